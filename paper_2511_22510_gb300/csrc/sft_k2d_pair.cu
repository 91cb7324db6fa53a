// sft_k2d_pair.cu -- row pass of the 2-D real-field step (cubic term) on rows
// of 1024 points, two rows per warp.
//
// The row pass takes P[a_x][y] (the state transformed back along y, masked and
// scaled, a_x < ncols) to psi(x, y), cubes it and transforms q = psi^3 forward
// along x into Q[a_x][y] (Sec. IV boxed algorithm, steps 1-3 along x).  Two
// real rows y, y + 1 go through one complex 1024-point transform:
//   Z[k] = X_y[k] + i X_{y+1}[k]   (X[1024 - k] = conj X[k] for k > 512),
//   IFFT(Z) = psi_y + i psi_{y+1},  q = (Re^3, Im^3),  W = FFT(q),
//   Q_y[k] = (W[k] + conj W[1024 - k]) / 2,  Q_{y+1}[k] = (W[k] - conj W[1024 - k]) / (2i),
// so no real-to-complex twiddle step is needed.  A block takes 16 rows of one
// replica: the tile of every carried column's 16 values (128 contiguous bytes
// per column) arrives by a TMA tensor load into a 128-byte-swizzled shared
// tile, completing on an mbarrier with a bounded wait; Q leaves the same tile
// by a TMA tensor store.  Under 2/3 truncation the transform inputs with
// 342 <= |k| are zero in ten whole slots, which the first DFT stage skips.
#include <cudaTypedefs.h>

#include <mutex>

#include "sft_step_common.cuh"
#include "sft_warpfft.cuh"

namespace sft {

namespace {

constexpr int kPairNX = 1024;     // row length
constexpr int kPairRows = 16;     // rows per block: 128 bytes of every column
constexpr int kPairWarps = 8;     // one warp per row pair
constexpr int kPairBoxCols = 176; // columns per tensor box (<= 256; a multiple of 8 keeps each box 1024-byte aligned)

template <bool DEAL>
struct PairCfg {
    static constexpr int NC = DEAL ? kPairNX / 3 + 1 : kPairNX / 2 + 1;  // carried columns: 342 or 513
    static constexpr int NBOX = (NC + kPairBoxCols - 1) / kPairBoxCols;
    static constexpr int TILEW = NBOX * kPairBoxCols;                     // columns in the tile
    static constexpr size_t TILE_BYTES = (size_t)TILEW * 128;
    static constexpr size_t XB_BYTES = (size_t)kPairWarps * kPairNX * sizeof(float2);
    static constexpr size_t SMEM = 1024 + TILE_BYTES + XB_BYTES;  // + alignment slack
    // slots e (index lane + 32 e) that are zero in every lane: 342 <= k <= 682
    static constexpr uint32_t ZIN = DEAL ? 0x001FF800u : 0u;
    static constexpr int EOUT = (NC - 1) / 32;  // last slot holding an output column
};

// Address (in float2) of the pair (X_y[c], X_{y+1}[c]) of pair j in the 128-byte-swizzled tile:
// column c occupies 128 bytes; its 16-byte chunk j is stored at chunk j ^ (c mod 8).
__device__ __forceinline__ int tile_pos(int c, int j) { return c * 16 + ((j ^ (c & 7)) << 1); }

template <bool DEAL>
__global__ void __launch_bounds__(kPairWarps * 32, 2)
    k2_rows_pair(const StepArgs a, const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout) {
    using C = PairCfg<DEAL>;
    extern __shared__ unsigned char smraw[];
    __shared__ uint64_t bar;
    __shared__ unsigned abort_flag;
    unsigned char* base =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    float2* tile = reinterpret_cast<float2*>(base);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    float2* xb = reinterpret_cast<float2*>(base + C::TILE_BYTES) + warp * kPairNX;
    const int y0 = blockIdx.x * kPairRows, rep = blockIdx.y;
    const float2* __restrict__ tw32 = a.tw_32;

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (uint32_t)C::TILE_BYTES);
#pragma unroll
        for (int b = 0; b < C::NBOX; ++b)
            tma_load_3d(tile + b * kPairBoxCols * 16, &tin, 2 * y0, b * kPairBoxCols, rep, &bar);
    }
    if (!mbar_wait_bounded(&bar, 0, wait_iters(a))) atomicOr(&abort_flag, 1u);
    __syncthreads();
    if (abort_flag) {
        // the wait ran out: report it, let the tile copy land (bounded) and stop
        if (threadIdx.x == 0) {
            atomicOr(a.status, 2u);
            mbar_wait_bounded(&bar, 0);
        }
        return;
    }

    // Z[k] = X_y[k] + i X_{y+1}[k], k = lane + 32 e, rows y0 + 2 warp and y0 + 2 warp + 1
    float2 v[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        if ((C::ZIN >> e) & 1u) {
            v[e] = czero();
            continue;
        }
        const bool lo = e < 16;  // k < 512: the stored column k; else the mirror 1024 - k
        const int c = lo ? lane + 32 * e : 32 * (32 - e) - lane;
        const bool may_exceed = lo ? (31 + 32 * e >= C::TILEW) : (32 * (32 - e) >= C::TILEW);
        if (may_exceed && c >= C::TILEW) {
            v[e] = czero();
            continue;
        }
        const float4 p = *reinterpret_cast<const float4*>(tile + tile_pos(c, warp));
        // lo: X_y + i X_{y+1}; mirror: conj X_y + i conj X_{y+1}
        v[e] = lo ? make_float2(p.x - p.w, p.y + p.z) : make_float2(p.x + p.w, p.z - p.y);
    }
    __syncthreads();  // every warp has read the tile: it is free for Q

    fft1024_warp<true, C::ZIN>(v, xb, lane, tw32);
#pragma unroll
    for (int e = 0; e < 32; ++e) v[e] = __fmul2_rn(__fmul2_rn(v[e], v[e]), v[e]);
    fft1024_warp<false, 0u>(v, xb, lane, tw32);

    // Q_y[k], Q_{y+1}[k] for the carried columns k = lane + 32 e < NC; W[1024 - k] comes from lane
    // (32 - lane) mod 32, slot 31 - e (lane 0: slot (32 - e) mod 32)
    const int src = (32 - lane) & 31;
#pragma unroll
    for (int e = 0; e <= C::EOUT; ++e) {
        const float2 mine = lane == 0 ? v[(32 - e) & 31] : v[31 - e];
        float2 wm;
        wm.x = __shfl_sync(0xffffffffu, mine.x, src);
        wm.y = __shfl_sync(0xffffffffu, mine.y, src);
        const int k = lane + 32 * e;
        if (32 * e + 31 < C::NC || k < C::NC) {
            const float2 w = v[e];
            const float2 qa = __fmul2_rn(f2(0.5f), __fadd2_rn(w, make_float2(wm.x, -wm.y)));
            const float2 qb = __fmul2_rn(f2(0.5f), __fadd2_rn(make_float2(w.y, wm.x), make_float2(wm.y, -w.x)));
            const float4 q = make_float4(qa.x, qa.y, qb.x, qb.y);
            *reinterpret_cast<float4*>(tile + tile_pos(k, warp)) = q;
        }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int b = 0; b < C::NBOX; ++b) tma_store_3d(&tout, 2 * y0, b * kPairBoxCols, rep, tile + b * kPairBoxCols * 16);
        tma_store_commit();
        tma_store_wait_read();
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

// Tensor map over an intermediate (P or Q) of R replicas: floats, dims {2 ny, ncols, R},
// strides {ny 8, hx ny 8} bytes, box {32 floats = 16 rows, kPairBoxCols columns, 1}.
cudaError_t encode_pq(CUtensorMap* m, const float2* base, int ny, int ncols, int hx, int R) {
    std::call_once(g_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_encode) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)2 * ny, (cuuint64_t)ncols, (cuuint64_t)R};
    const cuuint64_t strides[2] = {(cuuint64_t)ny * sizeof(float2), (cuuint64_t)hx * ny * sizeof(float2)};
    const cuuint32_t box[3] = {32, (cuuint32_t)kPairBoxCols, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(base), dims, strides, box,
                               estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <bool DEAL>
cudaError_t run_pair(const StepArgs& a, cudaStream_t s) {
    using C = PairCfg<DEAL>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k2_rows_pair<DEAL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (a.ncols != C::NC || !a.tw_32) return cudaErrorInvalidValue;
    CUtensorMap tin, tout;
    cudaError_t e = encode_pq(&tin, a.pin, a.ny, a.ncols, a.hx, a.R);
    if (e == cudaSuccess) e = encode_pq(&tout, a.qout, a.ny, a.ncols, a.hx, a.R);
    if (e != cudaSuccess) return e;
    dim3 grid(a.ny / kPairRows, a.R);
    k2_rows_pair<DEAL><<<grid, kPairWarps * 32, C::SMEM, s>>>(a, tin, tout);
    return cudaGetLastError();
}

}  // namespace

bool k2_pair_supported(int nx, int ny, int nl, int dealias) {
    return nx == kPairNX && ny >= kPairRows && ny % kPairRows == 0 && nl == NL_CUBIC && (dealias == 0 || dealias == 1);
}

cudaError_t launch_k2_rows_pair(const StepArgs& a, int nl, cudaStream_t s) {
    if (!k2_pair_supported(a.nx, a.ny, nl, a.pshift ? 2 : a.dealias)) return cudaErrorInvalidValue;
    return a.dealias ? run_pair<true>(a, s) : run_pair<false>(a, s);
}

}  // namespace sft
