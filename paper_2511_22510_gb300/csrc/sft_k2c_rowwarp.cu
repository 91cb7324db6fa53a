// sft_k2c_rowwarp.cu -- row pass of the complex 2-D step (the CGL term of
// Sec. V.C, steps 1-3 of the Sec. IV boxed algorithm along x) on rows of
// NX = 1024 H points (H = 1, 2) under 2/3 truncation, built on the
// warp-resident 1024-point transform of sft_warpfft.cuh.
//
// P[c][y] holds the carried x-modes of each row in compact order (c < m: a_x =
// c; c >= m: a_x = c + (NX - ncols)).  A block takes ROWS = 8 / H rows of one
// replica: the tile of every carried column's ROWS values (64 / H contiguous
// bytes per column) arrives by TMA tensor loads into a swizzled shared tile,
// completing on an mbarrier with a bounded wait, and Q leaves the same tile by
// TMA tensor stores.  Row r is held by H warps.  With H = 2 the inverse
// transform splits the modes by halves (decimation in frequency): warp 0
// transforms X[k] + X[k + 1024] into the even samples A(2n), warp 1 transforms
// (X[k] - X[k + 1024]) W^{-k} into the odd samples A(2n + 1); after the
// pointwise |A|^2 A each warp transforms its parity class forward and the two
// combine through shared memory (decimation in time): warp 0 keeps
// X[k] = E[k] + W^k O[k], warp 1 keeps X[k + 1024] = E[k] - W^k O[k].
// W = e^{-2 pi i / NX}.  Both transforms are unnormalised, as in the general
// complex row pass (P carries the 1/N^2 of the column pass).
#include <cudaTypedefs.h>

#include <mutex>

#include "sft_step_common.cuh"
#include "sft_warpfft.cuh"

namespace sft {

namespace {

constexpr int kCrWarps = 8;

template <int H>
struct CrCfg {
    static constexpr int NX = 1024 * H;
    static constexpr int ROWS = kCrWarps / H;             // rows per block
    static constexpr int PIECE = ROWS * 8;                 // bytes of one column in the tile (32 or 64)
    static constexpr int NC = 2 * (NX / 3) + 1;            // carried columns under 2/3 truncation: 683, 1365
    static constexpr int M = NX / 3 + 1;                   // compact columns c < M hold a_x = c
    static constexpr int BOXC = H == 2 ? 128 : 176;        // columns per tensor box (box bytes: multiples of 1 KB)
    static constexpr int NBOX = (NC + BOXC - 1) / BOXC;
    static constexpr int TILEW = NBOX * BOXC;
    static constexpr size_t TILE_BYTES = (size_t)TILEW * PIECE;
    static constexpr size_t XB_BYTES = (size_t)kCrWarps * 1024 * sizeof(float2);
    static constexpr size_t SMEM = 1024 + TILE_BYTES + XB_BYTES;  // + alignment slack
    // H = 1: slots e (index lane + 32 e) that are zero in every lane on input: 342 <= a_x <= 682
    static constexpr uint32_t ZIN = H == 1 ? 0x001FF800u : 0u;
};

// Byte offset of (column c, row r) in the tile: column pieces of PIECE bytes, stored with the tensor map's
// swizzle (32-byte pieces: SWIZZLE_32B, bit 7 into bit 4; 64-byte pieces: SWIZZLE_64B, bits 7-8 into bits 4-5)
template <int H>
__device__ __forceinline__ uint32_t cr_off(int c, int r) {
    const uint32_t o = (uint32_t)c * CrCfg<H>::PIECE + (uint32_t)r * 8u;
    return H == 2 ? o ^ (((o >> 7) & 1u) << 4) : o ^ (((o >> 7) & 3u) << 4);
}

// barrier of the H = 2 warps that hold row r: named barrier 1 + r, 64 threads (0 is __syncthreads)
__device__ __forceinline__ void row_pair_sync(int r) {
    switch (r) {
        case 0: asm volatile("bar.sync 1, 64;" ::: "memory"); break;
        case 1: asm volatile("bar.sync 2, 64;" ::: "memory"); break;
        case 2: asm volatile("bar.sync 3, 64;" ::: "memory"); break;
        default: asm volatile("bar.sync 4, 64;" ::: "memory"); break;
    }
}

template <int H>
__global__ void __launch_bounds__(kCrWarps * 32, 2)
    k2c_rows_warp(const StepArgs a, const __grid_constant__ CUtensorMap tin, const __grid_constant__ CUtensorMap tout) {
    using C = CrCfg<H>;
    extern __shared__ unsigned char smraw[];
    __shared__ uint64_t bar;
    __shared__ unsigned abort_flag;
    unsigned char* tile =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int r = warp / H, h = warp % H;
    float2* xb = reinterpret_cast<float2*>(tile + C::TILE_BYTES) + warp * 1024;
    const float2* xo = reinterpret_cast<const float2*>(tile + C::TILE_BYTES) + (warp ^ (H - 1)) * 1024;
    const int y0 = blockIdx.x * C::ROWS, rep = blockIdx.y;
    const float2* __restrict__ tw32 = a.tw_32;
    const float2* __restrict__ twN = a.tw_a;  // W_NX^k, k < NX

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(&bar, (uint32_t)C::TILE_BYTES);
#pragma unroll 1
        for (int b = 0; b < C::NBOX; ++b) tma_load_3d(tile + (size_t)b * C::BOXC * C::PIECE, &tin, 2 * y0, b * C::BOXC, rep, &bar);
    }
    if (!mbar_wait_bounded(&bar, 0, wait_iters(a))) atomicOr(&abort_flag, 1u);
    __syncthreads();
    if (abort_flag) {
        // the wait ran out: report it, let the tile copies land (bounded) and stop
        if (threadIdx.x == 0) {
            atomicOr(a.status, 2u);
            mbar_wait_bounded(&bar, 0);
        }
        return;
    }

    // the inverse transform's input, k = lane + 32 e.  The swizzle reads address bits 7 and up only below bit 10
    // (32-byte pieces: bit 7; 64-byte pieces: bits 7-8), so a step of 32 columns (1 KB or 2 KB) keeps it: one
    // swizzled base per lane for the low and one for the high (negative) columns, plus a multiple of 32 columns.
    constexpr int ESTEP = 32 * C::PIECE;
    constexpr int CSH = C::NX - C::NC;  // compact column of a high mode a_x: a_x - CSH
    constexpr int EH = (C::NX - C::M + 1 + 31) / 32;  // first slot whose every index is a high mode (H = 1)
    const int base_lo = (int)cr_off<H>(lane, r);
    const int base_hi = (int)(H == 1 ? cr_off<H>(lane + 32 * EH - CSH, r) : cr_off<H>(lane + 1024 - CSH, r));
    // W_NX^k for k = lane + 32 e, e = 2 j + p, as W_NX^{lane + 32 p} times the constant W_32^j (H = 2)
    float2 wl[2] = {czero(), czero()};
    if constexpr (H == 2) {
        wl[0] = __ldg(&twN[lane]);
        wl[1] = __ldg(&twN[lane + 32]);
    }
    float2 v[32];
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        const int k = lane + 32 * e;
        if constexpr (H == 1) {
            if ((C::ZIN >> e) & 1u) {
                v[e] = czero();
                continue;
            }
            // a_x = k carried when k < M (column k) or k >= NX - M + 1 (column k - CSH)
            const bool lo = k < C::M, hi = k >= C::NX - C::M + 1;
            const int o = lo ? base_lo + ESTEP * e : base_hi + ESTEP * (e - EH);
            v[e] = (lo || hi) ? *reinterpret_cast<const float2*>(tile + o) : czero();
        } else {
            // X[k] (carried for k < M) and X[k + 1024] (carried for k + 1024 >= NX - M + 1)
            const bool lo = k < C::M, hi = k + 1024 >= C::NX - C::M + 1;
            const float2 x0 = lo ? *reinterpret_cast<const float2*>(tile + base_lo + ESTEP * e) : czero();
            const float2 x1 = hi ? *reinterpret_cast<const float2*>(tile + base_hi + ESTEP * e) : czero();
            v[e] = h == 0 ? padd(x0, x1) : twiddle_const<true>(cmul(psub(x0, x1), cconj(wl[e & 1])), e >> 1, 32);
        }
    }
    __syncthreads();  // every warp has read the tile: it is free for Q

    fft1024_warp<true, C::ZIN>(v, xb, lane, tw32);
#pragma unroll
    for (int e = 0; e < 32; ++e) v[e] = cscale(v[e], v[e].x * v[e].x + v[e].y * v[e].y);
    fft1024_warp<false, 0u>(v, xb, lane, tw32);

    if constexpr (H == 2) {
        // warp 0 holds E[k] (even samples), warp 1 O[k]; X[k] = E + W^k O, X[k + 1024] = E - W^k O
        if (h == 1) {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = twiddle_const<false>(cmul(v[e], wl[e & 1]), e >> 1, 32);
        }
#pragma unroll
        for (int e = 0; e < 32; ++e) xb[lane + 32 * e] = v[e];
        row_pair_sync(r);
#pragma unroll
        for (int e = 0; e < 32; ++e) {
            const float2 o = xo[lane + 32 * e];
            v[e] = h == 0 ? padd(v[e], o) : psub(o, v[e]);
        }
    }

    // Q: the carried modes a_x = 1024 h + k into their compact columns
#pragma unroll
    for (int e = 0; e < 32; ++e) {
        const int ax = 1024 * h + lane + 32 * e;
        const bool lo = ax < C::M, hi = ax >= C::NX - C::M + 1;
        if (lo || hi) {
            const int o = H == 1 ? (lo ? base_lo + ESTEP * e : base_hi + ESTEP * (e - EH))
                                      : (h == 0 ? base_lo : base_hi) + ESTEP * e;
            *reinterpret_cast<float2*>(tile + o) = v[e];
        }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll 1
        for (int b = 0; b < C::NBOX; ++b) tma_store_3d(&tout, 2 * y0, b * C::BOXC, rep, tile + (size_t)b * C::BOXC * C::PIECE);
        tma_store_commit();
        tma_store_wait_read();
    }
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
PFN_cuTensorMapEncodeTiled_v12000 g_cr_encode = nullptr;
std::once_flag g_cr_encode_once;

// Tensor map over a complex intermediate (P or Q) of R replicas: floats, dims {2 ny, ncols, R}, strides
// {ny 8, hx ny 8} bytes, box {2 ROWS floats, BOXC columns, 1}, swizzle matching the piece width
template <int H>
cudaError_t encode_cr(CUtensorMap* m, const float2* base, int ny, int ncols, int hx, int R) {
    using C = CrCfg<H>;
    std::call_once(g_cr_encode_once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_cr_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!g_cr_encode) return cudaErrorNotSupported;
    const cuuint64_t dims[3] = {(cuuint64_t)2 * ny, (cuuint64_t)ncols, (cuuint64_t)R};
    const cuuint64_t strides[2] = {(cuuint64_t)ny * sizeof(float2), (cuuint64_t)hx * ny * sizeof(float2)};
    const cuuint32_t box[3] = {(cuuint32_t)(2 * C::ROWS), (cuuint32_t)C::BOXC, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult res =
        g_cr_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float2*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, H == 2 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return res == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int H>
cudaError_t run_crw(const StepArgs& a, cudaStream_t s) {
    using C = CrCfg<H>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(k2c_rows_warp<H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    CUtensorMap tin, tout;
    cudaError_t e = encode_cr<H>(&tin, a.pin, a.ny, a.ncols, a.hx, a.R);
    if (e == cudaSuccess) e = encode_cr<H>(&tout, a.qout, a.ny, a.ncols, a.hx, a.R);
    if (e != cudaSuccess) return e;
    k2c_rows_warp<H><<<dim3(a.ny / C::ROWS, a.R), kCrWarps * 32, C::SMEM, s>>>(a, tin, tout);
    return cudaGetLastError();
}

}  // namespace

// rows of 1024 or 2048 points under 2/3 truncation, a whole number of 8 / H-row tiles
bool k2c_rowwarp_supported(int nx, int ny, int dealias) {
    const int rows = nx == 1024 ? 8 : 4;
    return (nx == 1024 || nx == 2048) && dealias == 1 && ny >= rows && ny % rows == 0;
}

cudaError_t launch_k2c_rows_warp(const StepArgs& a, cudaStream_t s) {
    if (!k2c_rowwarp_supported(a.nx, a.ny, a.pshift ? 2 : a.dealias) || !a.tw_32 || !a.tw_a ||
        a.ncols != 2 * (a.nx / 3) + 1 || a.hx != a.nx)
        return cudaErrorInvalidValue;
    return a.nx == 1024 ? run_crw<1>(a, s) : run_crw<2>(a, s);
}

}  // namespace sft
