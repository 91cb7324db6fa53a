// sft_tcfft.cu -- the split-BF16x3 tensor-core transform of the precision
// study (sft_config.precision = 1), and the complex 2-D step built on it.
//
// An N-point complex DFT, N = 64 R (R = 16 or 32), is split n = n1 + R n2,
// k = k2 + 64 k1:
//   Y[n1][k2] = sum_{n2} x[n1 + R n2] W_64^{n2 k2}                (stage 1)
//   X[k2 + 64 k1] = sum_{n1} W_R^{n1 k1} (W_N^{n1 k2} Y[n1][k2])  (stage 2)
// Stage 1 is a real matrix product per line, [Re Y | Im Y] (R x 128) =
// [Re x | Im x] (R x 128) times the 128 x 128 real form of the DFT-64 matrix,
// on the tensor cores (mma.sync m16n8k16, bf16 operands, FP32 accumulation)
// with every FP32 operand split in two bf16 parts, a = a_hi + a_lo, and three
// products a_hi b_hi + a_hi b_lo + a_lo b_hi ("split-BF16x3"; the dropped
// a_lo b_lo is 2^-16 relative).  Stage 2 (twiddles and the R-point DFT) is
// FP32 in registers.  The step (Sec. IV boxed algorithm for the CGL term of
// Sec. V.C) runs as separate passes: masked scaled state -> inverse
// transforms along y and x (with a transpose between) -> |A|^2 A -> forward
// transforms along x and y -> the SETD update of every mode with the same
// Philox noise as the FP32 path.  The study compares this path with the FP32
// path against the FP64 oracle; it is slower by construction (materialised
// intermediates, two transposes per transform pair).
#include <cuda_bf16.h>

#include "sft_step_common.cuh"

namespace sft {

namespace {

constexpr int kTcLines = 4;     // lines per block
constexpr int kTcThreads = 256;
constexpr int kXS = 36;         // n2 stride (float2) of the stage-1 operand: conflict-free fragment loads
constexpr int kYS = 68;         // row stride (float2) of the stage-1 result
constexpr int kWS = 136;        // row stride (bf16) of the transposed real DFT-64 matrix

template <int N>
struct TcCfg {
    static constexpr int R = N / 64;  // stage-2 length = stage-1 rows
    static_assert(N == 1024 || N == 2048, "64 x 16 or 64 x 32 points");
    static constexpr int MT = R / 16;                  // 16-row tiles per line
    static constexpr int PAIRS = kTcLines * MT;        // (line, row tile) pairs per block
    static constexpr int WPP = 8 / PAIRS;              // warps per pair
    static constexpr int NT = 16 / WPP;                // 8-column tiles per warp
    static constexpr int XB = kXS * 64;                // float2 per line
    static constexpr int YB = R * kYS;
    static constexpr size_t SMEM = sizeof(float2) * (size_t)kTcLines * (XB + YB) +
                                   2 * sizeof(__nv_bfloat16) * (size_t)128 * kWS;
};

__device__ __forceinline__ uint32_t bf2_bits(__nv_bfloat162 v) { return *reinterpret_cast<uint32_t*>(&v); }

// hi and lo bf16 parts of a complex value (re in the low half, im in the high half)
__device__ __forceinline__ void split_bf16(float2 v, uint32_t& hi, uint32_t& lo) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(v.x, v.y);
    const float2 hf = __bfloat1622float2(h);
    const __nv_bfloat162 l = __floats2bfloat162_rn(v.x - hf.x, v.y - hf.y);
    hi = bf2_bits(h);
    lo = bf2_bits(l);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
        "{%0, %1, %2, %3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// In-place unnormalised N-point DFT (forward e^{-2 pi i}, inverse e^{+2 pi i}) of nlines contiguous lines.
// twN[m] = W_N^m (forward sign).
template <int N, bool INV>
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_fft(float2* data, long long nlines, const float2* __restrict__ twN) {
    using C = TcCfg<N>;
    constexpr int R = C::R;
    extern __shared__ __align__(16) unsigned char sm_raw[];
    float2* X = reinterpret_cast<float2*>(sm_raw);
    float2* Y = X + (size_t)kTcLines * C::XB;
    __nv_bfloat16* Wh = reinterpret_cast<__nv_bfloat16*>(Y + (size_t)kTcLines * C::YB);
    __nv_bfloat16* Wl = Wh + 128 * kWS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, q = lane & 3;

    // the real form of W_64^{+-n2 k2}: row nu = (k2, d) of the transposed matrix, column kappa = (n2, c):
    // d = 0 (Re Y): c = 0 -> Re W, c = 1 -> -Im W;  d = 1 (Im Y): c = 0 -> Im W, c = 1 -> Re W
    for (int i = tid; i < 128 * 128; i += kTcThreads) {
        const int nu = i >> 7, kap = i & 127;
        const int k2 = nu >> 1, d = nu & 1, n2 = kap >> 1, c = kap & 1;
        double sn, cs;
        sincospi(2.0 * (double)((n2 * k2) & 63) / 64.0, &sn, &cs);
        const float wr = (float)cs, wi = INV ? (float)sn : (float)-sn;
        const float w = d == 0 ? (c == 0 ? wr : -wi) : (c == 0 ? wi : wr);
        const __nv_bfloat16 h = __float2bfloat16_rn(w);
        Wh[nu * kWS + kap] = h;
        Wl[nu * kWS + kap] = __float2bfloat16_rn(w - __bfloat162float(h));
    }
    for (long long l0 = (long long)blockIdx.x * kTcLines; l0 < nlines; l0 += (long long)gridDim.x * kTcLines) {
        const int nl = (int)min((long long)kTcLines, nlines - l0);
        __syncthreads();  // the previous group is done with X and Y
        for (int i = tid; i < kTcLines * N; i += kTcThreads) {
            const int l = i / N, n = i % N;
            X[l * C::XB + (n % R) + kXS * (n / R)] = l < nl ? data[(l0 + l) * N + n] : czero();
        }
        __syncthreads();
        // stage 1: warp -> (line, 16-row tile), NT column tiles of 8
        {
            const int pair = warp / C::WPP, part = warp % C::WPP;
            const int line = pair / C::MT, mt = pair % C::MT;
            const float2* Xl = X + line * C::XB;
            float acc[C::NT][4];
#pragma unroll
            for (int j = 0; j < C::NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
            const int r0 = 16 * mt + g;
#pragma unroll
            for (int ks = 0; ks < 8; ++ks) {
                const int n2 = 8 * ks + q;
                uint32_t ah[4], al[4];
                split_bf16(Xl[r0 + kXS * n2], ah[0], al[0]);
                split_bf16(Xl[r0 + 8 + kXS * n2], ah[1], al[1]);
                split_bf16(Xl[r0 + kXS * (n2 + 4)], ah[2], al[2]);
                split_bf16(Xl[r0 + 8 + kXS * (n2 + 4)], ah[3], al[3]);
#pragma unroll
                for (int j = 0; j < C::NT; ++j) {
                    const int nu = 8 * (part * C::NT + j) + g;
                    const int kap = 16 * ks + 2 * q;
                    const uint32_t bh0 = *reinterpret_cast<const uint32_t*>(Wh + nu * kWS + kap);
                    const uint32_t bh1 = *reinterpret_cast<const uint32_t*>(Wh + nu * kWS + kap + 8);
                    const uint32_t bl0 = *reinterpret_cast<const uint32_t*>(Wl + nu * kWS + kap);
                    const uint32_t bl1 = *reinterpret_cast<const uint32_t*>(Wl + nu * kWS + kap + 8);
                    mma_bf16(acc[j], ah, bh0, bh1);
                    mma_bf16(acc[j], ah, bl0, bl1);
                    mma_bf16(acc[j], al, bh0, bh1);
                }
            }
            float2* Yl = Y + line * C::YB;
#pragma unroll
            for (int j = 0; j < C::NT; ++j) {
                const int k2 = 4 * (part * C::NT + j) + q;
                Yl[r0 * kYS + k2] = make_float2(acc[j][0], acc[j][1]);
                Yl[(r0 + 8) * kYS + k2] = make_float2(acc[j][2], acc[j][3]);
            }
        }
        __syncthreads();
        // stage 2: thread -> (line, k2), R values
        {
            const int line = tid >> 6, k2 = tid & 63;
            float2 v[R];
            const float2* Yl = Y + line * C::YB;
#pragma unroll
            for (int n1 = 0; n1 < R; ++n1) {
                float2 w = __ldg(&twN[n1 * k2]);
                if (INV) w.y = -w.y;
                v[n1] = cmul(Yl[n1 * kYS + k2], w);
            }
            dft_reg<R, INV>(v);
            if (line < nl) {
#pragma unroll
                for (int k1 = 0; k1 < R; ++k1) data[(l0 + line) * N + k2 + 64 * k1] = v[k1];
            }
        }
    }
}

// state -> the masked, scaled spectrum, column a_x of replica r contiguous along y (the state's own layout)
__global__ void k_tc_prep(const float2* __restrict__ phi, float2* __restrict__ out, long long total, int nx, int ny,
                          int dealias, float scale) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const int ay = (int)(i % ny), ax = (int)((i / ny) % nx);
    const bool keep = !dealias || (3 * abs(signed_idx(ax, nx)) < nx && 3 * abs(signed_idx(ay, ny)) < ny);
    out[i] = keep ? cscale(phi[i], scale) : czero();
}

// out[r][c][rr] = in[r][rr][c]: rows x cols matrices of every replica transposed
__global__ void k_tc_transpose(const float2* __restrict__ in, float2* __restrict__ out, int rows, int cols) {
    __shared__ float2 tile[32][33];
    const size_t base = (size_t)blockIdx.z * rows * cols;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = in[base + (size_t)r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const int c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[base + (size_t)c * rows + r] = tile[threadIdx.x][k];
    }
}

__global__ void k_tc_cube(float2* a, long long total) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= total) return;
    const float2 A = a[i];
    a[i] = cscale(A, A.x * A.x + A.y * A.y);
}

// the SETD update of every mode (complex coefficients, complex noise, SETD2 history): F = M s DFT[q]
__global__ void k_tc_update(const StepArgs a, const float2* __restrict__ dq) {
    const long long nm = (long long)a.hx * a.ny;
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)a.R * nm) return;
    const int r = (int)(i / nm);
    const long long j = i % nm;  // mode index within the replica (x-major): the noise counter
    const int ay = (int)(j % a.ny), ax = (int)(j / a.ny);
    const int axs = signed_idx(ax, a.nx), ays = signed_idx(ay, a.ny);
    const long long step = current_step(a);
    const bool first = (a.scheme == 2) && (step == *a.first_step);
    const bool inm = !a.dealias || (3 * abs(axs) < a.nx && 3 * abs(ays) < a.ny);
    const float2 F = inm ? cmul(make_float2(a.s0, a.s0i), dq[i]) : czero();
    const Coefs co = load_coefs<true>(a.tab, abs(axs) * (a.ny / 2 + 1) + abs(ays), first);
    const float2 Fp = a.scheme == 2 ? a.fprev[i] : czero();
    const float2 z = normal_pair_for_index(a.seed, (uint64_t)j, (uint32_t)step, (uint32_t)(a.rep0 + r), 0u);
    const float2 o = setd_update<true>(co, a.phi[i], F, Fp, eta_of(z, false));
    a.phi[i] = o;
    if (a.scheme == 2) a.fprev[i] = F;
    flag_nonfinite(a, o, step);
}

template <int N, bool INV>
cudaError_t run_tc_fft(float2* data, long long nlines, const float2* twN, cudaStream_t s) {
    using C = TcCfg<N>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tc_fft<N, INV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const long long groups = (nlines + kTcLines - 1) / kTcLines;
    const unsigned blocks = (unsigned)(groups < 1216 ? groups : 1216);
    k_tc_fft<N, INV><<<blocks, kTcThreads, C::SMEM, s>>>(data, nlines, twN);
    return cudaGetLastError();
}

cudaError_t tc_fft(int n, bool inv, float2* data, long long nlines, const float2* twN, cudaStream_t s) {
    if (n == 1024) return inv ? run_tc_fft<1024, true>(data, nlines, twN, s) : run_tc_fft<1024, false>(data, nlines, twN, s);
    if (n == 2048) return inv ? run_tc_fft<2048, true>(data, nlines, twN, s) : run_tc_fft<2048, false>(data, nlines, twN, s);
    return cudaErrorInvalidValue;
}

}  // namespace

bool tc_supported(int nx, int ny) { return nx == ny && (nx == 1024 || nx == 2048); }

// One step of the complex 2-D field through the tensor-core transforms: b1, b2 are scratch buffers of the
// state's size; twN the N-point table.  a: the step's arguments (phi, fprev, tab, counters).
cudaError_t launch_tc_step(const StepArgs& a, float2* b1, float2* b2, const float2* twN, cudaStream_t s) {
    const int nx = a.nx, ny = a.ny;
    if (!tc_supported(nx, ny)) return cudaErrorInvalidValue;
    const long long total = (long long)a.R * nx * ny;
    const unsigned eb = (unsigned)((total + 255) / 256);
    const dim3 tgrid((ny + 31) / 32, (nx + 31) / 32, a.R), tblock(32, 8);
    // A = IDFT_2D(M phi) / N^2: columns (along y), transpose, rows (along x)
    k_tc_prep<<<eb, 256, 0, s>>>(a.phi, b1, total, nx, ny, a.dealias, a.scale);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = tc_fft(ny, true, b1, (long long)a.R * nx, twN, s);
    if (e == cudaSuccess) {
        k_tc_transpose<<<tgrid, tblock, 0, s>>>(b1, b2, nx, ny);  // [a_x][y] -> [y][x]
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = tc_fft(nx, true, b2, (long long)a.R * ny, twN, s);
    if (e == cudaSuccess) {
        k_tc_cube<<<eb, 256, 0, s>>>(b2, total);
        e = cudaGetLastError();
    }
    // DFT_2D[|A|^2 A]: rows, transpose back, columns
    if (e == cudaSuccess) e = tc_fft(nx, false, b2, (long long)a.R * ny, twN, s);
    if (e == cudaSuccess) {
        const dim3 tg2((nx + 31) / 32, (ny + 31) / 32, a.R);
        k_tc_transpose<<<tg2, tblock, 0, s>>>(b2, b1, ny, nx);  // [y][a_x] -> [a_x][y]
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = tc_fft(ny, false, b1, (long long)a.R * nx, twN, s);
    if (e == cudaSuccess) {
        k_tc_update<<<eb, 256, 0, s>>>(a, b1);
        e = cudaGetLastError();
    }
    return e;
}

// Batched N-point transform of contiguous lines through the tensor-core path (tests of the transform alone).
cudaError_t launch_tc_fft(int n, int inverse, float2* data, long long nlines, const float2* twN, cudaStream_t s) {
    return tc_fft(n, inverse != 0, data, nlines, twN, s);
}

}  // namespace sft
