// sft_k2c_colwarp.cu -- column pass of the complex 2-D step (the CGL term of
// Sec. V.C, the Sec. IV boxed algorithm) on columns of 1024 or 2048 points,
// built on the warp-resident 1024-point transform of sft_warpfft.cuh.
//
// A column of NY = 1024 H points is held by H warps.  With H = 2 the forward
// transform splits the samples by parity (decimation in time): warp h
// transforms the samples 2 m + h, the odd half is multiplied by W_2048^k, and
// the two halves are exchanged through shared memory so that warp 0 holds
// X[k] = E[k] + W^k O[k] and warp 1 holds X[k + 1024] = E[k] - W^k O[k]
// (k < 1024).  The inverse transform runs the other way (decimation in
// frequency): warp 0 transforms X[k] + X[k + 1024] into the even samples, warp
// 1 transforms (X[k] - X[k + 1024]) W^{-k} into the odd ones.  Between the
// transforms each warp updates its 1024 modes a_y = 1024 h + t + 32 e in a
// rolled loop, two slots per trip, with the same Philox counters and the same
// complex SETD update as the other complex column passes (complex noise on
// every mode, no Hermitian constraint).
#include "sft_step_common.cuh"
#include "sft_warpfft.cuh"

namespace sft {

namespace {

constexpr int kCcWarps = 4;
constexpr int kCcRpb = 2;  // replicas per block

// compact x-column order of the complex intermediates P, Q (the complex row pass's layout): column cx < m holds
// a_x = cx, column cx >= m holds a_x = cx + (nx - ncols), ncols = 2m - 1 (ncols = nx without truncation)
__device__ __forceinline__ bool cw_mask_x(int ax, int nx, int ncols) {
    const int m = (ncols + 1) / 2;
    return ax < m || ax >= nx - ncols / 2;
}
__device__ __forceinline__ int cw_comp_x(int ax, int nx, int ncols) {
    const int m = (ncols + 1) / 2;
    return ax < m ? ax : ax - (nx - ncols);
}

// barrier of the two warps that hold one column: named barrier 1 + (column within the block), 64 threads (0 is
// __syncthreads); immediate ids, so that the kernel reserves only the barriers it uses
__device__ __forceinline__ void pair_sync(int pc) {
    if (pc == 0)
        asm volatile("bar.sync 1, 64;" ::: "memory");
    else
        asm volatile("bar.sync 2, 64;" ::: "memory");
}

// The update of this warp's 1024 modes a_y = 1024 h + lane + 32 e, two slots (one Philox call) per trip of a loop
// that is not unrolled; the state and the SETD2 history of the next pair of slots are loaded one trip ahead; xb
// holds DFT[q] on entry and receives the masked, scaled new state.  HASF: the column carries F and P; S2: SETD2
// (the history F_prev).  Returns the non-finite accumulator.
template <int H, bool DEAL, bool HASF, bool S2>
__device__ __forceinline__ float ccw_update(const StepArgs& a, float2* xb, size_t colbase, int c, int lane, int h,
                                            long long step, int rep, bool first, int tabrow, float2 s) {
    constexpr int NY = 1024 * H;
    constexpr bool HIST = S2 && HASF;
    const float2* __restrict__ phin = a.phi + colbase + 1024 * h;
    const float2* fpin = HIST ? a.fprev + colbase + 1024 * h : nullptr;
    float nf = 0.f;
    float2 ph0 = phin[lane], ph1 = phin[lane + 32];
    float2 fp0 = czero(), fp1 = czero();
    if constexpr (HIST) {
        fp0 = fpin[lane];
        fp1 = fpin[lane + 32];
    }
#pragma unroll 1
    for (int e = 0; e < 32; e += 2) {
        float2 nx0 = czero(), nx1 = czero(), nf0 = czero(), nf1 = czero();
        if (e + 2 < 32) {
            nx0 = phin[lane + 32 * (e + 2)];
            nx1 = phin[lane + 32 * (e + 3)];
            if constexpr (HIST) {
                nf0 = fpin[lane + 32 * (e + 2)];
                nf1 = fpin[lane + 32 * (e + 3)];
            }
        }
        float2 z0, z1;
        team_normal_pair_ks<32>(a.ks, (uint64_t)c * NY + 1024 * h, lane, e, (uint32_t)step,
                                (uint32_t)(a.rep0 + rep), z0, z1);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int k = lane + 32 * (e + hh);
            const int ay = 1024 * h + k;
            const int ays = signed_idx(ay, NY);
            const bool inm = HASF && (!DEAL || 3 * abs(ays) < NY);
            const float2 F = inm ? cmul(s, xb[k]) : czero();
            const Coefs co = load_coefs<true>(a.tab, tabrow + abs(ays), S2 && first);
            const float2 eta = eta_of(hh ? z1 : z0, false);
            const float2 ph = hh ? ph1 : ph0;
            float2 out = cadd(cmul(co.f1, ph), cmul(co.A, F));
            if constexpr (HIST) out = cadd(out, cmul(co.B, hh ? fp1 : fp0));
            out = cadd(out, cmul(co.g, eta));
            if constexpr (HIST) a.fprev[colbase + ay] = F;
            a.phi[colbase + ay] = out;
            nf = nonfinite_acc(nf, out);
            xb[k] = inm ? cscale(out, a.scale) : czero();
        }
        ph0 = nx0;
        ph1 = nx1;
        fp0 = nf0;
        fp1 = nf1;
    }
    return nf;
}

// 5 blocks (20 warps) per SM: the register budget of the real warp column pass
template <int H, bool DEAL>
__global__ void __launch_bounds__(kCcWarps * 32, 5) k2c_cols_warp(const StepArgs a) {
    constexpr int NY = 1024 * H;
    constexpr int CPB = kCcWarps / H;  // columns per block
    // H = 1 with 2/3 truncation: slots e (index lane + 32 e) outside |a_y| < 342 in every lane, e = 11 .. 20
    constexpr uint32_t ZMASK = (DEAL && H == 1) ? 0x001FF800u : 0u;
    __shared__ __align__(16) float2 xbuf[kCcWarps][1024];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = warp % H, pc = warp / H;
    const int c = blockIdx.x * CPB + pc;  // a_x
    if (c >= a.hx) return;                // every warp of the column
    float2* xb = xbuf[warp];
    const float2* xo = xbuf[warp ^ (H - 1)];  // the other half's buffer (H = 2)
    const int nx = a.nx, ncols = a.ncols;
    const bool has_f = !DEAL || cw_mask_x(c, nx, ncols);
    const int tabrow = abs(signed_idx(c, nx)) * (NY / 2 + 1);
    const long long step = current_step(a);
    const bool first = (a.scheme == 2) && (step == *a.first_step);
    const float2* __restrict__ tw32 = a.tw_32;
    const float2* __restrict__ twN = a.tw_a;  // W_NY^k
    const float2 s = make_float2(a.s0, a.s0i);
    const int bar = pc;  // H = 2: two columns per block, barriers 1 and 2
    // kCcRpb replicas per block, one after the other: the column's coefficient rows (complex, 32 bytes per mode)
    // are then read from the caches for every replica after the first
    for (int ri = 0; ri < kCcRpb; ++ri) {
    const int rep = blockIdx.y * kCcRpb + ri;
    if (rep >= a.R) break;  // every warp of the column
    const size_t colbase = ((size_t)rep * a.hx + c) * NY;
    const size_t cbase = ((size_t)rep * a.hx + (has_f ? cw_comp_x(c, nx, ncols) : 0)) * NY;

    // DFT_y[q] of this warp's half into xb, natural slot order (modes 1024 h + lane + 32 e)
    if (has_f) {
        float2 v[32];
#pragma unroll
        for (int e = 0; e < 32; ++e) v[e] = a.qin[cbase + H * (lane + 32 * e) + h];
        fft1024_warp<false, 0u>(v, xb, lane, tw32);
        if constexpr (H == 2) {
            if (h == 1) {
                // W_NY^k for k = lane + 32 e, e = 2 j + p: W_NY^{lane + 32 p} times the constant W_32^j
                const float2 w0 = __ldg(&twN[lane]), w1 = __ldg(&twN[lane + 32]);
#pragma unroll
                for (int e = 0; e < 32; ++e) v[e] = twiddle_const<false>(cmul(v[e], (e & 1) ? w1 : w0), e >> 1, 32);
            }
#pragma unroll
            for (int e = 0; e < 32; ++e) xb[lane + 32 * e] = v[e];
            pair_sync(bar);
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const float2 o = xo[lane + 32 * e];
                v[e] = (h == 0) ? cadd(v[e], o) : csub(o, v[e]);
            }
            pair_sync(bar);  // both halves read before either buffer is overwritten
        }
#pragma unroll
        for (int e = 0; e < 32; ++e) xb[lane + 32 * e] = v[e];
    }
    __syncwarp();

    // the update (ccw_update), with the column's run-time-uniform choices resolved once
    const float nf = has_f ? (a.scheme == 2 ? ccw_update<H, DEAL, true, true>(a, xb, colbase, c, lane, h, step, rep,
                                                                              first, tabrow, s)
                                            : ccw_update<H, DEAL, true, false>(a, xb, colbase, c, lane, h, step, rep,
                                                                               first, tabrow, s))
                           : (a.scheme == 2 ? ccw_update<H, DEAL, false, true>(a, xb, colbase, c, lane, h, step, rep,
                                                                               first, tabrow, s)
                                            : ccw_update<H, DEAL, false, false>(a, xb, colbase, c, lane, h, step,
                                                                                rep, first, tabrow, s));
    flag_nonfinite_acc(a, nf, step);
    __syncwarp();

    // P <- IFFT_y(M phi / N^2) into the compact column
    if (has_f) {
        float2 v[32];
        if constexpr (H == 2) {
            const float2 w0 = cconj(__ldg(&twN[lane])), w1 = cconj(__ldg(&twN[lane + 32]));
            pair_sync(bar);  // both halves of the new column are in the buffers
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int k = lane + 32 * e;
                const float2 lo = (h == 0) ? xb[k] : xo[k], hi = (h == 0) ? xo[k] : xb[k];
                v[e] = (h == 0) ? cadd(lo, hi)
                                : twiddle_const<true>(cmul(csub(lo, hi), (e & 1) ? w1 : w0), e >> 1, 32);
            }
            pair_sync(bar);
        } else {
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = ((ZMASK >> e) & 1u) ? czero() : xb[lane + 32 * e];
            __syncwarp();
        }
        fft1024_warp<true, ZMASK>(v, xb, lane, tw32);
#pragma unroll
        for (int e = 0; e < 32; ++e) a.pout[cbase + H * (lane + 32 * e) + h] = v[e];
    }
    __syncwarp();
    }  // replicas
}

template <int H, bool DEAL>
cudaError_t run_ccw(const StepArgs& a, cudaStream_t s) {
    constexpr int CPB = kCcWarps / H;
    dim3 grid((a.hx + CPB - 1) / CPB, (a.R + kCcRpb - 1) / kCcRpb);
    k2c_cols_warp<H, DEAL><<<grid, kCcWarps * 32, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool k2c_colwarp_supported(int ny) { return ny == 1024 || ny == 2048; }

cudaError_t launch_k2c_cols_warp(const StepArgs& a, cudaStream_t s) {
    if (!k2c_colwarp_supported(a.ny) || !a.tw_32 || !a.tw_a || a.rec_phi || a.noise_in || a.pshift)
        return cudaErrorInvalidValue;
    if (a.ny == 1024) return a.dealias ? run_ccw<1, true>(a, s) : run_ccw<1, false>(a, s);
    return a.dealias ? run_ccw<2, true>(a, s) : run_ccw<2, false>(a, s);
}

}  // namespace sft
