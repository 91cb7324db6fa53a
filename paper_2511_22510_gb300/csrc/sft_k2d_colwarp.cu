// sft_k2d_colwarp.cu -- column pass of the 2-D real-field step on columns of
// 1024 points, one warp per column (cubic term).
//
// Same step as the column pass of sft_k2d_cols.cuh (Sec. IV boxed algorithm,
// the y half of steps 3-5): Q --FFT along y--> DFT[q]; F = M s DFT[q];
// phi <- f1 phi + A F + B F_prev + g eta with the Philox noise of App. B;
// Hermitian fix-up on the self-conjugate columns; P <- IFFT_y(M phi / N^2).
// The column's 1024 values are held by the warp in registers (32 per lane,
// index lane + 32 e) through each transform, with one transpose per transform
// through the warp's 8 KB shared buffer; between the transforms the column
// waits in that buffer in natural order while a loop that is not unrolled (so
// the kernel's code stays small enough for the instruction cache) updates two
// slots per trip, loading the state one trip ahead.  The global loads and
// stores of a slot are whole 256-byte lines of the column.  The noise of every mode
// is drawn exactly as in the other column passes (the same counters, the same
// words and the same Box-Muller recipe), so the result is the same step.
#include "sft_step_common.cuh"
#include "sft_warpfft.cuh"

namespace sft {

namespace {

constexpr int kCwNY = 1024;
constexpr int kCwWarps = 4;  // columns per block

// The update of one column (all 1024 modes a_y = lane + 32 e), two slots (one Philox call) per trip of a loop
// that is not unrolled: the column's DFT[q] waits in xb in natural order, the state of the next pair of slots is
// loaded one trip ahead, and xb receives what the inverse transform needs (the masked, scaled new state; on the
// self-conjugate columns the raw new state, fixed up by the caller).  The run-time-uniform choices are template
// parameters: MB (Model B: s = -Gamma u k^2), S2 (SETD2: the history F_prev), PLANE (a_x in {0, nx/2}), HASF
// (the column carries F and P).  Returns the non-finite accumulator.
template <bool DEAL, bool MB, bool S2, bool PLANE, bool HASF>
__device__ __forceinline__ float cw_update(const StepArgs& a, float2* xb, float2* __restrict__ phc,
                                           float2* __restrict__ fpc, const float4* __restrict__ trow, int cc,
                                           int lane, long long step, uint32_t rep, bool first, float sB) {
    constexpr int NY = kCwNY;
    float nf = 0.f;
    float2 ph0 = phc[lane], ph1 = phc[lane + 32];
#pragma unroll 1
    for (int e = 0; e < 32; e += 2) {
        float2 nx0 = czero(), nx1 = czero();
        if (e + 2 < 32) {
            nx0 = phc[lane + 32 * (e + 2)];
            nx1 = phc[lane + 32 * (e + 3)];
        }
        float2 z0, z1;
        team_normal_pair_ks<32>(a.ks, (uint64_t)cc * NY, lane, e, (uint32_t)step, rep, z0, z1);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int ay = lane + 32 * (e + h);
            const int ays = ay < NY / 2 ? ay : ay - NY;  // signed index (ay = 512 -> -512)
            const int aya = ays < 0 ? -ays : ays;
            const bool inm = HASF && (!DEAL || 3 * aya < NY);
            float2 F = czero();
            if (HASF && inm) {
                const float sq = MB ? sB * (float)(cc * cc + ays * ays) : sB;
                F = cscale(xb[ay], sq);
            }
            const float4 t = __ldg(&trow[aya]);  // {f1, A, B, g}
            const float2 ph = h ? ph1 : ph0;
            const float2 eta = eta_of(h ? z1 : z0, PLANE && (ay == 0 || ay == NY / 2));
            float2 out;
            if constexpr (S2 && HASF) {
                // SETD2 (the SETD1 pair A + B, B = 0 at the step that starts the history)
                const float A = first ? t.y + t.z : t.y, B = first ? 0.f : t.z;
                const float2 Fp = fpc[ay];
                out = make_float2(t.x * ph.x + A * F.x + B * Fp.x + t.w * eta.x,
                                  t.x * ph.y + A * F.y + B * Fp.y + t.w * eta.y);
                fpc[ay] = F;
            } else {
                const float A = (S2 && first) ? t.y + t.z : t.y;
                out = make_float2(t.x * ph.x + A * F.x + t.w * eta.x, t.x * ph.y + A * F.y + t.w * eta.y);
            }
            if constexpr (PLANE) {
                xb[ay] = out;  // stored after the fix-up by the caller
            } else {
                phc[ay] = out;
                nf = nonfinite_acc(nf, out);
                xb[ay] = (HASF && inm) ? cscale(out, a.scale) : czero();
            }
        }
        ph0 = nx0;
        ph1 = nx1;
    }
    return nf;
}

// 5 blocks (20 warps) per SM caps the kernel at 96 registers; the latency-bound update loop gains more from the
// extra warps than the transforms lose to the tighter budget.  MB / S2: Model B, SETD2 (see cw_update).
template <bool DEAL, bool MB, bool S2>
__global__ void __launch_bounds__(kCwWarps * 32, 5) k2_cols_warp(const StepArgs a) {
    constexpr int NY = kCwNY;
    // slots e (index lane + 32 e) outside the 2/3 band |a_y| < 342 in every lane: e = 11 .. 20
    constexpr uint32_t ZMASK = DEAL ? 0x001FF800u : 0u;
    __shared__ __align__(16) float2 xbuf[kCwWarps][NY];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cc = blockIdx.x * kCwWarps + warp;
    if (cc >= a.hx) return;  // whole warp
    float2* xb = xbuf[warp];
    const float2* __restrict__ tw32 = a.tw_32;
    const long long step = current_step(a);
    const bool first = (a.scheme == 2) && (step == *a.first_step);
    const bool has_f = cc < a.ncols;
    const bool plane = (cc == 0 || 2 * cc == a.nx);
    const float sB = a.model == 1 ? a.s0 * a.dk * a.dk : a.s0;  // Model B: s = -Gamma u k^2
    const float4* __restrict__ trow = a.tab + (size_t)cc * (NY / 2 + 1);
    for (int ri = 0; ri < a.rpb; ++ri) {
        const int rep = blockIdx.y * a.rpb + ri;
        if (rep >= a.R) break;
        const size_t colbase = ((size_t)rep * a.hx + cc) * NY;
        // DFT_y[q] of the column into xb in natural order (zero outside the carried columns)
        if (has_f) {
            float2 v[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = a.qin[colbase + lane + 32 * e];
            fft1024_warp<false, 0u>(v, xb, lane, tw32);
#pragma unroll
            for (int e = 0; e < 32; ++e) xb[lane + 32 * e] = v[e];
        }
        __syncwarp();
        // the update (cw_update), with the run-time-uniform choices of this column resolved once
        const uint32_t rp = (uint32_t)(a.rep0 + rep);
        float2* phc = a.phi + colbase;
        float2* fpc = S2 ? a.fprev + colbase : nullptr;
        float nf;
        if (plane)
            nf = has_f ? cw_update<DEAL, MB, S2, true, true>(a, xb, phc, fpc, trow, cc, lane, step, rp, first, sB)
                       : cw_update<DEAL, MB, S2, true, false>(a, xb, phc, fpc, trow, cc, lane, step, rp, first, sB);
        else
            nf = has_f ? cw_update<DEAL, MB, S2, false, true>(a, xb, phc, fpc, trow, cc, lane, step, rp, first, sB)
                       : cw_update<DEAL, MB, S2, false, false>(a, xb, phc, fpc, trow, cc, lane, step, rp, first, sB);
        __syncwarp();
        if (plane) {
            // partners a_y > 512 take the conjugate of 1024 - a_y, self-conjugate modes are real; then the
            // state is stored and the masked, scaled column is left in xb
            float2 w[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int ay = lane + 32 * e;
                w[e] = (2 * ay > NY) ? cconj(xb[NY - ay]) : xb[ay];
                if (ay == 0 || 2 * ay == NY) w[e].y = 0.f;
            }
            __syncwarp();
#pragma unroll
            for (int e = 0; e < 32; ++e) {
                const int ay = lane + 32 * e;
                const int aya = ay <= NY / 2 ? ay : NY - ay;
                a.phi[colbase + ay] = w[e];
                nf = nonfinite_acc(nf, w[e]);
                xb[ay] = (has_f && (!DEAL || 3 * aya < NY)) ? cscale(w[e], a.scale) : czero();
            }
            __syncwarp();
        }
        flag_nonfinite_acc(a, nf, step);
        if (has_f) {
            // P <- IFFT_y(M phi / N^2): the masked slots are zero in every lane
            float2 v[32];
#pragma unroll
            for (int e = 0; e < 32; ++e) v[e] = ((ZMASK >> e) & 1u) ? czero() : xb[lane + 32 * e];
            __syncwarp();
            fft1024_warp<true, ZMASK>(v, xb, lane, tw32);
#pragma unroll
            for (int e = 0; e < 32; ++e) a.pout[colbase + lane + 32 * e] = v[e];
        }
        __syncwarp();
    }
}

template <bool DEAL, bool MB, bool S2>
cudaError_t run_cw(const StepArgs& a, cudaStream_t s) {
    StepArgs b = a;
    if (b.rpb < 1) b.rpb = 4;
    dim3 grid((a.hx + kCwWarps - 1) / kCwWarps, (a.R + b.rpb - 1) / b.rpb);
    k2_cols_warp<DEAL, MB, S2><<<grid, kCwWarps * 32, 0, s>>>(b);
    return cudaGetLastError();
}

template <bool DEAL>
cudaError_t run_cw_for(const StepArgs& a, cudaStream_t s) {
    const bool mb = a.model == 1, s2 = a.scheme == 2;
    if (mb) return s2 ? run_cw<DEAL, true, true>(a, s) : run_cw<DEAL, true, false>(a, s);
    return s2 ? run_cw<DEAL, false, true>(a, s) : run_cw<DEAL, false, false>(a, s);
}

}  // namespace

bool k2_colwarp_supported(int nx, int ny, int nl, int dealias) {
    (void)nx;
    return ny == kCwNY && nl == NL_CUBIC && (dealias == 0 || dealias == 1);
}

cudaError_t launch_k2_cols_warp(const StepArgs& a, int nl, cudaStream_t s) {
    if (!k2_colwarp_supported(a.nx, a.ny, nl, a.pshift ? 2 : a.dealias) || !a.tw_32 || a.rec_phi || a.noise_in)
        return cudaErrorInvalidValue;
    return a.dealias ? run_cw_for<true>(a, s) : run_cw_for<false>(a, s);
}

}  // namespace sft
