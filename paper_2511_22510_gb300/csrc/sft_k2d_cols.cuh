// sft_k2d_cols.cuh -- two-pass 2-D step for real fields (Model A/B, KPZ):
// column pass (kernel templates and launchers, instantiated by sft_k2d_cols.cu
// for power-of-two columns and by sft_k2d_cols_mixed.cu for p x 2^k columns).  Layout and the split of the step between the row pass
// (sft_k2d.cu) and this pass:
//
//   column pass (k2_cols): Q --FFT along y--> DFT[q]; F = M s DFT[q];
//                          phi <- f1 phi + A F + B F_prev + g eta (Philox);
//                          Hermitian fix-up; P <- IFFT_y(M phi / N^2)
//
// with phi[a_x][a_y] (a_x in [0, nx/2], a_y in [0, ny)) and P, Q restricted to
// the x-columns inside the dealiasing band (Sec. IV boxed algorithm).
#pragma once
#include "sft_async.cuh"
#include "sft_step_common.cuh"

// Column pass on columns of 512 points and more: SFT_COL_EMAX values per
// thread, SFT_COL_CTA threads per block and SFT_COL_THREADS_SM resident threads
// per SM (more warps in flight hide the HBM and L1 latency of the streaming
// update better than longer per-thread FFT radices).  Shorter columns use 16
// values per thread, 128-thread blocks and 4 blocks per SM.
#ifndef SFT_COL_EMAX
#define SFT_COL_EMAX 8
#endif
#ifndef SFT_COL_CTA
#define SFT_COL_CTA 256
#endif
#ifndef SFT_COL_THREADS_SM
#define SFT_COL_THREADS_SM 768
#endif
#ifndef SFT_RPB
#define SFT_RPB 4  // default replicas per column-pass block: the column's table and twiddle reads then hit L1
#endif

namespace sft {

// Schedules of the column pass of the step on columns of 512 points and more
// (radix schedule and block shape), chosen per lattice by the plan autotuner:
//   0: SFT_COL_EMAX values per thread (1024 = 8 x 8 x 8 x 2), SFT_COL_CTA-thread
//      blocks, SFT_COL_THREADS_SM threads per SM
//   1: 8 values per thread, 256-thread blocks, 1024 threads per SM
//   2: 16 values per thread (1024 = 16 x 16 x 4), 128-thread blocks, 512 per SM
template <int SH>
struct ColShape {
    static constexpr int EM = SFT_COL_EMAX, CTA = SFT_COL_CTA, PER_SM = SFT_COL_THREADS_SM;
};
template <>
struct ColShape<1> {
    static constexpr int EM = 8, CTA = 256, PER_SM = 1024;
};
template <>
struct ColShape<2> {
    static constexpr int EM = 16, CTA = 128, PER_SM = 512;
};

template <int NY, int SH = 0>
struct ColCfg {
    static constexpr bool WIDE = NY >= 512;
    static constexpr int EM = ColShape<SH>::EM;
    using PL = FftPlan<NY, EM>;
    static constexpr int T = PL::T;
    static constexpr int CTA = WIDE ? ColShape<SH>::CTA : 128;
    static constexpr int COLS = T >= CTA ? 1 : CTA / T;
    static constexpr int THREADS = COLS * T;
    static constexpr int PER_SM = WIDE ? ColShape<SH>::PER_SM : 512;
    static constexpr int MINB = PER_SM / THREADS > 1 ? PER_SM / THREADS : 1;
    static constexpr int XB = PL::BUF;
    // the step stages each column's state (and SETD2 history) in shared memory
    // behind the exchange buffers, at a 16-byte aligned offset
    static constexpr int SOFF = (COLS * XB + 1) / 2 * 2;
    static constexpr size_t smem() { return sizeof(float2) * (size_t)COLS * XB; }
    static constexpr size_t smem_step() { return sizeof(float2) * ((size_t)SOFF + 2 * (size_t)COLS * NY); }
};

// Asynchronous copy of one column (NY values) into shared memory, 16 bytes per copy.
template <int NY, int T>
__device__ __forceinline__ void stage_column(float2* dst, const float2* src, int t) {
#pragma unroll
    for (int i = t; i < NY / 2; i += T) cp_async_16_cg(dst + 2 * i, src + 2 * i);
}

// Hermitian fix-up of one column held by a team on the planes a_x in {0, nx/2}:
// partners (a_y > ny/2) take the conjugate of a_y' = ny - a_y, self-conjugate
// modes drop their imaginary part.  Warp-uniform when teams share a warp.
template <int NY, int EM>
__device__ __forceinline__ void fixup_plane(float2 (&out)[FftPlan<NY, EM>::E], float2* xb, int t, bool plane) {
    using PL = FftPlan<NY, EM>;
    constexpr int T = PL::T, E = PL::E;
    if (plane || T < 32) {
        team_sync<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) xb[xpos<NY, EM>(t + T * e)] = out[e];
        team_sync<T>();
        if (plane) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ay = t + T * e;
                if (2 * ay > NY) out[e] = cconj(xb[xpos<NY, EM>(NY - ay)]);
                if (ay == 0 || 2 * ay == NY) out[e].y = 0.f;
            }
        }
    }
}

// Dealiasing mask of mode (cc, a_y) on a 2-D real lattice: 2/3 truncation
// (a.dealias), or, with phase-shift dealiasing (PS), every mode off the
// Nyquist lines.
template <bool PS>
__device__ __forceinline__ bool keep_mode(const StepArgs& a, int cc, int ays, int ny) {
    if constexpr (PS) return 2 * cc != a.nx && 2 * abs(ays) != ny;
    return !a.dealias || (3 * cc < a.nx && 3 * abs(ays) < ny);
}

// e^{-i pi s / N} for the signed index s, |s| < N (half-cell shift phase, conjugated)
__device__ __forceinline__ float2 shift_phase_conj(const float2* __restrict__ tw_ps, int s) {
    const float2 w = __ldg(&tw_ps[abs(s)]);
    return s >= 0 ? w : cconj(w);
}

// P <- IFFT_y(M phi / N^2) for one column (and, for KPZ, P_y <- IFFT_y(i k_y M phi / N^2)):
// the dealiased input of the next row pass.
template <int NY, int NL, int EM>
__device__ __forceinline__ void emit_p(const StepArgs& a, const float2 (&out)[FftPlan<NY, EM>::E], bool has_p, int cc,
                                       size_t colbase, float2* xb, int t) {
    using PL = FftPlan<NY, EM>;
    constexpr int T = PL::T, E = PL::E;
    if (!(has_p || T < 32)) return;
    float2 v[E];
    float2 vy[NL == NL_GRAD2 ? E : 1];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int ay = t + T * e;
        const int ays = signed_idx(ay, NY);
        const bool inm = keep_mode<false>(a, cc, ays, NY);
        v[e] = (has_p && inm) ? cscale(out[e], a.scale) : czero();
        if constexpr (NL == NL_GRAD2) vy[e] = cscale(cmuli(v[e]), a.dk * (float)odd_idx(ay, NY));
    }
    fft_line<NY, true, EM>(v, xb, t, a.tw_a);
    if constexpr (NL == NL_GRAD2) fft_line<NY, true, EM>(vy, xb, t, a.tw_a);
    if (has_p) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            a.pout[colbase + t + T * e] = v[e];
            if constexpr (NL == NL_GRAD2) a.pyout[colbase + t + T * e] = vy[e];
        }
    }
}

// The same under phase-shift dealiasing: P0 and the copy shifted by half a cell
// along y, P1 <- IFFT_y(M phi e^{i pi a_y / N} / N^2) at a.ps_off behind P (KPZ: P_y
// and P_y1 as well), every mode off the Nyquist lines kept; one transform at a time.
template <int NY, int NL, int EM>
__device__ __forceinline__ void emit_p_ps(const StepArgs& a, const float2 (&out)[FftPlan<NY, EM>::E], bool has_p,
                                          int cc, size_t colbase, float2* xb, int t) {
    using PL = FftPlan<NY, EM>;
    constexpr int T = PL::T, E = PL::E;
    if (!(has_p || T < 32)) return;
    // kind: bit 0 the y derivative i k_y, bit 1 the half-cell shift
    auto one = [&](float2* dst, int kind) {
        float2 v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int ay = t + T * e;
            const int ays = signed_idx(ay, NY);
            const bool inm = keep_mode<true>(a, cc, ays, NY);
            float2 x = (has_p && inm) ? cscale(out[e], a.scale) : czero();
            if (kind & 1) x = cscale(cmuli(x), a.dk * (float)odd_idx(ay, NY));
            if (kind & 2) x = cmul(x, cconj(shift_phase_conj(a.tw_ps, ays)));
            v[e] = x;
        }
        fft_line<NY, true, EM>(v, xb, t, a.tw_a);
        if (has_p) {
#pragma unroll
            for (int e = 0; e < E; ++e) dst[colbase + t + T * e] = v[e];
        }
    };
    one(a.pout, 0);
    if constexpr (NL == NL_GRAD2) one(a.pyout, 1);
    one(a.pout + a.ps_off, 2);
    if constexpr (NL == NL_GRAD2) one(a.pyout + a.ps_off, 3);
}

template <int NY, int NL, int MODE, int SH = 0>
__global__ void __launch_bounds__(ColCfg<NY, SH>::THREADS, ColCfg<NY, SH>::MINB) k2_cols_real(const StepArgs a) {
    using C = ColCfg<NY, SH>;
    constexpr int EM = C::EM;
    using PL = FftPlan<NY, EM>;
    constexpr int T = PL::T, E = PL::E, COLS = C::COLS, XB = C::XB;
    extern __shared__ float2 sm[];
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const int c = blockIdx.x * COLS + team;
    const bool valid = c < a.hx;
    const int cc = valid ? c : a.hx - 1;
    const int M = a.nx / 2;
    float2* xb = sm + team * XB;
    const float2* __restrict__ tw = a.tw_a;
    const bool plane = (cc == 0 || cc == M);
    for (int ri = 0; ri < a.rpb; ++ri) {
    const int rep = blockIdx.y * a.rpb + ri;
    if (rep >= a.R) break;
    const size_t colbase = ((size_t)rep * a.hx + cc) * NY;
    float2 v[E];

    if constexpr (MODE == MODE_FWD) {
        if (!valid && T >= 32) return;
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = a.qin[colbase + t + T * e];
        fft_line<NY, false, EM>(v, xb, t, tw);
        team_sync<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) xb[xpos<NY, EM>(t + T * e)] = v[e];
        team_sync<T>();
        if (plane) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ay = t + T * e;
                if (2 * ay > NY) v[e] = cconj(xb[xpos<NY, EM>(NY - ay)]);
                if (ay == 0 || 2 * ay == NY) v[e].y = 0.f;
            }
        }
        if (valid) {
#pragma unroll
            for (int e = 0; e < E; ++e) a.phi[colbase + t + T * e] = v[e];
        }
    } else if constexpr (MODE == MODE_INV) {
        if (!valid && T >= 32) return;
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = cscale(a.phi[colbase + t + T * e], a.scale);
        fft_line<NY, true, EM>(v, xb, t, tw);
        if (valid) {
#pragma unroll
            for (int e = 0; e < E; ++e) a.pout[colbase + t + T * e] = v[e];
        }
    } else if constexpr (MODE == MODE_STEP || MODE == MODE_STEP_REC || MODE == MODE_STEP_RSN ||
                         MODE == MODE_STEP_PS) {
        constexpr bool PS = MODE == MODE_STEP_PS;
        if (!valid && T >= 32) return;
        const long long step = current_step(a);
        const bool first = (a.scheme == 2) && (step == *a.first_step);
        const bool has_f = valid && cc < a.ncols;
        // the state column (and SETD2 history) streams into shared memory while the FFT of Q runs
        float2* sphi = sm + C::SOFF + team * NY;
        float2* sfp = sm + C::SOFF + (COLS + team) * NY;
        team_sync<T>();  // this team's reads of the staging rows (previous replica) are complete
        if (valid) {
            stage_column<NY, T>(sphi, a.phi + colbase, t);
            if (a.scheme == 2 && has_f) stage_column<NY, T>(sfp, a.fprev + colbase, t);
        }
        cp_async_commit();
        if (has_f || T < 32) {
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = has_f ? a.qin[colbase + t + T * e] : czero();
        }
        float2 v1[PS ? E : 1];  // phase shift: Q1, the row pass's result on the grid shifted along y
        if constexpr (PS) {
            if (has_f || T < 32) {
#pragma unroll
                for (int e = 0; e < E; ++e) v1[e] = has_f ? a.qin[a.ps_off + colbase + t + T * e] : czero();
            }
        }
        // the noise depends on no loaded value: drawn while the loads of Q are in flight
        float2 out[E];
        if constexpr (MODE == MODE_STEP_RSN) {
#pragma unroll
            for (int e = 0; e < E; ++e) out[e] = cscale(a.noise_in[colbase + t + T * e], a.noise_scale);
        } else {
#pragma unroll
            for (int e = 0; e < E; e += 2)
                team_normal_pair_ks<T>(a.ks, (uint64_t)cc * NY, t, e, (uint32_t)step, (uint32_t)(a.rep0 + rep), out[e],
                                    out[e + 1]);
        }
        if (has_f || T < 32) fft_line<NY, false, EM>(v, xb, t, tw);
        if constexpr (PS) {
            if (has_f || T < 32) fft_line<NY, false, EM>(v1, xb, t, tw);
        }
        cp_async_wait_all();
        team_sync<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int ay = t + T * e;
            const int ays = signed_idx(ay, NY);
            const int q = cc * cc + ays * ays;
            const bool inm = keep_mode<PS>(a, cc, ays, NY);
            float2 F = czero();
            if constexpr (PS) {
                // mean over the grids shifted along y by 0 and half a cell (each already
                // averaged over the two x shifts by the row pass)
                if (has_f && inm)
                    F = cscale(cadd(v[e], cmul(v1[e], shift_phase_conj(a.tw_ps, ays))), 0.5f * nl_prefactor(a, q).x);
            } else {
                if (has_f && inm) F = cscale(v[e], nl_prefactor(a, q).x);
            }
            const Coefs co = load_coefs<false>(a.tab, cc * (NY / 2 + 1) + abs(ays), first);
            const float2 ph = sphi[ay];
            float2 Fp = czero();
            if (a.scheme == 2 && has_f) Fp = sfp[ay];
            const bool selfc = plane && (ay == 0 || 2 * ay == NY);
            // partners on the self-conjugate planes are overwritten by the fix-up below
            const float2 eta = (MODE == MODE_STEP_RSN) ? make_float2(out[e].x, selfc ? 0.f : out[e].y)
                                                        : eta_of(out[e], selfc);
            out[e] = setd_update<false>(co, ph, F, Fp, eta);
            if (a.scheme == 2 && has_f && valid) a.fprev[colbase + ay] = F;
            if constexpr (MODE == MODE_STEP_REC) {
                const long long kk = step - a.rec_start;
                if (valid && kk >= 0 && kk % a.rec_every == 0 && kk / a.rec_every < a.rec_M) {
                    const size_t ri = (size_t)(kk / a.rec_every) * (size_t)a.rec_n + colbase + ay;
                    a.rec_phi[ri] = ph;
                    a.rec_F[ri] = F;
                }
            }
        }
        if (plane || T < 32) {
            team_sync<T>();
#pragma unroll
            for (int e = 0; e < E; ++e) xb[xpos<NY, EM>(t + T * e)] = out[e];
            team_sync<T>();
            if (plane) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int ay = t + T * e;
                    if (2 * ay > NY) out[e] = cconj(xb[xpos<NY, EM>(NY - ay)]);
                    if (ay == 0 || 2 * ay == NY) out[e].y = 0.f;
                }
            }
        }
        if (valid) {
            float nf = 0.f;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                a.phi[colbase + t + T * e] = out[e];
                nf = nonfinite_acc(nf, out[e]);
            }
            flag_nonfinite_acc(a, nf, step);
        }
        if constexpr (PS)
            emit_p_ps<NY, NL, EM>(a, out, valid && cc < a.ncols, cc, colbase, xb, t);
        else
            emit_p<NY, NL, EM>(a, out, valid && cc < a.ncols, cc, colbase, xb, t);
    } else if constexpr (MODE == MODE_TAN) {
        // primal step as in MODE_STEP, plus the tangent dphi <- f1 dphi + A M s DFT[q'] (no noise)
        if (!valid && T >= 32) return;
        const long long step = current_step(a);
        const bool first = (a.scheme == 2) && (step == *a.first_step);
        const bool has_f = valid && cc < a.ncols;
        float2 dv[E];
        if (has_f || T < 32) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                v[e] = has_f ? a.qin[colbase + t + T * e] : czero();
                dv[e] = has_f ? a.dqin[colbase + t + T * e] : czero();
            }
            fft_line<NY, false, EM>(v, xb, t, tw);
            fft_line<NY, false, EM>(dv, xb, t, tw);
        }
        float2 out[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if ((e & 1) == 0)
                team_normal_pair_ks<T>(a.ks, (uint64_t)cc * NY, t, e, (uint32_t)step, (uint32_t)(a.rep0 + rep), out[e],
                                    out[e + 1]);
            const int ay = t + T * e;
            const int ays = signed_idx(ay, NY);
            const int q = cc * cc + ays * ays;
            const bool inm = !a.dealias || (3 * cc < a.nx && 3 * abs(ays) < NY);
            const float sq = nl_prefactor(a, q).x;
            const float2 F = (has_f && inm) ? cscale(v[e], sq) : czero();
            const float2 dF = (has_f && inm) ? cscale(dv[e], sq) : czero();
            const Coefs co = load_coefs<false>(a.tab, cc * (NY / 2 + 1) + abs(ays), first);
            const bool selfc = plane && (ay == 0 || 2 * ay == NY);
            // SETD2: B F_prev for the primal, B dF_prev with the tangent's own history (zero at the seed)
            float2 Fp = czero(), dFp = czero();
            if (a.scheme == 2 && has_f) {
                Fp = a.fprev[colbase + ay];
                dFp = a.dfprev[colbase + ay];
            }
            out[e] = setd_update<false>(co, a.phi[colbase + ay], F, Fp, eta_of(out[e], selfc));
            dv[e] = setd_update<false>(co, a.dphi[colbase + ay], dF, dFp, czero());
            if (a.scheme == 2 && has_f) {
                a.fprev[colbase + ay] = F;
                a.dfprev[colbase + ay] = dF;
            }
        }
        fixup_plane<NY, EM>(out, xb, t, plane);
        fixup_plane<NY, EM>(dv, xb, t, plane);
        if (valid) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                a.phi[colbase + t + T * e] = out[e];
                a.dphi[colbase + t + T * e] = dv[e];
                flag_nonfinite(a, out[e], step);
            }
        }
        emit_p<NY, NL, EM>(a, out, valid && cc < a.ncols, cc, colbase, xb, t);
        StepArgs b = a;
        b.pout = a.dpout;
        b.pyout = a.dpyout;
        emit_p<NY, NL, EM>(b, dv, valid && cc < a.ncols, cc, colbase, xb, t);
    } else if constexpr (MODE == MODE_ADJ || MODE == MODE_ADJ_PRIME) {
        // adjoint of step n: lam_n = f1 lam_{n+1} + M DFT[v] (v from the row pass), mu_{n-1} = B_n lam_{n+1}
        // (SETD2), then W = IDFT_y(M s (A_{n-1} lam_n + mu_{n-1}) / N^2) for step n - 1.  ADJ_PRIME: W from
        // lam_N alone (mu = 0).
        if (!valid && T >= 32) return;
        const bool has_f = valid && cc < a.ncols;
        float2 lam[E];
        float2 mu[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            lam[e] = a.dphi[colbase + t + T * e];
            mu[e] = czero();
        }
        if constexpr (MODE == MODE_ADJ) {
            if (has_f || T < 32) {
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = has_f ? a.dqin[colbase + t + T * e] : czero();
                fft_line<NY, false, EM>(v, xb, t, tw);
                if constexpr (NL == NL_GRAD2) {
                    // KPZ: dqin = DFT_x(v_x), qin = DFT_x(v_y); the transposed gradients give
                    // -i (k_x DFT[v_x] + k_y DFT[v_y]) (odd multipliers: zero at the Nyquist indices)
                    float2 vy[E];
#pragma unroll
                    for (int e = 0; e < E; ++e) vy[e] = has_f ? a.qin[colbase + t + T * e] : czero();
                    fft_line<NY, false, EM>(vy, xb, t, tw);
                    const float kx = a.dk * (float)odd_idx(cc, a.nx);
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const float ky = a.dk * (float)odd_idx(t + T * e, NY);
                        const float2 w = make_float2(kx * v[e].x + ky * vy[e].x, kx * v[e].y + ky * vy[e].y);
                        v[e] = make_float2(w.y, -w.x);
                    }
                }
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ay = t + T * e;
                const int ays = signed_idx(ay, NY);
                const bool inm = !a.dealias || (3 * cc < a.nx && 3 * abs(ays) < NY);
                const float f1 = __ldg(&a.tab[cc * (NY / 2 + 1) + abs(ays)]).x;
                const float2 dv = (has_f && inm) ? v[e] : czero();
                if (a.scheme == 2 && !a.adj_first_n) {
                    const float b = __ldg(&a.tab[cc * (NY / 2 + 1) + abs(ays)]).z;
                    mu[e] = cscale(lam[e], b);
                }
                lam[e] = make_float2(f1 * lam[e].x + dv.x, f1 * lam[e].y + dv.y);
            }
            fixup_plane<NY, EM>(lam, xb, t, plane);
            if (valid) {
#pragma unroll
                for (int e = 0; e < E; ++e) a.dphi[colbase + t + T * e] = lam[e];
            }
        }
        const bool has_p = valid && cc < a.ncols;
        if (has_p || T < 32) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ay = t + T * e;
                const int ays = signed_idx(ay, NY);
                const int q = cc * cc + ays * ays;
                const bool inm = !a.dealias || (3 * cc < a.nx && 3 * abs(ays) < NY);
                const Coefs co = load_coefs<false>(a.tab, cc * (NY / 2 + 1) + abs(ays), a.adj_first_prev != 0);
                const float2 nu = make_float2(co.A.x * lam[e].x + mu[e].x, co.A.x * lam[e].y + mu[e].y);
                v[e] = (has_p && inm) ? cscale(nu, nl_prefactor(a, q).x * a.scale) : czero();
            }
            fft_line<NY, true, EM>(v, xb, t, tw);
            if (has_p) {
#pragma unroll
                for (int e = 0; e < E; ++e) a.dpout[colbase + t + T * e] = v[e];
            }
        }
    } else if constexpr (MODE == MODE_PRIME) {
        if (!valid && T >= 32) return;
        const bool has_p = valid && cc < a.ncols;
        float2 out[E];
#pragma unroll
        for (int e = 0; e < E; ++e) out[e] = has_p ? a.phi[colbase + t + T * e] : czero();
        if (a.pshift)
            emit_p_ps<NY, NL, EM>(a, out, has_p, cc, colbase, xb, t);
        else
            emit_p<NY, NL, EM>(a, out, has_p, cc, colbase, xb, t);
    }
    }  // replicas
}

// ----------------------------------------------------------------- launchers
template <int NY, int NL, int MODE, int SH = 0>
static cudaError_t run_cols(const StepArgs& a, cudaStream_t s) {
    using C = ColCfg<NY, SH>;
    const size_t sm = (MODE == MODE_STEP || MODE == MODE_STEP_REC || MODE == MODE_STEP_RSN || MODE == MODE_STEP_PS)
                          ? C::smem_step()
                          : C::smem();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k2_cols_real<NY, NL, MODE, SH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    StepArgs b = a;
    if (b.rpb < 1) b.rpb = SFT_RPB;
    dim3 grid((a.hx + C::COLS - 1) / C::COLS, (a.R + b.rpb - 1) / b.rpb);
    k2_cols_real<NY, NL, MODE, SH><<<grid, C::THREADS, sm, s>>>(b);
    return cudaGetLastError();
}

template <int NY, int NL>
static cudaError_t cols_step(const StepArgs& a, cudaStream_t s, int shape) {
    if (a.rec_phi) return run_cols<NY, NL, MODE_STEP_REC, 0>(a, s);  // recording: the default schedule
    if (a.noise_in) return run_cols<NY, NL, MODE_STEP_RSN, 0>(a, s);  // real-space noise: the default schedule
    if (a.pshift) return run_cols<NY, NL, MODE_STEP_PS, 0>(a, s);  // phase-shift dealiasing
    if constexpr (ColCfg<NY>::WIDE) {
        if (shape == 1) return run_cols<NY, NL, MODE_STEP, 1>(a, s);
        if (shape == 2) return run_cols<NY, NL, MODE_STEP, 2>(a, s);
    }
    return run_cols<NY, NL, MODE_STEP, 0>(a, s);
}

template <int NY>
static cudaError_t cols_for(const StepArgs& a, int mode, int nl, cudaStream_t s, int shape) {
    if (mode == MODE_FWD) return run_cols<NY, NL_CUBIC, MODE_FWD>(a, s);
    if (mode == MODE_INV) return run_cols<NY, NL_CUBIC, MODE_INV>(a, s);
    if (mode == MODE_STEP && nl == NL_CUBIC) return cols_step<NY, NL_CUBIC>(a, s, shape);
    if (mode == MODE_STEP && nl == NL_GRAD2) return cols_step<NY, NL_GRAD2>(a, s, shape);
    if (mode == MODE_PRIME && nl == NL_CUBIC) return run_cols<NY, NL_CUBIC, MODE_PRIME>(a, s);
    if (mode == MODE_PRIME && nl == NL_GRAD2) return run_cols<NY, NL_GRAD2, MODE_PRIME>(a, s);
    if (mode == MODE_TAN && nl == NL_CUBIC) return run_cols<NY, NL_CUBIC, MODE_TAN>(a, s);
    if (mode == MODE_TAN && nl == NL_GRAD2) return run_cols<NY, NL_GRAD2, MODE_TAN>(a, s);
    if (mode == MODE_ADJ && nl == NL_CUBIC) return run_cols<NY, NL_CUBIC, MODE_ADJ>(a, s);
    if (mode == MODE_ADJ_PRIME && nl == NL_CUBIC) return run_cols<NY, NL_CUBIC, MODE_ADJ_PRIME>(a, s);
    if (mode == MODE_ADJ && nl == NL_GRAD2) return run_cols<NY, NL_GRAD2, MODE_ADJ>(a, s);
    if (mode == MODE_ADJ_PRIME && nl == NL_GRAD2) return run_cols<NY, NL_GRAD2, MODE_ADJ_PRIME>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace sft
