// sft_k1d.cuh -- whole-step 1-D kernels (templates and launchers, instantiated
// by sft_k1d.cu for power-of-two lines and by sft_k1d_mixed.cu for p x 2^k
// lines): one team of threads holds one replica's
// spectrum in registers for the entire step (Sec. IV boxed algorithm), so the
// only HBM traffic is one read and one write of the state (plus the SETD2
// history).  Real fields keep the Hermitian half a in [0, N/2] and transform
// through the N/2-point complex FFT; complex fields (CGL) use full C2C lines.
#pragma once
#include "sft_step_common.cuh"

namespace sft {

// the step and transforms on real lines of p x 2^k points, p in {3, 5, 7} (sft_k1d_mixed.cu)
cudaError_t launch_k1_line_mixed(const StepArgs& a, int mode, int nl, cudaStream_t s);

// Index of the mirrored entry (M - k) mod M of an M-point line.
template <int M>
__device__ __forceinline__ int line_mirror(int k) {
    if constexpr ((M & (M - 1)) == 0)
        return (M - k) & (M - 1);
    else
        return k == 0 ? 0 : M - k;
}

template <int M>
struct LineCfg {
    using PL = FftPlan<M>;
    static constexpr int T = PL::T;
    static constexpr int LINES = T >= 128 ? 1 : 128 / T;
    static constexpr int THREADS = LINES * T;
    static constexpr int XB = PL::BUF;
    static constexpr size_t smem() { return sizeof(float2) * (size_t)LINES * XB; }
};

// R2C post-processing of a line held by a team: Xq[e] = X[t + T e] for the
// N/2 = M lowest modes, XqM = the Nyquist mode (valid in every thread).
template <int M>
__device__ __forceinline__ void line_post(float2 (&z)[FftPlan<M>::E], float2* xb, int t,
                                          const float2* __restrict__ twN, float2 (&Xq)[FftPlan<M>::E], float2& XqM) {
    using PL = FftPlan<M>;
    constexpr int T = PL::T, E = PL::E;
    team_sync<T>();
#pragma unroll
    for (int e = 0; e < E; ++e) xb[xpos<M>(t + T * e)] = z[e];
    team_sync<T>();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + T * e;
        Xq[e] = r2c_post(z[e], cconj(xb[xpos<M>(line_mirror<M>(k))]), __ldg(&twN[k]));
    }
    const float2 z0 = xb[0];
    XqM = make_float2(z0.x - z0.y, 0.f);
}

// One SETD step of one real 1-D replica held by a team of T threads (Sec. IV
// boxed algorithm): inverse transform of the masked state, nonlinearity,
// forward transform, update with Philox noise.  r: replica (clamped when the
// team is idle, valid = false); xb: the team's exchange buffer.
template <int M, int NL>
__device__ __forceinline__ void line_step(const StepArgs& a, int r, bool valid, int t, float2* xb) {
    using PL = FftPlan<M>;
    constexpr int T = PL::T, E = PL::E;
    constexpr int NX = 2 * M;
    const float2* __restrict__ twM = a.tw_a;
    const float2* __restrict__ twN = a.tw_b;
    float2* ph = a.phi + (size_t)r * (M + 1);
    const float sc = a.scale;
    float2 z[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + T * e;
        float2 X = ph[k], Xm = ph[M - k];
        X = (!a.dealias || 3 * k < NX) ? cscale(X, sc) : czero();
        Xm = (!a.dealias || 3 * (M - k) < NX) ? cscale(Xm, sc) : czero();
        if constexpr (NL == NL_GRAD2) {
            X = cscale(cmuli(X), a.dk * (float)k);
            Xm = cscale(cmuli(Xm), k == 0 ? 0.f : a.dk * (float)(M - k));
        }
        z[e] = c2r_pre(X, Xm, __ldg(&twN[k]));
    }
    fft_line<M, true>(z, xb, t, twM);
#pragma unroll
    for (int e = 0; e < E; ++e) {
        if constexpr (NL == NL_GRAD2)
            z[e] = make_float2(z[e].x * z[e].x, z[e].y * z[e].y);
        else
            z[e] = make_float2(z[e].x * z[e].x * z[e].x, z[e].y * z[e].y * z[e].y);
    }
    fft_line<M, false>(z, xb, t, twM);
    float2 Xq[E];
    float2 XqM;
    line_post<M>(z, xb, t, twN, Xq, XqM);
    const long long step = current_step(a);
    const bool first = (a.scheme == 2) && (step == *a.first_step);
    float2* fp = a.fprev + (size_t)r * (M + 1);
    const uint32_t rep = (uint32_t)(a.rep0 + r);
    float2 zn0, zn1;
    // modes k = t + T e, then (thread 0) the Nyquist mode k = M
#pragma unroll
    for (int e = 0; e <= E; ++e) {
        if (e < E && (e & 1) == 0) team_normal_pair_ks<T>(a.ks, 0, t, e, (uint32_t)step, rep, zn0, zn1);
        if (e == E && t != 0) break;
        const int k = (e < E) ? t + T * e : M;
        const float2 xq = (e < E) ? Xq[e] : XqM;
        const bool inm = !a.dealias || 3 * k < NX;
        const float2 F = inm ? cscale(xq, nl_prefactor(a, k * k).x) : czero();
        const Coefs co = load_coefs<false>(a.tab, k, first);
        const float2 phv = ph[k];
        const float2 Fp = (a.scheme == 2) ? fp[k] : czero();
        const bool selfc = (k == 0 || k == M);
        const float2 eta = (e < E) ? eta_of((e & 1) ? zn1 : zn0, selfc)
                                   : fourier_noise(a.seed, (uint64_t)k, (uint32_t)step, rep, selfc);
        float2 o = setd_update<false>(co, phv, F, Fp, eta);
        if (selfc) o.y = 0.f;
        if (valid) {
            ph[k] = o;
            if (a.scheme == 2) fp[k] = F;
            flag_nonfinite(a, o, step);
        }
    }
}

// Variants of the 1-D step (the alternatives of Sec. IV steps 1 and 2), on one line per team:
//   MODE_STEP_PS: phase-shift dealiasing -- the nonlinear term is the mean of its evaluation on the plain grid
//     and on the grid shifted by half a cell (input phases e^{i pi k / N}, output phases e^{-i pi k / N}); the
//     Nyquist mode is masked on input and output and every other mode is kept;
//   MODE_STEP_RSN: real-space noise -- site s of the line takes normal s & 3 of Philox(s >> 2, step, replica,
//     tag 3), and the update uses eta_k = DFT[eta]_k / sqrt(N) (a.noise_scale = 1 / sqrt(N)).
// The plain evaluation of the nonlinear term waits in a.qout (M + 1 entries per line, each thread reading back
// the entries it wrote) while the second transform pair runs, so that two spectra are never live in registers.
template <int M, int NL, int MODE>
__device__ __forceinline__ void line_step_var(const StepArgs& a, int r, bool valid, int t, float2* xb) {
    using PL = FftPlan<M>;
    constexpr int T = PL::T, E = PL::E;
    constexpr int NX = 2 * M;
    constexpr bool PS = MODE == MODE_STEP_PS;
    constexpr bool G = NL == NL_GRAD2;
    static_assert(NL == NL_CUBIC || G, "1-D variants: cubic or gradient-squared term");
    const float2* __restrict__ twM = a.tw_a;
    const float2* __restrict__ twN = a.tw_b;
    const float2* __restrict__ tps = a.tw_ps;  // e^{-i pi m / N}
    float2* ph = a.phi + (size_t)r * (M + 1);
    const float sc = a.scale;
    const long long step = current_step(a);
    const uint32_t rep = (uint32_t)(a.rep0 + r);
    // the nonlinear term evaluated on the plain grid (shift = false) or the shifted one: Xq[e] for the modes
    // k = t + T e, XqM for the Nyquist mode
    auto q_of = [&](bool shift, float2 (&Xq)[E], float2& XqM) {
        float2 z[E];
        // unrolled in groups of four: fewer input loads in flight, so the long lines do not spill
#pragma unroll 4
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            float2 X = ph[k], Xm = ph[M - k];
            if constexpr (PS) {
                X = cscale(X, sc);
                Xm = (k == 0) ? czero() : cscale(Xm, sc);  // the Nyquist mode is masked
            } else {
                X = (!a.dealias || 3 * k < NX) ? cscale(X, sc) : czero();
                Xm = (!a.dealias || 3 * (M - k) < NX) ? cscale(Xm, sc) : czero();
            }
            if constexpr (G) {
                X = cscale(cmuli(X), a.dk * (float)k);
                Xm = cscale(cmuli(Xm), k == 0 ? 0.f : a.dk * (float)(M - k));
            }
            if (shift) {
                X = cmul(X, cconj(__ldg(&tps[k])));
                Xm = cmul(Xm, cconj(__ldg(&tps[M - k])));
            }
            z[e] = c2r_pre(X, Xm, __ldg(&twN[k]));
        }
        fft_line<M, true>(z, xb, t, twM);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if constexpr (G)
                z[e] = make_float2(z[e].x * z[e].x, z[e].y * z[e].y);
            else
                z[e] = make_float2(z[e].x * z[e].x * z[e].x, z[e].y * z[e].y * z[e].y);
        }
        fft_line<M, false>(z, xb, t, twM);
        line_post<M>(z, xb, t, twN, Xq, XqM);
        if (shift) {
#pragma unroll
            for (int e = 0; e < E; ++e) Xq[e] = cmul(Xq[e], __ldg(&tps[t + T * e]));
        }
    };
    float2* qs = a.qout + (size_t)r * (M + 1);
    {
        float2 Xp[E], XpM;
        q_of(false, Xp, XpM);
        if (valid) {
#pragma unroll
            for (int e = 0; e < E; ++e) qs[t + T * e] = Xp[e];
            if (t == 0) qs[M] = XpM;
        }
    }
    // PS: Xq <- the shifted evaluation, averaged with the plain one below; RSN: Xq <- the noise spectrum
    float2 Xq[E], XqM;
    if constexpr (PS) {
        q_of(true, Xq, XqM);
    } else {
        // the packed pair m = t + T e holds sites 2m, 2m + 1: normal pair m of the tag-3 stream
#pragma unroll
        for (int e = 0; e < E; e += 2)
            team_normal_pair_ks<T>(a.ks, 0, t, e, (uint32_t)step, rep, Xq[e], Xq[e + 1], 3u);
        fft_line<M, false>(Xq, xb, t, twM);
        line_post<M>(Xq, xb, t, twN, Xq, XqM);
    }
    const bool first = (a.scheme == 2) && (step == *a.first_step);
    float2* fp = a.fprev + (size_t)r * (M + 1);
    float2 zn0 = czero(), zn1 = czero();
    // modes k = t + T e, then (thread 0) the Nyquist mode k = M
#pragma unroll
    for (int e = 0; e <= E; ++e) {
        if constexpr (PS) {
            if (e < E && (e & 1) == 0) team_normal_pair_ks<T>(a.ks, 0, t, e, (uint32_t)step, rep, zn0, zn1);
        }
        if (e == E && t != 0) break;
        const int k = (e < E) ? t + T * e : M;
        const float2 xv = (e < E) ? Xq[e] : XqM;
        float2 xq = qs[k];  // the plain evaluation, written by this thread
        if constexpr (PS) xq = cscale(cadd(xq, xv), 0.5f);
        const bool inm = PS ? (k != M) : (!a.dealias || 3 * k < NX);
        const float2 F = inm ? cscale(xq, nl_prefactor(a, k * k).x) : czero();
        const Coefs co = load_coefs<false>(a.tab, k, first);
        const float2 phv = ph[k];
        const float2 Fp = (a.scheme == 2) ? fp[k] : czero();
        const bool selfc = (k == 0 || k == M);
        float2 eta;
        if constexpr (PS) {
            eta = (e < E) ? eta_of((e & 1) ? zn1 : zn0, selfc)
                          : fourier_noise(a.seed, (uint64_t)k, (uint32_t)step, rep, selfc);
        } else {
            eta = cscale(xv, a.noise_scale);
            if (selfc) eta.y = 0.f;
        }
        float2 o = setd_update<false>(co, phv, F, Fp, eta);
        if (selfc) o.y = 0.f;
        if (valid) {
            ph[k] = o;
            if (a.scheme == 2) fp[k] = F;
            flag_nonfinite(a, o, step);
        }
    }
}

// Real field, N = 2M points.  Mode k of replica r sits at phi[r * (M + 1) + k].
template <int M, int NL, int MODE>
__global__ void __launch_bounds__(LineCfg<M>::THREADS) k1_real(const StepArgs a) {
    using C = LineCfg<M>;
    using PL = FftPlan<M>;
    constexpr int T = PL::T, E = PL::E, LINES = C::LINES, XB = C::XB;
    constexpr int NX = 2 * M;
    extern __shared__ float2 sm[];
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const int r = blockIdx.x * LINES + team;
    const bool valid = r < a.R;
    const int rr = valid ? r : a.R - 1;
    float2* xb = sm + team * XB;
    const float2* __restrict__ twM = a.tw_a;
    const float2* __restrict__ twN = a.tw_b;
    float2* ph = a.phi + (size_t)rr * (M + 1);
    float2 z[E];

    if constexpr (MODE == MODE_STEP_PS || MODE == MODE_STEP_RSN) {
        line_step_var<M, NL, MODE>(a, rr, valid, t, xb);
        return;
    }
    if constexpr (MODE == MODE_TAN || MODE == MODE_ADJ) {
        // TAN: primal step plus dphi <- f1 dphi + A M s DFT[q'] with q' = 3 psi^2 dpsi (cubic,
        // dpsi = IDFT(M dphi)) or 2 g dg (KPZ, g = IDFT(i k M phi), dg = IDFT(i k M dphi)).
        // ADJ: lam <- f1 lam + M DFT[3 psi^2 w] (cubic) or (-i k) M DFT[2 g w] (KPZ: the transpose of the
        // odd multiplier i k), w = IDFT(A s M lam), psi and g from the primal state phi.
        static_assert(NL == NL_CUBIC || NL == NL_GRAD2, "tangent/adjoint: cubic or gradient-squared term");
        constexpr bool G = NL == NL_GRAD2;
        float2* dp = a.dphi + (size_t)rr * (M + 1);
        const float sc = a.scale;
        float2 zd[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            const bool i1 = !a.dealias || 3 * k < NX, i2 = !a.dealias || 3 * (M - k) < NX;
            const float2 tw = __ldg(&twN[k]);
            // KPZ: i k on the primal (and on the tangent), k = 0 at the Nyquist mode M - 0
            const float k1 = a.dk * (float)k, k2 = k == 0 ? 0.f : a.dk * (float)(M - k);
            float2 X1 = i1 ? cscale(ph[k], sc) : czero(), X2 = i2 ? cscale(ph[M - k], sc) : czero();
            if constexpr (G) {
                X1 = cscale(cmuli(X1), k1);
                X2 = cscale(cmuli(X2), k2);
            }
            z[e] = c2r_pre(X1, X2, tw);
            float w1 = sc, w2 = sc;
            float2 L1 = dp[k], L2 = dp[M - k];
            if constexpr (MODE == MODE_ADJ) {
                // nu_n = A_n lam_{n+1} + mu_n (SETD2 history cotangent, kept between the steps in dmu)
                const bool fa = a.adj_first_n != 0;
                L1 = cscale(L1, load_coefs<false>(a.tab, k, fa).A.x);
                L2 = cscale(L2, load_coefs<false>(a.tab, M - k, fa).A.x);
                if (a.scheme == 2) {
                    const float2* mu = a.dmu + (size_t)rr * (M + 1);
                    L1 = cadd(L1, mu[k]);
                    L2 = cadd(L2, mu[M - k]);
                }
                w1 *= nl_prefactor(a, k * k).x;
                w2 *= nl_prefactor(a, (M - k) * (M - k)).x;
            }
            float2 D1 = i1 ? cscale(L1, w1) : czero(), D2 = i2 ? cscale(L2, w2) : czero();
            if constexpr (G && MODE == MODE_TAN) {
                D1 = cscale(cmuli(D1), k1);
                D2 = cscale(cmuli(D2), k2);
            }
            zd[e] = c2r_pre(D1, D2, tw);
        }
        fft_line<M, true>(z, xb, t, twM);
        fft_line<M, true>(zd, xb, t, twM);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float2 p = z[e];
            if constexpr (G) {
                zd[e] = make_float2(2.f * p.x * zd[e].x, 2.f * p.y * zd[e].y);
                z[e] = make_float2(p.x * p.x, p.y * p.y);
            } else {
                zd[e] = make_float2(3.f * p.x * p.x * zd[e].x, 3.f * p.y * p.y * zd[e].y);
                z[e] = make_float2(p.x * p.x * p.x, p.y * p.y * p.y);
            }
        }
        fft_line<M, false>(zd, xb, t, twM);
        float2 dXq[E];
        float2 dXqM;
        line_post<M>(zd, xb, t, twN, dXq, dXqM);
        if constexpr (MODE == MODE_ADJ) {
#pragma unroll
            for (int e = 0; e <= E; ++e) {
                if (e == E && t != 0) break;
                const int k = (e < E) ? t + T * e : M;
                const bool inm = !a.dealias || 3 * k < NX;
                float2 v = inm ? ((e < E) ? dXq[e] : dXqM) : czero();
                if constexpr (G) v = cscale(cmuli(v), k == M ? 0.f : -a.dk * (float)k);  // (-i k), odd: 0 at Nyquist
                const float4 tk = __ldg(&a.tab[k]);
                const float2 lk = dp[k];
                float2 o = make_float2(tk.x * lk.x + v.x, tk.x * lk.y + v.y);
                if (k == 0 || k == M) o.y = 0.f;
                if (valid) {
                    dp[k] = o;
                    // SETD2: mu_{n-1} = B_n lam_{n+1}
                    if (a.scheme == 2) a.dmu[(size_t)rr * (M + 1) + k] = a.adj_first_n ? czero() : cscale(lk, tk.z);
                }
            }
            return;
        } else {
            fft_line<M, false>(z, xb, t, twM);
            float2 Xq[E];
            float2 XqM;
            line_post<M>(z, xb, t, twN, Xq, XqM);
            const long long step = current_step(a);
            const bool first = (a.scheme == 2) && (step == *a.first_step);
            const uint32_t rep = (uint32_t)(a.rep0 + rr);
            float2* fp = a.fprev + (size_t)rr * (M + 1);
            float2* dfp = a.dfprev + (size_t)rr * (M + 1);
            float2 zn0, zn1;
#pragma unroll
            for (int e = 0; e <= E; ++e) {
                if (e < E && (e & 1) == 0) team_normal_pair_ks<T>(a.ks, 0, t, e, (uint32_t)step, rep, zn0, zn1);
                if (e == E && t != 0) break;
                const int k = (e < E) ? t + T * e : M;
                const bool inm = !a.dealias || 3 * k < NX;
                const float sq = nl_prefactor(a, k * k).x;
                const float2 F = inm ? cscale((e < E) ? Xq[e] : XqM, sq) : czero();
                const float2 dF = inm ? cscale((e < E) ? dXq[e] : dXqM, sq) : czero();
                const Coefs co = load_coefs<false>(a.tab, k, first);
                const bool selfc = (k == 0 || k == M);
                const float2 eta = (e < E) ? eta_of((e & 1) ? zn1 : zn0, selfc)
                                           : fourier_noise(a.seed, (uint64_t)k, (uint32_t)step, rep, selfc);
                // SETD2: B F_prev for the primal, B dF_prev with the tangent's own history (zero at the seed)
                const float2 Fp = (a.scheme == 2) ? fp[k] : czero();
                const float2 dFp = (a.scheme == 2) ? dfp[k] : czero();
                float2 o = setd_update<false>(co, ph[k], F, Fp, eta);
                float2 d = setd_update<false>(co, dp[k], dF, dFp, czero());
                if (selfc) {
                    o.y = 0.f;
                    d.y = 0.f;
                }
                if (valid) {
                    ph[k] = o;
                    dp[k] = d;
                    if (a.scheme == 2) {
                        fp[k] = F;
                        dfp[k] = dF;
                    }
                    flag_nonfinite(a, o, step);
                }
            }
            return;
        }
    }

    if constexpr (MODE == MODE_STEP) {
        line_step<M, NL>(a, rr, valid, t, xb);
        return;
    }
    if constexpr (MODE == MODE_FWD) {
        const float* src = a.real_io + (size_t)rr * NX;
#pragma unroll
        for (int e = 0; e < E; ++e) z[e] = *reinterpret_cast<const float2*>(src + 2 * (t + T * e));
    } else {
        const float sc = a.scale;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            float2 X = ph[k], Xm = ph[M - k];
            if constexpr (MODE == MODE_STEP) {
                X = (!a.dealias || 3 * k < NX) ? cscale(X, sc) : czero();
                Xm = (!a.dealias || 3 * (M - k) < NX) ? cscale(Xm, sc) : czero();
                if constexpr (NL == NL_GRAD2) {
                    X = cscale(cmuli(X), a.dk * (float)k);
                    Xm = cscale(cmuli(Xm), k == 0 ? 0.f : a.dk * (float)(M - k));
                }
            } else {
                X = cscale(X, sc);
                Xm = cscale(Xm, sc);
            }
            z[e] = c2r_pre(X, Xm, __ldg(&twN[k]));
        }
        fft_line<M, true>(z, xb, t, twM);
        if constexpr (MODE == MODE_INV) {
            if (valid) {
                float* dst = a.real_io + (size_t)rr * NX;
#pragma unroll
                for (int e = 0; e < E; ++e) *reinterpret_cast<float2*>(dst + 2 * (t + T * e)) = z[e];
            }
            return;
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if constexpr (NL == NL_GRAD2)
                    z[e] = make_float2(z[e].x * z[e].x, z[e].y * z[e].y);
                else
                    z[e] = make_float2(z[e].x * z[e].x * z[e].x, z[e].y * z[e].y * z[e].y);
            }
        }
    }
    if constexpr (MODE != MODE_INV) {
        fft_line<M, false>(z, xb, t, twM);
        team_sync<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) xb[xpos<M>(t + T * e)] = z[e];
        team_sync<T>();
        float2 Xq[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            Xq[e] = r2c_post(z[e], cconj(xb[xpos<M>(line_mirror<M>(k))]), __ldg(&twN[k]));
        }
        const float2 z0 = xb[0];
        const float2 XqM = make_float2(z0.x - z0.y, 0.f);
        if constexpr (MODE == MODE_FWD) {
            if (valid) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    float2 v = Xq[e];
                    if (t + T * e == 0) v.y = 0.f;
                    ph[t + T * e] = v;
                }
                if (t == 0) ph[M] = XqM;
            }
        } else {
            const long long step = current_step(a);
            const bool first = (a.scheme == 2) && (step == *a.first_step);
            float2* fp = a.fprev + (size_t)rr * (M + 1);
            const uint32_t rep = (uint32_t)(a.rep0 + rr);
            float2 zn0, zn1;
            // modes k = t + T e, then (thread 0) the Nyquist mode k = M
#pragma unroll
            for (int e = 0; e <= E; ++e) {
                if (e < E && (e & 1) == 0) team_normal_pair_ks<T>(a.ks, 0, t, e, (uint32_t)step, rep, zn0, zn1);
                if (e == E && t != 0) break;
                const int k = (e < E) ? t + T * e : M;
                const float2 xq = (e < E) ? Xq[e] : XqM;
                const bool inm = !a.dealias || 3 * k < NX;
                const int q = k * k;
                const float2 F = inm ? cscale(xq, nl_prefactor(a, q).x) : czero();
                const Coefs co = load_coefs<false>(a.tab, k, first);
                const float2 phv = ph[k];
                const float2 Fp = (a.scheme == 2) ? fp[k] : czero();
                const bool selfc = (k == 0 || k == M);
                const float2 eta = (e < E) ? eta_of((e & 1) ? zn1 : zn0, selfc)
                                           : fourier_noise(a.seed, (uint64_t)k, (uint32_t)step, rep, selfc);
                float2 o = setd_update<false>(co, phv, F, Fp, eta);
                if (selfc) o.y = 0.f;
                if (valid) {
                    ph[k] = o;
                    if (a.scheme == 2) fp[k] = F;
                    flag_nonfinite(a, o, step);
                }
            }
        }
    }
}

// Complex field of N points (CGL).  Mode k of replica r at phi[r * N + k].
template <int N, int MODE>
__global__ void __launch_bounds__(LineCfg<N>::THREADS) k1_cplx(const StepArgs a) {
    using C = LineCfg<N>;
    using PL = FftPlan<N>;
    constexpr int T = PL::T, E = PL::E, LINES = C::LINES, XB = C::XB;
    extern __shared__ float2 sm[];
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const int r = blockIdx.x * LINES + team;
    const bool valid = r < a.R;
    const int rr = valid ? r : a.R - 1;
    float2* xb = sm + team * XB;
    const float2* __restrict__ tw = a.tw_a;
    float2* ph = a.phi + (size_t)rr * N;
    float2 z[E];
    if constexpr (MODE == MODE_FWD) {
        const float2* src = a.cplx_io + (size_t)rr * N;
#pragma unroll
        for (int e = 0; e < E; ++e) z[e] = src[t + T * e];
        fft_line<N, false>(z, xb, t, tw);
        if (valid) {
#pragma unroll
            for (int e = 0; e < E; ++e) ph[t + T * e] = z[e];
        }
        return;
    }
    float2 raw[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + T * e;
        raw[e] = ph[k];
        const bool inm = !a.dealias || 3 * abs(signed_idx(k, N)) < N;
        z[e] = (MODE == MODE_INV || inm) ? cscale(raw[e], a.scale) : czero();
    }
    fft_line<N, true>(z, xb, t, tw);
    if constexpr (MODE == MODE_INV) {
        if (valid) {
            float2* dst = a.cplx_io + (size_t)rr * N;
#pragma unroll
            for (int e = 0; e < E; ++e) dst[t + T * e] = z[e];
        }
        return;
    } else if constexpr (MODE == MODE_ADJ) {
        // adjoint for the real inner product Re sum conj(u) v: every Fourier multiplier transposes to its
        // conjugate and the pointwise 2 |A|^2 dA + A^2 conj(dA) is its own transpose (Sec. V.C linearised):
        //   nu = conj(a_n) lam + mu,  w = IDFT(M conj(s) nu),  lam <- conj(f1) lam + M DFT[2 |A|^2 w + A^2 conj(w)],
        //   mu <- conj(b_n) lam (SETD2 history cotangent; zero at the step that starts SETD2)
        float2* dp = a.dphi + (size_t)rr * N;
        float2* mu = a.scheme == 2 ? a.dmu + (size_t)rr * N : nullptr;
        const bool fa = a.adj_first_n != 0;
        const float2 sw = make_float2(a.s0 * a.scale, -a.s0i * a.scale);  // conj(s) / N
        float2 lam[E], zw[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            const int ks = signed_idx(k, N);
            const bool inm = !a.dealias || 3 * abs(ks) < N;
            lam[e] = dp[k];
            const Coefs co = load_coefs<true>(a.tab, abs(ks), fa);
            float2 nu = cmul(cconj(co.A), lam[e]);
            if (mu) nu = cadd(nu, mu[k]);
            zw[e] = inm ? cmul(sw, nu) : czero();
        }
        fft_line<N, true>(zw, xb, t, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float2 A = z[e], w = zw[e];
            zw[e] = cadd(cscale(w, 2.f * (A.x * A.x + A.y * A.y)), cmul(cmul(A, A), cconj(w)));
        }
        fft_line<N, false>(zw, xb, t, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            const int ks = signed_idx(k, N);
            const bool inm = !a.dealias || 3 * abs(ks) < N;
            const Coefs co = load_coefs<true>(a.tab, abs(ks), fa);
            const float2 o = cadd(cmul(cconj(co.f1), lam[e]), inm ? zw[e] : czero());
            if (valid) {
                dp[k] = o;
                if (mu) mu[k] = fa ? czero() : cmul(cconj(co.B), lam[e]);
            }
        }
        return;
    } else {
        // tangent (MODE_TAN): dq = 2 |A|^2 dA + A^2 conj(dA), the linearisation of |A|^2 A, with
        // dA = IDFT(M dphi); the tangent update has no noise and its own SETD2 history
        constexpr bool TAN = MODE == MODE_TAN;
        float2* dp = TAN ? a.dphi + (size_t)rr * N : nullptr;
        float2 draw[TAN ? E : 1], zd[TAN ? E : 1];
        if constexpr (TAN) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = t + T * e;
                draw[e] = dp[k];
                const bool inm = !a.dealias || 3 * abs(signed_idx(k, N)) < N;
                zd[e] = inm ? cscale(draw[e], a.scale) : czero();
            }
            fft_line<N, true>(zd, xb, t, tw);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const float2 A = z[e], dA = zd[e];
                zd[e] = cadd(cscale(dA, 2.f * (A.x * A.x + A.y * A.y)), cmul(cmul(A, A), cconj(dA)));
            }
            fft_line<N, false>(zd, xb, t, tw);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) z[e] = cscale(z[e], z[e].x * z[e].x + z[e].y * z[e].y);
        fft_line<N, false>(z, xb, t, tw);
        const long long step = current_step(a);
        const bool first = (a.scheme == 2) && (step == *a.first_step);
        float2* fp = a.fprev + (size_t)rr * N;
        float2* dfp = TAN ? a.dfprev + (size_t)rr * N : nullptr;
        const uint32_t rep = (uint32_t)(a.rep0 + rr);
        const float2 s = make_float2(a.s0, a.s0i);
        float2 zn0, zn1;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if ((e & 1) == 0) team_normal_pair_ks<T>(a.ks, 0, t, e, (uint32_t)step, rep, zn0, zn1);
            const int k = t + T * e;
            const int ks = signed_idx(k, N);
            const bool inm = !a.dealias || 3 * abs(ks) < N;
            const float2 F = inm ? cmul(s, z[e]) : czero();
            const Coefs co = load_coefs<true>(a.tab, abs(ks), first);
            const float2 Fp = (a.scheme == 2) ? fp[k] : czero();
            const float2 o = setd_update<true>(co, raw[e], F, Fp, eta_of((e & 1) ? zn1 : zn0, false));
            if (valid) {
                ph[k] = o;
                if (a.scheme == 2) fp[k] = F;
                flag_nonfinite(a, o, step);
            }
            if constexpr (TAN) {
                const float2 dF = inm ? cmul(s, zd[e]) : czero();
                const float2 dFp = (a.scheme == 2) ? dfp[k] : czero();
                const float2 d = setd_update<true>(co, draw[e], dF, dFp, czero());
                if (valid) {
                    dp[k] = d;
                    if (a.scheme == 2) dfp[k] = dF;
                }
            }
        }
    }
}

template <int M, int NL, int MODE>
static cudaError_t run_k1_real(const StepArgs& a, cudaStream_t s) {
    using C = LineCfg<M>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k1_real<M, NL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)C::smem());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k1_real<M, NL, MODE><<<(a.R + C::LINES - 1) / C::LINES, C::THREADS, C::smem(), s>>>(a);
    return cudaGetLastError();
}

template <int N, int MODE>
static cudaError_t run_k1_cplx(const StepArgs& a, cudaStream_t s) {
    using C = LineCfg<N>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(k1_cplx<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k1_cplx<N, MODE><<<(a.R + C::LINES - 1) / C::LINES, C::THREADS, C::smem(), s>>>(a);
    return cudaGetLastError();
}

template <int M>
static cudaError_t k1r_for(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    if (mode == MODE_FWD) return run_k1_real<M, NL_CUBIC, MODE_FWD>(a, s);
    if (mode == MODE_INV) return run_k1_real<M, NL_CUBIC, MODE_INV>(a, s);
    if (mode == MODE_STEP && nl == NL_CUBIC) return run_k1_real<M, NL_CUBIC, MODE_STEP>(a, s);
    if (mode == MODE_STEP && nl == NL_GRAD2) return run_k1_real<M, NL_GRAD2, MODE_STEP>(a, s);
    if (mode == MODE_TAN && nl == NL_CUBIC) return run_k1_real<M, NL_CUBIC, MODE_TAN>(a, s);
    if (mode == MODE_ADJ && nl == NL_CUBIC) return run_k1_real<M, NL_CUBIC, MODE_ADJ>(a, s);
    if (mode == MODE_TAN && nl == NL_GRAD2) return run_k1_real<M, NL_GRAD2, MODE_TAN>(a, s);
    if (mode == MODE_ADJ && nl == NL_GRAD2) return run_k1_real<M, NL_GRAD2, MODE_ADJ>(a, s);
    return cudaErrorInvalidValue;
}

template <int N>
static cudaError_t k1c_for(const StepArgs& a, int mode, cudaStream_t s) {
    if (mode == MODE_FWD) return run_k1_cplx<N, MODE_FWD>(a, s);
    if (mode == MODE_INV) return run_k1_cplx<N, MODE_INV>(a, s);
    if (mode == MODE_STEP) return run_k1_cplx<N, MODE_STEP>(a, s);
    if (mode == MODE_TAN) return run_k1_cplx<N, MODE_TAN>(a, s);
    if (mode == MODE_ADJ) return run_k1_cplx<N, MODE_ADJ>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace sft
