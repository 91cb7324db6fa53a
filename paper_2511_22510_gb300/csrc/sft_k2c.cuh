// sft_k2c.cuh -- two-pass 2-D step for complex fields (complex Ginzburg-Landau):
// the row and column kernels (instantiated in sft_k2c.cu and sft_k2c_cols.cu).
//
// Layout (x-major): spectrum phi[a_x][a_y] over the full a_x in [0, nx).  The
// intermediates P, Q keep only the x-columns inside the dealiasing band, in
// compact order: column cx < m holds a_x = cx, column cx >= m holds
// a_x = cx + (nx - ncols) (the negative indices), with ncols = 2m - 1
// (ncols = nx without dealiasing).
//   row pass:    P --IFFT_x--> A(x, y) --(|A|^2 A)--> FFT_x --> Q
//   column pass: Q --FFT_y--> F = M s DFT[|A|^2 A], s = -(1 + i beta);
//                phi <- f1 phi + A F + B F_prev + g eta (complex coefficients,
//                complex noise on every mode); P <- IFFT_y(M phi / N^2)
#pragma once
#include "sft_async.cuh"
#include "sft_step_common.cuh"

namespace sft {

__device__ __forceinline__ bool cmask_x(int ax, int nx, int ncols) {
    const int m = (ncols + 1) / 2;
    return ax < m || ax >= nx - ncols / 2;
}
__device__ __forceinline__ int ccomp_x(int ax, int nx, int ncols) {
    const int m = (ncols + 1) / 2;
    return ax < m ? ax : ax - (nx - ncols);
}

// e^{-i pi s / N} for the signed index s, |s| <= N / 2, from tw_ps[m] = e^{-i pi m / N} (half-cell shift phase)
__device__ __forceinline__ float2 cps_phase_conj(const float2* __restrict__ tw_ps, int s) {
    const float2 w = __ldg(&tw_ps[abs(s)]);
    return s >= 0 ? w : cconj(w);
}

template <int N>
struct CRowCfg {
    using PL = FftPlan<N>;
    static constexpr int T = PL::T;
    static constexpr int ROWS = T >= 128 ? 4 : (T >= 32 ? 128 / T : 128 / T);
    static constexpr int THREADS = ROWS * T;
    static constexpr int TS = PL::BUF | 1;  // a row is also its team's exchange buffer
    static constexpr size_t smem() { return sizeof(float2) * (size_t)ROWS * TS; }
};

template <int N, int MODE>
__global__ void __launch_bounds__(CRowCfg<N>::THREADS) k2_rows_cplx(const StepArgs a) {
    using C = CRowCfg<N>;
    using PL = FftPlan<N>;
    constexpr int T = PL::T, E = PL::E, ROWS = C::ROWS, TS = C::TS;
    extern __shared__ float2 sm[];
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const int rep = blockIdx.y;
    const int ny = a.ny, hx = a.hx, ncols = a.ncols, nx = N;
    const int y0 = blockIdx.x * ROWS;
    const int y = y0 + team;
    const bool yok = y < ny;
    float2* trow = sm + team * TS;
    const float2* __restrict__ tw = a.tw_a;
    float2 z[E];
    if constexpr (MODE == MODE_TAN || MODE == MODE_ADJ) {
        // tangent: A = IDFT_x(P), dA = IDFT_x(dP); Q = DFT_x(|A|^2 A) and dQ = DFT_x(2 |A|^2 dA + A^2 conj(dA)),
        // the linearisation of |A|^2 A.  Tile 0: P (then Q), tile 1: dP (then dQ); each team row is also its
        // transform's exchange buffer.  Adjoint: the same map applied to W = IDFT(M conj(s) nu) (dP) is its own
        // transpose for the real inner product Re sum conj(u) v, and Q is not needed.
        constexpr bool TAN = MODE == MODE_TAN;
        float2* drow = sm + (ROWS + team) * TS;
        auto load = [&](const float2* src, float2* dst) {
            block_copy<C::THREADS, ROWS * N>(
                ROWS * ncols,
                [&](int f) {
                    const int c = f / ROWS, yy = f % ROWS;
                    return (y0 + yy < ny) ? src[((size_t)rep * hx + c) * ny + y0 + yy] : czero();
                },
                [&](int f, float2 v) { dst[(f % ROWS) * TS + f / ROWS] = v; });
        };
        load(a.pin, sm);
        load(a.dpin, sm + ROWS * TS);
        __syncthreads();
        float2 zd[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int ax = t + T * e;
            const bool in = cmask_x(ax, nx, ncols);
            z[e] = in ? trow[ccomp_x(ax, nx, ncols)] : czero();
            zd[e] = in ? drow[ccomp_x(ax, nx, ncols)] : czero();
        }
        fft_line<N, true>(z, trow, t, tw);
        fft_line<N, true>(zd, drow, t, tw);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float2 A = z[e], dA = zd[e];
            const float a2 = A.x * A.x + A.y * A.y;
            zd[e] = cadd(cscale(dA, 2.f * a2), cmul(cmul(A, A), cconj(dA)));
            z[e] = cscale(A, a2);
        }
        if constexpr (TAN) fft_line<N, false>(z, trow, t, tw);
        fft_line<N, false>(zd, drow, t, tw);
        team_sync<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int ax = t + T * e;
            if (cmask_x(ax, nx, ncols)) {
                if constexpr (TAN) trow[ccomp_x(ax, nx, ncols)] = z[e];
                drow[ccomp_x(ax, nx, ncols)] = zd[e];
            }
        }
        __syncthreads();
        auto store = [&](const float2* src, float2* dst) {
            block_copy<C::THREADS, ROWS * N>(
                ROWS * ncols, [&](int f) { return src[(f % ROWS) * TS + f / ROWS]; },
                [&](int f, float2 v) {
                    const int c = f / ROWS, yy = f % ROWS;
                    if (y0 + yy < ny) dst[((size_t)rep * hx + c) * ny + y0 + yy] = v;
                });
        };
        if constexpr (TAN) store(sm, a.qout);
        store(sm + ROWS * TS, a.dqout);
        return;
    }
    if constexpr (MODE == MODE_STEP_PS) {
        // phase-shift dealiasing along x (the alternative of Sec. IV step 1): |A|^2 A on the plain grid and on the
        // grid shifted by half a cell along x (input phases e^{i pi a_x / N}, output e^{-i pi a_x / N}, signed
        // a_x), averaged.  The block's rows are those of one copy of P (plain or shifted along y: blockIdx.y runs
        // over 2R copies); tile 1 holds a second copy of the rows for the shifted evaluation.  The compact columns
        // are every a_x but the Nyquist one.
        float2* srow = sm + (ROWS + team) * TS;
        auto load = [&](float2* dst) {
            block_copy<C::THREADS, ROWS * N>(
                ROWS * ncols,
                [&](int f) {
                    const int c = f / ROWS, yy = f % ROWS;
                    return (y0 + yy < ny) ? a.pin[((size_t)rep * hx + c) * ny + y0 + yy] : czero();
                },
                [&](int f, float2 v) { dst[(f % ROWS) * TS + f / ROWS] = v; });
        };
        load(sm);
        load(sm + ROWS * TS);
        __syncthreads();
        const float2* __restrict__ tps = a.tw_ps;
        auto eval = [&](float2* row, bool shift) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ax = t + T * e;
                float2 v = cmask_x(ax, nx, ncols) ? row[ccomp_x(ax, nx, ncols)] : czero();
                if (shift) v = cmul(v, cconj(cps_phase_conj(tps, signed_idx(ax, nx))));
                z[e] = v;
            }
            fft_line<N, true>(z, row, t, tw);
#pragma unroll
            for (int e = 0; e < E; ++e) z[e] = cscale(z[e], z[e].x * z[e].x + z[e].y * z[e].y);
            fft_line<N, false>(z, row, t, tw);
            team_sync<T>();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ax = t + T * e;
                if (cmask_x(ax, nx, ncols))
                    row[ccomp_x(ax, nx, ncols)] = shift ? cmul(z[e], cps_phase_conj(tps, signed_idx(ax, nx))) : z[e];
            }
        };
        eval(trow, false);
        eval(srow, true);
        // each thread reads back the entries it wrote itself
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int ax = t + T * e;
            if (cmask_x(ax, nx, ncols)) {
                const int cc = ccomp_x(ax, nx, ncols);
                trow[cc] = cscale(cadd(trow[cc], srow[cc]), 0.5f);
            }
        }
        __syncthreads();
        block_copy<C::THREADS, ROWS * N>(
            ROWS * ncols, [&](int f) { return sm[(f % ROWS) * TS + f / ROWS]; },
            [&](int f, float2 v) {
                const int c = f / ROWS, yy = f % ROWS;
                if (y0 + yy < ny) a.qout[((size_t)rep * hx + c) * ny + y0 + yy] = v;
            });
        return;
    }
    if constexpr (MODE == MODE_FWD) {
        const float2* src = a.cplx_io + ((size_t)rep * ny + (yok ? y : 0)) * N;
#pragma unroll
        for (int e = 0; e < E; ++e) z[e] = yok ? src[t + T * e] : czero();
    } else {
        block_copy<C::THREADS, ROWS * N>(
            ROWS * ncols,
            [&](int f) {
                const int c = f / ROWS, yy = f % ROWS;
                return (y0 + yy < ny) ? a.pin[((size_t)rep * hx + c) * ny + y0 + yy] : czero();
            },
            [&](int f, float2 v) { sm[(f % ROWS) * TS + f / ROWS] = v; });
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int ax = t + T * e;
            z[e] = cmask_x(ax, nx, ncols) ? trow[ccomp_x(ax, nx, ncols)] : czero();
        }
        fft_line<N, true>(z, trow, t, tw);
        if constexpr (MODE == MODE_INV) {
            if (yok) {
                float2* dst = a.cplx_io + ((size_t)rep * ny + y) * N;
#pragma unroll
                for (int e = 0; e < E; ++e) dst[t + T * e] = z[e];
            }
            return;
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) z[e] = cscale(z[e], z[e].x * z[e].x + z[e].y * z[e].y);
        }
    }
    if constexpr (MODE != MODE_INV) {
        fft_line<N, false>(z, trow, t, tw);
        team_sync<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int ax = t + T * e;
            if (cmask_x(ax, nx, ncols)) trow[ccomp_x(ax, nx, ncols)] = z[e];
        }
        __syncthreads();
        block_copy<C::THREADS, ROWS * N>(
            ROWS * ncols, [&](int f) { return sm[(f % ROWS) * TS + f / ROWS]; },
            [&](int f, float2 v) {
                const int c = f / ROWS, yy = f % ROWS;
                if (y0 + yy < ny) a.qout[((size_t)rep * hx + c) * ny + y0 + yy] = v;
            });
    }
}

// Replicas per column-pass block: the column's coefficient and twiddle reads
// then hit the caches for every replica after the first.
constexpr int kCRpb = 4;

template <int NY>
struct CColCfg {
    using PL = FftPlan<NY>;
    static constexpr int T = PL::T;
    static constexpr int COLS = T >= 128 ? 1 : 128 / T;
    static constexpr int THREADS = COLS * T;
    static constexpr int XB = PL::BUF;
    // the step stages each column's state and SETD2 history behind the exchange
    // buffers, at a 16-byte aligned offset
    static constexpr int SOFF = (COLS * XB + 1) / 2 * 2;
    static constexpr size_t smem() { return sizeof(float2) * (size_t)COLS * XB; }
    static constexpr size_t smem_step() { return sizeof(float2) * ((size_t)SOFF + 2 * (size_t)COLS * NY); }
};

template <int NY, int T>
__device__ __forceinline__ void stage_ccolumn(float2* dst, const float2* src, int t) {
#pragma unroll
    for (int i = t; i < NY / 2; i += T) cp_async_16_cg(dst + 2 * i, src + 2 * i);
}

template <int NY, int MODE>
__global__ void __launch_bounds__(CColCfg<NY>::THREADS, 512 / CColCfg<NY>::THREADS) k2_cols_cplx(const StepArgs a) {
    using C = CColCfg<NY>;
    using PL = FftPlan<NY>;
    constexpr int T = PL::T, E = PL::E, COLS = C::COLS, XB = C::XB;
    extern __shared__ float2 sm[];
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const int c = blockIdx.x * COLS + team;  // a_x
    const bool valid = c < a.hx;
    const int ax = valid ? c : a.hx - 1;
    const int nx = a.nx, ncols = a.ncols;
    float2* xb = sm + team * XB;
    const float2* __restrict__ tw = a.tw_a;
    // carried x-column: 2/3 truncation or phase shifts (every column but the Nyquist one) use the compact order
    const bool inx = (!a.dealias && !a.pshift) || cmask_x(ax, nx, ncols);
    const int axs = signed_idx(ax, nx);
    if (!valid && T >= 32) return;
    for (int ri = 0; ri < kCRpb; ++ri) {
        const int rep = blockIdx.y * kCRpb + ri;
        if (rep >= a.R) break;
        const size_t colbase = ((size_t)rep * a.hx + ax) * NY;
        const size_t cbase = ((size_t)rep * a.hx + (inx ? ccomp_x(ax, nx, ncols) : 0)) * NY;
        float2 v[E];
        if constexpr (MODE == MODE_FWD) {
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = a.qin[colbase + t + T * e];
            fft_line<NY, false>(v, xb, t, tw);
            if (valid) {
#pragma unroll
                for (int e = 0; e < E; ++e) a.phi[colbase + t + T * e] = v[e];
            }
        } else if constexpr (MODE == MODE_INV) {
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = cscale(a.phi[colbase + t + T * e], a.scale);
            fft_line<NY, true>(v, xb, t, tw);
            if (valid) {
#pragma unroll
                for (int e = 0; e < E; ++e) a.pout[colbase + t + T * e] = v[e];
            }
        } else {
            float2 out[E];
            if constexpr (MODE == MODE_STEP) {
                const long long step = current_step(a);
                const bool first = (a.scheme == 2) && (step == *a.first_step);
                const bool has_f = valid && inx;
                // the state column (and SETD2 history) streams into shared memory during the FFT of Q
                float2* sphi = sm + C::SOFF + team * NY;
                float2* sfp = sm + C::SOFF + (COLS + team) * NY;
                team_sync<T>();  // this team's reads of the staging rows (previous replica) are complete
                if (valid) {
                    stage_ccolumn<NY, T>(sphi, a.phi + colbase, t);
                    if (a.scheme == 2 && has_f) stage_ccolumn<NY, T>(sfp, a.fprev + colbase, t);
                }
                cp_async_commit();
                if (has_f || T < 32) {
#pragma unroll
                    for (int e = 0; e < E; ++e) v[e] = has_f ? a.qin[cbase + t + T * e] : czero();
                    fft_line<NY, false>(v, xb, t, tw);
                }
                cp_async_wait_all();
                team_sync<T>();
                const float2 s = make_float2(a.s0, a.s0i);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if ((e & 1) == 0)
                        team_normal_pair_ks<T>(a.ks, (uint64_t)ax * NY, t, e, (uint32_t)step, (uint32_t)(a.rep0 + rep),
                                            out[e], out[e + 1]);
                    const int ay = t + T * e;
                    const int ays = signed_idx(ay, NY);
                    const bool inm = has_f && (!a.dealias || 3 * abs(ays) < NY);
                    const float2 F = inm ? cmul(s, v[e]) : czero();
                    const Coefs co = load_coefs<true>(a.tab, abs(axs) * (NY / 2 + 1) + abs(ays), first);
                    float2 Fp = czero();
                    if (a.scheme == 2 && has_f) Fp = sfp[ay];
                    out[e] = setd_update<true>(co, sphi[ay], F, Fp, eta_of(out[e], false));
                    if (a.scheme == 2 && has_f && valid) a.fprev[colbase + ay] = F;
                }
                if (valid) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        a.phi[colbase + t + T * e] = out[e];
                        flag_nonfinite(a, out[e], step);
                    }
                }
            } else if constexpr (MODE == MODE_STEP_PS) {
                // phase-shift dealiasing: F = M s (Q0^ + e^{-i pi a_y / N} Q1^) / 2 from the row pass's plain (Q0)
                // and y-shifted (Q1) copies, each already averaged over its two x shifts; M keeps every mode off
                // the Nyquist lines; P0, P1 are emitted below
                const long long step = current_step(a);
                const bool first = (a.scheme == 2) && (step == *a.first_step);
                const bool has_f = valid && inx;
                float2 v1[E];
                if (has_f || T < 32) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        v[e] = has_f ? a.qin[cbase + t + T * e] : czero();
                        v1[e] = has_f ? a.qin[a.ps_off + cbase + t + T * e] : czero();
                    }
                    fft_line<NY, false>(v, xb, t, tw);
                    fft_line<NY, false>(v1, xb, t, tw);
                }
                const float2 s = make_float2(a.s0, a.s0i);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if ((e & 1) == 0)
                        team_normal_pair_ks<T>(a.ks, (uint64_t)ax * NY, t, e, (uint32_t)step, (uint32_t)(a.rep0 + rep),
                                               out[e], out[e + 1]);
                    const int ay = t + T * e;
                    const int ays = signed_idx(ay, NY);
                    const bool inm = has_f && 2 * abs(ays) != NY;
                    const float2 qa = cscale(cadd(v[e], cmul(v1[e], cps_phase_conj(a.tw_ps, ays))), 0.5f);
                    const float2 F = inm ? cmul(s, qa) : czero();
                    const Coefs co = load_coefs<true>(a.tab, abs(axs) * (NY / 2 + 1) + abs(ays), first);
                    const float2 Fp = (a.scheme == 2 && has_f) ? a.fprev[colbase + ay] : czero();
                    out[e] = setd_update<true>(co, a.phi[colbase + ay], F, Fp, eta_of(out[e], false));
                    if (a.scheme == 2 && has_f && valid) a.fprev[colbase + ay] = F;
                }
                if (valid) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        a.phi[colbase + t + T * e] = out[e];
                        flag_nonfinite(a, out[e], step);
                    }
                }
            } else if constexpr (MODE == MODE_TAN) {
                // the primal step (as MODE_STEP, without staging) and the tangent update of Eq. SETD1/SETD2
                // linearised: dphi <- f1 dphi + A M s DFT[dq] + B dF_prev, no noise; P and dP emitted below
                const long long step = current_step(a);
                const bool first = (a.scheme == 2) && (step == *a.first_step);
                const bool has_f = valid && inx;
                float2 dv[E];
                if (has_f || T < 32) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        v[e] = has_f ? a.qin[cbase + t + T * e] : czero();
                        dv[e] = has_f ? a.dqin[cbase + t + T * e] : czero();
                    }
                    fft_line<NY, false>(v, xb, t, tw);
                    fft_line<NY, false>(dv, xb, t, tw);
                }
                const float2 s = make_float2(a.s0, a.s0i);
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    if ((e & 1) == 0)
                        team_normal_pair_ks<T>(a.ks, (uint64_t)ax * NY, t, e, (uint32_t)step, (uint32_t)(a.rep0 + rep),
                                               out[e], out[e + 1]);
                    const int ay = t + T * e;
                    const int ays = signed_idx(ay, NY);
                    const bool inm = has_f && (!a.dealias || 3 * abs(ays) < NY);
                    const float2 F = inm ? cmul(s, v[e]) : czero();
                    const float2 dF = inm ? cmul(s, dv[e]) : czero();
                    const Coefs co = load_coefs<true>(a.tab, abs(axs) * (NY / 2 + 1) + abs(ays), first);
                    float2 Fp = czero(), dFp = czero();
                    if (a.scheme == 2 && has_f) {
                        Fp = a.fprev[colbase + ay];
                        dFp = a.dfprev[colbase + ay];
                    }
                    out[e] = setd_update<true>(co, a.phi[colbase + ay], F, Fp, eta_of(out[e], false));
                    dv[e] = setd_update<true>(co, a.dphi[colbase + ay], dF, dFp, czero());
                    if (a.scheme == 2 && has_f && valid) {
                        a.fprev[colbase + ay] = F;
                        a.dfprev[colbase + ay] = dF;
                    }
                }
                if (valid) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        a.phi[colbase + t + T * e] = out[e];
                        a.dphi[colbase + t + T * e] = dv[e];
                        flag_nonfinite(a, out[e], step);
                    }
                }
                // dP <- IFFT_y(M dphi / N^2)
                const bool has_dp = valid && inx;
                if (has_dp || T < 32) {
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int ay = t + T * e;
                        const bool inm = has_dp && (!a.dealias || 3 * abs(signed_idx(ay, NY)) < NY);
                        dv[e] = inm ? cscale(dv[e], a.scale) : czero();
                    }
                    fft_line<NY, true>(dv, xb, t, tw);
                    if (has_dp) {
#pragma unroll
                        for (int e = 0; e < E; ++e) a.dpout[cbase + t + T * e] = dv[e];
                    }
                }
            } else if constexpr (MODE == MODE_ADJ || MODE == MODE_ADJ_PRIME) {
                // adjoint of step n for the real inner product Re sum conj(u) v (multipliers conjugated):
                // lam_n = conj(f1) lam_{n+1} + M DFT_y[dQ] (dQ from the row pass), mu_{n-1} = conj(B_n) lam_{n+1}
                // (SETD2), then W = IDFT_y(M conj(s) (conj(A_{n-1}) lam_n + mu_{n-1}) / N^2) for step n - 1.
                // ADJ_PRIME: W from lam_N alone (mu = 0).
                const bool has_f = valid && inx;
                float2 lam[E], mu[E];
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    lam[e] = a.dphi[colbase + t + T * e];
                    mu[e] = czero();
                }
                if constexpr (MODE == MODE_ADJ) {
                    if (has_f || T < 32) {
#pragma unroll
                        for (int e = 0; e < E; ++e) v[e] = has_f ? a.dqin[cbase + t + T * e] : czero();
                        fft_line<NY, false>(v, xb, t, tw);
                    }
                    const bool fa = a.adj_first_n != 0;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int ays = signed_idx(t + T * e, NY);
                        const bool inm = has_f && (!a.dealias || 3 * abs(ays) < NY);
                        const Coefs co = load_coefs<true>(a.tab, abs(axs) * (NY / 2 + 1) + abs(ays), fa);
                        if (a.scheme == 2 && !fa) mu[e] = cmul(cconj(co.B), lam[e]);
                        lam[e] = cadd(cmul(cconj(co.f1), lam[e]), inm ? v[e] : czero());
                    }
                    if (valid) {
#pragma unroll
                        for (int e = 0; e < E; ++e) a.dphi[colbase + t + T * e] = lam[e];
                    }
                }
                const bool has_p = valid && inx;
                if (has_p || T < 32) {
                    const float2 sw = make_float2(a.s0 * a.scale, -a.s0i * a.scale);  // conj(s) / N^2
                    const bool fp = a.adj_first_prev != 0;
#pragma unroll
                    for (int e = 0; e < E; ++e) {
                        const int ays = signed_idx(t + T * e, NY);
                        const bool inm = has_p && (!a.dealias || 3 * abs(ays) < NY);
                        const Coefs co = load_coefs<true>(a.tab, abs(axs) * (NY / 2 + 1) + abs(ays), fp);
                        const float2 nu = cadd(cmul(cconj(co.A), lam[e]), mu[e]);
                        v[e] = inm ? cmul(sw, nu) : czero();
                    }
                    fft_line<NY, true>(v, xb, t, tw);
                    if (has_p) {
#pragma unroll
                        for (int e = 0; e < E; ++e) a.dpout[cbase + t + T * e] = v[e];
                    }
                }
                continue;
            } else {  // MODE_PRIME
#pragma unroll
                for (int e = 0; e < E; ++e) out[e] = a.phi[colbase + t + T * e];
            }
            const bool has_p = valid && inx;
            if (a.pshift) {
                // phase shifts: P0 <- IFFT_y(M phi / N^2), P1 <- IFFT_y(M phi e^{i pi a_y / N} / N^2) at ps_off
                if (has_p || T < 32) {
#pragma unroll
                    for (int cp = 0; cp < 2; ++cp) {
#pragma unroll
                        for (int e = 0; e < E; ++e) {
                            const int ays = signed_idx(t + T * e, NY);
                            const bool inm = has_p && 2 * abs(ays) != NY;
                            float2 x = cscale(out[e], a.scale);
                            if (cp) x = cmul(x, cconj(cps_phase_conj(a.tw_ps, ays)));
                            v[e] = inm ? x : czero();
                        }
                        fft_line<NY, true>(v, xb, t, tw);
                        if (has_p) {
#pragma unroll
                            for (int e = 0; e < E; ++e) a.pout[cp * a.ps_off + cbase + t + T * e] = v[e];
                        }
                    }
                }
            } else if (has_p || T < 32) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int ay = t + T * e;
                    const bool inm = has_p && (!a.dealias || 3 * abs(signed_idx(ay, NY)) < NY);
                    v[e] = inm ? cscale(out[e], a.scale) : czero();
                }
                fft_line<NY, true>(v, xb, t, tw);
                if (has_p) {
#pragma unroll
                    for (int e = 0; e < E; ++e) a.pout[cbase + t + T * e] = v[e];
                }
            }
        }
    }
}

template <int N, int MODE>
static cudaError_t run_crows(const StepArgs& a, cudaStream_t s) {
    using C = CRowCfg<N>;
    const size_t sm = (MODE == MODE_TAN || MODE == MODE_ADJ || MODE == MODE_STEP_PS ? 2 : 1) * C::smem();
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(k2_rows_cplx<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k2_rows_cplx<N, MODE><<<dim3((a.ny + C::ROWS - 1) / C::ROWS, a.R), C::THREADS, sm, s>>>(a);
    return cudaGetLastError();
}

template <int NY, int MODE>
static cudaError_t run_ccols(const StepArgs& a, cudaStream_t s) {
    using C = CColCfg<NY>;
    const size_t sm = MODE == MODE_STEP ? C::smem_step() : C::smem();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k2_cols_cplx<NY, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k2_cols_cplx<NY, MODE><<<dim3((a.hx + C::COLS - 1) / C::COLS, (a.R + kCRpb - 1) / kCRpb), C::THREADS, sm, s>>>(a);
    return cudaGetLastError();
}

template <int N>
static cudaError_t crows_for(const StepArgs& a, int mode, cudaStream_t s) {
    switch (mode) {
        case MODE_STEP: return run_crows<N, MODE_STEP>(a, s);
        case MODE_FWD: return run_crows<N, MODE_FWD>(a, s);
        case MODE_INV: return run_crows<N, MODE_INV>(a, s);
        case MODE_TAN: return run_crows<N, MODE_TAN>(a, s);
        case MODE_ADJ: return run_crows<N, MODE_ADJ>(a, s);
        case MODE_STEP_PS: return run_crows<N, MODE_STEP_PS>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int NY>
static cudaError_t ccols_for(const StepArgs& a, int mode, cudaStream_t s) {
    switch (mode) {
        case MODE_STEP: return run_ccols<NY, MODE_STEP>(a, s);
        case MODE_FWD: return run_ccols<NY, MODE_FWD>(a, s);
        case MODE_INV: return run_ccols<NY, MODE_INV>(a, s);
        case MODE_PRIME: return run_ccols<NY, MODE_PRIME>(a, s);
        case MODE_TAN: return run_ccols<NY, MODE_TAN>(a, s);
        case MODE_ADJ: return run_ccols<NY, MODE_ADJ>(a, s);
        case MODE_ADJ_PRIME: return run_ccols<NY, MODE_ADJ_PRIME>(a, s);
        case MODE_STEP_PS: return run_ccols<NY, MODE_STEP_PS>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
