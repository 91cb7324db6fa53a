// sft_k2d.cu -- two-pass 2-D step for real fields (Model A/B, KPZ).
//
// Layout (x-major, per replica): spectrum phi[a_x][a_y], a_x in [0, nx/2],
// a_y in [0, ny); intermediates P, Q with the same layout restricted to the
// x-columns inside the dealiasing band.  One step (Sec. IV boxed algorithm):
//
//   row pass    (k2_rows): P[a_x][y] --C2R along x--> psi(x, y) --q(psi)-->
//                          q(x, y) --R2C along x--> Q[a_x][y]
//   column pass (k2_cols): Q --FFT along y--> DFT[q]; F = M s DFT[q];
//                          phi <- f1 phi + A F + B F_prev + g eta (Philox);
//                          Hermitian fix-up; P <- IFFT_y(M phi / N^2)
//
// so every step moves the state once through HBM plus two dealiased
// intermediates.  Real-length-N transforms use the N/2-point complex FFT with
// the even/odd split (z[m] = x[2m] + i x[2m+1]).
#include "sft_async.cuh"
#include "sft_step_common.cuh"

// Launch shape of the row pass: SFT_ROW_CTA threads per block (16 values per
// thread), SFT_ROW_MINB resident blocks per SM requested from the register
// allocator.
#ifndef SFT_ROW_CTA
#define SFT_ROW_CTA 128
#endif
#ifndef SFT_ROW_MINB
#define SFT_ROW_MINB 4
#endif
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
#define SFT_RPB 4  // replicas per column-pass block: the column's table and twiddle reads then hit L1
#endif

namespace sft {

// R2C post-processing of one row held by a team (z = FFT_M of the packed real
// line) into the spectral row trow[0..ncols); xb is the team's exchange buffer
// (it may alias trow).
template <int M>
__device__ __forceinline__ void row_post(float2 (&z)[FftPlan<M>::E], float2* xb, float2* trow, int ncols, int t,
                                         const float2* __restrict__ twN) {
    using PL = FftPlan<M>;
    constexpr int T = PL::T, E = PL::E;
    team_sync<T>();
#pragma unroll
    for (int e = 0; e < E; ++e) xb[xpos<M>(t + T * e)] = z[e];
    team_sync<T>();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + T * e;
        z[e] = r2c_post(z[e], cconj(xb[xpos<M>((M - k) & (M - 1))]), __ldg(&twN[k]));
    }
    const float2 z0 = xb[0];
    team_sync<T>();
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + T * e;
        if (k < ncols) trow[k] = z[e];
    }
    if (t == 0 && M < ncols) trow[M] = make_float2(z0.x - z0.y, 0.f);
}

template <int M_>
struct RowCfg {
    static constexpr int M = M_;
    using PL = FftPlan<M>;
    static constexpr int T = PL::T;
    static constexpr int ROWS = T >= SFT_ROW_CTA ? 1 : SFT_ROW_CTA / T;
    static constexpr int THREADS = ROWS * T;
    // row stride of the spectral tile (a row also serves as its team's FFT exchange buffer):
    // the transposing tile loads/stores of a half-warp touch ROWS rows x 16/ROWS columns, which
    // fall on distinct banks when TS = 16/ROWS (mod 16); an odd stride when ROWS >= 16
    static constexpr int TSM = ROWS >= 16 ? 1 : 16 / ROWS;
    static constexpr int TS = ROWS >= 16 ? (PL::BUF | 1) : ((PL::BUF + 15) / 16) * 16 + TSM;
    static constexpr size_t smem(int ntile) { return sizeof(float2) * (size_t)ntile * ROWS * TS; }
};

// Spectral tile of a row-pass block: tile[yy][c] = src[rowbase + c ny + y0 + yy]
// for the ROWS rows y0 + yy and the columns c < ncols; columns ncols..M are
// zero (outside the dealiasing band).
template <class C>
__device__ __forceinline__ void load_tile(float2* tile, const float2* __restrict__ src, size_t rowbase, int ncols,
                                          int ny, int y0) {
    constexpr int ROWS = C::ROWS, TS = C::TS, NEL = C::ROWS * (C::M + 1);
    block_copy<C::THREADS, NEL>(
        NEL,
        [&](int f) {
            const int c = f / ROWS, yy = f % ROWS;
            return (c < ncols && y0 + yy < ny) ? src[rowbase + (size_t)c * ny + y0 + yy] : czero();
        },
        [&](int f, float2 v) { tile[(f % ROWS) * TS + f / ROWS] = v; });
}

// dst[rowbase + c ny + y0 + yy] = tile[yy][c] for c < ncols
template <class C>
__device__ __forceinline__ void store_tile(const float2* tile, float2* __restrict__ dst, size_t rowbase, int ncols,
                                           int ny, int y0) {
    constexpr int ROWS = C::ROWS, TS = C::TS;
    block_copy<C::THREADS, C::ROWS * (C::M + 1)>(
        ROWS * ncols, [&](int f) { return tile[(f % ROWS) * TS + f / ROWS]; },
        [&](int f, float2 v) {
            const int c = f / ROWS, yy = f % ROWS;
            if (y0 + yy < ny) dst[rowbase + (size_t)c * ny + y0 + yy] = v;
        });
}

template <int M, int NL, int MODE>
__global__ void __launch_bounds__(RowCfg<M>::THREADS, SFT_ROW_MINB) k2_rows_real(const StepArgs a) {
    using C = RowCfg<M>;
    using PL = FftPlan<M>;
    constexpr int T = PL::T, E = PL::E, ROWS = C::ROWS, TS = C::TS;
    constexpr bool GRAD = (NL == NL_GRAD2) && (MODE == MODE_STEP);
    static_assert(!((MODE == MODE_TAN || MODE == MODE_ADJ) && NL != NL_CUBIC), "tangent/adjoint: cubic term");
    extern __shared__ float2 sm[];
    float2* tile = sm;
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    const int rep = blockIdx.y;
    const int ny = a.ny, hx = a.hx, ncols = a.ncols;
    const int y0 = blockIdx.x * ROWS;
    const int y = y0 + team;
    const bool yok = y < ny;
    const size_t rowbase = (size_t)rep * hx * ny;
    float2* xb = tile + team * TS;  // the team's own tile row doubles as its exchange buffer
    const float2* __restrict__ twM = a.tw_a;
    const float2* __restrict__ twN = a.tw_b;
    float2 z[E];

    if constexpr (MODE == MODE_TAN || MODE == MODE_ADJ) {
        // tangent: q' = 3 psi^2 dpsi next to q = psi^3; adjoint: v = 3 psi^2 w.
        // tile 0: primal P (psi), tile 1: tangent dP (dpsi) or adjoint W.
        load_tile<C>(tile, a.pin, rowbase, ncols, ny, y0);
        load_tile<C>(tile + ROWS * TS, a.dpin, rowbase, ncols, ny, y0);
        __syncthreads();
        const float2* trow = tile + team * TS;
        float2* drow = tile + ROWS * TS + team * TS;
        float2 zd[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            const float2 tw = __ldg(&twN[k]);
            z[e] = c2r_pre(trow[k], trow[M - k], tw);
            zd[e] = c2r_pre(drow[k], drow[M - k], tw);
        }
        fft_line<M, true>(z, xb, t, twM);
        fft_line<M, true>(zd, xb, t, twM);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const float2 p = z[e];
            zd[e] = make_float2(3.f * p.x * p.x * zd[e].x, 3.f * p.y * p.y * zd[e].y);
            if constexpr (MODE == MODE_TAN) z[e] = make_float2(p.x * p.x * p.x, p.y * p.y * p.y);
        }
        fft_line<M, false>(zd, xb, t, twM);
        // second output first: its post-processing uses tile row 0 as the exchange buffer
        row_post<M>(zd, xb, drow, ncols, t, twN);
        if constexpr (MODE == MODE_TAN) {
            fft_line<M, false>(z, xb, t, twM);
            row_post<M>(z, xb, tile + team * TS, ncols, t, twN);
        }
        __syncthreads();
        store_tile<C>(tile + ROWS * TS, a.dqout, rowbase, ncols, ny, y0);
        if constexpr (MODE == MODE_TAN) store_tile<C>(tile, a.qout, rowbase, ncols, ny, y0);
        return;
    }
    if constexpr (MODE == MODE_FWD) {
        const float* src = a.real_io + ((size_t)rep * ny + (yok ? y : 0)) * (2 * M);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int m = t + T * e;
            z[e] = yok ? *reinterpret_cast<const float2*>(src + 2 * m) : czero();
        }
    } else {
        load_tile<C>(tile, a.pin, rowbase, ncols, ny, y0);
        if constexpr (GRAD) load_tile<C>(tile + ROWS * TS, a.pyin, rowbase, ncols, ny, y0);
        __syncthreads();
        const float2* trow = tile + team * TS;
        if constexpr (GRAD) {
            // grad_x h from i k_x P (k_x = 0 at the Nyquist column), grad_y h from P_y
            const float2* tyrow = tile + ROWS * TS + team * TS;
            float2 zy[E];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = t + T * e;
                const float2 tw = __ldg(&twN[k]);
                const float kx = a.dk * (float)k, kxm = (k == 0) ? 0.f : a.dk * (float)(M - k);
                const float2 X = cscale(cmuli(trow[k]), kx), Xm = cscale(cmuli(trow[M - k]), kxm);
                z[e] = c2r_pre(X, Xm, tw);
                zy[e] = c2r_pre(tyrow[k], tyrow[M - k], tw);
            }
            fft_line<M, true>(z, xb, t, twM);
            fft_line<M, true>(zy, xb, t, twM);
#pragma unroll
            for (int e = 0; e < E; ++e)
                z[e] = make_float2(z[e].x * z[e].x + zy[e].x * zy[e].x, z[e].y * z[e].y + zy[e].y * zy[e].y);
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = t + T * e;
                z[e] = c2r_pre(trow[k], trow[M - k], __ldg(&twN[k]));
            }
            fft_line<M, true>(z, xb, t, twM);
            if constexpr (MODE == MODE_INV) {
                if (yok) {
                    float* dst = a.real_io + ((size_t)rep * ny + y) * (2 * M);
#pragma unroll
                    for (int e = 0; e < E; ++e) *reinterpret_cast<float2*>(dst + 2 * (t + T * e)) = z[e];
                }
                return;
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) z[e] = make_float2(z[e].x * z[e].x * z[e].x, z[e].y * z[e].y * z[e].y);
            }
        }
    }
    if constexpr (MODE != MODE_INV) {
        fft_line<M, false>(z, xb, t, twM);
        team_sync<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) xb[xpos<M>(t + T * e)] = z[e];
        team_sync<T>();
        float2* trow = tile + team * TS;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            z[e] = r2c_post(z[e], cconj(xb[xpos<M>((M - k) & (M - 1))]), __ldg(&twN[k]));
        }
        const float2 z0 = xb[0];
        team_sync<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            if (k < ncols) trow[k] = z[e];
        }
        if (t == 0 && M < ncols) trow[M] = make_float2(z0.x - z0.y, 0.f);
        __syncthreads();
        store_tile<C>(tile, a.qout, rowbase, ncols, ny, y0);
    }
}

constexpr int kColEM = SFT_COL_EMAX;

template <int NY>
struct ColCfg {
    static constexpr bool WIDE = NY >= 512;
    using PL = FftPlan<NY, kColEM>;
    static constexpr int T = PL::T;
    static constexpr int CTA = WIDE ? SFT_COL_CTA : 128;
    static constexpr int COLS = T >= CTA ? 1 : CTA / T;
    static constexpr int THREADS = COLS * T;
    static constexpr int PER_SM = WIDE ? SFT_COL_THREADS_SM : 512;
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
template <int NY>
__device__ __forceinline__ void fixup_plane(float2 (&out)[FftPlan<NY, kColEM>::E], float2* xb, int t, bool plane) {
    using PL = FftPlan<NY, kColEM>;
    constexpr int T = PL::T, E = PL::E;
    if (plane || T < 32) {
        team_sync<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) xb[xpos<NY, kColEM>(t + T * e)] = out[e];
        team_sync<T>();
        if (plane) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ay = t + T * e;
                if (2 * ay > NY) out[e] = cconj(xb[xpos<NY, kColEM>(NY - ay)]);
                if (ay == 0 || 2 * ay == NY) out[e].y = 0.f;
            }
        }
    }
}

// P <- IFFT_y(M phi / N^2) for one column (and, for KPZ, P_y <- IFFT_y(i k_y M phi / N^2)):
// the dealiased input of the next row pass.
template <int NY, int NL>
__device__ __forceinline__ void emit_p(const StepArgs& a, const float2 (&out)[FftPlan<NY, kColEM>::E], bool has_p, int cc,
                                       size_t colbase, float2* xb, int t) {
    using PL = FftPlan<NY, kColEM>;
    constexpr int T = PL::T, E = PL::E;
    if (!(has_p || T < 32)) return;
    float2 v[E];
    float2 vy[NL == NL_GRAD2 ? E : 1];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int ay = t + T * e;
        const int ays = signed_idx(ay, NY);
        const bool inm = !a.dealias || (3 * cc < a.nx && 3 * abs(ays) < NY);
        v[e] = (has_p && inm) ? cscale(out[e], a.scale) : czero();
        if constexpr (NL == NL_GRAD2) vy[e] = cscale(cmuli(v[e]), a.dk * (float)odd_idx(ay, NY));
    }
    fft_line<NY, true, kColEM>(v, xb, t, a.tw_a);
    if constexpr (NL == NL_GRAD2) fft_line<NY, true, kColEM>(vy, xb, t, a.tw_a);
    if (has_p) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            a.pout[colbase + t + T * e] = v[e];
            if constexpr (NL == NL_GRAD2) a.pyout[colbase + t + T * e] = vy[e];
        }
    }
}

template <int NY, int NL, int MODE>
__global__ void __launch_bounds__(ColCfg<NY>::THREADS, ColCfg<NY>::MINB) k2_cols_real(const StepArgs a) {
    using C = ColCfg<NY>;
    using PL = FftPlan<NY, kColEM>;
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
    for (int ri = 0; ri < SFT_RPB; ++ri) {
    const int rep = blockIdx.y * SFT_RPB + ri;
    if (rep >= a.R) break;
    const size_t colbase = ((size_t)rep * a.hx + cc) * NY;
    float2 v[E];

    if constexpr (MODE == MODE_FWD) {
        if (!valid && T >= 32) return;
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = a.qin[colbase + t + T * e];
        fft_line<NY, false, kColEM>(v, xb, t, tw);
        team_sync<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) xb[xpos<NY, kColEM>(t + T * e)] = v[e];
        team_sync<T>();
        if (plane) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ay = t + T * e;
                if (2 * ay > NY) v[e] = cconj(xb[xpos<NY, kColEM>(NY - ay)]);
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
        fft_line<NY, true, kColEM>(v, xb, t, tw);
        if (valid) {
#pragma unroll
            for (int e = 0; e < E; ++e) a.pout[colbase + t + T * e] = v[e];
        }
    } else if constexpr (MODE == MODE_STEP) {
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
            fft_line<NY, false, kColEM>(v, xb, t, tw);
        }
        cp_async_wait_all();
        team_sync<T>();
        float2 out[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if ((e & 1) == 0)
                team_normal_pair<T>(a.seed, (uint64_t)cc * NY, t, e, (uint32_t)step, (uint32_t)(a.rep0 + rep), out[e],
                                    out[e + 1]);
            const int ay = t + T * e;
            const int ays = signed_idx(ay, NY);
            const int q = cc * cc + ays * ays;
            const bool inm = !a.dealias || (3 * cc < a.nx && 3 * abs(ays) < NY);
            float2 F = czero();
            if (has_f && inm) F = cscale(v[e], nl_prefactor(a, q).x);
            const Coefs co = load_coefs<false>(a.tab, cc * (NY / 2 + 1) + abs(ays), first);
            const float2 ph = sphi[ay];
            float2 Fp = czero();
            if (a.scheme == 2 && has_f) Fp = sfp[ay];
            const bool selfc = plane && (ay == 0 || 2 * ay == NY);
            // partners on the self-conjugate planes are overwritten by the fix-up below
            out[e] = setd_update<false>(co, ph, F, Fp, eta_of(out[e], selfc));
            if (a.scheme == 2 && has_f && valid) a.fprev[colbase + ay] = F;
        }
        if (plane || T < 32) {
            team_sync<T>();
#pragma unroll
            for (int e = 0; e < E; ++e) xb[xpos<NY, kColEM>(t + T * e)] = out[e];
            team_sync<T>();
            if (plane) {
#pragma unroll
                for (int e = 0; e < E; ++e) {
                    const int ay = t + T * e;
                    if (2 * ay > NY) out[e] = cconj(xb[xpos<NY, kColEM>(NY - ay)]);
                    if (ay == 0 || 2 * ay == NY) out[e].y = 0.f;
                }
            }
        }
        if (valid) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                a.phi[colbase + t + T * e] = out[e];
                flag_nonfinite(a, out[e], step);
            }
        }
        emit_p<NY, NL>(a, out, valid && cc < a.ncols, cc, colbase, xb, t);
    } else if constexpr (MODE == MODE_TAN) {
        // primal step as in MODE_STEP, plus the tangent dphi <- f1 dphi + A M s DFT[q'] (no noise)
        if (!valid && T >= 32) return;
        const long long step = current_step(a);
        const bool has_f = valid && cc < a.ncols;
        float2 dv[E];
        if (has_f || T < 32) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                v[e] = has_f ? a.qin[colbase + t + T * e] : czero();
                dv[e] = has_f ? a.dqin[colbase + t + T * e] : czero();
            }
            fft_line<NY, false, kColEM>(v, xb, t, tw);
            fft_line<NY, false, kColEM>(dv, xb, t, tw);
        }
        float2 out[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if ((e & 1) == 0)
                team_normal_pair<T>(a.seed, (uint64_t)cc * NY, t, e, (uint32_t)step, (uint32_t)(a.rep0 + rep), out[e],
                                    out[e + 1]);
            const int ay = t + T * e;
            const int ays = signed_idx(ay, NY);
            const int q = cc * cc + ays * ays;
            const bool inm = !a.dealias || (3 * cc < a.nx && 3 * abs(ays) < NY);
            const float sq = nl_prefactor(a, q).x;
            const float2 F = (has_f && inm) ? cscale(v[e], sq) : czero();
            const float2 dF = (has_f && inm) ? cscale(dv[e], sq) : czero();
            const Coefs co = load_coefs<false>(a.tab, cc * (NY / 2 + 1) + abs(ays), false);
            const bool selfc = plane && (ay == 0 || 2 * ay == NY);
            out[e] = setd_update<false>(co, a.phi[colbase + ay], F, czero(), eta_of(out[e], selfc));
            dv[e] = setd_update<false>(co, a.dphi[colbase + ay], dF, czero(), czero());
        }
        fixup_plane<NY>(out, xb, t, plane);
        fixup_plane<NY>(dv, xb, t, plane);
        if (valid) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                a.phi[colbase + t + T * e] = out[e];
                a.dphi[colbase + t + T * e] = dv[e];
                flag_nonfinite(a, out[e], step);
            }
        }
        emit_p<NY, NL>(a, out, valid && cc < a.ncols, cc, colbase, xb, t);
        StepArgs b = a;
        b.pout = a.dpout;
        emit_p<NY, NL>(b, dv, valid && cc < a.ncols, cc, colbase, xb, t);
    } else if constexpr (MODE == MODE_ADJ || MODE == MODE_ADJ_PRIME) {
        // adjoint: lam <- f1 lam + M DFT[v] (v from the row pass), then W = IDFT_y(A s M lam / N^2)
        if (!valid && T >= 32) return;
        const bool has_f = valid && cc < a.ncols;
        float2 lam[E];
#pragma unroll
        for (int e = 0; e < E; ++e) lam[e] = a.dphi[colbase + t + T * e];
        if constexpr (MODE == MODE_ADJ) {
            if (has_f || T < 32) {
#pragma unroll
                for (int e = 0; e < E; ++e) v[e] = has_f ? a.dqin[colbase + t + T * e] : czero();
                fft_line<NY, false, kColEM>(v, xb, t, tw);
            }
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ay = t + T * e;
                const int ays = signed_idx(ay, NY);
                const bool inm = !a.dealias || (3 * cc < a.nx && 3 * abs(ays) < NY);
                const float f1 = __ldg(&a.tab[cc * (NY / 2 + 1) + abs(ays)]).x;
                const float2 dv = (has_f && inm) ? v[e] : czero();
                lam[e] = make_float2(f1 * lam[e].x + dv.x, f1 * lam[e].y + dv.y);
            }
            fixup_plane<NY>(lam, xb, t, plane);
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
                const Coefs co = load_coefs<false>(a.tab, cc * (NY / 2 + 1) + abs(ays), false);
                v[e] = (has_p && inm) ? cscale(lam[e], co.A.x * nl_prefactor(a, q).x * a.scale) : czero();
            }
            fft_line<NY, true, kColEM>(v, xb, t, tw);
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
        emit_p<NY, NL>(a, out, has_p, cc, colbase, xb, t);
    }
    }  // replicas
}

// ----------------------------------------------------------------- launchers
template <int M, int NL, int MODE>
static cudaError_t run_rows(const StepArgs& a, cudaStream_t s) {
    using C = RowCfg<M>;
    constexpr int NTILE = ((NL == NL_GRAD2 && MODE == MODE_STEP) || MODE == MODE_TAN || MODE == MODE_ADJ) ? 2 : 1;
    const size_t sm = C::smem(NTILE);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k2_rows_real<M, NL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((a.ny + C::ROWS - 1) / C::ROWS, a.R);
    k2_rows_real<M, NL, MODE><<<grid, C::THREADS, sm, s>>>(a);
    return cudaGetLastError();
}

template <int NY, int NL, int MODE>
static cudaError_t run_cols(const StepArgs& a, cudaStream_t s) {
    using C = ColCfg<NY>;
    const size_t sm = MODE == MODE_STEP ? C::smem_step() : C::smem();
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k2_cols_real<NY, NL, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((a.hx + C::COLS - 1) / C::COLS, (a.R + SFT_RPB - 1) / SFT_RPB);
    k2_cols_real<NY, NL, MODE><<<grid, C::THREADS, sm, s>>>(a);
    return cudaGetLastError();
}

template <int M>
static cudaError_t rows_for(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    if (mode == MODE_FWD) return run_rows<M, NL_CUBIC, MODE_FWD>(a, s);
    if (mode == MODE_INV) return run_rows<M, NL_CUBIC, MODE_INV>(a, s);
    if (mode == MODE_STEP && nl == NL_CUBIC) return run_rows<M, NL_CUBIC, MODE_STEP>(a, s);
    if (mode == MODE_STEP && nl == NL_GRAD2) return run_rows<M, NL_GRAD2, MODE_STEP>(a, s);
    if (mode == MODE_TAN && nl == NL_CUBIC) return run_rows<M, NL_CUBIC, MODE_TAN>(a, s);
    if (mode == MODE_ADJ && nl == NL_CUBIC) return run_rows<M, NL_CUBIC, MODE_ADJ>(a, s);
    return cudaErrorInvalidValue;
}

template <int NY>
static cudaError_t cols_for(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    if (mode == MODE_FWD) return run_cols<NY, NL_CUBIC, MODE_FWD>(a, s);
    if (mode == MODE_INV) return run_cols<NY, NL_CUBIC, MODE_INV>(a, s);
    if (mode == MODE_STEP && nl == NL_CUBIC) return run_cols<NY, NL_CUBIC, MODE_STEP>(a, s);
    if (mode == MODE_STEP && nl == NL_GRAD2) return run_cols<NY, NL_GRAD2, MODE_STEP>(a, s);
    if (mode == MODE_PRIME && nl == NL_CUBIC) return run_cols<NY, NL_CUBIC, MODE_PRIME>(a, s);
    if (mode == MODE_PRIME && nl == NL_GRAD2) return run_cols<NY, NL_GRAD2, MODE_PRIME>(a, s);
    if (mode == MODE_TAN && nl == NL_CUBIC) return run_cols<NY, NL_CUBIC, MODE_TAN>(a, s);
    if (mode == MODE_ADJ && nl == NL_CUBIC) return run_cols<NY, NL_CUBIC, MODE_ADJ>(a, s);
    if (mode == MODE_ADJ_PRIME && nl == NL_CUBIC) return run_cols<NY, NL_CUBIC, MODE_ADJ_PRIME>(a, s);
    return cudaErrorInvalidValue;
}

bool k2_supported(int nx, int ny, int complex_field) {
    if (complex_field) return false;
    auto ok = [](int n) { return n >= 16 && n <= 4096 && (n & (n - 1)) == 0; };
    return ok(nx) && ok(ny);
}

cudaError_t launch_k2_rows(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    switch (a.nx / 2) {
        case 8: return rows_for<8>(a, mode, nl, s);
        case 16: return rows_for<16>(a, mode, nl, s);
        case 32: return rows_for<32>(a, mode, nl, s);
        case 64: return rows_for<64>(a, mode, nl, s);
        case 128: return rows_for<128>(a, mode, nl, s);
        case 256: return rows_for<256>(a, mode, nl, s);
        case 512: return rows_for<512>(a, mode, nl, s);
        case 1024: return rows_for<1024>(a, mode, nl, s);
        case 2048: return rows_for<2048>(a, mode, nl, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_k2_cols(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    switch (a.ny) {
        case 16: return cols_for<16>(a, mode, nl, s);
        case 32: return cols_for<32>(a, mode, nl, s);
        case 64: return cols_for<64>(a, mode, nl, s);
        case 128: return cols_for<128>(a, mode, nl, s);
        case 256: return cols_for<256>(a, mode, nl, s);
        case 512: return cols_for<512>(a, mode, nl, s);
        case 1024: return cols_for<1024>(a, mode, nl, s);
        case 2048: return cols_for<2048>(a, mode, nl, s);
        case 4096: return cols_for<4096>(a, mode, nl, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
