// sft_k2d.cuh -- two-pass 2-D step for real fields (Model A/B, KPZ): row pass
// (kernel templates and launchers, instantiated by sft_k2d.cu for power-of-two
// rows and by sft_k2d_mixed.cu for p x 2^k rows; the column pass is in
// sft_k2d_cols.cuh).
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
#pragma once
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
namespace sft {

// Index of the mirrored entry (M - k) mod M of an M-point line.
template <int M>
__device__ __forceinline__ int mirror_idx(int k) {
    if constexpr ((M & (M - 1)) == 0)
        return (M - k) & (M - 1);
    else
        return k == 0 ? 0 : M - k;
}

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
        z[e] = r2c_post(z[e], cconj(xb[xpos<M>(mirror_idx<M>(k))]), __ldg(&twN[k]));
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

// Schedules of the row pass of the step, chosen per lattice by the plan
// autotuner: 0 = SFT_ROW_CTA threads per block at SFT_ROW_MINB blocks per SM;
// 1 = 256-thread blocks (twice the rows per tile) at 2 blocks per SM;
// 2 = 512-thread blocks at 1 per SM (16 rows per tile on 512-point rows: the
// transposing tile reads whole 128-byte segments of every column).
template <int SH>
struct RowShape {
    static constexpr int CTA = SFT_ROW_CTA, MINB = SFT_ROW_MINB;
};
template <>
struct RowShape<1> {
    static constexpr int CTA = 256, MINB = 2;
};
template <>
struct RowShape<2> {
    static constexpr int CTA = 512, MINB = 1;
};

template <int M_, int SH = 0>
struct RowCfg {
    static constexpr int M = M_;
    using PL = FftPlan<M>;
    static constexpr int T = PL::T;
    static constexpr int CTA = RowShape<SH>::CTA, MINB = RowShape<SH>::MINB;
    static constexpr int ROWS = T >= CTA ? 1 : CTA / T;
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

template <int M, int NL, int MODE, int SH = 0>
__global__ void __launch_bounds__(RowCfg<M, SH>::THREADS, RowCfg<M, SH>::MINB) k2_rows_real(const StepArgs a) {
    using C = RowCfg<M, SH>;
    using PL = FftPlan<M>;
    constexpr int T = PL::T, E = PL::E, ROWS = C::ROWS, TS = C::TS;
    constexpr bool GRAD = (NL == NL_GRAD2) && (MODE == MODE_STEP);
    static_assert(!(MODE == MODE_ADJ && NL != NL_CUBIC && NL != NL_GRAD2), "adjoint: cubic or KPZ term");
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

    if constexpr (MODE == MODE_TAN && NL == NL_GRAD2) {
        // KPZ tangent: q = g_x^2 + g_y^2 and q' = 2 (g_x dg_x + g_y dg_y), g_x = IDFT_x(i k_x P), g_y = IDFT_x(P_y),
        // dg likewise from dP, dP_y (Sec. V.B linearised).  Tiles: 0 P (then Q), 1 P_y, 2 dP (then dQ), 3 dP_y;
        // tile rows 0 and then 1 serve as the team's exchange buffer once read.
        load_tile<C>(tile, a.pin, rowbase, ncols, ny, y0);
        load_tile<C>(tile + ROWS * TS, a.pyin, rowbase, ncols, ny, y0);
        load_tile<C>(tile + 2 * ROWS * TS, a.dpin, rowbase, ncols, ny, y0);
        load_tile<C>(tile + 3 * ROWS * TS, a.dpyin, rowbase, ncols, ny, y0);
        __syncthreads();
        float2* r0 = tile + team * TS;
        float2* r1 = tile + ROWS * TS + team * TS;
        float2* r2 = tile + 2 * ROWS * TS + team * TS;
        float2* r3 = tile + 3 * ROWS * TS + team * TS;
        float2 zd[E], zy[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            const float2 tw = __ldg(&twN[k]);
            const float kx = a.dk * (float)k, kxm = (k == 0) ? 0.f : a.dk * (float)(M - k);
            z[e] = c2r_pre(cscale(cmuli(r0[k]), kx), cscale(cmuli(r0[M - k]), kxm), tw);
            zd[e] = c2r_pre(cscale(cmuli(r2[k]), kx), cscale(cmuli(r2[M - k]), kxm), tw);
            zy[e] = c2r_pre(r1[k], r1[M - k], tw);
        }
        fft_line<M, true>(z, r0, t, twM);
        fft_line<M, true>(zd, r0, t, twM);
        fft_line<M, true>(zy, r0, t, twM);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            zd[e] = make_float2(2.f * z[e].x * zd[e].x, 2.f * z[e].y * zd[e].y);
            z[e] = make_float2(z[e].x * z[e].x + zy[e].x * zy[e].x, z[e].y * z[e].y + zy[e].y * zy[e].y);
        }
        fft_line<M, false>(z, r0, t, twM);
        row_post<M>(z, r0, r0, ncols, t, twN);  // Q in tile 0
        // dg_y from dP_y (tile 3), exchanging through tile 1
        team_sync<T>();
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            z[e] = c2r_pre(r3[k], r3[M - k], __ldg(&twN[k]));
        }
        fft_line<M, true>(z, r1, t, twM);
#pragma unroll
        for (int e = 0; e < E; ++e)
            zd[e] = make_float2(zd[e].x + 2.f * zy[e].x * z[e].x, zd[e].y + 2.f * zy[e].y * z[e].y);
        fft_line<M, false>(zd, r1, t, twM);
        row_post<M>(zd, r1, r2, ncols, t, twN);  // dQ in tile 2
        __syncthreads();
        store_tile<C>(tile, a.qout, rowbase, ncols, ny, y0);
        store_tile<C>(tile + 2 * ROWS * TS, a.dqout, rowbase, ncols, ny, y0);
        return;
    }
    if constexpr (MODE == MODE_ADJ && NL == NL_GRAD2) {
        // KPZ adjoint (the transpose of q' = 2 (g_x dg_x + g_y dg_y), Sec. V.B linearised): with w the row of
        // W = IDFT(M s nu), v_x = 2 g_x w and v_y = 2 g_y w; the row pass returns DFT_x(v_x) and DFT_x(v_y),
        // and the column pass applies the transposed gradient multipliers -i k_x, -i k_y.  Tiles: 0 P (then
        // DFT_x(v_x)), 1 P_y (then DFT_x(v_y)), 2 W; tile rows 0 and 1 serve as the team's exchange buffers.
        load_tile<C>(tile, a.pin, rowbase, ncols, ny, y0);
        load_tile<C>(tile + ROWS * TS, a.pyin, rowbase, ncols, ny, y0);
        load_tile<C>(tile + 2 * ROWS * TS, a.dpin, rowbase, ncols, ny, y0);
        __syncthreads();
        float2* r0 = tile + team * TS;
        float2* r1 = tile + ROWS * TS + team * TS;
        const float2* r2 = tile + 2 * ROWS * TS + team * TS;
        float2 zw[E], zy[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            const float2 tw = __ldg(&twN[k]);
            const float kx = a.dk * (float)k, kxm = (k == 0) ? 0.f : a.dk * (float)(M - k);
            z[e] = c2r_pre(cscale(cmuli(r0[k]), kx), cscale(cmuli(r0[M - k]), kxm), tw);
            zy[e] = c2r_pre(r1[k], r1[M - k], tw);
            zw[e] = c2r_pre(r2[k], r2[M - k], tw);
        }
        fft_line<M, true>(z, r0, t, twM);
        fft_line<M, true>(zy, r0, t, twM);
        fft_line<M, true>(zw, r0, t, twM);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            z[e] = make_float2(2.f * z[e].x * zw[e].x, 2.f * z[e].y * zw[e].y);
            zy[e] = make_float2(2.f * zy[e].x * zw[e].x, 2.f * zy[e].y * zw[e].y);
        }
        fft_line<M, false>(z, r0, t, twM);
        row_post<M>(z, r0, r0, ncols, t, twN);
        team_sync<T>();
        fft_line<M, false>(zy, r1, t, twM);
        row_post<M>(zy, r1, r1, ncols, t, twN);
        __syncthreads();
        store_tile<C>(tile, a.dqout, rowbase, ncols, ny, y0);
        store_tile<C>(tile + ROWS * TS, a.qout, rowbase, ncols, ny, y0);
        return;
    }
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
    if constexpr (MODE == MODE_STEP_PS) {
        // phase-shift dealiasing along x: q on the plain grid and on the grid shifted by half a
        // cell along x (input phases e^{i pi k / N}, output phases e^{-i pi k / N}), averaged.
        // The block's rows are those of one copy of P (plain or shifted along y: blockIdx.y runs
        // over 2R copies).  Tile 0 holds the row for the plain grid, tile 1 a second copy for the
        // shifted one (each team row is also its evaluation's exchange buffer); KPZ adds the
        // matching rows of P_y in tiles 2 and 3.
        constexpr bool G = NL == NL_GRAD2;
        static_assert(NL == NL_CUBIC || G, "phase-shift dealiasing: cubic or gradient-squared term");
        load_tile<C>(tile, a.pin, rowbase, ncols, ny, y0);
        load_tile<C>(tile + ROWS * TS, a.pin, rowbase, ncols, ny, y0);
        if constexpr (G) {
            load_tile<C>(tile + 2 * ROWS * TS, a.pyin, rowbase, ncols, ny, y0);
            load_tile<C>(tile + 3 * ROWS * TS, a.pyin, rowbase, ncols, ny, y0);
        }
        __syncthreads();
        float2* r0 = tile + team * TS;
        float2* r1 = tile + ROWS * TS + team * TS;
        const float2* __restrict__ tps = a.tw_ps;
        // q on one grid from the P row (and the P_y row), phase e^{i pi k / N} on the shifted one; xb: the P row
        auto q_of = [&](const float2* prow, const float2* pyrow, bool shift, float2* xbuf) {
            float2 zy[G ? E : 1];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = t + T * e;
                const float2 ph = shift ? cconj(__ldg(&tps[k])) : make_float2(1.f, 0.f);
                const float2 phm = shift ? cconj(__ldg(&tps[M - k])) : make_float2(1.f, 0.f);
                const float2 tw = __ldg(&twN[k]);
                if constexpr (G) {
                    // grad_x h from i k_x P (k_x = 0 at the Nyquist column), grad_y h from P_y
                    const float kx = a.dk * (float)k, kxm = (k == 0) ? 0.f : a.dk * (float)(M - k);
                    z[e] = c2r_pre(cmul(cscale(cmuli(prow[k]), kx), ph), cmul(cscale(cmuli(prow[M - k]), kxm), phm),
                                   tw);
                    zy[e] = c2r_pre(cmul(pyrow[k], ph), cmul(pyrow[M - k], phm), tw);
                } else {
                    z[e] = c2r_pre(cmul(prow[k], ph), cmul(prow[M - k], phm), tw);
                }
            }
            fft_line<M, true>(z, xbuf, t, twM);
            if constexpr (G) {
                fft_line<M, true>(zy, xbuf, t, twM);
#pragma unroll
                for (int e = 0; e < E; ++e)
                    z[e] = make_float2(z[e].x * z[e].x + zy[e].x * zy[e].x, z[e].y * z[e].y + zy[e].y * zy[e].y);
            } else {
#pragma unroll
                for (int e = 0; e < E; ++e) z[e] = make_float2(z[e].x * z[e].x * z[e].x, z[e].y * z[e].y * z[e].y);
            }
            fft_line<M, false>(z, xbuf, t, twM);
            row_post<M>(z, xbuf, xbuf, ncols, t, twN);
        };
        q_of(r0, G ? tile + 2 * ROWS * TS + team * TS : nullptr, false, r0);
        q_of(r1, G ? tile + 3 * ROWS * TS + team * TS : nullptr, true, r1);
        // each thread reads back the entries k = t + T e that it wrote itself
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = t + T * e;
            if (k < ncols) r0[k] = cscale(cadd(r0[k], cmul(r1[k], __ldg(&tps[k]))), 0.5f);
        }
        __syncthreads();
        store_tile<C>(tile, a.qout, rowbase, ncols, ny, y0);
        return;
    }
    if constexpr (MODE == MODE_FWD) {
        const float* src = a.real_io + ((size_t)rep * ny + (yok ? y : 0)) * (2 * M);
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int m = t + T * e;
            z[e] = yok ? *reinterpret_cast<const float2*>(src + 2 * m) : czero();
        }
    } else if constexpr (MODE == MODE_FWD_NOISE) {
        // real-space noise of the step (Sec. IV step 2): site s = y nx + x takes normal s & 3 of
        // Philox(ctr = (s >> 2, step, replica, 3)); the packed pair m of row y (sites 2m, 2m + 1) is
        // normal pair y M + m, drawn here instead of being read from memory
        const long long step = current_step(a);
#pragma unroll
        for (int e = 0; e < E; e += 2)
            team_normal_pair_ks<T>(a.ks, (uint64_t)(yok ? y : 0) * M, t, e, (uint32_t)step, (uint32_t)(a.rep0 + rep),
                                z[e], z[e + 1], 3u);
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
            z[e] = r2c_post(z[e], cconj(xb[xpos<M>(mirror_idx<M>(k))]), __ldg(&twN[k]));
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

// ----------------------------------------------------------------- launchers
template <int M, int NL, int MODE, int SH = 0>
static cudaError_t run_rows(const StepArgs& a, cudaStream_t s) {
    using C = RowCfg<M, SH>;
    constexpr int NTILE =
        (NL == NL_GRAD2 && (MODE == MODE_STEP_PS || MODE == MODE_TAN))
            ? 4
            : ((NL == NL_GRAD2 && MODE == MODE_ADJ)
                   ? 3
                   : (((NL == NL_GRAD2 && MODE == MODE_STEP) || MODE == MODE_TAN || MODE == MODE_ADJ ||
                       MODE == MODE_STEP_PS)
                          ? 2
                          : 1));
    const size_t sm = C::smem(NTILE);
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k2_rows_real<M, NL, MODE, SH>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    dim3 grid((a.ny + C::ROWS - 1) / C::ROWS, a.R);
    k2_rows_real<M, NL, MODE, SH><<<grid, C::THREADS, sm, s>>>(a);
    return cudaGetLastError();
}

template <int M, int NL>
static cudaError_t rows_step(const StepArgs& a, cudaStream_t s, int shape) {
    if (shape == 1) return run_rows<M, NL, MODE_STEP, 1>(a, s);
    if (shape == 2) return run_rows<M, NL, MODE_STEP, 2>(a, s);
    return run_rows<M, NL, MODE_STEP, 0>(a, s);
}

template <int M>
static cudaError_t rows_for(const StepArgs& a, int mode, int nl, cudaStream_t s, int shape) {
    if (mode == MODE_FWD) return run_rows<M, NL_CUBIC, MODE_FWD>(a, s);
    if (mode == MODE_FWD_NOISE) return run_rows<M, NL_CUBIC, MODE_FWD_NOISE>(a, s);
    if (mode == MODE_INV) return run_rows<M, NL_CUBIC, MODE_INV>(a, s);
    if (mode == MODE_STEP && nl == NL_CUBIC) return rows_step<M, NL_CUBIC>(a, s, shape);
    if (mode == MODE_STEP && nl == NL_GRAD2) return rows_step<M, NL_GRAD2>(a, s, shape);
    if (mode == MODE_STEP_PS && nl == NL_CUBIC) return run_rows<M, NL_CUBIC, MODE_STEP_PS>(a, s);
    if (mode == MODE_STEP_PS && nl == NL_GRAD2) return run_rows<M, NL_GRAD2, MODE_STEP_PS>(a, s);
    if (mode == MODE_TAN && nl == NL_CUBIC) return run_rows<M, NL_CUBIC, MODE_TAN>(a, s);
    if (mode == MODE_TAN && nl == NL_GRAD2) return run_rows<M, NL_GRAD2, MODE_TAN>(a, s);
    if (mode == MODE_ADJ && nl == NL_CUBIC) return run_rows<M, NL_CUBIC, MODE_ADJ>(a, s);
    if (mode == MODE_ADJ && nl == NL_GRAD2) return run_rows<M, NL_GRAD2, MODE_ADJ>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace sft
