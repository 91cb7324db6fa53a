// sft_step_common.cuh -- per-mode pieces of the SETD update shared by the
// 1-D, 2-D and 3-D kernels: coefficient lookup, nonlinear prefactor, Fourier
// noise, the update itself and the status word.
#pragma once
#include "sft_device.cuh"
#include "sft_internal.h"

namespace sft {

__device__ __forceinline__ int signed_idx(int i, int n) { return (2 * i < n) ? i : i - n; }

// Odd-derivative wavenumber index: zero at the Nyquist index.
__device__ __forceinline__ int odd_idx(int i, int n) { return (2 * i == n) ? 0 : signed_idx(i, n); }

// 2/3-rule truncation on one axis: 3 |a| < n (axes of length 1 always pass).
__device__ __forceinline__ bool keep_axis(int a_signed, int n) { return n == 1 || 3 * abs(a_signed) < n; }

struct Coefs {
    float2 f1, A, B, g;
};

// Coefficients of mode class q = |a|^2 (Sec. II: f1 = e^{ch}; A, B from the
// scheme; g the noise amplitude).  SETD2's first step uses the SETD1 pair:
// A + B = h phi1 = f2 and B = 0.
template <bool CPLX>
__device__ __forceinline__ Coefs load_coefs(const float4* __restrict__ tab, int q, bool setd2_first) {
    Coefs c;
    if constexpr (CPLX) {
        const float4 t0 = __ldg(&tab[2 * q]);
        const float4 t1 = __ldg(&tab[2 * q + 1]);
        c.f1 = make_float2(t0.x, t0.y);
        c.A = make_float2(t0.z, t0.w);
        c.B = make_float2(t1.x, t1.y);
        c.g = make_float2(t1.z, t1.w);
    } else {
        const float4 t = __ldg(&tab[q]);
        c.f1 = make_float2(t.x, 0.f);
        c.A = make_float2(t.y, 0.f);
        c.B = make_float2(t.z, 0.f);
        c.g = make_float2(t.w, 0.f);
    }
    if (setd2_first) {
        c.A = cadd(c.A, c.B);
        c.B = czero();
    }
    return c;
}

// Nonlinear prefactor s_a of F_a = M_a s_a DFT[q] (Sec. V):
// Model A: -Gamma u; Model B: -Gamma u k^2; KPZ: lambda/2; CGL: -(1 + i beta).
__device__ __forceinline__ float2 nl_prefactor(const StepArgs& a, int q) {
    if (a.model == 1) return make_float2(a.s0 * a.dk * a.dk * (float)q, 0.f);
    return make_float2(a.s0, a.s0i);
}

// Fourier noise eta of one stored mode (App. B).  j: x-major counter index.
// selfc: self-conjugate mode of a real field (real N(0,1)); otherwise complex
// (A + iB)/sqrt2 with A, B ~ N(0,1).
__device__ __forceinline__ float2 fourier_noise(uint64_t seed, uint64_t j, uint32_t step, uint32_t replica,
                                                bool selfc) {
    const float2 z = normal_pair_for_index(seed, j, step, replica, 0u);
    if (selfc) return make_float2(z.x, 0.f);
    const float r2 = 0x1.6a09e6p-1f;  // 1/sqrt(2)
    return make_float2(z.x * r2, z.y * r2);
}

// Normal pairs of two modes a team holds, j(e) = jbase + t + T e and j(e+1)
// (jbase even, T even or 1, e even), with one Philox call per counter: the two
// modes 2m, 2m+1 of counter m sit in lanes t, t^1 (or slots e, e+1 when
// T = 1).  The even lane draws the counter of its mode at e, the odd lane the
// counter of its mode at e+1; each keeps one Box-Muller pair and hands the
// other to its partner lane with one shuffle.  Every lane of the warp must
// call this (warp shuffles).
template <int T>
__device__ __forceinline__ void team_normal_pair(uint64_t seed, uint64_t jbase, int t, int e, uint32_t step,
                                                 uint32_t replica, float2& z0, float2& z1, uint32_t tag = 0u) {
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    if constexpr (T == 1) {
        const uint64_t j = jbase + e;
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(j >> 1), step, replica, tag), key);
        z0 = recipe_bm_pair(w.x, w.y);
        z1 = recipe_bm_pair(w.z, w.w);
    } else {
        const bool odd = (t & 1) != 0;
        const uint64_t j = jbase + t + (uint64_t)T * (e + (odd ? 1 : 0));
        const uint4 w = philox4x32_10(make_uint4((uint32_t)(j >> 1), step, replica, tag), key);
        const float2 p0 = recipe_bm_pair(w.x, w.y), p1 = recipe_bm_pair(w.z, w.w);
        const float2 send = odd ? p0 : p1;
        float2 recv;
        recv.x = __shfl_xor_sync(0xffffffffu, send.x, 1);
        recv.y = __shfl_xor_sync(0xffffffffu, send.y, 1);
        z0 = odd ? recv : p0;
        z1 = odd ? p1 : recv;
    }
}

// team_normal_pair with the round keys of the seed precomputed (StepArgs::ks): the same words.
template <int T>
__device__ __forceinline__ void team_normal_pair_ks(const uint32_t (&ks)[20], uint64_t jbase, int t, int e,
                                                    uint32_t step, uint32_t replica, float2& z0, float2& z1,
                                                    uint32_t tag = 0u) {
    if constexpr (T == 1) {
        const uint64_t j = jbase + e;
        const uint4 w = philox4x32_10_ks(make_uint4((uint32_t)(j >> 1), step, replica, tag), ks);
        const float4 pp = recipe_bm_pair2(w.x, w.y, w.z, w.w);
        z0 = make_float2(pp.x, pp.y);
        z1 = make_float2(pp.z, pp.w);
    } else {
        const bool odd = (t & 1) != 0;
        const uint64_t j = jbase + t + (uint64_t)T * (e + (odd ? 1 : 0));
        const uint4 w = philox4x32_10_ks(make_uint4((uint32_t)(j >> 1), step, replica, tag), ks);
        const float4 pp = recipe_bm_pair2(w.x, w.y, w.z, w.w);
        const float2 p0 = make_float2(pp.x, pp.y), p1 = make_float2(pp.z, pp.w);
        const float2 send = odd ? p0 : p1;
        float2 recv;
        recv.x = __shfl_xor_sync(0xffffffffu, send.x, 1);
        recv.y = __shfl_xor_sync(0xffffffffu, send.y, 1);
        z0 = odd ? recv : p0;
        z1 = odd ? p1 : recv;
    }
}

// eta from a normal pair: self-conjugate modes real N(0,1), others (z0 + i z1)/sqrt2.
__device__ __forceinline__ float2 eta_of(float2 z, bool selfc) {
    if (selfc) return make_float2(z.x, 0.f);
    const float r2 = 0x1.6a09e6p-1f;
    return make_float2(z.x * r2, z.y * r2);
}

// Block-wide copy of the elements f in [0, n), n <= NMAX: thread i takes
// f = i, i + THREADS, ... (THREADS = blockDim.x).  Loads are issued in batches
// of up to 24 per thread before the matching stores, so a whole batch of
// global loads is in flight at once; a loop with one load and one dependent
// store per trip would wait a full memory latency per trip.
template <int THREADS, int NMAX, class Load, class Store>
__device__ __forceinline__ void block_copy(int n, Load&& load, Store&& store) {
    constexpr int NIT = (NMAX + THREADS - 1) / THREADS;
    constexpr int B = NIT <= 24 ? NIT : 16;
#pragma unroll
    for (int i0 = 0; i0 < NIT; i0 += B) {
        decltype(load(0)) v[B];
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int f = (int)threadIdx.x + (i0 + u) * THREADS;
            if (i0 + u < NIT && f < n) v[u] = load(f);
        }
#pragma unroll
        for (int u = 0; u < B; ++u) {
            const int f = (int)threadIdx.x + (i0 + u) * THREADS;
            if (i0 + u < NIT && f < n) store(f, v[u]);
        }
    }
}

__device__ __forceinline__ long long current_step(const StepArgs& a) { return *a.step_base + a.k_in_chunk; }

// Iteration limit of the launch's bounded waits (StepArgs::wait_limit).
__device__ __forceinline__ uint32_t wait_iters(const StepArgs& a) {
    return a.wait_limit == 0 ? (1u << 22) : (a.wait_limit < 0 ? 0u : (uint32_t)a.wait_limit);
}

__device__ __forceinline__ void flag_nonfinite(const StepArgs& a, float2 v, long long step) {
    if (!isfinite(v.x) || !isfinite(v.y)) {
        atomicOr(a.status, 1u);
        atomicMin((unsigned long long*)a.bad_step, (unsigned long long)step);
    }
}

// Branch-free form of the check above for a set of values: x * 0 is NaN exactly
// when x is infinite or NaN (and +-0 otherwise, which leaves acc unchanged), so
// acc stays 0 while every value is finite; one flag_nonfinite_acc at the end.
__device__ __forceinline__ float nonfinite_acc(float acc, float2 v) {
    return __fmaf_rn(v.y, 0.f, __fmaf_rn(v.x, 0.f, acc));
}
__device__ __forceinline__ void flag_nonfinite_acc(const StepArgs& a, float acc, long long step) {
    if (acc != acc) {
        atomicOr(a.status, 1u);
        atomicMin((unsigned long long*)a.bad_step, (unsigned long long)step);
    }
}

// phi_new = f1 phi + A F + B F_prev + g eta   (complex arithmetic throughout;
// for real fields the imaginary parts of the coefficients are zero).
template <bool CPLX>
__device__ __forceinline__ float2 setd_update(const Coefs& c, float2 phi, float2 F, float2 Fp, float2 eta) {
    if constexpr (CPLX) {
        float2 r = cmul(c.f1, phi);
        r = cadd(r, cmul(c.A, F));
        r = cadd(r, cmul(c.B, Fp));
        r = cadd(r, cmul(c.g, eta));
        return r;
    } else {
        return make_float2(c.f1.x * phi.x + c.A.x * F.x + c.B.x * Fp.x + c.g.x * eta.x,
                           c.f1.x * phi.y + c.A.x * F.y + c.B.x * Fp.y + c.g.x * eta.y);
    }
}

// ------------------------------------------------------------ real-FFT helpers
// Half-spectrum X[0..M] of a real line of N = 2M points -> Z[k] such that the
// unnormalised inverse M-point FFT of Z gives N (x[2m] + i x[2m+1]):
//   Z[k] = (X[k] + conj X[M-k]) + i W_N^{-k} (X[k] - conj X[M-k]).
__device__ __forceinline__ float2 c2r_pre(float2 Xk, float2 Xm, float2 twk) {
    const float2 cm = cconj(Xm);
    const float2 e = cadd(Xk, cm);
    const float2 o = cmul(csub(Xk, cm), cconj(twk));
    return cadd(e, cmuli(o));
}
// Z[k] = FFT_M(x[2m] + i x[2m+1]) -> X[k] = E + W_N^k O with
// E = (Z[k] + conj Z[M-k]) / 2, O = (Z[k] - conj Z[M-k]) / (2i).  Bc = conj Z[M-k].
__device__ __forceinline__ float2 r2c_post(float2 A, float2 Bc, float2 twk) {
    const float2 e = cadd(A, Bc);
    const float2 d = cmul(csub(A, Bc), twk);
    return make_float2(0.5f * (e.x + d.y), 0.5f * (e.y - d.x));  // (e - i d) / 2
}

}  // namespace sft
