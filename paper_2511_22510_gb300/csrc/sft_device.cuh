// sft_device.cuh -- device building blocks of the stochastic-ETD stepper:
// complex arithmetic, the Philox4x32-10 counter generator, the single-precision
// Box-Muller recipe (bit-reproducible: only correctly rounded IEEE operations
// through the __f*_rn intrinsics, never contracted), and a shared-memory
// Stockham FFT engine in which a team of T threads holds a line of N complex
// values (E per thread), with warp/named-barrier synchronisation.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sft {

// ----------------------------------------------------------------- complex
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float2 cmuli(float2 a) { return make_float2(-a.y, a.x); }  // i * a
__device__ __forceinline__ float2 czero() { return make_float2(0.f, 0.f); }

// ------------------------------------------------------------------ Philox
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of the 4x32
// bijection with multipliers 0xD2511F53 / 0xCD9E8D57, key bumped by the Weyl
// constants 0x9E3779B9 / 0xBB67AE85 between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        if (i > 0) {
            k.x += 0x9E3779B9u;
            k.y += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

// The same generator with the ten round keys given (ks[2i], ks[2i + 1] = key +
// i Weyl constants): kernels pass the schedule of their seed as a kernel
// parameter, so no key additions are issued per call.
__device__ __forceinline__ uint4 philox4x32_10_ks(uint4 c, const uint32_t (&ks)[20]) {
#pragma unroll
    for (int i = 0; i < 10; ++i) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ ks[2 * i], lo1, hi0 ^ c.w ^ ks[2 * i + 1], lo0);
    }
    return c;
}

// --------------------------------------------------------- Box-Muller recipe
// ln x for x in [2^-24, 1]: x = 2^e m, m in (1/sqrt2, sqrt2]; ln m = 2 atanh(s),
// s = (m-1)/(m+1), odd Taylor series of atanh through s^11; ln 2 split in a
// short head and a tail.  Each step is one correctly rounded binary32 op.
__device__ __forceinline__ float recipe_log(float x) {
    const uint32_t b = __float_as_uint(x);
    int e = (int)(b >> 23) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > 0x1.6a09e6p+0f) {
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float p = __fmaf_rn(s2, 0x1.745d18p-4f, 0x1.c71c72p-4f);
    p = __fmaf_rn(s2, p, 0x1.24924ap-3f);
    p = __fmaf_rn(s2, p, 0x1.99999ap-3f);
    p = __fmaf_rn(s2, p, 0x1.555556p-2f);
    const float t = __fmul_rn(s2, p);
    const float two_s = __fadd_rn(s, s);
    const float lnm = __fmaf_rn(two_s, t, two_s);
    const float ef = __int2float_rn(e);
    return __fmaf_rn(ef, 0x1.62e4p-1f, __fmaf_rn(ef, 0x1.7f7d1cp-20f, lnm));
}

// sin and cos of 2 pi k / 2^24: exact integer reduction to the nearest quarter
// turn, Taylor series of sin (through x^11) and cos (through x^10) on [-pi/4, pi/4).
__device__ __forceinline__ void recipe_sincos_turn(uint32_t k24, float& sn, float& cs) {
    const uint32_t qq = (k24 + 0x200000u) >> 22;
    const int32_t r = (int32_t)k24 - (int32_t)(qq << 22);
    const uint32_t q = qq & 3u;
    const float x = __fmul_rn(__int2float_rn(r), 0x1.921fb6p-22f);
    const float x2 = __fmul_rn(x, x);
    float ps = __fmaf_rn(x2, -0x1.ae6456p-26f, 0x1.71de3ap-19f);
    ps = __fmaf_rn(x2, ps, -0x1.a01a02p-13f);
    ps = __fmaf_rn(x2, ps, 0x1.111112p-7f);
    ps = __fmaf_rn(x2, ps, -0x1.555556p-3f);
    const float sx = __fmaf_rn(__fmul_rn(x, x2), ps, x);
    float pc = __fmaf_rn(x2, -0x1.27e4fcp-22f, 0x1.a01a02p-16f);
    pc = __fmaf_rn(x2, pc, -0x1.6c16c2p-10f);
    pc = __fmaf_rn(x2, pc, 0x1.555556p-5f);
    pc = __fmaf_rn(x2, pc, -0.5f);
    const float cx = __fmaf_rn(x2, pc, 1.0f);
    switch (q) {
        case 0: sn = sx; cs = cx; break;
        case 1: sn = cx; cs = -sx; break;
        case 2: sn = -sx; cs = -cx; break;
        default: sn = -cx; cs = sx; break;
    }
}

// One Box-Muller pair from two 32-bit words:
//   u1 = ((wa >> 8) + 1) 2^-24 in (0, 1], turn = (wb >> 8) 2^-24,
//   z0 = sqrt(-2 ln u1) cos(2 pi turn), z1 = sqrt(-2 ln u1) sin(2 pi turn).
__device__ __forceinline__ float2 recipe_bm_pair(uint32_t wa, uint32_t wb) {
    const float u1 = __fmul_rn(__uint2float_rn((wa >> 8) + 1u), 0x1p-24f);
    const float rad = __fsqrt_rn(__fmul_rn(-2.0f, recipe_log(u1)));
    float sn, cs;
    recipe_sincos_turn(wb >> 8, sn, cs);
    return make_float2(__fmul_rn(rad, cs), __fmul_rn(rad, sn));
}

// The recipe for two pairs at once, (wa0, wb0) and (wa1, wb1), with the paired
// single-precision instructions of sm_100 and later (__fadd2_rn, __fmul2_rn,
// __ffma2_rn: per component the same correctly rounded operation as the
// scalar one): every floating-point step of recipe_log, recipe_sincos_turn
// and recipe_bm_pair, in the same order, so each pair has exactly the bits of
// recipe_bm_pair.  Returns (z0, z1) of the first pair in .x, .y and of the
// second in .z, .w.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

__device__ __forceinline__ float2 recipe_log2(float2 x) {
    const uint32_t b0 = __float_as_uint(x.x), b1 = __float_as_uint(x.y);
    int e0 = (int)(b0 >> 23) - 127, e1 = (int)(b1 >> 23) - 127;
    float2 m = make_float2(__uint_as_float((b0 & 0x007FFFFFu) | 0x3F800000u),
                           __uint_as_float((b1 & 0x007FFFFFu) | 0x3F800000u));
    // m > sqrt2: halve it (an exact product) and bump the exponent
    const bool h0 = m.x > 0x1.6a09e6p+0f, h1 = m.y > 0x1.6a09e6p+0f;
    m = __fmul2_rn(m, make_float2(h0 ? 0.5f : 1.0f, h1 ? 0.5f : 1.0f));
    e0 += h0 ? 1 : 0;
    e1 += h1 ? 1 : 0;
    const float2 num = __fadd2_rn(m, f2(-1.0f)), den = __fadd2_rn(m, f2(1.0f));
    const float2 s = make_float2(__fdiv_rn(num.x, den.x), __fdiv_rn(num.y, den.y));
    const float2 s2 = __fmul2_rn(s, s);
    float2 p = __ffma2_rn(s2, f2(0x1.745d18p-4f), f2(0x1.c71c72p-4f));
    p = __ffma2_rn(s2, p, f2(0x1.24924ap-3f));
    p = __ffma2_rn(s2, p, f2(0x1.99999ap-3f));
    p = __ffma2_rn(s2, p, f2(0x1.555556p-2f));
    const float2 t = __fmul2_rn(s2, p);
    const float2 two_s = __fadd2_rn(s, s);
    const float2 lnm = __ffma2_rn(two_s, t, two_s);
    const float2 ef = make_float2(__int2float_rn(e0), __int2float_rn(e1));
    return __ffma2_rn(ef, f2(0x1.62e4p-1f), __ffma2_rn(ef, f2(0x1.7f7d1cp-20f), lnm));
}

__device__ __forceinline__ void recipe_sincos_turn2(uint32_t k0, uint32_t k1, float2& sn, float2& cs) {
    const uint32_t qq0 = (k0 + 0x200000u) >> 22, qq1 = (k1 + 0x200000u) >> 22;
    const int32_t r0 = (int32_t)k0 - (int32_t)(qq0 << 22), r1 = (int32_t)k1 - (int32_t)(qq1 << 22);
    const float2 x = __fmul2_rn(make_float2(__int2float_rn(r0), __int2float_rn(r1)), f2(0x1.921fb6p-22f));
    const float2 x2 = __fmul2_rn(x, x);
    float2 ps = __ffma2_rn(x2, f2(-0x1.ae6456p-26f), f2(0x1.71de3ap-19f));
    ps = __ffma2_rn(x2, ps, f2(-0x1.a01a02p-13f));
    ps = __ffma2_rn(x2, ps, f2(0x1.111112p-7f));
    ps = __ffma2_rn(x2, ps, f2(-0x1.555556p-3f));
    const float2 sx = __ffma2_rn(__fmul2_rn(x, x2), ps, x);
    float2 pc = __ffma2_rn(x2, f2(-0x1.27e4fcp-22f), f2(0x1.a01a02p-16f));
    pc = __ffma2_rn(x2, pc, f2(-0x1.6c16c2p-10f));
    pc = __ffma2_rn(x2, pc, f2(0x1.555556p-5f));
    pc = __ffma2_rn(x2, pc, f2(-0.5f));
    const float2 cx = __ffma2_rn(x2, pc, f2(1.0f));
    auto quad = [](uint32_t q, float s, float c, float& so, float& co) {
        switch (q & 3u) {
            case 0: so = s; co = c; break;
            case 1: so = c; co = -s; break;
            case 2: so = -s; co = -c; break;
            default: so = -c; co = s; break;
        }
    };
    quad(qq0, sx.x, cx.x, sn.x, cs.x);
    quad(qq1, sx.y, cx.y, sn.y, cs.y);
}

__device__ __forceinline__ float4 recipe_bm_pair2(uint32_t wa0, uint32_t wb0, uint32_t wa1, uint32_t wb1) {
    const float2 u1 = __fmul2_rn(make_float2(__uint2float_rn((wa0 >> 8) + 1u), __uint2float_rn((wa1 >> 8) + 1u)),
                                 f2(0x1p-24f));
    const float2 l = __fmul2_rn(f2(-2.0f), recipe_log2(u1));
    const float2 rad = make_float2(__fsqrt_rn(l.x), __fsqrt_rn(l.y));
    float2 sn, cs;
    recipe_sincos_turn2(wb0 >> 8, wb1 >> 8, sn, cs);
    const float2 z0 = __fmul2_rn(rad, cs), z1 = __fmul2_rn(rad, sn);
    return make_float4(z0.x, z1.x, z0.y, z1.y);
}

// The normal pair belonging to counter index j (x-major mode enumeration):
// Philox(ctr = (j >> 1, step, replica, tag), key = seed) -> words w0..w3;
// even j takes the pair of (w0, w1), odd j the pair of (w2, w3).
__device__ __forceinline__ float2 normal_pair_for_index(uint64_t seed, uint64_t j, uint32_t step, uint32_t replica,
                                                        uint32_t tag) {
    const uint4 w = philox4x32_10(make_uint4((uint32_t)(j >> 1), step, replica, tag),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    return (j & 1) ? recipe_bm_pair(w.z, w.w) : recipe_bm_pair(w.x, w.y);
}

// ------------------------------------------------------------- FFT engine
// Compile-time plan for an N-point line: E values per thread (32 for lines of
// 512 points and more, else up to 16), T = N / E threads per line, and the
// radix of every Stockham pass; every radix divides E, so each thread runs
// E / R butterflies per pass.  Lines of 1024 points take two radix-32 passes
// and a single shared-memory exchange.
#ifndef SFT_EMAX
#define SFT_EMAX 16
#endif
//
// Lines of N = p x 2^k points with an odd prime p in {3, 5, 7} (MIXED) take 4p
// values per thread: one radix-p pass, then radix-4 passes and a radix-2
// remainder.
template <int N, int EM = SFT_EMAX>
struct FftPlan {
    static constexpr int PR = N % 3 == 0 ? 3 : (N % 5 == 0 ? 5 : (N % 7 == 0 ? 7 : 1));  // odd factor
    static constexpr bool MIXED = PR > 1;
    static_assert(N >= 2 && ((N & (N - 1)) == 0 || (MIXED && N >= 4 * PR && ((N / PR) & (N / PR - 1)) == 0)),
                  "2^k or p x 2^k points, p in {3, 5, 7}");
    static constexpr int log2(int v) { return v <= 1 ? 0 : 1 + log2(v / 2); }
    static constexpr int L = log2(MIXED ? N / PR : N);  // the power-of-two factor
    static constexpr int E = MIXED ? 4 * PR : (N <= 16 ? N : (N >= 512 ? EM : (N <= 32 && EM >= 32 ? N : 16)));
    static constexpr int T = N / E;
    static constexpr int R0 = MIXED ? PR : E;  // first radix
    static constexpr int E2 = MIXED ? 4 : E;  // radix of the power-of-two passes
    // remaining log2 after the first pass, split into radix-E2 passes and a remainder
    static constexpr int LE = log2(E2);
    static constexpr int LR = MIXED ? L : L - log2(R0);
    static constexpr int P = 1 + (LR + LE - 1) / LE;
    static constexpr int radix(int p) {
        return p == 0 ? R0 : (p < P - 1 ? E2 : (LR % LE == 0 ? E2 : (1 << (LR % LE))));
    }
    // padded exchange buffer: one pad element per R0 (first-pass radix) elements
    static constexpr int PAD = R0 >= 16 ? R0 : 16;
    static constexpr int BUF = N + N / PAD + 1;
};

// padded position of element i in an exchange buffer of plan N
template <int N, int EM = SFT_EMAX>
__device__ __forceinline__ int xpos(int i) {
    return i + i / FftPlan<N, EM>::PAD;
}

// Team barrier: teams of T <= 32 threads live inside one warp and use the
// warp barrier (all lanes of the warp must take part); larger teams use a
// named barrier per team (ids 1..15).
template <int T>
__device__ __forceinline__ void team_sync() {
    if constexpr (T <= 32) {
        __syncwarp();
    } else {
        const int id = 1 + (int)(threadIdx.x / T);
        asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(T) : "memory");
    }
}

// cos / sin of 2 pi m / 32
__device__ constexpr float kCos32[32] = {
    1.0f, 0.98078528040323044f, 0.92387953251128674f, 0.83146961230254524f, 0.70710678118654752f,
    0.55557023301960218f, 0.38268343236508977f, 0.19509032201612826f, 0.0f, -0.19509032201612826f,
    -0.38268343236508977f, -0.55557023301960218f, -0.70710678118654752f, -0.83146961230254524f,
    -0.92387953251128674f, -0.98078528040323044f, -1.0f, -0.98078528040323044f, -0.92387953251128674f,
    -0.83146961230254524f, -0.70710678118654752f, -0.55557023301960218f, -0.38268343236508977f,
    -0.19509032201612826f, 0.0f, 0.19509032201612826f, 0.38268343236508977f, 0.55557023301960218f,
    0.70710678118654752f, 0.83146961230254524f, 0.92387953251128674f, 0.98078528040323044f};

// z * W_R^m with W_R = e^{-2 pi i / R} (forward) or its conjugate (inverse);
// m and R are compile-time constants after unrolling.  Angles are counted in
// 32nds of a turn; quarter turns are swaps, odd multiples of 1/8 turn use the
// (a +- b)/sqrt2 form.
template <bool INV>
__device__ __forceinline__ float2 twiddle_const(float2 z, int m, int R) {
    const int q = (m * 32 / R) & 31;
    if (q == 0) return z;
    if (q == 16) return make_float2(-z.x, -z.y);
    if (q == 8) return INV ? make_float2(-z.y, z.x) : make_float2(z.y, -z.x);
    if (q == 24) return INV ? make_float2(z.y, -z.x) : make_float2(-z.y, z.x);
    const float c = kCos32[q];
    const float sn = kCos32[(q + 24) & 31];  // sin(2 pi q / 32) = cos(2 pi (q - 8) / 32)
    const float s = INV ? sn : -sn;
    if ((q & 7) == 4) {
        const float r = 0.70710678118654752f;
        // c = +-r, s = +-r
        return make_float2(r * ((c > 0 ? z.x : -z.x) - (s > 0 ? z.y : -z.y)),
                           r * ((s > 0 ? z.x : -z.x) + (c > 0 ? z.y : -z.y)));
    }
    return make_float2(z.x * c - z.y * s, z.x * s + z.y * c);
}

template <int R>
__device__ constexpr int bitrev(int k) {
    int r = 0;
    for (int b = 1; b < R; b <<= 1) {
        r = (r << 1) | (k & 1);
        k >>= 1;
    }
    return r;
}

// In-register DFT of R values (R = 1, 2, 4, ..., 32): radix-2 decimation in
// frequency, then the bit-reversal permutation (resolved at compile time).
// cos and sin of 2 pi j / R for the radix-5 and radix-7 passes
__device__ constexpr float kCos5[5] = {1.0f, 0.309016994374947451f, -0.809016994374947340f, -0.809016994374947562f,
                                       0.309016994374947229f};
__device__ constexpr float kSin5[5] = {0.0f, 0.951056516295153531f, 0.587785252292473248f, -0.587785252292473026f,
                                       -0.951056516295153642f};
__device__ constexpr float kCos7[7] = {1.0f, 0.623489801858733594f, -0.222520933956314337f, -0.900968867902419035f,
                                       -0.900968867902419146f, -0.222520933956314587f, 0.623489801858733372f};
__device__ constexpr float kSin7[7] = {0.0f, 0.781831482468029804f, 0.974927912181823619f, 0.433883739117558231f,
                                       -0.433883739117558009f, -0.974927912181823619f, -0.781831482468029915f};

// DFT of an odd number R of values from its definition, pairing m with R - m:
// with s_m = x_m + x_{R-m}, d_m = x_m - x_{R-m} and theta = 2 pi k m / R,
// A_k = x_0 + sum_m s_m cos(theta), B_k = sum_m d_m sin(theta), and
// y_k = A_k -+ i B_k, y_{R-k} = A_k +- i B_k (forward / inverse).
template <int R>
__device__ __forceinline__ float odd_cos(int j) {
    if constexpr (R == 5) return kCos5[j]; else return kCos7[j];
}
template <int R>
__device__ __forceinline__ float odd_sin(int j) {
    if constexpr (R == 5) return kSin5[j]; else return kSin7[j];
}

template <int R, bool INV>
__device__ __forceinline__ void dft_odd(float2* x) {
    constexpr int H = (R - 1) / 2;
    float2 s[H], d[H];
    float2 y0 = x[0];
#pragma unroll
    for (int m = 1; m <= H; ++m) {
        s[m - 1] = cadd(x[m], x[R - m]);
        d[m - 1] = csub(x[m], x[R - m]);
        y0 = cadd(y0, s[m - 1]);
    }
    float2 y[R];
    y[0] = y0;
#pragma unroll
    for (int k = 1; k <= H; ++k) {
        float2 A = x[0], B = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 1; m <= H; ++m) {
            const float c = odd_cos<R>((k * m) % R), sv = odd_sin<R>((k * m) % R);
            A = make_float2(A.x + c * s[m - 1].x, A.y + c * s[m - 1].y);
            B = make_float2(B.x + sv * d[m - 1].x, B.y + sv * d[m - 1].y);
        }
        const float2 iB = make_float2(-B.y, B.x);
        y[k] = INV ? cadd(A, iB) : csub(A, iB);
        y[R - k] = INV ? csub(A, iB) : cadd(A, iB);
    }
#pragma unroll
    for (int k = 0; k < R; ++k) x[k] = y[k];
}

template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2* x) {
    if constexpr (R == 5 || R == 7) {
        dft_odd<R, INV>(x);
    } else if constexpr (R == 3) {
        // y1 = a + w b + w^2 c, y2 = a + w^2 b + w c with w = e^{-+2 pi i / 3} = -1/2 -+ i sqrt(3)/2
        const float2 a = x[0], s = cadd(x[1], x[2]), d = csub(x[1], x[2]);
        const float2 t = make_float2(a.x - 0.5f * s.x, a.y - 0.5f * s.y);
        const float h = 0.866025403784438647f;  // sin(2 pi / 3)
        const float2 ihd = make_float2(-h * d.y, h * d.x);  // i h d
        x[0] = cadd(a, s);
        x[1] = INV ? cadd(t, ihd) : csub(t, ihd);
        x[2] = INV ? csub(t, ihd) : cadd(t, ihd);
    } else if constexpr (R > 1) {
#pragma unroll
        for (int span = R / 2; span >= 1; span >>= 1) {
#pragma unroll
            for (int blk = 0; blk < R; blk += 2 * span) {
#pragma unroll
                for (int i = 0; i < span; ++i) {
                    const float2 a = x[blk + i], b = x[blk + i + span];
                    x[blk + i] = cadd(a, b);
                    x[blk + i + span] = twiddle_const<INV>(csub(a, b), i * (R / (2 * span)), R);
                }
            }
        }
        float2 y[R];
#pragma unroll
        for (int k = 0; k < R; ++k) y[k] = x[bitrev<R>(k)];
#pragma unroll
        for (int k = 0; k < R; ++k) x[k] = y[k];
    }
}

// Stockham pass PASS of an N-point FFT.  Thread t of the team holds v[e] =
// x[t + T e]; after the last pass it holds X[t + T e] in natural order.
// Passes other than the last exchange through the padded team buffer `buf`.
// tw: table of W_N^m = e^{-2 pi i m / N}, m in [0, N).
template <int N, bool INV, int PASS, int NS, int EM>
struct StockhamPass {
    static __device__ __forceinline__ void run(float2 (&v)[FftPlan<N, EM>::E], float2* buf, int t,
                                               const float2* __restrict__ tw) {
        using PL = FftPlan<N, EM>;
        constexpr int E = PL::E, T = PL::T;
        constexpr int R = PL::radix(PASS);
        constexpr int NB = E / R;
        constexpr bool FIRST = (PASS == 0);
        constexpr bool LAST = (NS * R == N);
        float2 x[NB][R];
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = t + T * b;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if constexpr (FIRST)
                    x[b][r] = v[b + r * NB];
                else
                    x[b][r] = buf[xpos<N, EM>(j + r * (N / R))];
            }
            if constexpr (!FIRST) {
                const int k = j % NS;
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    float2 w = __ldg(&tw[r * k * (N / (NS * R))]);
                    if (INV) w.y = -w.y;
                    x[b][r] = cmul(x[b][r], w);
                }
            }
            dft_reg<R, INV>(x[b]);
        }
        if constexpr (LAST) {
#pragma unroll
            for (int b = 0; b < NB; ++b)
#pragma unroll
                for (int s = 0; s < R; ++s) v[b + s * NB] = x[b][s];
        } else {
            team_sync<T>();
#pragma unroll
            for (int b = 0; b < NB; ++b) {
                const int j = t + T * b;
                const int k = j % NS;
                const int base = (j / NS) * NS * R + k;
#pragma unroll
                for (int s = 0; s < R; ++s) buf[xpos<N, EM>(base + s * NS)] = x[b][s];
            }
            team_sync<T>();
            StockhamPass<N, INV, PASS + 1, NS * R, EM>::run(v, buf, t, tw);
        }
    }
};

// Unnormalised N-point FFT of a line held by a team (forward: e^{-2 pi i}).
template <int N, bool INV, int EM = SFT_EMAX>
__device__ __forceinline__ void fft_line(float2 (&v)[FftPlan<N, EM>::E], float2* buf, int t,
                                         const float2* __restrict__ tw) {
    StockhamPass<N, INV, 0, 1, EM>::run(v, buf, t, tw);
}

}  // namespace sft
