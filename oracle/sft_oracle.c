/*
 * sft_oracle.c -- plain serial FP64 reference of the pseudo-spectral stochastic
 * exponential-time-differencing (SETD) step of Johnsrud & Rana, "Efficient
 * Pseudo-spectral Algorithms for Statistical Field Theories" (arXiv 2511.22510).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * constant generator with the CUDA library, and it never calls into it.
 *
 * Everything is written for clarity, not speed: the spectrum is kept as a FULL
 * complex array (no half-spectrum tricks), transforms are a textbook radix-2
 * FFT (pinned against a brute-force DFT; lengths p x 2^k split by radix 2 down to
 * the odd length, whose DFT is its definition), and every mode is updated in a
 * plain loop.  Floating point is double precision except for the Gaussian-noise
 * recipe, which is specified in single precision so that both implementations
 * produce bit-identical normal deviates (they are widened to double here).
 *
 * Paper passages followed (section / equation):
 *   Sec. II, Eq. (setd-beg): exact variation-of-constants identity.
 *   Sec. II: f1 = e^{ch}, f2 = (e^{ch}-1)/c, f3 = e^{ch/2}, f4^2 = (e^{2ch}-1)/(2c).
 *   Sec. II, Eqs. (SETD-EM), (SETD1), (SETD2): the three additive-noise schemes.
 *   Sec. IV, boxed algorithm: per-mode pseudo-spectral step with dealiasing and
 *     the noise factor (N^2/L)^{d/2}; EM limit for small c.
 *   Sec. V.A: Model A / Model B, c(k) = -k^Delta (r + k^2), D(k) = k^Delta D.
 *   Sec. V.B: KPZ, c = -nu k^2, F = (lambda/2) F[|grad h|^2].
 *   Sec. V.C: complex Ginzburg-Landau.
 *   App. A: DFT conventions and the (N^2/L)^d noise variance in Fourier space.
 *   App. B: Hermitian structure of the noise for real fields.
 *   App. C: equal-time correlator C_ET(k) = (L/N^2)^d |phi_a|^2 and shell average;
 *     dynamic correlation C(k, omega), noise-inferred susceptibility chi(k, omega)
 *     and the FDT deviation of Sec. V.A from recorded series (or_dyn_estimators).
 *   Sec. III: 0-d SDE ensembles (SAO, GBM) under the five update rules of the
 *     stability table.
 *   Sec. IV step 1, alternative: phase-shift dealiasing (mean of the nonlinear
 *     term over the 2^d half-cell-shifted grids).
 *   Sec. IV step 2, alternative: noise drawn per real-space site and transformed.
 *   Sec. V.A footnote: the r phi term placed in F (Model A/B, p[4] != 0).
 *
 * Readings where the paper is silent or inconsistent (each also listed in the
 * design notes of the repository):
 *   - DFT sign: forward e^{-2 pi i a.n/N}, inverse (1/N^d) e^{+...} (FFTW); the
 *     paper's App. A prints the opposite sign with an unnormalised inverse.
 *   - Dealiasing by truncation: box mask M_a = 1 iff 3|a_i| < N_i on every axis;
 *     applied to the state before the inverse transform and to F afterwards.
 *   - For complex c the noise amplitude is g^2 = (N/dx)^d 2 D h phi1(2 Re(c) h),
 *     the exact variance of int e^{c s} dW; for real c this is f4^2 2D.
 *   - SETD2's first step uses the SETD1 coefficients (no F at t-h exists).
 *   - Odd derivatives (KPZ gradient) use k = 0 at the Nyquist index.
 *   - Hermitian fix-up after every update: partner modes take the conjugate of
 *     their canonical mode and self-conjugate modes drop their imaginary part.
 *   - Phase-shift dealiasing masks the Nyquist modes (their shifted copies are
 *     not spectra of real fields) and keeps every other mode.
 *   - Real-space noise: eta_a = DFT[eta]_a / sqrt(N^d), site s taking normal
 *     s & 3 of Philox(s >> 2, step, replica, tag 3).
 *
 * Parity unpinned: the noise counter map (which Philox counter and which word
 * pair each mode or site takes) is a convention of this implementation; the
 * paper fixes only the distribution of the noise, whose structure (App. B
 * deviate counts, Hermitian symmetry, variances) is pinned.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

#define OR_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------- */
/* Philox4x32-10, Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11.  Ten rounds of the 4x32 bijection, key bumped     */
/* by the Weyl constants between rounds.                                      */
/* ------------------------------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* ------------------------------------------------------------------------- */
/* Single-precision Box-Muller recipe.  Every operation is one IEEE-754       */
/* correctly rounded binary32 operation (+, -, *, /, sqrt, fma), evaluated in */
/* a fixed order, so any conforming implementation gets the same bits.        */
/*   u1 = ((w0 >> 8) + 1) 2^-24 in (0, 1],   turn = (w1 >> 8) 2^-24 in [0,1)  */
/*   z0 = sqrt(-2 ln u1) cos(2 pi turn),     z1 = sqrt(-2 ln u1) sin(2 pi turn)*/
/* ln: argument split x = 2^e m with m in (1/sqrt2, sqrt2], then             */
/*     ln m = 2 atanh(s), s = (m-1)/(m+1), by its odd Taylor series.          */
/* sin/cos: exact integer reduction of the 24-bit turn count to the nearest  */
/*     quarter turn, then the Taylor series of sin and cos on [-pi/4, pi/4). */
/* ------------------------------------------------------------------------- */
static float f32_from_bits(uint32_t b) {
    float f;
    memcpy(&f, &b, sizeof f);
    return f;
}
static uint32_t f32_bits(float f) {
    uint32_t b;
    memcpy(&b, &f, sizeof b);
    return b;
}

float or_bm_log(float x) {
    uint32_t b = f32_bits(x);
    int e = (int)(b >> 23) - 127;
    float m = f32_from_bits((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > 0x1.6a09e6p+0f) {
        m = m * 0.5f;
        e += 1;
    }
    float s = (m - 1.0f) / (m + 1.0f);
    float s2 = s * s;
    /* atanh(s)/s - 1 = s^2/3 + s^4/5 + ... + s^10/11 */
    float p = fmaf(s2, 0x1.745d18p-4f, 0x1.c71c72p-4f); /* 1/11, 1/9 */
    p = fmaf(s2, p, 0x1.24924ap-3f);                    /* 1/7 */
    p = fmaf(s2, p, 0x1.99999ap-3f);                    /* 1/5 */
    p = fmaf(s2, p, 0x1.555556p-2f);                    /* 1/3 */
    float t = s2 * p;
    float two_s = s + s;
    float lnm = fmaf(two_s, t, two_s);
    float ef = (float)e;
    /* ln 2 split into a short head (exact products) and a tail */
    return fmaf(ef, 0x1.62e4p-1f, fmaf(ef, 0x1.7f7d1cp-20f, lnm));
}

void or_bm_sincos_turn(uint32_t k24, float* sn, float* cs) {
    /* angle = 2 pi k24 / 2^24 */
    uint32_t qq = (k24 + 0x200000u) >> 22; /* nearest quarter turn, 0..4 */
    int32_t r = (int32_t)k24 - (int32_t)(qq << 22);
    uint32_t q = qq & 3u;
    float x = (float)r * 0x1.921fb6p-22f; /* r * 2 pi / 2^24, |x| <= pi/4 */
    float x2 = x * x;
    float ps = fmaf(x2, -0x1.ae6456p-26f, 0x1.71de3ap-19f); /* -1/11!, 1/9! */
    ps = fmaf(x2, ps, -0x1.a01a02p-13f);                     /* -1/7! */
    ps = fmaf(x2, ps, 0x1.111112p-7f);                       /* 1/5! */
    ps = fmaf(x2, ps, -0x1.555556p-3f);                      /* -1/3! */
    float sx = fmaf(x * x2, ps, x);
    float pc = fmaf(x2, -0x1.27e4fcp-22f, 0x1.a01a02p-16f); /* -1/10!, 1/8! */
    pc = fmaf(x2, pc, -0x1.6c16c2p-10f);                     /* -1/6! */
    pc = fmaf(x2, pc, 0x1.555556p-5f);                       /* 1/4! */
    pc = fmaf(x2, pc, -0.5f);                                /* -1/2! */
    float cx = fmaf(x2, pc, 1.0f);
    switch (q) {
        case 0: *sn = sx; *cs = cx; break;
        case 1: *sn = cx; *cs = -sx; break;
        case 2: *sn = -sx; *cs = -cx; break;
        default: *sn = -cx; *cs = sx; break;
    }
}

void or_bm_pair(uint32_t wa, uint32_t wb, float* z0, float* z1) {
    float u1 = (float)((wa >> 8) + 1u) * 0x1p-24f;
    float rad = sqrtf(-2.0f * or_bm_log(u1));
    float sn, cs;
    or_bm_sincos_turn(wb >> 8, &sn, &cs);
    *z0 = rad * cs;
    *z1 = rad * sn;
}

/* Normal pair for counter index j: one Philox call serves indices 2m, 2m+1. */
static void normals_for_index(uint64_t seed, uint32_t jhalf_word, uint32_t step_word, uint32_t replica,
                              uint32_t tag, float z[4]) {
    uint32_t ctr[4] = {jhalf_word, step_word, replica, tag};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t w[4];
    or_philox4x32_10(ctr, key, w);
    or_bm_pair(w[0], w[1], &z[0], &z[1]);
    or_bm_pair(w[2], w[3], &z[2], &z[3]);
}

void or_normals4(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, float out[4]) {
    normals_for_index(seed, c0, c1, c2, c3, out);
}

/* ------------------------------------------------------------------------- */
/* Transforms.  Forward: X_a = sum_n e^{-2 pi i a.n/N} x_n (unnormalised).   */
/* Inverse (sign +1) is also unnormalised here; callers divide by N^d.       */
/* ------------------------------------------------------------------------- */
static int is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static void fft1d_radix2(cplx* x, int n, int sign) {
    /* bit-reversal permutation */
    for (int i = 1, j = 0; i < n; ++i) {
        int bit = n >> 1;
        for (; j & bit; bit >>= 1) j ^= bit;
        j ^= bit;
        if (i < j) {
            cplx t = x[i];
            x[i] = x[j];
            x[j] = t;
        }
    }
    for (int len = 2; len <= n; len <<= 1) {
        int half = len / 2;
        for (int k = 0; k < half; ++k) {
            double ang = (double)sign * 2.0 * OR_PI * (double)k / (double)len;
            cplx w = cos(ang) + I * sin(ang);
            for (int s = 0; s < n; s += len) {
                cplx u = x[s + k];
                cplx v = x[s + k + half] * w;
                x[s + k] = u + v;
                x[s + k + half] = u - v;
            }
        }
    }
}

/* Lengths that are not powers of two (p x 2^k lattices, p odd): radix-2 decimation in
 * time down to an odd length, whose DFT is taken from its definition (phase
 * (k m mod n) / n of a turn). */
static void fft1d_split(cplx* x, int n, int sign) {
    if (n % 2) {
        cplx* y = (cplx*)malloc(sizeof(cplx) * (size_t)n);
        for (int k = 0; k < n; ++k) {
            cplx acc = 0;
            for (int m = 0; m < n; ++m) {
                double ang = (double)sign * 2.0 * OR_PI * (double)((long)k * m % n) / (double)n;
                acc += x[m] * (cos(ang) + I * sin(ang));
            }
            y[k] = acc;
        }
        memcpy(x, y, sizeof(cplx) * (size_t)n);
        free(y);
        return;
    }
    int h = n / 2;
    cplx* ev = (cplx*)malloc(sizeof(cplx) * (size_t)h);
    cplx* od = (cplx*)malloc(sizeof(cplx) * (size_t)h);
    for (int i = 0; i < h; ++i) {
        ev[i] = x[2 * i];
        od[i] = x[2 * i + 1];
    }
    fft1d_split(ev, h, sign);
    fft1d_split(od, h, sign);
    for (int k = 0; k < h; ++k) {
        double ang = (double)sign * 2.0 * OR_PI * (double)k / (double)n;
        cplx w = (cos(ang) + I * sin(ang)) * od[k];
        x[k] = ev[k] + w;
        x[k + h] = ev[k] - w;
    }
    free(ev);
    free(od);
}

/* In-place d-dimensional FFT of a row-major [n2][n1][n0] array (n0 fastest). */
int or_fft_nd(int d, const int* n_in, double* data_ri, int sign) {
    int n[3] = {1, 1, 1};
    for (int i = 0; i < d; ++i) n[i] = n_in[i];
    for (int i = 0; i < 3; ++i)
        if (n[i] < 1) return -1;
    cplx* a = (cplx*)data_ri;
    int maxn = n[0] > n[1] ? n[0] : n[1];
    if (n[2] > maxn) maxn = n[2];
    cplx* line = (cplx*)malloc(sizeof(cplx) * (size_t)maxn);
    size_t stride[3] = {1, (size_t)n[0], (size_t)n[0] * n[1]};
    for (int ax = 0; ax < 3; ++ax) {
        if (n[ax] == 1) continue;
        int o1 = (ax + 1) % 3, o2 = (ax + 2) % 3;
        for (int i1 = 0; i1 < n[o1]; ++i1)
            for (int i2 = 0; i2 < n[o2]; ++i2) {
                size_t base = i1 * stride[o1] + i2 * stride[o2];
                for (int t = 0; t < n[ax]; ++t) line[t] = a[base + t * stride[ax]];
                if (is_pow2(n[ax]))
                    fft1d_radix2(line, n[ax], sign);
                else
                    fft1d_split(line, n[ax], sign);
                for (int t = 0; t < n[ax]; ++t) a[base + t * stride[ax]] = line[t];
            }
    }
    free(line);
    return 0;
}

/* Brute-force O(N^2d) DFT, any sizes. */
void or_dft_naive(int d, const int* n_in, const double* in_ri, double* out_ri, int sign) {
    int n[3] = {1, 1, 1};
    for (int i = 0; i < d; ++i) n[i] = n_in[i];
    const cplx* x = (const cplx*)in_ri;
    cplx* X = (cplx*)out_ri;
    for (int a2 = 0; a2 < n[2]; ++a2)
        for (int a1 = 0; a1 < n[1]; ++a1)
            for (int a0 = 0; a0 < n[0]; ++a0) {
                cplx acc = 0;
                for (int m2 = 0; m2 < n[2]; ++m2)
                    for (int m1 = 0; m1 < n[1]; ++m1)
                        for (int m0 = 0; m0 < n[0]; ++m0) {
                            /* phase in turns, each term reduced exactly mod N_i */
                            double turns = (double)((long)a0 * m0 % n[0]) / n[0] +
                                           (double)((long)a1 * m1 % n[1]) / n[1] +
                                           (double)((long)a2 * m2 % n[2]) / n[2];
                            double ang = (double)sign * 2.0 * OR_PI * turns;
                            acc += x[((size_t)m2 * n[1] + m1) * n[0] + m0] * (cos(ang) + I * sin(ang));
                        }
                X[((size_t)a2 * n[1] + a1) * n[0] + a0] = acc;
            }
}

/* ------------------------------------------------------------------------- */
/* phi-functions phi1(z) = (e^z-1)/z, phi2(z) = (e^z-1-z)/z^2 (Sec. II, and  */
/* the small-c remark of Sec. IV read as their exact limits 1 and 1/2).      */
/* ------------------------------------------------------------------------- */
static void phi12(cplx z, cplx* p1, cplx* p2) {
    double az = cabs(z);
    if (cimag(z) == 0.0) {
        double x = creal(z);
        if (x == 0.0) {
            *p1 = 1.0;
            *p2 = 0.5;
            return;
        }
        *p1 = expm1(x) / x;
        if (fabs(x) < 0.5) {
            /* phi2 = sum_{k>=0} x^k / (k+2)! */
            double term = 0.5, sum = 0.0;
            for (int k = 0; k < 30; ++k) {
                sum += term;
                term *= x / (double)(k + 3);
            }
            *p2 = sum;
        } else {
            *p2 = (expm1(x) - x) / (x * x);
        }
        return;
    }
    if (az < 1.0) {
        cplx t1 = 1.0, t2 = 0.5, s1 = 0.0, s2 = 0.0;
        for (int k = 0; k < 40; ++k) {
            s1 += t1;
            s2 += t2;
            t1 *= z / (double)(k + 2);
            t2 *= z / (double)(k + 3);
        }
        *p1 = s1;
        *p2 = s2;
    } else {
        cplx em1 = cexp(z) - 1.0;
        *p1 = em1 / z;
        *p2 = (em1 - z) / (z * z);
    }
}

void or_phi12(double zr, double zi, double out[4]) {
    cplx p1, p2;
    phi12(zr + I * zi, &p1, &p2);
    out[0] = creal(p1);
    out[1] = cimag(p1);
    out[2] = creal(p2);
    out[3] = cimag(p2);
}

/* ------------------------------------------------------------------------- */
/* Configuration and state                                                    */
/* ------------------------------------------------------------------------- */
enum { OR_MODEL_A = 0, OR_MODEL_B = 1, OR_KPZ = 2, OR_CGL = 3, OR_CUSTOM = 4 };
enum { OR_NL_NONE = 0, OR_NL_CUBIC = 1, OR_NL_GRAD2 = 2, OR_NL_CGL = 3 };
enum { OR_EM = 0, OR_SETD1 = 1, OR_SETD2 = 2 };

typedef struct {
    int d;
    int n[3];
    double dx[3];
    int replicas;
    int model;
    double p[8];
    int nl; /* OR_CUSTOM only */
    int complex_field; /* OR_CUSTOM only */
    const double* c_re;
    const double* c_im;
    const double* noise_D;
    const double* nl_re;
    const double* nl_im;
    int scheme;
    double h;
    uint64_t seed;
    int dealias;
    int replica0; /* global index of replica 0: Philox counter word 2 of replica r is replica0 + r */
    int noise_space; /* 0: Fourier-space draw (App. B); 1: real-space draw, then the DFT (Sec. IV step 2) */
} or_config;

typedef struct {
    or_config cfg;
    int nl;
    int cplx_field;
    int n[3]; /* x, y, z with unused = 1 */
    size_t ntot;
    double* tab_c_re;
    double* tab_c_im;
    double* tab_D;
    double* tab_s_re;
    double* tab_s_im;
    size_t ntab;
    cplx* phi;    /* replicas * ntot */
    cplx* fprev;  /* SETD2 */
    int have_fprev;
    int64_t step;
    cplx* snap;   /* two-time mark */
    cplx* dphi;   /* tangent */
    cplx* dfprev;
    cplx* dseed;
    int have_dseed;
    /* scratch */
    cplx* w0;
    cplx* w1;
    cplx* w2;
    cplx* w3;
} or_state;

static void idx3(const or_state* st, size_t idx, int* ix, int* iy, int* iz) {
    *ix = (int)(idx % st->n[0]);
    *iy = (int)((idx / st->n[0]) % st->n[1]);
    *iz = (int)(idx / ((size_t)st->n[0] * st->n[1]));
}
static size_t lin3(const or_state* st, int ix, int iy, int iz) {
    return ((size_t)iz * st->n[1] + iy) * st->n[0] + ix;
}
static int signed_index(int i, int n) { return (2 * i < n) ? i : i - n; }

static double axis_k(const or_state* st, int ax, int i) {
    double L = st->n[ax] * st->cfg.dx[ax];
    return 2.0 * OR_PI * signed_index(i, st->n[ax]) / L;
}
/* k used in odd derivatives: zero at the Nyquist index */
static double axis_k_odd(const or_state* st, int ax, int i) {
    if (st->n[ax] % 2 == 0 && 2 * i == st->n[ax]) return 0.0;
    return axis_k(st, ax, i);
}

static long mode_a2(const or_state* st, size_t idx) {
    int ix, iy, iz;
    idx3(st, idx, &ix, &iy, &iz);
    long ax = signed_index(ix, st->n[0]), ay = signed_index(iy, st->n[1]), az = signed_index(iz, st->n[2]);
    return ax * ax + ay * ay + az * az;
}
static double mode_k2(const or_state* st, size_t idx) {
    int ix, iy, iz;
    idx3(st, idx, &ix, &iy, &iz);
    double kx = axis_k(st, 0, ix), ky = axis_k(st, 1, iy), kz = axis_k(st, 2, iz);
    return kx * kx + ky * ky + kz * kz;
}
/* Dealiasing mask M_a (Sec. IV step 1): dealias = 1 truncates by the 2/3 rule;
 * dealias = 2 (phase-shift dealiasing) keeps every mode but the Nyquist ones,
 * whose shifted copies are not the spectrum of a real field. */
static double mode_mask(const or_state* st, size_t idx) {
    if (!st->cfg.dealias) return 1.0;
    int i3[3];
    idx3(st, idx, &i3[0], &i3[1], &i3[2]);
    for (int ax = 0; ax < 3; ++ax) {
        int a = signed_index(i3[ax], st->n[ax]);
        if (st->n[ax] > 1 && (st->cfg.dealias == 2 ? 2 * abs(a) == st->n[ax] : 3 * abs(a) >= st->n[ax])) return 0.0;
    }
    return 1.0;
}

/* Phase of a shift of the grid by half a cell along the axes in the bit set
 * sigma: e^{+i pi sum_{ax in sigma} a_ax / n_ax}, a_ax the signed index. */
static cplx half_cell_phase(const or_state* st, size_t idx, int sigma) {
    int i3[3];
    idx3(st, idx, &i3[0], &i3[1], &i3[2]);
    double ang = 0.0;
    for (int ax = 0; ax < 3; ++ax)
        if (sigma & (1 << ax)) ang += OR_PI * (double)signed_index(i3[ax], st->n[ax]) / (double)st->n[ax];
    return cos(ang) + I * sin(ang);
}

/* Linear operator c, noise strength D and nonlinear prefactor s of mode idx
 * (Sec. V: Model A/B with Gamma, KPZ, CGL; CUSTOM from |a|^2 tables). */
/* Model A/B with p[4] != 0 place the r phi term in F instead of c (the variant
 * of the Sec. V.A footnote, so that c does not change sign with k^2). */
static int r_in_F(const or_state* st) {
    return (st->cfg.model == OR_MODEL_A || st->cfg.model == OR_MODEL_B) && st->cfg.p[4] != 0.0;
}

static void mode_operator(const or_state* st, size_t idx, cplx* c, double* D, cplx* s) {
    const double* p = st->cfg.p;
    double k2 = mode_k2(st, idx);
    const double r = r_in_F(st) ? 0.0 : p[1];
    switch (st->cfg.model) {
        case OR_MODEL_A: /* p = Gamma, r, u, T[, r in F] */
            *c = -p[0] * (r + k2);
            *D = p[0] * p[3];
            *s = -p[0] * p[2];
            break;
        case OR_MODEL_B:
            *c = -p[0] * k2 * (r + k2);
            *D = p[0] * p[3] * k2;
            *s = -p[0] * p[2] * k2;
            break;
        case OR_KPZ: /* p = nu, lambda, D */
            *c = -p[0] * k2;
            *D = p[2];
            *s = 0.5 * p[1];
            break;
        case OR_CGL: /* p = alpha, beta, eps: c = 1 - (1 + i alpha) k^2, s = -(1 + i beta) */
            *c = 1.0 - (1.0 + I * p[0]) * k2;
            *D = p[2];
            *s = -(1.0 + I * p[1]);
            break;
        default: {
            long q = mode_a2(st, idx);
            *c = st->tab_c_re[q] + I * (st->tab_c_im ? st->tab_c_im[q] : 0.0);
            *D = st->tab_D[q];
            *s = (st->tab_s_re ? st->tab_s_re[q] : 0.0) + I * (st->tab_s_im ? st->tab_s_im[q] : 0.0);
        }
    }
}

static double noise_norm(const or_state* st) {
    /* (N^2/L)^{d/2} = prod_i sqrt(N_i / dx_i)   (App. A) */
    double v = 1.0;
    for (int ax = 0; ax < st->cfg.d; ++ax) v *= sqrt(st->n[ax] / st->cfg.dx[ax]);
    return v;
}

/* SETD coefficients of one mode (Sec. II and the boxed algorithm of Sec. IV):
 *   phi <- f1 phi + a F + b F_prev + g eta */
static void mode_coefs(const or_state* st, size_t idx, int first_step, cplx* f1, cplx* a, cplx* b, cplx* g) {
    cplx c, s;
    double D;
    mode_operator(st, idx, &c, &D, &s);
    double h = st->cfg.h;
    cplx z = c * h;
    cplx p1, p2;
    phi12(z, &p1, &p2);
    *f1 = cexp(z);
    double nf = noise_norm(st);
    int scheme = st->cfg.scheme;
    if (scheme == OR_EM) {
        *a = h * p1;
        *b = 0.0;
        *g = nf * sqrt(2.0 * D * h) * cexp(0.5 * z); /* f3 G dW, dW = sqrt(h) N(0,1) */
        return;
    }
    cplx q1, q2;
    phi12(2.0 * creal(z), &q1, &q2);
    *g = nf * sqrt(2.0 * D * h * creal(q1)); /* f4 G, exact I1 variance */
    if (scheme == OR_SETD1 || first_step) {
        *a = h * p1;
        *b = 0.0;
    } else {
        *a = h * (p1 + p2);
        *b = -h * p2;
    }
}

void or_mode_coefs(const or_state* st, size_t idx, int first_step, double out[8]) {
    cplx f1, a, b, g;
    mode_coefs(st, idx, first_step, &f1, &a, &b, &g);
    out[0] = creal(f1); out[1] = cimag(f1);
    out[2] = creal(a); out[3] = cimag(a);
    out[4] = creal(b); out[5] = cimag(b);
    out[6] = creal(g); out[7] = cimag(g);
}

/* Hermitian classification for real fields (App. B).
 * Stored half: ix in [0, nx/2].  Off the planes ix in {0, nx/2} every stored
 * mode is canonical.  On those planes the mode is canonical when its (iz, iy)
 * tuple is lexicographically below that of its negative, self-conjugate when
 * equal.  Modes with ix > nx/2 are partners.
 * Returns 0 canonical, 1 self-conjugate, 2 partner. */
static int herm_class(const or_state* st, size_t idx) {
    int ix, iy, iz;
    idx3(st, idx, &ix, &iy, &iz);
    int nx = st->n[0];
    if (2 * ix > nx) return 2;
    if (ix != 0 && 2 * ix != nx) return 0;
    int miz = (st->n[2] - iz) % st->n[2];
    int miy = (st->n[1] - iy) % st->n[1];
    if (iz < miz || (iz == miz && iy < miy)) return 0;
    if (iz == miz && iy == miy) return 1;
    return 2;
}
static size_t neg_index(const or_state* st, size_t idx) {
    int ix, iy, iz;
    idx3(st, idx, &ix, &iy, &iz);
    return lin3(st, (st->n[0] - ix) % st->n[0], (st->n[1] - iy) % st->n[1], (st->n[2] - iz) % st->n[2]);
}

static void hermitian_fixup(const or_state* st, cplx* phi) {
    if (st->cplx_field) return;
    for (size_t i = 0; i < st->ntot; ++i) {
        int cl = herm_class(st, i);
        if (cl == 1) phi[i] = creal(phi[i]);
    }
    for (size_t i = 0; i < st->ntot; ++i)
        if (herm_class(st, i) == 2) phi[i] = conj(phi[neg_index(st, i)]);
}

/* Noise counter index of a stored mode: x-major enumeration
 *   j = (ix * nz + iz) * ny + iy. */
static uint64_t noise_index(const or_state* st, size_t idx) {
    int ix, iy, iz;
    idx3(st, idx, &ix, &iy, &iz);
    return ((uint64_t)ix * st->n[2] + iz) * st->n[1] + iy;
}

/* Fourier-space noise eta_a of one replica at one step (App. B):
 * canonical complex modes (A + iB), A, B ~ N(0, 1/2); self-conjugate modes real
 * N(0, 1); partners conjugate.  Complex fields: every mode complex. */
static void draw_noise(const or_state* st, int replica, int64_t step, cplx* eta) {
    const double inv_sqrt2 = 0.70710678118654752440;
    for (size_t i = 0; i < st->ntot; ++i) {
        int cl = st->cplx_field ? 0 : herm_class(st, i);
        if (cl == 2) continue;
        uint64_t j = noise_index(st, i);
        float z[4];
        normals_for_index(st->cfg.seed, (uint32_t)(j >> 1), (uint32_t)step, (uint32_t)(st->cfg.replica0 + replica),
                          0u, z);
        int o = (int)(j & 1) * 2;
        if (cl == 1)
            eta[i] = (double)z[o];
        else
            eta[i] = ((double)z[o] + I * (double)z[o + 1]) * inv_sqrt2;
    }
    if (!st->cplx_field)
        for (size_t i = 0; i < st->ntot; ++i)
            if (herm_class(st, i) == 2) eta[i] = conj(eta[neg_index(st, i)]);
}

/* Real-space noise of one replica at one step (the alternative of Sec. IV
 * step 2): eta(x) iid N(0, 1) per site -- site s = lin3(x) takes normal s & 3 of
 * Philox tag 3, counter (s / 4, step, replica, 3) -- and eta_a = DFT[eta]_a / sqrt(N).
 * The DFT of a real field is Hermitian; the self-conjugate modes are real
 * N(0, 1) and every other mode has E|eta_a|^2 = 1, as in the Fourier draw. */
static void fft_full(const or_state* st, cplx* a, int sign);
static void draw_noise_real(const or_state* st, int replica, int64_t step, cplx* eta) {
    for (size_t s = 0; s < st->ntot; ++s) {
        float z[4];
        normals_for_index(st->cfg.seed, (uint32_t)(s >> 2), (uint32_t)step, (uint32_t)(st->cfg.replica0 + replica),
                          3u, z);
        eta[s] = (double)z[s & 3];
    }
    fft_full(st, eta, -1);
    const double inv_sqrt_n = 1.0 / sqrt((double)st->ntot);
    for (size_t i = 0; i < st->ntot; ++i) eta[i] *= inv_sqrt_n;
    hermitian_fixup(st, eta);
}

int or_noise(const or_state* st, int replica, int64_t step, double* eta_ri) {
    if (st->cfg.noise_space)
        draw_noise_real(st, replica, step, (cplx*)eta_ri);
    else
        draw_noise(st, replica, step, (cplx*)eta_ri);
    return 0;
}

static size_t tab_len(const or_config* cfg) {
    long q = 0;
    for (int ax = 0; ax < cfg->d; ++ax) q += (long)(cfg->n[ax] / 2) * (cfg->n[ax] / 2);
    return (size_t)q + 1;
}

or_state* or_create(const or_config* cfg) {
    if (cfg->d < 1 || cfg->d > 3 || cfg->replicas < 1 || !(cfg->h > 0) || cfg->dealias < 0 || cfg->dealias > 2 ||
        cfg->noise_space < 0 || cfg->noise_space > 1)
        return NULL;
    or_state* st = (or_state*)calloc(1, sizeof(or_state));
    st->cfg = *cfg;
    st->n[0] = st->n[1] = st->n[2] = 1;
    for (int ax = 0; ax < cfg->d; ++ax) {
        if (cfg->n[ax] < 1 || (cfg->n[ax] > 1 && cfg->n[ax] % 2) || !(cfg->dx[ax] > 0)) {  /* 1 or even */
            free(st);
            return NULL;
        }
        st->n[ax] = cfg->n[ax];
    }
    for (int ax = cfg->d; ax < 3; ++ax) st->cfg.dx[ax] = 1.0;
    st->ntot = (size_t)st->n[0] * st->n[1] * st->n[2];
    switch (cfg->model) {
        case OR_MODEL_A: case OR_MODEL_B: st->nl = OR_NL_CUBIC; st->cplx_field = 0; break;
        case OR_KPZ: st->nl = OR_NL_GRAD2; st->cplx_field = 0; break;
        case OR_CGL: st->nl = OR_NL_CGL; st->cplx_field = 1; break;
        default:
            st->nl = cfg->nl;
            st->cplx_field = cfg->complex_field;
            st->ntab = tab_len(cfg);
            st->tab_c_re = (double*)calloc(st->ntab, sizeof(double));
            st->tab_c_im = (double*)calloc(st->ntab, sizeof(double));
            st->tab_D = (double*)calloc(st->ntab, sizeof(double));
            st->tab_s_re = (double*)calloc(st->ntab, sizeof(double));
            st->tab_s_im = (double*)calloc(st->ntab, sizeof(double));
            for (size_t q = 0; q < st->ntab; ++q) {
                st->tab_c_re[q] = cfg->c_re ? cfg->c_re[q] : 0.0;
                st->tab_c_im[q] = cfg->c_im ? cfg->c_im[q] : 0.0;
                st->tab_D[q] = cfg->noise_D ? cfg->noise_D[q] : 0.0;
                st->tab_s_re[q] = cfg->nl_re ? cfg->nl_re[q] : 0.0;
                st->tab_s_im[q] = cfg->nl_im ? cfg->nl_im[q] : 0.0;
            }
            st->cfg.c_re = st->cfg.c_im = st->cfg.noise_D = st->cfg.nl_re = st->cfg.nl_im = NULL;
    }
    size_t tot = st->ntot * (size_t)cfg->replicas;
    st->phi = (cplx*)calloc(tot, sizeof(cplx));
    st->fprev = (cplx*)calloc(tot, sizeof(cplx));
    st->snap = (cplx*)calloc(tot, sizeof(cplx));
    st->dphi = (cplx*)calloc(tot, sizeof(cplx));
    st->dfprev = (cplx*)calloc(tot, sizeof(cplx));
    st->dseed = (cplx*)calloc(tot, sizeof(cplx));
    st->w0 = (cplx*)calloc(st->ntot, sizeof(cplx));
    st->w1 = (cplx*)calloc(st->ntot, sizeof(cplx));
    st->w2 = (cplx*)calloc(st->ntot, sizeof(cplx));
    st->w3 = (cplx*)calloc(st->ntot, sizeof(cplx));
    return st;
}

void or_destroy(or_state* st) {
    if (!st) return;
    free(st->tab_c_re); free(st->tab_c_im); free(st->tab_D); free(st->tab_s_re); free(st->tab_s_im);
    free(st->phi); free(st->fprev); free(st->snap); free(st->dphi); free(st->dfprev); free(st->dseed);
    free(st->w0); free(st->w1); free(st->w2); free(st->w3);
    free(st);
}

size_t or_ntot(const or_state* st) { return st->ntot; }
int64_t or_get_step(const or_state* st) { return st->step; }
void or_set_step(or_state* st, int64_t s) { st->step = s; }

static void fft_full(const or_state* st, cplx* a, int sign) { or_fft_nd(3, st->n, (double*)a, sign); }

/* Real-space field (real: ntot doubles; complex: ntot pairs) -> spectrum. */
int or_set_field(or_state* st, int replica, const double* field) {
    cplx* phi = st->phi + (size_t)replica * st->ntot;
    for (size_t i = 0; i < st->ntot; ++i)
        phi[i] = st->cplx_field ? field[2 * i] + I * field[2 * i + 1] : field[i];
    fft_full(st, phi, -1);
    hermitian_fixup(st, phi);
    st->have_fprev = 0;
    return 0;
}

int or_get_field(const or_state* st, int replica, double* out) {
    cplx* w = st->w0;
    memcpy(w, st->phi + (size_t)replica * st->ntot, st->ntot * sizeof(cplx));
    fft_full(st, w, +1);
    for (size_t i = 0; i < st->ntot; ++i) {
        cplx v = w[i] / (double)st->ntot;
        if (st->cplx_field) {
            out[2 * i] = creal(v);
            out[2 * i + 1] = cimag(v);
        } else {
            out[i] = creal(v);
        }
    }
    return 0;
}

int or_get_spectrum(const or_state* st, int replica, double* out_ri) {
    memcpy(out_ri, st->phi + (size_t)replica * st->ntot, st->ntot * sizeof(cplx));
    return 0;
}
int or_set_spectrum(or_state* st, int replica, const double* in_ri) {
    memcpy(st->phi + (size_t)replica * st->ntot, in_ri, st->ntot * sizeof(cplx));
    return 0;
}
int or_get_fprev(const or_state* st, int replica, double* out_ri) {
    memcpy(out_ri, st->fprev + (size_t)replica * st->ntot, st->ntot * sizeof(cplx));
    return st->have_fprev;
}

/* Initial condition: iid N(0, sigma^2) per real-space site (complex fields:
 * sigma (N(0,1) + i N(0,1))), Philox tag 1, counter word 0 = site / 4 (real)
 * or site / 2 (complex), then the forward transform. */
int or_init_random(or_state* st, double sigma) {
    double* buf = (double*)malloc(sizeof(double) * 2 * st->ntot);
    for (int r = 0; r < st->cfg.replicas; ++r) {
        for (size_t s = 0; s < st->ntot; ++s) {
            float z[4];
            if (st->cplx_field) {
                normals_for_index(st->cfg.seed, (uint32_t)(s >> 1), 0u, (uint32_t)(st->cfg.replica0 + r), 1u, z);
                int o = (int)(s & 1) * 2;
                buf[2 * s] = sigma * (double)z[o];
                buf[2 * s + 1] = sigma * (double)z[o + 1];
            } else {
                normals_for_index(st->cfg.seed, (uint32_t)(s >> 2), 0u, (uint32_t)(st->cfg.replica0 + r), 1u, z);
                buf[s] = sigma * (double)z[s & 3];
            }
        }
        or_set_field(st, r, buf);
    }
    free(buf);
    return 0;
}

/* DFT of the real-space nonlinearity q of the masked state, evaluated on the
 * grid shifted by half a cell along the axes in sigma (sigma = 0: the plain
 * grid): P = M phi e^{i pi sigma.a/N}, psi = IDFT(P), Q_a = DFT[q(psi)]_a
 * e^{-i pi sigma.a/N} (Sec. IV step 1, Sec. V model terms). */
static void nonlinear_dft(or_state* st, const cplx* phi, int sigma, cplx* q) {
    size_t nt = st->ntot;
    cplx* g = st->w2;
    if (st->nl == OR_NL_GRAD2) {
        memset(q, 0, nt * sizeof(cplx));
        for (int ax = 0; ax < st->cfg.d; ++ax) {
            for (size_t i = 0; i < nt; ++i) {
                int i3[3];
                idx3(st, i, &i3[0], &i3[1], &i3[2]);
                g[i] = I * axis_k_odd(st, ax, i3[ax]) * mode_mask(st, i) * phi[i];
                if (sigma) g[i] *= half_cell_phase(st, i, sigma);
            }
            fft_full(st, g, +1);
            for (size_t i = 0; i < nt; ++i) {
                double gr = creal(g[i]) / (double)nt;
                q[i] += gr * gr;
            }
        }
    } else {
        for (size_t i = 0; i < nt; ++i) q[i] = mode_mask(st, i) * phi[i] * (sigma ? half_cell_phase(st, i, sigma) : 1.0);
        fft_full(st, q, +1);
        for (size_t i = 0; i < nt; ++i) {
            cplx v = q[i] / (double)nt;
            if (st->nl == OR_NL_CUBIC) {
                double p = creal(v);
                q[i] = p * p * p;
            } else { /* CGL: |A|^2 A */
                q[i] = (creal(v) * creal(v) + cimag(v) * cimag(v)) * v;
            }
        }
    }
    fft_full(st, q, -1);
    if (sigma)
        for (size_t i = 0; i < nt; ++i) q[i] *= conj(half_cell_phase(st, i, sigma));
}

/* F_a = M_a s_a Q_a, with Q the plain DFT of q (dealias 0 or 1) or, for
 * phase-shift dealiasing (dealias = 2), the mean of Q over the 2^d grids
 * shifted by half a cell along every subset of the axes: on a grid shifted
 * along ax, the alias of output mode a from input modes with
 * a_1 + a_2 + a_3 = a + j N carries the factor (-1)^{j_ax}, so the mean keeps
 * only the terms whose j has every component even (phase shifts after
 * Rogallo, cited in Sec. IV step 1). */
static void nonlinear_term(or_state* st, const cplx* phi, cplx* F) {
    size_t nt = st->ntot;
    cplx* q = st->w1;
    if (st->nl == OR_NL_NONE) {
        memset(q, 0, nt * sizeof(cplx));
    } else if (st->cfg.dealias == 2) {
        cplx* acc = st->w0;  /* free here: the noise is drawn after the force */
        memset(acc, 0, nt * sizeof(cplx));
        const int nshift = 1 << st->cfg.d;
        for (int sigma = 0; sigma < nshift; ++sigma) {
            nonlinear_dft(st, phi, sigma, q);
            for (size_t i = 0; i < nt; ++i) acc[i] += q[i] / (double)nshift;
        }
        memcpy(q, acc, nt * sizeof(cplx));
    } else {
        nonlinear_dft(st, phi, 0, q);
    }
    for (size_t i = 0; i < nt; ++i) {
        cplx c, s;
        double D;
        mode_operator(st, i, &c, &D, &s);
        F[i] = mode_mask(st, i) * s * q[i];
        if (r_in_F(st)) /* the linear term -Gamma r k^Delta phi, no dealiasing needed */
            F[i] += -st->cfg.p[0] * st->cfg.p[1] * (st->cfg.model == OR_MODEL_B ? mode_k2(st, i) : 1.0) * phi[i];
    }
}

/* One SETD step of one replica (boxed algorithm of Sec. IV). */
static void step_replica(or_state* st, int r, int first) {
    size_t nt = st->ntot;
    cplx* phi = st->phi + (size_t)r * nt;
    cplx* fprev = st->fprev + (size_t)r * nt;
    cplx* F = st->w3;
    nonlinear_term(st, phi, F);
    cplx* eta = st->w0;
    if (st->cfg.noise_space)
        draw_noise_real(st, r, st->step, eta);
    else
        draw_noise(st, r, st->step, eta);
    for (size_t i = 0; i < nt; ++i) {
        cplx f1, a, b, g;
        mode_coefs(st, i, first, &f1, &a, &b, &g);
        phi[i] = f1 * phi[i] + a * F[i] + b * fprev[i] + g * eta[i];
    }
    hermitian_fixup(st, phi);
    memcpy(fprev, F, nt * sizeof(cplx));
}

int or_step(or_state* st, int64_t nsteps) {
    for (int64_t t = 0; t < nsteps; ++t) {
        int first = (st->cfg.scheme == OR_SETD2) && !st->have_fprev;
        for (int r = 0; r < st->cfg.replicas; ++r) step_replica(st, r, first);
        st->have_fprev = 1;
        st->step++;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Observables (App. C)                                                      */
/* ------------------------------------------------------------------------- */
static long isqrt_ceil(long q) {
    long j = (long)floor(sqrt((double)q));
    while (j * j < q) ++j;
    while (j > 0 && (j - 1) * (j - 1) >= q) --j;
    return j;
}

int or_nshells(const or_state* st) {
    long q = 0;
    for (int ax = 0; ax < st->cfg.d; ++ax) q += (long)(st->n[ax] / 2) * (st->n[ax] / 2);
    return (int)isqrt_ceil(q) + 1;
}

static double ct_norm(const or_state* st) {
    /* (L/N^2)^d = prod_i dx_i / N_i */
    double v = 1.0;
    for (int ax = 0; ax < st->cfg.d; ++ax) v *= st->cfg.dx[ax] / st->n[ax];
    return v;
}

/* Shell of mode: j = ceil(|a|), so that k_j - dk < |k| <= k_j (App. C). */
static int shell_of(const or_state* st, size_t idx) { return (int)isqrt_ceil(mode_a2(st, idx)); }

/* kind 0: C_ET shell average of (L/N^2)^d |phi_a|^2, replica-averaged.
 * kind 1: two-time shell average of (L/N^2)^d Re(phi_a(t) conj(phi_a(t0))).
 * counts receives N_k. */
int or_observe_shells(const or_state* st, int kind, double* out, double* counts) {
    int ns = or_nshells(st);
    for (int j = 0; j < ns; ++j) out[j] = counts[j] = 0.0;
    double nrm = ct_norm(st);
    for (size_t i = 0; i < st->ntot; ++i) counts[shell_of(st, i)] += 1.0;
    for (int r = 0; r < st->cfg.replicas; ++r) {
        const cplx* phi = st->phi + (size_t)r * st->ntot;
        const cplx* snap = st->snap + (size_t)r * st->ntot;
        for (size_t i = 0; i < st->ntot; ++i) {
            double v = kind == 0 ? creal(phi[i] * conj(phi[i])) : creal(phi[i] * conj(snap[i]));
            out[shell_of(st, i)] += nrm * v;
        }
    }
    for (int j = 0; j < ns; ++j)
        if (counts[j] > 0) out[j] /= counts[j] * st->cfg.replicas;
    return ns;
}

int or_mark(or_state* st) {
    memcpy(st->snap, st->phi, st->ntot * (size_t)st->cfg.replicas * sizeof(cplx));
    return 0;
}

/* KPZ width squared per replica, w^2 = N^{-2d} sum_{a != 0} |phi_a|^2
 * (Sec. V.B with the box equal to the whole system; Parseval). */
int or_roughness(const or_state* st, double* out) {
    double n2 = (double)st->ntot * (double)st->ntot;
    for (int r = 0; r < st->cfg.replicas; ++r) {
        const cplx* phi = st->phi + (size_t)r * st->ntot;
        double acc = 0.0;
        for (size_t i = 1; i < st->ntot; ++i) acc += creal(phi[i] * conj(phi[i]));
        out[r] = acc / n2;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Tangent (forward-mode linearisation) of the step, advanced together with   */
/* the primal on the same noise path.  dF = M s DFT[dq] with                  */
/*   cubic: dq = 3 psi^2 dpsi;  KPZ: dq = 2 sum_j g_j dg_j;                    */
/*   CGL: dq = 2 |A|^2 dA + A^2 conj(dA).                                     */
/* ------------------------------------------------------------------------- */
static void tangent_term(or_state* st, const cplx* phi, const cplx* dphi, cplx* dF) {
    size_t nt = st->ntot;
    cplx* psi = (cplx*)malloc(nt * sizeof(cplx));
    cplx* dpsi = (cplx*)malloc(nt * sizeof(cplx));
    cplx* dq = (cplx*)calloc(nt, sizeof(cplx));
    if (st->nl == OR_NL_GRAD2) {
        for (int ax = 0; ax < st->cfg.d; ++ax) {
            for (size_t i = 0; i < nt; ++i) {
                int i3[3];
                idx3(st, i, &i3[0], &i3[1], &i3[2]);
                cplx ik = I * axis_k_odd(st, ax, i3[ax]) * mode_mask(st, i);
                psi[i] = ik * phi[i];
                dpsi[i] = ik * dphi[i];
            }
            fft_full(st, psi, +1);
            fft_full(st, dpsi, +1);
            for (size_t i = 0; i < nt; ++i) dq[i] += 2.0 * (creal(psi[i]) / nt) * (creal(dpsi[i]) / nt);
        }
    } else if (st->nl != OR_NL_NONE) {
        for (size_t i = 0; i < nt; ++i) {
            psi[i] = mode_mask(st, i) * phi[i];
            dpsi[i] = mode_mask(st, i) * dphi[i];
        }
        fft_full(st, psi, +1);
        fft_full(st, dpsi, +1);
        for (size_t i = 0; i < nt; ++i) {
            cplx v = psi[i] / (double)nt, dv = dpsi[i] / (double)nt;
            if (st->nl == OR_NL_CUBIC)
                dq[i] = 3.0 * creal(v) * creal(v) * creal(dv);
            else
                dq[i] = 2.0 * (creal(v) * creal(v) + cimag(v) * cimag(v)) * dv + v * v * conj(dv);
        }
    }
    fft_full(st, dq, -1);
    for (size_t i = 0; i < nt; ++i) {
        cplx c, s;
        double D;
        mode_operator(st, i, &c, &D, &s);
        dF[i] = mode_mask(st, i) * s * dq[i];
    }
    free(psi);
    free(dpsi);
    free(dq);
}

/* dphi0: real-space tangent seed (replicas x field), or NULL to continue. */
int or_tangent_step(or_state* st, const double* dphi0, int64_t nsteps, double* dphi_out) {
    if (st->cfg.dealias == 2) return -1; /* linearised about the truncated nonlinear term only */
    size_t nt = st->ntot;
    int R = st->cfg.replicas;
    if (dphi0) {
        for (int r = 0; r < R; ++r) {
            cplx* d = st->dphi + (size_t)r * nt;
            for (size_t i = 0; i < nt; ++i)
                d[i] = st->cplx_field ? dphi0[(size_t)r * 2 * nt + 2 * i] + I * dphi0[(size_t)r * 2 * nt + 2 * i + 1]
                                      : dphi0[(size_t)r * nt + i];
            fft_full(st, d, -1);
            hermitian_fixup(st, d);
            memset(st->dfprev + (size_t)r * nt, 0, nt * sizeof(cplx));
        }
        memcpy(st->dseed, st->dphi, nt * (size_t)R * sizeof(cplx));
        st->have_dseed = 1;
    }
    cplx* dF = (cplx*)malloc(nt * sizeof(cplx));
    for (int64_t t = 0; t < nsteps; ++t) {
        int first = (st->cfg.scheme == OR_SETD2) && !st->have_fprev;
        for (int r = 0; r < R; ++r) {
            cplx* phi = st->phi + (size_t)r * nt;
            cplx* dphi = st->dphi + (size_t)r * nt;
            cplx* dfp = st->dfprev + (size_t)r * nt;
            tangent_term(st, phi, dphi, dF);
            for (size_t i = 0; i < nt; ++i) {
                cplx f1, a, b, g;
                mode_coefs(st, i, first, &f1, &a, &b, &g);
                dphi[i] = f1 * dphi[i] + a * dF[i] + b * dfp[i];
            }
            hermitian_fixup(st, dphi);
            memcpy(dfp, dF, nt * sizeof(cplx));
            step_replica(st, r, first);
        }
        st->have_fprev = 1;
        st->step++;
    }
    free(dF);
    if (dphi_out) {
        cplx* w = (cplx*)malloc(nt * sizeof(cplx));
        for (int r = 0; r < R; ++r) {
            memcpy(w, st->dphi + (size_t)r * nt, nt * sizeof(cplx));
            fft_full(st, w, +1);
            for (size_t i = 0; i < nt; ++i) {
                cplx v = w[i] / (double)nt;
                if (st->cplx_field) {
                    dphi_out[(size_t)r * 2 * nt + 2 * i] = creal(v);
                    dphi_out[(size_t)r * 2 * nt + 2 * i + 1] = cimag(v);
                } else {
                    dphi_out[(size_t)r * nt + i] = creal(v);
                }
            }
        }
        free(w);
    }
    return 0;
}

int or_get_tangent_spectrum(const or_state* st, int replica, double* out_ri) {
    memcpy(out_ri, st->dphi + (size_t)replica * st->ntot, st->ntot * sizeof(cplx));
    return 0;
}

/* Linear response per shell: sum Re(dphi_a(t) conj(dphi_a(t0))) / sum |dphi_a(t0)|^2,
 * summed over replicas, for shells where the seed has weight. */
int or_observe_response(const or_state* st, double* out) {
    int ns = or_nshells(st);
    double* den = (double*)calloc((size_t)ns, sizeof(double));
    for (int j = 0; j < ns; ++j) out[j] = 0.0;
    for (int r = 0; r < st->cfg.replicas; ++r) {
        const cplx* d = st->dphi + (size_t)r * st->ntot;
        const cplx* s = st->dseed + (size_t)r * st->ntot;
        for (size_t i = 0; i < st->ntot; ++i) {
            int j = shell_of(st, i);
            out[j] += creal(d[i] * conj(s[i]));
            den[j] += creal(s[i] * conj(s[i]));
        }
    }
    for (int j = 0; j < ns; ++j) out[j] = den[j] > 0 ? out[j] / den[j] : 0.0;
    free(den);
    return ns;
}

/* ------------------------------------------------------------------------- */
/* Adjoint (transpose of the tangent with respect to the real-space inner    */
/* product sum_x u(x) v(x)), real fields.  With C(m) the real-space Fourier  */
/* multiplier by m (symmetric when m is real and even) and L_n = C(M s) D(q'_n) */
/* C(M) the linearised nonlinear term of step n, the tangent of Eq. SETD2 is  */
/*   dF_n = L_n dphi_n,  dphi_{n+1} = f1 dphi_n + a_n dF_n + b_n dF_{n-1}     */
/* (dF_{-1} = 0 at the seed; SETD-EM and SETD1 have b = 0).  Its transpose    */
/* runs backward from the cotangent lam_N of dphi_N with mu_{N-1} = 0:        */
/*   nu_n = a_n lam_{n+1} + mu_n          (the cotangent of dF_n),            */
/*   lam_n = f1 lam_{n+1} + L_n^T nu_n,   L_n^T = C(M) D(q'_n) C(M s),        */
/*   mu_{n-1} = b_n lam_{n+1},                                                */
/* with the SETD1 pair at the step that starts SETD2 (no F_{-1} exists).  For */
/* KPZ the gradient multiplier i k is odd, so its transpose is -i k.          */
/* Complex fields (CGL, Sec. V.C) take the real inner product                 */
/* Re sum_x conj(u(x)) v(x); every Fourier multiplier m then transposes to    */
/* conj(m) (f1, a, b and the prefactor s are complex), and the pointwise      */
/* linearisation dA -> 2 |A|^2 dA + A^2 conj(dA) of |A|^2 A is its own        */
/* transpose, so L_n^T = C(M) D(q'_n) C(conj(M s)).                           */
/* ------------------------------------------------------------------------- */
int or_adjoint(or_state* st, const double* lam_in, int64_t nsteps, double* grad_out) {
    if (st->cfg.dealias == 2) return -1;
    if (st->cplx_field && st->nl != OR_NL_CGL && st->nl != OR_NL_NONE) return -1;
    const int cf = st->cplx_field;
    size_t nt = st->ntot;
    int R = st->cfg.replicas;
    cplx* traj = (cplx*)malloc(nt * (size_t)R * (size_t)(nsteps > 0 ? nsteps : 1) * sizeof(cplx));
    /* step t of the recorded trajectory used the SETD1 pair if it started the SETD2 history */
    int* first_of = (int*)calloc((size_t)(nsteps > 0 ? nsteps : 1), sizeof(int));
    for (int64_t t = 0; t < nsteps; ++t) {
        memcpy(traj + (size_t)t * nt * R, st->phi, nt * (size_t)R * sizeof(cplx));
        first_of[t] = (st->cfg.scheme == OR_SETD2) && !st->have_fprev;
        or_step(st, 1);
    }
    cplx* lam = (cplx*)malloc(nt * sizeof(cplx));
    cplx* mu = (cplx*)malloc(nt * sizeof(cplx));
    cplx* w = (cplx*)malloc(nt * sizeof(cplx));
    cplx* g = (cplx*)malloc(nt * sizeof(cplx));
    cplx* acc = (cplx*)malloc(nt * sizeof(cplx));
    for (int r = 0; r < R; ++r) {
        for (size_t i = 0; i < nt; ++i) {
            lam[i] = cf ? lam_in[2 * ((size_t)r * nt + i)] + I * lam_in[2 * ((size_t)r * nt + i) + 1]
                        : lam_in[(size_t)r * nt + i];
            mu[i] = 0.0;
        }
        fft_full(st, lam, -1);
        hermitian_fixup(st, lam);
        for (int64_t t = nsteps - 1; t >= 0; --t) {
            const cplx* phi = traj + (size_t)t * nt * R + (size_t)r * nt;
            /* W = IDFT(M s nu), nu = a lam + mu; then mu <- b lam (lam of step t + 1) */
            for (size_t i = 0; i < nt; ++i) {
                cplx f1, a, b, gg, c, s;
                double D;
                mode_coefs(st, i, first_of[t], &f1, &a, &b, &gg);
                mode_operator(st, i, &c, &D, &s);
                w[i] = mode_mask(st, i) * conj(s) * (conj(a) * lam[i] + mu[i]);
                mu[i] = conj(b) * lam[i];
            }
            fft_full(st, w, +1);
            for (size_t i = 0; i < nt; ++i) w[i] = (cf ? w[i] : creal(w[i])) / (double)nt;
            for (size_t i = 0; i < nt; ++i) acc[i] = 0.0;
            if (st->nl == OR_NL_CGL) {
                /* q' = 2 |A|^2 w + A^2 conj(w), A = IDFT(M phi) */
                for (size_t i = 0; i < nt; ++i) g[i] = mode_mask(st, i) * phi[i];
                fft_full(st, g, +1);
                for (size_t i = 0; i < nt; ++i) {
                    const cplx A = g[i] / (double)nt;
                    g[i] = 2.0 * (creal(A) * creal(A) + cimag(A) * cimag(A)) * w[i] + A * A * conj(w[i]);
                }
                fft_full(st, g, -1);
                for (size_t i = 0; i < nt; ++i) acc[i] = mode_mask(st, i) * g[i];
            } else if (st->nl == OR_NL_CUBIC) {
                for (size_t i = 0; i < nt; ++i) g[i] = mode_mask(st, i) * phi[i];
                fft_full(st, g, +1);
                for (size_t i = 0; i < nt; ++i) {
                    double p = creal(g[i]) / (double)nt;
                    g[i] = 3.0 * p * p * creal(w[i]);
                }
                fft_full(st, g, -1);
                for (size_t i = 0; i < nt; ++i) acc[i] = mode_mask(st, i) * g[i];
            } else if (st->nl == OR_NL_GRAD2) {
                cplx* v = (cplx*)malloc(nt * sizeof(cplx));
                for (int ax = 0; ax < st->cfg.d; ++ax) {
                    for (size_t i = 0; i < nt; ++i) {
                        int i3[3];
                        idx3(st, i, &i3[0], &i3[1], &i3[2]);
                        g[i] = I * axis_k_odd(st, ax, i3[ax]) * mode_mask(st, i) * phi[i];
                    }
                    fft_full(st, g, +1);
                    for (size_t i = 0; i < nt; ++i) v[i] = 2.0 * (creal(g[i]) / (double)nt) * creal(w[i]);
                    fft_full(st, v, -1);
                    for (size_t i = 0; i < nt; ++i) {
                        int i3[3];
                        idx3(st, i, &i3[0], &i3[1], &i3[2]);
                        acc[i] += -I * axis_k_odd(st, ax, i3[ax]) * mode_mask(st, i) * v[i];
                    }
                }
                free(v);
            }
            for (size_t i = 0; i < nt; ++i) {
                cplx f1, a, b, gg;
                mode_coefs(st, i, first_of[t], &f1, &a, &b, &gg);
                lam[i] = conj(f1) * lam[i] + acc[i];
            }
            hermitian_fixup(st, lam);
            hermitian_fixup(st, mu);
        }
        memcpy(w, lam, nt * sizeof(cplx));
        fft_full(st, w, +1);
        for (size_t i = 0; i < nt; ++i) {
            const cplx v = w[i] / (double)nt;
            if (cf) {
                grad_out[2 * ((size_t)r * nt + i)] = creal(v);
                grad_out[2 * ((size_t)r * nt + i) + 1] = cimag(v);
            } else {
                grad_out[(size_t)r * nt + i] = creal(v);
            }
        }
    }
    free(traj);
    free(first_of);
    free(mu);
    free(lam);
    free(w);
    free(g);
    free(acc);
    return 0;
}

/* One step of every replica with caller-supplied Fourier noise (replicas x
 * full spectrum) instead of the Philox draw; used to build coarse noise paths
 * from fine ones in the strong-convergence study (Sec. III). */
int or_step_noise(or_state* st, const double* eta_ri) {
    size_t nt = st->ntot;
    int first = (st->cfg.scheme == OR_SETD2) && !st->have_fprev;
    const cplx* eta_all = (const cplx*)eta_ri;
    for (int r = 0; r < st->cfg.replicas; ++r) {
        cplx* phi = st->phi + (size_t)r * nt;
        cplx* fprev = st->fprev + (size_t)r * nt;
        cplx* F = st->w3;
        nonlinear_term(st, phi, F);
        const cplx* eta = eta_all + (size_t)r * nt;
        for (size_t i = 0; i < nt; ++i) {
            cplx f1, a, b, g;
            mode_coefs(st, i, first, &f1, &a, &b, &g);
            phi[i] = f1 * phi[i] + a * F[i] + b * fprev[i] + g * eta[i];
        }
        hermitian_fixup(st, phi);
        memcpy(fprev, F, nt * sizeof(cplx));
    }
    st->have_fprev = 1;
    st->step++;
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 0-d SDE ensembles (Sec. III): independent paths of the Ito SDE              */
/*   du = c u dt + F(u) dt + G(u) dW                                          */
/* kind 0, SAO (Eq. sao), p = {Gamma, T, b}: c = -Gamma, F = -Gamma b u^3,     */
/*   G = sqrt(2 Gamma T);                                                      */
/* kind 1, GBM (Eq. gbm), p = {lambda, mu, delta}: c = lambda - delta,         */
/*   F = delta u, G = mu u.                                                    */
/* Schemes (the update rules of the stability table of Sec. III):             */
/*   0 EM:            u + (c u + F) h + G dW                                   */
/*   1 Milstein:      EM + G G' (dW^2 - h) / 2                                 */
/*   2 SETD-EM:       f1 u + f2 F + f3 G dW                       (Eq. SETD-EM) */
/*   3 SETD-Milstein: f1 u + f2 F + f3 G [dW + G' (dW^2 - h)/2]   (Eq. SETD-Miltstein) */
/*   4 SETD1:         f1 u + f2 F + f4 G N,  N = dW / sqrt(h)     (Eq. SETD1)  */
/* f1 = e^{ch}, f2 = (e^{ch} - 1)/c, f3 = e^{ch/2}, f4 = sqrt((e^{2ch} - 1)/(2c)). */
/* Wiener increments: step n of size h = K h_f is the sum over i < K of        */
/* sqrt(h_f) z(p, (step0 + n) K + i), z(p, m) the normal p & 3 of             */
/* Philox(ctr = (p >> 2, m, 0, 2), key = seed); runs with different K on one  */
/* seed therefore follow one Wiener path.  w (optional) accumulates W.        */
/* ------------------------------------------------------------------------- */
int or_sde0d(int kind, const double* p, int scheme, double h, int substeps, uint64_t seed, int64_t step0,
             int64_t nsteps, int64_t npaths, double* u, double* w) {
    if (kind < 0 || kind > 1 || scheme < 0 || scheme > 4 || !(h > 0) || substeps < 1) return 1;
    const double c = kind == 0 ? -p[0] : p[0] - p[2];
    const double ch = c * h;
    const double f1 = exp(ch);
    const double f2 = c != 0.0 ? expm1(ch) / c : h;
    const double f3 = exp(0.5 * ch);
    const double f4 = c != 0.0 ? sqrt(expm1(2.0 * ch) / (2.0 * c)) : sqrt(h);
    const double sqhf = sqrt(h / substeps);
    for (int64_t pa = 0; pa < npaths; ++pa) {
        double x = u[pa], wsum = w ? w[pa] : 0.0;
        for (int64_t n = 0; n < nsteps; ++n) {
            double dW = 0.0;
            for (int i = 0; i < substeps; ++i) {
                const int64_t m = (step0 + n) * substeps + i;
                float z[4];
                normals_for_index(seed, (uint32_t)(pa >> 2), (uint32_t)m, 0u, 2u, z);
                dW += sqhf * (double)z[pa & 3];
            }
            double F, G, Gp;
            if (kind == 0) {
                F = -p[0] * p[2] * x * x * x;
                G = sqrt(2.0 * p[0] * p[1]);
                Gp = 0.0;
            } else {
                F = p[2] * x;
                G = p[1] * x;
                Gp = p[1];
            }
            double xn;
            switch (scheme) {
                case 0: xn = x + (c * x + F) * h + G * dW; break;
                case 1: xn = x + (c * x + F) * h + G * dW + 0.5 * G * Gp * (dW * dW - h); break;
                case 2: xn = f1 * x + f2 * F + f3 * G * dW; break;
                case 3: xn = f1 * x + f2 * F + f3 * G * (dW + 0.5 * Gp * (dW * dW - h)); break;
                default: xn = f1 * x + f2 * F + f4 * G * (dW / sqrt(h)); break;
            }
            x = xn;
            wsum += dW;
        }
        u[pa] = x;
        if (w) w[pa] = wsum;
    }
    return 0;
}

/* Width over boxes (Sec. V.B): for replica r, the mean over the boxes of ell^d
 * sites tiling the lattice of the variance of the real-space field in the box,
 * <h^2>_box - <h>_box^2.  ell must divide every n_i.  out: R values. */
int or_box_width(const or_state* st, int ell, double* out) {
    if (st->cplx_field || ell < 1) return 1;
    for (int ax = 0; ax < st->cfg.d; ++ax)
        if (st->n[ax] % ell) return 1;
    const int nx = st->n[0], ny = st->n[1], nz = st->n[2];
    const int lx = ell, ly = st->cfg.d >= 2 ? ell : 1, lz = st->cfg.d >= 3 ? ell : 1;
    const int bx = nx / lx, by = ny / ly, bz = nz / lz;
    double* h = (double*)malloc(sizeof(double) * st->ntot);
    for (int r = 0; r < st->cfg.replicas; ++r) {
        or_get_field(st, r, h);
        double acc = 0.0;
        for (int kz = 0; kz < bz; ++kz)
            for (int ky = 0; ky < by; ++ky)
                for (int kx = 0; kx < bx; ++kx) {
                    double s1 = 0.0, s2 = 0.0;
                    for (int z = kz * lz; z < (kz + 1) * lz; ++z)
                        for (int y = ky * ly; y < (ky + 1) * ly; ++y)
                            for (int x = kx * lx; x < (kx + 1) * lx; ++x) {
                                const double v = h[((size_t)z * ny + y) * nx + x];
                                s1 += v;
                                s2 += v * v;
                            }
                    const double n = (double)lx * ly * lz, m = s1 / n;
                    acc += s2 / n - m * m;
                }
        out[r] = acc / ((double)bx * by * bz);
    }
    free(h);
    return 0;
}

/* The nonlinear term F_a = M_a s_a DFT[q(psi)]_a of the current state of one
 * replica (Sec. IV step 1-3, full spectrum): with c_a phi_a it is the
 * deterministic force K_a of the noise-inferred susceptibility (App. C). */
int or_force(or_state* st, int replica, double* out_ri) {
    if (replica < 0 || replica >= st->cfg.replicas) return 1;
    nonlinear_term(st, st->phi + (size_t)replica * st->ntot, (cplx*)out_ri);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Dynamic observables of App. C from an ensemble of recorded time series.     */
/*                                                                             */
/* Input: S series (replicas) of n modes, each sampled at M times m = 0..M-1   */
/* spanning the record duration T; phi[(s n + a) M + m] and F[...] complex     */
/* (interleaved re, im): the state phi_a and the nonlinear term F_a at each    */
/* sample; c[a] (complex, interleaved) the linear operator, D[a] the noise     */
/* strength; norm = (L/N^2)^d.  The steps, in the paper's order:               */
/*   1. time DFT of every series, phi_{a,b} = sum_m e^{+2 pi i b m / M}        */
/*      phi_{a,m} (the printed exponent divides by T; read as M, the number    */
/*      of samples, so that b indexes the M frequencies), and likewise K;      */
/*   2. the deterministic force K = c phi + F (the Langevin drift K[phi] of    */
/*      the Onsager-Machlup functional, in Fourier space);                     */
/*   3. omega_b = 2 pi b / T with b the signed frequency index;                */
/*   4. C_{a,b} = norm (T / M^2) <|phi_{a,b}|^2>_s;                            */
/*   5. chi_{a,b} = norm (T / M^2) (1 / 2 D_a) <phi_{a,b} conj(-i omega_b       */
/*      phi_{a,b} - K_{a,b})>_s;                                               */
/*   6. Delta_{a,b} = 2 Im chi_{a,b} - (omega_b / D_a) C_{a,b} (Sec. V.A) and   */
/*      Dbar = the mean of |Delta| over the frequencies and the modes.         */
/* Readings: the ensemble sum over s is taken as the ensemble mean (1/S), as   */
/* an estimator of the expectation; modes with D_a = 0 carry no noise, so      */
/* chi is left zero there and they are left out of Dbar.  The DFT is the plain */
/* O(M^2) sum of its definition.  C_out[a M + b] (real), chi_out[a M + b]      */
/* (complex, interleaved), *dbar_out.                                          */
/* ------------------------------------------------------------------------- */
int or_dyn_estimators(int S, long n, int M, const double* phi_ri, const double* F_ri, const double* c_ri,
                      const double* D, double T, double norm, double* C_out, double* chi_out, double* dbar_out) {
    if (S < 1 || n < 1 || M < 1 || !(T > 0)) return 1;
    const cplx* phi = (const cplx*)phi_ri;
    const cplx* F = (const cplx*)F_ri;
    const cplx* c = (const cplx*)c_ri;
    cplx* chi = (cplx*)chi_out;
    cplx* X = (cplx*)malloc(sizeof(cplx) * (size_t)M);
    cplx* Y = (cplx*)malloc(sizeof(cplx) * (size_t)M);
    if (!X || !Y) {
        free(X);
        free(Y);
        return 2;
    }
    for (long i = 0; i < n * M; ++i) {
        C_out[i] = 0.0;
        chi[i] = 0.0;
    }
    const double pref = norm * T / ((double)M * M) / (double)S;
    for (int s = 0; s < S; ++s) {
        for (long a = 0; a < n; ++a) {
            const cplx* ps = phi + ((size_t)s * n + a) * M;
            const cplx* fs = F + ((size_t)s * n + a) * M;
            /* step 1: time DFT with the + sign */
            for (int b = 0; b < M; ++b) {
                cplx xs = 0.0, ys = 0.0;
                for (int m = 0; m < M; ++m) {
                    const cplx e = cexp(2.0 * OR_PI * I * (double)(((long)b * m) % M) / (double)M);
                    xs += e * ps[m];
                    ys += e * fs[m];
                }
                X[b] = xs;
                Y[b] = ys;
            }
            for (int b = 0; b < M; ++b) {
                /* steps 2, 3 */
                const cplx K = c[a] * X[b] + Y[b];
                const int bs = 2 * b < M ? b : b - M;
                const double om = 2.0 * OR_PI * (double)bs / T;
                /* steps 4, 5 */
                C_out[a * M + b] += pref * creal(X[b] * conj(X[b]));
                if (D[a] > 0.0) chi[a * M + b] += pref / (2.0 * D[a]) * X[b] * conj(-I * om * X[b] - K);
            }
        }
    }
    /* step 6 */
    double acc = 0.0;
    long cnt = 0;
    for (long a = 0; a < n; ++a) {
        if (!(D[a] > 0.0)) continue;
        for (int b = 0; b < M; ++b) {
            const int bs = 2 * b < M ? b : b - M;
            const double om = 2.0 * OR_PI * (double)bs / T;
            acc += fabs(2.0 * cimag(chi[a * M + b]) - om / D[a] * C_out[a * M + b]);
            ++cnt;
        }
    }
    *dbar_out = cnt ? acc / (double)cnt : 0.0;
    free(X);
    free(Y);
    return 0;
}

/* The linear operator c_a and the noise strength D_a of every mode of the full
 * spectrum (Sec. V, per model), for the dynamic observables: out[3 idx] =
 * Re c, out[3 idx + 1] = Im c, out[3 idx + 2] = D. */
void or_mode_operators(const or_state* st, double* out) {
    for (size_t idx = 0; idx < st->ntot; ++idx) {
        cplx c, s;
        double D;
        mode_operator(st, idx, &c, &D, &s);
        out[3 * idx] = creal(c);
        out[3 * idx + 1] = cimag(c);
        out[3 * idx + 2] = D;
    }
}
