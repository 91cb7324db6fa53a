// sft_misc.cu -- per-context set-up and bookkeeping kernels: the FP64
// coefficient tables, the Philox initial condition, the step counter, and the
// shell-averaged observables.
#include <type_traits>
#include "sft_step_common.cuh"

namespace sft {

// ------------------------------------------------------------------ tables
// phi1(z) = (e^z - 1)/z, phi2(z) = (e^z - 1 - z)/z^2 (Sec. II), in FP64:
// real z by expm1 with a Taylor series for phi2 when |z| < 1/2; complex z by
// the Taylor series for |z| < 1 and the direct formula otherwise.  The c -> 0
// limits (1 and 1/2) are the small-c fallback of Sec. IV.
__device__ void phi12_real(double x, double& p1, double& p2) {
    if (x == 0.0) {
        p1 = 1.0;
        p2 = 0.5;
        return;
    }
    const double em1 = expm1(x);
    p1 = em1 / x;
    if (fabs(x) < 0.5) {
        double term = 0.5, sum = 0.0;
        for (int k = 0; k < 30; ++k) {
            sum += term;
            term *= x / (double)(k + 3);
        }
        p2 = sum;
    } else {
        p2 = (em1 - x) / (x * x);
    }
}

__device__ __forceinline__ double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 zdiv(double2 a, double2 b) {
    const double d = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 zexp(double2 z) {
    double s, c;
    sincos(z.y, &s, &c);
    const double m = exp(z.x);
    return make_double2(m * c, m * s);
}

__device__ void phi12_cplx(double2 z, double2& p1, double2& p2) {
    if (z.y == 0.0) {
        double a, b;
        phi12_real(z.x, a, b);
        p1 = make_double2(a, 0.0);
        p2 = make_double2(b, 0.0);
        return;
    }
    if (z.x * z.x + z.y * z.y < 1.0) {
        double2 t1 = make_double2(1.0, 0.0), t2 = make_double2(0.5, 0.0);
        double2 s1 = make_double2(0.0, 0.0), s2 = make_double2(0.0, 0.0);
        for (int k = 0; k < 40; ++k) {
            s1.x += t1.x; s1.y += t1.y;
            s2.x += t2.x; s2.y += t2.y;
            t1 = zmul(t1, make_double2(z.x / (k + 2), z.y / (k + 2)));
            t2 = zmul(t2, make_double2(z.x / (k + 3), z.y / (k + 3)));
        }
        p1 = s1;
        p2 = s2;
    } else {
        double2 em1 = zexp(z);
        em1.x -= 1.0;
        p1 = zdiv(em1, z);
        p2 = zdiv(make_double2(em1.x - z.x, em1.y - z.y), zmul(z, z));
    }
}

// One entry per class of modes with equal |k| (isotropic lattice; see the
// table layouts in sft_internal.h), k^2 = dk^2 |a|^2:
//   z = c h, f1 = e^z;
//   SETD-EM: A = h phi1(z), B = 0, g = nf sqrt(2 D h) e^{z/2}      (f3 G dW)
//   SETD1:   A = h phi1(z), B = 0, g = nf sqrt(2 D h phi1(2 Re z))  (f4 G, exact I1)
//   SETD2:   A = h (phi1 + phi2), B = -h phi2, g as SETD1            (Eq. SETD2)
// nf = (N^2/L)^{d/2} (App. A).  Real models store {f1, A, B, g}; CGL stores
// {f1, A} and {B, g} as complex pairs.
__global__ void k_build_table(const TableArgs t) {
    const long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (q >= t.nq) return;
    const double k2 = t.dk * t.dk * (double)table_k2_index(t.d, t.hy, q);
    const double* p = t.p;
    double2 c = make_double2(0.0, 0.0);
    double D = 0.0;
    double2 s = make_double2(1.0, 0.0);  // nonlinear prefactor folded into A, B (SFT_CUSTOM only)
    // Model A/B with p[4] != 0: the r phi term is part of F (explicit), not of c; for SETD-EM and
    // SETD1 it folds into f1 below: f1 phi + A (F_nl + s_r phi) = (f1 + A s_r) phi + A F_nl
    const bool rf = (t.model == 0 || t.model == 1) && p[4] != 0.0;
    const double rr = rf ? 0.0 : p[1];
    switch (t.model) {
        case 0: c.x = -p[0] * (rr + k2); D = p[0] * p[3]; break;
        case 1: c.x = -p[0] * k2 * (rr + k2); D = p[0] * p[3] * k2; break;
        case 2: c.x = -p[0] * k2; D = p[2]; break;
        case 3: c.x = 1.0 - k2; c.y = -p[0] * k2; D = p[2]; break;
        default: {  // tables over |a|^2 (general Fourier-space form, Sec. IV)
            const long long a2 = table_k2_index(t.d, t.hy, q);
            const long long n = t.ncust;
            c = make_double2(t.cust[a2], t.cust[n + a2]);
            D = t.cust[2 * n + a2];
            s = make_double2(t.cust[3 * n + a2], t.cust[4 * n + a2]);
        }
    }
    const double h = t.h;
    const double2 z = make_double2(c.x * h, c.y * h);
    double2 p1, p2;
    phi12_cplx(z, p1, p2);
    const double2 f1 = zexp(z);
    double2 A, B = make_double2(0.0, 0.0), g;
    if (t.scheme == 0) {
        A = make_double2(h * p1.x, h * p1.y);
        const double2 e2 = zexp(make_double2(0.5 * z.x, 0.5 * z.y));
        const double amp = t.noise_norm * sqrt(2.0 * D * h);
        g = make_double2(amp * e2.x, amp * e2.y);
    } else {
        double q1, q2;
        phi12_real(2.0 * z.x, q1, q2);
        g = make_double2(t.noise_norm * sqrt(2.0 * D * h * q1), 0.0);
        if (t.scheme == 1) {
            A = make_double2(h * p1.x, h * p1.y);
        } else {
            A = make_double2(h * (p1.x + p2.x), h * (p1.y + p2.y));
            B = make_double2(-h * p2.x, -h * p2.y);
        }
    }
    double2 f1v = f1;
    if (rf) {
        const double sr = -p[0] * p[1] * (t.model == 1 ? k2 : 1.0);
        f1v = make_double2(f1.x + A.x * sr, f1.y + A.y * sr);
    }
    A = make_double2(A.x * s.x - A.y * s.y, A.x * s.y + A.y * s.x);
    B = make_double2(B.x * s.x - B.y * s.y, B.x * s.y + B.y * s.x);
    if (t.complex_field) {
        t.out[2 * q] = make_float4((float)f1v.x, (float)f1v.y, (float)A.x, (float)A.y);
        t.out[2 * q + 1] = make_float4((float)B.x, (float)B.y, (float)g.x, (float)g.y);
    } else {
        t.out[q] = make_float4((float)f1v.x, (float)A.x, (float)B.x, (float)g.x);
    }
}

cudaError_t launch_build_table(const TableArgs& t, cudaStream_t s) {
    const int th = 128;
    k_build_table<<<(unsigned)((t.nq + th - 1) / th), th, 0, s>>>(t);
    return cudaGetLastError();
}

// ------------------------------------------------------- twiddle tables
// tw[m] = W_L^m = e^{-2 pi i m / L}, m < L: sin and cos of pi (2m / L) in FP64
// (exact zeros at the quarter turns), rounded to float.
__global__ void k_twiddles(float2* tw, int L) {
    const int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= L) return;
    double sn, cs;
    sincospi(2.0 * (double)m / (double)L, &sn, &cs);
    tw[m] = make_float2((float)cs, (float)-sn);
}

cudaError_t launch_twiddles(float2* tw, int L, cudaStream_t s) {
    if (L < 1) return cudaSuccess;
    k_twiddles<<<(L + 127) / 128, 128, 0, s>>>(tw, L);
    return cudaGetLastError();
}

// tw[k1 32 + t] = W_1024^{t k1} for t, k1 < 32 (the 1024-point warp transforms)
__global__ void k_twiddles32(float2* tw) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= 1024) return;
    double sn, cs;
    sincospi(2.0 * (double)((i >> 5) * (i & 31)) / 1024.0, &sn, &cs);
    tw[i] = make_float2((float)cs, (float)-sn);
}

cudaError_t launch_twiddles32(float2* tw, cudaStream_t s) {
    k_twiddles32<<<8, 128, 0, s>>>(tw);
    return cudaGetLastError();
}

// ------------------------------------------------------- initial condition
// Real fields: site s of replica r is sigma * z[s & 3] of the four normals of
// Philox(ctr = (s >> 2, 0, r, 1)); complex fields: sigma (z_a + i z_b) of the
// pair (s & 1) of Philox(ctr = (s >> 1, 0, r, 1)).
__global__ void k_init_random(float* real_out, float2* cplx_out, long long sites, int R, int rep0, uint64_t seed,
                              float sigma) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    if (real_out) {
        const long long s0 = 4 * g;
        if (s0 >= sites) return;
        const uint4 w = philox4x32_10(make_uint4((uint32_t)g, 0u, (uint32_t)(rep0 + r), 1u), key);
        const float2 a = recipe_bm_pair(w.x, w.y), b = recipe_bm_pair(w.z, w.w);
        const float z[4] = {a.x, a.y, b.x, b.y};
        for (int i = 0; i < 4 && s0 + i < sites; ++i) real_out[(size_t)r * sites + s0 + i] = sigma * z[i];
    } else {
        const long long s0 = 2 * g;
        if (s0 >= sites) return;
        const uint4 w = philox4x32_10(make_uint4((uint32_t)g, 0u, (uint32_t)(rep0 + r), 1u), key);
        const float2 a = recipe_bm_pair(w.x, w.y), b = recipe_bm_pair(w.z, w.w);
        cplx_out[(size_t)r * sites + s0] = make_float2(sigma * a.x, sigma * a.y);
        if (s0 + 1 < sites) cplx_out[(size_t)r * sites + s0 + 1] = make_float2(sigma * b.x, sigma * b.y);
    }
}

cudaError_t launch_init_random(float* real_out, float2* cplx_out, long long sites, int R, int rep0, uint64_t seed,
                               float sigma, cudaStream_t s) {
    const long long per = real_out ? 4 : 2;
    const long long threads = (sites + per - 1) / per;
    dim3 grid((unsigned)((threads + 255) / 256), R);
    k_init_random<<<grid, 256, 0, s>>>(real_out, cplx_out, sites, R, rep0, seed, sigma);
    return cudaGetLastError();
}

__global__ void k_advance(long long* step_base, int by) { *step_base += by; }

cudaError_t launch_advance(long long* step_base, int by, cudaStream_t s) {
    k_advance<<<1, 1, 0, s>>>(step_base, by);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- observables
// Shell sums in a fixed order with compensation, so that repeated evaluations
// give the same bits and long sums keep FP64 accuracy (App. C estimators):
// the stored modes are enumerated shell by shell (ObsArgs::order, built once
// per lattice on the host) and cut into chunks of at most kObsChunkLen modes
// inside one shell.  One warp per chunk and replica: each lane sums a fixed
// stride of the chunk (at most 32 modes) in single-precision pairs made of
// error-free transformations -- products split exactly by a fused
// multiply-add (x x = p + e, Dekker), sums by Knuth's two-sum -- so that no
// bit of a term is lost, then converts its pair to FP64; lanes are combined by
// a fixed shuffle tree and chunks in order, both with Neumaier's compensated
// FP64 summation.  (This GPU's FP64 rate is a small fraction of its FP32 rate:
// two FP64 operations per mode would cost more than the gather.)  For real
// fields the stored half carries weight 2 off the planes a_x in {0, nx/2} and
// 1 on them (exact in FP32).

// s + x with its rounding error carried in c (Neumaier)
__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
}

// (hi, lo) += x exactly up to the rounding of lo: Knuth's two-sum of hi and x, the error into lo
__device__ __forceinline__ void ff_add(float& hi, float& lo, float x) {
    const float s = hi + x, bb = s - hi;
    lo += (hi - (s - bb)) + (x - bb);
    hi = s;
}

// (hi, lo) += w (a b + c d), each product split exactly (a b = p + fma(a, b, -p)); w in {1, 2}
__device__ __forceinline__ void ff_add_dot2(float& hi, float& lo, float w, float a, float b, float c, float d) {
    const float p1 = a * b, p2 = c * d;
    const float e1 = fmaf(a, b, -p1), e2 = fmaf(c, d, -p2);
    ff_add(hi, lo, w * p1);
    ff_add(hi, lo, w * p2);
    lo += w * (e1 + e2);
}

template <int KIND>
__global__ void k_obs_chunks(const ObsArgs o) {
    const int chunk = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
    const int r = blockIdx.y;
    if (chunk >= o.nchunks) return;  // whole warp
    const int4 ch = o.chunks[chunk];
    const size_t nm = (size_t)o.hx * o.nz * o.ny;
    const float2* phi = o.phi ? o.phi + (size_t)r * nm : nullptr;
    const float2* ref = o.ref ? o.ref + (size_t)r * nm : nullptr;
    const int plane = o.nz * o.ny;
    // two independent pairs per lane (entries lane + 64 u and lane + 64 u + 32), so two gathers are in flight
    float hi[2] = {0.f, 0.f}, lo[2] = {0.f, 0.f};
    auto term = [&](int i, int k) {
        const int m = o.order[ch.y + i];
        const int ax = m / plane;
        const float w = (!o.complex_field && ax != 0 && 2 * ax != o.nx) ? 2.f : 1.f;
        if constexpr (KIND == 0) {
            const float2 v = phi[m];
            ff_add_dot2(hi[k], lo[k], w, v.x, v.x, v.y, v.y);
        } else if constexpr (KIND == 1) {
            const float2 v = phi[m], u = ref[m];
            ff_add_dot2(hi[k], lo[k], w, v.x, u.x, v.y, u.y);
        } else {
            const float2 u = ref[m];
            ff_add_dot2(hi[k], lo[k], w, u.x, u.x, u.y, u.y);
        }
    };
    int i = lane;
    for (; i + 32 < ch.z; i += 64) {
        term(i, 0);
        term(i + 32, 1);
    }
    if (i < ch.z) term(i, 0);
    double s = (double)hi[0], c = (double)lo[0];
    neumaier_add(s, c, (double)hi[1]);
    c += (double)lo[1];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double s2 = __shfl_down_sync(0xffffffffu, s, off), c2 = __shfl_down_sync(0xffffffffu, c, off);
        neumaier_add(s, c, s2);
        c += c2;
    }
    if (lane == 0) o.part[(size_t)r * o.nchunks + chunk] = make_double2(s, c);
}

// shell_sum[r][j] = norm * (the chunks of shell j combined in order)
__global__ void k_obs_shells(const ObsArgs o) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= (long long)o.R * o.nshells) return;
    const int r = (int)(i / o.nshells), j = (int)(i % o.nshells);
    const double2* p = o.part + (size_t)r * o.nchunks;
    double s = 0.0, c = 0.0;
    for (int k = o.first_chunk[j]; k < o.first_chunk[j + 1]; ++k) {
        neumaier_add(s, c, p[k].x);
        c += p[k].y;
    }
    o.shell_sum[i] = (s + c) * o.norm;
}

cudaError_t launch_observe(const ObsArgs& o, cudaStream_t s) {
    if (o.nchunks < 1) return cudaErrorInvalidValue;
    dim3 g1((unsigned)((o.nchunks + 7) / 8), o.R);
    if (o.kind == 1)
        k_obs_chunks<1><<<g1, 256, 0, s>>>(o);
    else if (o.kind == 2)
        k_obs_chunks<2><<<g1, 256, 0, s>>>(o);
    else
        k_obs_chunks<0><<<g1, 256, 0, s>>>(o);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const long long n = (long long)o.R * o.nshells;
    k_obs_shells<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(o);
    return cudaGetLastError();
}

// Time accumulator of S(k, t): acc[j] += sum over replicas r (in order) of shell_sum[r][j], as a
// compensated (sum, correction) pair.
__global__ void k_obs_time_acc(const double* shell_sum, int R, int nshells, double2* acc) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nshells) return;
    double s = acc[j].x, c = acc[j].y;
    for (int r = 0; r < R; ++r) neumaier_add(s, c, shell_sum[(size_t)r * nshells + j]);
    acc[j] = make_double2(s, c);
}

cudaError_t launch_obs_time_acc(const double* shell_sum, int R, int nshells, double2* acc, cudaStream_t s) {
    k_obs_time_acc<<<(nshells + 127) / 128, 128, 0, s>>>(shell_sum, R, nshells, acc);
    return cudaGetLastError();
}

}  // namespace sft

namespace sft {

// Fourier noise eta of every stored mode at one step (unit variance; the
// amplitude g_a is applied by the update).  Same classification as the step
// kernels: partners on the self-conjugate planes a_x in {0, nx/2} carry the
// conjugate of their canonical mode.
__global__ void k_draw_noise(int nx, int ny, int nz, int hx, int cplx, int R, int rep0, uint64_t seed,
                             long long step, float2* out) {
    const long long nm = (long long)hx * nz * ny;
    const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (m >= nm) return;
    const int ay = (int)(m % ny), az = (int)((m / ny) % nz), ax = (int)(m / ((long long)ny * nz));
    int cz = az, cy = ay;
    bool selfc = false, partner = false;
    if (!cplx && (ax == 0 || 2 * ax == nx)) {
        const int mz = (nz - az) % nz, my = (ny - ay) % ny;
        if (az > mz || (az == mz && ay > my)) {
            partner = true;
            cz = mz;
            cy = my;
        } else if (az == mz && ay == my) {
            selfc = true;
        }
    }
    const uint64_t j = ((uint64_t)ax * nz + cz) * ny + cy;
    float2 eta = fourier_noise(seed, j, (uint32_t)step, (uint32_t)(rep0 + r), selfc);
    if (partner) eta = cconj(eta);
    out[(size_t)r * nm + m] = eta;
}

cudaError_t launch_draw_noise(int nx, int ny, int nz, int hx, int cplx, int R, int rep0, uint64_t seed,
                              long long step, float2* out, cudaStream_t s) {
    const long long nm = (long long)hx * nz * ny;
    dim3 grid((unsigned)((nm + 255) / 256), R);
    k_draw_noise<<<grid, 256, 0, s>>>(nx, ny, nz, hx, cplx, R, rep0, seed, step, out);
    return cudaGetLastError();
}

// ------------------------------------------------------------- box width
// KPZ width over boxes (Sec. V.B): block b of the flattened (replica, box) grid
// sums h and h^2 over the ell^d sites of its box in FP64 and adds the box
// variance <h^2> - <h>^2 to its replica's accumulator.
__global__ void k_box_width(const float* __restrict__ real, int nx, int ny, int nz, int d, int ell, long long nboxes,
                            double* out) {
    const long long b = blockIdx.x;
    const int r = (int)(b / nboxes);
    const long long box = b % nboxes;
    const int bx = nx / ell, by = d >= 2 ? ny / ell : 1;
    const int x0 = (int)(box % bx) * ell, y0 = (int)((box / bx) % by) * ell, z0 = (int)(box / ((long long)bx * by)) * ell;
    const int lx = ell, ly = d >= 2 ? ell : 1, lz = d >= 3 ? ell : 1;
    const long long ncell = (long long)lx * ly * lz;
    const float* base = real + (size_t)r * ((size_t)nx * ny * nz);
    double s1 = 0.0, s2 = 0.0;
    for (long long i = threadIdx.x; i < ncell; i += blockDim.x) {
        const int x = x0 + (int)(i % lx), y = y0 + (int)((i / lx) % ly), z = z0 + (int)(i / ((long long)lx * ly));
        const double h = base[((size_t)z * ny + y) * nx + x];
        s1 += h;
        s2 += h * h;
    }
    __shared__ double red[2][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
        s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        red[0][wid] = s1;
        red[1][wid] = s2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            t1 += red[0][w];
            t2 += red[1][w];
        }
        const double m = t1 / (double)ncell;
        atomicAdd(&out[r], t2 / (double)ncell - m * m);
    }
}

cudaError_t launch_box_width(const float* real, int nx, int ny, int nz, int d, int ell, int R, double* out,
                             cudaStream_t s) {
    long long nboxes = nx / ell;
    if (d >= 2) nboxes *= ny / ell;
    if (d >= 3) nboxes *= nz / ell;
    const long long blocks = nboxes * R;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_box_width<<<(unsigned)blocks, 256, 0, s>>>(real, nx, ny, nz, d, ell, nboxes, out);
    return cudaGetLastError();
}

// ------------------------------------------------------ dynamic observables
// C_ab and chi_ab of App. C from the time transforms of the recorded series, one
// thread per (mode a, frequency b), the ensemble sum over replicas in FP64.  The
// paper's time transform is phi_b = sum_m e^{+2 pi i b m / M} phi_m: our forward
// transform (e^{-i}) at index (M - b) mod M; omega_b = 2 pi b / T, b signed.
//   C_ab   = norm sum_s |phi_ab|^2
//   chi_ab = norm / (2 D_a) sum_s phi_ab conj(-i omega_b phi_ab - K_ab),  K = c_a phi + F
__global__ void k_dyn_reduce(const DynArgs d) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= d.nmodes * d.M) return;
    const long long a = i / d.M;
    const int b = (int)(i % d.M);
    const int bb = (d.M - b) % d.M;
    const int sb = b < d.M / 2 ? b : b - d.M;
    const double w = 2.0 * 3.14159265358979323846 * (double)sb / d.T;
    const double ca = d.c[a];
    double cs = 0.0, xr = 0.0, xi = 0.0;
    for (int r = 0; r < d.R; ++r) {
        const size_t idx = ((size_t)r * d.nmodes + a) * d.M + bb;
        const float2 X = d.Phi[idx], Fb = d.Fw[idx];
        const double x = X.x, y = X.y;
        const double kx = ca * x + Fb.x, ky = ca * y + Fb.y;  // K = c phi + F
        const double yr = w * y - kx, yi = -w * x - ky;        // -i omega phi - K
        cs += x * x + y * y;
        xr += x * yr + y * yi;  // phi conj(Y)
        xi += y * yr - x * yi;
    }
    d.C[i] = cs * d.norm;
    const double f = d.D[a] > 0.0 ? d.norm / (2.0 * d.D[a]) : 0.0;
    d.chi[i] = make_double2(xr * f, xi * f);
}

cudaError_t launch_dyn_reduce(const DynArgs& d, cudaStream_t s) {
    const long long n = d.nmodes * d.M;
    k_dyn_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(d);
    return cudaGetLastError();
}

// complex transpose through 32 x 32 shared-memory tiles (padded against bank conflicts)
__global__ void k_transpose_c(const float2* __restrict__ in, float2* __restrict__ out, long long rows, long long cols) {
    __shared__ float2 tile[32][33];
    const long long c0 = (long long)blockIdx.x * 32, r0 = (long long)blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const long long r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[i][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const long long c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][i];
    }
}

cudaError_t launch_transpose_c(const float2* in, float2* out, long long rows, long long cols, cudaStream_t s) {
    const long long gx = (cols + 31) / 32, gy = (rows + 31) / 32;
    if (gx > 0x7fffffffLL || gy > 65535) return cudaErrorInvalidValue;
    k_transpose_c<<<dim3((unsigned)gx, (unsigned)gy), dim3(32, 8), 0, s>>>(in, out, rows, cols);
    return cudaGetLastError();
}

}  // namespace sft
