// sft_sde0d.cu -- ensembles of 0-d SDEs (Sec. III): the stochastic anharmonic
// oscillator (Eq. sao) and geometric Brownian motion (Eq. gbm) under the
// Euler-Maruyama, Milstein, SETD-EM (Eq. SETD-EM), SETD-Milstein
// (Eq. SETD-Miltstein) and SETD1 (Eq. SETD1) update rules of the stability
// table of Sec. III, for the convergence, steady-state and stability studies.
//
// One thread advances four paths through all steps in registers: path p takes
// normal p & 3 of Philox4x32-10(ctr = (p >> 2, m, 0, 2), key = seed) for fine
// increment m, the same Box-Muller recipe as the field noise.  A step of size
// h = K h_f sums K fine increments sqrt(h_f) z, so runs with different K on one
// seed follow one Wiener path.  State and coefficients are FP64; every
// operation is one correctly rounded IEEE operation in a fixed order, so the
// results do not depend on the compiler's contraction choices.
#include <cmath>

#include "../../include/sft.h"
#include "sft_device.cuh"

namespace sft {

struct SdeArgs {
    int kind, scheme, substeps;
    double p0, p1, p2;
    double h, c, f1, f2, f3, f4, sqhf, sqh;
    uint64_t seed;
    long long step0, nsteps, npaths;
    double* u;
    double* w;
};

__device__ __forceinline__ double dm(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double da(double a, double b) { return __dadd_rn(a, b); }

// one step of one path: x <- S(x, dW) (update rules of the stability table, Sec. III)
__device__ __forceinline__ double sde_update(const SdeArgs& a, double x, double dW) {
    double F, G, Gp;
    if (a.kind == SFT_SDE_SAO) {  // c = -Gamma, F = -Gamma b u^3, G = sqrt(2 Gamma T)
        F = dm(dm(dm(dm(-a.p0, a.p2), x), x), x);
        G = __dsqrt_rn(dm(dm(2.0, a.p0), a.p1));
        Gp = 0.0;
    } else {  // GBM: c = lambda - delta, F = delta u, G = mu u
        F = dm(a.p2, x);
        G = dm(a.p1, x);
        Gp = a.p1;
    }
    const double h = a.h;
    switch (a.scheme) {
        case SFT_SDE_EM: return da(da(x, dm(da(dm(a.c, x), F), h)), dm(G, dW));
        case SFT_SDE_MILSTEIN:
            return da(da(da(x, dm(da(dm(a.c, x), F), h)), dm(G, dW)),
                      dm(dm(dm(0.5, G), Gp), __dsub_rn(dm(dW, dW), h)));
        case SFT_SDE_SETD_EM: return da(da(dm(a.f1, x), dm(a.f2, F)), dm(dm(a.f3, G), dW));
        case SFT_SDE_SETD_MILSTEIN:
            return da(da(dm(a.f1, x), dm(a.f2, F)),
                      dm(dm(a.f3, G), da(dW, dm(dm(0.5, Gp), __dsub_rn(dm(dW, dW), h)))));
        default: return da(da(dm(a.f1, x), dm(a.f2, F)), dm(dm(a.f4, G), __ddiv_rn(dW, a.sqh)));
    }
}

__global__ void k_sde0d(const SdeArgs a) {
    const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;  // paths 4g .. 4g+3
    const long long p0 = 4 * g;
    if (p0 >= a.npaths) return;
    const int np = a.npaths - p0 < 4 ? (int)(a.npaths - p0) : 4;
    double x[4], ws[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        x[j] = j < np ? a.u[p0 + j] : 0.0;
        ws[j] = (j < np && a.w) ? a.w[p0 + j] : 0.0;
    }
    const uint2 key = make_uint2((uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    for (long long n = 0; n < a.nsteps; ++n) {
        double dW[4] = {0.0, 0.0, 0.0, 0.0};
        for (int i = 0; i < a.substeps; ++i) {
            const long long m = (a.step0 + n) * a.substeps + i;
            const uint4 wv = philox4x32_10(make_uint4((uint32_t)g, (uint32_t)m, 0u, 2u), key);
            const float2 z01 = recipe_bm_pair(wv.x, wv.y), z23 = recipe_bm_pair(wv.z, wv.w);
            dW[0] = da(dW[0], dm(a.sqhf, (double)z01.x));
            dW[1] = da(dW[1], dm(a.sqhf, (double)z01.y));
            dW[2] = da(dW[2], dm(a.sqhf, (double)z23.x));
            dW[3] = da(dW[3], dm(a.sqhf, (double)z23.y));
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            x[j] = sde_update(a, x[j], dW[j]);
            ws[j] = da(ws[j], dW[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
        if (j < np) {
            a.u[p0 + j] = x[j];
            if (a.w) a.w[p0 + j] = ws[j];
        }
}

}  // namespace sft

using namespace sft;

extern "C" sft_status sft_sde0d(int kind, const double* p, int scheme, double h, int substeps, uint64_t seed,
                                int64_t step0, int64_t nsteps, int64_t npaths, void* u_dev, void* w_dev,
                                void* stream) {
    if ((kind != SFT_SDE_SAO && kind != SFT_SDE_GBM) || scheme < SFT_SDE_EM || scheme > SFT_SDE_SETD1 || !p ||
        !(h > 0) || !std::isfinite(h) || substeps < 1 || step0 < 0 || nsteps < 0 || npaths < 0 ||
        (npaths > 0 && !u_dev))
        return SFT_EINVAL;
    if ((step0 + nsteps) * (int64_t)substeps > (int64_t)0xFFFFFFFFLL) return SFT_EINVAL;  // fine-increment counter
    if (kind == SFT_SDE_SAO && !(p[0] > 0 && p[1] >= 0)) return SFT_EINVAL;
    if (npaths == 0 || nsteps == 0) return SFT_OK;
    SdeArgs a{};
    a.kind = kind;
    a.scheme = scheme;
    a.substeps = substeps;
    a.p0 = p[0];
    a.p1 = p[1];
    a.p2 = p[2];
    a.h = h;
    // coefficients of Sec. III: f1 = e^{ch}, f2 = (e^{ch} - 1)/c, f3 = e^{ch/2}, f4 = sqrt((e^{2ch} - 1)/(2c))
    a.c = kind == SFT_SDE_SAO ? -p[0] : p[0] - p[2];
    const double ch = a.c * h;
    a.f1 = std::exp(ch);
    a.f2 = a.c != 0.0 ? std::expm1(ch) / a.c : h;
    a.f3 = std::exp(0.5 * ch);
    a.f4 = a.c != 0.0 ? std::sqrt(std::expm1(2.0 * ch) / (2.0 * a.c)) : std::sqrt(h);
    a.sqhf = std::sqrt(h / substeps);
    a.sqh = std::sqrt(h);
    a.seed = seed;
    a.step0 = step0;
    a.nsteps = nsteps;
    a.npaths = npaths;
    a.u = (double*)u_dev;
    a.w = (double*)w_dev;
    const long long groups = (npaths + 3) / 4;
    const int th = 128;
    k_sde0d<<<(unsigned)((groups + th - 1) / th), th, 0, (cudaStream_t)stream>>>(a);
    return cudaGetLastError() == cudaSuccess ? SFT_OK : SFT_ECUDA;
}
