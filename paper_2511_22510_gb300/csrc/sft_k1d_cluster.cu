// sft_k1d_cluster.cu -- whole-step kernel for 1-D real lattices of 65536 points.
//
// The half-length complex line (32768 values) does not fit one block's shared
// memory in FP32, so one replica is held by a cluster of 4 blocks of 512
// threads: the 2048 threads hold 16 values each in registers, and the padded
// exchange buffer of the Stockham passes is split in four quarters, one in
// each block's shared memory, addressed through distributed shared memory;
// cluster-wide barriers replace the team barriers.  Same arithmetic as the
// single-block line kernel (Sec. IV boxed algorithm).
#include <cooperative_groups.h>

#include "sft_step_common.cuh"

namespace cg = cooperative_groups;

namespace sft {

constexpr int kClM = 32768;  // half length
constexpr int kCl = 4;       // blocks per cluster
constexpr int kClThreads = 512;
using ClPlan = FftPlan<kClM, 16>;
static_assert(ClPlan::T == kCl * kClThreads, "one value group per thread");
constexpr int kClQuarter = (ClPlan::BUF + kCl - 1) / kCl;

struct DistBuf {
    float2* part[kCl];
    __device__ __forceinline__ float2& operator[](int p) const {
        const int r = p / kClQuarter;
        return part[r][p - r * kClQuarter];
    }
};

__device__ __forceinline__ void cl_sync() { cg::this_cluster().sync(); }

// Stockham pass over the distributed buffer (same plan and indexing as fft_line).
template <bool INV, int PASS, int NS>
__device__ __forceinline__ void cl_pass(float2 (&v)[ClPlan::E], const DistBuf& buf, int t,
                                        const float2* __restrict__ tw) {
    constexpr int N = kClM, E = ClPlan::E, T = ClPlan::T;
    constexpr int R = ClPlan::radix(PASS);
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
                x[b][r] = buf[xpos<N, 16>(j + r * (N / R))];
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
        cl_sync();
#pragma unroll
        for (int b = 0; b < NB; ++b) {
            const int j = t + T * b;
            const int k = j % NS;
            const int base = (j / NS) * NS * R + k;
#pragma unroll
            for (int s = 0; s < R; ++s) buf[xpos<N, 16>(base + s * NS)] = x[b][s];
        }
        cl_sync();
        cl_pass<INV, PASS + 1, NS * R>(v, buf, t, tw);
    }
}

template <int MODE, int NL>
__global__ void __cluster_dims__(kCl, 1, 1) __launch_bounds__(kClThreads) k1_cluster(const StepArgs a) {
    constexpr int M = kClM, NX = 2 * M, E = ClPlan::E, T = ClPlan::T;
    extern __shared__ float2 sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    DistBuf buf;
#pragma unroll
    for (int r = 0; r < kCl; ++r) buf.part[r] = cl.map_shared_rank(sm, r);
    const int t = rank * kClThreads + threadIdx.x;
    const int rr = blockIdx.x / kCl;  // replica
    const float2* __restrict__ twM = a.tw_a;
    const float2* __restrict__ twN = a.tw_b;
    float2* ph = a.phi + (size_t)rr * (M + 1);
    float2 z[E];
    cl_sync();  // every block of the cluster is running before remote shared memory is touched
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
        cl_pass<true, 0, 1>(z, buf, t, twM);
        if constexpr (MODE == MODE_INV) {
            float* dst = a.real_io + (size_t)rr * NX;
#pragma unroll
            for (int e = 0; e < E; ++e) *reinterpret_cast<float2*>(dst + 2 * (t + T * e)) = z[e];
            cl_sync();
            return;
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if constexpr (NL == NL_GRAD2)
                z[e] = make_float2(z[e].x * z[e].x, z[e].y * z[e].y);
            else
                z[e] = make_float2(z[e].x * z[e].x * z[e].x, z[e].y * z[e].y * z[e].y);
        }
    }
    cl_pass<false, 0, 1>(z, buf, t, twM);
    // R2C post-processing through the distributed buffer
    cl_sync();
#pragma unroll
    for (int e = 0; e < E; ++e) buf[xpos<M, 16>(t + T * e)] = z[e];
    cl_sync();
    float2 Xq[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = t + T * e;
        Xq[e] = r2c_post(z[e], cconj(buf[xpos<M, 16>((M - k) & (M - 1))]), __ldg(&twN[k]));
    }
    const float2 z0 = buf[0];
    const float2 XqM = make_float2(z0.x - z0.y, 0.f);
    if constexpr (MODE == MODE_FWD) {
#pragma unroll
        for (int e = 0; e < E; ++e) {
            float2 v = Xq[e];
            if (t + T * e == 0) v.y = 0.f;
            ph[t + T * e] = v;
        }
        if (t == 0) ph[M] = XqM;
    } else {
        const long long step = current_step(a);
        const bool first = (a.scheme == 2) && (step == *a.first_step);
        float2* fp = a.fprev + (size_t)rr * (M + 1);
        const uint32_t rep = (uint32_t)(a.rep0 + rr);
        float2 zn0, zn1;
#pragma unroll
        for (int e = 0; e <= E; ++e) {
            if (e < E && (e & 1) == 0) team_normal_pair<T>(a.seed, 0, t, e, (uint32_t)step, rep, zn0, zn1);
            if (e == E && t != 0) break;
            const int k = (e < E) ? t + T * e : M;
            const float2 xq = (e < E) ? Xq[e] : XqM;
            const bool inm = !a.dealias || 3 * k < NX;
            const float2 F = inm ? cscale(xq, nl_prefactor(a, k * k).x) : czero();
            const Coefs co = load_coefs<false>(a.tab, k, first);
            const float2 Fp = (a.scheme == 2) ? fp[k] : czero();
            const bool selfc = (k == 0 || k == M);
            const float2 eta = (e < E) ? eta_of((e & 1) ? zn1 : zn0, selfc)
                                       : fourier_noise(a.seed, (uint64_t)k, (uint32_t)step, rep, selfc);
            float2 o = setd_update<false>(co, ph[k], F, Fp, eta);
            if (selfc) o.y = 0.f;
            ph[k] = o;
            if (a.scheme == 2) fp[k] = F;
            flag_nonfinite(a, o, step);
        }
    }
    cl_sync();  // no block leaves while others may still read its shared memory
}

template <int MODE, int NL>
static cudaError_t run_cluster(const StepArgs& a, cudaStream_t s) {
    static bool attr = false;
    const size_t sm = sizeof(float2) * (size_t)kClQuarter;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k1_cluster<MODE, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k1_cluster<MODE, NL><<<kCl * a.R, kClThreads, sm, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_k1_cluster(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    if (mode == MODE_FWD) return run_cluster<MODE_FWD, NL_CUBIC>(a, s);
    if (mode == MODE_INV) return run_cluster<MODE_INV, NL_CUBIC>(a, s);
    if (mode == MODE_STEP && nl == NL_CUBIC) return run_cluster<MODE_STEP, NL_CUBIC>(a, s);
    if (mode == MODE_STEP && nl == NL_GRAD2) return run_cluster<MODE_STEP, NL_GRAD2>(a, s);
    return cudaErrorInvalidValue;
}

}  // namespace sft
