// sft_k1d_cluster.cu -- whole-step kernel for long 1-D real lattices, one
// replica per thread-block cluster.
//
// 65536 points: the half-length complex line (M = 32768 values, packed
// z[m] = x[2m] + i x[2m+1]) does not fit one block's shared memory in FP32.
// 16384 and 32768 points fit one block, but a block per replica leaves most SMs
// idle when there are fewer replicas than SMs.  So one replica is held by a
// cluster of P blocks of L / 8 threads (8 values per thread, 64 registers), and
// every M-point transform is split four-step style into L = M / P-point FFTs
// that each block runs in its own shared memory, plus one P-point stage across
// the blocks (P, L) = (4, 8192), (2, 8192), (2, 4096) for 65536, 32768, 16384
// points:
//
//   inverse, m = P l + p, n = n1 + L n2:
//     T_p[n1] = W_M^{-p n1} IFFT_L(Z[P l + p])[n1]        (block p, local)
//     y[n1 + L n2] = sum_p W_P^{-p n2} T_p[n1]             (block q: n1 in its quarter; reads T_p remotely)
//   forward, k = P k1 + k2:
//     U_k2[n1] = W_M^{n1 k2} sum_n2 q[n1 + L n2] W_P^{n2 k2} (the thread that holds q[n1 + L n2])
//     Q[P k1 + k2] = FFT_L(U_k2)[k1]                        (block k2, after U_k2 is written into it)
//
// so distributed shared memory is touched only by the cross-block stage, the
// redistribution before the forward FFT and the r2c partner reads, not by every
// FFT pass.  Same arithmetic as the single-block line kernel otherwise (Sec. IV
// boxed algorithm): dealias + scale, C2R, q(psi), R2C, SETD update with the
// Philox Fourier noise.
#include <cooperative_groups.h>

#include "sft_step_common.cuh"

namespace cg = cooperative_groups;

namespace sft {

template <int L>
using ClPlan = FftPlan<L, 8>;

template <int L>
__device__ __forceinline__ int clpos(int i) { return xpos<L, 8>(i); }

template <int P, int L, int MODE, int NL>
__global__ void __launch_bounds__(ClPlan<L>::T, 1024 / ClPlan<L>::T) k1_cluster(const StepArgs a) {
    constexpr int M = P * L, NX = 2 * M, E = ClPlan<L>::E, T = ClPlan<L>::T;
    static_assert(E == 8, "8 values per thread");
    constexpr int NI = L / (P * T);  // n1 values per thread in the cross-block stage
    static_assert(NI * P == E, "cross-block stage keeps E values per thread");
    extern __shared__ float2 sm[];
    cg::cluster_group cl = cg::this_cluster();
    const int q = (int)cl.block_rank();  // block of the cluster
    const int t = threadIdx.x;
    const int rr = blockIdx.x / P;  // replica
    const float2* __restrict__ twL = a.tw_c;  // W_L
    const float2* __restrict__ twM = a.tw_a;  // W_M
    const float2* __restrict__ twN = a.tw_b;  // W_NX
    float2* ph = a.phi + (size_t)rr * (M + 1);
    float2* rem[P];
#pragma unroll
    for (int r = 0; r < P; ++r) rem[r] = cl.map_shared_rank(sm, r);
    float2 y[E];  // y[i P + n2] = value at n = n1(i) + L n2, n1(i) = q L/P + t + T i
    cl.sync();    // every block of the cluster is running before remote shared memory is touched

    if constexpr (MODE == MODE_FWD) {
        const float* src = a.real_io + (size_t)rr * NX;
#pragma unroll
        for (int i = 0; i < NI; ++i)
#pragma unroll
            for (int n2 = 0; n2 < P; ++n2) {
                const int n = q * (L / P) + t + T * i + L * n2;
                y[i * P + n2] = *reinterpret_cast<const float2*>(src + 2 * n);
            }
    } else {
        // inverse, block-local part: T_p[n1] for p = q
        float2 z[E];
        const float sc = a.scale;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = P * (t + T * e) + q;
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
        fft_line<L, true, 8>(z, sm, t, twL);
        __syncthreads();  // the FFT's last reads of the buffer are done
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int n1 = t + T * e;
            float2 w = __ldg(&twM[q * n1]);
            w.y = -w.y;
            sm[clpos<L>(n1)] = cmul(z[e], w);
        }
        cl.sync();
        // cross-block inverse P-point stage for this block's quarter of n1
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int n1 = q * (L / P) + t + T * i;
            float2 x[P];
#pragma unroll
            for (int p = 0; p < P; ++p) x[p] = rem[p][clpos<L>(n1)];
            dft_reg<P, true>(x);
#pragma unroll
            for (int n2 = 0; n2 < P; ++n2) y[i * P + n2] = x[n2];
        }
        if constexpr (MODE == MODE_INV) {
            float* dst = a.real_io + (size_t)rr * NX;
#pragma unroll
            for (int i = 0; i < NI; ++i)
#pragma unroll
                for (int n2 = 0; n2 < P; ++n2) {
                    const int n = q * (L / P) + t + T * i + L * n2;
                    *reinterpret_cast<float2*>(dst + 2 * n) = y[i * P + n2];
                }
        } else {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if constexpr (NL == NL_GRAD2)
                    y[e] = make_float2(y[e].x * y[e].x, y[e].y * y[e].y);
                else
                    y[e] = make_float2(y[e].x * y[e].x * y[e].x, y[e].y * y[e].y * y[e].y);
            }
        }
    }

    if constexpr (MODE != MODE_INV) {
        // forward: U_k2[n1] for this thread's n1, written into block k2
        cl.sync();  // every remote read of the cross-block inverse stage is done
#pragma unroll
        for (int i = 0; i < NI; ++i) {
            const int n1 = q * (L / P) + t + T * i;
            float2 x[P];
#pragma unroll
            for (int n2 = 0; n2 < P; ++n2) x[n2] = y[i * P + n2];
            dft_reg<P, false>(x);
#pragma unroll
            for (int k2 = 0; k2 < P; ++k2) rem[k2][clpos<L>(n1)] = cmul(x[k2], __ldg(&twM[n1 * k2]));
        }
        cl.sync();
        float2 v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = sm[clpos<L>(t + T * e)];
        fft_line<L, false, 8>(v, sm, t, twL);  // v[e] = Q[P (t + T e) + q]
        __syncthreads();
#pragma unroll
        for (int e = 0; e < E; ++e) sm[clpos<L>(t + T * e)] = v[e];
        cl.sync();

        // R2C post-processing and the update of the modes k in [q L, (q + 1) L) (block q)
        auto Qat = [&](int k) -> float2 { return rem[k % P][clpos<L>(k / P)]; };
        float2 Xq[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = q * L + t + T * e;
            Xq[e] = r2c_post(Qat(k), cconj(Qat((M - k) & (M - 1))), __ldg(&twN[k]));
        }
        const float2 z0 = rem[0][clpos<L>(0)];
        const float2 XqM = make_float2(z0.x - z0.y, 0.f);
        const bool last_owner = (q == 0 && t == 0);  // also handles the Nyquist mode k = M
        if constexpr (MODE == MODE_FWD) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int k = q * L + t + T * e;
                float2 o = Xq[e];
                if (k == 0) o.y = 0.f;
                ph[k] = o;
            }
            if (last_owner) ph[M] = XqM;
        } else {
            const long long step = current_step(a);
            const bool first = (a.scheme == 2) && (step == *a.first_step);
            float2* fp = a.fprev + (size_t)rr * (M + 1);
            const uint32_t rep = (uint32_t)(a.rep0 + rr);
            float2 zn0, zn1;
            float nf = 0.f;
#pragma unroll
            for (int e = 0; e <= E; ++e) {
                if (e < E && (e & 1) == 0)
                    team_normal_pair_ks<T>(a.ks, (uint64_t)q * L, t, e, (uint32_t)step, rep, zn0, zn1);
                if (e == E && !last_owner) break;
                const int k = (e < E) ? q * L + t + T * e : M;
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
                nf = nonfinite_acc(nf, o);
            }
            flag_nonfinite_acc(a, nf, step);
        }
    }
    cl.sync();  // no block leaves while others may still read its shared memory
}

template <int P, int L, int MODE, int NL>
static cudaError_t run_cluster(const StepArgs& a, cudaStream_t s) {
    static bool attr = false;
    const size_t sm = sizeof(float2) * (size_t)ClPlan<L>::BUF;
    if (!a.tw_a || !a.tw_b || !a.tw_c) return cudaErrorInvalidValue;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(k1_cluster<P, L, MODE, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(P * a.R), 1, 1);
    cfg.blockDim = dim3(ClPlan<L>::T, 1, 1);
    cfg.dynamicSmemBytes = sm;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = P;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k1_cluster<P, L, MODE, NL>, a);
}

template <int P, int L>
static cudaError_t cluster_for(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    if (mode == MODE_FWD) return run_cluster<P, L, MODE_FWD, NL_CUBIC>(a, s);
    if (mode == MODE_INV) return run_cluster<P, L, MODE_INV, NL_CUBIC>(a, s);
    if (mode == MODE_STEP && nl == NL_CUBIC) return run_cluster<P, L, MODE_STEP, NL_CUBIC>(a, s);
    if (mode == MODE_STEP && nl == NL_GRAD2) return run_cluster<P, L, MODE_STEP, NL_GRAD2>(a, s);
    return cudaErrorInvalidValue;
}

int k1_cluster_fft_len(int nx) {
    switch (nx) {
        case 65536:
        case 32768: return 8192;
        case 16384: return 4096;
        default: return 0;
    }
}

bool k1_use_cluster(int nx, int R, int mode) {
    if (nx == 65536) return true;
    if (!k1_cluster_fft_len(nx) || !(mode == MODE_STEP || mode == MODE_FWD || mode == MODE_INV)) return false;
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 1;
    }
    return R < 2 * nsm;  // a block per replica would leave SMs idle
}

cudaError_t launch_k1_cluster(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    switch (a.nx) {
        case 65536: return cluster_for<4, 8192>(a, mode, nl, s);
        case 32768: return cluster_for<2, 8192>(a, mode, nl, s);
        case 16384: return cluster_for<2, 4096>(a, mode, nl, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
