// sft_k3d.cu -- plane pass of the 3-D step (real fields, cubic term).
//
// Layout (x-major): spectrum phi[a_x][a_z][a_y], each a_x plane N x N
// contiguous.  The x-direction (row) pass is the 2-D row pass with the pair
// (z, y) as the row index.  This kernel holds one a_x plane of one replica in
// shared memory and does, in order:
//   y-FFT of the rows, z-FFT of the columns  -> DFT[q] on the plane;
//   SETD update per mode (Philox noise, counter index (a_x nz + a_z) ny + a_y);
//   Hermitian fix-up on the planes a_x in {0, nx/2}: the mode (a_z, a_y) is a
//   partner when (a_z, a_y) is lexicographically above (-a_z, -a_y) mod N;
//   dealiased inverse z- and y-FFTs -> the next step's row-pass input.
#include "sft_step_common.cuh"

namespace sft {

template <int N>
struct PlaneCfg {
    using PL = FftPlan<N>;
    static constexpr int T = PL::T;
    // a 128^2 plane fills most of an SM's shared memory (one block per SM), so
    // that block takes 512 threads; smaller planes run several 256-thread blocks
    static constexpr int TT = N >= 128 ? 512 : 256;
    static constexpr int TEAMS = T >= TT ? 1 : TT / T;
    static constexpr int THREADS = TEAMS * T;
    static constexpr int RS = N + 1;  // odd row stride of the plane
    static constexpr int XB = PL::BUF;
    static constexpr int ITERS = (N + TEAMS - 1) / TEAMS;  // lines per team per phase
    static constexpr size_t smem() { return sizeof(float2) * ((size_t)N * RS + (size_t)TEAMS * XB); }
};

// FFT of every row (ROW = true) or column of the plane held in shared memory.
template <int N, bool ROW, bool INV>
__device__ __forceinline__ void plane_fft(float2* S, float2* xb, int team, int t, const float2* __restrict__ tw) {
    using C = PlaneCfg<N>;
    using PL = FftPlan<N>;
    constexpr int T = PL::T, E = PL::E;
    for (int it = 0; it < C::ITERS; ++it) {
        const int line = team + it * C::TEAMS;
        const int l = line < N ? line : N - 1;
        float2 v[E];
#pragma unroll
        for (int e = 0; e < E; ++e) v[e] = ROW ? S[l * C::RS + t + T * e] : S[(t + T * e) * C::RS + l];
        fft_line<N, INV>(v, xb, t, tw);
        if (line < N) {
#pragma unroll
            for (int e = 0; e < E; ++e) {
                if (ROW)
                    S[l * C::RS + t + T * e] = v[e];
                else
                    S[(t + T * e) * C::RS + l] = v[e];
            }
        }
        team_sync<T>();
    }
}

template <int N, int MODE>
__global__ void __launch_bounds__(PlaneCfg<N>::THREADS) k3_planes(const StepArgs a) {
    using C = PlaneCfg<N>;
    using PL = FftPlan<N>;
    constexpr int T = PL::T, E = PL::E, RS = C::RS;
    extern __shared__ float2 sm[];
    float2* S = sm;
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    float2* xb = sm + (size_t)N * RS + (size_t)team * C::XB;
    const int c = blockIdx.x, rep = blockIdx.y;
    const int M = a.nx / 2;
    const size_t base = ((size_t)rep * a.hx + c) * (size_t)N * N;
    const float2* __restrict__ tw = a.tw_a;
    const bool plane = (c == 0 || c == M);

    // modes: STEP (primal, with noise); TAN (tangent only: dphi <- f1 dphi + A M s DFT[q']);
    // ADJ (lam <- f1 lam + M DFT[v], then W = IDFT(A s M lam / N^3)); ADJ_PRIME (W from lam only)
    constexpr bool DIFF = (MODE == MODE_TAN || MODE == MODE_ADJ || MODE == MODE_ADJ_PRIME);
    const float2* qsrc = DIFF ? a.dqin : a.qin;
    float2* state = DIFF ? a.dphi : a.phi;
    float2* pdst = DIFF ? a.dpout : a.pout;
    if constexpr (MODE == MODE_FWD || MODE == MODE_STEP || MODE == MODE_TAN || MODE == MODE_ADJ) {
        const bool has_f = (MODE == MODE_FWD) || c < a.ncols;
        block_copy<C::THREADS, N * N>(
            N * N, [&](int f) { return has_f ? qsrc[base + f] : czero(); },
            [&](int f, float2 v) { S[(f / N) * RS + f % N] = v; });
        __syncthreads();
        if (has_f) {
            plane_fft<N, true, false>(S, xb, team, t, tw);
            __syncthreads();
            plane_fft<N, false, false>(S, xb, team, t, tw);
            __syncthreads();
        }
    } else {
        // INV / PRIME / ADJ_PRIME: the state goes straight to the inverse transforms
        block_copy<C::THREADS, N * N>(
            N * N, [&](int f) { return state[base + f]; }, [&](int f, float2 v) { S[(f / N) * RS + f % N] = v; });
        __syncthreads();
    }

    if constexpr (MODE == MODE_STEP || MODE == MODE_TAN || MODE == MODE_ADJ) {
        const long long step = current_step(a);
        const bool first = (MODE == MODE_STEP || MODE == MODE_TAN) && (a.scheme == 2) && (step == *a.first_step);
        const bool has_f = c < a.ncols;
        for (int it = 0; it < C::ITERS; ++it) {
            const int line = team + it * C::TEAMS;
            const int az = line < N ? line : N - 1;
            const int azs = signed_idx(az, N);
#pragma unroll
            for (int e = 0; e < E; e += 2) {
                float2 zz[2] = {czero(), czero()};
                // Fourier-space draw, unless the step reads the transformed real-space draw (noise_in)
                if constexpr (MODE == MODE_STEP) {
                    if (!a.noise_in)
                        team_normal_pair_ks<T>(a.ks, ((uint64_t)c * N + az) * N, t, e, (uint32_t)step,
                                               (uint32_t)(a.rep0 + rep), zz[0], zz[1]);
                }
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int ay = t + T * (e + h);
                    const int ays = signed_idx(ay, N);
                    const int q = c * c + ays * ays + azs * azs;
                    const bool inm = !a.dealias || (3 * c < a.nx && 3 * abs(ays) < N && 3 * abs(azs) < N);
                    const float2 Fh = (has_f && inm) ? S[az * RS + ay] : czero();
                    const Coefs co = load_coefs<false>(a.tab, q, first);
                    const size_t idx = base + (size_t)az * N + ay;
                    const int mz = (N - az) % N, my = (N - ay) % N;
                    const bool selfc = plane && az == mz && ay == my;
                    float2 o;
                    if constexpr (MODE == MODE_STEP) {
                        const float2 F = cscale(Fh, nl_prefactor(a, q).x);
                        float2 Fp = czero();
                        if (a.scheme == 2 && has_f) Fp = a.fprev[idx];
                        float2 eta;
                        if (a.noise_in) {
                            // real-space noise (Sec. IV step 2): eta_a = DFT[eta]_a / sqrt(N^3)
                            const float2 nv = a.noise_in[idx];
                            eta = make_float2(nv.x * a.noise_scale, selfc ? 0.f : nv.y * a.noise_scale);
                        } else {
                            eta = eta_of(zz[h], selfc);
                        }
                        o = setd_update<false>(co, state[idx], F, Fp, eta);
                        if (line < N && a.scheme == 2 && has_f) a.fprev[idx] = F;
                    } else if constexpr (MODE == MODE_TAN) {
                        // SETD2: B dF_prev with the tangent's own history (zero at the seed)
                        const float2 dF = cscale(Fh, nl_prefactor(a, q).x);
                        float2 dFp = czero();
                        if (a.scheme == 2 && has_f) dFp = a.dfprev[idx];
                        o = setd_update<false>(co, state[idx], dF, dFp, czero());
                        if (line < N && a.scheme == 2 && has_f) a.dfprev[idx] = dF;
                    } else {
                        // adjoint of step n: lam_n = f1 lam_{n+1} + M DFT[v]; SETD2: mu_{n-1} = B_n lam_{n+1}
                        const float2 l = state[idx];
                        o = make_float2(co.f1.x * l.x + Fh.x, co.f1.x * l.y + Fh.y);
                        if (a.scheme == 2 && line < N)
                            a.dmu[idx] = a.adj_first_n ? czero() : cscale(l, __ldg(&a.tab[q]).z);
                    }
                    if (selfc) o.y = 0.f;
                    if (line < N) S[az * RS + ay] = o;
                }
            }
        }
        __syncthreads();
        if (plane) {
            // partners take the conjugate of their canonical mode (canonical entries are not written here)
            for (int f = threadIdx.x; f < N * N; f += blockDim.x) {
                const int az = f / N, ay = f % N;
                const int mz = (N - az) % N, my = (N - ay) % N;
                if (az > mz || (az == mz && ay > my)) S[az * RS + ay] = cconj(S[mz * RS + my]);
            }
            __syncthreads();
        }
        for (int f = threadIdx.x; f < N * N; f += blockDim.x) {
            const int az = f / N, ay = f % N;
            const float2 o = S[az * RS + ay];
            state[base + f] = o;
            if (MODE == MODE_STEP) flag_nonfinite(a, o, step);
        }
    }
    if constexpr (MODE == MODE_FWD) {
        if (plane) {
            for (int f = threadIdx.x; f < N * N; f += blockDim.x) {
                const int az = f / N, ay = f % N;
                const int mz = (N - az) % N, my = (N - ay) % N;
                if (az > mz || (az == mz && ay > my)) S[az * RS + ay] = cconj(S[mz * RS + my]);
                if (az == mz && ay == my) S[az * RS + ay].y = 0.f;
            }
            __syncthreads();
        }
        block_copy<C::THREADS, N * N>(
            N * N, [&](int f) { return S[(f / N) * RS + f % N]; }, [&](int f, float2 v) { a.phi[base + f] = v; });
        return;
    } else {
        // inverse transforms of M phi / N^3 (INV: no mask; adjoint: times A s) -> row-pass input
        const bool emit = (MODE == MODE_INV) || c < a.ncols;
        if (!emit) return;  // whole block
        __syncthreads();
        for (int f = threadIdx.x; f < N * N; f += blockDim.x) {
            const int az = f / N, ay = f % N;
            const int ays = signed_idx(ay, N), azs = signed_idx(az, N);
            const bool inm = (MODE == MODE_INV) || !a.dealias || (3 * c < a.nx && 3 * abs(ays) < N && 3 * abs(azs) < N);
            float w = a.scale;
            float2 o = S[az * RS + ay];
            if constexpr (MODE == MODE_ADJ || MODE == MODE_ADJ_PRIME) {
                // W = IDFT(M s (A_{n-1} lam_n + mu_{n-1}) / N^3); ADJ_PRIME: mu = 0
                const int q = c * c + ays * ays + azs * azs;
                const Coefs co = load_coefs<false>(a.tab, q, a.adj_first_prev != 0);
                o = cscale(o, co.A.x);
                if (MODE == MODE_ADJ && a.scheme == 2) o = cadd(o, a.dmu[base + f]);
                w *= nl_prefactor(a, q).x;
            }
            S[az * RS + ay] = inm ? cscale(o, w) : czero();
        }
        __syncthreads();
        plane_fft<N, false, true>(S, xb, team, t, tw);
        __syncthreads();
        plane_fft<N, true, true>(S, xb, team, t, tw);
        __syncthreads();
        block_copy<C::THREADS, N * N>(
            N * N, [&](int f) { return S[(f / N) * RS + f % N]; }, [&](int f, float2 v) { pdst[base + f] = v; });
    }
}

// Phase-shift dealiasing in 3-D (the alternative of Sec. IV step 1): the nonlinear term is the mean over the 8 grids
// shifted by half a cell along every subset of the axes.  The row pass runs over four copies of P, one per shift
// (s_y, s_z) of the y and z axes (copy s_y + 2 s_z at ps_off (s_y + 2 s_z) behind P), each row averaged over its two
// x shifts; this plane pass combines the four copies of Q,
//   F = M s (1/4) sum_{s_y, s_z} e^{-i pi (s_y a_y + s_z a_z) / N} DFT_yz[Q_{s_y, s_z}],
// updates (Fourier noise, as the plain step) and emits the four copies P_{s_y, s_z} = IDFT_yz(M phi
// e^{+i pi (s_y a_y + s_z a_z) / N} / N^3) for the next row pass.  M keeps every mode off the Nyquist planes.  Two
// planes of shared memory (the work plane and the accumulated force, then the new state): planes up to 64^2.
// STEP = false (prime): the emission only, from the current state.
__device__ __forceinline__ float2 ps_phase_conj(const float2* __restrict__ tw_ps, int s) {
    const float2 w = __ldg(&tw_ps[abs(s)]);  // e^{-i pi |s| / N}
    return s >= 0 ? w : cconj(w);
}

template <int N, bool STEP>
__global__ void __launch_bounds__(PlaneCfg<N>::THREADS) k3_planes_ps(const StepArgs a) {
    using C = PlaneCfg<N>;
    using PL = FftPlan<N>;
    constexpr int T = PL::T, E = PL::E, RS = C::RS;
    static_assert(N <= 64, "two planes of shared memory");
    extern __shared__ float2 sm[];
    float2* S = sm;
    float2* A = sm + (size_t)N * RS;
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    float2* xb = sm + 2 * (size_t)N * RS + (size_t)team * C::XB;
    const int c = blockIdx.x, rep = blockIdx.y;
    const int M = a.nx / 2;
    const size_t base = ((size_t)rep * a.hx + c) * (size_t)N * N;
    const float2* __restrict__ tw = a.tw_a;
    const float2* __restrict__ tps = a.tw_ps;
    const bool plane = (c == 0 || c == M);
    const bool has_f = c < a.ncols;  // every x-mode but the Nyquist one
    // the phase e^{-i pi (s_y a_y + s_z a_z) / N} of copy cp = s_y + 2 s_z at plane entry (az, ay)
    auto phase = [&](int cp, int az, int ay) {
        float2 ph = make_float2(1.f, 0.f);
        if (cp & 1) ph = ps_phase_conj(tps, signed_idx(ay, N));
        if (cp & 2) ph = cmul(ph, ps_phase_conj(tps, signed_idx(az, N)));
        return ph;
    };
    if constexpr (STEP) {
        for (int f = threadIdx.x; f < N * N; f += blockDim.x) A[(f / N) * RS + f % N] = czero();
        __syncthreads();
        if (has_f) {
            for (int cp = 0; cp < 4; ++cp) {
                const float2* q = a.qin + (size_t)cp * a.ps_off + base;
                block_copy<C::THREADS, N * N>(
                    N * N, [&](int f) { return q[f]; }, [&](int f, float2 v) { S[(f / N) * RS + f % N] = v; });
                __syncthreads();
                plane_fft<N, true, false>(S, xb, team, t, tw);
                __syncthreads();
                plane_fft<N, false, false>(S, xb, team, t, tw);
                __syncthreads();
                for (int f = threadIdx.x; f < N * N; f += blockDim.x) {
                    const int az = f / N, ay = f % N;
                    A[az * RS + ay] = cadd(A[az * RS + ay], cmul(S[az * RS + ay], phase(cp, az, ay)));
                }
                __syncthreads();
            }
        }
        const long long step = current_step(a);
        const bool first = (a.scheme == 2) && (step == *a.first_step);
        for (int it = 0; it < C::ITERS; ++it) {
            const int line = team + it * C::TEAMS;
            const int az = line < N ? line : N - 1;
            const int azs = signed_idx(az, N);
#pragma unroll
            for (int e = 0; e < E; e += 2) {
                float2 zz[2];
                team_normal_pair_ks<T>(a.ks, ((uint64_t)c * N + az) * N, t, e, (uint32_t)step,
                                       (uint32_t)(a.rep0 + rep), zz[0], zz[1]);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int ay = t + T * (e + h);
                    const int ays = signed_idx(ay, N);
                    const int q = c * c + ays * ays + azs * azs;
                    const bool inm = has_f && 2 * abs(ays) != N && 2 * abs(azs) != N;
                    const float2 F = inm ? cscale(A[az * RS + ay], 0.25f * nl_prefactor(a, q).x) : czero();
                    const Coefs co = load_coefs<false>(a.tab, q, first);
                    const size_t idx = base + (size_t)az * N + ay;
                    const int mz = (N - az) % N, my = (N - ay) % N;
                    const bool selfc = plane && az == mz && ay == my;
                    float2 Fp = czero();
                    if (a.scheme == 2 && has_f) Fp = a.fprev[idx];
                    float2 o = setd_update<false>(co, a.phi[idx], F, Fp, eta_of(zz[h], selfc));
                    if (line < N && a.scheme == 2 && has_f) a.fprev[idx] = F;
                    if (selfc) o.y = 0.f;
                    if (line < N) A[az * RS + ay] = o;
                }
            }
        }
        __syncthreads();
        if (plane) {
            for (int f = threadIdx.x; f < N * N; f += blockDim.x) {
                const int az = f / N, ay = f % N;
                const int mz = (N - az) % N, my = (N - ay) % N;
                if (az > mz || (az == mz && ay > my)) A[az * RS + ay] = cconj(A[mz * RS + my]);
            }
            __syncthreads();
        }
        for (int f = threadIdx.x; f < N * N; f += blockDim.x) {
            const float2 o = A[(f / N) * RS + f % N];
            a.phi[base + f] = o;
            flag_nonfinite(a, o, step);
        }
    } else {
        block_copy<C::THREADS, N * N>(
            N * N, [&](int f) { return a.phi[base + f]; }, [&](int f, float2 v) { A[(f / N) * RS + f % N] = v; });
    }
    if (!has_f) return;  // whole block: P carries the x-modes off the Nyquist one
    for (int cp = 0; cp < 4; ++cp) {
        __syncthreads();
        for (int f = threadIdx.x; f < N * N; f += blockDim.x) {
            const int az = f / N, ay = f % N;
            const bool inm = 2 * abs(signed_idx(ay, N)) != N && 2 * abs(signed_idx(az, N)) != N;
            S[az * RS + ay] = inm ? cscale(cmul(A[az * RS + ay], cconj(phase(cp, az, ay))), a.scale) : czero();
        }
        __syncthreads();
        plane_fft<N, false, true>(S, xb, team, t, tw);
        __syncthreads();
        plane_fft<N, true, true>(S, xb, team, t, tw);
        __syncthreads();
        float2* dst = a.pout + (size_t)cp * a.ps_off + base;
        block_copy<C::THREADS, N * N>(
            N * N, [&](int f) { return S[(f / N) * RS + f % N]; }, [&](int f, float2 v) { dst[f] = v; });
    }
}

template <int N, bool STEP>
static cudaError_t run_planes_ps(const StepArgs& a, cudaStream_t s) {
    using C = PlaneCfg<N>;
    const size_t sm = C::smem() + sizeof(float2) * (size_t)N * C::RS;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k3_planes_ps<N, STEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k3_planes_ps<N, STEP><<<dim3(a.hx, a.R), C::THREADS, sm, s>>>(a);
    return cudaGetLastError();
}

template <int N>
static cudaError_t planes_ps_for(const StepArgs& a, int mode, cudaStream_t s) {
    if (mode == MODE_STEP) return run_planes_ps<N, true>(a, s);
    if (mode == MODE_PRIME) return run_planes_ps<N, false>(a, s);
    return cudaErrorInvalidValue;
}

template <int N, int MODE>
static cudaError_t run_planes(const StepArgs& a, cudaStream_t s) {
    using C = PlaneCfg<N>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e =
            cudaFuncSetAttribute(k3_planes<N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem());
        if (e != cudaSuccess) return e;
        attr = true;
    }
    k3_planes<N, MODE><<<dim3(a.hx, a.R), C::THREADS, C::smem(), s>>>(a);
    return cudaGetLastError();
}

template <int N>
static cudaError_t planes_for(const StepArgs& a, int mode, cudaStream_t s) {
    switch (mode) {
        case MODE_STEP: return run_planes<N, MODE_STEP>(a, s);
        case MODE_FWD: return run_planes<N, MODE_FWD>(a, s);
        case MODE_INV: return run_planes<N, MODE_INV>(a, s);
        case MODE_PRIME: return run_planes<N, MODE_PRIME>(a, s);
        case MODE_TAN: return run_planes<N, MODE_TAN>(a, s);
        case MODE_ADJ: return run_planes<N, MODE_ADJ>(a, s);
        case MODE_ADJ_PRIME: return run_planes<N, MODE_ADJ_PRIME>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

bool k3_supported(int nx, int ny, int nz, int complex_field) {
    if (complex_field || ny != nz) return false;
    auto ok = [](int n) { return n == 16 || n == 32 || n == 64 || n == 128; };
    return ok(ny) && nx >= 16 && nx <= 4096 && (nx & (nx - 1)) == 0;
}

cudaError_t launch_k3_planes(const StepArgs& a, int mode, int nl, cudaStream_t s) {
    if (nl != NL_CUBIC) return cudaErrorInvalidValue;
    if (a.pshift && (mode == MODE_STEP || mode == MODE_PRIME)) {
        if (!a.tw_ps) return cudaErrorInvalidValue;
        switch (a.ny) {
            case 16: return planes_ps_for<16>(a, mode, s);
            case 32: return planes_ps_for<32>(a, mode, s);
            case 64: return planes_ps_for<64>(a, mode, s);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (a.ny) {
        case 16: return planes_for<16>(a, mode, s);
        case 32: return planes_for<32>(a, mode, s);
        case 64: return planes_for<64>(a, mode, s);
        case 128: return planes_for<128>(a, mode, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
