// sft_k2d_pipe.cu -- persistent, bulk-copy pipelined column pass of the 2-D
// step (real fields, columns of 1024 points and longer).
//
// Same arithmetic as the column pass of sft_k2d.cu (forward FFT along y of
// the row-pass output, SETD update with Philox noise, Hermitian fix-up,
// dealiased inverse FFT), organised for latency hiding: one CTA per SM, each
// team of T threads walks a strided list of (column, replica) items and keeps
// two shared-memory stages; while it computes item k, the next item's row-pass
// column and state column stream in with cp.async.bulk, completing on a
// per-stage mbarrier.  Waits are bounded (StepArgs::wait_limit): a wait that
// runs out sets status bit 1 (time-out), lets its copies in flight land
// (bounded) and stops.
#include "sft_async.cuh"
#include "sft_step_common.cuh"

namespace sft {

template <int NY>
struct ColPipeCfg {
    using PL = FftPlan<NY, 32>;
    static constexpr int T = PL::T;
    static_assert(T >= 32, "pipelined column pass needs whole-warp teams");
    static constexpr int TEAMS = T >= 128 ? 1 : (T == 64 ? 3 : 6);
    static constexpr int THREADS = TEAMS * T;
    static constexpr int QB = (PL::BUF + 1) & ~1;  // row-pass column + exchange buffer (16-byte multiple)
    static constexpr int STAGE = QB + NY;          // + state column
    static constexpr int BARB = 16 * ((2 * TEAMS * 8 + 15) / 16);
    static constexpr size_t smem() { return BARB + sizeof(float2) * (size_t)TEAMS * 2 * STAGE; }
};

template <int NY, int NL>
__global__ void __launch_bounds__(ColPipeCfg<NY>::THREADS, 1) k2_cols_pipe(const StepArgs a) {
    using C = ColPipeCfg<NY>;
    using PL = FftPlan<NY, 32>;
    constexpr int T = C::T, E = PL::E, TEAMS = C::TEAMS, QB = C::QB;
    extern __shared__ __align__(16) unsigned char smraw[];
    uint64_t* bars = reinterpret_cast<uint64_t*>(smraw);
    float2* region = reinterpret_cast<float2*>(smraw + C::BARB);
    const int team = threadIdx.x / T, t = threadIdx.x % T;
    float2* stage[2] = {region + (size_t)team * 2 * C::STAGE, region + (size_t)team * 2 * C::STAGE + C::STAGE};
    uint64_t* bar = bars + 2 * team;
    __shared__ unsigned team_abort[TEAMS];
    const long long total = (long long)a.hx * a.R;
    const long long G = (long long)gridDim.x * TEAMS;
    const long long g = (long long)blockIdx.x * TEAMS + team;
    if (g >= total) return;  // whole team
    const long long step = current_step(a);
    const bool first = (a.scheme == 2) && (step == *a.first_step);
    const int M = a.nx / 2;
    const float2* __restrict__ tw = a.tw_a;

    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        team_abort[team] = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    team_sync<T>();

    auto issue = [&](long long i, int s) {
        const int c = (int)(i / a.R), r = (int)(i % a.R);
        const size_t colbase = ((size_t)r * a.hx + c) * NY;
        const bool hf = c < a.ncols;
        mbar_arrive_expect_tx(&bar[s], (uint32_t)(NY * sizeof(float2) * (hf ? 2 : 1)));
        bulk_load(stage[s] + QB, a.phi + colbase, NY * sizeof(float2), &bar[s]);
        if (hf) bulk_load(stage[s], a.qin + colbase, NY * sizeof(float2), &bar[s]);
    };
    if (t == 0) issue(g, 0);

    for (long long k = 0;; ++k) {
        const long long i = g + k * G;
        if (i >= total) break;
        const int s = (int)(k & 1);
        fence_proxy_async_smem();
        team_sync<T>();  // the team is done with the other stage
        if (t == 0 && i + G < total) issue(i + G, 1 - s);
        if (!mbar_wait_bounded(&bar[s], (uint32_t)((k >> 1) & 1), wait_iters(a))) atomicOr(&team_abort[team], 1u);
        team_sync<T>();
        if (team_abort[team]) {
            // report the time-out, let both stages' copies in flight land (bounded waits) and stop
            if (t == 0) {
                atomicOr(a.status, 2u);
                mbar_wait_bounded(&bar[s], (uint32_t)((k >> 1) & 1));
                if (i + G < total) mbar_wait_bounded(&bar[1 - s], (uint32_t)(((k + 1) >> 1) & 1));
            }
            return;
        }
        const int c = (int)(i / a.R), rep = (int)(i % a.R);
        const size_t colbase = ((size_t)rep * a.hx + c) * NY;
        const bool has_f = c < a.ncols;
        const bool plane = (c == 0 || c == M);
        float2* Qs = stage[s];
        const float2* Ps = stage[s] + QB;
        float2 v[E];
        if (has_f) {
#pragma unroll
            for (int e = 0; e < E; ++e) v[e] = Qs[t + T * e];
            fft_line<NY, false, 32>(v, Qs, t, tw);
        }
        float2 out[E];
#pragma unroll
        for (int e = 0; e < E; ++e) {
            if ((e & 1) == 0)
                team_normal_pair_ks<T>(a.ks, (uint64_t)c * NY, t, e, (uint32_t)step, (uint32_t)(a.rep0 + rep), out[e],
                                    out[e + 1]);
            const int ay = t + T * e;
            const int ays = signed_idx(ay, NY);
            const int q = c * c + ays * ays;
            const bool inm = !a.dealias || (3 * c < a.nx && 3 * abs(ays) < NY);
            float2 F = czero();
            if (has_f && inm) F = cscale(v[e], nl_prefactor(a, q).x);
            const Coefs co = load_coefs<false>(a.tab, c * (NY / 2 + 1) + abs(ays), first);
            float2 Fp = czero();
            if (a.scheme == 2 && has_f) Fp = a.fprev[colbase + ay];
            const bool selfc = plane && (ay == 0 || 2 * ay == NY);
            out[e] = setd_update<false>(co, Ps[ay], F, Fp, eta_of(out[e], selfc));
            if (a.scheme == 2 && has_f) a.fprev[colbase + ay] = F;
        }
        if (plane) {
            team_sync<T>();
#pragma unroll
            for (int e = 0; e < E; ++e) Qs[xpos<NY, 32>(t + T * e)] = out[e];
            team_sync<T>();
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ay = t + T * e;
                if (2 * ay > NY) out[e] = cconj(Qs[xpos<NY, 32>(NY - ay)]);
                if (ay == 0 || 2 * ay == NY) out[e].y = 0.f;
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            a.phi[colbase + t + T * e] = out[e];
            flag_nonfinite(a, out[e], step);
        }
        if (has_f) {
            float2 vy[NL == NL_GRAD2 ? E : 1];
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int ay = t + T * e;
                const bool inm = !a.dealias || (3 * c < a.nx && 3 * abs(signed_idx(ay, NY)) < NY);
                v[e] = inm ? cscale(out[e], a.scale) : czero();
                if constexpr (NL == NL_GRAD2) vy[e] = cscale(cmuli(v[e]), a.dk * (float)odd_idx(ay, NY));
            }
            fft_line<NY, true, 32>(v, Qs, t, tw);
            if constexpr (NL == NL_GRAD2) fft_line<NY, true, 32>(vy, Qs, t, tw);
#pragma unroll
            for (int e = 0; e < E; ++e) {
                a.pout[colbase + t + T * e] = v[e];
                if constexpr (NL == NL_GRAD2) a.pyout[colbase + t + T * e] = vy[e];
            }
        }
    }
}

template <int NY, int NL>
static cudaError_t run_pipe(const StepArgs& a, cudaStream_t s) {
    using C = ColPipeCfg<NY>;
    static int nsm = 0;
    if (!nsm) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k2_cols_pipe<NY, NL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::smem());
        if (e != cudaSuccess) {
            nsm = 0;
            return e;
        }
    }
    k2_cols_pipe<NY, NL><<<nsm, C::THREADS, C::smem(), s>>>(a);
    return cudaGetLastError();
}

bool k2_pipe_supported(int nx, int ny, int complex_field) {
    (void)nx;
    return !complex_field && (ny == 1024 || ny == 2048 || ny == 4096);
}

cudaError_t launch_k2_cols_pipe(const StepArgs& a, int nl, cudaStream_t s) {
    if (nl != NL_CUBIC && nl != NL_GRAD2) return cudaErrorInvalidValue;
    switch (a.ny) {
        case 1024: return nl == NL_CUBIC ? run_pipe<1024, NL_CUBIC>(a, s) : run_pipe<1024, NL_GRAD2>(a, s);
        case 2048: return nl == NL_CUBIC ? run_pipe<2048, NL_CUBIC>(a, s) : run_pipe<2048, NL_GRAD2>(a, s);
        case 4096: return nl == NL_CUBIC ? run_pipe<4096, NL_CUBIC>(a, s) : run_pipe<4096, NL_GRAD2>(a, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace sft
