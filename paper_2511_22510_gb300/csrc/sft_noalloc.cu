// sft_noalloc.cu -- a 2-D step entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: code that runs where the allocator is
// owned by someone else (an embedding runtime with its own pool, a plug-in
// that must not grow the device footprint after start-up, a real-time loop
// where an allocation may stall).  sft_step2d_noalloc serves them: the caller
// passes the state (and the SETD2 history) in device memory it owns, and all
// scratch the two-pass 2-D step needs -- the row/column intermediates, the
// coefficient table, the twiddle tables, the step counter and the status word
// -- lives in one file-scope device array of fixed size, below.
//
// That array exists once per GPU that loads this library and stays allocated
// until the process exits.  Its address is looked up once per device, with the
// device current, on that device's first call (cudaGetSymbolAddress); make
// that first call before any stream capture.  The address is kept for the rest
// of the process, so the entry point must not be called after anything that
// destroys the device's primary context (cudaDeviceReset): the module is then
// loaded again elsewhere and the kept address is stale.  Every call shares the
// array and it keeps the previous call's contents, so calls whose work
// overlaps on the GPU (different streams, or different host threads on one
// stream without ordering) race on it: order them.
//
// A configuration passes the same checks as sft_create (validate_config) and
// then the limits of the scratch below.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>
#include <string>

#include "../../include/sft.h"
#include "sft_internal.h"

namespace sft {
namespace {

// limits of the scratch (see include/sft.h)
constexpr int kNoAllocMaxN = 512;             // points per axis
constexpr long long kNoAllocMaxModes = 1 << 18;  // R * (nx/2 + 1) * ny, per intermediate
constexpr long long kTabMax = (long long)(kNoAllocMaxN / 2 + 1) * (kNoAllocMaxN / 2 + 1);
constexpr long long kTwMax = 3 * kNoAllocMaxN;

// byte offsets inside the scratch array (all 256-byte aligned)
constexpr size_t kOffP = 0;
constexpr size_t kOffQ = kOffP + sizeof(float2) * kNoAllocMaxModes;
constexpr size_t kOffPy = kOffQ + sizeof(float2) * kNoAllocMaxModes;
constexpr size_t kOffTab = kOffPy + sizeof(float2) * kNoAllocMaxModes;
constexpr size_t kOffTw = kOffTab + sizeof(float4) * ((kTabMax + 15) / 16 * 16);
constexpr size_t kOffCnt = kOffTw + sizeof(float2) * ((kTwMax + 31) / 32 * 32);
constexpr size_t kScratchBytes = kOffCnt + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mu;
unsigned char* g_addr[64] = {nullptr};

// counters: [0] step base, [1] SETD2 first step, [2] bad step; status word after them
__global__ void k_noalloc_counters(long long* cnt, unsigned* status, long long step0, long long first) {
    cnt[0] = step0;
    cnt[1] = first;
    cnt[2] = 0x7fffffffffffffffLL;
    *status = 0u;
}

}  // namespace
sft_status validate_config(const sft_config* cfg, std::string& why);  // sft_api.cu: the checks of sft_create
}  // namespace sft

using namespace sft;

extern "C" sft_status sft_step2d_noalloc(const sft_config* cfg, void* phi_dev, void* fprev_dev, int history_valid,
                                         int64_t step0, int64_t nsteps) {
    if (!cfg || !phi_dev || nsteps < 0 || step0 < 0) return SFT_EINVAL;
    std::string why;
    const sft_status vs = validate_config(cfg, why);
    if (vs != SFT_OK) {
        fprintf(stderr, "sft_step2d_noalloc: %s\n", why.c_str());
        return vs;
    }
    // the variants this entry point carries: 2-D real fields (Model A/B, KPZ), power-of-two sizes,
    // Fourier-space noise, 2/3 truncation or none
    if (cfg->d != 2 || cfg->model == SFT_CGL || cfg->model == SFT_CUSTOM || cfg->noise_space != 0 || cfg->dealias == 2 ||
        (cfg->n[0] & (cfg->n[0] - 1)) != 0) {
        fprintf(stderr, "sft_step2d_noalloc: built for 2-D real fields (Model A, Model B, KPZ) of power-of-two sizes "
                        "with Fourier-space noise and 2/3 truncation or none\n");
        return SFT_EUNSUPPORTED;
    }
    const int nx = cfg->n[0], ny = cfg->n[1];
    if (nx > kNoAllocMaxN) {
        fprintf(stderr, "sft_step2d_noalloc: %d points per axis is above the scratch limit of %d\n", nx, kNoAllocMaxN);
        return SFT_EINVAL;
    }
    if (cfg->scheme == SFT_SETD2 && !fprev_dev) {
        fprintf(stderr, "sft_step2d_noalloc: SETD2 needs the history buffer fprev_dev\n");
        return SFT_EINVAL;
    }
    const int hx = nx / 2 + 1;
    const long long modes = (long long)cfg->replicas * hx * ny;
    if (modes > kNoAllocMaxModes) {
        fprintf(stderr, "sft_step2d_noalloc: R (n/2 + 1) n = %lld modes is above the scratch limit of %lld\n", modes,
                kNoAllocMaxModes);
        return SFT_EINVAL;
    }
    if (step0 + nsteps > (long long)0xFFFFFFFFLL) {
        fprintf(stderr, "sft_step2d_noalloc: step0 + nsteps must stay below 2^32 (the noise counter)\n");
        return SFT_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)cfg->stream;

    // once per device, with that device current: the scratch array's device address
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SFT_ECUDA;
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (!g_addr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return SFT_ECUDA;
            g_addr[dev] = (unsigned char*)p;
        }
        base = g_addr[dev];
    }
    float2* P = (float2*)(base + kOffP);
    float2* Q = (float2*)(base + kOffQ);
    float2* Py = (float2*)(base + kOffPy);
    float4* tab = (float4*)(base + kOffTab);
    float2* tw = (float2*)(base + kOffTw);
    long long* cnt = (long long*)(base + kOffCnt);
    unsigned* status = (unsigned*)(base + kOffCnt + 4 * sizeof(long long));

    // per-call set-up inside the scratch (it keeps the last call's contents)
    const int nl = cfg->model == SFT_KPZ ? NL_GRAD2 : NL_CUBIC;
    // twiddle tables of the three transform lengths, by the builder sft_create uses
    if (launch_twiddles(tw, nx / 2, st) != cudaSuccess || launch_twiddles(tw + nx / 2, nx, st) != cudaSuccess ||
        launch_twiddles(tw + nx / 2 + nx, ny, st) != cudaSuccess)
        return SFT_ECUDA;
    const float2* twM = tw;
    const float2* twN = tw + nx / 2;
    const float2* twY = tw + nx / 2 + nx;
    TableArgs t{};
    t.model = cfg->model;
    t.scheme = cfg->scheme;
    t.complex_field = 0;
    t.d = 2;
    t.hy = ny / 2 + 1;
    for (int i = 0; i < 8; ++i) t.p[i] = cfg->p[i];
    t.h = cfg->h;
    t.dk = 2.0 * M_PI / (nx * cfg->dx[0]);
    t.noise_norm = std::sqrt(nx / cfg->dx[0]) * std::sqrt(ny / cfg->dx[1]);
    t.nq = (long long)(nx / 2 + 1) * (ny / 2 + 1);
    t.out = tab;
    if (launch_build_table(t, st) != cudaSuccess) return SFT_ECUDA;
    const long long first = (cfg->scheme == SFT_SETD2 && !history_valid) ? step0 : -1;
    k_noalloc_counters<<<1, 1, 0, st>>>(cnt, status, step0, first);

    StepArgs a{};
    a.nx = nx;
    a.ny = ny;
    a.nz = 1;
    a.hx = hx;
    int mx = 0;
    for (int c = 0; c < hx; ++c)
        if (!cfg->dealias || 3 * c < nx) mx = c + 1;
    a.ncols = mx;
    a.R = cfg->replicas;
    a.rep0 = cfg->replica0;
    a.scale = (float)(1.0 / ((double)nx * ny));
    a.dk = (float)t.dk;
    a.dealias = cfg->dealias;
    a.model = cfg->model;
    a.scheme = cfg->scheme;
    a.s0 = cfg->model == SFT_KPZ ? (float)(0.5 * cfg->p[1]) : (float)(-cfg->p[0] * cfg->p[2]);
    a.s0i = 0.f;
    a.seed = cfg->seed;
    philox_key_schedule(a.seed, a.ks);
    a.tab = tab;
    a.phi = (float2*)phi_dev;
    a.fprev = (float2*)fprev_dev;
    a.step_base = cnt;
    a.first_step = cnt + 1;
    a.status = status;
    a.bad_step = cnt + 2;

    // P (and P_y) from the caller's state, then nsteps row + column passes
    StepArgs pr = a;
    pr.pout = P;
    pr.pyout = Py;
    pr.tw_a = twY;
    if (launch_k2_cols(pr, MODE_PRIME, nl, st) != cudaSuccess) return SFT_ECUDA;
    for (int64_t i = 0; i < nsteps; ++i) {
        StepArgs r = a;
        r.pin = P;
        r.pyin = Py;
        r.qout = Q;
        r.tw_a = twM;
        r.tw_b = twN;
        if (launch_k2_rows(r, MODE_STEP, nl, st) != cudaSuccess) return SFT_ECUDA;
        StepArgs c = a;
        c.qin = Q;
        c.pout = P;
        c.pyout = Py;
        c.tw_a = twY;
        if (launch_k2_cols(c, MODE_STEP, nl, st) != cudaSuccess) return SFT_ECUDA;
        if (launch_advance(cnt, 1, st) != cudaSuccess) return SFT_ECUDA;
    }
    unsigned hs = 0;
    if (cudaMemcpyAsync(&hs, status, sizeof hs, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return SFT_ECUDA;
    return (hs & 1u) ? SFT_ENONFINITE : SFT_OK;
}
