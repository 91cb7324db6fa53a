// sft_api.cu -- host runtime behind the C ABI of include/sft.h: context and
// buffer management, the per-step launch sequence, CUDA-graph chunks of steps,
// observables, checkpoints and error reporting.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/sft.h"
#include "sft_internal.h"

namespace sft {
// complex 2-D step on columns of 1024 or 2048 points, one warp per 1024 points (sft_k2c_colwarp.cu)
bool k2c_colwarp_supported(int ny);
cudaError_t launch_k2c_cols_warp(const StepArgs& a, cudaStream_t s);
bool k2c_rowwarp_supported(int nx, int ny, int dealias);
cudaError_t launch_k2c_rows_warp(const StepArgs& a, cudaStream_t s);
}  // namespace sft

using namespace sft;

namespace {

constexpr int kGraphChunk = 16;  // steps per captured graph

struct Twiddles {
    std::vector<int> lens;
    std::vector<size_t> offs;
    float2* dev = nullptr;
    const float2* get(int L) const {
        for (size_t i = 0; i < lens.size(); ++i)
            if (lens[i] == L) return dev + offs[i];
        return nullptr;
    }
};

}  // namespace

struct sft_ctx {
    sft_config cfg{};
    int d = 0, nx = 1, ny = 1, nz = 1;
    int cplx = 0, nl = NL_CUBIC;
    int hx = 0, mx = 0;
    long long sites = 0, nmodes = 0;
    int R = 0;
    int rep0 = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // device buffers
    float2 *phi = nullptr, *fprev = nullptr, *P = nullptr, *Q = nullptr, *Py = nullptr, *snap = nullptr;
    float* real = nullptr;
    float2* cfield = nullptr;
    float4* tab = nullptr;
    long long* dstep = nullptr;   // [0] step base, [1] SETD2 first step, [2] bad step
    unsigned* dstatus = nullptr;
    double* dshell = nullptr;
    double* drough = nullptr;
    // observation: the stored modes shell by shell, cut into chunks (ObsArgs), chunk partials, and the
    // device time accumulator of S(k, t) (compensated pairs) with its sample count
    int* d_order = nullptr;
    int4* d_chunks = nullptr;
    int* d_first_chunk = nullptr;
    int nchunks = 0;
    double2* d_part = nullptr;
    double2* d_tacc = nullptr;
    long long tacc_count = 0;
    Twiddles tw;
    float2* tw32 = nullptr;  // W_1024^{t k1} for t, k1 < 32 (1024-point warp transforms)
    int wait_limit = 0;      // StepArgs::wait_limit (SFT_WAIT_LIMIT; tests of the time-out path)
    // tangent / adjoint
    float2 *dphi = nullptr, *dseed = nullptr, *dP = nullptr, *dQ = nullptr, *dPy = nullptr;
    float2* dfprev = nullptr;  // SETD2: the tangent's history dF of the previous step
    float2* dmu = nullptr;     // SETD2 adjoint: the cotangent of the history term
    float2 *tcb1 = nullptr, *tcb2 = nullptr;  // precision study: scratch of the tensor-core step
    bool dp_valid = false;
    // host mirrors
    long long step = 0;
    long long first_step = -1;
    bool p_valid = false;
    int nshells = 0;
    std::vector<double> counts;
    cudaGraphExec_t graph = nullptr;
    bool warmed = false;
    int launches_per_step = 0;
    int ckpt_segment = 100;
    long long launches = 0;
    bool pipe_cols = false;  // pipelined (bulk-copy) column pass
    bool pipe_forced = false;  // chosen by SFT_COLUMN_PASS, not by the plan
    // schedule of the step's passes (plan autotuner)
    bool planned = false;
    int row_shape = 0, col_shape = 0, rpb = 0;
    uint64_t cust_hash = 0;  // SFT_CUSTOM: hash of the copied tables (checkpoint compatibility)
    std::vector<double> cust_c, cust_D;  // SFT_CUSTOM: real c and D over |a|^2 (dynamic observables)
    // recording for the dynamic observables
    float2 *rec_phi = nullptr, *rec_F = nullptr;
    long long rec_start = 0;
    // real-space noise: the transformed draw of the current step (R x nmodes)
    float2* noise_spec = nullptr;
    int rec_every = 1, rec_M = 0;
    // batch context: members advanced together (1-D lattices of uneven sizes in one persistent launch)
    bool is_batch = false;
    std::vector<sft_ctx*> members;
    std::vector<long long> rep_offset;  // global replica index of each member's replica 0
    std::vector<int> solo;              // members stepped by their own kernels on a forked branch
    BatchMember* d_members = nullptr;
    BatchItem* d_items = nullptr;
    int nitems = 0;
    int* d_head = nullptr;
    int batch_blocks = 0;
    std::vector<cudaStream_t> sides;   // one forked graph branch per solo member
    std::vector<cudaEvent_t> ev_joins;
    cudaEvent_t ev_fork = nullptr;
    std::string err;
};

static sft_status fail(sft_ctx* c, sft_status s, const std::string& msg) {
    if (c) c->err = msg;
    return s;
}

#define CK(call)                                                                                              \
    do {                                                                                                      \
        cudaError_t e_ = (call);                                                                              \
        if (e_ != cudaSuccess)                                                                                \
            return fail(ctx, SFT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));                  \
    } while (0)

static bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

static long long isqrt_ceil(long long q) {
    long long j = (long long)std::floor(std::sqrt((double)q));
    while (j * j < q) ++j;
    while (j > 0 && (j - 1) * (j - 1) >= q) --j;
    return j;
}

// Field kind and nonlinearity of a configuration.  SFT_CUSTOM without a
// nonlinearity runs the cubic (real) or |A|^2 A (complex) kernels with s = 0.
static void model_kind(const sft_config* c, int* cplx, int* nl) {
    if (c->model == SFT_CUSTOM) {
        *cplx = c->complex_field ? 1 : 0;
        if (c->custom_nl == SFT_NL_GRAD2)
            *nl = NL_GRAD2;
        else if (c->custom_nl == SFT_NL_CGL)
            *nl = NL_CGL;
        else
            *nl = *cplx ? NL_CGL : NL_CUBIC;
        return;
    }
    *cplx = c->model == SFT_CGL;
    *nl = c->model == SFT_KPZ ? NL_GRAD2 : (*cplx ? NL_CGL : NL_CUBIC);
}

// Entries of the SFT_CUSTOM tables: |a|^2 = 0 .. sum_i (n_i/2)^2.
static long long custom_len(const sft_config* c) {
    long long q = 0;
    for (int i = 0; i < c->d; ++i) q += (long long)(c->n[i] / 2) * (c->n[i] / 2);
    return q + 1;
}

static StepArgs base_args(const sft_ctx* c) {
    StepArgs a{};
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz;
    a.hx = c->hx;
    a.ncols = c->mx;
    a.R = c->R;
    a.rep0 = c->rep0;
    a.scale = (float)(1.0 / (double)c->sites);
    a.dk = (float)(2.0 * M_PI / (c->nx * c->cfg.dx[0]));
    a.dealias = c->cfg.dealias == 1;
    a.pshift = c->cfg.dealias == 2;
    a.tw_ps = a.pshift ? c->tw.get(2 * c->nx) : nullptr;
    a.ps_off = (long long)c->R * c->nmodes;
    a.model = c->cfg.model;
    a.scheme = c->cfg.scheme;
    const double* p = c->cfg.p;
    switch (c->cfg.model) {
        case SFT_MODEL_A:
        case SFT_MODEL_B: a.s0 = (float)(-p[0] * p[2]); a.s0i = 0.f; break;
        case SFT_KPZ: a.s0 = (float)(0.5 * p[1]); a.s0i = 0.f; break;
        case SFT_CUSTOM: a.s0 = 1.f; a.s0i = 0.f; break;  // s is folded into the coefficient table
        default: a.s0 = -1.f; a.s0i = (float)(-p[1]); break;
    }
    a.seed = c->cfg.seed;
    philox_key_schedule(a.seed, a.ks);
    a.tab = c->tab;
    a.phi = c->phi;
    a.fprev = c->fprev;
    a.step_base = c->dstep;
    a.first_step = c->dstep + 1;
    a.status = c->dstatus;
    a.bad_step = c->dstep + 2;
    a.rpb = c->rpb;
    a.tw_32 = c->tw32;
    a.wait_limit = c->wait_limit;
    a.tw_c = (c->d == 1 && !c->cplx && k1_cluster_fft_len(c->nx)) ? c->tw.get(k1_cluster_fft_len(c->nx)) : nullptr;
    a.rec_phi = c->rec_phi;
    a.rec_F = c->rec_F;
    a.rec_start = c->rec_start;
    a.rec_n = (long long)c->R * c->nmodes;
    a.rec_every = c->rec_every;
    a.rec_M = c->rec_M;
    return a;
}

// Row pass: in 3-D the pair (z, y) is the row index of the x-major layout.
static cudaError_t launch_rows(const sft_ctx* ctx, StepArgs a, int mode) {
    a.ny = ctx->ny * ctx->nz;
    a.nz = 1;
    if (ctx->cplx) {
        a.tw_a = ctx->tw.get(ctx->nx);
        // the step on complex rows of 1024 or 2048 points under 2/3 truncation: warp-resident transforms
        if (mode == MODE_STEP && ctx->d == 2 && a.tw_32 && !a.pshift &&
            k2c_rowwarp_supported(ctx->nx, ctx->ny, ctx->cfg.dealias))
            return launch_k2c_rows_warp(a, ctx->stream);
        return launch_k2c_rows(a, mode, ctx->stream);
    }
    return launch_k2_rows(a, mode, ctx->nl, ctx->stream, mode == MODE_STEP ? ctx->row_shape : 0);
}

// Second pass: columns (2-D) or a_x planes (3-D).
static cudaError_t launch_second(const sft_ctx* ctx, const StepArgs& a, int mode) {
    if (ctx->d == 3) return launch_k3_planes(a, mode, ctx->nl, ctx->stream);
    if (ctx->cplx) {
        // the step on complex columns of 1024 or 2048 points: warp-resident transforms
        if (mode == MODE_STEP && k2c_colwarp_supported(ctx->ny) && a.tw_32 && !a.rec_phi && !a.noise_in && !a.pshift)
            return launch_k2c_cols_warp(a, ctx->stream);
        return launch_k2c_cols(a, mode, ctx->stream);
    }
    return launch_k2_cols(a, mode, ctx->nl, ctx->stream);
}

static cudaError_t launch_cols_step(const sft_ctx* ctx, const StepArgs& a) {
    if (ctx->pipe_cols && !a.rec_phi && !a.noise_in && !a.pshift) return launch_k2_cols_pipe(a, ctx->nl, ctx->stream);
    if (ctx->d == 2 && !ctx->cplx) return launch_k2_cols(a, MODE_STEP, ctx->nl, ctx->stream, ctx->col_shape);
    return launch_second(ctx, a, MODE_STEP);
}

// Twiddle tables of a 1-D line launch: complex fields transform N-point lines (tw_a); real fields N/2-point
// lines with the N-point table of the real-to-complex post-processing (tw_b).  False if one is missing.
// Mode of the 1-D step kernel: the plain step or one of its variants (phase shifts, real-space noise); the
// variants keep the plain evaluation of the nonlinear term in Q (one line of M + 1 entries per replica).
static int line_step_mode(const sft_ctx* ctx, StepArgs& a) {
    a.qout = ctx->Q;
    if (ctx->cfg.noise_space == 1) {
        a.noise_scale = (float)(1.0 / std::sqrt((double)ctx->sites));
        return MODE_STEP_RSN;
    }
    return ctx->cfg.dealias == 2 ? MODE_STEP_PS : MODE_STEP;
}

static bool set_line_twiddles(const sft_ctx* ctx, StepArgs& a) {
    if (ctx->cplx) {
        a.tw_a = ctx->tw.get(ctx->nx);
        a.tw_b = nullptr;
        return a.tw_a != nullptr;
    }
    a.tw_a = ctx->tw.get(ctx->nx / 2);
    a.tw_b = ctx->tw.get(ctx->nx);
    return a.tw_a != nullptr && a.tw_b != nullptr;
}

// ------------------------------------------------------------ transforms
// state <- forward transform of the real-space buffer (c->real / c->cfield),
// for R replicas starting at replica r0.
static sft_status forward_from_buffer(sft_ctx* ctx, int r0, int R, float2* dst = nullptr) {
    StepArgs a = base_args(ctx);
    a.R = R;
    a.phi = (dst ? dst : ctx->phi) + (size_t)r0 * ctx->nmodes;
    a.real_io = ctx->real + (size_t)r0 * ctx->sites;
    a.cplx_io = ctx->cfield ? ctx->cfield + (size_t)r0 * ctx->sites : nullptr;
    if (ctx->d == 1) {
        if (!set_line_twiddles(ctx, a)) return fail(ctx, SFT_EINVAL, "twiddle table missing");
        CK(launch_k1_line(a, MODE_FWD, ctx->nl, ctx->stream));
        ctx->launches += 1;
    } else {
        ctx->launches += 2;
        a.ncols = ctx->hx;
        a.qout = ctx->Q + (size_t)r0 * ctx->nmodes;
        a.tw_a = ctx->tw.get(ctx->nx / 2);
        a.tw_b = ctx->tw.get(ctx->nx);
        CK(launch_rows(ctx, a, MODE_FWD));
        a.qin = a.qout;
        a.tw_a = ctx->tw.get(ctx->ny);
        CK(launch_second(ctx, a, MODE_FWD));
    }
    if (!dst) ctx->p_valid = false;
    return SFT_OK;
}

// real-space buffer <- inverse transform of the state (Q used as scratch).
static sft_status inverse_to_buffer(sft_ctx* ctx, const float2* src, int r0, int R) {
    StepArgs a = base_args(ctx);
    a.R = R;
    a.phi = const_cast<float2*>(src) + (size_t)r0 * ctx->nmodes;
    a.real_io = ctx->real + (size_t)r0 * ctx->sites;
    a.cplx_io = ctx->cfield ? ctx->cfield + (size_t)r0 * ctx->sites : nullptr;
    if (ctx->d == 1) {
        if (!set_line_twiddles(ctx, a)) return fail(ctx, SFT_EINVAL, "twiddle table missing");
        CK(launch_k1_line(a, MODE_INV, ctx->nl, ctx->stream));
        ctx->launches += 1;
    } else {
        ctx->launches += 2;
        a.ncols = ctx->hx;
        a.pout = ctx->Q + (size_t)r0 * ctx->nmodes;
        a.tw_a = ctx->tw.get(ctx->ny);
        CK(launch_second(ctx, a, MODE_INV));
        a.pin = a.pout;
        a.tw_a = ctx->tw.get(ctx->nx / 2);
        a.tw_b = ctx->tw.get(ctx->nx);
        CK(launch_rows(ctx, a, MODE_INV));
    }
    return SFT_OK;
}

// Advance the step counter(s) read by the step kernels (a batch: its own and
// those of the members that run their own kernels).
static cudaError_t advance_all(sft_ctx* ctx, int by) {
    cudaError_t e = launch_advance(ctx->dstep, by, ctx->stream);
    for (int m : ctx->solo)
        if (e == cudaSuccess) e = launch_advance(ctx->members[m]->dstep, by, ctx->stream);
    return e;
}
static int advances_per_chunk(const sft_ctx* ctx) { return 1 + (int)ctx->solo.size(); }

// P (and P_y) <- dealiased inverse y-transform of the state, the input of the
// next row pass.
static sft_status prime(sft_ctx* ctx) {
    if (ctx->is_batch) {
        for (int m : ctx->solo) {
            sft_status s = prime(ctx->members[m]);
            if (s != SFT_OK) return fail(ctx, s, ctx->members[m]->err);
            ctx->launches += 1;
        }
        ctx->p_valid = true;
        return SFT_OK;
    }
    if (ctx->d == 1) {
        ctx->p_valid = true;
        return SFT_OK;
    }
    StepArgs a = base_args(ctx);
    a.pout = ctx->P;
    a.pyout = ctx->Py;
    a.tw_a = ctx->tw.get(ctx->ny);
    CK(launch_second(ctx, a, MODE_PRIME));
    ctx->launches += 1;
    ctx->p_valid = true;
    return SFT_OK;
}


// One primal step with explicit intermediates: reads P from pin, leaves the
// next step's P in pout (2-D); used by the adjoint's segment recompute.
static sft_status enqueue_step_io(sft_ctx* ctx, const float2* pin, float2* pout, const float2* pyin = nullptr,
                                  float2* pyout = nullptr) {
    StepArgs a = base_args(ctx);
    if (ctx->d == 1) {
        if (!set_line_twiddles(ctx, a)) return fail(ctx, SFT_EINVAL, "twiddle table missing");
        CK(launch_k1_line(a, MODE_STEP, ctx->nl, ctx->stream));
    } else {
        a.pin = pin;
        a.pyin = pyin ? pyin : ctx->Py;
        a.pyout = pyout ? pyout : ctx->Py;
        a.qout = ctx->Q;
        a.tw_a = ctx->tw.get(ctx->nx / 2);
        a.tw_b = ctx->tw.get(ctx->nx);
        CK(launch_rows(ctx, a, MODE_STEP));
        a.qin = ctx->Q;
        a.pout = pout;
        a.tw_a = ctx->tw.get(ctx->ny);
        CK(launch_cols_step(ctx, a));
    }
    CK(launch_advance(ctx->dstep, 1, ctx->stream));
    ctx->launches += ctx->launches_per_step + 1;
    return SFT_OK;
}

static sft_status enqueue_step(sft_ctx* ctx, int k);

// One step of a batch: queue reset + the persistent 1-D kernel on the batch
// stream, every other member's own kernels on a forked branch of its own (so
// members too large for the persistent kernel run side by side), all joined at
// the end.
static sft_status enqueue_batch_step(sft_ctx* ctx, int k) {
    if (!ctx->solo.empty()) {
        CK(cudaEventRecord(ctx->ev_fork, ctx->stream));
        for (size_t i = 0; i < ctx->solo.size(); ++i) {
            CK(cudaStreamWaitEvent(ctx->sides[i], ctx->ev_fork, 0));
            sft_ctx* mb = ctx->members[ctx->solo[i]];
            cudaStream_t keep = mb->stream;
            mb->stream = ctx->sides[i];
            sft_status s = enqueue_step(mb, k);
            mb->stream = keep;
            if (s != SFT_OK) return fail(ctx, s, mb->err);
        }
    }
    if (ctx->nitems > 0) {
        CK(cudaMemsetAsync(ctx->d_head, 0, sizeof(int), ctx->stream));
        CK(launch_k1_batch(ctx->d_members, ctx->d_items, ctx->nitems, ctx->d_head, ctx->nl, k, ctx->batch_blocks,
                           ctx->stream));
    }
    for (size_t i = 0; i < ctx->solo.size(); ++i) {
        CK(cudaEventRecord(ctx->ev_joins[i], ctx->sides[i]));
        CK(cudaStreamWaitEvent(ctx->stream, ctx->ev_joins[i], 0));
    }
    return SFT_OK;
}

// The kernels of a 2-D step before its column pass (k_in_chunk = k): the
// real-space noise and its transform where configured, and the row pass; a is
// left set up for the column pass.
static sft_status enqueue_front(sft_ctx* ctx, StepArgs& a, int k) {
    if (ctx->noise_spec) {
        // real-space noise (Sec. IV step 2): iid N(0, 1) per site, drawn inside the forward row pass
        // (Q as scratch, overwritten by the step's row pass below), then the column transform into
        // noise_spec; the column pass reads eta_a = DFT[eta]_a / sqrt(N^d)
        StepArgs f = a;
        f.k_in_chunk = k;
        f.ncols = ctx->hx;
        f.qout = ctx->Q;
        f.tw_a = ctx->tw.get(ctx->nx / 2);
        f.tw_b = ctx->tw.get(ctx->nx);
        CK(launch_rows(ctx, f, MODE_FWD_NOISE));
        f.qin = ctx->Q;
        f.phi = ctx->noise_spec;
        f.tw_a = ctx->tw.get(ctx->ny);
        CK(launch_second(ctx, f, MODE_FWD));
        a.noise_in = ctx->noise_spec;
        a.noise_scale = (float)(1.0 / std::sqrt((double)ctx->sites));
    }
    a.pin = ctx->P;
    a.pyin = ctx->Py;
    a.qout = ctx->Q;
    a.tw_a = ctx->tw.get(ctx->nx / 2);
    a.tw_b = ctx->tw.get(ctx->nx);
    if (a.pshift) {
        // phase-shift dealiasing: the row pass runs over every copy of P (2-D: plain and shifted along y; 3-D: the
        // four shifts of y and z), each averaging its two x shifts
        StepArgs r = a;
        r.R = (ctx->d == 3 ? 4 : 2) * ctx->R;  // every copy of P (2-D: y shifts; 3-D: y and z shifts)
        CK(launch_rows(ctx, r, MODE_STEP_PS));
    } else {
        CK(launch_rows(ctx, a, MODE_STEP));
    }
    a.qin = ctx->Q;
    a.pout = ctx->P;
    a.pyout = ctx->Py;
    a.tw_a = ctx->tw.get(ctx->ny);
    return SFT_OK;
}

// Enqueue the kernels of one step (k_in_chunk = k).
static sft_status enqueue_step(sft_ctx* ctx, int k) {
    if (ctx->is_batch) return enqueue_batch_step(ctx, k);
    StepArgs a = base_args(ctx);
    a.k_in_chunk = k;
    if (ctx->d == 1) {
        if (!set_line_twiddles(ctx, a)) return fail(ctx, SFT_EINVAL, "twiddle table missing");
        CK(launch_k1_line(a, line_step_mode(ctx, a), ctx->nl, ctx->stream));
        return SFT_OK;
    }
    if (ctx->cfg.precision == 1) {
        // precision study: the step through the split-BF16x3 tensor-core transforms
        CK(launch_tc_step(a, ctx->tcb1, ctx->tcb2, ctx->tw.get(ctx->nx), ctx->stream));
        return SFT_OK;
    }
    sft_status s = enqueue_front(ctx, a, k);
    if (s != SFT_OK) return s;
    CK(launch_cols_step(ctx, a));
    return SFT_OK;
}

// ------------------------------------------------------------ plan autotuner
// The schedule of the step's passes -- the radix schedule and block shape of
// the 2-D column pass, replicas per column block, the block shape of the row
// pass and the pipelined column pass -- is chosen per lattice by timing every
// variant built for it with CUDA events on scratch copies of the state (the
// context's own state is left untouched), once per configuration in the
// process.  SFT_AUTOTUNE=0 keeps the defaults.
namespace {
struct PlanKey {
    int d, nx, ny, nz, R, nl, scheme, dealias, dev;
    bool operator<(const PlanKey& o) const {
        return std::tie(d, nx, ny, nz, R, nl, scheme, dealias, dev) <
               std::tie(o.d, o.nx, o.ny, o.nz, o.R, o.nl, o.scheme, o.dealias, o.dev);
    }
};
struct PlanChoice {
    int row_shape, col_shape, rpb, pipe;
};
std::mutex g_plan_mu;
std::map<PlanKey, PlanChoice> g_plans;
constexpr int kRpbChoices[] = {1, 2, 4, 8};
constexpr int kPlanReps = 4;
}  // namespace

// mean time of kPlanReps launches after one untimed launch
template <class F>
static cudaError_t time_launch(cudaStream_t s, F&& launch, float* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    for (int i = 0; i < kPlanReps && e == cudaSuccess; ++i) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    *ms = t / kPlanReps;
    return e;
}

static void apply_plan(sft_ctx* ctx, const PlanChoice& p) {
    ctx->row_shape = p.row_shape;
    ctx->col_shape = p.col_shape;
    ctx->rpb = p.rpb;
    if (!ctx->pipe_forced) ctx->pipe_cols = p.pipe != 0;
}

static sft_status prime(sft_ctx* ctx);

// Whether row-pass schedule sh is built for the context's lattice and term.
static bool row_shape_ok(const sft_ctx* ctx, int sh) {
    if (sh < 0 || sh >= k2_row_shapes(ctx->nx)) return false;
    if (sh == 3) return k2_pair_supported(ctx->nx, ctx->ny * ctx->nz, ctx->nl, ctx->cfg.dealias) && ctx->tw32;
    return true;
}

// Whether column-pass schedule sh is built for the context's lattice and term.
static bool col_shape_ok(const sft_ctx* ctx, int sh) {
    if (sh < 0 || sh >= (ctx->d == 2 ? k2_col_shapes(ctx->ny) : 1)) return false;
    if (sh == 3) return k2_colwarp_supported(ctx->nx, ctx->ny, ctx->nl, ctx->cfg.dealias) && ctx->tw32;
    return true;
}

static sft_status plan_step(sft_ctx* ctx) {
    if (ctx->planned) return SFT_OK;
    ctx->planned = true;
    if (ctx->is_batch) {
        for (int m : ctx->solo) {
            sft_status s = plan_step(ctx->members[m]);
            if (s != SFT_OK) return fail(ctx, s, ctx->members[m]->err);
        }
        return SFT_OK;
    }
    const char* env = getenv("SFT_AUTOTUNE");
    if ((env && env[0] == '0') || ctx->cplx || ctx->d < 2 || ctx->cfg.dealias == 2 || !is_pow2(ctx->nx)) return SFT_OK;
    // SFT_PLAN="row,col,rpb,pipe" fixes the schedule (as sft_set_plan; e.g. to profile the one a timed run chose)
    if (const char* fixed = getenv("SFT_PLAN")) {
        int v[4];
        if (sscanf(fixed, "%d,%d,%d,%d", &v[0], &v[1], &v[2], &v[3]) == 4) {
            const bool ok = row_shape_ok(ctx, v[0]) && col_shape_ok(ctx, v[1]) && v[2] >= 1 && v[2] <= 64 &&
                            (v[3] == 0 || (ctx->d == 2 && k2_pipe_supported(ctx->nx, ctx->ny, 0)));
            if (!ok) return fail(ctx, SFT_EINVAL, "SFT_PLAN names a schedule not built for this lattice");
            apply_plan(ctx, PlanChoice{v[0], v[1], v[2], v[3]});
            return SFT_OK;
        }
        return fail(ctx, SFT_EINVAL, "SFT_PLAN must read row,col,rpb,pipe");
    }
    int dev = 0;
    CK(cudaGetDevice(&dev));
    const PlanKey key{ctx->d, ctx->nx, ctx->ny, ctx->nz, ctx->R, ctx->nl, ctx->cfg.scheme, ctx->cfg.dealias, dev};
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        auto it = g_plans.find(key);
        if (it != g_plans.end()) {
            apply_plan(ctx, it->second);
            return SFT_OK;
        }
    }
    if (!ctx->p_valid) {
        sft_status s = prime(ctx);
        if (s != SFT_OK) return s;
    }
    PlanChoice best{0, 0, 0, 0};
    // row pass: reads P, writes the scratch Q (the state is not touched)
    StepArgs a = base_args(ctx);
    a.pin = ctx->P;
    a.pyin = ctx->Py;
    a.qout = ctx->Q;
    a.ny = ctx->ny * ctx->nz;
    a.nz = 1;
    a.tw_a = ctx->tw.get(ctx->nx / 2);
    a.tw_b = ctx->tw.get(ctx->nx);
    float best_ms = 1e30f;
    for (int sh = 0; sh < k2_row_shapes(ctx->nx); ++sh) {
        if (!row_shape_ok(ctx, sh)) continue;
        float ms = 0.f;
        CK(time_launch(ctx->stream, [&] { return launch_k2_rows(a, MODE_STEP, ctx->nl, ctx->stream, sh); }, &ms));
        if (ms < best_ms) best_ms = ms, best.row_shape = sh;
    }
    CK(launch_k2_rows(a, MODE_STEP, ctx->nl, ctx->stream, best.row_shape));  // Q as the chosen pass leaves it
    if (ctx->d == 2) {
        // column pass on copies of the state and history, writing a scratch P (and P_y); the
        // intermediates use the state's layout (replica stride hx columns), so every scratch
        // buffer has the state's size, as the context's own P, Q, P_y do
        const size_t sb = (size_t)ctx->R * ctx->nmodes * sizeof(float2);
        const size_t pb = sb;
        const bool grad = ctx->nl == NL_GRAD2, hist = ctx->cfg.scheme == SFT_SETD2;
        float2 *tphi = nullptr, *tfp = nullptr, *tP = nullptr, *tPy = nullptr;
        cudaError_t me = cudaMalloc(&tphi, sb);
        if (me == cudaSuccess) me = cudaMalloc(&tP, pb);
        if (me == cudaSuccess && hist) me = cudaMalloc(&tfp, sb);
        if (me == cudaSuccess && grad) me = cudaMalloc(&tPy, pb);
        if (me == cudaSuccess) {
            StepArgs c = base_args(ctx);
            c.rec_phi = c.rec_F = nullptr;  // trial passes record nothing
            c.qin = ctx->Q;
            c.phi = tphi;
            c.fprev = tfp;
            c.pout = tP;
            c.pyout = tPy;
            c.tw_a = ctx->tw.get(ctx->ny);
            cudaError_t e = cudaMemcpyAsync(tphi, ctx->phi, sb, cudaMemcpyDeviceToDevice, ctx->stream);
            if (e == cudaSuccess && hist) e = cudaMemcpyAsync(tfp, ctx->fprev, sb, cudaMemcpyDeviceToDevice, ctx->stream);
            best_ms = 1e30f;
            for (int sh = 0; sh < k2_col_shapes(ctx->ny) && e == cudaSuccess; ++sh) {
                if (!col_shape_ok(ctx, sh)) continue;
                for (int rpb : kRpbChoices) {
                    c.rpb = rpb;
                    float ms = 0.f;
                    e = time_launch(ctx->stream, [&] { return launch_k2_cols(c, MODE_STEP, ctx->nl, ctx->stream, sh); },
                                    &ms);
                    if (e != cudaSuccess) break;
                    if (ms < best_ms) best_ms = ms, best.col_shape = sh, best.rpb = rpb;
                }
            }
            if (e == cudaSuccess && !ctx->pipe_forced && k2_pipe_supported(ctx->nx, ctx->ny, 0)) {
                float ms = 0.f;
                e = time_launch(ctx->stream, [&] { return launch_k2_cols_pipe(c, ctx->nl, ctx->stream); }, &ms);
                if (e == cudaSuccess && ms < best_ms) best_ms = ms, best.pipe = 1;
            }
            cudaError_t se = cudaStreamSynchronize(ctx->stream);
            if (e == cudaSuccess) e = se;
            cudaFree(tphi);
            cudaFree(tP);
            if (tfp) cudaFree(tfp);
            if (tPy) cudaFree(tPy);
            if (e != cudaSuccess) return fail(ctx, SFT_ECUDA, std::string("plan autotuner: ") + cudaGetErrorString(e));
        } else {
            // not enough device memory for the scratch copies: keep the default column schedule
            cudaGetLastError();
            if (tphi) cudaFree(tphi);
            if (tP) cudaFree(tP);
            if (tfp) cudaFree(tfp);
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_plan_mu);
        g_plans[key] = best;
    }
    apply_plan(ctx, best);
    return SFT_OK;
}

static sft_status capture_graph(sft_ctx* ctx) {
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    sft_status st = SFT_OK;
    for (int k = 0; k < kGraphChunk && st == SFT_OK; ++k) st = enqueue_step(ctx, k);
    if (st == SFT_OK) {
        cudaError_t e = advance_all(ctx, kGraphChunk);
        if (e != cudaSuccess) st = fail(ctx, SFT_ECUDA, cudaGetErrorString(e));
    }
    cudaError_t ee = cudaStreamEndCapture(ctx->stream, &g);
    if (st != SFT_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ee != cudaSuccess) return fail(ctx, SFT_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
    cudaError_t ie = cudaGraphInstantiate(&ctx->graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return fail(ctx, SFT_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    return SFT_OK;
}

static sft_status build_twiddles(sft_ctx* ctx, const std::vector<int>& lens) {
    size_t total = 0;
    for (int L : lens) {
        bool dup = false;
        for (int x : ctx->tw.lens) dup |= (x == L);
        if (dup || L < 2) continue;
        ctx->tw.lens.push_back(L);
        ctx->tw.offs.push_back(total);
        total += (size_t)L;
    }
    CK(cudaMalloc(&ctx->tw.dev, std::max<size_t>(total, 1) * sizeof(float2)));
    for (size_t i = 0; i < ctx->tw.lens.size(); ++i)
        CK(launch_twiddles(ctx->tw.dev + ctx->tw.offs[i], ctx->tw.lens[i], ctx->stream));
    return SFT_OK;
}

namespace sft {
sft_status validate_config(const sft_config* cfg, std::string& why);
}

static sft_status validate(const sft_config* cfg, std::string& why) { return sft::validate_config(cfg, why); }

// The checks every configuration passes before any device work (also used by the allocation-free entry point).
sft_status sft::validate_config(const sft_config* cfg, std::string& why) {
    if (!cfg) return why = "null config", SFT_EINVAL;
    if (cfg->d < 1 || cfg->d > 3) return why = "d must be 1, 2 or 3", SFT_EINVAL;
    for (int i = 0; i < cfg->d; ++i) {
        if (!is_pow2(cfg->n[i]) && !k2_mixed_size(cfg->n[i]))
            return why = "lattice sizes must be powers of two (or p x 2^k, p in {3, 5, 7}, 16p .. 768, for 1-D and 2-D "
                         "real fields)", SFT_EINVAL;
        if (!(cfg->dx[i] > 0)) return why = "dx must be positive", SFT_EINVAL;
        if (cfg->n[i] != cfg->n[0] || cfg->dx[i] != cfg->dx[0])
            return why = "anisotropic lattices are not supported (coefficients are tabulated by |a|^2)",
                   SFT_EUNSUPPORTED;
    }
    if (cfg->replicas < 1) return why = "replicas must be >= 1", SFT_EINVAL;
    if (cfg->replica0 < 0) return why = "replica0 must be >= 0", SFT_EINVAL;
    if (!(cfg->h > 0) || !std::isfinite(cfg->h)) return why = "h must be positive and finite", SFT_EINVAL;
    if (cfg->model < SFT_MODEL_A || cfg->model > SFT_CUSTOM) return why = "unknown model", SFT_EINVAL;
    if (cfg->scheme < SFT_SETD_EM || cfg->scheme > SFT_SETD2) return why = "unknown scheme", SFT_EINVAL;
    if (cfg->precision != 0) {
        // 1: the split-BF16x3 tensor-core transforms of the precision study, complex 2-D fields of 1024^2
        // or 2048^2 points with Fourier-space noise
        int cp = 0, nl1 = 0;
        model_kind(cfg, &cp, &nl1);
        if (cfg->precision != 1) return why = "precision must be 0 (FP32) or 1 (split-BF16x3 study)", SFT_EINVAL;
        if (!cp || cfg->d != 2 || !tc_supported(cfg->n[0], cfg->n[1]) || cfg->noise_space != 0 || cfg->dealias == 2)
            return why = "the split-BF16x3 tensor-core path is built for complex 2-D fields of 1024^2 or 2048^2 "
                         "points, Fourier-space noise, 2/3 truncation or none",
                   SFT_EUNSUPPORTED;
    }
    if ((cfg->model == SFT_MODEL_A || cfg->model == SFT_MODEL_B) && cfg->p[4] != 0.0 && cfg->scheme == SFT_SETD2)
        return why = "r placed in F (p[4] != 0) is built for SETD-EM and SETD1", SFT_EUNSUPPORTED;
    if (cfg->dealias < 0 || cfg->dealias > 2)
        return why = "dealias must be 0 (none), 1 (2/3 truncation) or 2 (phase shifts)", SFT_EINVAL;
    int cplx = 0, nlk = 0;
    model_kind(cfg, &cplx, &nlk);
    if (cfg->noise_space != 0 && cfg->noise_space != 1) return why = "noise_space must be 0 or 1", SFT_EINVAL;
    // the 1-D variants run in the single-line kernel: power-of-two lines of up to 16384 points
    const bool line_var_ok = cfg->d == 1 && !cplx && is_pow2(cfg->n[0]) && cfg->n[0] <= 16384 &&
                             (nlk == NL_CUBIC || nlk == NL_GRAD2);
    if (cfg->noise_space == 1 && !((cfg->d >= 2 && !cplx) || line_var_ok))
        return why = "real-space noise is built for 2-D and 3-D real fields and 1-D real lines of up to 16384 points "
                     "(cubic or gradient-squared term)",
               SFT_EUNSUPPORTED;
    if (!is_pow2(cfg->n[0]) &&
        (cfg->d == 3 || cplx || cfg->dealias == 2 || cfg->noise_space != 0 || cfg->model == SFT_CUSTOM))
        return why = "lattices of p x 2^k points are built for 1-D and 2-D real fields (Model A/B, KPZ) with "
                     "Fourier-space noise and 2/3 truncation (or none)",
               SFT_EUNSUPPORTED;
    // 3-D: the plane pass keeps two planes in shared memory (planes up to 64^2); complex fields: 2-D, |A|^2 A
    const bool ps3_ok = cfg->d == 3 && !cplx && nlk == NL_CUBIC && cfg->n[0] <= 64;
    const bool psc_ok = cfg->d == 2 && cplx && nlk == NL_CGL && cfg->precision == 0;
    const bool ps_real = (cfg->d == 2 && !cplx) || line_var_ok || ps3_ok;
    if (cfg->dealias == 2 && (!(ps_real || psc_ok) || (!psc_ok && nlk != NL_CUBIC && nlk != NL_GRAD2) ||
                              cfg->noise_space != 0))
        return why = "phase-shift dealiasing is built for 2-D real fields, 1-D real lines of up to 16384 points (cubic "
                     "or gradient-squared term), 3-D real fields of up to 64^3 (cubic term) and 2-D complex fields "
                     "(|A|^2 A), with Fourier-space noise",
               SFT_EUNSUPPORTED;
    if (cfg->model == SFT_CUSTOM) {
        const int nl = cfg->custom_nl;
        if (nl < SFT_NL_NONE || nl > SFT_NL_CGL) return why = "unknown custom nonlinearity", SFT_EINVAL;
        if (cplx ? !(nl == SFT_NL_CGL || nl == SFT_NL_NONE) : nl == SFT_NL_CGL)
            return why = "custom nonlinearity does not match the field (|A|^2 A needs a complex field, psi^3 and "
                         "grad^2 a real one)",
                   SFT_EINVAL;
        if (!cfg->c_re || !cfg->noise_D) return why = "SFT_CUSTOM needs the c_re and noise_D tables", SFT_EINVAL;
        const long long n = custom_len(cfg);
        for (long long q = 0; q < n; ++q) {
            const double ci = cfg->c_im ? cfg->c_im[q] : 0.0, si = cfg->nl_im ? cfg->nl_im[q] : 0.0;
            const double sr = cfg->nl_re ? cfg->nl_re[q] : 0.0;
            if (!std::isfinite(cfg->c_re[q]) || !std::isfinite(ci) || !std::isfinite(sr) || !std::isfinite(si))
                return why = "custom tables must be finite", SFT_EINVAL;
            if (!(cfg->noise_D[q] >= 0.0) || !std::isfinite(cfg->noise_D[q]))
                return why = "custom noise strength D must be finite and >= 0", SFT_EINVAL;
            if (!cplx && (ci != 0.0 || si != 0.0))
                return why = "a real field needs real c and s (Hermitian symmetry)", SFT_EINVAL;
        }
    }
    if (cfg->d == 1 && !k1_supported(cfg->n[0], cplx)) return why = "1-D size outside the built plans", SFT_EUNSUPPORTED;
    if (cfg->d == 2 && !(cplx ? k2c_supported(cfg->n[0], cfg->n[1]) : k2_supported(cfg->n[0], cfg->n[1], 0)))
        return why = "2-D size outside the built plans", SFT_EUNSUPPORTED;
    if (cfg->d == 3 && (cplx || nlk == NL_GRAD2 || !k3_supported(cfg->n[0], cfg->n[1], cfg->n[2], cplx)))
        return why = "3-D lattices are built for real fields with the cubic term and 16..128 points per axis",
               SFT_EUNSUPPORTED;
    return SFT_OK;
}

extern "C" {

sft_status sft_create(const sft_config* cfg, sft_ctx** out) {
    if (!out) return SFT_EINVAL;
    *out = nullptr;
    std::string why;
    sft_status vs = validate(cfg, why);
    if (vs != SFT_OK) {
        fprintf(stderr, "sft_create: %s\n", why.c_str());
        return vs;
    }
    sft_ctx* ctx = new (std::nothrow) sft_ctx();
    if (!ctx) return SFT_ENOMEM;
    ctx->cfg = *cfg;
    ctx->d = cfg->d;
    ctx->nx = cfg->n[0];
    ctx->ny = cfg->d >= 2 ? cfg->n[1] : 1;
    ctx->nz = cfg->d >= 3 ? cfg->n[2] : 1;
    model_kind(cfg, &ctx->cplx, &ctx->nl);
    ctx->cfg.c_re = ctx->cfg.c_im = ctx->cfg.noise_D = ctx->cfg.nl_re = ctx->cfg.nl_im = nullptr;  // host tables: copied below
    if (cfg->model != SFT_CUSTOM) ctx->cfg.custom_nl = ctx->cfg.complex_field = 0;
    ctx->hx = ctx->cplx ? ctx->nx : ctx->nx / 2 + 1;
    ctx->mx = 0;
    for (int c = 0; c < ctx->hx; ++c) {
        // real fields: the first mx x-modes; complex fields: the mx x-modes with 3|a_x| < nx (compact order)
        const int cs = ctx->cplx && 2 * c >= ctx->nx ? ctx->nx - c : c;
        if (!cfg->dealias || (cfg->dealias == 1 ? 3 * cs < ctx->nx : 2 * cs < ctx->nx))
            ctx->mx = ctx->cplx ? ctx->mx + 1 : c + 1;
    }
    ctx->sites = (long long)ctx->nx * ctx->ny * ctx->nz;
    ctx->nmodes = (long long)ctx->hx * ctx->ny * ctx->nz;
    ctx->R = cfg->replicas;
    ctx->rep0 = cfg->replica0;
    auto cleanup = [&](sft_status s) {
        sft_destroy(ctx);
        return s;
    };
    if (cfg->stream) {
        ctx->stream = (cudaStream_t)cfg->stream;
    } else {
        if (cudaStreamCreate(&ctx->stream) != cudaSuccess) return cleanup(SFT_ECUDA);
        ctx->own_stream = true;
    }
    const size_t ms = (size_t)ctx->R * ctx->nmodes * sizeof(float2);
    const size_t rs = (size_t)ctx->R * ctx->sites * (ctx->cplx ? sizeof(float2) : sizeof(float));
    auto dalloc = [&](void** p, size_t bytes) { return cudaMalloc(p, bytes) == cudaSuccess; };
    // phase-shift dealiasing keeps further copies of P and Q behind the first: one per shift of the axes after x
    // (2-D: y; 3-D: y, z and both)
    const size_t pq = cfg->dealias == 2 ? (cfg->d == 3 ? 4 : 2) * ms : ms;
    bool ok = dalloc((void**)&ctx->phi, ms) && dalloc((void**)&ctx->Q, pq);
    if (ok && ctx->d >= 2) ok = dalloc((void**)&ctx->P, pq);
    if (ok && ctx->d >= 2 && ctx->nl == NL_GRAD2) ok = dalloc((void**)&ctx->Py, pq);
    if (ok && cfg->scheme == SFT_SETD2) ok = dalloc((void**)&ctx->fprev, ms);
    if (ok && cfg->noise_space == 1 && ctx->d >= 2) ok = dalloc((void**)&ctx->noise_spec, ms);
    if (ok && cfg->precision == 1) ok = dalloc((void**)&ctx->tcb1, ms) && dalloc((void**)&ctx->tcb2, ms);
    if (ok) {
        if (ctx->cplx)
            ok = dalloc((void**)&ctx->cfield, rs);
        else
            ok = dalloc((void**)&ctx->real, rs);
    }
    long long qmax = 0;
    for (int i = 0; i < ctx->d; ++i) qmax += (long long)(cfg->n[i] / 2) * (cfg->n[i] / 2);
    long long nq = qmax + 1;  // d = 3: one entry per |a|^2
    if (ctx->d == 1) nq = ctx->nx / 2 + 1;
    if (ctx->d == 2) nq = (long long)(ctx->nx / 2 + 1) * (ctx->ny / 2 + 1);
    if (ok) ok = dalloc((void**)&ctx->tab, (size_t)nq * (ctx->cplx ? 2 : 1) * sizeof(float4));
    if (ok) ok = dalloc((void**)&ctx->dstep, 4 * sizeof(long long)) && dalloc((void**)&ctx->dstatus, sizeof(unsigned));
    ctx->nshells = (int)isqrt_ceil(qmax) + 1;
    if (ok)
        ok = dalloc((void**)&ctx->dshell, (size_t)ctx->R * ctx->nshells * sizeof(double)) &&
             dalloc((void**)&ctx->drough, (size_t)ctx->R * sizeof(double));
    if (!ok) {
        fprintf(stderr, "sft_create: device allocation failed\n");
        return cleanup(SFT_ENOMEM);
    }
    if (cudaMemset(ctx->phi, 0, ms) != cudaSuccess || cudaMemset(ctx->Q, 0, pq) != cudaSuccess)
        return cleanup(SFT_ECUDA);
    if (ctx->P && cudaMemset(ctx->P, 0, pq) != cudaSuccess) return cleanup(SFT_ECUDA);
    if (ctx->Py && cudaMemset(ctx->Py, 0, pq) != cudaSuccess) return cleanup(SFT_ECUDA);
    if (ctx->fprev && cudaMemset(ctx->fprev, 0, ms) != cudaSuccess) return cleanup(SFT_ECUDA);
    long long init[4] = {0, cfg->scheme == SFT_SETD2 ? 0 : -1, (long long)0x7fffffffffffffffLL, 0};
    ctx->first_step = init[1];
    if (cudaMemcpy(ctx->dstep, init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(ctx->dstatus, 0, sizeof(unsigned)) != cudaSuccess)
        return cleanup(SFT_ECUDA);
    std::vector<int> lens;
    if (ctx->cplx) {
        lens.push_back(ctx->nx);
    } else {
        lens.push_back(ctx->nx / 2);
        lens.push_back(ctx->nx);
    }
    if (ctx->d >= 2) lens.push_back(ctx->ny);
    if (cfg->dealias == 2) lens.push_back(2 * ctx->nx);  // half-cell shift phases
    if (ctx->d == 1 && !ctx->cplx && k1_cluster_fft_len(ctx->nx))
        lens.push_back(k1_cluster_fft_len(ctx->nx));  // per-block FFT of the cluster kernel
    if (build_twiddles(ctx, lens) != SFT_OK) return cleanup(SFT_ECUDA);
    if (ctx->d >= 2 && (ctx->cplx ? (ctx->d == 2 && (k2c_colwarp_supported(ctx->ny) ||
                                                     k2c_rowwarp_supported(ctx->nx, ctx->ny, cfg->dealias)))
                                  : (ctx->nx == 1024 || ctx->ny == 1024))) {
        // twiddles of the 1024-point warp transforms: entry k1 32 + t = W_1024^{t k1}
        if (!dalloc((void**)&ctx->tw32, 1024 * sizeof(float2)) || launch_twiddles32(ctx->tw32, ctx->stream) != cudaSuccess)
            return cleanup(SFT_ECUDA);
    }
    if (const char* wl = getenv("SFT_WAIT_LIMIT")) ctx->wait_limit = atoi(wl);
    // FP64 coefficient tables
    TableArgs t{};
    t.model = cfg->model;
    t.scheme = cfg->scheme;
    t.complex_field = ctx->cplx;
    t.d = ctx->d;
    t.hy = ctx->ny / 2 + 1;
    for (int i = 0; i < 8; ++i) t.p[i] = cfg->p[i];
    t.h = cfg->h;
    t.dk = 2.0 * M_PI / (ctx->nx * cfg->dx[0]);
    double nf = 1.0;
    for (int i = 0; i < ctx->d; ++i) nf *= std::sqrt(cfg->n[i] / cfg->dx[i]);
    t.noise_norm = nf;
    t.nq = nq;
    t.out = ctx->tab;
    double* dcust = nullptr;
    if (cfg->model == SFT_CUSTOM) {
        // c_re, c_im, D, s_re, s_im over |a|^2, copied to the device for the FP64 table build
        const long long n = custom_len(cfg);
        std::vector<double> host((size_t)(5 * n), 0.0);
        const bool with_s = cfg->custom_nl != SFT_NL_NONE;
        uint64_t hsh = 1469598103934665603ULL;
        for (long long q = 0; q < n; ++q) {
            host[q] = cfg->c_re[q];
            host[n + q] = cfg->c_im ? cfg->c_im[q] : 0.0;
            host[2 * n + q] = cfg->noise_D[q];
            host[3 * n + q] = (with_s && cfg->nl_re) ? cfg->nl_re[q] : 0.0;
            host[4 * n + q] = (with_s && cfg->nl_im) ? cfg->nl_im[q] : 0.0;
        }
        const unsigned char* b = (const unsigned char*)host.data();
        for (size_t i = 0; i < host.size() * sizeof(double); ++i) {
            hsh ^= b[i];
            hsh *= 1099511628211ULL;
        }
        ctx->cust_hash = hsh;
        ctx->cust_c.assign(host.begin(), host.begin() + n);
        ctx->cust_D.assign(host.begin() + 2 * n, host.begin() + 3 * n);
        if (cudaMalloc(&dcust, host.size() * sizeof(double)) != cudaSuccess) return cleanup(SFT_ENOMEM);
        if (cudaMemcpy(dcust, host.data(), host.size() * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
            cudaFree(dcust);
            return cleanup(SFT_ECUDA);
        }
        t.cust = dcust;
        t.ncust = n;
    }
    const cudaError_t te = launch_build_table(t, ctx->stream);
    if (dcust) {
        cudaStreamSynchronize(ctx->stream);
        cudaFree(dcust);
    }
    if (te != cudaSuccess) return cleanup(SFT_ECUDA);
    // shell counts with the half-spectrum weights
    ctx->counts.assign(ctx->nshells, 0.0);
    for (int ax = 0; ax < ctx->hx; ++ax) {
        const long long sx = ctx->cplx ? (2 * ax < ctx->nx ? ax : ax - ctx->nx) : ax;
        const double w = (!ctx->cplx && ax != 0 && 2 * ax != ctx->nx) ? 2.0 : 1.0;
        for (int az = 0; az < ctx->nz; ++az) {
            const long long sz = 2 * az < ctx->nz ? az : az - ctx->nz;
            for (int ay = 0; ay < ctx->ny; ++ay) {
                const long long sy = 2 * ay < ctx->ny ? ay : ay - ctx->ny;
                ctx->counts[isqrt_ceil(sx * sx + sy * sy + sz * sz)] += w;
            }
        }
    }
    {
        // the stored modes shell by shell (index order inside a shell), cut into chunks of at most
        // kObsChunkLen modes inside one shell: the fixed summation order of every observation
        const long long nm = ctx->nmodes;
        std::vector<int> shell_of_mode((size_t)nm), fill(ctx->nshells + 1, 0);
        for (int ax = 0; ax < ctx->hx; ++ax) {
            const long long sx = ctx->cplx ? (2 * ax < ctx->nx ? ax : ax - ctx->nx) : ax;
            for (int az = 0; az < ctx->nz; ++az) {
                const long long sz = 2 * az < ctx->nz ? az : az - ctx->nz;
                for (int ay = 0; ay < ctx->ny; ++ay) {
                    const long long sy = 2 * ay < ctx->ny ? ay : ay - ctx->ny;
                    const long long m = ((long long)ax * ctx->nz + az) * ctx->ny + ay;
                    shell_of_mode[(size_t)m] = (int)isqrt_ceil(sx * sx + sy * sy + sz * sz);
                }
            }
        }
        std::vector<int> start(ctx->nshells + 1, 0);
        for (long long m = 0; m < nm; ++m) ++start[shell_of_mode[(size_t)m] + 1];
        for (int j = 0; j < ctx->nshells; ++j) start[j + 1] += start[j];
        std::vector<int> order((size_t)nm);
        for (long long m = 0; m < nm; ++m) {
            const int j = shell_of_mode[(size_t)m];
            order[(size_t)(start[j] + fill[j]++)] = (int)m;
        }
        std::vector<int4> chunks;
        std::vector<int> first(ctx->nshells + 1, 0);
        for (int j = 0; j < ctx->nshells; ++j) {
            first[j] = (int)chunks.size();
            for (int b = start[j]; b < start[j + 1]; b += kObsChunkLen)
                chunks.push_back(make_int4(j, b, std::min(kObsChunkLen, start[j + 1] - b), 0));
        }
        first[ctx->nshells] = (int)chunks.size();
        ctx->nchunks = (int)chunks.size();
        if (!dalloc((void**)&ctx->d_order, order.size() * sizeof(int)) ||
            !dalloc((void**)&ctx->d_chunks, chunks.size() * sizeof(int4)) ||
            !dalloc((void**)&ctx->d_first_chunk, first.size() * sizeof(int)) ||
            !dalloc((void**)&ctx->d_part, (size_t)ctx->R * chunks.size() * sizeof(double2)) ||
            !dalloc((void**)&ctx->d_tacc, (size_t)ctx->nshells * sizeof(double2)))
            return cleanup(SFT_ENOMEM);
        if (cudaMemcpy(ctx->d_order, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
            cudaMemcpy(ctx->d_chunks, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(ctx->d_first_chunk, first.data(), first.size() * sizeof(int), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemset(ctx->d_tacc, 0, (size_t)ctx->nshells * sizeof(double2)) != cudaSuccess)
            return cleanup(SFT_ECUDA);
    }
    ctx->launches_per_step = ctx->d == 1 ? 1 : 2;
    // 2-D real-space noise: the forward transform of the noise (drawn in its row pass); 1-D lines transform it
    // inside the step kernel
    if (cfg->noise_space == 1 && ctx->d >= 2) ctx->launches_per_step += 2;
    if (cfg->precision == 1) ctx->launches_per_step = 9;     // prep, 4 transforms, 2 transposes, |A|^2 A, update
    {
        // column-pass variant: chosen by the plan autotuner unless SFT_COLUMN_PASS forces the
        // persistent bulk-copy pipelined kernel ("pipelined", where it is built) or the
        // multi-block kernel ("multiblock")
        const char* v = getenv("SFT_COLUMN_PASS");
        if (v && (strcmp(v, "pipelined") == 0 || strcmp(v, "multiblock") == 0)) {
            ctx->pipe_forced = true;
            ctx->pipe_cols = ctx->d == 2 && strcmp(v, "pipelined") == 0 && k2_pipe_supported(ctx->nx, ctx->ny, ctx->cplx);
        }
    }
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return cleanup(SFT_ECUDA);
    *out = ctx;
    return SFT_OK;
}

sft_status sft_create_batch(const sft_config* cfgs, int count, sft_ctx** out) {
    if (!out) return SFT_EINVAL;
    *out = nullptr;
    if (!cfgs || count < 1) return SFT_EINVAL;
    for (int i = 0; i < count; ++i) {
        std::string why;
        sft_status vs = validate(&cfgs[i], why);
        if (vs != SFT_OK) {
            fprintf(stderr, "sft_create_batch: member %d: %s\n", i, why.c_str());
            return vs;
        }
        if (cfgs[i].model != cfgs[0].model || cfgs[i].scheme != cfgs[0].scheme ||
            (cfgs[0].model == SFT_CUSTOM &&
             (cfgs[i].custom_nl != cfgs[0].custom_nl || cfgs[i].complex_field != cfgs[0].complex_field))) {
            fprintf(stderr, "sft_create_batch: members must share the model and the scheme\n");
            return SFT_EUNSUPPORTED;
        }
    }
    sft_ctx* ctx = new (std::nothrow) sft_ctx();
    if (!ctx) return SFT_ENOMEM;
    auto cleanup = [&](sft_status s) {
        sft_destroy(ctx);
        return s;
    };
    ctx->is_batch = true;
    ctx->cfg = cfgs[0];
    ctx->d = cfgs[0].d;
    model_kind(&cfgs[0], &ctx->cplx, &ctx->nl);
    ctx->cfg.c_re = ctx->cfg.c_im = ctx->cfg.noise_D = ctx->cfg.nl_re = ctx->cfg.nl_im = nullptr;
    if (cfgs[0].stream) {
        ctx->stream = (cudaStream_t)cfgs[0].stream;
    } else {
        if (cudaStreamCreate(&ctx->stream) != cudaSuccess) return cleanup(SFT_ECUDA);
        ctx->own_stream = true;
    }
    if (cudaEventCreateWithFlags(&ctx->ev_fork, cudaEventDisableTiming) != cudaSuccess) return cleanup(SFT_ECUDA);
    if (cudaMalloc(&ctx->dstep, 4 * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&ctx->dstatus, sizeof(unsigned)) != cudaSuccess || cudaMalloc(&ctx->d_head, sizeof(int)) != cudaSuccess)
        return cleanup(SFT_ENOMEM);
    long long init[4] = {0, -1, (long long)0x7fffffffffffffffLL, 0};
    if (cudaMemcpy(ctx->dstep, init, sizeof(init), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(ctx->dstatus, 0, sizeof(unsigned)) != cudaSuccess)
        return cleanup(SFT_ECUDA);
    std::vector<BatchMember> hm;
    std::vector<std::pair<int, BatchItem>> items;  // (M, item)
    long long roff = 0;
    for (int i = 0; i < count; ++i) {
        sft_config c = cfgs[i];
        c.stream = ctx->stream;
        sft_ctx* m = nullptr;
        sft_status st = sft_create(&c, &m);
        if (st != SFT_OK) return cleanup(st);
        ctx->members.push_back(m);
        ctx->rep_offset.push_back(roff);
        roff += m->R;
        const int M = m->nx / 2;
        // lines the persistent kernel takes; longer ones that the cluster kernel runs better (few replicas) go solo
        // members with a step variant (real-space noise, phase shifts) or p x 2^k points run their own kernels
        // on a graph branch of their own
        const bool plain_line = m->d == 1 && !m->cplx && c.noise_space == 0 && c.dealias != 2 && is_pow2(m->nx);
        const int lines = (plain_line && !k1_use_cluster(m->nx, m->R, MODE_STEP)) ? batch_lines_per_item(M) : 0;
        if (lines > 0) {
            BatchMember bm{};
            bm.a = base_args(m);
            bm.a.tw_a = m->tw.get(m->nx / 2);
            bm.a.tw_b = m->tw.get(m->nx);
            bm.a.step_base = ctx->dstep;  // one counter for every member of the persistent launch
            bm.a.status = ctx->dstatus;
            bm.a.bad_step = ctx->dstep + 2;
            bm.M = M;
            for (int r0 = 0; r0 < m->R; r0 += lines)
                items.push_back({M, BatchItem{(int)hm.size(), r0}});
            hm.push_back(bm);
        } else {
            ctx->solo.push_back(i);
        }
    }
    ctx->R = (int)roff;
    // largest lattices first, so the long items do not finish last
    std::stable_sort(items.begin(), items.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
    std::vector<BatchItem> hi;
    for (auto& it : items) hi.push_back(it.second);
    ctx->nitems = (int)hi.size();
    if (!hm.empty()) {
        if (cudaMalloc(&ctx->d_members, hm.size() * sizeof(BatchMember)) != cudaSuccess ||
            cudaMalloc(&ctx->d_items, hi.size() * sizeof(BatchItem)) != cudaSuccess)
            return cleanup(SFT_ENOMEM);
        if (cudaMemcpy(ctx->d_members, hm.data(), hm.size() * sizeof(BatchMember), cudaMemcpyHostToDevice) !=
                cudaSuccess ||
            cudaMemcpy(ctx->d_items, hi.data(), hi.size() * sizeof(BatchItem), cudaMemcpyHostToDevice) != cudaSuccess)
            return cleanup(SFT_ECUDA);
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        ctx->batch_blocks = std::max(1, std::min(nsm, ctx->nitems));
    }
    for (size_t i = 0; i < ctx->solo.size(); ++i) {
        cudaStream_t st = nullptr;
        cudaEvent_t ev = nullptr;
        if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return cleanup(SFT_ECUDA);
        ctx->sides.push_back(st);
        if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return cleanup(SFT_ECUDA);
        ctx->ev_joins.push_back(ev);
    }
    ctx->launches_per_step = ctx->nitems > 0 ? 1 : 0;
    for (int m : ctx->solo) ctx->launches_per_step += ctx->members[m]->launches_per_step;
    *out = ctx;
    return SFT_OK;
}

// batch: global replica -> (member, local replica)
static sft_ctx* member_of(sft_ctx* ctx, int replica, int* local) {
    for (size_t i = 0; i < ctx->members.size(); ++i) {
        const long long o = ctx->rep_offset[i];
        if (replica >= o && replica < o + ctx->members[i]->R) {
            *local = (int)(replica - o);
            return ctx->members[i];
        }
    }
    return nullptr;
}

static size_t field_bytes(const sft_ctx* m) { return (size_t)m->sites * (m->cplx ? sizeof(float2) : sizeof(float)); }

static sft_status check_replica(sft_ctx* ctx, int replica, size_t bytes, size_t per, int* r0, int* R) {
    if (replica < -1 || replica >= ctx->R) return fail(ctx, SFT_EINVAL, "replica out of range");
    *r0 = replica < 0 ? 0 : replica;
    *R = replica < 0 ? ctx->R : 1;
    if (bytes != per * (size_t)(*R)) return fail(ctx, SFT_EINVAL, "buffer size does not match the field");
    return SFT_OK;
}

sft_status sft_set_field(sft_ctx* ctx, int replica, const void* host, size_t bytes) {
    if (!ctx || !host) return SFT_EINVAL;
    if (ctx->is_batch) {
        if (replica >= 0) {
            int local = 0;
            sft_ctx* m = member_of(ctx, replica, &local);
            if (!m) return fail(ctx, SFT_EINVAL, "replica out of range");
            sft_status st = sft_set_field(m, local, host, bytes);
            return st == SFT_OK ? SFT_OK : fail(ctx, st, m->err);
        }
        size_t total = 0;
        for (sft_ctx* m : ctx->members) total += field_bytes(m) * m->R;
        if (bytes != total) return fail(ctx, SFT_EINVAL, "buffer size does not match the batch");
        const char* p = (const char*)host;
        for (sft_ctx* m : ctx->members) {
            sft_status st = sft_set_field(m, -1, p, field_bytes(m) * m->R);
            if (st != SFT_OK) return fail(ctx, st, m->err);
            p += field_bytes(m) * m->R;
        }
        ctx->p_valid = false;
        return SFT_OK;
    }
    const size_t per = (size_t)ctx->sites * (ctx->cplx ? sizeof(float2) : sizeof(float));
    int r0, R;
    sft_status s = check_replica(ctx, replica, bytes, per, &r0, &R);
    if (s != SFT_OK) return s;
    void* dst = ctx->cplx ? (void*)(ctx->cfield + (size_t)r0 * ctx->sites) : (void*)(ctx->real + (size_t)r0 * ctx->sites);
    CK(cudaMemcpyAsync(dst, host, bytes, cudaMemcpyHostToDevice, ctx->stream));
    s = forward_from_buffer(ctx, r0, R);
    if (s != SFT_OK) return s;
    if (ctx->cfg.scheme == SFT_SETD2) {
        ctx->first_step = ctx->step;
        CK(cudaMemcpyAsync(ctx->dstep + 1, &ctx->first_step, sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return SFT_OK;
}

sft_status sft_init_random(sft_ctx* ctx, double sigma) {
    if (!ctx || !(sigma >= 0)) return SFT_EINVAL;
    if (ctx->is_batch) {
        for (sft_ctx* m : ctx->members) {
            sft_status st = sft_init_random(m, sigma);
            if (st != SFT_OK) return fail(ctx, st, m->err);
        }
        ctx->p_valid = false;
        return SFT_OK;
    }
    CK(launch_init_random(ctx->real, ctx->cfield, ctx->sites, ctx->R, ctx->rep0, ctx->cfg.seed, (float)sigma,
                          ctx->stream));
    ctx->launches += 1;
    sft_status s = forward_from_buffer(ctx, 0, ctx->R);
    if (s != SFT_OK) return s;
    if (ctx->cfg.scheme == SFT_SETD2) {
        ctx->first_step = ctx->step;
        CK(cudaMemcpyAsync(ctx->dstep + 1, &ctx->first_step, sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return SFT_OK;
}

static sft_status read_status(sft_ctx* ctx) {
    for (sft_ctx* m : ctx->members) {
        sft_status s = read_status(m);
        if (s != SFT_OK) return fail(ctx, s, m->err);
    }
    unsigned st = 0;
    long long bad = 0;
    CK(cudaMemcpyAsync(&st, ctx->dstatus, sizeof(unsigned), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&bad, ctx->dstep + 2, sizeof(long long), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    if (st & 2u) return fail(ctx, SFT_ETIMEOUT, "a bounded device-side wait ran out; the step was abandoned");
    if (st & 1u) {
        char buf[128];
        snprintf(buf, sizeof buf, "non-finite state first seen at step %lld", bad);
        return fail(ctx, SFT_ENONFINITE, buf);
    }
    return SFT_OK;
}

sft_status sft_sync(sft_ctx* ctx) {
    if (!ctx) return SFT_EINVAL;
    CK(cudaStreamSynchronize(ctx->stream));
    return read_status(ctx);
}

// ------------------------------------------------------------ dynamic observables
static void drop_graph(sft_ctx* ctx) {
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    ctx->warmed = false;  // the next chunk runs plain first, then is captured with the new arguments
}

static void stop_recording(sft_ctx* ctx) {
    if (ctx->rec_phi) cudaFree(ctx->rec_phi);
    if (ctx->rec_F) cudaFree(ctx->rec_F);
    ctx->rec_phi = ctx->rec_F = nullptr;
    ctx->rec_M = 0;
    drop_graph(ctx);
}

sft_status sft_dyn_start(sft_ctx* ctx, int M, int every) {
    if (!ctx) return SFT_EINVAL;
    if (ctx->is_batch) return fail(ctx, SFT_EUNSUPPORTED, "not available on a batch context; use its members' configurations individually");
    if (ctx->d != 2 || ctx->cplx)
        return fail(ctx, SFT_EUNSUPPORTED, "dynamic observables are built for 2-D real fields");
    if (ctx->noise_spec || ctx->cfg.dealias == 2 || !is_pow2(ctx->nx))
        return fail(ctx, SFT_EUNSUPPORTED,
                    "dynamic observables are built for power-of-two lattices with the Fourier-space noise and 2/3 "
                    "truncation (or none)");
    if (M < 16 || M > 16384 || (M & (M - 1)) || every < 1)
        return fail(ctx, SFT_EINVAL, "M must be a power of two in [16, 16384] and every >= 1");
    CK(cudaStreamSynchronize(ctx->stream));
    stop_recording(ctx);
    const size_t n = (size_t)ctx->R * ctx->nmodes * M;
    if (cudaMalloc(&ctx->rec_phi, n * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&ctx->rec_F, n * sizeof(float2)) != cudaSuccess) {
        cudaGetLastError();
        stop_recording(ctx);
        return fail(ctx, SFT_ENOMEM, "no device memory for the recorded series");
    }
    CK(cudaMemsetAsync(ctx->rec_phi, 0, n * sizeof(float2), ctx->stream));
    CK(cudaMemsetAsync(ctx->rec_F, 0, n * sizeof(float2), ctx->stream));
    ctx->rec_start = ctx->step;
    ctx->rec_every = every;
    ctx->rec_M = M;
    return SFT_OK;
}

sft_status sft_dyn_result(sft_ctx* ctx, double* C_out, double* chi_out, size_t cap, double* dbar) {
    if (!ctx || !C_out || !chi_out) return SFT_EINVAL;
    if (!ctx->rec_phi) return fail(ctx, SFT_EINVAL, "no recording: call sft_dyn_start first");
    const int M = ctx->rec_M;
    if (ctx->step < ctx->rec_start + (long long)M * ctx->rec_every)
        return fail(ctx, SFT_EINVAL, "the recording is not complete: step M * every times after sft_dyn_start");
    const long long nm = ctx->nmodes;
    if (cap < (size_t)(nm * M)) return fail(ctx, SFT_EINVAL, "output too small");
    CK(cudaStreamSynchronize(ctx->stream));
    sft_status st = read_status(ctx);
    if (st != SFT_OK) return st;
    const size_t n = (size_t)ctx->R * nm * M;
    // time transforms of every (replica, mode) series: the complex line FFT
    std::vector<float2> tw(M);
    for (int m = 0; m < M; ++m) {
        const double ang = 2.0 * M_PI * (double)m / (double)M;
        tw[m] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
    }
    float2 *dtw = nullptr, *Phi = nullptr, *Fw = nullptr;
    double *dc = nullptr, *dD = nullptr, *dC = nullptr;
    double2* dchi = nullptr;
    auto release = [&]() {
        for (void* p : {(void*)dtw, (void*)Phi, (void*)Fw, (void*)dc, (void*)dD, (void*)dC, (void*)dchi})
            if (p) cudaFree(p);
    };
    if (cudaMalloc(&dtw, M * sizeof(float2)) != cudaSuccess || cudaMalloc(&Phi, n * sizeof(float2)) != cudaSuccess ||
        cudaMalloc(&Fw, n * sizeof(float2)) != cudaSuccess || cudaMalloc(&dc, nm * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dD, nm * sizeof(double)) != cudaSuccess || cudaMalloc(&dC, nm * M * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&dchi, nm * M * sizeof(double2)) != cudaSuccess) {
        cudaGetLastError();
        release();
        return fail(ctx, SFT_ENOMEM, "no device memory for the time transforms");
    }
    // c_a and D_a of every stored mode (Sec. V model terms; tables for SFT_CUSTOM)
    std::vector<double> hc(nm), hD(nm);
    const double dk = 2.0 * M_PI / (ctx->nx * ctx->cfg.dx[0]);
    const double* p = ctx->cfg.p;
    for (int cc = 0; cc < ctx->hx; ++cc)
        for (int ay = 0; ay < ctx->ny; ++ay) {
            const long long ays = (2 * ay < ctx->ny) ? ay : ay - ctx->ny;
            const long long q = (long long)cc * cc + ays * ays;
            const double k2 = dk * dk * (double)q;
            double c = 0.0, D = 0.0;
            switch (ctx->cfg.model) {
                case SFT_MODEL_A: c = -p[0] * (p[1] + k2); D = p[0] * p[3]; break;
                case SFT_MODEL_B: c = -p[0] * k2 * (p[1] + k2); D = p[0] * p[3] * k2; break;
                case SFT_KPZ: c = -p[0] * k2; D = p[2]; break;
                default: c = ctx->cust_c[q]; D = ctx->cust_D[q]; break;
            }
            hc[(size_t)cc * ctx->ny + ay] = c;
            hD[(size_t)cc * ctx->ny + ay] = D;
        }
    cudaError_t e = cudaMemcpyAsync(dtw, tw.data(), M * sizeof(float2), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dc, hc.data(), nm * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dD, hD.data(), nm * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
        // step-major record -> one contiguous series per (replica, mode), then its FFT in place
        float2* ser = pass == 0 ? Phi : Fw;
        e = launch_transpose_c(pass == 0 ? ctx->rec_phi : ctx->rec_F, ser, M, (long long)ctx->R * nm, ctx->stream);
        StepArgs t{};
        t.nx = M;
        t.ny = t.nz = 1;
        t.hx = M;
        t.R = (int)(ctx->R * nm);
        t.cplx_io = ser;
        t.phi = ser;
        t.tw_a = dtw;
        if (e == cudaSuccess) e = launch_k1_line(t, MODE_FWD, NL_CGL, ctx->stream);
        ctx->launches += 2;
    }
    DynArgs dv{};
    dv.Phi = Phi;
    dv.Fw = Fw;
    dv.c = dc;
    dv.D = dD;
    dv.R = ctx->R;
    dv.M = M;
    dv.nmodes = nm;
    dv.T = (double)M * ctx->rec_every * ctx->cfg.h;
    double Ld = 1.0;
    for (int i = 0; i < ctx->d; ++i) Ld *= ctx->cfg.dx[i] / ctx->cfg.n[i];  // (L / N^2)^d = (dx / N)^d
    dv.norm = Ld * dv.T / ((double)M * M) / ctx->R;
    dv.C = dC;
    dv.chi = dchi;
    if (e == cudaSuccess) e = launch_dyn_reduce(dv, ctx->stream);
    ctx->launches += 1;
    if (e == cudaSuccess) e = cudaMemcpyAsync(C_out, dC, nm * M * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(chi_out, dchi, nm * M * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    release();
    if (e != cudaSuccess) return fail(ctx, SFT_ECUDA, std::string("dynamic observables: ") + cudaGetErrorString(e));
    // average absolute deviation from the FDT over the modes with noise (Eq. average-deviation)
    if (dbar) {
        double acc = 0.0;
        long long cnt = 0;
        for (long long a = 0; a < nm; ++a) {
            if (!(hD[a] > 0.0)) continue;
            for (int b = 0; b < M; ++b) {
                const int sb = b < M / 2 ? b : b - M;
                const double w = 2.0 * M_PI * sb / dv.T;
                acc += std::fabs(2.0 * chi_out[2 * (a * M + b) + 1] - w / hD[a] * C_out[a * M + b]);
                ++cnt;
            }
        }
        *dbar = cnt ? acc / (double)cnt : 0.0;
    }
    stop_recording(ctx);
    return SFT_OK;
}

sft_status sft_box_width(sft_ctx* ctx, int ell, double* host_out, size_t cap, size_t* written) {
    if (!ctx || !host_out) return SFT_EINVAL;
    if (written) *written = 0;
    if (ctx->is_batch) return fail(ctx, SFT_EUNSUPPORTED, "not available on a batch context; use its members' configurations individually");
    if (ctx->cplx) return fail(ctx, SFT_EUNSUPPORTED, "the box width is defined for real fields");
    const int n[3] = {ctx->nx, ctx->ny, ctx->nz};
    if (ell < 1) return fail(ctx, SFT_EINVAL, "box size must be >= 1");
    for (int i = 0; i < ctx->d; ++i)
        if (n[i] % ell != 0) return fail(ctx, SFT_EINVAL, "box size must divide every lattice size");
    if (cap < (size_t)ctx->R) return fail(ctx, SFT_EINVAL, "output too small");
    sft_status s = inverse_to_buffer(ctx, ctx->phi, 0, ctx->R);
    if (s != SFT_OK) return s;
    CK(cudaMemsetAsync(ctx->drough, 0, sizeof(double) * ctx->R, ctx->stream));
    CK(launch_box_width(ctx->real, ctx->nx, ctx->ny, ctx->nz, ctx->d, ell, ctx->R, ctx->drough, ctx->stream));
    ctx->launches += 1;
    std::vector<double> acc(ctx->R);
    CK(cudaMemcpyAsync(acc.data(), ctx->drough, sizeof(double) * ctx->R, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    double nboxes = 1.0;
    for (int i = 0; i < ctx->d; ++i) nboxes *= (double)(n[i] / ell);
    for (int r = 0; r < ctx->R; ++r) host_out[r] = acc[r] / nboxes;
    if (written) *written = (size_t)ctx->R;
    return read_status(ctx);
}

sft_status sft_get_field(sft_ctx* ctx, int replica, void* host_out, size_t bytes) {
    if (!ctx || !host_out) return SFT_EINVAL;
    if (ctx->is_batch) {
        if (replica >= 0) {
            int local = 0;
            sft_ctx* m = member_of(ctx, replica, &local);
            if (!m) return fail(ctx, SFT_EINVAL, "replica out of range");
            sft_status st = sft_get_field(m, local, host_out, bytes);
            return st == SFT_OK ? SFT_OK : fail(ctx, st, m->err);
        }
        size_t total = 0;
        for (sft_ctx* m : ctx->members) total += field_bytes(m) * m->R;
        if (bytes != total) return fail(ctx, SFT_EINVAL, "buffer size does not match the batch");
        char* p = (char*)host_out;
        for (sft_ctx* m : ctx->members) {
            sft_status st = sft_get_field(m, -1, p, field_bytes(m) * m->R);
            if (st != SFT_OK) return fail(ctx, st, m->err);
            p += field_bytes(m) * m->R;
        }
        return read_status(ctx);
    }
    const size_t per = (size_t)ctx->sites * (ctx->cplx ? sizeof(float2) : sizeof(float));
    int r0, R;
    sft_status s = check_replica(ctx, replica, bytes, per, &r0, &R);
    if (s != SFT_OK) return s;
    s = inverse_to_buffer(ctx, ctx->phi, r0, R);
    if (s != SFT_OK) return s;
    const void* src =
        ctx->cplx ? (const void*)(ctx->cfield + (size_t)r0 * ctx->sites) : (const void*)(ctx->real + (size_t)r0 * ctx->sites);
    CK(cudaMemcpyAsync(host_out, src, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    return read_status(ctx);
}

sft_status sft_get_spectrum(sft_ctx* ctx, void* host_out, size_t bytes) {
    if (!ctx || !host_out) return SFT_EINVAL;
    if (ctx->is_batch) return fail(ctx, SFT_EUNSUPPORTED, "not available on a batch context; use its members' configurations individually");
    if (bytes != (size_t)ctx->R * ctx->nmodes * sizeof(float2)) return fail(ctx, SFT_EINVAL, "spectrum size mismatch");
    CK(cudaMemcpyAsync(host_out, ctx->phi, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    return read_status(ctx);
}

sft_status sft_set_spectrum(sft_ctx* ctx, const void* host_in, size_t bytes) {
    if (!ctx || !host_in) return SFT_EINVAL;
    if (ctx->is_batch) return fail(ctx, SFT_EUNSUPPORTED, "not available on a batch context; use its members' configurations individually");
    if (bytes != (size_t)ctx->R * ctx->nmodes * sizeof(float2)) return fail(ctx, SFT_EINVAL, "spectrum size mismatch");
    CK(cudaMemcpyAsync(ctx->phi, host_in, bytes, cudaMemcpyHostToDevice, ctx->stream));
    ctx->p_valid = false;
    if (ctx->cfg.scheme == SFT_SETD2) {
        ctx->first_step = ctx->step;
        CK(cudaMemcpyAsync(ctx->dstep + 1, &ctx->first_step, sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return SFT_OK;
}

static sft_status step_impl(sft_ctx* ctx, int64_t nsteps, bool use_graph) {
    if (!ctx || nsteps < 0) return SFT_EINVAL;
    if (ctx->step + nsteps > (long long)0xFFFFFFFFLL)
        return fail(ctx, SFT_EINVAL, "the noise counter holds 2^32 steps per context");
    if (!ctx->p_valid) {
        sft_status s = prime(ctx);
        if (s != SFT_OK) return s;
    }
    if (!ctx->planned) {
        sft_status s = plan_step(ctx);
        if (s != SFT_OK) return s;
    }
    int64_t left = nsteps;
    if (use_graph && left >= kGraphChunk) {
        if (!ctx->warmed) {
            // first chunk runs as plain launches (sets kernel attributes outside capture)
            for (int k = 0; k < kGraphChunk; ++k) {
                sft_status s = enqueue_step(ctx, k);
                if (s != SFT_OK) return s;
            }
            CK(advance_all(ctx, kGraphChunk));
            ctx->launches += (long long)kGraphChunk * ctx->launches_per_step + advances_per_chunk(ctx);
            left -= kGraphChunk;
            ctx->warmed = true;
        }
        if (left >= kGraphChunk && !ctx->graph) {
            sft_status s = capture_graph(ctx);
            if (s != SFT_OK) return s;
        }
        while (left >= kGraphChunk) {
            CK(cudaGraphLaunch(ctx->graph, ctx->stream));
            ctx->launches += (long long)kGraphChunk * ctx->launches_per_step + advances_per_chunk(ctx);
            left -= kGraphChunk;
        }
    }
    for (int64_t i = 0; i < left; ++i) {
        sft_status s = enqueue_step(ctx, 0);
        if (s != SFT_OK) return s;
        CK(advance_all(ctx, 1));
        ctx->launches += ctx->launches_per_step + advances_per_chunk(ctx);
    }
    ctx->step += nsteps;
    for (sft_ctx* m : ctx->members) m->step += nsteps;
    return SFT_OK;
}

sft_status sft_step(sft_ctx* ctx, int64_t nsteps) { return step_impl(ctx, nsteps, true); }

sft_status sft_prepare(sft_ctx* ctx) {
    if (!ctx) return SFT_EINVAL;
    if (!ctx->p_valid) {
        sft_status s = prime(ctx);
        if (s != SFT_OK) return s;
    }
    if (!ctx->planned) {
        sft_status s = plan_step(ctx);
        if (s != SFT_OK) return s;
    }
    if (!ctx->graph) {
        // capture only: the graph is instantiated, nothing runs and the state is untouched
        sft_status s = capture_graph(ctx);
        if (s != SFT_OK) return s;
    }
    ctx->warmed = true;
    CK(cudaStreamSynchronize(ctx->stream));
    return SFT_OK;
}

sft_status sft_get_plan(sft_ctx* ctx, int* out, int cap) {
    if (!ctx || !out || cap < 4) return SFT_EINVAL;
    if (ctx->is_batch) return fail(ctx, SFT_EUNSUPPORTED, "not available on a batch context; use its members' configurations individually");
    if (!ctx->p_valid) {
        sft_status s = prime(ctx);
        if (s != SFT_OK) return s;
    }
    sft_status s = plan_step(ctx);
    if (s != SFT_OK) return s;
    out[0] = ctx->row_shape;
    out[1] = ctx->col_shape;
    out[2] = ctx->rpb > 0 ? ctx->rpb : 4;
    out[3] = ctx->pipe_cols ? 1 : 0;
    return SFT_OK;
}

sft_status sft_set_plan(sft_ctx* ctx, const int* plan, int n) {
    if (!ctx || !plan || n < 4) return SFT_EINVAL;
    if (ctx->is_batch) return fail(ctx, SFT_EUNSUPPORTED, "not available on a batch context; use its members' configurations individually");
    const bool real2 = ctx->d >= 2 && !ctx->cplx;
    if (plan[0] < 0 || (real2 ? !row_shape_ok(ctx, plan[0]) : plan[0] != 0) || plan[1] < 0 ||
        (real2 && ctx->d == 2 ? !col_shape_ok(ctx, plan[1]) : plan[1] != 0) || plan[2] < 1 || plan[2] > 64 ||
        (plan[3] != 0 && !(ctx->d == 2 && k2_pipe_supported(ctx->nx, ctx->ny, ctx->cplx))))
        return fail(ctx, SFT_EINVAL, "schedule outside the variants built for this lattice");
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->planned = true;
    ctx->row_shape = plan[0];
    ctx->col_shape = plan[1];
    ctx->rpb = plan[2];
    ctx->pipe_cols = plan[3] != 0;
    ctx->pipe_forced = true;
    if (ctx->graph) {
        cudaGraphExecDestroy(ctx->graph);
        ctx->graph = nullptr;
    }
    ctx->warmed = false;  // the next chunk runs plain first (kernel attributes outside capture)
    return SFT_OK;
}
sft_status sft_step_plain(sft_ctx* ctx, int64_t nsteps) { return step_impl(ctx, nsteps, false); }

sft_status sft_observe(sft_ctx* ctx, int kind, double* host_out, size_t cap, size_t* written) {
    if (!ctx) return SFT_EINVAL;
    if (written) *written = 0;
    if (ctx->is_batch) {
        if (kind != SFT_OBS_ROUGHNESS)
            return fail(ctx, SFT_EUNSUPPORTED, "a batch of uneven lattices supports the per-replica roughness only");
        if (!host_out || cap < (size_t)ctx->R) return fail(ctx, SFT_EINVAL, "output too small");
        size_t w = 0;
        for (sft_ctx* m : ctx->members) {
            size_t wm = 0;
            sft_status st = sft_observe(m, kind, host_out + w, cap - w, &wm);
            if (st != SFT_OK) return fail(ctx, st, m->err);
            w += wm;
        }
        if (written) *written = w;
        return SFT_OK;
    }
    const int ns = ctx->nshells;
    if (kind == SFT_OBS_NSHELLS) {
        if (!host_out || cap < 1) return fail(ctx, SFT_EINVAL, "output too small");
        host_out[0] = ns;
        if (written) *written = 1;
        return SFT_OK;
    }
    if (kind == SFT_OBS_MARK) {
        if (!ctx->snap) CK(cudaMalloc(&ctx->snap, (size_t)ctx->R * ctx->nmodes * sizeof(float2)));
        CK(cudaMemcpyAsync(ctx->snap, ctx->phi, (size_t)ctx->R * ctx->nmodes * sizeof(float2),
                           cudaMemcpyDeviceToDevice, ctx->stream));
        return read_status(ctx);
    }
    if (kind == SFT_OBS_SK_RESET) {
        CK(cudaMemsetAsync(ctx->d_tacc, 0, (size_t)ns * sizeof(double2), ctx->stream));
        ctx->tacc_count = 0;
        return SFT_OK;
    }
    if (kind == SFT_OBS_SK_TIME_MEAN) {
        if (!host_out || cap < (size_t)ns + 1) return fail(ctx, SFT_EINVAL, "output too small");
        std::vector<double2> acc(ns);
        CK(cudaMemcpyAsync(acc.data(), ctx->d_tacc, (size_t)ns * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
        sft_status s = read_status(ctx);
        if (s != SFT_OK) return s;
        const double samples = (double)ctx->tacc_count * ctx->R;
        for (int j = 0; j < ns; ++j)
            host_out[j] = (ctx->counts[j] > 0 && samples > 0) ? (acc[j].x + acc[j].y) / (ctx->counts[j] * samples) : 0.0;
        host_out[ns] = (double)ctx->tacc_count;
        if (written) *written = ns + 1;
        return SFT_OK;
    }
    if (kind < 0 || kind > SFT_OBS_SK_RESET) return fail(ctx, SFT_EINVAL, "unknown observable");
    if (!host_out && kind != SFT_OBS_SK_ACCUM) return SFT_EINVAL;
    if (kind == SFT_OBS_CKT && !ctx->snap) return fail(ctx, SFT_EINVAL, "two-time correlation needs SFT_OBS_MARK first");
    if (kind == SFT_OBS_RESPONSE && !ctx->dseed) return fail(ctx, SFT_EINVAL, "response needs a seeded tangent");
    ObsArgs o{};
    o.nx = ctx->nx;
    o.ny = ctx->ny;
    o.nz = ctx->nz;
    o.hx = ctx->hx;
    o.R = ctx->R;
    o.complex_field = ctx->cplx;
    o.nshells = ns;
    o.order = ctx->d_order;
    o.chunks = ctx->d_chunks;
    o.first_chunk = ctx->d_first_chunk;
    o.nchunks = ctx->nchunks;
    o.part = ctx->d_part;
    double norm = 1.0;
    for (int i = 0; i < ctx->d; ++i) norm *= ctx->cfg.dx[i] / ctx->cfg.n[i];
    const size_t nsum = (size_t)ctx->R * ns;
    std::vector<double> sums(nsum), sums2;
    if (kind == SFT_OBS_SK_ACCUM) {
        // S(k) of the current state added to the device time accumulator; nothing comes back
        o.phi = ctx->phi;
        o.norm = norm;
        o.kind = 0;
        o.shell_sum = ctx->dshell;
        CK(launch_observe(o, ctx->stream));
        CK(launch_obs_time_acc(ctx->dshell, ctx->R, ns, ctx->d_tacc, ctx->stream));
        ctx->launches += 3;
        ctx->tacc_count += 1;
        return SFT_OK;
    }
    if (kind == SFT_OBS_RESPONSE) {
        o.phi = ctx->dphi;
        o.ref = ctx->dseed;
        o.norm = 1.0;
        o.kind = 1;
        o.shell_sum = ctx->dshell;
        CK(launch_observe(o, ctx->stream));
        ctx->launches += 2;
        CK(cudaMemcpyAsync(sums.data(), ctx->dshell, nsum * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));
        sums2.resize(nsum);
        o.kind = 2;
        CK(launch_observe(o, ctx->stream));
        ctx->launches += 2;
        CK(cudaMemcpyAsync(sums2.data(), ctx->dshell, nsum * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        sft_status s = read_status(ctx);
        if (s != SFT_OK) return s;
        if (cap < (size_t)ns) return fail(ctx, SFT_EINVAL, "output too small");
        for (int j = 0; j < ns; ++j) {
            double num = 0, den = 0;
            for (int r = 0; r < ctx->R; ++r) {
                num += sums[(size_t)r * ns + j];
                den += sums2[(size_t)r * ns + j];
            }
            host_out[j] = den > 0 ? num / den : 0.0;
        }
        if (written) *written = ns;
        return SFT_OK;
    }
    o.phi = ctx->phi;
    o.ref = kind == SFT_OBS_CKT ? ctx->snap : nullptr;
    o.norm = norm;
    o.kind = kind == SFT_OBS_CKT ? 1 : 0;
    o.shell_sum = ctx->dshell;
    CK(launch_observe(o, ctx->stream));
    ctx->launches += 2;
    CK(cudaMemcpyAsync(sums.data(), ctx->dshell, nsum * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    sft_status s = read_status(ctx);
    if (s != SFT_OK) return s;
    if (kind == SFT_OBS_ROUGHNESS) {
        // w^2 = N^{-2d} sum_{a != 0} |phi_a|^2: every shell but j = 0 (which holds a = 0 alone), summed
        // in shell order with compensation
        if (cap < (size_t)ctx->R) return fail(ctx, SFT_EINVAL, "output too small");
        const double n2 = (double)ctx->sites * (double)ctx->sites;
        for (int r = 0; r < ctx->R; ++r) {
            double acc = 0.0, c = 0.0;
            for (int j = 1; j < ns; ++j) {
                const double x = sums[(size_t)r * ns + j], t = acc + x;
                c += std::fabs(acc) >= std::fabs(x) ? (acc - t) + x : (x - t) + acc;
                acc = t;
            }
            host_out[r] = (acc + c) / norm / n2;
        }
        if (written) *written = ctx->R;
        return SFT_OK;
    }
    if (kind == SFT_OBS_SK_REPLICAS) {
        if (cap < nsum) return fail(ctx, SFT_EINVAL, "output too small");
        for (int r = 0; r < ctx->R; ++r)
            for (int j = 0; j < ns; ++j)
                host_out[(size_t)r * ns + j] = ctx->counts[j] > 0 ? sums[(size_t)r * ns + j] / ctx->counts[j] : 0.0;
        if (written) *written = nsum;
        return SFT_OK;
    }
    if (cap < (size_t)ns) return fail(ctx, SFT_EINVAL, "output too small");
    for (int j = 0; j < ns; ++j) {
        double acc = 0;
        for (int r = 0; r < ctx->R; ++r) acc += sums[(size_t)r * ns + j];
        host_out[j] = ctx->counts[j] > 0 ? acc / (ctx->counts[j] * ctx->R) : 0.0;
    }
    size_t w = ns;
    if (cap >= 2 * (size_t)ns) {
        for (int j = 0; j < ns; ++j) host_out[ns + j] = ctx->counts[j];
        w = 2 * ns;
    }
    if (written) *written = w;
    return SFT_OK;
}

// adjoint: whether the adjoint (not only the tangent) is asked for
static sft_status diff_supported(sft_ctx* ctx, bool adjoint) {
    // tangent: the cubic term in 1-D, 2-D and 3-D; the KPZ term and the complex |A|^2 A term (CGL) in 1-D and
    // 2-D (complex rows up to 2048 points); adjoint: the cubic term and the KPZ and CGL terms in 1-D and 2-D
    const bool tan_term = ctx->nl == NL_CUBIC ||
                          (ctx->d <= 2 && ctx->nl == NL_GRAD2) ||
                          (ctx->nl == NL_CGL && (ctx->d == 1 || (ctx->d == 2 && ctx->nx <= 2048)));
    const bool adj_term = ctx->nl == NL_CUBIC || (ctx->d <= 2 && ctx->nl == NL_GRAD2) ||
                          (ctx->nl == NL_CGL && (ctx->d == 1 || (ctx->d == 2 && ctx->nx <= 2048)));
    if (!(adjoint ? adj_term : tan_term) || (ctx->d == 1 && ctx->nx > 32768) || ctx->cfg.dealias == 2 ||
        !is_pow2(ctx->nx) || ctx->cfg.noise_space != 0)
        return fail(ctx, SFT_EUNSUPPORTED,
                    "the tangent is built for the cubic term (Model A/B, d = 1..3) and the KPZ and CGL terms "
                    "(d = 1, 2; complex rows up to 2048 points); the adjoint likewise; "
                    "every scheme; 1-D lines up to 32768 points, power-of-two lattices, 2/3 truncation or "
                    "none, Fourier-space noise");
    const size_t ms = (size_t)ctx->R * ctx->nmodes * sizeof(float2);
    if (!ctx->dphi) {
        CK(cudaMalloc(&ctx->dphi, ms));
        CK(cudaMemsetAsync(ctx->dphi, 0, ms, ctx->stream));
    }
    if (ctx->cfg.scheme == SFT_SETD2 && !ctx->dfprev) {
        CK(cudaMalloc(&ctx->dfprev, ms));
        CK(cudaMemsetAsync(ctx->dfprev, 0, ms, ctx->stream));
    }
    if (adjoint && ctx->cfg.scheme == SFT_SETD2 && !ctx->dmu) CK(cudaMalloc(&ctx->dmu, ms));
    if (!ctx->dseed) CK(cudaMalloc(&ctx->dseed, ms));
    if (ctx->d >= 2 && !ctx->dP) {
        CK(cudaMalloc(&ctx->dP, ms));
        CK(cudaMalloc(&ctx->dQ, ms));
        CK(cudaMemsetAsync(ctx->dP, 0, ms, ctx->stream));
        CK(cudaMemsetAsync(ctx->dQ, 0, ms, ctx->stream));
    }
    if (ctx->d >= 2 && ctx->nl == NL_GRAD2 && !ctx->dPy) {
        CK(cudaMalloc(&ctx->dPy, ms));
        CK(cudaMemsetAsync(ctx->dPy, 0, ms, ctx->stream));
    }
    return SFT_OK;
}

static sft_status set_step_counter(sft_ctx* ctx, long long step) {
    ctx->step = step;
    CK(cudaMemcpyAsync(ctx->dstep, &step, sizeof(long long), cudaMemcpyHostToDevice, ctx->stream));
    return SFT_OK;
}

// dst spectrum <- forward transform of R real-space fields at a device pointer
static sft_status spectrum_from_device_field(sft_ctx* ctx, const void* dev_field, float2* dst) {
    const size_t rs = (size_t)ctx->R * ctx->sites * (ctx->cplx ? sizeof(float2) : sizeof(float));
    CK(cudaMemcpyAsync(ctx->cplx ? (void*)ctx->cfield : (void*)ctx->real, dev_field, rs, cudaMemcpyDeviceToDevice,
                       ctx->stream));
    sft_status s = forward_from_buffer(ctx, 0, ctx->R, dst);
    if (s != SFT_OK) return s;
    ctx->launches += ctx->d == 1 ? 1 : 2;
    return SFT_OK;
}

static sft_status device_field_from_spectrum(sft_ctx* ctx, const float2* src, void* dev_field) {
    sft_status s = inverse_to_buffer(ctx, src, 0, ctx->R);
    if (s != SFT_OK) return s;
    ctx->launches += ctx->d == 1 ? 1 : 2;
    CK(cudaMemcpyAsync(dev_field, ctx->cplx ? (const void*)ctx->cfield : (const void*)ctx->real,
                       (size_t)ctx->R * ctx->sites * (ctx->cplx ? sizeof(float2) : sizeof(float)),
                       cudaMemcpyDeviceToDevice, ctx->stream));
    return SFT_OK;
}

sft_status sft_tangent_step(sft_ctx* ctx, const void* dphi0_dev, int64_t nsteps, void* dphi_out_dev) {
    if (!ctx || nsteps < 0) return SFT_EINVAL;
    if (ctx->is_batch) return fail(ctx, SFT_EUNSUPPORTED, "not available on a batch context; use its members' configurations individually");
    sft_status s = diff_supported(ctx, false);
    if (s != SFT_OK) return s;
    const size_t ms = (size_t)ctx->R * ctx->nmodes * sizeof(float2);
    if (dphi0_dev) {
        s = spectrum_from_device_field(ctx, dphi0_dev, ctx->dphi);
        if (s != SFT_OK) return s;
        CK(cudaMemcpyAsync(ctx->dseed, ctx->dphi, ms, cudaMemcpyDeviceToDevice, ctx->stream));
        // a perturbation seeded now leaves the nonlinear term of the previous step unchanged
        if (ctx->dfprev) CK(cudaMemsetAsync(ctx->dfprev, 0, ms, ctx->stream));
        ctx->dp_valid = false;
    }
    if (!ctx->p_valid) {
        s = prime(ctx);
        if (s != SFT_OK) return s;
    }
    if (ctx->d >= 2 && !ctx->dp_valid) {
        StepArgs a = base_args(ctx);
        a.phi = ctx->dphi;
        a.pout = ctx->dP;
        a.pyout = ctx->dPy;
        a.tw_a = ctx->tw.get(ctx->ny);
        CK(launch_second(ctx, a, MODE_PRIME));
        ctx->launches += 1;
        ctx->dp_valid = true;
    }
    for (int64_t i = 0; i < nsteps; ++i) {
        StepArgs a = base_args(ctx);
        a.dphi = ctx->dphi;
        a.dfprev = ctx->dfprev;
        if (ctx->d == 1) {
            // complex lines: one C2C length; real lines: the half length and the full length
            if (!set_line_twiddles(ctx, a)) return fail(ctx, SFT_EINVAL, "twiddle table missing");
            CK(launch_k1_line(a, MODE_TAN, ctx->nl, ctx->stream));
            ctx->launches += 1;
        } else {
            a.pin = ctx->P;
            a.dpin = ctx->dP;
            a.pyin = ctx->Py;
            a.dpyin = ctx->dPy;
            a.qout = ctx->Q;
            a.dqout = ctx->dQ;
            a.tw_a = ctx->tw.get(ctx->nx / 2);
            a.tw_b = ctx->tw.get(ctx->nx);
            CK(launch_rows(ctx, a, MODE_TAN));
            a.qin = ctx->Q;
            a.dqin = ctx->dQ;
            a.pout = ctx->P;
            a.dpout = ctx->dP;
            a.pyout = ctx->Py;
            a.dpyout = ctx->dPy;
            a.tw_a = ctx->tw.get(ctx->ny);
            if (ctx->d == 3) {
                // the plane pass runs the primal step, then the (noise-free) tangent update
                CK(launch_second(ctx, a, MODE_STEP));
                CK(launch_second(ctx, a, MODE_TAN));
                ctx->launches += 1;
            } else {
                CK(launch_second(ctx, a, MODE_TAN));
            }
            ctx->launches += 2;
        }
        CK(launch_advance(ctx->dstep, 1, ctx->stream));
        ctx->launches += 1;
    }
    ctx->step += nsteps;
    if (dphi_out_dev) {
        s = device_field_from_spectrum(ctx, ctx->dphi, dphi_out_dev);
        if (s != SFT_OK) return s;
    }
    return read_status(ctx);
}

sft_status sft_adjoint(sft_ctx* ctx, const void* cot_dev, int64_t nsteps, void* grad_dev) {
    if (!ctx || !cot_dev || !grad_dev || nsteps < 1) return SFT_EINVAL;
    if (ctx->is_batch) return fail(ctx, SFT_EUNSUPPORTED, "not available on a batch context; use its members' configurations individually");
    sft_status s = diff_supported(ctx, true);
    if (s != SFT_OK) return s;
    const size_t ms = (size_t)ctx->R * ctx->nmodes * sizeof(float2);
    const int64_t K = ctx->ckpt_segment;
    const int64_t nseg = (nsteps + K - 1) / K;
    const long long step0 = ctx->step;
    float2 *ckpt = nullptr, *traj = nullptr, *trajy = nullptr, *phiN = nullptr;
    auto release = [&]() {
        if (ckpt) cudaFree(ckpt);
        if (traj) cudaFree(traj);
        if (trajy) cudaFree(trajy);
        if (phiN) cudaFree(phiN);
    };
#define CKA(call)                                                                                     \
    do {                                                                                              \
        cudaError_t e_ = (call);                                                                      \
        if (e_ != cudaSuccess) {                                                                      \
            release();                                                                                \
            return fail(ctx, SFT_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_));          \
        }                                                                                             \
    } while (0)
#define SKA(expr)                   \
    do {                            \
        sft_status s_ = (expr);     \
        if (s_ != SFT_OK) {         \
            release();              \
            return s_;              \
        }                           \
    } while (0)
    // a checkpoint holds the state and, for SETD2, the history F_prev that the next step reads
    const bool hist = ctx->cfg.scheme == SFT_SETD2;
    const size_t cs = hist ? 2 * ms : ms;
    const size_t cm = hist ? 2 * (size_t)ctx->R * ctx->nmodes : (size_t)ctx->R * ctx->nmodes;  // in float2
    if (cudaMalloc(&ckpt, cs * (size_t)nseg) != cudaSuccess || cudaMalloc(&traj, ms * (size_t)(K + 1)) != cudaSuccess ||
        cudaMalloc(&phiN, cs) != cudaSuccess) {
        release();
        return fail(ctx, SFT_ENOMEM, "adjoint checkpoint buffers");
    }
    // the KPZ term in 2-D also keeps each step's second intermediate P_y = IDFT_y(i k_y M phi)
    const bool grad2d = ctx->d >= 2 && ctx->nl == NL_GRAD2;
    if (grad2d && cudaMalloc(&trajy, ms * (size_t)(K + 1)) != cudaSuccess) {
        release();
        return fail(ctx, SFT_ENOMEM, "adjoint checkpoint buffers");
    }
    // forward sweep: state at the start of every segment
    for (int64_t sg = 0; sg < nseg; ++sg) {
        CKA(cudaMemcpyAsync(ckpt + (size_t)sg * cm, ctx->phi, ms, cudaMemcpyDeviceToDevice, ctx->stream));
        if (hist)
            CKA(cudaMemcpyAsync(ckpt + (size_t)sg * cm + cm / 2, ctx->fprev, ms, cudaMemcpyDeviceToDevice,
                                ctx->stream));
        SKA(step_impl(ctx, std::min<int64_t>(K, nsteps - sg * K), true));
    }
    CKA(cudaMemcpyAsync(phiN, ctx->phi, ms, cudaMemcpyDeviceToDevice, ctx->stream));
    if (hist) CKA(cudaMemcpyAsync(phiN + cm / 2, ctx->fprev, ms, cudaMemcpyDeviceToDevice, ctx->stream));
    // lambda_N; the SETD2 history cotangent mu_{N-1} = 0
    SKA(spectrum_from_device_field(ctx, cot_dev, ctx->dphi));
    if (ctx->dmu) CKA(cudaMemsetAsync(ctx->dmu, 0, ms, ctx->stream));
    // whether step n of the sweep (global index step0 + n) took the SETD1 pair that starts SETD2
    auto starts_setd2 = [&](int64_t n) {
        return ctx->cfg.scheme == SFT_SETD2 && n >= 0 && step0 + n == ctx->first_step ? 1 : 0;
    };
    bool w_valid = false;
    for (int64_t sg = nseg - 1; sg >= 0; --sg) {
        const int64_t n0 = sg * K, len = std::min<int64_t>(K, nsteps - n0);
        // recompute the segment, keeping each step's primal input
        CKA(cudaMemcpyAsync(ctx->phi, ckpt + (size_t)sg * cm, ms, cudaMemcpyDeviceToDevice, ctx->stream));
        if (hist)
            CKA(cudaMemcpyAsync(ctx->fprev, ckpt + (size_t)sg * cm + cm / 2, ms, cudaMemcpyDeviceToDevice,
                                ctx->stream));
        SKA(set_step_counter(ctx, step0 + n0));
        const size_t sl = (size_t)ctx->R * ctx->nmodes;  // one trajectory slot, in float2
        if (ctx->d >= 2) {
            StepArgs a = base_args(ctx);
            a.pout = traj;
            a.pyout = grad2d ? trajy : ctx->Py;
            a.tw_a = ctx->tw.get(ctx->ny);
            CKA(launch_second(ctx, a, MODE_PRIME));
        }
        for (int64_t i = 0; i < len; ++i) {
            float2* slot = traj + (size_t)i * sl;
            if (ctx->d == 1) {
                CKA(cudaMemcpyAsync(slot, ctx->phi, ms, cudaMemcpyDeviceToDevice, ctx->stream));
                SKA(enqueue_step_io(ctx, nullptr, nullptr));
            } else if (grad2d) {
                float2* sloty = trajy + (size_t)i * sl;
                SKA(enqueue_step_io(ctx, slot, slot + sl, sloty, sloty + sl));
            } else {
                SKA(enqueue_step_io(ctx, slot, slot + sl));
            }
        }
        // reverse sweep over the segment
        for (int64_t i = len - 1; i >= 0; --i) {
            float2* slot = traj + (size_t)i * ctx->R * ctx->nmodes;
            StepArgs a = base_args(ctx);
            a.dphi = ctx->dphi;
            a.dmu = ctx->dmu;
            a.adj_first_n = starts_setd2(n0 + i);
            a.adj_first_prev = starts_setd2(n0 + i - 1);
            if (ctx->d == 1) {
                a.phi = slot;
                if (!set_line_twiddles(ctx, a)) {
                    release();
                    return fail(ctx, SFT_EINVAL, "twiddle table missing");
                }
                CKA(launch_k1_line(a, MODE_ADJ, ctx->nl, ctx->stream));
                ctx->launches += 1;
            } else {
                if (!w_valid) {
                    // W_{N-1} = IDFT(M s A_{N-1} lam_N)
                    StepArgs b = a;
                    b.dpout = ctx->dP;
                    b.tw_a = ctx->tw.get(ctx->ny);
                    b.adj_first_prev = starts_setd2(n0 + i);
                    CKA(launch_second(ctx, b, MODE_ADJ_PRIME));
                    w_valid = true;
                }
                a.pin = slot;
                a.dpin = ctx->dP;
                a.dqout = ctx->dQ;
                if (grad2d) {
                    // KPZ: P_y of the step in, DFT_x(v_y) out through Q (free during the backward sweep)
                    a.pyin = trajy + (size_t)i * ctx->R * ctx->nmodes;
                    a.qout = ctx->Q;
                }
                a.tw_a = ctx->tw.get(ctx->nx / 2);
                a.tw_b = ctx->tw.get(ctx->nx);
                CKA(launch_rows(ctx, a, MODE_ADJ));
                a.dqin = ctx->dQ;
                a.qin = ctx->Q;
                a.dpout = ctx->dP;
                a.tw_a = ctx->tw.get(ctx->ny);
                CKA(launch_second(ctx, a, MODE_ADJ));
                ctx->launches += 2;
            }
        }
    }
    SKA(device_field_from_spectrum(ctx, ctx->dphi, grad_dev));
    // the primal ends at step0 + nsteps, as after nsteps of sft_step
    CKA(cudaMemcpyAsync(ctx->phi, phiN, ms, cudaMemcpyDeviceToDevice, ctx->stream));
    if (hist) CKA(cudaMemcpyAsync(ctx->fprev, phiN + cm / 2, ms, cudaMemcpyDeviceToDevice, ctx->stream));
    SKA(set_step_counter(ctx, step0 + nsteps));
    ctx->p_valid = false;
    ctx->dp_valid = false;
    s = read_status(ctx);
    release();
#undef CKA
#undef SKA
    return s;
}

sft_status sft_set_checkpoint_interval(sft_ctx* ctx, int segment) {
    if (!ctx || segment < 1) return SFT_EINVAL;
    ctx->ckpt_segment = segment;
    return SFT_OK;
}

// ------------------------------------------------------------ checkpoints
struct CkptHeader {
    char magic[8];
    uint64_t version;
    uint64_t cfg_hash;
    int64_t step;
    int64_t first_step;
    int64_t R;
    int64_t nmodes;
    int64_t has_fprev;
};

static uint64_t config_hash(const sft_config& c, uint64_t tables) {
    uint64_t h = 1469598103934665603ULL ^ tables;
    auto mix = [&](const void* p, size_t n) {
        const unsigned char* b = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ULL;
        }
    };
    mix(&c.d, sizeof c.d);
    mix(c.n, sizeof c.n);
    mix(c.dx, sizeof c.dx);
    mix(&c.replicas, sizeof c.replicas);
    mix(&c.model, sizeof c.model);
    mix(c.p, sizeof c.p);
    mix(&c.scheme, sizeof c.scheme);
    mix(&c.h, sizeof c.h);
    mix(&c.seed, sizeof c.seed);
    mix(&c.dealias, sizeof c.dealias);
    mix(&c.precision, sizeof c.precision);
    mix(&c.custom_nl, sizeof c.custom_nl);
    mix(&c.complex_field, sizeof c.complex_field);
    if (c.noise_space) mix(&c.noise_space, sizeof c.noise_space);
    return h;
}

sft_status sft_checkpoint(sft_ctx* ctx, void* host_buf, size_t cap, size_t* written) {
    if (!ctx) return SFT_EINVAL;
    if (ctx->is_batch) return fail(ctx, SFT_EUNSUPPORTED, "not available on a batch context; use its members' configurations individually");
    const size_t ms = (size_t)ctx->R * ctx->nmodes * sizeof(float2);
    const size_t need = sizeof(CkptHeader) + ms * (ctx->fprev ? 2 : 1);
    if (written) *written = need;
    if (!host_buf) return SFT_OK;
    if (cap < need) return fail(ctx, SFT_EINVAL, "checkpoint buffer too small");
    CkptHeader hd{};
    memcpy(hd.magic, "SFTCKPT1", 8);
    hd.version = 1;
    hd.cfg_hash = config_hash(ctx->cfg, ctx->cust_hash);
    hd.step = ctx->step;
    hd.first_step = ctx->first_step;
    hd.R = ctx->R;
    hd.nmodes = ctx->nmodes;
    hd.has_fprev = ctx->fprev ? 1 : 0;
    char* b = (char*)host_buf;
    memcpy(b, &hd, sizeof hd);
    CK(cudaMemcpyAsync(b + sizeof hd, ctx->phi, ms, cudaMemcpyDeviceToHost, ctx->stream));
    if (ctx->fprev) CK(cudaMemcpyAsync(b + sizeof hd + ms, ctx->fprev, ms, cudaMemcpyDeviceToHost, ctx->stream));
    return read_status(ctx);
}

sft_status sft_restore(sft_ctx* ctx, const void* host_buf, size_t bytes) {
    if (!ctx || !host_buf) return SFT_EINVAL;
    if (ctx->is_batch) return fail(ctx, SFT_EUNSUPPORTED, "not available on a batch context; use its members' configurations individually");
    CkptHeader hd{};
    if (bytes < sizeof hd) return fail(ctx, SFT_ECHECKPOINT, "checkpoint truncated");
    memcpy(&hd, host_buf, sizeof hd);
    const size_t ms = (size_t)ctx->R * ctx->nmodes * sizeof(float2);
    if (memcmp(hd.magic, "SFTCKPT1", 8) != 0 || hd.version != 1) return fail(ctx, SFT_ECHECKPOINT, "not a checkpoint");
    if (hd.cfg_hash != config_hash(ctx->cfg, ctx->cust_hash) || hd.R != ctx->R || hd.nmodes != ctx->nmodes ||
        hd.has_fprev != (ctx->fprev ? 1 : 0))
        return fail(ctx, SFT_ECHECKPOINT, "checkpoint written for another configuration");
    if (bytes != sizeof hd + ms * (hd.has_fprev ? 2 : 1)) return fail(ctx, SFT_ECHECKPOINT, "checkpoint size mismatch");
    const char* b = (const char*)host_buf;
    CK(cudaMemcpyAsync(ctx->phi, b + sizeof hd, ms, cudaMemcpyHostToDevice, ctx->stream));
    if (ctx->fprev) CK(cudaMemcpyAsync(ctx->fprev, b + sizeof hd + ms, ms, cudaMemcpyHostToDevice, ctx->stream));
    ctx->step = hd.step;
    ctx->first_step = hd.first_step;
    long long vals[2] = {hd.step, hd.first_step};
    CK(cudaMemcpyAsync(ctx->dstep, vals, sizeof vals, cudaMemcpyHostToDevice, ctx->stream));
    ctx->p_valid = false;
    CK(cudaStreamSynchronize(ctx->stream));
    return SFT_OK;
}

// Per-kernel timing: nsteps steps launched one kernel at a time with CUDA
// events around every launch on the context stream; out_ms receives the mean
// duration of each kernel of the step in launch order (row pass, column pass;
// or the line kernel in 1-D) followed by the mean whole-step duration.
sft_status sft_profile(sft_ctx* ctx, int64_t nsteps, double* out_ms, int cap, int* nkernels) {
    if (!ctx || !out_ms || nsteps < 1) return SFT_EINVAL;
    if (ctx->is_batch) {
        // out: [persistent 1-D kernel, the other members' kernels, step]
        if (cap < 3) return fail(ctx, SFT_EINVAL, "output too small");
        if (!ctx->p_valid) {
            sft_status s = prime(ctx);
            if (s != SFT_OK) return s;
        }
        cudaEvent_t e0, e1, e2;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        CK(cudaEventCreate(&e2));
        double t1 = 0, t2 = 0;
        for (int64_t i = 0; i < nsteps; ++i) {
            CK(cudaEventRecord(e0, ctx->stream));
            if (ctx->nitems > 0) {
                CK(cudaMemsetAsync(ctx->d_head, 0, sizeof(int), ctx->stream));
                CK(launch_k1_batch(ctx->d_members, ctx->d_items, ctx->nitems, ctx->d_head, ctx->nl, 0,
                                   ctx->batch_blocks, ctx->stream));
            }
            CK(cudaEventRecord(e1, ctx->stream));
            for (int m : ctx->solo) {
                sft_status s = enqueue_step(ctx->members[m], 0);
                if (s != SFT_OK) return fail(ctx, s, ctx->members[m]->err);
            }
            CK(cudaEventRecord(e2, ctx->stream));
            CK(advance_all(ctx, 1));
            ctx->launches += ctx->launches_per_step + advances_per_chunk(ctx);
            CK(cudaEventSynchronize(e2));
            float a = 0, b = 0;
            CK(cudaEventElapsedTime(&a, e0, e1));
            CK(cudaEventElapsedTime(&b, e1, e2));
            t1 += a;
            t2 += b;
        }
        ctx->step += nsteps;
        for (sft_ctx* m : ctx->members) m->step += nsteps;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaEventDestroy(e2);
        out_ms[0] = t1 / nsteps;
        out_ms[1] = t2 / nsteps;
        out_ms[2] = (t1 + t2) / nsteps;
        if (nkernels) *nkernels = 2;
        return read_status(ctx);
    }
    const int nk = ctx->d == 1 ? 1 : 2;
    if (cap < nk + 1) return fail(ctx, SFT_EINVAL, "output too small");
    if (!ctx->p_valid) {
        sft_status s = prime(ctx);
        if (s != SFT_OK) return s;
    }
    std::vector<cudaEvent_t> ev((size_t)nsteps * (nk + 1));
    for (auto& e : ev) CK(cudaEventCreate(&e));
    for (int64_t i = 0; i < nsteps; ++i) {
        cudaEvent_t* e = &ev[(size_t)i * (nk + 1)];
        StepArgs a = base_args(ctx);
        CK(cudaEventRecord(e[0], ctx->stream));
        if (ctx->d == 1) {
            if (!set_line_twiddles(ctx, a)) return fail(ctx, SFT_EINVAL, "twiddle table missing");
            CK(launch_k1_line(a, line_step_mode(ctx, a), ctx->nl, ctx->stream));
            CK(cudaEventRecord(e[1], ctx->stream));
        } else if (ctx->cfg.precision == 1) {
            // precision study: the whole tensor-core step, reported as the first entry (the second is empty)
            CK(launch_tc_step(a, ctx->tcb1, ctx->tcb2, ctx->tw.get(ctx->nx), ctx->stream));
            CK(cudaEventRecord(e[1], ctx->stream));
            CK(cudaEventRecord(e[2], ctx->stream));
        } else {
            sft_status s = enqueue_front(ctx, a, 0);
            if (s != SFT_OK) return s;
            CK(cudaEventRecord(e[1], ctx->stream));
            CK(launch_cols_step(ctx, a));
            CK(cudaEventRecord(e[2], ctx->stream));
        }
        CK(launch_advance(ctx->dstep, 1, ctx->stream));
        ctx->launches += ctx->launches_per_step + 1;  // the step's kernels (with any noise transform) + advance
    }
    ctx->step += nsteps;
    CK(cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k <= nk; ++k) out_ms[k] = 0.0;
    for (int64_t i = 0; i < nsteps; ++i) {
        cudaEvent_t* e = &ev[(size_t)i * (nk + 1)];
        for (int k = 0; k < nk; ++k) {
            float ms = 0.f;
            CK(cudaEventElapsedTime(&ms, e[k], e[k + 1]));
            out_ms[k] += ms / nsteps;
            out_ms[nk] += ms / nsteps;
        }
    }
    for (auto& e : ev) cudaEventDestroy(e);
    if (nkernels) *nkernels = nk;
    return read_status(ctx);
}

sft_status sft_draw_noise(sft_ctx* ctx, int64_t step, void* host_out, size_t bytes) {
    if (!ctx || !host_out || step < 0) return SFT_EINVAL;
    if (ctx->is_batch) return fail(ctx, SFT_EUNSUPPORTED, "not available on a batch context; use its members' configurations individually");
    const size_t ms = (size_t)ctx->R * ctx->nmodes * sizeof(float2);
    if (bytes != ms) return fail(ctx, SFT_EINVAL, "noise buffer size mismatch");
    CK(launch_draw_noise(ctx->nx, ctx->ny, ctx->nz, ctx->hx, ctx->cplx, ctx->R, ctx->rep0, ctx->cfg.seed, step,
                         ctx->Q, ctx->stream));
    CK(cudaMemcpyAsync(host_out, ctx->Q, ms, cudaMemcpyDeviceToHost, ctx->stream));
    return read_status(ctx);
}

sft_status sft_get_step(const sft_ctx* ctx, int64_t* step) {
    if (!ctx || !step) return SFT_EINVAL;
    *step = ctx->step;
    return SFT_OK;
}

sft_status sft_launches_per_step(const sft_ctx* ctx, int* launches) {
    if (!ctx || !launches) return SFT_EINVAL;
    *launches = ctx->launches_per_step;
    return SFT_OK;
}

sft_status sft_kernel_launches(const sft_ctx* ctx, int64_t* count) {
    if (!ctx || !count) return SFT_EINVAL;
    *count = ctx->launches;
    return SFT_OK;
}

const char* sft_last_error(const sft_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

void sft_destroy(sft_ctx* ctx) {
    if (!ctx) return;
    if (ctx->graph) cudaGraphExecDestroy(ctx->graph);
    for (sft_ctx* m : ctx->members) sft_destroy(m);
    if (ctx->d_members) cudaFree(ctx->d_members);
    if (ctx->d_items) cudaFree(ctx->d_items);
    if (ctx->d_head) cudaFree(ctx->d_head);
    if (ctx->rec_phi) cudaFree(ctx->rec_phi);
    if (ctx->rec_F) cudaFree(ctx->rec_F);
    for (cudaStream_t st : ctx->sides) cudaStreamDestroy(st);
    for (cudaEvent_t ev : ctx->ev_joins) cudaEventDestroy(ev);
    if (ctx->ev_fork) cudaEventDestroy(ctx->ev_fork);
    void* bufs[] = {ctx->phi,   ctx->fprev,  ctx->P,      ctx->Q,      ctx->Py,     ctx->snap, ctx->real,
                    ctx->cfield, ctx->tab,   ctx->dstep,  ctx->dstatus, ctx->dshell, ctx->drough, ctx->tw.dev,
                    ctx->dphi,  ctx->dseed, ctx->dP,     ctx->dQ,      ctx->noise_spec, ctx->tw32, ctx->dfprev, ctx->dmu, ctx->dPy, ctx->tcb1, ctx->tcb2,
                    ctx->d_order, ctx->d_chunks, ctx->d_first_chunk, ctx->d_part, ctx->d_tacc};
    for (void* p : bufs)
        if (p) cudaFree(p);
    if (ctx->own_stream && ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

}  // extern "C"
