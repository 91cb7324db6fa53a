// sft_internal.h -- host/device parameter blocks and kernel launchers shared by
// the translation units of the stepper library (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sft {

enum Nonlinearity { NL_CUBIC = 0, NL_GRAD2 = 1, NL_CGL = 2, NL_NONE = 3 };
enum KernelMode {
    MODE_STEP = 0,
    MODE_FWD = 1,
    MODE_INV = 2,
    MODE_TAN = 3,
    MODE_ADJ = 4,
    MODE_PRIME = 5,
    MODE_ADJ_PRIME = 6,
    MODE_STEP_REC = 7,  // the step, also recording the state and the nonlinear force (dynamic observables)
    MODE_STEP_RSN = 8,  // the step with the noise read from a transformed real-space draw
    MODE_STEP_PS = 9,   // the step with phase-shift dealiasing (grids shifted by half a cell)
    MODE_FWD_NOISE = 10 // row pass: forward transform of the step's real-space noise, drawn in registers
};

// Everything a step kernel needs, passed by value.
struct StepArgs {
    // lattice (real-space points per axis; unused axes = 1)
    int nx, ny, nz;
    int hx;        // stored x modes: nx/2 + 1 (real field) or nx (complex field)
    int ncols;     // x columns carried by the P/Q intermediates in this launch
    int R;         // replicas in the launch
    int rep0;      // replica index of the first replica (noise counter word 2)
    float scale;   // 1 / (nx ny nz): folds the inverse-transform normalisation
    float dk;      // 2 pi / L
    int dealias;   // 1: 2/3 truncation
    int pshift;    // 1: phase-shift dealiasing (the kernels' mask keeps all but the Nyquist modes)
    const float2* tw_ps;  // e^{-i pi m / N}, m < 2N: half-cell shift phases (N = nx = ny)
    long long ps_off;     // phase shift: offset of the shifted copies P1, Q1 behind P0, Q0 (R x modes)
    int model;     // sft_model
    int scheme;    // sft_scheme
    float s0, s0i; // nonlinear prefactor: A: -Gamma u; B: -Gamma u (times k^2); KPZ: lambda/2; CGL: -(1 + i beta)
    uint64_t seed;
    uint32_t ks[20];    // Philox round keys of the seed: ks[2i], ks[2i + 1] = seed words + i Weyl constants
    const float4* tab;  // per |a|^2 coefficients {f1, A, B, g} (complex: 2 float4 per entry)
    // buffers (x-major layouts, replica-major)
    float2* phi;        // state
    float2* fprev;      // SETD2 history
    const float2* qin;  // row-pass output / column-pass input
    float2* pout;       // column-pass output / row-pass input
    float2* qout;
    const float2* pin;
    const float2* pyin; // KPZ: second intermediate (i k_y M phi)
    float2* pyout;
    float* real_io;     // real-space field (FWD input / INV output), real fields
    float2* cplx_io;    // complex real-space field, complex fields
    // tangent / adjoint streams
    float2* dphi;
    float2* dfprev;
    const float2* dqin;
    float2* dpout;
    float2* dqout;
    const float2* dpin;
    const float2* dpyin;
    float2* dpyout;
    // SETD2 adjoint (Eq. SETD2 transposed): the history cotangent mu (1-D lines keep it between steps) and
    // whether step n (adj_first_n) or step n - 1 (adj_first_prev) of the backward sweep is the step that
    // starts the SETD2 history (SETD1 pair: A + B and B = 0)
    float2* dmu;
    int adj_first_n, adj_first_prev;
    // twiddle tables for the transform lengths used by the kernel
    const float2* tw_a;  // table for the first transform length
    const float2* tw_b;  // table for the second transform length
    const float2* tw_c;  // 1-D lines of 65536 points: table of the 8192-point per-block FFT
    const float2* tw_32; // 1024-point warp transforms: tw_32[k1 32 + t] = W_1024^{t k1} (t, k1 < 32)
    // step bookkeeping
    const long long* step_base;  // device: step index of k_in_chunk = 0
    int k_in_chunk;
    const long long* first_step;  // SETD2: the step that uses SETD1 coefficients
    unsigned* status;             // bit 0: non-finite state
    long long* bad_step;
    int rpb;                      // 2-D column pass: replicas per block (< 1: the default)
    int wait_limit;               // iterations of a bounded device wait: 0 the default (2^22); < 0 none, so
                                  // the first wait of a launch times out (exercises the time-out path)
    // recording for the dynamic observables (2-D real fields): at steps rec_start + m rec_every,
    // m < rec_M, mode j (state layout index, replicas included) writes phi_j and F_j to
    // rec_*[m rec_n + j] (step-major, coalesced), rec_n = R n_modes
    float2* rec_phi;
    float2* rec_F;
    long long rec_start, rec_n;
    int rec_every, rec_M;
    const float2* noise_in;  // real-space noise: DFT of the draw (state layout); eta = noise_scale * noise_in
    float noise_scale;
};

// Round keys of Philox4x32-10 for a seed: the key, then bumped by the Weyl constants 0x9E3779B9 / 0xBB67AE85
// before each further round (StepArgs::ks).
inline void philox_key_schedule(uint64_t seed, uint32_t (&ks)[20]) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int i = 0; i < 10; ++i) {
        ks[2 * i] = k0;
        ks[2 * i + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// launchers (return cudaGetLastError of the launch); each picks the template
// instance for the lattice size and returns cudaErrorInvalidValue if none.
cudaError_t launch_k1_line(const StepArgs& a, int mode, int nl, cudaStream_t s);
cudaError_t launch_k1_cluster(const StepArgs& a, int mode, int nl, cudaStream_t s);
int k1_cluster_fft_len(int nx);            // per-block FFT length of the cluster kernel for lines of nx points (0: none)
bool k1_use_cluster(int nx, int R, int mode);  // whether a 1-D launch of R replicas takes the cluster kernel
// shape: schedule variant of the step mode (0 = default; see k2_row_shapes / k2_col_shapes)
cudaError_t launch_k2_rows(const StepArgs& a, int mode, int nl, cudaStream_t s, int shape = 0);
cudaError_t launch_k2_cols(const StepArgs& a, int mode, int nl, cudaStream_t s, int shape = 0);
int k2_row_shapes(int nx);  // schedule variants of the 2-D row pass for lattices of nx points
cudaError_t launch_k2_rows_mixed(const StepArgs& a, int mode, int nl, cudaStream_t s);  // p x 2^k rows
cudaError_t launch_k2_cols_mixed(const StepArgs& a, int mode, int nl, cudaStream_t s);  // p x 2^k columns
bool k2_mixed_size(int n);   // p x 2^k points, p in {3, 5, 7}, 16p .. 768: 2-D real fields, transforms and step only
int k2_col_shapes(int ny);  // schedule variants of the 2-D column pass for columns of ny points
cudaError_t launch_k2_cols_pipe(const StepArgs& a, int nl, cudaStream_t s);
// row pass of the step on rows of 1024 points, two rows per warp, TMA tiles (cubic term)
bool k2_pair_supported(int nx, int ny, int nl, int dealias);
cudaError_t launch_k2_rows_pair(const StepArgs& a, int nl, cudaStream_t s);
// column pass of the step on columns of 1024 points, one warp per column (cubic term)
bool k2_colwarp_supported(int nx, int ny, int nl, int dealias);
cudaError_t launch_k2_cols_warp(const StepArgs& a, int nl, cudaStream_t s);
// precision study (sft_config.precision = 1): complex 2-D step through split-BF16x3 tensor-core transforms
bool tc_supported(int nx, int ny);
cudaError_t launch_tc_step(const StepArgs& a, float2* b1, float2* b2, const float2* twN, cudaStream_t s);
cudaError_t launch_tc_fft(int n, int inverse, float2* data, long long nlines, const float2* twN, cudaStream_t s);
cudaError_t launch_k3_planes(const StepArgs& a, int mode, int nl, cudaStream_t s);
cudaError_t launch_k2c_rows(const StepArgs& a, int mode, cudaStream_t s);
cudaError_t launch_k2c_cols(const StepArgs& a, int mode, cudaStream_t s);
bool k2c_supported(int nx, int ny);
bool k3_supported(int nx, int ny, int nz, int complex_field);
bool k2_pipe_supported(int nx, int ny, int complex_field);
bool k1_supported(int nx, int complex_field);
bool k2_supported(int nx, int ny, int complex_field);

// batches of 1-D lattices of uneven sizes advanced by one persistent launch
struct BatchMember {
    StepArgs a;  // the member's arguments (step_base shared by the batch)
    int M;       // half length: the member's lattice has 2M points
};
struct BatchItem {
    int member;  // index into the member table
    int r0;      // first replica of the item
};
int batch_lines_per_item(int M);
cudaError_t launch_k1_batch(const BatchMember* members, const BatchItem* items, int nitems, int* head, int nl,
                            int k_in_chunk, int blocks, cudaStream_t s);

// coefficient tables (FP64 on the device, stored as float)
// Table layouts (entry index -> k^2 / dk^2):
//   d = 1: entry i = |a|            -> i^2
//   d = 2: entry i * (ny/2 + 1) + j,  i = |a_x|, j = |a_y|  -> i^2 + j^2
//   d = 3: entry q = |a|^2          -> q
struct TableArgs {
    int model, scheme, complex_field;
    int d, hy;  // hy = ny/2 + 1 (d = 2)
    double p[8];
    double h, dk, noise_norm;
    long long nq;
    float4* out;
    // SFT_CUSTOM: device copies of c_re, c_im, D, s_re, s_im over |a|^2 = 0 .. ncust-1 (consecutive blocks);
    // the prefactor s is folded into A and B
    const double* cust;
    long long ncust;
};
__host__ __device__ inline long long table_k2_index(int d, int hy, long long entry) {
    if (d == 1) return entry * entry;
    if (d == 2) {
        const long long i = entry / hy, j = entry % hy;
        return i * i + j * j;
    }
    return entry;
}
cudaError_t launch_build_table(const TableArgs& t, cudaStream_t s);
// tw[m] = e^{-2 pi i m / L} for m < L (every twiddle table of the step kernels)
cudaError_t launch_twiddles(float2* tw, int L, cudaStream_t s);
// tw[k1 32 + t] = W_1024^{t k1} for t, k1 < 32 (1024-point warp transforms)
cudaError_t launch_twiddles32(float2* tw, cudaStream_t s);

// initial condition (Philox tag 1) into a real-space buffer
cudaError_t launch_init_random(float* real_out, float2* cplx_out, long long sites, int R, int rep0, uint64_t seed,
                               float sigma, cudaStream_t s);
// unit-variance Fourier noise of one step for every stored mode (diagnostics)
cudaError_t launch_draw_noise(int nx, int ny, int nz, int hx, int cplx, int R, int rep0, uint64_t seed,
                              long long step, float2* out, cudaStream_t s);
// step counter advance (one thread)
cudaError_t launch_advance(long long* step_base, int by, cudaStream_t s);

// observables
struct ObsArgs {
    int nx, ny, nz, hx, R, complex_field, nshells;
    const float2* phi;
    const float2* ref;  // snapshot for two-time, tangent seed for response
    double norm;        // (L/N^2)^d
    int kind;           // 0: |phi|^2, 1: Re(phi conj(ref)), 2: |ref|^2 (response denominator)
    double* shell_sum;  // [R][nshells] out: norm times the weighted shell sums
    // the stored modes of one replica shell by shell (built once per lattice): order[] lists the
    // mode indices of shell 0, then shell 1, ...; chunks[c] = {shell, start, length, 0} cuts it into
    // runs of at most kObsChunkLen modes inside one shell; the chunks of shell j are
    // first_chunk[j] .. first_chunk[j + 1] - 1
    const int* order;
    const int4* chunks;
    const int* first_chunk;
    int nchunks;
    double2* part;      // [R][nchunks] scratch: compensated chunk sums (sum, correction)
};
constexpr int kObsChunkLen = 1024;
cudaError_t launch_observe(const ObsArgs& o, cudaStream_t s);
// acc[j] += sum_r shell_sum[r][j] (compensated pairs): the device time accumulator of S(k, t)
cudaError_t launch_obs_time_acc(const double* shell_sum, int R, int nshells, double2* acc, cudaStream_t s);
// per replica: sum over the boxes of ell^d sites of the height variance in the box (out zeroed by the caller)
cudaError_t launch_box_width(const float* real, int nx, int ny, int nz, int d, int ell, int R, double* out,
                             cudaStream_t s);
// dynamic observables: C_ab and chi_ab from the time transforms of the recorded series (see sft_dyn_result)
struct DynArgs {
    const float2* Phi;  // [R][nmodes][M] time transforms of phi (forward, e^{-i})
    const float2* Fw;   // same for the nonlinear force F
    const double* c;    // [nmodes] linear operator c_a (real fields)
    const double* D;    // [nmodes] noise strength D_a
    int R, M;
    long long nmodes;
    double T, norm;     // record duration, (L/N^2)^d T / M^2 / R
    double* C;          // [nmodes][M] out
    double2* chi;       // [nmodes][M] out
};
cudaError_t launch_dyn_reduce(const DynArgs& d, cudaStream_t s);
// out[c rows + r] = in[r cols + c] (complex, tiled through shared memory)
cudaError_t launch_transpose_c(const float2* in, float2* out, long long rows, long long cols, cudaStream_t s);
cudaError_t launch_shell_counts(int nx, int ny, int nz, int hx, int complex_field, int nshells, double* counts,
                                cudaStream_t s);

}  // namespace sft
