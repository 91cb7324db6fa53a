/*
 * sft.h -- C ABI of the GB300 stochastic-field stepper.
 *
 * The library advances R independent replicas of a real or complex field on a
 * periodic d-dimensional lattice (d = 1, 2, 3) by the pseudo-spectral
 * stochastic exponential-time-differencing (SETD) schemes of Johnsrud & Rana,
 * "Efficient Pseudo-spectral Algorithms for Statistical Field Theories"
 * (arXiv 2511.22510).  In Fourier space every mode obeys (Sec. IV, eq.
 * general_fourier)
 *
 *     d phi_a / dt = c_a phi_a + F_a[phi] + sqrt(2 D_a) eta_a(t),
 *
 * with a diagonal linear operator c_a, a nonlinearity F evaluated in real
 * space and dealiased (2/3 truncation), and additive noise.  One step is the
 * boxed algorithm of Sec. IV: inverse transform of the masked state, the
 * real-space nonlinearity, forward transform, and the diagonal update
 *
 *     phi_a <- f1_a phi_a + A_a F_a + B_a F_a(t-h) + g_a eta_a
 *
 * with the coefficients of SETD-EM (Sec. II, Eq. SETD-EM), SETD1 (Eq. SETD1)
 * or SETD2 (Eq. SETD2), and Philox4x32-10 Gaussian noise drawn directly in
 * Fourier space with the Hermitian structure of App. B.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an sft_status; nothing aborts and no C++
 *    exception crosses the ABI.  sft_last_error() gives a message.
 *  - Lattice axis 0 is x, the fastest-varying real-space axis.  A real-space
 *    field of one replica is a row-major array [n2][n1][n0] (x fastest) of
 *    float (real fields) or interleaved float pairs (complex fields); R
 *    replicas are stored one after another.
 *  - The state lives on the device in Fourier space.  Its internal layout is
 *    "x-major": mode (a_x, a_z, a_y) of replica r sits at
 *        ((r * HX + a_x) * n2 + a_z) * n1 + a_y
 *    with HX = n0/2 + 1 stored x-modes for real fields (Hermitian half) and
 *    HX = n0 for complex fields; indices are the unsigned FFT indices
 *    0 .. n-1.  sft_get_spectrum returns exactly this layout.
 *  - The caller owns every host and device buffer it passes; the library
 *    copies what it needs and retains no caller pointer after returning.
 *  - A context owns all of its device memory and is not thread-safe.
 *  - Work is enqueued on cfg.stream (NULL = the legacy default stream).
 *    sft_step returns after enqueueing; calls that return data to the host
 *    synchronise the stream first and then report any device-side status.
 */
#ifndef SFT_H
#define SFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sft_ctx sft_ctx;

typedef enum {
    SFT_OK = 0,
    SFT_EINVAL = 1,        /* invalid argument or configuration */
    SFT_ENOMEM = 2,        /* device or host allocation failed */
    SFT_ECUDA = 3,         /* a CUDA runtime call failed */
    SFT_ENONFINITE = 4,    /* a non-finite value appeared in the state */
    SFT_ETIMEOUT = 5,      /* a bounded device-side wait expired */
    SFT_EUNSUPPORTED = 6,  /* valid request that this build does not implement */
    SFT_ECHECKPOINT = 7    /* checkpoint buffer malformed or for another config */
} sft_status;

/* Built-in models (Sec. V).  Parameters p[] per model:
 *   SFT_MODEL_A: p = {Gamma, r, u, T}:  c = -Gamma (r + k^2), D_a = Gamma T,
 *                F = -Gamma u DFT[psi^3]                        (Sec. V.A, Delta = 0)
 *   SFT_MODEL_B: p = {Gamma, r, u, T}:  c = -Gamma k^2 (r + k^2), D_a = Gamma T k^2,
 *                F = -Gamma u k^2 DFT[psi^3]                    (Sec. V.A, Delta = 2)
 *   Model A/B with p[4] != 0: the r phi term is placed in F instead of c (the
 *                variant of the Sec. V.A footnote, c = -Gamma k^Delta k^2 never
 *                changes sign): F = -Gamma k^Delta (r phi + u DFT[psi^3]);
 *                SETD-EM and SETD1 only (SFT_EUNSUPPORTED with SETD2).
 *   SFT_KPZ:     p = {nu, lambda, D}:   c = -nu k^2, D_a = D,
 *                F = (lambda/2) DFT[|grad h|^2]                 (Sec. V.B, noise sqrt(2D) eta)
 *   SFT_CGL:     p = {alpha, beta, eps}: complex field, c = 1 - (1 + i alpha) k^2,
 *                D_a = eps, F = -(1 + i beta) DFT[|A|^2 A]       (Sec. V.C with b = alpha,
 *                c = beta, D = eps)
 *   SFT_CUSTOM:  the general Fourier-space form of Sec. IV,
 *                d phi_a/dt = c_a phi_a + F_a + sqrt(2 D_a) eta_a,  F = s_a DFT[q(psi)],
 *                with c, D and s given as tables over |a|^2 and q one of sft_nonlinearity
 *                (see the SFT_CUSTOM fields of sft_config).
 * psi, grad h and A are the inverse transforms of the dealiased state. */
typedef enum { SFT_MODEL_A = 0, SFT_MODEL_B = 1, SFT_KPZ = 2, SFT_CGL = 3, SFT_CUSTOM = 4 } sft_model;

/* Real-space nonlinearity q of SFT_CUSTOM: none; psi^3 (real field); sum_j (d_j psi)^2
 * with the spectral gradient (real field); |A|^2 A (complex field). */
typedef enum { SFT_NL_NONE = 0, SFT_NL_CUBIC = 1, SFT_NL_GRAD2 = 2, SFT_NL_CGL = 3 } sft_nonlinearity;

/* Schemes of Sec. II: SETD-EM (Eq. SETD-EM), SETD1 (Eq. SETD1), SETD2 (Eq. SETD2). */
typedef enum { SFT_SETD_EM = 0, SFT_SETD1 = 1, SFT_SETD2 = 2 } sft_scheme;

typedef struct {
    int d;             /* 1, 2 or 3 */
    int n[3];          /* points per axis (x first), all equal (isotropic): powers of two, or, for
                        * 1-D and 2-D real fields (Model A/B, KPZ) with Fourier-space noise and truncation
                        * (or none), p x 2^k with p in {3, 5, 7} and 16p <= n <= 768 (a radix-p
                        * pass ahead of the radix-4/2 passes; no tangent/adjoint, dynamic recording
                        * or batches) */
    double dx[3];      /* lattice spacing per axis; all equal */
    int replicas;      /* R >= 1 independent noise realisations */
    sft_model model;
    double p[8];       /* model parameters, see sft_model */
    sft_scheme scheme;
    double h;          /* time step, > 0 */
    uint64_t seed;     /* Philox key */
    int dealias;       /* 1: 2/3-rule truncation (3|a_i| < n_i), 0: none, 2: phase-shift
                        * dealiasing (Sec. IV step 1): the nonlinear term is the mean over the
                        * 2^d grids shifted by half a cell along every subset of the axes, every
                        * mode but the Nyquist ones kept (alias-free for the cubic and the gradient-
                        * squared terms); built for 2-D real fields and power-of-two 1-D real lines of up
                        * to 16384 points (Model A/B, KPZ), 3-D real fields up to 64^3 (cubic term) and
                        * 2-D complex fields (CGL), with noise_space 0, at two (2-D) or four (3-D) times the P/Q memory and two to
                        * four times the transform work of a step */
    int precision;     /* 0: FP32 state and transforms; 1: the split-BF16x3 tensor-core transforms of
                        * the precision study (complex 2-D fields of 1024^2 or 2048^2 points) */
    void* stream;      /* cudaStream_t, or NULL for the default stream */
    int replica0;      /* global index of replica 0 (Philox counter word 2): ranks that shard one
                          ensemble pass disjoint offsets; 0 for a stand-alone context */
    /* SFT_CUSTOM only (ignored otherwise).  Host tables indexed by q = |a|^2 = sum_i a_i^2,
     * q = 0 .. sum_i (n_i/2)^2, copied by sft_create (the caller keeps ownership):
     * c_re/c_im the linear operator c_a (c_im NULL: real), noise_D the noise strength
     * D_a >= 0, nl_re/nl_im the nonlinear prefactor s_a (NULL: zero).  A real field needs
     * real c and s (Hermitian symmetry); complex_field = 1 takes SFT_NL_CGL or SFT_NL_NONE,
     * a real field SFT_NL_NONE, SFT_NL_CUBIC or SFT_NL_GRAD2 (3-D: NONE or CUBIC).
     * SFT_EINVAL for a missing c_re / noise_D, a negative D or a complex table on a real
     * field. */
    int custom_nl;         /* sft_nonlinearity */
    int complex_field;
    const double* c_re;
    const double* c_im;
    const double* noise_D;
    const double* nl_re;
    const double* nl_im;
    /* Noise (Sec. IV step 2): 0 draws eta_a in Fourier space with the Hermitian
     * structure of App. B; 1 draws iid N(0,1) per real-space site (Philox
     * ctr = (site >> 2, step, replica, 3), normal site & 3) and takes
     * eta_a = DFT[eta]_a / sqrt(N^d): one extra forward transform per step.
     * 1 is built for 2-D and 3-D real fields and power-of-two 1-D real lines
     * of up to 16384 points (cubic or gradient-squared term). */
    int noise_space;
} sft_config;

/* Observables for sft_observe (App. C; shells j = ceil(|a|), i.e. the shell
 * (k_j - dk, k_j] with dk = 2 pi / L). */
typedef enum {
    SFT_OBS_SK = 0,          /* C_ET shell average (L/N^2)^d <|phi_a|^2>, replica-averaged:
                                writes nshells values, then nshells mode counts N_k if cap allows */
    SFT_OBS_SK_REPLICAS = 1, /* same per replica: R * nshells values */
    SFT_OBS_MARK = 2,        /* store phi(t0) for SFT_OBS_CKT; writes nothing */
    SFT_OBS_CKT = 3,         /* two-time shell average (L/N^2)^d Re<phi_a(t) conj(phi_a(t0))> */
    SFT_OBS_ROUGHNESS = 4,   /* per replica w^2 = N^{-2d} sum_{a != 0} |phi_a|^2 (Sec. V.B, box = L) */
    SFT_OBS_RESPONSE = 5,    /* per shell sum Re(dphi_a(t) conj(dphi_a(t0))) / sum |dphi_a(t0)|^2 over
                                replicas, dphi the tangent seeded at t0 by sft_tangent_step */
    SFT_OBS_NSHELLS = 6,     /* writes one value: the number of shells */
    SFT_OBS_SK_ACCUM = 7,    /* adds the current S(k) of every replica to a device time accumulator
                                (compensated FP64 pairs); writes nothing, does not synchronise */
    SFT_OBS_SK_TIME_MEAN = 8,/* nshells values: the time and replica mean of S(k) over the accumulated
                                observations, then their count; synchronises */
    SFT_OBS_SK_RESET = 9     /* clears the time accumulator; writes nothing */
} sft_observable;
/* Every shell sum is taken in a fixed order (the modes enumerated shell by
 * shell), so repeated evaluations of the same state give the same bits: runs
 * of at most 32 modes in single-precision pairs built from error-free
 * transformations (exact products by fused multiply-add, two-sum), the runs
 * combined with compensated FP64 summation. */

/* Create a context (allocates all device memory, builds the FP64 coefficient
 * tables of Sec. II on the device, zero state).  *out receives the context or
 * NULL on failure.  Errors: SFT_EINVAL (bad config), SFT_EUNSUPPORTED
 * (anisotropic lattice, sizes outside this build's transform plans),
 * SFT_ENOMEM, SFT_ECUDA. */
sft_status sft_create(const sft_config* cfg, sft_ctx** out);

/* Create one context that advances several configurations together (uneven
 * lattice sizes, the same model and scheme; custom members the same
 * nonlinearity and field type): each sft_step of the batch context advances
 * every member by one step inside one CUDA-graph launch.  Plain power-of-two
 * 1-D real lines share one persistent kernel (lines of up to 8192 points, and
 * 16384-point lines with at least twice as many replicas as SMs); every other
 * member (2-D, 3-D, complex, longer lines, p x 2^k points, real-space noise,
 * phase shifts) runs its own kernels on a parallel branch of the same graph.
 * Replica r of the batch is member m's replica r - offset(m).
 * SFT_EUNSUPPORTED for members of different models or schemes. */
sft_status sft_create_batch(const sft_config* cfgs, int count, sft_ctx** out);

/* Copy a host real-space field of ONE replica (bytes = n0*n1*n2*sizeof(float),
 * doubled for complex fields) into the state (forward transform, Hermitian
 * fix-up of App. B).  replica = -1 writes all replicas from R consecutive
 * fields.  Resets the SETD2 history.  Errors: SFT_EINVAL on size mismatch. */
sft_status sft_set_field(sft_ctx* ctx, int replica, const void* host_real_space, size_t bytes);

/* Initial condition drawn on the device: iid N(0, sigma^2) per site (complex:
 * sigma (N(0,1) + i N(0,1))), Philox counter (site/4 | site/2, 0, replica, 1). */
sft_status sft_init_random(sft_ctx* ctx, double sigma);

/* Inverse transform of one replica's state into a host buffer (replica = -1:
 * all replicas).  Synchronises the stream. */
sft_status sft_get_field(sft_ctx* ctx, int replica, void* host_out, size_t bytes);

/* Copy the device spectrum of all replicas (internal x-major layout, complex
 * float pairs) to a host buffer of bytes = R * HX * n1 * n2 * 8. */
sft_status sft_get_spectrum(sft_ctx* ctx, void* host_out, size_t bytes);
sft_status sft_set_spectrum(sft_ctx* ctx, const void* host_in, size_t bytes);

/* Advance every replica by nsteps SETD steps (Sec. IV boxed algorithm).
 * Enqueued on the context stream as CUDA-graph replays; returns without
 * waiting.  A non-finite state is reported by the next synchronising call
 * (sft_sync, sft_observe, sft_get_field) as SFT_ENONFINITE. */
sft_status sft_step(sft_ctx* ctx, int64_t nsteps);

/* One-time preparation of sft_step, without advancing or touching the state:
 * the schedule is chosen (as sft_get_plan) and the graph of a chunk of steps
 * is captured and instantiated.  sft_step otherwise does this on its first
 * call (running its first chunk as plain launches); calling sft_prepare first
 * keeps that set-up out of a timed region.  Synchronises.  No counterpart in
 * the paper. */
sft_status sft_prepare(sft_ctx* ctx);

/* Advance with the SAME kernels launched one by one from the host (no graph),
 * the plain unbatched form used for timing comparisons. */
sft_status sft_step_plain(sft_ctx* ctx, int64_t nsteps);

/* Schedule of the step's passes.  On the first step (or here, if no step has
 * run yet) a plan autotuner times every variant built for the lattice with
 * CUDA events on scratch copies of the state and keeps the fastest; the
 * choice is cached per configuration for the process (SFT_AUTOTUNE=0 in the
 * environment keeps the defaults; SFT_PLAN="row,col,rpb,pipe" fixes the
 * schedule).  out[0]: row-pass shape (0: 128-thread blocks at 4 per SM, 1:
 * 256-thread blocks at 2 per SM, 2: 512-thread blocks at 1 per SM; 3, rows of
 * 1024 points with the cubic term: two rows per warp as one complex 1024-point
 * transform in registers, tiles moved by TMA); out[1]: 2-D column
 * pass radix schedule and block shape (0: 8 values per thread, 256-thread
 * blocks, 3 per SM; 1: same, 4 per SM; 2: 16 values per thread, 128-thread
 * blocks, 4 per SM; 3, columns of 1024 points with the cubic term: one warp
 * per column, the column in registers through both transforms and the update;
 * columns shorter than 512 points have only 0); out[2]:
 * replicas per column-pass block; out[3]: 1 when the pipelined bulk-copy
 * column pass runs.  cap >= 4.  The schedule changes no result beyond
 * rounding order: every variant computes the same step.  Not on batch
 * contexts.  No counterpart in the paper (its code calls FFTW). */
sft_status sft_get_plan(sft_ctx* ctx, int* out, int cap);
/* Force a schedule (values as sft_get_plan, n >= 4); SFT_EINVAL for a
 * variant not built for the lattice.  Synchronises the context stream. */
sft_status sft_set_plan(sft_ctx* ctx, const int* plan, int n);

/* Wait for the context stream and report the device status word. */
sft_status sft_sync(sft_ctx* ctx);

/* Evaluate an observable (sft_observable) into host_out (cap doubles);
 * *written receives the number of doubles written.  Synchronises. */
sft_status sft_observe(sft_ctx* ctx, int kind, double* host_out, size_t cap, size_t* written);

/* Dynamic correlation C(k, omega) and noise-inferred susceptibility chi(k, omega)
 * (App. C), 2-D real fields.  sft_dyn_start arms a recording: at the steps
 * s0 + m every (s0 = the next step, m = 0 .. M-1) every mode of every replica
 * writes its state phi_a and its nonlinear force F_a (the F of that step) to
 * device buffers (2 R * n_modes * M complex floats, allocated here; step-major,
 * so the recording steps write coalesced).  After
 * M * every further steps sft_dyn_result transforms the series in time on the
 * GPU (the paper's convention phi_b = sum_m e^{+2 pi i b m / M} phi_m, omega_b =
 * 2 pi b / T, T = M every h, b signed with b = -M/2 .. M/2 - 1 at index
 * (b mod M)) and reduces over the replicas (the ensemble):
 *   C[a M + b]   = (L/N^2)^d T / M^2 <|phi_ab|^2>
 *   chi[a M + b] = (L/N^2)^d T / M^2 / (2 D_a) <phi_ab conj(-i omega_b phi_ab - K_ab)>,
 *                  K = c_a phi + F (the deterministic force),
 * a the stored mode (x-major half-spectrum order, n_modes = (n0/2 + 1) n1),
 * chi as (re, im) pairs, cap >= n_modes M; *dbar (if not NULL) receives the
 * average |2 Im chi - (omega / D) C| over the modes with D_a > 0 and all
 * frequencies (Eq. average-deviation).  The result ends the recording.
 * M: power of two in [16, 16384]; every >= 1.  Synchronises. */
sft_status sft_dyn_start(sft_ctx* ctx, int M, int every);
sft_status sft_dyn_result(sft_ctx* ctx, double* C_out, double* chi_out, size_t cap, double* dbar);

/* Width over boxes (Sec. V.B, the KPZ width w_ell): for every replica, the mean
 * over the boxes of ell^d sites that tile the lattice of the variance of the
 * real-space field in the box, w_ell^2 = < <h^2>_box - <h>_box^2 >_boxes (FP64
 * sums).  ell = n gives the global width of SFT_OBS_ROUGHNESS, ell = 1 gives 0.
 * ell must divide every n_i; host_out receives R doubles (cap >= R).  Real
 * fields, not on batch contexts.  Synchronises. */
sft_status sft_box_width(sft_ctx* ctx, int ell, double* host_out, size_t cap, size_t* written);

/* Linear response by forward-mode differentiation of the step (tangent map,
 * Sec. II schemes linearised; the response of Sec. V.A), advanced together
 * with the primal on the same noise path:
 *   dphi <- f1 dphi + A dF + B dF(t-h),  dF = M s DFT[q'(psi) IDFT(M dphi)],
 * with the tangent's own history dF(t-h) under SETD2 (zero at the seed).
 * dphi0_dev: DEVICE pointer to R real-space fields (layout as set_field) that
 * seed the tangent, or NULL to continue the current tangent.  dphi_out_dev:
 * DEVICE pointer receiving the R real-space tangent fields after nsteps, or
 * NULL.  Advances the primal by nsteps.  Built for the cubic term (d = 1..3),
 * the KPZ term (d = 1, 2) and the CGL term (d = 1, 2; rows up to 2048 points),
 * every scheme, power-of-two lattices, truncation or no dealiasing,
 * Fourier-space noise, 1-D lines up to 32768 points; otherwise
 * SFT_EUNSUPPORTED before any device work. */
sft_status sft_tangent_step(sft_ctx* ctx, const void* dphi0_dev, int64_t nsteps, void* dphi_out_dev);

/* Reverse-mode differentiation (the transpose of the tangent above): given a
 * cotangent lambda on the real-space fields after nsteps (DEVICE pointer, R
 * fields), writes into grad_out_dev (DEVICE, R fields) the gradient of
 * sum_x lambda(x) phi_{t+n}(x) (complex fields: Re sum_x conj(lambda(x))
 * phi_{t+n}(x)) with respect to phi_t(x), the real-space state at the call.
 * SETD2 is transposed with a history cotangent.  The primal is advanced by
 * nsteps; the backward sweep recomputes it from device checkpoints (state and
 * SETD2 history) taken every `segment` steps (sft_set_checkpoint_interval,
 * default 100), regenerating the noise from its Philox counters.  Same
 * coverage as sft_tangent_step; SFT_ENOMEM if the checkpoint buffers cannot be
 * allocated. */
sft_status sft_adjoint(sft_ctx* ctx, const void* cotangent_dev, int64_t nsteps, void* grad_out_dev);
sft_status sft_set_checkpoint_interval(sft_ctx* ctx, int segment);

/* Serialise the full state (spectrum, SETD2 history, step counter, seed and a
 * configuration hash) into a host buffer.  With host_buf = NULL only *written
 * (the required size) is set.  sft_restore accepts only a buffer written for
 * an identical configuration (SFT_ECHECKPOINT otherwise); resuming is
 * bit-identical to an uninterrupted run because the noise is a pure function
 * of (seed, step, replica, mode). */
sft_status sft_checkpoint(sft_ctx* ctx, void* host_buf, size_t cap, size_t* written);
sft_status sft_restore(sft_ctx* ctx, const void* host_buf, size_t bytes);

/* Diagnostics: the unit-variance Fourier noise eta_a (App. B structure) that
 * step `step` draws for every stored mode of every replica, written to a host
 * buffer in the spectrum layout (bytes = R * HX * n1 * n2 * 8).  The update
 * multiplies it by the amplitude g_a.  Synchronises. */
sft_status sft_draw_noise(sft_ctx* ctx, int64_t step, void* host_out, size_t bytes);

/* Tracing: advance nsteps steps launching one kernel at a time, with CUDA
 * events recorded on the context stream around every launch.  out_ms (cap >=
 * kernels per step + 1) receives the mean duration in milliseconds of each
 * kernel of the step in launch order (2-D: row pass, column pass; 1-D: the
 * line kernel) followed by the mean step duration; *nkernels the kernel count.
 * With real-space noise the first entry also holds the noise's forward
 * transform (the two kernels before the row pass).
 * The state advances exactly as with sft_step_plain.  Synchronises. */
sft_status sft_profile(sft_ctx* ctx, int64_t nsteps, double* out_ms, int cap, int* nkernels);

/* Current step counter (steps taken since creation or restore). */
sft_status sft_get_step(const sft_ctx* ctx, int64_t* step);

/* Number of kernel launches the context issues per step (for accounting). */
sft_status sft_launches_per_step(const sft_ctx* ctx, int* launches);

/* Total kernels this context has launched since creation (kernel nodes of
 * graph replays included). */
sft_status sft_kernel_launches(const sft_ctx* ctx, int64_t* count);

/* 0-d SDE ensembles (Sec. III): npaths independent paths of the Ito SDE
 * du = c u dt + F(u) dt + G(u) dW,
 *   SFT_SDE_SAO (Eq. sao), p = {Gamma, T, b}: c = -Gamma, F = -Gamma b u^3,
 *                G = sqrt(2 Gamma T) (additive noise);
 *   SFT_SDE_GBM (Eq. gbm), p = {lambda, mu, delta}: c = lambda - delta,
 *                F = delta u, G = mu u (multiplicative; delta = 0 makes the
 *                deterministic part of the SETD schemes exact),
 * advanced by the update rules of the stability table of Sec. III:
 *   EM u + (c u + F) h + G dW;  Milstein EM + G G' (dW^2 - h)/2;
 *   SETD-EM f1 u + f2 F + f3 G dW;  SETD-Milstein f1 u + f2 F + f3 G [dW + G' (dW^2 - h)/2];
 *   SETD1 f1 u + f2 F + f4 G dW/sqrt(h),
 * f1 = e^{ch}, f2 = (e^{ch} - 1)/c, f3 = e^{ch/2}, f4 = sqrt((e^{2ch} - 1)/(2c)).
 * Step n (counting from step0) of size h uses dW = sum_{i < substeps}
 * sqrt(h/substeps) z_p((step0 + n) substeps + i), z_p(m) the normal p & 3 of
 * Philox4x32-10(ctr = (p >> 2, m, 0, 2), key = seed): runs with different
 * substeps (h) on one seed follow one Wiener path (strong-convergence studies).
 *   u_dev: DEVICE array of npaths doubles, in/out.  w_dev: DEVICE array of
 *   npaths doubles accumulating W (the sum of the dW), or NULL.  Both owned by
 *   the caller.  stream: cudaStream_t or NULL.  FP64 state and coefficients.
 * Enqueues one kernel and returns (no synchronisation); SFT_EINVAL for an
 * unknown kind or scheme, h <= 0, substeps < 1, negative counts, a missing
 * u_dev or more than 2^32 fine increments; SFT_ECUDA if the launch fails. */
typedef enum { SFT_SDE_SAO = 0, SFT_SDE_GBM = 1 } sft_sde_kind;
typedef enum {
    SFT_SDE_EM = 0,
    SFT_SDE_MILSTEIN = 1,
    SFT_SDE_SETD_EM = 2,
    SFT_SDE_SETD_MILSTEIN = 3,
    SFT_SDE_SETD1 = 4
} sft_sde_scheme;
sft_status sft_sde0d(int kind, const double* p, int scheme, double h, int substeps, uint64_t seed, int64_t step0,
                     int64_t nsteps, int64_t npaths, void* u_dev, void* w_dev, void* stream);

/* No counterpart in the paper: an entry point for callers that cannot allocate
 * device memory (an embedding runtime that owns the allocator, a plug-in that
 * must not grow its footprint after start-up, a real-time loop where an
 * allocation could stall).  Advances nsteps SETD steps of a 2-D real field
 * (Model A, Model B or KPZ; n[0] == n[1] <= 512) without a context and without
 * calling cudaMalloc or cudaFree.
 *   cfg:       configuration as for sft_create (d = 2); cfg->stream is used.
 *   phi_dev:   DEVICE state, in/out, spectrum layout of sft_get_spectrum
 *              (R * (n0/2 + 1) * n1 complex float pairs), owned by the caller.
 *   fprev_dev: DEVICE SETD2 history of the same size (in/out), or NULL for
 *              SETD-EM and SETD1.
 *   history_valid: 1 if fprev_dev holds F of the step before step0 (a
 *              continued SETD2 run); 0 makes the first step use SETD1.
 *   step0:     index of the first step (the noise counter).
 * All other scratch -- intermediates, coefficient table, twiddles, counters --
 * lives in one fixed device array of about 7 MiB that every GPU loading this
 * library holds until exit; sizes beyond it (R * (n0/2 + 1) * n1 > 262144 modes,
 * or n > 512) return SFT_EINVAL.  The first call on a device looks that array
 * up and must come before any stream capture.  The address is kept for the
 * process: do not call this entry point after a cudaDeviceReset (or anything
 * else that destroys the device's primary context).  Calls share the array:
 * calls that overlap on the GPU race.  The configuration passes the checks of
 * sft_create first.  Synchronises cfg->stream; returns SFT_ENONFINITE if the
 * state became non-finite. */
sft_status sft_step2d_noalloc(const sft_config* cfg, void* phi_dev, void* fprev_dev, int history_valid,
                              int64_t step0, int64_t nsteps);

const char* sft_last_error(const sft_ctx* ctx);
void sft_destroy(sft_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* SFT_H */
