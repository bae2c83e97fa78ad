/*
 * mstep.h -- C ABI of the GB300 (sm_103a) library for the multi-step
 * reconstruction of radio-interferometric images (Wang, Prunet, Mignot,
 * Ferrari, "Multi-Step Reconstruction of Radio-Interferometric Images").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Every function returns an ms_status; nothing throws or exits across the
 *   ABI.  On failure, ms_last_error(plan) describes the cause (a string owned
 *   by the plan, valid until its next call).
 * - The CALLER owns all data buffers.  "dev" pointers are CUDA device memory
 *   on the plan's device (any allocator, e.g. PyTorch); "host" pointers are
 *   ordinary host memory.  The PLAN owns everything it derives: sorted
 *   visibility indices, kernel and deapodization tables, PSF spectra,
 *   filters, work lists, workspaces and cuFFT plans.
 * - Real arrays are float64 for MS_FP64 plans and float32 otherwise; complex
 *   visibilities are interleaved (re, im) pairs of the same type.  Images are
 *   N x N row-major; pixel (p, q) sits at l = (q - N/2) dl, m = (p - N/2) dl.
 *   Wavelet coefficients are M planes of N x N in Mallat layout (see
 *   ms_dictionary_synthesis).
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *   stream-ordered; results that come back to the host (ms_stats, counts)
 *   are complete when the call returns.  A plan is not thread-safe: use it
 *   from one host thread and one stream at a time.
 * - Device-side waits inside kernels are bounded; a wait that runs out
 *   returns MS_ERR_TIMEOUT.
 */
#ifndef MSTEP_H
#define MSTEP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MS_OK = 0,
  MS_ERR_ARG = 1,          /* invalid argument or unsupported size */
  MS_ERR_CUDA = 2,         /* CUDA / cuFFT error */
  MS_ERR_OOM = 3,          /* device allocation failed */
  MS_ERR_NUMERIC = 4,      /* NaN / Inf seen, or a degenerate problem */
  MS_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out */
  MS_ERR_NOT_CONVERGED = 6,
  MS_ERR_STATE = 7,        /* call out of order */
  MS_ERR_UNSUPPORTED = 8
} ms_status;

typedef enum { MS_FP64 = 0, MS_FP32 = 1, MS_FP32_KAHAN = 2 } ms_precision;

/* Minor-cycle dictionaries (App. A.1).  DAUBECHIES: W = [Psi_1 .. Psi_M],
 * the periodized orthonormal 2-D db1..dbM transforms (W W^H = M I, step size
 * 2 M max K^ in closed form, Sect. 3.4).  IUWT: W = T^H, T the isotropic
 * undecimated "a trous" B3-spline transform with J levels (J + 1 planes
 * [w_1 .. w_J, c_J], T^H T not a multiple of I), step size by power
 * iteration (Sect. 3.4): 100 iterations in FP64 reductions from a fixed
 * pseudo-random start, once per minor-cycle problem. */
typedef enum { MS_DICT_DAUBECHIES = 0, MS_DICT_IUWT = 1 } ms_dictionary;

/* The PSF operator H of the minor cycle (Sects. 3.2-3.4).  CIRCULAR: the
 * N x N circular convolution by the PSF, diagonal in the N x N DFT (K^ =
 * |H^|^2 ..., step size 2 M max K^, the closed form of Sect. 3.4).  LINEAR:
 * the linear convolution that A^H A / sum(w) is on images of the N x N
 * field, H x = P F2^-1(H2^ . F2(P^T x)) with P^T the zero padding to
 * 2N x 2N and H2^ the spectrum of the PSF of the same partition on a
 * 2N x 2N field with the same pixel size (computed once at plan creation,
 * from a temporary 2N plan).  H is then not circulant and 2 M max K^ holds
 * only as a bound (2 M max H2^2, or 2 M (max g_H^2 max H2^2 + max g_L^2),
 * since ||P H P^T|| <= max |H2^|, 2-5x above the constant on small
 * cases), so the step size is a power iteration as for the IUWT (100
 * iterations from the same fixed start, once per minor-cycle problem).  LINEAR
 * needs the Daubechies dictionary and N <= 8192 (MS_ERR_ARG otherwise). */
typedef enum { MS_CONV_CIRCULAR = 0, MS_CONV_LINEAR = 1 } ms_convolution;

/* Baseline partitions of Sect. 3.1: L = {r <= ell + delta} (short baselines),
 * H = {r >= ell - delta} (long baselines), ALL = every unflagged row. */
typedef enum { MS_PART_L = 0, MS_PART_H = 1, MS_PART_ALL = 2 } ms_part;

/* Minor-cycle problems: LOW = Eq. LowRes (Sect. 3.2) on V_L, FULL = Eq. FullRes
 * (Sect. 3.3) on V_H, SINGLE = the LowRes problem on all rows (Sect. 5).  The
 * interleaved pipeline (ms_reconstruct_interleaved) adds LOW_H = the LowRes
 * problem on V_H, and FULL_L = Eq. FullRes on V_L with the two sides of the
 * band exchanged: data term ||G'_L (i~ - H x)||^2, prior ||G'_H (l - x)||^2,
 * G'_L, G'_H Sect. 3.3's filters with sigma^2 and eta^2 exchanged (weight
 * 1/sigma^2 below ell - delta on the data, 1/eta^2 above ell + delta on the
 * prior image). */
typedef enum {
  MS_STEP_LOW = 0, MS_STEP_FULL = 1, MS_STEP_SINGLE = 2, MS_STEP_LOW_H = 3, MS_STEP_FULL_L = 4
} ms_step;

/* lambda rules: NORM2_2N is lambda_n = c ||i~_n||_2 2^n (Sect. 5, App. A.2);
 * MAX_FIXED is lambda = c max|i~_1|, held for all cycles of a step. */
typedef enum { MS_LAMBDA_NORM2_2N = 0, MS_LAMBDA_MAX_FIXED = 1 } ms_lambda_rule;

typedef struct ms_plan ms_plan;
typedef struct ms_unet ms_unet;   /* the learned warm start's network (below) */

typedef struct {
  const double* u;        /* host [nchan * nvis] baseline u, wavelengths        */
  const double* v;        /* host [nchan * nvis] baseline v, wavelengths        */
  const uint8_t* flags;   /* host [nchan * nvis], nonzero = flagged; may be NULL */
  int64_t nvis;           /* rows per channel, 1 .. 2^31-1                      */
  int32_t nchan;          /* channels, >= 1                                     */
  int32_t npix;           /* image side N: multiple of 16 and of 2^levels       */
  double pixel_size;      /* dl in radians                                      */
  double ell_px;          /* partition centre ell, pixel units of the N x N DFT */
  double delta_px;        /* partition half width delta (> 0)                   */
  int32_t kernel_width;   /* ES kernel support W in cells; 7                    */
  int32_t oversample;     /* grid oversampling; 2                               */
  double es_beta;         /* ES shape; <= 0 selects 2.30 * W                    */
  int32_t levels;         /* wavelet levels J, 1..8                             */
  int32_t n_bases;        /* dictionary size M, 1..8 (db1 .. dbM)               */
  int32_t precision;      /* ms_precision                                       */
  int32_t tile;           /* gridding tile side: 0 = default (16), or 16 / 32 */
  int32_t chunk;          /* visibilities per work item: 0 = automatic          */
  int32_t device;         /* CUDA device ordinal                                */
  int32_t dictionary;     /* ms_dictionary; MS_DICT_IUWT ignores n_bases        */
  int32_t convolution;    /* ms_convolution of the minor cycle's PSF operator    */
} ms_plan_desc;

typedef struct {
  int32_t iterations;     /* prox steps taken in the last minor cycle         */
  int32_t converged;      /* 1 if the relative-objective test stopped it      */
  int32_t major_cycles;   /* major cycles run by a reconstruct call           */
  int32_t total_iterations; /* prox steps over all minor cycles of the call   */
  double objective;       /* F at the returned coefficients (FP64)            */
  double lambda;          /* lambda of the last minor cycle                   */
  double theta;           /* Lipschitz constant used (2 M max K^)             */
  double sigma2;          /* sigma^2 used by step two (0 if none)             */
  double eta2;            /* eta^2 used by step two (0 if none)               */
  double elapsed_ms;      /* device time of the call (CUDA events)            */
  double grid_ms;         /* of which: gridding + degridding kernels          */
  double fft_ms;          /* of which: the Ng x Ng FFTs of the major cycles   */
  double minor_ms;        /* of which: minor cycles                           */
  int64_t gridded_vis;    /* visibilities passed through one degrid + grid pair,
                             summed over the residual images of the call      */
  const double* objective_trace; /* plan-owned host array: F(beta_0..beta_k) of
                             the last minor cycle, length iterations + 1;
                             valid until the plan's next call                 */
} ms_stats;

typedef struct {
  int32_t n_major;        /* major cycles per step (Sect. 5: 5)               */
  int32_t fista_iters;    /* FISTA iterations per minor cycle (Sect. 5: 100)  */
  double rel_tol;         /* stop when |F_k - F_k-1| <= rel_tol |F_k|; 0 = off */
  int32_t lambda_rule;    /* ms_lambda_rule                                   */
  double lambda_low;      /* c for step one (paper: 0.05)                     */
  double lambda_full;     /* c for step two (paper: 0.05)                     */
  double lambda_single;   /* c for the single-step method (paper: 0.01)       */
  double sigma2;          /* <= 0: estimate on i~_H1 (Sect. 4.3)              */
  double eta2;            /* <= 0: 1e-3 sigma^2 (Sect. 4.3)                   */
  ms_unet* warm_start;    /* NULL, or a network on the plan's device: step
                             two's first minor cycle then starts from
                             ms_warm_start_coefficients(net, i^_L, i~_H1)
                             instead of zero (ms_reconstruct_two_step only)   */
} ms_recon_opts;

/* ------------------------------------------------------------------ plan */

/* Builds a plan (Sect. 3.1 partition + the gridding set-up the paper leaves
 * open): classifies every row of every channel into L / H by
 * r = |uv| N dl against ell +- delta (closed intervals), computes each row's
 * ES footprint on the 2x oversampled grid (first cell floor(g - W/2) + 1,
 * g = u Ng dl), sorts each partition by grid tile with a stable radix sort (so
 * rows keep their original order inside a tile), splits tiles into work
 * items, builds the deapodization table, the Daubechies filters db1..dbM and
 * the cuFFT plans.  u, v, flags are copied; the caller may free them after
 * the call.  Errors: MS_ERR_ARG (sizes, W != 7, oversample != 2, N not a
 * multiple of 16 or 2^levels), MS_ERR_OOM, MS_ERR_CUDA. */
ms_status ms_plan_create(const ms_plan_desc* desc, ms_plan** out);
ms_status ms_plan_destroy(ms_plan* plan);
const char* ms_last_error(const ms_plan* plan);

/* Row counts of a partition (Sect. 3.1): out[0] = |V_L|, out[1] = |V_H|,
 * out[2] = |V_L n V_H|, out[3] = unflagged rows, for channel chan. */
ms_status ms_partition_counts(ms_plan* plan, int32_t chan, int64_t out[4]);

/* Gridding layout of a partition: out[0] = its work items, out[1] = cells
 * of one work item's scratch tile ((tile + 6)^2), out[2] = bytes per
 * scratch cell (8 for FP32, 16 for FP64 and the compensated FP32 form). */
ms_status ms_partition_layout(ms_plan* plan, int32_t part, int32_t chan, int64_t out[3]);

/* The rows of partition `part` in the plan's sorted (tile) order, copied to
 * host `rows` [count]; count = ms_partition_counts of that partition. */
ms_status ms_partition_rows(ms_plan* plan, int32_t part, int32_t chan, int32_t* rows);

/* ------------------------------------------------------ measurement operator */

/* Degridding, A x (Sect. 2): image -> visibilities of the rows of `part`.
 * image: dev N*N real.  vis_obs: dev complex [nvis] in original row order, or
 * NULL.  vis_out: dev complex [nvis]; only the partition's rows are written,
 * with vis_obs - A x (the residual visibilities) if vis_obs is given, else
 * A x.  A = G F Z D with the ES kernel (W = 7, 2x oversampling). */
ms_status ms_degrid(ms_plan* plan, int32_t part, int32_t chan, const void* image,
                    const void* vis_obs, void* vis_out, void* stream);

/* Gridding, A^H y / sum(w) (Sect. 2): the rows of `part` of vis (dev complex
 * [nvis], original order) -> dirty image dev N*N real, natural weights. */
ms_status ms_grid(ms_plan* plan, int32_t part, int32_t chan, const void* vis,
                  void* dirty, void* stream);

/* ms_grid with the gridding kernel's per-work-item tiles in a fixed 64 MiB
 * array that is part of the library's device image, so this call obtains no
 * device memory (no cudaMalloc / cudaFree, no allocating library).  It is
 * meant for callers that may not allocate while they run: a process whose
 * device memory is already held by another allocator, or a pipeline that
 * cannot take the device-wide synchronization an allocation or free implies.
 * The paper has no counterpart of this call; its result equals ms_grid's.
 * Arguments, layouts and ownership are those of ms_grid; the plan's own
 * buffers (created by ms_plan_create) are used as in ms_grid.
 * Scratch need: (work items of the partition) x (tile + 6)^2 cells x 8 bytes
 * (FP32) or 16 bytes (FP64, FP32 compensated); a larger need returns
 * MS_ERR_ARG with the sizes in ms_last_error, and nothing is launched.
 * Nothing in the array has to start at zero (each tile is written in full
 * before it is read).  The array is shared by every plan and stream of a
 * device: calls whose executions overlap on one device race on it, so the
 * caller orders them (one stream, or events).  The first call on a device
 * looks up the array's address (cudaGetSymbolAddress, which may load the
 * module); make that first call before beginning any stream capture. */
ms_status ms_grid_static_scratch(ms_plan* plan, int32_t part, int32_t chan, const void* vis,
                                 void* dirty, void* stream);

/* ----------------------------------------------------------- batched form */

/* Gridding of several (channel, partition) jobs at once: the work items of
 * all jobs go through one gridding launch and one fold launch, the grids
 * through one batched inverse FFT and one crop.  chans, parts, vis, dirty are
 * HOST arrays of njobs entries; vis[j] is a dev complex [nvis] array of
 * channel chans[j] in original row order, dirty[j] a dev N*N real image that
 * receives A^H y / sum(w) of the rows of parts[j] (as ms_grid would).  The
 * plan grows its batch workspaces (grids, tiles, rows) when a call needs more
 * than an earlier one; later calls of the same or smaller size allocate
 * nothing.  Errors: MS_ERR_ARG (a NULL array or entry, channel or partition
 * out of range), MS_ERR_OOM, MS_ERR_CUDA. */
ms_status ms_grid_batch(ms_plan* plan, int32_t njobs, const int32_t* chans,
                        const int32_t* parts, const void* const* vis, void* const* dirty,
                        void* stream);

/* Degridding of several jobs at once (one pad, one batched FFT, one
 * degridding launch over all jobs' work items): images[j] (dev N*N real) ->
 * vis_out[j] (dev complex [nvis], only the rows of parts[j] written) = A x,
 * or vis_obs[j] - A x when vis_obs is not NULL.  Host arrays as in
 * ms_grid_batch; vis_obs may be NULL as a whole. */
ms_status ms_degrid_batch(ms_plan* plan, int32_t njobs, const int32_t* chans,
                          const int32_t* parts, const void* const* images,
                          const void* const* vis_obs, void* const* vis_out, void* stream);

/* Batched minor cycles (the batched form's "one CUDA graph per minor
 * cycle"): njobs independent FISTA problems (Algorithm 1 on Eq. LowRes or
 * FullRes) of this plan's geometry run together, each pass kernel launched
 * once over all jobs (blockIdx.z = job) and 8 passes per graph launch, each
 * job stopping on its own (rel_tol, max_iters).  Job j: step steps[j] on
 * channel chans[j] (its partition's PSF), residual residuals[j] (dev N*N),
 * for FULL l_lows[j] (dev N*N), sigma2s[j], eta2s[j] (> 0); lambdas[j];
 * B_0 = 0.  models_out[j] (dev N*N) receives W beta of the job's last prox
 * output; stats[j] (may be NULL) its iteration count, objective, lambda,
 * theta and the batch's elapsed time; traces (host, may be NULL)
 * [njobs][max_iters + 1] receives F(beta_0..) of each job (entries past
 * stats[j].iterations + 1 unspecified).  All arrays are HOST arrays of njobs
 * entries.  The workspace (about 155 MB per job at N = 1024, FP32, M = 8)
 * grows on demand and is kept.  Needs N a power of two, the Daubechies
 * dictionary and the circular PSF operator (MS_ERR_UNSUPPORTED otherwise). */
ms_status ms_minor_cycle_batch(ms_plan* plan, int32_t njobs, const int32_t* steps,
                               const int32_t* chans, const void* const* residuals,
                               const void* const* l_lows, const double* lambdas,
                               const double* sigma2s, const double* eta2s, int32_t max_iters,
                               double rel_tol, void* const* models_out, ms_stats* stats,
                               double* traces, void* stream);

/* The method on several channels at once (the batched form): as
 * ms_reconstruct_two_step / ms_reconstruct_single_step for each channel
 * chans[j] with visibilities vis[j] (dev complex [nvis], original order),
 * with every major cycle's residual images through one batched degridding
 * and gridding pass over all jobs and every minor cycle through the batched
 * FISTA loop of ms_minor_cycle_batch.  low_out[j] / img_out[j]: dev N*N;
 * stats[j] (may be NULL): per job (elapsed_ms is the whole call's).
 * opts->warm_start must be NULL.  Same requirements as
 * ms_minor_cycle_batch. */
ms_status ms_reconstruct_two_step_batch(ms_plan* plan, int32_t njobs, const int32_t* chans,
                                        const void* const* vis, const ms_recon_opts* opts,
                                        void* const* low_out, void* const* img_out,
                                        ms_stats* stats, void* stream);
ms_status ms_reconstruct_single_step_batch(ms_plan* plan, int32_t njobs, const int32_t* chans,
                                           const void* const* vis, const ms_recon_opts* opts,
                                           void* const* img_out, ms_stats* stats,
                                           void* stream);

/* Autotuner of the gridding layout: builds a plan from *desc for every grid
 * tile side T in {16, 32} (dividing 2N) and work-item size in {512, 1024,
 * 2048, 4096, 8192} rows, times `reps` degrid + grid pairs of channel chan's
 * full row set on this GPU (CUDA events, after one untimed pair) and returns
 * the fastest tile and chunk (to be put into desc->tile, desc->chunk) and its
 * time per pair in ms.  desc is not modified. */
ms_status ms_plan_autotune(const ms_plan_desc* desc, int32_t chan, int32_t reps,
                           int32_t* best_tile, int32_t* best_chunk, double* best_ms);

/* Major-cycle residual image i~ = F^H G^H (v - G F x) / sum(w) (Sect. 2) for
 * the rows of `part`: degrid, subtract, grid, in one call.  model: dev N*N
 * real; vis_obs: dev complex [nvis] original order; out: dev N*N real. */
ms_status ms_residual_image(ms_plan* plan, int32_t part, int32_t chan,
                            const void* vis_obs, const void* model, void* out,
                            void* stream);

/* PSF of a partition: A^H A applied to a unit impulse at (N/2, N/2), divided
 * by sum(w) (peak ~1).  psf: dev N*N real. */
ms_status ms_psf(ms_plan* plan, int32_t part, int32_t chan, void* psf, void* stream);

/* ------------------------------------------------------------ dictionary */

/* W alpha = sum_m Psi_m alpha_m (Sect. 4.3, App. A.1): M periodized
 * orthonormal Daubechies (db1..dbM) syntheses with J levels.  alpha: dev
 * [M][N][N] Mallat layout (after a level on an n x n block: [0,n/2)^2
 * approximation, rows [0,n/2) x cols [n/2,n) low-y/high-x, rows [n/2,n) x
 * cols [0,n/2) high-y/low-x, [n/2,n)^2 high/high).  x: dev N*N. */
ms_status ms_dictionary_synthesis(ms_plan* plan, const void* alpha, void* x, void* stream);

/* W^H x = [Psi_1^H x, ..., Psi_M^H x].  x: dev N*N; alpha: dev [M][N][N]. */
ms_status ms_dictionary_analysis(ms_plan* plan, const void* x, void* alpha, void* stream);

/* ----------------------------------------------------------- minor cycle */

/* Noise variance estimate of Sect. 4.3: mean over all inside 5x5 windows of
 * the population variance of image (dev N*N).  Result to host *sigma2. */
ms_status ms_sigma2_hat(ms_plan* plan, const void* image, double* sigma2, void* stream);

/* Lipschitz constant of the gradient (Sect. 3.4) for a step of a partition:
 * *closed = the step size the minor cycle uses: the closed form 2 M max K^
 * (K^ = |H^|^2, or |g_H H^|^2 + |g_L|^2 for FULL with the given sigma2,
 * eta2), or, for the IUWT dictionary or the linear PSF operator, the
 * 100-iteration power estimate; and, if power_iters > 0, *power = 2 lambda_max
 * by a power iteration of that many steps through W (FP64 reductions, on the
 * plan's PSF operator).  Results to host. */
ms_status ms_lipschitz(ms_plan* plan, int32_t step, int32_t chan, double sigma2,
                       double eta2, int32_t power_iters, double* theta_closed,
                       double* theta_power, void* stream);

/* One minor cycle: FISTA (Algorithm 1) on Eq. LowRes (LOW, SINGLE) or
 * Eq. FullRes (FULL) with gradients Eq. GradL / Eq. GradH, step 1/theta with
 * theta = 2 M max K^ (Sect. 3.4), threshold lambda/theta.  residual: dev N*N
 * (i~_n); l_low: dev N*N (l_Ln), FULL only; sigma2, eta2: FULL only.
 * beta_inout: dev [M][N][N] start point (NULL = zero) and, if not NULL, the
 * result.  model_out: dev N*N, receives W beta.  Runs exactly max_iters prox
 * steps unless rel_tol > 0 and |F_k - F_k-1| <= rel_tol |F_k| first.  The
 * objective F is evaluated in FP64 at every prox output. */
ms_status ms_minor_cycle(ms_plan* plan, int32_t step, int32_t chan,
                         const void* residual, const void* l_low, double sigma2,
                         double eta2, double lambda, int32_t max_iters,
                         double rel_tol, void* beta_inout, void* model_out,
                         ms_stats* stats, void* stream);

/* Objective target of the plan's later minor cycles (ms_minor_cycle and
 * the reconstruct calls), for time-to-tolerance comparisons of the forms:
 * with a finite target, a minor cycle also stops (stats->converged = 1) at
 * the first k with F(beta_k) <= target (Algorithm 1's objective, evaluated
 * in FP64 as for the relative-change test).  target = -inf turns it off
 * (the default); NaN is MS_ERR_ARG. */
ms_status ms_set_objective_target(ms_plan* plan, double target);

/* ----------------------------------------------------------- reconstruct */

/* The two-step method: step one (Eq. LowRes) on V_L for n_major cycles, final
 * low-resolution image i^_L = i~_{L,N+1} + sum i_Ln; then step two (Eq.
 * FullRes) on V_H with l_Ln = i^_L - sum_{j<n} i_j, final image
 * i^ = i~_{H,N+1} + sum i_n.  vis: dev complex [nvis] original order.
 * img_low_out, img_out: dev N*N; model_out (optional) receives sum i_n. */
ms_status ms_reconstruct_two_step(ms_plan* plan, int32_t chan, const void* vis,
                                  const ms_recon_opts* opts, void* img_low_out,
                                  void* img_out, void* model_out, ms_stats* stats,
                                  void* stream);

/* The interleaved two-image pipeline (Sect. 6, Fig. InterleavedMultiStepPipeline),
 * in this reading: node L (V_L) and node H (V_H) each keep a model; in major
 * cycle 1 each solves Eq. LowRes on its residual (LOW, LOW_H); from cycle 2
 * node H solves Eq. FullRes with l = model_L - model_H (FULL) and node L the
 * mirrored problem with l = model_H - model_L (FULL_L), both on the models
 * of the previous cycle, so the two minor cycles of a major cycle run as one
 * batched launch (the pipeline's parallelism on one GPU).  sigma^2 of each
 * node: Sect. 4.3's estimate on its first residual, eta^2 = 1e-3 sigma^2
 * (opts->sigma2 / eta2 are not used); lambda_n = c ||i~_n||_2 2^n with c =
 * lambda_low (node L), lambda_full (node H).  Node images: last residual +
 * model (node_l_out, node_h_out, dev N*N, may be NULL); the combined image
 * (img_out, dev N*N) takes eta_H^2 g_L^2 of node L's image and sigma_H^2
 * g_H^2 of node H's in the Fourier domain (weights that sum to one; g_L, g_H
 * node H's filters).  stats: NULL or [2] (node L, node H).  Requirements of
 * ms_minor_cycle_batch; opts->warm_start must be NULL. */
ms_status ms_reconstruct_interleaved(ms_plan* plan, int32_t chan, const void* vis,
                                     const ms_recon_opts* opts, void* img_out,
                                     void* node_l_out, void* node_h_out, ms_stats* stats,
                                     void* stream);

/* One step of the method on its own, n_major major cycles: LOW (Eq. LowRes
 * on V_L), FULL (Eq. FullRes on V_H, l_n = low_image - sum_{j<n} i_j, the
 * filters at the plan's ell, delta) or SINGLE; the step's image (last
 * residual + model) to img_out (dev N*N), the model to model_out (optional).
 * The method with K > 2 bands (Sect. 6's "more than 2-steps"; bands V_1 =
 * {r <= ell_1 + delta}, V_k = {ell_k-1 - delta <= r <= ell_k + delta}, V_K =
 * {r >= ell_K-1 - delta}) runs LOW on a plan with ell_1 and FULL on, for each
 * later band k, a plan with ell_k-1 whose flags drop the rows above
 * ell_k + delta, each FULL step taking the previous step's image. */
ms_status ms_reconstruct_step(ms_plan* plan, int32_t step, int32_t chan, const void* vis,
                              const ms_recon_opts* opts, const void* low_image, void* img_out,
                              void* model_out, ms_stats* stats, void* stream);

/* The single-step baseline (Sect. 5): step one's problem on V_L u V_H. */
ms_status ms_reconstruct_single_step(ms_plan* plan, int32_t chan, const void* vis,
                                     const ms_recon_opts* opts, void* img_out,
                                     void* model_out, ms_stats* stats, void* stream);

/* --------------------------------------------------- learned warm start */
/* A small U-Net maps [step-one image i^_L, long-baseline dirty image i~_H1]
 * to a starting image x0 for step two (Sect. 3.3); its coefficients
 * W^H x0 / M are passed to ms_minor_cycle as beta_inout, so FISTA still runs
 * to its own tolerance and the network only moves the starting point.  The
 * paper has no network; this is the learned warm-start form.
 * Architecture (levels L, base width C): per encoder level two 3x3 conv +
 * ReLU (C 2^l channels) then 2x2 average pooling; bottom level two conv +
 * ReLU; per decoder level nearest 2x upsampling, concatenation with the
 * encoder's skip, two conv + ReLU; a 3x3 conv head to one channel plus the
 * input's first channel.  Weights and activations bfloat16, products on the
 * tensor cores with FP32 accumulation, FP32 master weights and Adam state.
 * Images are FP32 device arrays, channels last: in [H][W][2], out / target
 * [H][W]; H and W must be multiples of 4 * 2^(L-1) and at most max_side.
 * Parameters (host FP32, conv after conv in execution order): weights
 * [c_out][3][3][c_in] then biases [c_out].  ms_unet_create draws He-normal
 * weights from `seed` and zero biases, and starts the head at zero, so an
 * untrained network returns the step-one image. */
ms_status ms_unet_create(int32_t levels, int32_t width, int32_t max_side, uint64_t seed,
                         int32_t device, ms_unet** out);
ms_status ms_unet_destroy(ms_unet* net);
const char* ms_unet_last_error(const ms_unet* net);
ms_status ms_unet_param_count(const ms_unet* net, int64_t* n);
ms_status ms_unet_get_params(ms_unet* net, float* host, int64_t n);
/* also clears the Adam state */
ms_status ms_unet_set_params(ms_unet* net, const float* host, int64_t n);
/* out = net(in) */
ms_status ms_unet_forward(ms_unet* net, const float* in, int32_t H, int32_t W, float* out,
                          void* stream);
/* out = net(in); loss = mean((out - target)^2) (FP64); grads_host (NULL or
 * param_count floats) receives d loss / d params (for checking). */
ms_status ms_unet_gradients(ms_unet* net, const float* in, const float* target, int32_t H,
                            int32_t W, float* out, float* grads_host, double* loss,
                            void* stream);
/* Checking aids (no part of the method): keep = 1 makes later
 * ms_unet_gradients calls keep every layer's bfloat16 pre-activation
 * gradient (memory for max_side is allocated on the first enable).
 * ms_unet_layer_tensor copies to host FP32 `host` [H_l][W_l][c] (n floats,
 * H_l = H >> level of the layer, H x W of the last forward pass) layer
 * `layer`'s (execution order) stored bfloat16 input activation (which = 0,
 * c = c_in), its stored output after the ReLU (1, c = c_out; not the head)
 * or its kept pre-activation gradient (2, c = c_out), so that each layer's
 * products can be checked on exactly the values the device used.
 * Errors: MS_ERR_ARG (range, size, nothing kept). */
ms_status ms_unet_keep_intermediates(ms_unet* net, int32_t keep);
ms_status ms_unet_layer_tensor(ms_unet* net, int32_t layer, int32_t which, float* host,
                               int64_t n);
/* one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) at learning rate lr on the
 * mean squared error; *loss receives the loss before the step. */
ms_status ms_unet_train_step(ms_unet* net, const float* in, const float* target, int32_t H,
                             int32_t W, float lr, double* loss, void* stream);

/* lambda of major cycle n (>= 1) of a step from its residual image i~_n
 * (dev N*N), as the reconstruct calls set it: rule NORM2_2N gives
 * coef ||i~_n||_2 2^n (Sect. 5, App. A.2), MAX_FIXED gives coef max|i~_n|
 * (the residual taken as the step's first).  Reductions in FP64; result to
 * host *lambda.  Errors: MS_ERR_ARG (rule, n < 1, NULL pointers). */
ms_status ms_lambda(ms_plan* plan, int32_t rule, double coef, int32_t n,
                    const void* residual, double* lambda, void* stream);

/* The learned warm start of step two (Sect. 3.3's full-resolution problem):
 * s = max|i~_H1|, x0 = s net([i^_L, i~_H1] / s) (the network sees images
 * scaled to unit peak), beta = W^H x0 / M (dev [M][N][N]), so that
 * W beta = x0 (W W^H = M I).  low_image (i^_L) and residual_h1 (i~_H1) are
 * dev N*N; x0_out (dev N*N) may be NULL.  N must be a valid network size
 * (a multiple of 4 * 2^(levels-1), at most the network's max_side) and the
 * network must live on the plan's device.  The network runs on `stream`
 * (the plan's ordering rules apply). */
ms_status ms_warm_start_coefficients(ms_plan* plan, ms_unet* net, const void* low_image,
                                     const void* residual_h1, void* beta_out, void* x0_out,
                                     void* stream);

/* ------------------------------------------------------------- profiling */

/* Kernel families timed by the profiler.  SYNTH / ANALYSIS are the wavelet
 * levels 2..J, *_L1 the first level (the largest); ANALYSIS includes the
 * fused prox of the minor cycle; FFT_GRID is the Ng x Ng transform of the
 * major cycle, FFT_R2C / FFT_C2R the N x N transforms of the minor cycle
 * (for N a power of two: the row transforms, the inverse one with the
 * iteration control) and SPEC_MUL its spectral step (for N a power of two:
 * fused with the column transforms).  LINEAR_PSF is the 2N x 2N linear
 * PSF operator of the minor cycle (padding, transforms, multiply, crop) when
 * the plan uses MS_CONV_LINEAR; its objective and control kernels count as
 * SPEC_MUL. */
typedef enum {
  MS_K_DEGRID = 0, MS_K_GRID = 1, MS_K_FOLD = 2, MS_K_FFT_GRID = 3, MS_K_PAD_CROP = 4,
  MS_K_SYNTH = 5, MS_K_SYNTH_L1 = 6, MS_K_FFT_R2C = 7, MS_K_SPEC_MUL = 8,
  MS_K_FFT_C2R = 9, MS_K_ANALYSIS = 10, MS_K_ANALYSIS_L1 = 11, MS_K_LINEAR_PSF = 12,
  MS_K_COUNT = 13
} ms_kernel_family;

typedef struct {
  int64_t launches[16];   /* timed launches (groups of launches) per family   */
  double total_ms[16];    /* summed CUDA-event durations per family           */
} ms_kernel_profile;

/* on = 1: every subsequent call brackets each kernel family launch with CUDA
 * events on the plan's stream (the minor cycle then runs its passes as direct
 * launches instead of the captured graph).  on = 0 turns it off. */
ms_status ms_set_profiling(ms_plan* plan, int32_t on);

/* Waits for the plan's stream, then copies the accumulated per-family times
 * to *out; reset = 1 clears the accumulators afterwards. */
ms_status ms_get_kernel_profile(ms_plan* plan, ms_kernel_profile* out, int32_t reset);

#ifdef __cplusplus
}
#endif

#endif /* MSTEP_H */
