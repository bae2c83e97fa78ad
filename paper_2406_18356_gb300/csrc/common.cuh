// Internal declarations shared by the CUDA translation units of libmstep.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cufft.h>
#include <stdint.h>

namespace ms {

template <typename R> struct CplxOf;
template <> struct CplxOf<float> { using T = float2; };
template <> struct CplxOf<double> { using T = double2; };
template <typename R> using C2 = typename CplxOf<R>::T;

constexpr int kW = 7;          // ES kernel support in cells
constexpr int kHalfW = 3;      // (W - 1) / 2
constexpr int kMaxBases = 8;   // db1 .. db8
constexpr int kMaxTaps = 16;   // db8 has 16 taps
constexpr int kMaxLevels = 8;

// One unit of (de)gridding work: `count` sorted rows starting at `start`
// that all anchor in grid tile `tile`.
struct WorkItem {
  int32_t tile;
  int32_t start;
  int32_t count;
  int32_t pad;
};

// One job of the batched (multi-channel, multi-partition) operator: the
// plan's sorted geometry of one (channel, partition) pair, the caller's
// buffers of this call, and the job's place among all jobs' work items.
template <typename R> struct BatchJob {
  const WorkItem* items;      // the job's work items
  const uint32_t* cell;       // sorted packed anchor cells
  const C2<R>* frac;          // sorted sub-cell offsets
  const int32_t* idx;         // sorted position -> original row
  const int32_t* tile_items;  // first work item of each tile (and the total)
  C2<R>* sorted_in;           // gridding input / observed values, plan order
  C2<R>* sorted_out;          // degridding output, plan order
  C2<R>* grid;                // the job's Ng^2 grid
  const C2<R>* user_in;       // caller's visibilities (original order) or null
  C2<R>* user_out;            // caller's output visibilities (original order)
  const R* image_in;          // degridding: the caller's image
  R* image_out;               // gridding: the caller's dirty image
  int64_t n;                  // rows of the job
  int64_t item_base;          // index of the job's first item over all jobs
  int32_t nitems;
  int32_t pad;
  double inv_n;               // 1 / n (dirty-image scale; 0 when n = 0)
};

// Device-side state of a minor cycle, one per plan.  Read and written only by
// the library's kernels; the host reads it back after a cycle.
struct FistaCtl {
  int32_t k;          // iteration index (coefficients B[k] are current)
  int32_t done;       // stop flag (converged or iteration budget reached)
  int32_t converged;
  int32_t max_iters;
  int32_t error;
  int32_t pad[3];
  double lam;         // lambda
  double inv_theta;   // mu = 1/theta
  double theta;
  double c0;          // constant of the objective
  double rel_tol;
  double l1_cur;      // ||B[k]||_1
  double xkx, bx;     // <x, K x>, <b, x> of B[k]
  double F_prev, F_cur;
  double sigma2, eta2;
  double kmax;        // max K^ (unscaled)
  double norm2, absmax;  // reductions of the residual image
  double absmax_first;   // max |i~_1| of the current step
  // per-iteration scalars, computed once by the spectral kernel's final
  // block so no thread of the pass kernels spends FP64 work on them:
  // momentum t_k = (k-1)/(k+2) (0 for k < 2) in slot k & 1, step mu = 1/theta
  // and threshold lambda/theta, in FP32 and FP64
  float tf[2];
  float muf, thrf;
  double td[2];
  double mud, thrd;
  double F_target;    // stop once F <= F_target (-inf: no target)
};

template <typename R> __device__ __forceinline__ R ctl_t(const FistaCtl* c, int slot);
template <> __device__ __forceinline__ float ctl_t<float>(const FistaCtl* c, int slot) {
  return c->tf[slot];
}
template <> __device__ __forceinline__ double ctl_t<double>(const FistaCtl* c, int slot) {
  return c->td[slot];
}
template <typename R> __device__ __forceinline__ R ctl_mu(const FistaCtl* c) {
  return sizeof(R) == 8 ? (R)c->mud : (R)c->muf;
}
template <typename R> __device__ __forceinline__ R ctl_thr(const FistaCtl* c) {
  return sizeof(R) == 8 ? (R)c->thrd : (R)c->thrf;
}

// Error-free sum of two working-precision numbers: a + b = s + e exactly.
template <typename R> __device__ __forceinline__ void two_sum(R a, R b, R& s, R& e) {
  s = a + b;
  R bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Warp sum of per-lane compensated values hi + lo in the working precision
// (pairwise, each addition error-free up to the lo terms); lane 0 ends with
// the warp's (hi, lo), which the caller converts to FP64 there only.
template <typename R> __device__ __forceinline__ void warp_sum_comp(R& hi, R& lo) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    R h2 = __shfl_down_sync(0xffffffffu, hi, o);
    R l2 = __shfl_down_sync(0xffffffffu, lo, o);
    R s, e;
    two_sum(hi, h2, s, e);
    hi = s;
    lo = lo + l2 + e;
  }
}

// ES kernel phi(z) = exp(beta (sqrt(1 - z^2) - 1)) on |z| <= 1 (z = 2 t / W).
__device__ __forceinline__ float es_phi(float z, float beta) {
  float s = fmaxf(1.0f - z * z, 0.0f);
  return expf(beta * (sqrtf(s) - 1.0f));
}
__device__ __forceinline__ double es_phi(double z, double beta) {
  double s = fmax(1.0 - z * z, 0.0);
  return exp(beta * (sqrt(s) - 1.0));
}

// shared-memory address of a generic pointer into shared memory
__device__ __forceinline__ unsigned saddr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// asynchronous global -> shared copy of 4, 8 or 16 bytes (both addresses
// aligned to the size); completes at cp_async_wait after cp_async_commit
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  if (BYTES == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(saddr(dst)), "l"(src)
                 : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(saddr(dst)), "l"(src),
                 "n"(BYTES)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Programmatic dependent launch.  A kernel launched with
// launch_pdl may be scheduled while the preceding kernel of its stream is
// still running; it must call pdl_wait() before touching anything that
// kernel writes (pdl_wait returns once the predecessor has completed and its
// memory is visible; without the launch attribute it returns at once).
// pdl_trigger() lets the next kernel be scheduled early.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

#ifndef MS_PDL
#define MS_PDL 1   // programmatic dependent launch of the FISTA kernels
#endif
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = MS_PDL ? 1 : 0;   // without the attribute: an ordinary launch
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Streaming multiprocessors of the current device (queried once per device
// and cached): grid caps of the grid-stride kernels are multiples of it.
int sm_count();

// -------------------------------------------------------------------------
// launch wrappers (defined in the .cu files); all take the launch stream
// -------------------------------------------------------------------------

// plan_kernels.cu
void launch_classify(const double* u, const double* v, const uint8_t* flags, int64_t n,
                     int Ng, int npix, double dl, double ell, double delta, int tile,
                     int ntx, uint32_t* cell, double2* frac, uint32_t* tile_id,
                     uint8_t* member, cudaStream_t s);
void launch_make_keys(const uint32_t* tile_id, const uint32_t* cell, const uint8_t* member,
                      int64_t n, uint8_t mask, int log2_tile, uint32_t sentinel, uint32_t* keys,
                      int32_t* vals, cudaStream_t s);
// stable LSD radix sort of (keys, vals) on the low `bits` bits of keys;
// tmp buffers of n elements; returns the pointers holding the result
void radix_sort(uint32_t** keys, int32_t** vals, uint32_t* ktmp, int32_t* vtmp, int64_t n,
                int bits, int32_t* hist, int64_t hist_cap, cudaStream_t s);
int64_t radix_hist_size(int64_t n);
void launch_count_tiles(const uint32_t* keys, int64_t n, int shift, int32_t* counts,
                        cudaStream_t s);
void launch_exclusive_scan(const int32_t* in, int32_t* out, int n, cudaStream_t s);
void launch_chunks_per_tile(const int32_t* counts, int ntiles, int chunk, int32_t* nchunks,
                            cudaStream_t s);
void launch_make_items(const int32_t* counts, const int32_t* tile_start,
                       const int32_t* item_start, int ntiles, int chunk, WorkItem* items,
                       cudaStream_t s);
template <typename R>
void launch_gather_geometry(const int32_t* idx, int64_t n, const uint32_t* cell_all,
                            const double2* frac_all, uint32_t* cell, C2<R>* frac,
                            cudaStream_t s);
template <typename R>
void launch_gather_vis(const int32_t* idx, int64_t n, const C2<R>* src, C2<R>* dst,
                       cudaStream_t s);
template <typename R>
void launch_scatter_vis(const int32_t* idx, int64_t n, const C2<R>* src, C2<R>* dst,
                        cudaStream_t s);
void launch_deapodization(int npix, int ngrid, double beta, const double* nodes,
                          const double* weights, int nq, double* psi, cudaStream_t s);

// grid_kernels.cu
template <typename R>
void launch_pad(const R* image, const R* psi, int npix, int Ng, C2<R>* grid, cudaStream_t s);
template <typename R>
void launch_crop(const C2<R>* grid, const R* psi, int npix, int Ng, double scale, R* image,
                 cudaStream_t s);
template <typename R>
void launch_degrid(const CUtensorMap* tmap, const C2<R>* grid, const WorkItem* items,
                   int nitems, const uint32_t* cell, const C2<R>* frac, const C2<R>* obs,
                   C2<R>* out, int Ng, int tile, int ntx, double beta, int32_t* err,
                   cudaStream_t s);
template <typename R, bool KAHAN>
void launch_grid(const WorkItem* items, int nitems, const uint32_t* cell, const C2<R>* frac,
                 const C2<R>* vis, void* scratch, int Ng, int tile, int ntx, double beta,
                 cudaStream_t s);
template <typename R, bool KAHAN>
void launch_fold(const void* scratch, const int32_t* tile_items, int Ng, int tile, int ntx,
                 C2<R>* grid, cudaStream_t s);
size_t grid_scratch_cell_bytes(int precision);
// batched form (all launches take the device job table)
template <typename R>
void launch_job_of(const BatchJob<R>* jobs, int njobs, int max_items, int32_t* job_of,
                   cudaStream_t s);
template <typename R>
void launch_batch_gather(const BatchJob<R>* jobs, int njobs, int64_t max_n, cudaStream_t s);
template <typename R>
void launch_batch_scatter(const BatchJob<R>* jobs, int njobs, int64_t max_n, cudaStream_t s);
template <typename R, bool KAHAN>
void launch_grid_batch(const BatchJob<R>* jobs, const int32_t* job_of, int total_items,
                       void* scratch, int tile, int ntx, double beta, cudaStream_t s);
template <typename R, bool KAHAN>
void launch_fold_batch(const BatchJob<R>* jobs, int njobs, const void* scratch, int Ng,
                       int tile, int ntx, cudaStream_t s);
template <typename R>
void launch_degrid_batch(const CUtensorMap* tmap, const BatchJob<R>* jobs,
                         const int32_t* job_of, int total_items, bool has_obs, int Ng, int tile,
                         int ntx, double beta, int32_t* err, cudaStream_t s);
template <typename R>
void launch_pad_batch(const BatchJob<R>* jobs, int njobs, const R* psi, int npix, int Ng,
                      cudaStream_t s);
template <typename R>
void launch_crop_batch(const BatchJob<R>* jobs, int njobs, const R* psi, int npix, int Ng,
                       cudaStream_t s);

// wavelet_kernels.cu
void set_wavelet_filters(const double* h, const int* len, int nbases);   // host -> __constant__
struct WaveletGeom {
  int N, J, M;
};
// coef3 / B3 / Yh2 are DEVICE arrays of pointers; with a FistaCtl the kernels
// pick buffer k % 3 (and k % 2) from it and skip all work once ctl->done is set
template <typename R>
void launch_synthesis3(const R* const* coef3_dev, R* x, R* tmp, WaveletGeom g,
                       const FistaCtl* ctl, cudaStream_t s, int only_level = 0);
template <typename R>
void launch_analysis(const R* x, R* coef, R* tmp, WaveletGeom g, cudaStream_t s);
// Buffers of one minor-cycle pass, passed by value to the persistent pass
// kernels: the coefficient ring B0..B2 (B[k % 3] is current), the gradient
// image 2 (K W alpha_k - b) written by the inverse FFT, the synthesized image
// x = W B_k, the approximation ping-pong, the control block and the per-block
// partial sums of ||B_{k+1}||_1.
// CTAs of each basis's group in the one-launch coarse levels: basis m owns
// CTAs [first[m], first[m + 1]).
struct CoarseGroups {
  int first[kMaxBases + 1];
};
// Batched minor cycles: `jobs` independent FISTA problems whose state lives
// in arrays of equal per-job slices; a kernel's blockIdx.z is its job, and
// each buffer of job z starts z times its stride (elements) after job 0's.
// The default (one job, zero strides) is the plain minor cycle.
struct JobStride {
  int jobs = 1;
  int64_t coef = 0;    // coefficient ring entries B_k (M N^2)
  int64_t img = 0;     // images x, gradient (N^2)
  int64_t tmp = 0;     // wavelet temporaries
  int64_t spec = 0;    // half-plane spectra and multipliers (N (N/2+1))
  int64_t parts = 0;   // reduction partials (doubles)
  int64_t l1 = 0;      // l1 partials of the analysis levels
  int64_t trace = 0;   // objective trace entries
};                     // (the control blocks are consecutive: ctl + z)

template <typename R> struct FistaPass {
  R* B0;
  R* B1;
  R* B2;
  const R* grad;
  R* x;
  R* tmp;
  FistaCtl* ctl;
  double* l1_parts;
  int N, J, M;
  int coarse_ctas;     // CTAs of the one-launch coarse levels (0: one launch per level)
  int coarse_budget;   // their shared-memory budget per CTA (bytes)
  CoarseGroups coarse_groups;
  int* coarse_bar;     // group barrier state, two ints per basis, zero at rest
  JobStride js{};      // batched minor cycles (coarse_ctas must then be 0)
};

// this block's job's view of a (batched) pass
template <typename R> __device__ __forceinline__ FistaPass<R> job_slice(FistaPass<R> a) {
  const int64_t z = blockIdx.z;
  if (z != 0) {
    a.B0 += z * a.js.coef;
    a.B1 += z * a.js.coef;
    a.B2 += z * a.js.coef;
    a.grad += z * a.js.img;
    a.x += z * a.js.img;
    a.tmp += z * a.js.tmp;
    a.ctl += z;
    a.l1_parts += z * a.js.l1;
  }
  return a;
}
// The minor cycle's synthesis levels (J..1) and analysis + FISTA-update
// levels (1..J), one launch per level.  only_level: 0 = all levels, j > 0 =
// level j alone, -1 = all levels but level 1.  The analysis takes an optional
// TMA descriptor of the gradient image (nullptr: plain loads) and writes one
// l1 partial per block, analysis_prox_partials() in all.
template <typename R>
cudaError_t launch_synthesis_pass(const FistaPass<R>& a, cudaStream_t s, int only_level = 0);
template <typename R>
cudaError_t launch_analysis_pass(const FistaPass<R>& a, const CUtensorMap* grad_map,
                                 cudaStream_t s, int only_level = 0);
int analysis_prox_partials(WaveletGeom g);
void analysis_window_box(unsigned* cols, unsigned* rows);

// iuwt_kernels.cu: the IUWT dictionary W = T^H (J levels, J + 1 planes).
// fp = NULL: plain transforms of alpha / img; fp = the minor cycle's pass:
// synthesis of B_k into x, analysis of the gradient image into FISTA's step
// on B_k+1 (iuwt_prox_partials(J) l1 partials).  work: 3 N x N images.
template <typename R>
cudaError_t launch_iuwt_synthesis(const FistaPass<R>* fp, const R* alpha, R* x, R* work, int N,
                                  int J, cudaStream_t s);
template <typename R>
cudaError_t launch_iuwt_analysis(const FistaPass<R>* fp, const R* img, R* alpha, R* work, int N,
                                 int J, cudaStream_t s);
int iuwt_prox_partials(int J);
// The one-launch coarse levels (2..J of both transforms, one cooperative
// launch per transform) on the current device: the CTAs of each basis's
// group (in proportion to its filter length) and the shared-memory budget
// per CTA with which all of them are resident at once.  Returns the number
// of CTAs, or 0 when the geometry needs the per-level kernels (N not a power
// of two, N < 256, N >> J < 8, J < 2) or no such launch fits.
int coarse_groups(WaveletGeom g, size_t rsz, CoarseGroups* groups, int* budget);

// spectral_kernels.cu
int spectral_partials(int N);
template <typename R>
void launch_ifftshift_real(const R* in, R* out, int N, cudaStream_t s);
template <typename R>
void launch_real_part_spectrum(const C2<R>* in, R* out, int n, cudaStream_t s);
template <typename R>
void launch_filters(int N, double ell, double delta, const FistaCtl* ctl, R* gl2, R* gh2,
                    cudaStream_t s, int mirror = 0);
template <typename R>
void launch_combine_spectra(C2<R>* a, const C2<R>* b, const R* gl2, const R* gh2,
                            const FistaCtl* ctl, int N, cudaStream_t s);
template <typename R>
void launch_normal_spectrum(const R* Hhat, const R* gl2, const R* gh2, int N, int M, R* Ks,
                            double* parts, FistaCtl* ctl, int32_t* ticket, cudaStream_t s);
template <typename R>
void launch_b_spectrum(const C2<R>* Ihat, const C2<R>* Lhat, const R* Hhat, const R* gl2,
                       const R* gh2, int N, C2<R>* Bs, double* parts, FistaCtl* ctl,
                       int32_t* ticket, cudaStream_t s);
// the spectral step with the column FFTs fused in (N a power of two, 16 ..
// 8192); Z holds the row transforms of x_k on entry and the inverse column
// transforms of the gradient spectrum on exit; tw = exp(-2 pi i m / N),
// m < N; each warp leaves its sums of the objective terms in
// parts[i W + warp], i = 0..2 (W = spec_col_warps), for launch_row_c2r
template <typename R>
cudaError_t launch_spec_col(C2<R>* Z, C2<R>* Xk, const C2<R>* Xprev, const R* Ks,
                            const C2<R>* Bs, const C2<R>* tw, int N, double* parts,
                            const FistaCtl* ctl, const double* l1_parts, int n_l1,
                            cudaStream_t s, const JobStride& js = JobStride{});
int spec_col_blocks(int N, size_t complex_bytes);   // blocks of one launch (0: N unsupported)
int spec_col_warps(int N, size_t complex_bytes);    // warps of one launch (0: N unsupported)
// real row transforms of an N x N image (N a power of two, 16 <= N <= 8192)
// to / from the half-plane layout [N][N/2+1], through complex transforms of
// length N/2 in shared memory; the inverse is unnormalized and ignores the
// imaginary parts of columns 0 and N/2; tw as for launch_spec_col; both
// return at once when ctl->done.  With parts non-null, an extra block of the
// inverse sums the G warp sums launch_spec_col left and runs the iteration
// control (objective into trace, ctl update).  js: the batched form, each
// job's slices of x, Z (and the spectra), parts, trace and its ctl.
template <typename R>
cudaError_t launch_row_r2c(const R* x, C2<R>* Z, const C2<R>* tw, int N, const FistaCtl* ctl,
                           cudaStream_t s, const JobStride& js = JobStride{});
template <typename R>
cudaError_t launch_row_c2r(const C2<R>* Z, R* x, const C2<R>* tw, int N, FistaCtl* ctl,
                           const double* parts, int G, double* trace, cudaStream_t s,
                           const JobStride& js = JobStride{});
// dynamic shared memory of a block (SIZE_MAX: N unsupported)
size_t row_fft_smem(int N, size_t complex_bytes);
// dynamic shared memory of a block (SIZE_MAX: N unsupported)
size_t spec_col_smem(int N, size_t complex_bytes);
template <typename R>
void launch_spec_mul(const C2<R>* Xk, C2<R>* Xprev, const R* Ks, const C2<R>* Bs, int N,
                     double* parts, FistaCtl* ctl, double* trace, int32_t* ticket,
                     const double* l1_parts, int n_l1, cudaStream_t s);
template <typename R>
void launch_spec_apply(C2<R>* spec, const R* Ks, int N, cudaStream_t s);
template <typename R>
void launch_image_norms(const R* img, int64_t n, double* parts, FistaCtl* ctl, int32_t* ticket,
                        cudaStream_t s);
template <typename R>
void launch_sigma2_hat(const R* img, int N, double* parts, FistaCtl* ctl, int32_t* ticket,
                       int set_eta, cudaStream_t s);
void launch_set_lambda(FistaCtl* ctl, int rule, double coef, int n, int first, cudaStream_t s);
template <typename R>
void launch_axpby(const R* x, const R* y, R* out, double a, double b, int64_t n, cudaStream_t s);
template <typename R>
void launch_l1(const R* x, int64_t n, double* parts, double* out, int32_t* ticket,
               cudaStream_t s);
template <typename R>
void launch_dot(const R* x, const R* y, int64_t n, double* parts, double* out, int32_t* ticket,
                cudaStream_t s);
template <typename R>
void launch_normalize(R* x, int64_t n, const double* den, cudaStream_t s);
template <typename R>
void launch_hash_fill(R* x, int64_t n, uint64_t seed, cudaStream_t s);
// the linear PSF operator of the minor cycle (2N x 2N zero padding)
template <typename R>
void launch_lin_pad(const R* x, R* xp, int N, const FistaCtl* ctl, cudaStream_t s);
template <typename R>
void launch_lin_mul(C2<R>* S, const R* H2, int N, const FistaCtl* ctl, cudaStream_t s);
template <typename R>
void launch_lin_crop(const R* q, const R* add, R* out, int N, double scale, const FistaCtl* ctl,
                     cudaStream_t s);
template <typename R>
void launch_lin_low_step(const R* q, const R* res, R* ycur, const R* yprev, R* rp, int N,
                         double* parts, FistaCtl* ctl, double* trace, int32_t* ticket,
                         const double* l1_parts, int n_l1, cudaStream_t s);
template <typename R>
void launch_lin_full_diff(const R* q, const R* res, const R* x, const R* l, R* de, int N,
                          const FistaCtl* ctl, cudaStream_t s);
template <typename R>
void launch_lin_full_spec(const C2<R>* dek, const C2<R>* dep, const R* gl2, const R* gh2,
                          C2<R>* uv, int N, double* parts, FistaCtl* ctl, double* trace,
                          int32_t* ticket, const double* l1_parts, int n_l1, cudaStream_t s);
template <typename R>
void launch_lin_theta(const R* H2, int N, const R* gl2, const R* gh2, int M, double* parts,
                      FistaCtl* ctl, int32_t* ticket, cudaStream_t s);

}  // namespace ms
