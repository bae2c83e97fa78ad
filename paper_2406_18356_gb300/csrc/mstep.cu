// libmstep: plan object, C ABI and the orchestration of the method.
//
// Host code only sequences kernels: every step of the path (partitioning,
// sorting, gridding, the operator's FFTs through cuFFT, wavelets, FISTA with
// its own spectral-step transforms, reductions) runs on the device.  All work of a call is issued on a plan-owned stream
// that is ordered after the caller's stream at entry, and the caller's stream
// is ordered after it at exit.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cufft.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "common.cuh"
#include "mstep.h"

#ifndef MS_FUSED_SPEC_FP32
#define MS_FUSED_SPEC_FP32 1   // FP32 plans use the fused spectral step too
#endif
using namespace ms;

// the device a network was created on (defined with the network)
int ms_unet_device_of(const ms_unet* net);

namespace {

// ---------------------------------------------------------------- helpers
struct Fail {
  ms_status st;
  std::string msg;
};

void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Fail{e == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e)};
  }
}

void ckf(cufftResult r, const char* what) {
  if (r != CUFFT_SUCCESS)
    throw Fail{r == CUFFT_ALLOC_FAILED ? MS_ERR_OOM : MS_ERR_CUDA,
               std::string(what) + ": cuFFT error " + std::to_string((int)r)};
}

void arg(bool ok, const char* what) {
  if (!ok) throw Fail{MS_ERR_ARG, what};
}

template <typename T> T* dalloc(size_t n, const char* what) {
  void* p = nullptr;
  if (n == 0) n = 1;
  ck(cudaMalloc(&p, n * sizeof(T)), what);
  return static_cast<T*>(p);
}

// Daubechies low-pass filter db_p (2p taps, sum sqrt 2): roots y_i of
// P(y) = sum_{k<p} C(p-1+k, k) y^k by Durand-Kerner iteration in long double,
// each mapped to the root z of z + 1/z = 2 - 4 y_i with |z| > 1, then
// h ~ (1 + z)^p prod (z - z_i) in ascending powers of z.
std::vector<double> daubechies(int p) {
  typedef std::complex<long double> cx;
  if (p == 1) return {std::sqrt(0.5), std::sqrt(0.5)};
  const int deg = p - 1;
  std::vector<long double> c(p);
  for (int k = 0; k < p; ++k) {
    long double b = 1;   // C(p-1+k, k)
    for (int i = 1; i <= k; ++i) b = b * (p - 1 + i) / i;
    c[k] = b;
  }
  auto P = [&](cx y) {
    cx s = 0;
    for (int k = deg; k >= 0; --k) s = s * y + c[k];
    return s;
  };
  std::vector<cx> r(deg);
  for (int i = 0; i < deg; ++i) r[i] = std::pow(cx(0.4L, 0.9L), i);
  for (int it = 0; it < 2000; ++it) {
    long double moved = 0;
    for (int i = 0; i < deg; ++i) {
      cx den = c[deg];
      for (int j = 0; j < deg; ++j)
        if (j != i) den *= (r[i] - r[j]);
      cx d = P(r[i]) / den;
      r[i] -= d;
      moved = std::max(moved, std::abs(d));
    }
    if (moved < 1e-30L) break;
  }
  std::vector<cx> q(1, cx(1));   // ascending powers of z
  for (int i = 0; i < deg; ++i) {
    cx s = cx(1) - cx(2) * r[i];
    cx disc = std::sqrt(s * s - cx(1));
    cx z = s + disc;
    if (std::abs(z) < 1) z = s - disc;
    std::vector<cx> nq(q.size() + 1, cx(0));
    for (size_t k = 0; k < q.size(); ++k) {
      nq[k] -= z * q[k];
      nq[k + 1] += q[k];
    }
    q.swap(nq);
  }
  std::vector<cx> h(q.size() + p, cx(0));
  for (size_t k = 0; k < q.size(); ++k) {
    long double b = 1;
    for (int i = 0; i <= p; ++i) {
      h[k + i] += b * q[k];
      b = b * (p - i) / (i + 1);
    }
  }
  long double sum = 0;
  for (auto& v : h) sum += v.real();
  std::vector<double> out(h.size());
  for (size_t k = 0; k < h.size(); ++k)
    out[k] = (double)(h[k].real() * std::sqrt((long double)2) / sum);
  return out;
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton on the three-term
// recurrence of P_n).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  const long double pi = 3.141592653589793238462643383279502884L;
  for (int i = 0; i < n; ++i) {
    long double z = std::cos(pi * (i + 0.75L) / (n + 0.5L));
    long double dp = 0;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) {
        long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1);
      long double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-19L) break;
    }
    x[i] = (double)z;
    w[i] = (double)(2 / ((1 - z * z) * dp * dp));
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

__global__ void set_ptrs_kernel(void** dst, void* a, void* b, void* c) {
  dst[0] = a;
  dst[1] = b;
  dst[2] = c;
}

__global__ void init_ctl_kernel(FistaCtl* ctl, int max_iters, double rel_tol, double lam,
                                int set_lam, double sigma2, double eta2, int set_noise) {
  ctl->k = 0;
  ctl->done = 0;
  ctl->converged = 0;
  ctl->max_iters = max_iters;
  ctl->error = 0;
  ctl->rel_tol = rel_tol;
  if (set_lam) ctl->lam = lam;
  if (set_noise) {
    ctl->sigma2 = sigma2;
    ctl->eta2 = eta2;
  }
  ctl->F_prev = NAN;
  ctl->F_cur = NAN;
  ctl->tf[0] = ctl->tf[1] = 0.0f;   // t_0 = t_1 = 0
  ctl->td[0] = ctl->td[1] = 0.0;
}

__global__ void set_eta_kernel(FistaCtl* ctl, double eta2) { ctl->eta2 = eta2; }

__global__ void set_target_kernel(FistaCtl* ctl, double target) { ctl->F_target = target; }

__global__ void scale_scalar_kernel(const double* in, double a, double* out) { *out = a * *in; }

// step size from a device value (the IUWT's power iteration)
__global__ void set_theta_kernel(FistaCtl* ctl, const double* theta) {
  const double th = *theta;
  if (!(th > 0.0) || !isfinite(th)) {
    ctl->error = 4;
    return;
  }
  ctl->theta = th;
  ctl->inv_theta = 1.0 / th;
}

// Network input of the learned warm start: [i^_L, i~_H1] / max|i~_H1|,
// channels last (FP32 [n][2]); the peak comes from launch_image_norms.
template <typename R>
__global__ void ws_input_kernel(const R* __restrict__ low, const R* __restrict__ res,
                                const FistaCtl* __restrict__ ctl, int64_t n,
                                float* __restrict__ in) {
  const double a = ctl->absmax;
  const float sc = a > 0.0 ? (float)(1.0 / a) : 0.0f;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    in[2 * k] = (float)low[k] * sc;
    in[2 * k + 1] = (float)res[k] * sc;
  }
}

// x0 = max|i~_H1| times the network's output
template <typename R>
__global__ void ws_output_kernel(const float* __restrict__ out, const FistaCtl* __restrict__ ctl,
                                 int64_t n, R* __restrict__ x0) {
  const R a = (R)ctl->absmax;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    x0[k] = (R)out[k] * a;
}

__global__ void check_noise_kernel(FistaCtl* ctl) {
  if (!(ctl->sigma2 > 0.0) || !(ctl->eta2 > 0.0) || !isfinite(ctl->sigma2) ||
      !isfinite(ctl->eta2))
    ctl->error = 4;
}

}  // namespace

// ====================================================================== plan
// FULL-kind problems (Eq. FullRes, and its mirror on V_L)
inline bool step_full(int step) { return step == MS_STEP_FULL || step == MS_STEP_FULL_L; }

struct PartDev {
  int64_t n = 0;
  int32_t* idx = nullptr;
  uint32_t* cell = nullptr;
  void* frac = nullptr;
  WorkItem* items = nullptr;
  int nitems = 0;
  int32_t* tile_items = nullptr;
  void* Hhat = nullptr;
  bool have_psf = false;
  void* Hhat2 = nullptr;   // real spectrum of the PSF on the 2N x 2N field (linear operator)
};

// Batched minor cycles: each job's FISTA state as one slice of these arrays
// (JobStride), so one launch of each pass kernel covers every job; the
// reconstruct call adds each job's model, residual and l images.
struct FistaBatch {
  int cap = 0;         // jobs the arrays hold
  int trace_cap = 0;   // trace entries per job
  void* B[3] = {};
  void *x = nullptr, *y = nullptr, *F[2] = {}, *zrow = nullptr, *Ks = nullptr, *Bs = nullptr;
  void* tmp = nullptr;
  void *model = nullptr, *res = nullptr, *l = nullptr;
  FistaCtl* ctl = nullptr;
  double *trace = nullptr, *parts = nullptr, *l1 = nullptr;
  int64_t parts_stride = 0;
  CUtensorMap gmap{};   // the jobs' gradient images stacked: {N, cap N}
  bool have_gmap = false;
  cudaGraphExec_t exec = nullptr;
  int exec_jobs = 0;
  void release() {
    for (void* q : {B[0], B[1], B[2], x, y, F[0], F[1], zrow, Ks, Bs, tmp, model, res, l,
                    (void*)ctl, (void*)trace, (void*)parts, (void*)l1})
      if (q) cudaFree(q);
    if (exec) cudaGraphExecDestroy(exec);
    *this = FistaBatch{};
  }
};

struct ChanDev {
  PartDev part[3];
  int64_t counts[4] = {0, 0, 0, 0};
};

struct ms_plan {
  ms_plan_desc d{};
  int dev = 0, N = 0, Ng = 0, T = 0, S = 0, ntx = 0, ntiles = 0, J = 0, M = 0, prec = 0;
  int chunk = 0;
  size_t rsz = 8;
  double beta = 0;
  std::vector<ChanDev> ch;
  std::vector<void*> allocs;
  cudaStream_t ps = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<cudaEvent_t> tev;   // timing events
  // tables / workspaces
  void* psi = nullptr;
  void* grid = nullptr;
  void* scratch = nullptr;
  int max_items = 0;
  int64_t max_n = 0;
  void *vis_a = nullptr, *vis_b = nullptr;
  void* img[6] = {};
  void *B[3] = {}, *xwork = nullptr, *ywork = nullptr;
  void *F[2] = {};   // FISTA spectra X^_k / X^_{k-1} (ping-pong by pass parity)
  void *spec = nullptr, *spec2 = nullptr, *Ks = nullptr, *Bs = nullptr;
  void *gl2 = nullptr, *gh2 = nullptr, *wtmp = nullptr;
  void** api3_dev = nullptr;   // pointer table of the one-shot synthesis calls
  CUtensorMap grad_map{};   // TMA descriptor of the gradient image (ywork)
  bool have_grad_map = false;
  FistaCtl* ctl = nullptr;
  double* trace = nullptr;
  double* parts = nullptr;     // reduction partials (one reduction at a time)
  double* l1parts = nullptr;   // per-block |B_k+1| partials of the analysis levels
  int n_l1 = 0;                // their number
  int dict = MS_DICT_DAUBECHIES;   // minor-cycle dictionary
  int coarse_ctas = 0;         // CTAs of the one-launch coarse levels (0: one launch per level)
  int coarse_budget = 0;       // their shared-memory budget per CTA
  CoarseGroups coarse_gr{};    // their split over the bases
  int* coarse_bar = nullptr;   // their group barrier state
  int32_t* tickets = nullptr;
  double* scal = nullptr;
  int32_t* err = nullptr;
  int trace_cap = 0;
  cufftHandle c2c = 0, r2c = 0, c2r = 0;
  // fused spectral step (N a power of two whose blocks fit in shared
  // memory): the row-transform buffer and the twiddles
  bool fused_spec = false;
  void* zrow = nullptr;
  void* twid = nullptr;
  CUtensorMap tmap{};
  std::string msg;
  std::vector<double> htrace;
  double obj_target = -INFINITY;   // objective target of the minor cycles (-inf: none)
  // learned warm start: network input / output (FP32), x0 and beta_0
  float* ws_in = nullptr;
  float* ws_out = nullptr;
  void* ws_x0 = nullptr;
  void* ws_beta = nullptr;
  void* il_buf = nullptr;   // interleaved pipeline without the batched form: 6 images
  // profiling: CUDA-event spans per kernel family
  bool prof = false;
  bool capturing = false;
  std::vector<cudaEvent_t> evpool;
  struct Span {
    int fam;
    cudaEvent_t a, b;
  };
  std::vector<Span> pending;
  int64_t k_launch[16] = {};
  double k_ms[16] = {};
  // linear PSF operator of the minor cycle (MS_CONV_LINEAR): the 2N x 2N pad
  // and product images and their spectrum, the current problem's H2^, i~ and
  // l, the ring of H x_k (LOW / SINGLE), the stacked [D; E] images, their
  // spectra by pass parity, the filtered spectra [U^; V^] and their images
  int conv = MS_CONV_CIRCULAR;
  void *lp = nullptr, *lq = nullptr, *ls = nullptr, *lh2 = nullptr;
  void *lres = nullptr, *ll = nullptr, *ly[2] = {};
  void *lde = nullptr, *ldes[2] = {}, *luvs = nullptr, *luv = nullptr;
  cufftHandle r2c2 = 0, c2r2 = 0, r2cb = 0, c2rb = 0;
  cudaGraphExec_t lin_exec[2] = {};   // captured linear passes: LOW / SINGLE, FULL
  FistaBatch fb;   // batched minor cycles
  // captured FISTA passes
  cudaGraphExec_t fista_exec = nullptr;
  int fista_graph_step = -1;
  int fista_graph_passes = 0;

  template <typename T> T* alloc(size_t n, const char* what) {
    T* p = dalloc<T>(n, what);
    allocs.push_back(p);
    return p;
  }
  // batched form: workspaces grown on demand, freed with the plan
  struct Batch {
    int cap_jobs = 0;
    int64_t cap_items = 0, cap_rows = 0;
    void* jobs = nullptr;       // BatchJob<R>[cap_jobs]
    int32_t* job_of = nullptr;  // [cap_items]
    void* grids = nullptr;      // cap_jobs Ng^2 complex
    void* scratch = nullptr;    // cap_items tiles
    void* rows_a = nullptr;     // cap_rows complex (inputs in plan order)
    void* rows_b = nullptr;     // cap_rows complex (outputs in plan order)
    cufftHandle fft = 0;
    int fft_jobs = 0;
    CUtensorMap tmap{};
    int tmap_jobs = 0;
  } batch;
};

namespace {

constexpr int kPasses = 8;   // FISTA passes per captured graph launch

cudaEvent_t pool_event(ms_plan* p) {
  if (!p->evpool.empty()) {
    cudaEvent_t e = p->evpool.back();
    p->evpool.pop_back();
    return e;
  }
  cudaEvent_t e;
  ck(cudaEventCreate(&e), "event");
  return e;
}

// Sums the finished spans into the per-family accumulators (synchronizes).
void harvest(ms_plan* p) {
  if (p->pending.empty()) return;
  ck(cudaStreamSynchronize(p->ps), "synchronize");
  for (auto& s : p->pending) {
    float ms = 0;
    ck(cudaEventElapsedTime(&ms, s.a, s.b), "event time");
    p->k_ms[s.fam] += ms;
    p->k_launch[s.fam] += 1;
    p->evpool.push_back(s.a);
    p->evpool.push_back(s.b);
  }
  p->pending.clear();
}

// Brackets the launches of one kernel family with events when profiling.
struct KSpan {
  ms_plan* p;
  int fam;
  cudaEvent_t a = nullptr;
  KSpan(ms_plan* pl, int f) : p(pl), fam(f) {
    if (p->prof && !p->capturing) {
      a = pool_event(p);
      ck(cudaEventRecord(a, p->ps), "event record");
    }
  }
  ~KSpan() {
    if (!a) return;
    cudaEvent_t b = pool_event(p);
    cudaEventRecord(b, p->ps);
    p->pending.push_back({fam, a, b});
  }
};

struct Timer {
  ms_plan* p;
  std::vector<std::pair<int, int>> spans[3];   // grid, fft, minor
  int used = 0;
  explicit Timer(ms_plan* pl) : p(pl) {}
  int mark() {
    if (used >= (int)p->tev.size()) {
      cudaEvent_t e;
      ck(cudaEventCreate(&e), "event");
      p->tev.push_back(e);
    }
    ck(cudaEventRecord(p->tev[used], p->ps), "event record");
    return used++;
  }
  double total(int which) {
    double t = 0;
    for (auto& s : spans[which]) {
      float ms = 0;
      ck(cudaEventElapsedTime(&ms, p->tev[s.first], p->tev[s.second]), "event time");
      t += ms;
    }
    return t;
  }
};

// Restores the calling thread's current device when it goes out of scope.
struct DeviceGuard {
  int prev = 0;
  DeviceGuard() { cudaGetDevice(&prev); }
  ~DeviceGuard() { cudaSetDevice(prev); }
};

struct Scope {
  ms_plan* p;
  cudaStream_t user;
  int prev_dev = 0;
  Scope(ms_plan* pl, void* stream) : p(pl), user((cudaStream_t)stream) {
    cudaGetDevice(&prev_dev);
    ck(cudaSetDevice(p->dev), "set device");
    ck(cudaEventRecord(p->ev_in, user), "event record");
    ck(cudaStreamWaitEvent(p->ps, p->ev_in, 0), "stream wait");
  }
  void finish() {
    ck(cudaEventRecord(p->ev_out, p->ps), "event record");
    ck(cudaStreamWaitEvent(user, p->ev_out, 0), "stream wait");
    ck(cudaGetLastError(), "kernel launch");
  }
  ~Scope() { cudaSetDevice(prev_dev); }
};

template <typename F> ms_status guarded(ms_plan* p, F&& f) {
  if (!p) return MS_ERR_ARG;
  try {
    p->msg.clear();
    f();
    return MS_OK;
  } catch (const Fail& e) {
    p->msg = e.msg;
    return e.st;
  } catch (const std::exception& e) {
    p->msg = e.what();
    return MS_ERR_CUDA;
  } catch (...) {
    p->msg = "unknown failure";
    return MS_ERR_CUDA;
  }
}

void check_device_error(ms_plan* p) {
  int32_t e = 0;
  ck(cudaMemcpyAsync(&e, p->err, sizeof(e), cudaMemcpyDeviceToHost, p->ps), "read error flag");
  ck(cudaStreamSynchronize(p->ps), "synchronize");
  if (e) {
    ck(cudaMemsetAsync(p->err, 0, sizeof(int32_t), p->ps), "clear error flag");
    throw Fail{(ms_status)e, e == MS_ERR_TIMEOUT ? "a bounded device wait ran out"
                                                 : "device-side error"};
  }
}

PartDev& part_of(ms_plan* p, int part, int chan) {
  arg(chan >= 0 && chan < (int)p->ch.size(), "channel out of range");
  arg(part >= 0 && part <= 2, "partition must be MS_PART_L, MS_PART_H or MS_PART_ALL");
  return p->ch[chan].part[part];
}

// ------------------------------------------------------ measurement operator
template <typename R> void fft_c2c(ms_plan* p, int dir) {
  if (sizeof(R) == 8)
    ckf(cufftExecZ2Z(p->c2c, (cufftDoubleComplex*)p->grid, (cufftDoubleComplex*)p->grid, dir),
        "Z2Z");
  else
    ckf(cufftExecC2C(p->c2c, (cufftComplex*)p->grid, (cufftComplex*)p->grid, dir), "C2C");
}

template <typename R> void fft_r2c(ms_plan* p, const void* in, void* out) {
  if (sizeof(R) == 8)
    ckf(cufftExecD2Z(p->r2c, (cufftDoubleReal*)in, (cufftDoubleComplex*)out), "D2Z");
  else
    ckf(cufftExecR2C(p->r2c, (cufftReal*)in, (cufftComplex*)out), "R2C");
}

template <typename R> void fft_c2r(ms_plan* p, void* in, void* out) {
  if (sizeof(R) == 8)
    ckf(cufftExecZ2D(p->c2r, (cufftDoubleComplex*)in, (cufftDoubleReal*)out), "Z2D");
  else
    ckf(cufftExecC2R(p->c2r, (cufftComplex*)in, (cufftReal*)out), "C2R");
}

// real <-> half-plane transforms with a given cuFFT plan
template <typename R> void exec_r2c(cufftHandle h, const void* in, void* out) {
  if (sizeof(R) == 8)
    ckf(cufftExecD2Z(h, (cufftDoubleReal*)in, (cufftDoubleComplex*)out), "D2Z");
  else
    ckf(cufftExecR2C(h, (cufftReal*)in, (cufftComplex*)out), "R2C");
}
template <typename R> void exec_c2r(cufftHandle h, void* in, void* out) {
  if (sizeof(R) == 8)
    ckf(cufftExecZ2D(h, (cufftDoubleComplex*)in, (cufftDoubleReal*)out), "Z2D");
  else
    ckf(cufftExecC2R(h, (cufftComplex*)in, (cufftReal*)out), "C2R");
}

// model grid = F Z D image (centred)
template <typename R> void image_to_grid(ms_plan* p, const void* image, Timer* tm) {
  {
    KSpan k(p, MS_K_PAD_CROP);
    launch_pad<R>((const R*)image, (const R*)p->psi, p->N, p->Ng, (C2<R>*)p->grid, p->ps);
  }
  int a = tm ? tm->mark() : 0;
  {
    KSpan k(p, MS_K_FFT_GRID);
    fft_c2c<R>(p, CUFFT_FORWARD);
  }
  if (tm) tm->spans[1].push_back({a, tm->mark()});
}

// sorted visibilities -> model (or residual when obs given) with G
template <typename R>
void degrid_sorted(ms_plan* p, PartDev& pd, const void* obs_sorted, void* out_sorted, Timer* tm) {
  int a = tm ? tm->mark() : 0;
  {
    KSpan k(p, MS_K_DEGRID);
    launch_degrid<R>(&p->tmap, (const C2<R>*)p->grid, pd.items, pd.nitems, pd.cell,
                     (const C2<R>*)pd.frac, (const C2<R>*)obs_sorted, (C2<R>*)out_sorted, p->Ng,
                     p->T, p->ntx, p->beta, p->err, p->ps);
  }
  if (tm) tm->spans[0].push_back({a, tm->mark()});
}

// sorted visibilities -> image = Re(D Z^H F^H G^H y) / sum(w); the gridding
// kernel's per-work-item tiles go to `scratch` (NULL: the plan's buffer)
template <typename R>
void grid_sorted(ms_plan* p, PartDev& pd, const void* vis_sorted, void* image, Timer* tm,
                 void* scratch = nullptr) {
  if (!scratch) scratch = p->scratch;
  int a = tm ? tm->mark() : 0;
  if (p->prec == MS_FP32_KAHAN) {
    {
      KSpan k(p, MS_K_GRID);
      launch_grid<float, true>(pd.items, pd.nitems, pd.cell, (const float2*)pd.frac,
                               (const float2*)vis_sorted, scratch, p->Ng, p->T, p->ntx,
                               p->beta, p->ps);
    }
    KSpan k(p, MS_K_FOLD);
    launch_fold<float, true>(scratch, pd.tile_items, p->Ng, p->T, p->ntx, (float2*)p->grid,
                             p->ps);
  } else {
    {
      KSpan k(p, MS_K_GRID);
      launch_grid<R, false>(pd.items, pd.nitems, pd.cell, (const C2<R>*)pd.frac,
                            (const C2<R>*)vis_sorted, scratch, p->Ng, p->T, p->ntx, p->beta,
                            p->ps);
    }
    KSpan k(p, MS_K_FOLD);
    launch_fold<R, false>(scratch, pd.tile_items, p->Ng, p->T, p->ntx, (C2<R>*)p->grid,
                          p->ps);
  }
  int b = tm ? tm->mark() : 0;
  if (tm) tm->spans[0].push_back({a, b});
  {
    KSpan k(p, MS_K_FFT_GRID);
    fft_c2c<R>(p, CUFFT_INVERSE);
  }
  if (tm) tm->spans[1].push_back({b, tm->mark()});
  double sc = pd.n > 0 ? 1.0 / (double)pd.n : 0.0;
  KSpan k(p, MS_K_PAD_CROP);
  launch_crop<R>((const C2<R>*)p->grid, (const R*)p->psi, p->N, p->Ng, sc, (R*)image, p->ps);
}

// i~ = A^H (obs - A model) / sum(w), obs already sorted
template <typename R>
void residual_sorted(ms_plan* p, PartDev& pd, const void* obs_sorted, const void* model,
                     void* out, Timer* tm) {
  image_to_grid<R>(p, model, tm);
  degrid_sorted<R>(p, pd, obs_sorted, p->vis_b, tm);
  grid_sorted<R>(p, pd, p->vis_b, out, tm);
}

__global__ void impulse_kernel(void* img, int N, int is_double) {
  int64_t c = (int64_t)(N / 2) * N + N / 2;
  if (is_double)
    static_cast<double*>(img)[c] = 1.0;
  else
    static_cast<float*>(img)[c] = 1.0f;
}

// PSF = A^H A delta / sum(w), delta the unit impulse at (N/2, N/2)
template <typename R> void psf_image(ms_plan* p, PartDev& pd, void* out) {
  const int N = p->N;
  R* delta = (R*)p->img[5];
  ck(cudaMemsetAsync(delta, 0, sizeof(R) * N * N, p->ps), "memset");
  impulse_kernel<<<1, 1, 0, p->ps>>>(delta, N, sizeof(R) == 8);
  image_to_grid<R>(p, delta, nullptr);
  degrid_sorted<R>(p, pd, nullptr, p->vis_b, nullptr);
  grid_sorted<R>(p, pd, p->vis_b, out, nullptr);
}

template <typename R> void ensure_psf(ms_plan* p, PartDev& pd) {
  if (pd.have_psf) return;
  const int N = p->N;
  R* delta = (R*)p->img[5];
  R* psf = (R*)p->img[4];
  psf_image<R>(p, pd, psf);
  launch_ifftshift_real<R>(psf, delta, N, p->ps);
  fft_r2c<R>(p, delta, p->spec2);
  launch_real_part_spectrum<R>((const C2<R>*)p->spec2, (R*)pd.Hhat, N * (N / 2 + 1), p->ps);
  ck(cudaStreamSynchronize(p->ps), "psf");
  pd.have_psf = true;
}

// ------------------------------------------------------------- minor cycle
// One FISTA pass.  Pass i of a minor cycle has iteration index k = i, so the
// two spectrum buffers alternate with the pass parity: F[k % 2] receives
// X^_k, F[(k+1) % 2] holds X^_{k-1} and then the gradient spectrum.
template <typename R> FistaPass<R> fista_pass_args(ms_plan* p) {
  FistaPass<R> a;
  a.B0 = (R*)p->B[0];
  a.B1 = (R*)p->B[1];
  a.B2 = (R*)p->B[2];
  a.grad = (const R*)p->ywork;
  a.x = (R*)p->xwork;
  a.tmp = (R*)p->wtmp;
  a.ctl = p->ctl;
  a.l1_parts = p->l1parts;
  a.N = p->N;
  a.J = p->J;
  a.M = p->M;
  a.coarse_ctas = p->coarse_ctas;
  a.coarse_budget = p->coarse_budget;
  a.coarse_groups = p->coarse_gr;
  a.coarse_bar = p->coarse_bar;
  return a;
}

// What one FISTA pass reads and writes beyond the pass arguments: the
// spectra X^_k / X^_k-1 (by pass parity), the row-transform buffer, K^ and
// B^, the reduction partials, the objective trace and the gradient's TMA
// descriptor.  The plain minor cycle uses the plan's buffers; the batched one
// (a.js.jobs > 1) the per-job slices of its workspace.
template <typename R> struct PassView {
  FistaPass<R> a;
  C2<R>* F[2];
  C2<R>* zrow;
  const R* Ks;
  const C2<R>* Bs;
  double* parts;
  double* trace;
  const CUtensorMap* gmap;
};

template <typename R> PassView<R> plan_view(ms_plan* p) {
  PassView<R> v;
  v.a = fista_pass_args<R>(p);
  v.F[0] = (C2<R>*)p->F[0];
  v.F[1] = (C2<R>*)p->F[1];
  v.zrow = (C2<R>*)p->zrow;
  v.Ks = (const R*)p->Ks;
  v.Bs = (const C2<R>*)p->Bs;
  v.parts = p->parts;
  v.trace = p->trace;
  v.gmap = p->have_grad_map ? &p->grad_map : nullptr;
  return v;
}

// x_k = W B_k into a.x (levels J..1)
template <typename R> void record_synthesis(ms_plan* p, const FistaPass<R>& a) {
  if (p->dict == MS_DICT_IUWT) {
    KSpan k(p, MS_K_SYNTH_L1);
    ck(launch_iuwt_synthesis<R>(&a, nullptr, a.x, (R*)p->wtmp, p->N, p->J, p->ps),
       "IUWT synthesis");
    return;
  }
  if (p->J > 1) {
    KSpan k(p, MS_K_SYNTH);
    ck(launch_synthesis_pass<R>(a, p->ps, -1), "synthesis");
  }
  KSpan k(p, MS_K_SYNTH_L1);
  ck(launch_synthesis_pass<R>(a, p->ps, 1), "synthesis");
}

// B_k+1 = prox(z_k - mu W^H g) from the gradient image g in a.grad (levels 1..J)
template <typename R>
void record_analysis(ms_plan* p, const FistaPass<R>& a, const CUtensorMap* gmap) {
  if (p->dict == MS_DICT_IUWT) {
    KSpan k(p, MS_K_ANALYSIS_L1);
    ck(launch_iuwt_analysis<R>(&a, a.grad, nullptr, (R*)p->wtmp, p->N, p->J, p->ps),
       "IUWT analysis");
    return;
  }
  {
    KSpan k(p, MS_K_ANALYSIS_L1);
    ck(launch_analysis_pass<R>(a, gmap, p->ps, 1), "analysis");
  }
  if (p->J > 1) {
    KSpan k(p, MS_K_ANALYSIS);
    ck(launch_analysis_pass<R>(a, gmap, p->ps, -1), "analysis");
  }
}

// One FISTA iteration (Algorithm 1): synthesis x = W B_k (levels J..1),
// X^_k = F x, the spectral step (objective, iteration control, gradient
// spectrum with the momentum folded in), the inverse FFT to the gradient
// image, and analysis + prox into B_{k+1} (levels 1..J).
template <typename R> void record_fista_pass(ms_plan* p, int parity, const PassView<R>& v) {
  C2<R>* Fk = v.F[parity];
  C2<R>* Fo = v.F[parity ^ 1];
  const FistaPass<R>& a = v.a;
  record_synthesis<R>(p, a);
  if (p->fused_spec) {
    // row transforms, the spectral step with the column transforms fused in,
    // inverse row transforms (whose extra block runs the iteration control)
    const C2<R>* tw = (const C2<R>*)p->twid;
    {
      KSpan k(p, MS_K_FFT_R2C);
      ck(launch_row_r2c<R>(a.x, v.zrow, tw, p->N, a.ctl, p->ps, a.js), "row transforms");
    }
    {
      KSpan k(p, MS_K_SPEC_MUL);
      ck(launch_spec_col<R>(v.zrow, Fk, Fo, v.Ks, v.Bs, tw, p->N, v.parts, a.ctl, a.l1_parts,
                            p->n_l1, p->ps, a.js),
         "spectral step");
    }
    {
      KSpan k(p, MS_K_FFT_C2R);
      ck(launch_row_c2r<R>(v.zrow, (R*)a.grad, tw, p->N, a.ctl, v.parts,
                           spec_col_warps(p->N, sizeof(C2<R>)), v.trace, p->ps, a.js),
         "inverse row transforms");
    }
  } else {
    arg(a.js.jobs == 1, "batched minor cycles need the fused spectral step");
    {
      KSpan k(p, MS_K_FFT_R2C);
      fft_r2c<R>(p, a.x, Fk);
    }
    {
      KSpan k(p, MS_K_SPEC_MUL);
      launch_spec_mul<R>(Fk, Fo, v.Ks, v.Bs, p->N, v.parts, a.ctl, v.trace, p->tickets + 0,
                         a.l1_parts, p->n_l1, p->ps);
    }
    {
      KSpan k(p, MS_K_FFT_C2R);
      fft_c2r<R>(p, Fo, (R*)a.grad);   // gradient image 2 (K W alpha_k - b)
    }
  }
  record_analysis<R>(p, a, v.gmap);
}

// q = P^T-padded x through the 2N x 2N product with H2^ (lq holds the 2N x 2N
// result; P q = H x)
template <typename R> void linear_psf(ms_plan* p, const R* x, const FistaCtl* ctl) {
  KSpan k(p, MS_K_LINEAR_PSF);
  launch_lin_pad<R>(x, (R*)p->lp, p->N, ctl, p->ps);
  exec_r2c<R>(p->r2c2, p->lp, p->ls);
  launch_lin_mul<R>((C2<R>*)p->ls, (const R*)p->lh2, p->N, ctl, p->ps);
  exec_c2r<R>(p->c2r2, p->ls, p->lq);
}

// One FISTA iteration with the linear PSF operator (the pass of
// record_fista_pass with the smooth part evaluated in the image domain; the
// pass parity selects the ring slots of y_k / [D^_k; E^_k] as there).
template <typename R> void record_linear_pass(ms_plan* p, int parity, bool full) {
  const FistaPass<R> a = fista_pass_args<R>(p);
  const int N = p->N;
  const int64_t n2 = (int64_t)N * N;
  record_synthesis<R>(p, a);
  linear_psf<R>(p, (const R*)p->xwork, p->ctl);   // y_k = H x_k
  if (!full) {
    {
      KSpan k(p, MS_K_SPEC_MUL);
      launch_lin_low_step<R>((const R*)p->lq, (const R*)p->lres, (R*)p->ly[parity],
                             (const R*)p->ly[parity ^ 1], (R*)p->lp, N, p->parts, p->ctl,
                             p->trace, p->tickets + 0, p->l1parts, p->n_l1, p->ps);
    }
    KSpan k(p, MS_K_LINEAR_PSF);   // gradient image 2 H r
    exec_r2c<R>(p->r2c2, p->lp, p->ls);
    launch_lin_mul<R>((C2<R>*)p->ls, (const R*)p->lh2, N, p->ctl, p->ps);
    exec_c2r<R>(p->c2r2, p->ls, p->lq);
    launch_lin_crop<R>((const R*)p->lq, nullptr, (R*)p->ywork, N, 2.0, p->ctl, p->ps);
  } else {
    {
      KSpan k(p, MS_K_SPEC_MUL);
      launch_lin_full_diff<R>((const R*)p->lq, (const R*)p->lres, (const R*)p->xwork,
                              (const R*)p->ll, (R*)p->lde, N, p->ctl, p->ps);
      exec_r2c<R>(p->r2cb, p->lde, p->ldes[parity]);
      launch_lin_full_spec<R>((const C2<R>*)p->ldes[parity], (const C2<R>*)p->ldes[parity ^ 1],
                              (const R*)p->gl2, (const R*)p->gh2, (C2<R>*)p->luvs, N, p->parts,
                              p->ctl, p->trace, p->tickets + 0, p->l1parts, p->n_l1, p->ps);
      exec_c2r<R>(p->c2rb, p->luvs, p->luv);   // [u; v] = [G_H^2 D_z; G_L^2 E_z]
    }
    linear_psf<R>(p, (const R*)p->luv, p->ctl);
    KSpan k(p, MS_K_LINEAR_PSF);   // gradient image 2 (H u + v)
    launch_lin_crop<R>((const R*)p->lq, (const R*)p->luv + n2, (R*)p->ywork, N, 2.0, p->ctl,
                       p->ps);
  }
  record_analysis<R>(p, a, p->have_grad_map ? &p->grad_map : nullptr);
}

template <typename R> void record_pass(ms_plan* p, int parity, int step) {
  if (p->conv == MS_CONV_LINEAR)
    record_linear_pass<R>(p, parity, step_full(step));
  else
    record_fista_pass<R>(p, parity, plan_view<R>(p));
}

// the graph of kPasses passes of `step` (one for the circular operator;
// for the linear one, one per problem kind)
template <typename R> cudaGraphExec_t ensure_fista_graph(ms_plan* p, int step) {
  cudaGraphExec_t* exec = p->conv == MS_CONV_LINEAR
                              ? &p->lin_exec[step_full(step) ? 1 : 0]
                              : &p->fista_exec;
  if (*exec) return *exec;
  cudaGraph_t graph;
  ck(cudaStreamBeginCapture(p->ps, cudaStreamCaptureModeThreadLocal), "begin capture");
  p->capturing = true;
  try {
    for (int i = 0; i < kPasses; ++i) record_pass<R>(p, i & 1, step);
  } catch (...) {
    p->capturing = false;
    cudaStreamEndCapture(p->ps, &graph);
    throw;
  }
  p->capturing = false;
  ck(cudaStreamEndCapture(p->ps, &graph), "end capture");
  ck(cudaGraphInstantiate(exec, graph, 0), "graph instantiate");
  cudaGraphDestroy(graph);
  return *exec;
}

void drop_graphs(ms_plan* p) {
  for (cudaGraphExec_t* e : {&p->fista_exec, &p->lin_exec[0], &p->lin_exec[1]})
    if (*e) {
      cudaGraphExecDestroy(*e);
      *e = nullptr;
    }
}

// ------------------------------------------------------------- dictionary
// power iterations of the step size where the closed form does not hold
// (the IUWT dictionary, the linear PSF operator)
constexpr int kPowerIterations = 100;

// x = W alpha and alpha = W^H x with the plan's dictionary (plain calls)
template <typename R> void dict_synthesis(ms_plan* p, const R* alpha, R* x) {
  if (p->dict == MS_DICT_IUWT) {
    ck(launch_iuwt_synthesis<R>(nullptr, alpha, x, (R*)p->wtmp, p->N, p->J, p->ps),
       "IUWT synthesis");
    return;
  }
  set_ptrs_kernel<<<1, 1, 0, p->ps>>>(p->api3_dev, (void*)alpha, (void*)alpha, (void*)alpha);
  launch_synthesis3<R>((const R* const*)p->api3_dev, x, (R*)p->wtmp,
                       WaveletGeom{p->N, p->J, p->M}, nullptr, p->ps);
}
template <typename R> void dict_analysis(ms_plan* p, const R* x, R* alpha) {
  if (p->dict == MS_DICT_IUWT) {
    ck(launch_iuwt_analysis<R>(nullptr, x, alpha, (R*)p->wtmp, p->N, p->J, p->ps),
       "IUWT analysis");
    return;
  }
  launch_analysis<R>(x, alpha, (R*)p->wtmp, WaveletGeom{p->N, p->J, p->M}, p->ps);
}

// The normal operator of the current problem with the linear PSF operator,
// out = H H x (LOW / SINGLE) or H G_H^2 H x + G_L^2 x (FULL), plain launches.
template <typename R> void linear_normal(ms_plan* p, bool full, const R* x, R* out) {
  const int N = p->N;
  const int64_t n2 = (int64_t)N * N;
  linear_psf<R>(p, x, nullptr);
  if (!full) {
    launch_lin_crop<R>((const R*)p->lq, nullptr, (R*)p->luv, N, 1.0, nullptr, p->ps);
    linear_psf<R>(p, (const R*)p->luv, nullptr);
    launch_lin_crop<R>((const R*)p->lq, nullptr, out, N, 1.0, nullptr, p->ps);
    return;
  }
  // [H x; x] -> spectra -> [G_H^2 H x; G_L^2 x] -> images
  launch_lin_crop<R>((const R*)p->lq, nullptr, (R*)p->lde, N, 1.0, nullptr, p->ps);
  ck(cudaMemcpyAsync((R*)p->lde + n2, x, sizeof(R) * n2, cudaMemcpyDeviceToDevice, p->ps),
     "copy");
  exec_r2c<R>(p->r2cb, p->lde, p->ldes[0]);
  launch_lin_full_spec<R>((const C2<R>*)p->ldes[0], nullptr, (const R*)p->gl2, (const R*)p->gh2,
                          (C2<R>*)p->luvs, N, nullptr, nullptr, nullptr, nullptr, nullptr, 0,
                          p->ps);
  exec_c2r<R>(p->c2rb, p->luvs, p->luv);
  linear_psf<R>(p, (const R*)p->luv, nullptr);
  launch_lin_crop<R>((const R*)p->lq, (const R*)p->luv + n2, out, N, 1.0, nullptr, p->ps);
}

// 2 lambda_max(W^H K W) by power iteration (Sect. 3.4) into p->scal[2]
// (device), from the plan's K^ (or, with the linear PSF operator, the
// operator itself for the problem kind `full`): Rayleigh quotient of the
// normalized iterate, reductions in FP64.  Uses B[0], B[1] and the work
// images.
template <typename R> void power_theta(ms_plan* p, int iters, bool full) {
  const int64_t ncoef = (int64_t)p->M * p->N * p->N;
  R* v = (R*)p->B[0];
  R* w = (R*)p->B[1];
  double* sc = p->scal;
  launch_hash_fill<R>(v, ncoef, 12345, p->ps);
  for (int it = 0; it < iters; ++it) {
    launch_dot<R>(v, v, ncoef, p->parts, sc + 0, p->tickets + 7, p->ps);
    launch_normalize<R>(v, ncoef, sc + 0, p->ps);
    dict_synthesis<R>(p, v, (R*)p->xwork);
    if (p->conv == MS_CONV_LINEAR) {
      linear_normal<R>(p, full, (const R*)p->xwork, (R*)p->ywork);
    } else {
      fft_r2c<R>(p, p->xwork, p->spec);
      launch_spec_apply<R>((C2<R>*)p->spec, (const R*)p->Ks, p->N, p->ps);
      fft_c2r<R>(p, p->spec, p->ywork);
    }
    dict_analysis<R>(p, (const R*)p->ywork, w);
    launch_dot<R>(v, w, ncoef, p->parts, sc + 1, p->tickets + 8, p->ps);
    ck(cudaMemcpyAsync(v, w, sizeof(R) * ncoef, cudaMemcpyDeviceToDevice, p->ps), "copy");
  }
  scale_scalar_kernel<<<1, 1, 0, p->ps>>>(sc + 1, 2.0, sc + 2);
}

// Prepare K^, theta (once per step and channel) into the plan buffers.
// step: LOW/SINGLE use the partition PSF only; FULL adds the filters built
// from ctl->sigma2, ctl->eta2.
template <typename R> void build_normal(ms_plan* p, int step, PartDev& pd, double ell,
                                        double delta, FistaCtl* ctl = nullptr,
                                        R* Ks = nullptr) {
  ensure_psf<R>(p, pd);
  if (p->conv == MS_CONV_LINEAR) {
    // the problem's H2^ into the buffer the captured passes read
    ck(cudaMemcpyAsync(p->lh2, pd.Hhat2, sizeof(R) * 2 * p->N * (p->N + 1),
                       cudaMemcpyDeviceToDevice, p->ps),
       "copy");
    const bool full = step_full(step);
    if (full) {
      check_noise_kernel<<<1, 1, 0, p->ps>>>(p->ctl);
      launch_filters<R>(p->N, ell, delta, p->ctl, (R*)p->gl2, (R*)p->gh2, p->ps,
                        step == MS_STEP_FULL_L);
    }
    // the bound (and c0 = 0), then the step size itself: the operator is not
    // circulant, so the closed form is only a bound; power iteration from
    // the fixed start as for the IUWT
    launch_lin_theta<R>((const R*)p->lh2, p->N, full ? (const R*)p->gl2 : nullptr,
                        full ? (const R*)p->gh2 : nullptr, p->M, p->parts, p->ctl,
                        p->tickets + 2, p->ps);
    power_theta<R>(p, kPowerIterations, full);
    set_theta_kernel<<<1, 1, 0, p->ps>>>(p->ctl, p->scal + 2);
    return;
  }
  // (a batched job's own control block and K^ slice, else the plan's)
  FistaCtl* c = ctl ? ctl : p->ctl;
  R* K = Ks ? Ks : (R*)p->Ks;
  if (step_full(step)) {
    check_noise_kernel<<<1, 1, 0, p->ps>>>(c);
    launch_filters<R>(p->N, ell, delta, c, (R*)p->gl2, (R*)p->gh2, p->ps,
                      step == MS_STEP_FULL_L);
    launch_normal_spectrum<R>((const R*)pd.Hhat, (const R*)p->gl2, (const R*)p->gh2, p->N, p->M,
                              K, p->parts, c, p->tickets + 2, p->ps);
  } else {
    launch_normal_spectrum<R>((const R*)pd.Hhat, nullptr, nullptr, p->N, p->M, K, p->parts, c,
                              p->tickets + 2, p->ps);
  }
  if (p->dict == MS_DICT_IUWT) {
    // no closed form (T^H T is not a multiple of I): power iteration
    power_theta<R>(p, kPowerIterations, false);
    set_theta_kernel<<<1, 1, 0, p->ps>>>(p->ctl, p->scal + 2);
  }
}

// b^ and c0 of the circular operator's problem from the residual (and l_low
// for FULL; the filters of build_normal) into Bs and ctl
template <typename R>
void build_b(ms_plan* p, int step, PartDev& pd, const void* residual, const void* l_low,
             FistaCtl* ctl, C2<R>* Bs) {
  fft_r2c<R>(p, residual, p->spec);
  if (step_full(step)) {
    fft_r2c<R>(p, l_low, p->spec2);
    launch_b_spectrum<R>((const C2<R>*)p->spec, (const C2<R>*)p->spec2, (const R*)pd.Hhat,
                         (const R*)p->gl2, (const R*)p->gh2, p->N, Bs, p->parts, ctl,
                         p->tickets + 3, p->ps);
  } else {
    launch_b_spectrum<R>((const C2<R>*)p->spec, nullptr, (const R*)pd.Hhat, nullptr, nullptr,
                         p->N, Bs, p->parts, ctl, p->tickets + 3, p->ps);
  }
}

// b, c0 from the residual (and l_low for FULL), then the FISTA loop.  The
// result coefficients end in B[k % 3], W beta in xwork.
template <typename R>
void run_fista(ms_plan* p, int step, PartDev& pd, const void* residual, const void* l_low,
               const void* beta0, int max_iters, double rel_tol) {
  const int N = p->N;
  const int64_t npix2 = (int64_t)N * N;
  const int64_t ncoef = (int64_t)p->M * npix2;
  const int64_t nspec = (int64_t)N * (N / 2 + 1);
  if (p->conv == MS_CONV_LINEAR) {
    // i~ (and l) into the buffers the captured passes read; y_-1 and the
    // spectra of pass -1 zero (their weight t_0 is zero, but must be finite)
    ck(cudaMemcpyAsync(p->lres, residual, sizeof(R) * npix2, cudaMemcpyDeviceToDevice, p->ps),
       "copy");
    if (step_full(step)) {
      ck(cudaMemcpyAsync(p->ll, l_low, sizeof(R) * npix2, cudaMemcpyDeviceToDevice, p->ps),
         "copy");
      ck(cudaMemsetAsync(p->ldes[1], 0, sizeof(C2<R>) * 2 * nspec, p->ps), "memset");
    } else {
      ck(cudaMemsetAsync(p->ly[1], 0, sizeof(R) * npix2, p->ps), "memset");
    }
  } else {
    build_b<R>(p, step, pd, residual, l_low, p->ctl, (C2<R>*)p->Bs);
  }
  // B[0] = start, B[2] = B[0] and X^_{-1} = 0 (their weight is zero for k < 2)
  ck(cudaMemsetAsync(p->F[1], 0, sizeof(C2<R>) * nspec, p->ps), "memset");
  if (beta0)
    ck(cudaMemcpyAsync(p->B[0], beta0, sizeof(R) * ncoef, cudaMemcpyDeviceToDevice, p->ps),
       "copy");
  else
    ck(cudaMemsetAsync(p->B[0], 0, sizeof(R) * ncoef, p->ps), "memset");
  ck(cudaMemcpyAsync(p->B[2], p->B[0], sizeof(R) * ncoef, cudaMemcpyDeviceToDevice, p->ps),
     "copy");
  set_target_kernel<<<1, 1, 0, p->ps>>>(p->ctl, p->obj_target);
  // the coarse levels' group barriers start at rest (a wait that ran out
  // may have left a count behind)
  ck(cudaMemsetAsync(p->coarse_bar, 0, sizeof(int) * 2 * kMaxBases, p->ps), "memset");
  const bool poll = rel_tol > 0 || std::isfinite(p->obj_target);
  // ||B_0||_1 enters the first objective through the analysis partials
  ck(cudaMemsetAsync(p->l1parts, 0, sizeof(double) * p->n_l1, p->ps), "memset");
  launch_l1<R>((const R*)p->B[0], ncoef, p->parts, p->l1parts, p->tickets + 4, p->ps);
  // max_iters prox steps plus one pass that only evaluates F at the result
  const int passes = max_iters + 1;
  if (p->prof) {   // direct launches, each kernel family bracketed by events
    for (int i = 0; i < passes; ++i) {
      record_pass<R>(p, i & 1, step);
      if ((i + 1) % kPasses == 0 && p->pending.size() > 4096) harvest(p);
      if (poll && (i + 1) % (4 * kPasses) == 0 && i + 1 < passes) {
        int32_t done = 0;
        ck(cudaMemcpyAsync(&done, &p->ctl->done, sizeof(done), cudaMemcpyDeviceToHost, p->ps),
           "read done");
        ck(cudaStreamSynchronize(p->ps), "synchronize");
        if (done) break;
      }
    }
    return;
  }
  cudaGraphExec_t exec = ensure_fista_graph<R>(p, step);
  int launched = 0;
  while (launched < passes) {
    ck(cudaGraphLaunch(exec, p->ps), "graph launch");
    launched += kPasses;
    if (poll && launched < passes && (launched / kPasses) % 4 == 0) {
      int32_t done = 0;
      ck(cudaMemcpyAsync(&done, &p->ctl->done, sizeof(done), cudaMemcpyDeviceToHost, p->ps),
         "read done");
      ck(cudaStreamSynchronize(p->ps), "synchronize");
      if (done) break;
    }
  }
}

template <typename R> void fill_stats(ms_plan* p, ms_stats* st, bool copy_trace) {
  FistaCtl h{};
  ck(cudaMemcpyAsync(&h, p->ctl, sizeof(h), cudaMemcpyDeviceToHost, p->ps), "read ctl");
  ck(cudaStreamSynchronize(p->ps), "synchronize");
  if (h.error) throw Fail{(ms_status)h.error, "non-finite objective or invalid noise levels"};
  if (copy_trace) {
    p->htrace.assign(h.k + 1, 0.0);
    ck(cudaMemcpy(p->htrace.data(), p->trace, sizeof(double) * (h.k + 1),
                  cudaMemcpyDeviceToHost),
       "read trace");
  }
  if (st) {
    st->iterations = h.k;
    st->converged = h.converged;
    st->objective = h.F_cur;
    st->lambda = h.lam;
    st->theta = h.theta;
    st->sigma2 = h.sigma2;
    st->eta2 = h.eta2;
    st->objective_trace = p->htrace.data();
  }
}

int step_part(int step) {
  switch (step) {
    case MS_STEP_LOW: case MS_STEP_FULL_L: return MS_PART_L;
    case MS_STEP_FULL: case MS_STEP_LOW_H: return MS_PART_H;
    default: return MS_PART_ALL;
  }
}

// ------------------------------------------------------- learned warm start
// beta = W^H x0 / M with x0 = s net([i^_L, i~_H1] / s), s = max|i~_H1|
// (Sect. 3.3's problem, started from the network's image)
template <typename R>
void warm_start_beta(ms_plan* p, ms_unet* net, const void* low, const void* res, void* beta,
                     void* x0_out) {
  arg(net != nullptr, "warm start network is NULL");
  arg(p->dict == MS_DICT_DAUBECHIES,
      "the warm start's coefficients W^H x0 / M need the Daubechies dictionary (W W^H = M I)");
  arg(ms_unet_device_of(net) == p->dev, "the warm start network lives on another device");
  const int N = p->N;
  const int64_t n2 = (int64_t)N * N;
  if (!p->ws_in) {
    p->ws_in = p->alloc<float>(2 * n2, "warm start input");
    p->ws_out = p->alloc<float>(n2, "warm start output");
  }
  R* x0 = (R*)x0_out;
  if (!x0) {
    if (!p->ws_x0) p->ws_x0 = p->alloc<R>(n2, "warm start image");
    x0 = (R*)p->ws_x0;
  }
  launch_image_norms<R>((const R*)res, n2, p->parts, p->ctl, p->tickets + 5, p->ps);
  const int nb = (int)std::min<int64_t>((n2 + 255) / 256, (int64_t)sm_count() * 8);
  ws_input_kernel<R><<<nb, 256, 0, p->ps>>>((const R*)low, (const R*)res, p->ctl, n2, p->ws_in);
  const ms_status st = ms_unet_forward(net, p->ws_in, N, N, p->ws_out, p->ps);
  if (st != MS_OK)
    throw Fail{st, std::string("warm start network: ") + ms_unet_last_error(net)};
  ws_output_kernel<R><<<nb, 256, 0, p->ps>>>(p->ws_out, p->ctl, n2, x0);
  WaveletGeom g{p->N, p->J, p->M};
  launch_analysis<R>(x0, (R*)beta, (R*)p->wtmp, g, p->ps);
  launch_axpby<R>((const R*)beta, nullptr, (R*)beta, 1.0 / p->M, 0.0, (int64_t)p->M * n2,
                  p->ps);
  ck(cudaGetLastError(), "warm start kernels");
}

// ------------------------------------------------------------- reconstruct
// One step of the method on the partition of `step` (Sects. 3.2, 3.3): N_major
// major cycles, each a residual image, a lambda, a minor cycle, a model update.
// obs_sorted: the partition's visibilities in plan order (vis_a).
template <typename R>
void run_step(ms_plan* p, int step, int chan, const ms_recon_opts& o, const void* low_image,
              void* image_out, void* model_out, ms_stats* st, Timer& tm) {
  PartDev& pd = p->ch[chan].part[step_part(step)];
  const int N = p->N;
  const int64_t n2 = (int64_t)N * N;
  R* model = (R*)(model_out ? model_out : p->img[0]);
  R* res = (R*)p->img[1];
  R* l = (R*)p->img[2];
  ck(cudaMemsetAsync(model, 0, sizeof(R) * n2, p->ps), "memset");
  const double coef = step == MS_STEP_LOW ? o.lambda_low
                      : step == MS_STEP_FULL ? o.lambda_full : o.lambda_single;
  for (int n = 1; n <= o.n_major; ++n) {
    residual_sorted<R>(p, pd, p->vis_a, model, res, &tm);
    launch_image_norms<R>(res, n2, p->parts, p->ctl, p->tickets + 5, p->ps);
    if (n == 1) {
      init_ctl_kernel<<<1, 1, 0, p->ps>>>(p->ctl, o.fista_iters, o.rel_tol, 0.0, 0,
                                          o.sigma2, o.sigma2 > 0 && o.eta2 > 0 ? o.eta2
                                                                               : 1e-3 * o.sigma2,
                                          o.sigma2 > 0 ? 1 : 0);
      if (step == MS_STEP_FULL && !(o.sigma2 > 0)) {
        // sigma^2 estimated on i~_H1, eta^2 = 1e-3 sigma^2 unless given (Sect. 4.3)
        launch_sigma2_hat<R>(res, N, p->parts, p->ctl, p->tickets + 6, o.eta2 > 0 ? 0 : 1, p->ps);
        if (o.eta2 > 0) set_eta_kernel<<<1, 1, 0, p->ps>>>(p->ctl, o.eta2);
      }
      build_normal<R>(p, step, pd, p->d.ell_px, p->d.delta_px);
    }
    init_ctl_kernel<<<1, 1, 0, p->ps>>>(p->ctl, o.fista_iters, o.rel_tol, 0.0, 0, 0, 0, 0);
    launch_set_lambda(p->ctl, o.lambda_rule, coef, n, n == 1 ? 1 : 0, p->ps);
    if (step == MS_STEP_FULL)
      launch_axpby<R>((const R*)low_image, model, l, 1.0, -1.0, n2, p->ps);   // l = i^_L - sum i_j
    const void* beta0 = nullptr;
    if (step == MS_STEP_FULL && n == 1 && o.warm_start) {
      // the learned warm start: step two's first minor cycle starts from the
      // network's image of [i^_L, i~_H1]
      if (!p->ws_beta) p->ws_beta = p->alloc<R>((size_t)p->M * n2, "warm start coefficients");
      // (its norms of i~_H1 leave lambda, already set from them, unchanged)
      warm_start_beta<R>(p, o.warm_start, low_image, res, p->ws_beta, nullptr);
      beta0 = p->ws_beta;
    }
    int a = tm.mark();
    run_fista<R>(p, step, pd, res, step == MS_STEP_FULL ? l : nullptr, beta0, o.fista_iters,
                 o.rel_tol);
    tm.spans[2].push_back({a, tm.mark()});
    launch_axpby<R>(model, (const R*)p->xwork, model, 1.0, 1.0, n2, p->ps);   // i^ += W beta
    FistaCtl h{};
    ck(cudaMemcpyAsync(&h, p->ctl, sizeof(h), cudaMemcpyDeviceToHost, p->ps), "read ctl");
    ck(cudaStreamSynchronize(p->ps), "synchronize");
    if (h.error) throw Fail{(ms_status)h.error, "non-finite objective or invalid noise levels"};
    if (st) {
      st->total_iterations += h.k;
      st->gridded_vis += pd.n;
    }
  }
  residual_sorted<R>(p, pd, p->vis_a, model, res, &tm);   // i~_{N+1}
  if (st) st->gridded_vis += pd.n;
  launch_axpby<R>(res, model, (R*)image_out, 1.0, 1.0, n2, p->ps);
  fill_stats<R>(p, st, true);
  if (st) st->major_cycles += o.n_major;
}

void validate_opts(const ms_recon_opts* o) {
  arg(o != nullptr, "options must not be NULL");
  arg(o->n_major >= 1 && o->n_major <= 1000, "n_major must be 1..1000");
  arg(o->fista_iters >= 1 && o->fista_iters <= 1000000, "fista_iters must be 1..1e6");
  arg(o->lambda_rule == MS_LAMBDA_NORM2_2N || o->lambda_rule == MS_LAMBDA_MAX_FIXED,
      "unknown lambda rule");
  arg(o->rel_tol >= 0, "rel_tol must be >= 0");
}

void ensure_trace(ms_plan* p, int iters) {
  if (iters + 2 <= p->trace_cap) return;
  if (p->trace) {
    cudaFree(p->trace);
    auto it = std::find(p->allocs.begin(), p->allocs.end(), (void*)p->trace);
    if (it != p->allocs.end()) p->allocs.erase(it);
  }
  p->trace_cap = std::max(iters + 2, 1024);
  p->trace = p->alloc<double>(p->trace_cap, "trace");
  drop_graphs(p);   // the captured passes point at the old trace
}

template <typename R>
void two_step(ms_plan* p, int chan, const void* vis, const ms_recon_opts* o, void* low_out,
              void* img_out, void* model_out, ms_stats* st, void* stream) {
  Scope sc(p, stream);
  Timer tm(p);
  ensure_trace(p, o->fista_iters);
  if (st) std::memset(st, 0, sizeof(*st));
  int t0 = tm.mark();
  ChanDev& c = p->ch[chan];
  // step one on V_L
  PartDev& pl = c.part[MS_PART_L];
  launch_gather_vis<R>(pl.idx, pl.n, (const C2<R>*)vis, (C2<R>*)p->vis_a, p->ps);
  run_step<R>(p, MS_STEP_LOW, chan, *o, nullptr, low_out, nullptr, st, tm);
  // step two on V_H with i^_L
  PartDev& ph = c.part[MS_PART_H];
  launch_gather_vis<R>(ph.idx, ph.n, (const C2<R>*)vis, (C2<R>*)p->vis_a, p->ps);
  run_step<R>(p, MS_STEP_FULL, chan, *o, low_out, img_out, model_out, st, tm);
  int t1 = tm.mark();
  check_device_error(p);
  if (st) {
    float ms = 0;
    ck(cudaEventElapsedTime(&ms, p->tev[t0], p->tev[t1]), "event time");
    st->elapsed_ms = ms;
    st->grid_ms = tm.total(0);
    st->fft_ms = tm.total(1);
    st->minor_ms = tm.total(2);
  }
  sc.finish();
}

// ms_reconstruct_step: one step of the method on this plan's partition
template <typename R>
void one_step(ms_plan* p, int step, int chan, const void* vis, const ms_recon_opts* o,
              const void* low_image, void* img_out, void* model_out, ms_stats* st,
              void* stream) {
  Scope sc(p, stream);
  Timer tm(p);
  ensure_trace(p, o->fista_iters);
  if (st) std::memset(st, 0, sizeof(*st));
  int t0 = tm.mark();
  PartDev& pd = p->ch[chan].part[step_part(step)];
  launch_gather_vis<R>(pd.idx, pd.n, (const C2<R>*)vis, (C2<R>*)p->vis_a, p->ps);
  run_step<R>(p, step, chan, *o, low_image, img_out, model_out, st, tm);
  int t1 = tm.mark();
  check_device_error(p);
  if (st) {
    float ms = 0;
    ck(cudaEventElapsedTime(&ms, p->tev[t0], p->tev[t1]), "event time");
    st->elapsed_ms = ms;
    st->grid_ms = tm.total(0);
    st->fft_ms = tm.total(1);
    st->minor_ms = tm.total(2);
  }
  sc.finish();
}

template <typename R>
void single_step(ms_plan* p, int chan, const void* vis, const ms_recon_opts* o, void* img_out,
                 void* model_out, ms_stats* st, void* stream) {
  Scope sc(p, stream);
  Timer tm(p);
  ensure_trace(p, o->fista_iters);
  if (st) std::memset(st, 0, sizeof(*st));
  int t0 = tm.mark();
  PartDev& pa = p->ch[chan].part[MS_PART_ALL];
  launch_gather_vis<R>(pa.idx, pa.n, (const C2<R>*)vis, (C2<R>*)p->vis_a, p->ps);
  run_step<R>(p, MS_STEP_SINGLE, chan, *o, nullptr, img_out, model_out, st, tm);
  int t1 = tm.mark();
  check_device_error(p);
  if (st) {
    float ms = 0;
    ck(cudaEventElapsedTime(&ms, p->tev[t0], p->tev[t1]), "event time");
    st->elapsed_ms = ms;
    st->grid_ms = tm.total(0);
    st->fft_ms = tm.total(1);
    st->minor_ms = tm.total(2);
  }
  sc.finish();
}

// ------------------------------------------------------------- plan build
template <typename R> void build_plan(ms_plan* p, const ms_plan_desc* d) {
  const int N = p->N, Ng = p->Ng;
  const int64_t nvis = d->nvis;
  cudaStream_t s = p->ps;
  // Daubechies filters: the device's table holds db1..db8 whatever this
  // plan's M, so that plans of different M (and the temporary plans of the
  // linear PSF operator) leave it the same for each other
  {
    std::vector<double> h(kMaxBases * kMaxTaps, 0.0);
    std::vector<int> len(kMaxBases, 0);
    for (int m = 0; m < kMaxBases; ++m) {
      std::vector<double> f = daubechies(m + 1);
      len[m] = (int)f.size();
      for (size_t k = 0; k < f.size(); ++k) h[m * kMaxTaps + k] = f[k];
    }
    set_wavelet_filters(h.data(), len.data(), kMaxBases);
    ck(cudaGetLastError(), "wavelet filters");
  }
  // deapodization table
  {
    std::vector<double> x, w;
    gauss_legendre(96, x, w);
    double* dx = dalloc<double>(x.size(), "gl");
    double* dw = dalloc<double>(w.size(), "gl");
    double* psi = dalloc<double>(N, "psi");
    ck(cudaMemcpy(dx, x.data(), sizeof(double) * x.size(), cudaMemcpyHostToDevice), "copy");
    ck(cudaMemcpy(dw, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice), "copy");
    launch_deapodization(N, Ng, p->beta, dx, dw, (int)x.size(), psi, s);
    std::vector<double> hp(N);
    ck(cudaMemcpyAsync(hp.data(), psi, sizeof(double) * N, cudaMemcpyDeviceToHost, s), "copy");
    ck(cudaStreamSynchronize(s), "deapodization");
    std::vector<R> hr(hp.begin(), hp.end());
    p->psi = p->alloc<R>(N, "psi");
    ck(cudaMemcpy(p->psi, hr.data(), sizeof(R) * N, cudaMemcpyHostToDevice), "copy");
    cudaFree(dx);
    cudaFree(dw);
    cudaFree(psi);
  }
  // per channel: classify, sort, work items
  double* du = dalloc<double>(nvis, "u");
  double* dv = dalloc<double>(nvis, "v");
  uint8_t* dfl = d->flags ? dalloc<uint8_t>(nvis, "flags") : nullptr;
  uint32_t* cell_all = dalloc<uint32_t>(nvis, "cell");
  double2* frac_all = dalloc<double2>(nvis, "frac");
  uint32_t* tile_id = dalloc<uint32_t>(nvis, "tile");
  uint8_t* member = dalloc<uint8_t>(nvis, "member");
  uint32_t* keys = dalloc<uint32_t>(nvis, "keys");
  int32_t* vals = dalloc<int32_t>(nvis, "vals");
  uint32_t* ktmp = dalloc<uint32_t>(nvis, "keys");
  int32_t* vtmp = dalloc<int32_t>(nvis, "vals");
  int64_t hcap = radix_hist_size(nvis);
  int32_t* hist = dalloc<int32_t>(hcap, "hist");
  int32_t* counts = dalloc<int32_t>(p->ntiles + 1, "counts");
  int32_t* tstart = dalloc<int32_t>(p->ntiles + 2, "tstart");
  int32_t* nch = dalloc<int32_t>(p->ntiles + 1, "nchunks");
  // sort key: tile, then the anchor cell inside the tile (2 log2 T bits)
  int lg_t = 0;
  while ((1 << lg_t) < p->T) ++lg_t;
  int bits = 0;
  while ((1u << bits) <= (unsigned)p->ntiles) ++bits;
  bits = ((bits + 2 * lg_t + 7) / 8) * 8;
  const uint32_t sentinel = (uint32_t)p->ntiles << (2 * lg_t);
  const uint8_t masks[3] = {4 | 1, 4 | 2, 4};
  p->ch.resize(d->nchan);
  for (int c = 0; c < d->nchan; ++c) {
    ck(cudaMemcpy(du, d->u + (int64_t)c * nvis, sizeof(double) * nvis, cudaMemcpyHostToDevice),
       "copy u");
    ck(cudaMemcpy(dv, d->v + (int64_t)c * nvis, sizeof(double) * nvis, cudaMemcpyHostToDevice),
       "copy v");
    if (dfl)
      ck(cudaMemcpy(dfl, d->flags + (int64_t)c * nvis, nvis, cudaMemcpyHostToDevice),
         "copy flags");
    launch_classify(du, dv, dfl, nvis, Ng, N, d->pixel_size, d->ell_px, d->delta_px, p->T,
                    p->ntx, cell_all, frac_all, tile_id, member, s);
    for (int pt = 0; pt < 3; ++pt) {
      PartDev& pd = p->ch[c].part[pt];
      launch_make_keys(tile_id, cell_all, member, nvis, masks[pt], lg_t, sentinel, keys, vals, s);
      uint32_t* k = keys;
      int32_t* v = vals;
      radix_sort(&k, &v, ktmp, vtmp, nvis, bits, hist, hcap, s);
      ck(cudaMemsetAsync(counts, 0, sizeof(int32_t) * (p->ntiles + 1), s), "memset");
      launch_count_tiles(k, nvis, 2 * lg_t, counts, s);
      int32_t excluded = 0;
      ck(cudaMemcpyAsync(&excluded, counts + p->ntiles, sizeof(int32_t), cudaMemcpyDeviceToHost,
                         s),
         "copy");
      ck(cudaStreamSynchronize(s), "sort");
      pd.n = nvis - excluded;
      launch_exclusive_scan(counts, tstart, p->ntiles, s);
      launch_chunks_per_tile(counts, p->ntiles, p->chunk, nch, s);
      pd.tile_items = p->alloc<int32_t>(p->ntiles + 1, "tile items");
      launch_exclusive_scan(nch, pd.tile_items, p->ntiles, s);
      int32_t nitems = 0;
      ck(cudaMemcpyAsync(&nitems, pd.tile_items + p->ntiles, sizeof(int32_t),
                         cudaMemcpyDeviceToHost, s),
         "copy");
      ck(cudaStreamSynchronize(s), "items");
      pd.nitems = nitems;
      pd.items = p->alloc<WorkItem>(std::max(nitems, 1), "items");
      launch_make_items(counts, tstart, pd.tile_items, p->ntiles, p->chunk, pd.items, s);
      pd.idx = p->alloc<int32_t>(std::max<int64_t>(pd.n, 1), "idx");
      ck(cudaMemcpyAsync(pd.idx, v, sizeof(int32_t) * pd.n, cudaMemcpyDeviceToDevice, s), "copy");
      pd.cell = p->alloc<uint32_t>(std::max<int64_t>(pd.n, 1), "cell");
      pd.frac = p->alloc<C2<R>>(std::max<int64_t>(pd.n, 1), "frac");
      launch_gather_geometry<R>(pd.idx, pd.n, cell_all, frac_all, pd.cell, (C2<R>*)pd.frac, s);
      pd.Hhat = p->alloc<R>((size_t)N * (N / 2 + 1), "Hhat");
      p->max_items = std::max(p->max_items, pd.nitems);
      p->max_n = std::max(p->max_n, pd.n);
      p->ch[c].counts[pt == 2 ? 3 : pt] = pd.n;
    }
    ChanDev& cd = p->ch[c];
    cd.counts[2] = cd.counts[0] + cd.counts[1] - cd.counts[3];
  }
  ck(cudaStreamSynchronize(s), "plan");
  for (void* q : {(void*)du, (void*)dv, (void*)dfl, (void*)cell_all, (void*)frac_all,
                  (void*)tile_id, (void*)member, (void*)keys, (void*)vals, (void*)ktmp,
                  (void*)vtmp, (void*)hist, (void*)counts, (void*)tstart, (void*)nch})
    if (q) cudaFree(q);
  // workspaces
  const int64_t n2 = (int64_t)N * N;
  const int64_t nspec = (int64_t)N * (N / 2 + 1);
  const int64_t ncoef = (int64_t)p->M * n2;
  p->grid = p->alloc<C2<R>>((size_t)Ng * Ng, "grid");
  p->scratch = p->alloc<unsigned char>(
      (size_t)std::max(p->max_items, 1) * p->S * p->S * grid_scratch_cell_bytes(p->prec),
      "scratch");
  p->vis_a = p->alloc<C2<R>>(std::max<int64_t>(p->max_n, 1), "vis");
  p->vis_b = p->alloc<C2<R>>(std::max<int64_t>(p->max_n, 1), "vis");
  for (auto& im : p->img) im = p->alloc<R>(n2, "image");
  for (auto& b : p->B) b = p->alloc<R>(ncoef, "coefficients");
  p->xwork = p->alloc<R>(n2, "image");
  p->ywork = p->alloc<R>(n2, "image");
  for (auto& f : p->F) f = p->alloc<C2<R>>(nspec, "spectrum");
  p->spec = p->alloc<C2<R>>(nspec, "spectrum");
  p->spec2 = p->alloc<C2<R>>(nspec, "spectrum");
  p->Bs = p->alloc<C2<R>>(nspec, "spectrum");
  p->Ks = p->alloc<R>(nspec, "spectrum");
  p->gl2 = p->alloc<R>(nspec, "filter");
  p->gh2 = p->alloc<R>(nspec, "filter");
  // two LL buffers of M (N/2)^2 (Daubechies), or three work images (IUWT)
  p->wtmp = p->alloc<R>(std::max<int64_t>(ncoef, 3 * n2), "wavelet tmp");
  p->api3_dev = p->alloc<void*>(3, "ptrs");
  p->ctl = p->alloc<FistaCtl>(1, "ctl");
  p->parts = p->alloc<double>(std::max(4096, 3 * spec_col_warps(N, sizeof(C2<R>))), "partials");
  if (p->dict == MS_DICT_IUWT) {
    p->n_l1 = iuwt_prox_partials(p->J);
  } else {
    p->n_l1 = analysis_prox_partials(WaveletGeom{N, p->J, p->M});
    p->coarse_ctas =
        coarse_groups(WaveletGeom{N, p->J, p->M}, sizeof(R), &p->coarse_gr, &p->coarse_budget);
  }
  p->coarse_bar = p->alloc<int>(2 * kMaxBases, "coarse barrier");
  ck(cudaMemset(p->coarse_bar, 0, sizeof(int) * 2 * kMaxBases), "memset");
  p->l1parts = p->alloc<double>(p->n_l1, "partials");
  p->tickets = p->alloc<int32_t>(16, "tickets");
  p->scal = p->alloc<double>(16, "scalars");
  p->err = p->alloc<int32_t>(1, "error flag");
  ensure_trace(p, 1024);
  ck(cudaMemset(p->tickets, 0, sizeof(int32_t) * 16), "memset");
  ck(cudaMemset(p->err, 0, sizeof(int32_t)), "memset");
  ck(cudaMemset(p->ctl, 0, sizeof(FistaCtl)), "memset");
  // cuFFT plans
  cufftType tc = sizeof(R) == 8 ? CUFFT_Z2Z : CUFFT_C2C;
  cufftType tr = sizeof(R) == 8 ? CUFFT_D2Z : CUFFT_R2C;
  cufftType ti = sizeof(R) == 8 ? CUFFT_Z2D : CUFFT_C2R;
  ckf(cufftPlan2d(&p->c2c, Ng, Ng, tc), "plan C2C");
  ckf(cufftPlan2d(&p->r2c, N, N, tr), "plan R2C");
  ckf(cufftPlan2d(&p->c2r, N, N, ti), "plan C2R");
  for (cufftHandle h : {p->c2c, p->r2c, p->c2r}) ckf(cufftSetStream(h, s), "set stream");
  if (p->conv == MS_CONV_LINEAR) {
    const int64_t n4 = 4 * n2, s2 = (int64_t)2 * N * (N + 1);
    p->lp = p->alloc<R>(n4, "linear pad");
    p->lq = p->alloc<R>(n4, "linear product");
    p->ls = p->alloc<C2<R>>(s2, "linear spectrum");
    p->lh2 = p->alloc<R>(s2, "linear PSF spectrum");
    p->lres = p->alloc<R>(n2, "image");
    p->ll = p->alloc<R>(n2, "image");
    for (auto& y : p->ly) y = p->alloc<R>(n2, "image");
    p->lde = p->alloc<R>(2 * n2, "image");
    for (auto& q : p->ldes) q = p->alloc<C2<R>>(2 * nspec, "spectrum");
    p->luvs = p->alloc<C2<R>>(2 * nspec, "spectrum");
    p->luv = p->alloc<R>(2 * n2, "image");
    ckf(cufftPlan2d(&p->r2c2, 2 * N, 2 * N, tr), "plan R2C 2N");
    ckf(cufftPlan2d(&p->c2r2, 2 * N, 2 * N, ti), "plan C2R 2N");
    int nn[2] = {N, N};   // two stacked N x N transforms, contiguous
    ckf(cufftPlanMany(&p->r2cb, 2, nn, nullptr, 1, 0, nullptr, 1, 0, tr, 2), "plan R2C x2");
    ckf(cufftPlanMany(&p->c2rb, 2, nn, nullptr, 1, 0, nullptr, 1, 0, ti, 2), "plan C2R x2");
    for (cufftHandle h : {p->r2c2, p->c2r2, p->r2cb, p->c2rb})
      ckf(cufftSetStream(h, s), "set stream");
  }
  {
    int dev_smem = 0;
    ck(cudaDeviceGetAttribute(&dev_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->dev),
       "device attribute");
    // The fused step: shared-memory row transforms and Stockham column
    // transforms fused with the spectral step.  Measured at N = 1024 on
    // GB300 it beats the 2-D cuFFT transforms around spec_mul_kernel in both
    // precisions.
    p->fused_spec = (sizeof(R) == 8 || MS_FUSED_SPEC_FP32) && N >= 16 && N <= 8192 &&
                    (N & (N - 1)) == 0 && spec_col_smem(N, sizeof(C2<R>)) <= (size_t)dev_smem &&
                    row_fft_smem(N, sizeof(C2<R>)) <= (size_t)dev_smem;
  }
  if (p->fused_spec) {
    p->zrow = p->alloc<C2<R>>((size_t)N * (N / 2 + 1), "row spectra");
    // twiddles exp(-2 pi i m / N), m < N, in FP64 on the host
    std::vector<C2<R>> tw(N);
    for (int m = 0; m < N; ++m) {
      const double ang = -2.0 * M_PI * (double)m / (double)N;
      tw[m].x = (R)std::cos(ang);
      tw[m].y = (R)std::sin(ang);
    }
    p->twid = p->alloc<C2<R>>(N, "twiddles");
    ck(cudaMemcpy(p->twid, tw.data(), sizeof(C2<R>) * N, cudaMemcpyHostToDevice), "twiddles");
  }
  // TMA descriptor of the grid: {2 Ng scalars, Ng rows}, box {2 S, S}
  {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    ck(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                        &q),
       "driver entry point");
    arg(fn != nullptr && q == cudaDriverEntryPointSuccess, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)2 * Ng, (cuuint64_t)Ng};
    cuuint64_t strides[1] = {(cuuint64_t)2 * Ng * sizeof(R)};
    cuuint32_t box[2] = {(cuuint32_t)(2 * p->S), (cuuint32_t)p->S};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = ((EncodeTiledFn)fn)(
        &p->tmap, sizeof(R) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
        2, p->grid, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Fail{MS_ERR_CUDA, "cuTensorMapEncodeTiled failed"};
    // gradient image of the minor cycle: {N, N}, box = the analysis input
    // window {80, 78}; only images at least one window wide use it
    unsigned bc = 0, br = 0;
    analysis_window_box(&bc, &br);
    if ((unsigned)N >= bc) {
      cuuint64_t gd[2] = {(cuuint64_t)N, (cuuint64_t)N};
      cuuint64_t gs[1] = {(cuuint64_t)N * sizeof(R)};
      cuuint32_t gb[2] = {bc, br};
      r = ((EncodeTiledFn)fn)(
          &p->grad_map,
          sizeof(R) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
          p->ywork, gd, gs, gb, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) throw Fail{MS_ERR_CUDA, "cuTensorMapEncodeTiled failed (gradient)"};
      p->have_grad_map = true;
    }
  }
  ck(cudaStreamSynchronize(s), "plan");
  ck(cudaGetLastError(), "plan kernels");
}

template <typename R>
void lipschitz(ms_plan* p, int step, int chan, double sigma2, double eta2, int power_iters,
               double* closed, double* power) {
  PartDev& pd = part_of(p, step_part(step), chan);
  init_ctl_kernel<<<1, 1, 0, p->ps>>>(p->ctl, 1, 0.0, 0.0, 0, sigma2, eta2, 1);
  build_normal<R>(p, step, pd, p->d.ell_px, p->d.delta_px);
  FistaCtl h{};
  ck(cudaMemcpyAsync(&h, p->ctl, sizeof(h), cudaMemcpyDeviceToHost, p->ps), "read ctl");
  ck(cudaStreamSynchronize(p->ps), "synchronize");
  if (h.error) throw Fail{MS_ERR_NUMERIC, "invalid noise levels"};
  if (closed) *closed = h.theta;
  if (power) *power = 0.0;
  if (power_iters <= 0) return;
  power_theta<R>(p, power_iters, step_full(step));
  double* sc = p->scal;
  double rho = 0;
  ck(cudaMemcpyAsync(&rho, sc + 1, sizeof(double), cudaMemcpyDeviceToHost, p->ps), "copy");
  ck(cudaStreamSynchronize(p->ps), "synchronize");
  if (power) *power = 2.0 * rho;
}

template <typename R>
void minor_cycle(ms_plan* p, int step, int chan, const void* residual, const void* l_low,
                 double sigma2, double eta2, double lambda, int max_iters, double rel_tol,
                 void* beta_inout, void* model_out, ms_stats* st) {
  PartDev& pd = part_of(p, step_part(step), chan);
  arg(residual != nullptr && model_out != nullptr, "residual and model_out are required");
  arg(!step_full(step) || l_low != nullptr, "FULL needs l_low");
  arg(max_iters >= 1 && max_iters <= 1000000, "max_iters must be 1..1e6");
  arg(lambda >= 0 && std::isfinite(lambda), "lambda must be finite and >= 0");
  ensure_trace(p, max_iters);
  init_ctl_kernel<<<1, 1, 0, p->ps>>>(p->ctl, max_iters, rel_tol, lambda, 1, sigma2, eta2,
                                      step_full(step) ? 1 : 0);
  build_normal<R>(p, step, pd, p->d.ell_px, p->d.delta_px);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ck(cudaEventCreate(&e0), "event");
  ck(cudaEventCreate(&e1), "event");
  ck(cudaEventRecord(e0, p->ps), "event");
  run_fista<R>(p, step, pd, residual, l_low, beta_inout, max_iters, rel_tol);
  ck(cudaEventRecord(e1, p->ps), "event");
  const int64_t n2 = (int64_t)p->N * p->N;
  ck(cudaMemcpyAsync(model_out, p->xwork, sizeof(R) * n2, cudaMemcpyDeviceToDevice, p->ps),
     "copy");
  fill_stats<R>(p, st, true);
  if (beta_inout) {
    int k = st ? st->iterations : 0;
    if (!st) {
      FistaCtl h{};
      ck(cudaMemcpy(&h, p->ctl, sizeof(h), cudaMemcpyDeviceToHost), "read ctl");
      k = h.k;
    }
    ck(cudaMemcpyAsync(beta_inout, p->B[k % 3], sizeof(R) * p->M * n2, cudaMemcpyDeviceToDevice,
                       p->ps),
       "copy");
  }
  ck(cudaStreamSynchronize(p->ps), "synchronize");
  if (st) {
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    st->elapsed_ms = ms;
    st->minor_ms = ms;
    st->total_iterations = st->iterations;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
}

void destroy(ms_plan* p) {
  if (!p) return;
  DeviceGuard guard;
  cudaSetDevice(p->dev);
  drop_graphs(p);
  p->fb.release();
  for (cufftHandle h : {p->c2c, p->r2c, p->c2r, p->r2c2, p->c2r2, p->r2cb, p->c2rb})
    if (h) cufftDestroy(h);
  for (void* a : p->allocs) cudaFree(a);
  if (p->batch.fft) cufftDestroy(p->batch.fft);
  for (void* a : {p->batch.jobs, (void*)p->batch.job_of, p->batch.grids, p->batch.scratch,
                  p->batch.rows_a, p->batch.rows_b})
    if (a) cudaFree(a);
  for (auto e : p->tev) cudaEventDestroy(e);
  for (auto e : p->evpool) cudaEventDestroy(e);
  for (auto& sp : p->pending) {
    cudaEventDestroy(sp.a);
    cudaEventDestroy(sp.b);
  }
  if (p->ev_in) cudaEventDestroy(p->ev_in);
  if (p->ev_out) cudaEventDestroy(p->ev_out);
  if (p->ps) cudaStreamDestroy(p->ps);
  delete p;
}

#define DISPATCH(p, ...)            \
  do {                              \
    if ((p)->prec == MS_FP64) {     \
      typedef double R;             \
      __VA_ARGS__;                  \
    } else {                        \
      typedef float R;              \
      __VA_ARGS__;                  \
    }                               \
  } while (0)

// ------------------------------------------------------------ batched form
// All (channel, partition) jobs of one call share one gridding launch, one
// fold launch, one batched FFT and one crop (or one pad, one batched FFT, one
// degridding launch): the work items of all jobs form one launch, the job
// table says whose item a block holds.

struct BatchShape {
  int njobs = 0;
  int64_t items = 0, rows = 0, max_n = 0;
  int max_items = 0;
};

template <typename R>
BatchShape batch_jobs(ms_plan* p, int njobs, const int32_t* chans, const int32_t* parts,
                      std::vector<BatchJob<R>>& jobs) {
  arg(njobs > 0, "njobs must be positive");
  arg(chans && parts, "chans and parts are required");
  BatchShape sh;
  sh.njobs = njobs;
  jobs.assign(njobs, BatchJob<R>{});
  for (int j = 0; j < njobs; ++j) {
    PartDev& pd = part_of(p, parts[j], chans[j]);
    BatchJob<R>& b = jobs[j];
    b.items = pd.items;
    b.cell = pd.cell;
    b.frac = (const C2<R>*)pd.frac;
    b.idx = pd.idx;
    b.tile_items = pd.tile_items;
    b.n = pd.n;
    b.nitems = pd.nitems;
    b.item_base = sh.items;
    b.inv_n = pd.n > 0 ? 1.0 / (double)pd.n : 0.0;
    b.sorted_in = (C2<R>*)(intptr_t)sh.rows;    // offsets for now, pointers below
    sh.items += pd.nitems;
    sh.rows += pd.n;
    sh.max_n = std::max(sh.max_n, pd.n);
    sh.max_items = std::max(sh.max_items, pd.nitems);
  }
  arg(sh.items < (int64_t)1 << 31, "too many work items for one launch");
  return sh;
}

// grow the batch workspaces to hold `sh` (allocates only when it grows)
template <typename R> void batch_reserve(ms_plan* p, const BatchShape& sh) {
  auto& B = p->batch;
  const int Ng = p->Ng;
  auto grow = [&](void*& ptr, size_t bytes, const char* what) {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    ptr = dalloc<unsigned char>(bytes, what);
  };
  if (sh.njobs > B.cap_jobs) {
    grow(B.jobs, sizeof(BatchJob<R>) * sh.njobs, "batch jobs");
    grow(B.grids, sizeof(C2<R>) * (size_t)Ng * Ng * sh.njobs, "batch grids");
    B.cap_jobs = sh.njobs;
    B.tmap_jobs = 0;   // the stacked-grid descriptor names the old buffer
    if (B.fft) cufftDestroy(B.fft);
    B.fft = 0;
    B.fft_jobs = 0;
  }
  if (sh.items > B.cap_items) {
    void* jo = B.job_of;
    grow(jo, sizeof(int32_t) * std::max<int64_t>(sh.items, 1), "batch items");
    B.job_of = (int32_t*)jo;
    grow(B.scratch,
         (size_t)std::max<int64_t>(sh.items, 1) * p->S * p->S * grid_scratch_cell_bytes(p->prec),
         "batch scratch");
    B.cap_items = sh.items;
  }
  if (sh.rows > B.cap_rows) {
    grow(B.rows_a, sizeof(C2<R>) * std::max<int64_t>(sh.rows, 1), "batch rows");
    grow(B.rows_b, sizeof(C2<R>) * std::max<int64_t>(sh.rows, 1), "batch rows");
    B.cap_rows = sh.rows;
  }
  if (B.fft_jobs != sh.njobs) {
    if (B.fft) cufftDestroy(B.fft);
    B.fft = 0;
    int n[2] = {Ng, Ng};
    ckf(cufftPlanMany(&B.fft, 2, n, nullptr, 1, Ng * Ng, nullptr, 1, Ng * Ng,
                      sizeof(R) == 8 ? CUFFT_Z2Z : CUFFT_C2C, sh.njobs),
        "batched FFT plan");
    ckf(cufftSetStream(B.fft, p->ps), "set stream");
    B.fft_jobs = sh.njobs;
  }
  if (B.tmap_jobs != sh.njobs) {
    // the jobs' grids stacked: {2 Ng scalars, njobs Ng rows}, box {2 S, S}
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    ck(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                        &q),
       "driver entry point");
    arg(fn != nullptr && q == cudaDriverEntryPointSuccess, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)2 * Ng, (cuuint64_t)Ng * sh.njobs};
    cuuint64_t strides[1] = {(cuuint64_t)2 * Ng * sizeof(R)};
    cuuint32_t box[2] = {(cuuint32_t)(2 * p->S), (cuuint32_t)p->S};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = ((EncodeTiledFn)fn)(
        &B.tmap, sizeof(R) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
        2, B.grids, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Fail{MS_ERR_CUDA, "cuTensorMapEncodeTiled failed (batch)"};
    B.tmap_jobs = sh.njobs;
  }
}

// fill the workspace pointers of the jobs, upload the table, map items to jobs
template <typename R>
void batch_upload(ms_plan* p, const BatchShape& sh, std::vector<BatchJob<R>>& jobs) {
  auto& B = p->batch;
  const int64_t ng2 = (int64_t)p->Ng * p->Ng;
  for (int j = 0; j < sh.njobs; ++j) {
    const int64_t off = (int64_t)(intptr_t)jobs[j].sorted_in;
    jobs[j].sorted_in = (C2<R>*)B.rows_a + off;
    jobs[j].sorted_out = (C2<R>*)B.rows_b + off;
    jobs[j].grid = (C2<R>*)B.grids + j * ng2;
  }
  ck(cudaMemcpyAsync(B.jobs, jobs.data(), sizeof(BatchJob<R>) * sh.njobs,
                     cudaMemcpyHostToDevice, p->ps),
     "job table");
  launch_job_of<R>((const BatchJob<R>*)B.jobs, sh.njobs, sh.max_items, B.job_of, p->ps);
}

template <typename R> void batch_fft(ms_plan* p, int dir) {
  if (sizeof(R) == 8)
    ckf(cufftExecZ2Z(p->batch.fft, (cufftDoubleComplex*)p->batch.grids,
                     (cufftDoubleComplex*)p->batch.grids, dir),
        "batched Z2Z");
  else
    ckf(cufftExecC2C(p->batch.fft, (cufftComplex*)p->batch.grids,
                     (cufftComplex*)p->batch.grids, dir),
        "batched C2C");
}

template <typename R>
void grid_batch(ms_plan* p, int njobs, const int32_t* chans, const int32_t* parts,
                const void* const* vis, void* const* dirty) {
  arg(vis && dirty, "vis and dirty are required");
  std::vector<BatchJob<R>> jobs;
  BatchShape sh = batch_jobs<R>(p, njobs, chans, parts, jobs);
  for (int j = 0; j < njobs; ++j) {
    arg(vis[j] && dirty[j], "a job's vis or dirty pointer is NULL");
    jobs[j].user_in = (const C2<R>*)vis[j];
    jobs[j].image_out = (R*)dirty[j];
  }
  batch_reserve<R>(p, sh);
  batch_upload<R>(p, sh, jobs);
  const BatchJob<R>* jd = (const BatchJob<R>*)p->batch.jobs;
  launch_batch_gather<R>(jd, njobs, sh.max_n, p->ps);
  {
    KSpan k(p, MS_K_GRID);
    if (p->prec == MS_FP32_KAHAN)
      launch_grid_batch<float, true>((const BatchJob<float>*)jd, p->batch.job_of, (int)sh.items,
                                     p->batch.scratch, p->T, p->ntx, p->beta, p->ps);
    else
      launch_grid_batch<R, false>(jd, p->batch.job_of, (int)sh.items, p->batch.scratch, p->T,
                                  p->ntx, p->beta, p->ps);
  }
  {
    KSpan k(p, MS_K_FOLD);
    if (p->prec == MS_FP32_KAHAN)
      launch_fold_batch<float, true>((const BatchJob<float>*)jd, njobs, p->batch.scratch, p->Ng,
                                     p->T, p->ntx, p->ps);
    else
      launch_fold_batch<R, false>(jd, njobs, p->batch.scratch, p->Ng, p->T, p->ntx, p->ps);
  }
  {
    KSpan k(p, MS_K_FFT_GRID);
    batch_fft<R>(p, CUFFT_INVERSE);
  }
  KSpan k(p, MS_K_PAD_CROP);
  launch_crop_batch<R>(jd, njobs, (const R*)p->psi, p->N, p->Ng, p->ps);
}

template <typename R>
void degrid_batch(ms_plan* p, int njobs, const int32_t* chans, const int32_t* parts,
                  const void* const* images, const void* const* vis_obs, void* const* vis_out) {
  arg(images && vis_out, "images and vis_out are required");
  std::vector<BatchJob<R>> jobs;
  BatchShape sh = batch_jobs<R>(p, njobs, chans, parts, jobs);
  for (int j = 0; j < njobs; ++j) {
    arg(images[j] && vis_out[j], "a job's image or vis_out pointer is NULL");
    arg(!vis_obs || vis_obs[j], "a job's vis_obs pointer is NULL");
    jobs[j].image_in = (const R*)images[j];
    jobs[j].user_in = vis_obs ? (const C2<R>*)vis_obs[j] : nullptr;
    jobs[j].user_out = (C2<R>*)vis_out[j];
  }
  batch_reserve<R>(p, sh);
  batch_upload<R>(p, sh, jobs);
  const BatchJob<R>* jd = (const BatchJob<R>*)p->batch.jobs;
  if (vis_obs) launch_batch_gather<R>(jd, njobs, sh.max_n, p->ps);
  {
    KSpan k(p, MS_K_PAD_CROP);
    launch_pad_batch<R>(jd, njobs, (const R*)p->psi, p->N, p->Ng, p->ps);
  }
  {
    KSpan k(p, MS_K_FFT_GRID);
    batch_fft<R>(p, CUFFT_FORWARD);
  }
  {
    KSpan k(p, MS_K_DEGRID);
    launch_degrid_batch<R>(&p->batch.tmap, jd, p->batch.job_of, (int)sh.items, vis_obs != nullptr,
                           p->Ng, p->T, p->ntx, p->beta, p->err, p->ps);
  }
  launch_batch_scatter<R>(jd, njobs, sh.max_n, p->ps);
}

// ------------------------------------------------- batched minor cycles
// Grow the batched FISTA workspace to `jobs` jobs of up to max_iters
// iterations (frees and reallocates everything when it grows).
template <typename R> void ensure_fista_batch(ms_plan* p, int jobs, int max_iters) {
  FistaBatch& F = p->fb;
  if (jobs <= F.cap && max_iters + 2 <= F.trace_cap) return;
  const int cap = std::max(jobs, F.cap);
  const int tcap = std::max({max_iters + 2, F.trace_cap, 1024});
  F.release();
  const int N = p->N;
  const int64_t n2 = (int64_t)N * N, nspec = (int64_t)N * (N / 2 + 1), ncoef = (int64_t)p->M * n2;
  for (auto& b : F.B) b = dalloc<R>(ncoef * cap, "batch coefficients");
  F.x = dalloc<R>(n2 * cap, "batch images");
  F.y = dalloc<R>(n2 * cap, "batch images");
  for (auto& f : F.F) f = dalloc<C2<R>>(nspec * cap, "batch spectra");
  F.zrow = dalloc<C2<R>>(nspec * cap, "batch spectra");
  F.Ks = dalloc<R>(nspec * cap, "batch spectra");
  F.Bs = dalloc<C2<R>>(nspec * cap, "batch spectra");
  F.tmp = dalloc<R>(ncoef * cap, "batch wavelet tmp");
  F.model = dalloc<R>(n2 * cap, "batch images");
  F.res = dalloc<R>(n2 * cap, "batch images");
  F.l = dalloc<R>(n2 * cap, "batch images");
  F.ctl = dalloc<FistaCtl>(cap, "batch control");
  F.trace = dalloc<double>((int64_t)tcap * cap, "batch trace");
  F.parts_stride = std::max(4096, 3 * spec_col_warps(N, sizeof(C2<R>)));
  F.parts = dalloc<double>(F.parts_stride * cap, "batch partials");
  F.l1 = dalloc<double>((int64_t)p->n_l1 * cap, "batch partials");
  ck(cudaMemset(F.ctl, 0, sizeof(FistaCtl) * cap), "memset");
  F.cap = cap;
  F.trace_cap = tcap;
  // the stacked gradient images for the level-1 analysis's TMA window loads
  unsigned bc = 0, br = 0;
  analysis_window_box(&bc, &br);
  if (p->have_grad_map && (unsigned)N >= bc) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    ck(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                        &q),
       "driver entry point");
    arg(fn != nullptr && q == cudaDriverEntryPointSuccess, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t gd[2] = {(cuuint64_t)N, (cuuint64_t)N * cap};
    cuuint64_t gs[1] = {(cuuint64_t)N * sizeof(R)};
    cuuint32_t gb[2] = {bc, br};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = ((EncodeTiledFn)fn)(
        &F.gmap, sizeof(R) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
        2, F.y, gd, gs, gb, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
        CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) throw Fail{MS_ERR_CUDA, "cuTensorMapEncodeTiled failed (batch)"};
    F.have_gmap = true;
  }
}

template <typename R> PassView<R> batch_view(ms_plan* p, int jobs) {
  FistaBatch& F = p->fb;
  const int N = p->N;
  const int64_t n2 = (int64_t)N * N, nspec = (int64_t)N * (N / 2 + 1);
  PassView<R> v;
  v.a = fista_pass_args<R>(p);
  v.a.B0 = (R*)F.B[0];
  v.a.B1 = (R*)F.B[1];
  v.a.B2 = (R*)F.B[2];
  v.a.grad = (const R*)F.y;
  v.a.x = (R*)F.x;
  v.a.tmp = (R*)F.tmp;
  v.a.ctl = F.ctl;
  v.a.l1_parts = F.l1;
  v.a.coarse_ctas = 0;   // per-level launches: a cooperative launch cannot hold every job
  JobStride& js = v.a.js;
  js.jobs = jobs;
  js.coef = (int64_t)p->M * n2;
  js.img = n2;
  js.tmp = (int64_t)p->M * n2;
  js.spec = nspec;
  js.parts = F.parts_stride;
  js.l1 = p->n_l1;
  js.trace = F.trace_cap;
  v.F[0] = (C2<R>*)F.F[0];
  v.F[1] = (C2<R>*)F.F[1];
  v.zrow = (C2<R>*)F.zrow;
  v.Ks = (const R*)F.Ks;
  v.Bs = (const C2<R>*)F.Bs;
  v.parts = F.parts;
  v.trace = F.trace;
  v.gmap = F.have_gmap ? &F.gmap : nullptr;
  return v;
}

void check_batchable(ms_plan* p) {
  if (!p->fused_spec || p->dict != MS_DICT_DAUBECHIES || p->conv != MS_CONV_CIRCULAR)
    throw Fail{MS_ERR_UNSUPPORTED,
               "batched minor cycles need N a power of two, the Daubechies dictionary and the "
               "circular PSF operator"};
}

// The FISTA loop of `jobs` set-up problems (each job's control block, K^ and
// b^ slices ready): B_0 = 0, kPasses passes per graph launch, each kernel
// over all jobs; a job whose control block says done skips its share.
template <typename R> void run_fista_batch(ms_plan* p, int jobs, int max_iters, double rel_tol) {
  FistaBatch& F = p->fb;
  const int N = p->N;
  const int64_t n2 = (int64_t)N * N, nspec = (int64_t)N * (N / 2 + 1);
  const int64_t ncoef = (int64_t)p->M * n2;
  ck(cudaMemsetAsync(F.B[0], 0, sizeof(R) * ncoef * jobs, p->ps), "memset");
  ck(cudaMemsetAsync(F.B[2], 0, sizeof(R) * ncoef * jobs, p->ps), "memset");
  ck(cudaMemsetAsync(F.F[1], 0, sizeof(C2<R>) * nspec * jobs, p->ps), "memset");
  ck(cudaMemsetAsync(F.l1, 0, sizeof(double) * p->n_l1 * jobs, p->ps), "memset");   // ||B_0||_1
  for (int j = 0; j < jobs; ++j) set_target_kernel<<<1, 1, 0, p->ps>>>(F.ctl + j, p->obj_target);
  const PassView<R> v = batch_view<R>(p, jobs);
  const bool poll = rel_tol > 0 || std::isfinite(p->obj_target);
  std::vector<FistaCtl> h(jobs);
  auto all_done = [&]() {
    ck(cudaMemcpyAsync(h.data(), F.ctl, sizeof(FistaCtl) * jobs, cudaMemcpyDeviceToHost, p->ps),
       "read ctl");
    ck(cudaStreamSynchronize(p->ps), "synchronize");
    for (const FistaCtl& c : h)
      if (!c.done) return false;
    return true;
  };
  const int passes = max_iters + 1;
  if (p->prof) {
    for (int i = 0; i < passes; ++i) {
      record_fista_pass<R>(p, i & 1, v);
      if ((i + 1) % kPasses == 0 && p->pending.size() > 4096) harvest(p);
      if (poll && (i + 1) % (4 * kPasses) == 0 && i + 1 < passes && all_done()) break;
    }
    return;
  }
  if (F.exec && F.exec_jobs != jobs) {
    cudaGraphExecDestroy(F.exec);
    F.exec = nullptr;
  }
  if (!F.exec) {
    cudaGraph_t graph;
    ck(cudaStreamBeginCapture(p->ps, cudaStreamCaptureModeThreadLocal), "begin capture");
    p->capturing = true;
    try {
      for (int i = 0; i < kPasses; ++i) record_fista_pass<R>(p, i & 1, v);
    } catch (...) {
      p->capturing = false;
      cudaStreamEndCapture(p->ps, &graph);
      throw;
    }
    p->capturing = false;
    ck(cudaStreamEndCapture(p->ps, &graph), "end capture");
    ck(cudaGraphInstantiate(&F.exec, graph, 0), "graph instantiate");
    cudaGraphDestroy(graph);
    F.exec_jobs = jobs;
  }
  int launched = 0;
  while (launched < passes) {
    ck(cudaGraphLaunch(F.exec, p->ps), "graph launch");
    launched += kPasses;
    if (poll && launched < passes && (launched / kPasses) % 4 == 0 && all_done()) break;
  }
}

// job j's results: the statistics (and, with copy_trace, its trace)
template <typename R> void batch_stats(ms_plan* p, int jobs, ms_stats* stats) {
  if (!stats) return;
  FistaBatch& F = p->fb;
  std::vector<FistaCtl> h(jobs);
  ck(cudaMemcpyAsync(h.data(), F.ctl, sizeof(FistaCtl) * jobs, cudaMemcpyDeviceToHost, p->ps),
     "read ctl");
  ck(cudaStreamSynchronize(p->ps), "synchronize");
  for (int j = 0; j < jobs; ++j) {
    if (h[j].error)
      throw Fail{(ms_status)h[j].error, "non-finite objective or invalid noise levels"};
    ms_stats& st = stats[j];
    st.iterations = h[j].k;
    st.converged = h[j].converged;
    st.objective = h[j].F_cur;
    st.lambda = h[j].lam;
    st.theta = h[j].theta;
    st.sigma2 = h[j].sigma2;
    st.eta2 = h[j].eta2;
    st.objective_trace = nullptr;
  }
}

// ms_minor_cycle_batch: set up each job's problem, run the batched loop,
// copy each job's model image out
template <typename R>
void minor_cycle_batch(ms_plan* p, int njobs, const int32_t* steps, const int32_t* chans,
                       const void* const* residuals, const void* const* l_lows,
                       const double* lambdas, const double* sigma2s, const double* eta2s,
                       int max_iters, double rel_tol, void* const* models_out, ms_stats* stats,
                       double* traces) {
  check_batchable(p);
  arg(njobs >= 1 && njobs <= 4096, "njobs must be 1..4096");
  arg(steps && chans && residuals && lambdas && models_out, "a required array is NULL");
  arg(max_iters >= 1 && max_iters <= 1000000, "max_iters must be 1..1e6");
  ensure_fista_batch<R>(p, njobs, max_iters);
  FistaBatch& F = p->fb;
  const int N = p->N;
  const int64_t n2 = (int64_t)N * N, nspec = (int64_t)N * (N / 2 + 1);
  for (int j = 0; j < njobs; ++j) {
    const int step = steps[j];
    arg(step >= MS_STEP_LOW && step <= MS_STEP_FULL_L, "unknown step");
    arg(residuals[j] && models_out[j], "a job's residual or model pointer is NULL");
    const bool full = step_full(step);
    arg(!full || (l_lows && l_lows[j] && sigma2s && eta2s), "FULL jobs need l_low, sigma2, eta2");
    arg(lambdas[j] >= 0 && std::isfinite(lambdas[j]), "lambda must be finite and >= 0");
    PartDev& pd = part_of(p, step_part(step), chans[j]);
    FistaCtl* c = F.ctl + j;
    init_ctl_kernel<<<1, 1, 0, p->ps>>>(c, max_iters, rel_tol, lambdas[j], 1,
                                        full ? sigma2s[j] : 0.0, full ? eta2s[j] : 0.0,
                                        full ? 1 : 0);
    build_normal<R>(p, step, pd, p->d.ell_px, p->d.delta_px, c, (R*)F.Ks + j * nspec);
    build_b<R>(p, step, pd, residuals[j], full ? l_lows[j] : nullptr, c,
               (C2<R>*)F.Bs + j * nspec);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ck(cudaEventCreate(&e0), "event");
  ck(cudaEventCreate(&e1), "event");
  ck(cudaEventRecord(e0, p->ps), "event");
  run_fista_batch<R>(p, njobs, max_iters, rel_tol);
  ck(cudaEventRecord(e1, p->ps), "event");
  for (int j = 0; j < njobs; ++j)
    ck(cudaMemcpyAsync(models_out[j], (R*)F.x + j * n2, sizeof(R) * n2, cudaMemcpyDeviceToDevice,
                       p->ps),
       "copy");
  if (traces)   // [njobs][max_iters + 1], F(beta_0..) of each job (NaN past its last)
    for (int j = 0; j < njobs; ++j)
      ck(cudaMemcpyAsync(traces + (int64_t)j * (max_iters + 1), F.trace + (int64_t)j * F.trace_cap,
                         sizeof(double) * (max_iters + 1), cudaMemcpyDeviceToHost, p->ps),
         "copy");
  batch_stats<R>(p, njobs, stats);
  float ms = 0;
  ck(cudaEventSynchronize(e1), "event");
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (stats)
    for (int j = 0; j < njobs; ++j) {
      stats[j].elapsed_ms = stats[j].minor_ms = ms;
      stats[j].total_iterations = stats[j].iterations;
    }
}

// residual images of several (channel, partition) jobs at once: job j takes
// partition parts[j] of channel chans[j], obs = vis[j] (original order),
// model models + j N^2, residual res + j N^2;
// one pad / FFT / degridding launch over all jobs, then the residual rows
// (left in plan order) through one gridding / fold / FFT / crop
template <typename R>
void residual_batch(ms_plan* p, int njobs, const int32_t* chans, const int32_t* parts,
                    const void* const* vis, const R* models, R* res) {
  const int64_t n2 = (int64_t)p->N * p->N;
  std::vector<BatchJob<R>> jobs;
  const BatchShape sh = batch_jobs<R>(p, njobs, chans, parts, jobs);
  for (int j = 0; j < njobs; ++j) {
    arg(vis[j] != nullptr, "a job's visibilities are NULL");
    jobs[j].user_in = (const C2<R>*)vis[j];
    jobs[j].image_in = models + j * n2;
    jobs[j].image_out = res + j * n2;
  }
  batch_reserve<R>(p, sh);
  batch_upload<R>(p, sh, jobs);
  const BatchJob<R>* jd = (const BatchJob<R>*)p->batch.jobs;
  launch_batch_gather<R>(jd, njobs, sh.max_n, p->ps);
  {
    KSpan k(p, MS_K_PAD_CROP);
    launch_pad_batch<R>(jd, njobs, (const R*)p->psi, p->N, p->Ng, p->ps);
  }
  {
    KSpan k(p, MS_K_FFT_GRID);
    batch_fft<R>(p, CUFFT_FORWARD);
  }
  {
    KSpan k(p, MS_K_DEGRID);
    launch_degrid_batch<R>(&p->batch.tmap, jd, p->batch.job_of, (int)sh.items, true, p->Ng,
                           p->T, p->ntx, p->beta, p->err, p->ps);
  }
  // grid the residual rows obs - A x where the degridding left them
  for (auto& b : jobs) std::swap(b.sorted_in, b.sorted_out);
  ck(cudaMemcpyAsync(p->batch.jobs, jobs.data(), sizeof(BatchJob<R>) * njobs,
                     cudaMemcpyHostToDevice, p->ps),
     "job table");
  {
    KSpan k(p, MS_K_GRID);
    if (p->prec == MS_FP32_KAHAN)
      launch_grid_batch<float, true>((const BatchJob<float>*)jd, p->batch.job_of, (int)sh.items,
                                     p->batch.scratch, p->T, p->ntx, p->beta, p->ps);
    else
      launch_grid_batch<R, false>(jd, p->batch.job_of, (int)sh.items, p->batch.scratch, p->T,
                                  p->ntx, p->beta, p->ps);
  }
  {
    KSpan k(p, MS_K_FOLD);
    if (p->prec == MS_FP32_KAHAN)
      launch_fold_batch<float, true>((const BatchJob<float>*)jd, njobs, p->batch.scratch, p->Ng,
                                     p->T, p->ntx, p->ps);
    else
      launch_fold_batch<R, false>(jd, njobs, p->batch.scratch, p->Ng, p->T, p->ntx, p->ps);
  }
  {
    KSpan k(p, MS_K_FFT_GRID);
    batch_fft<R>(p, CUFFT_INVERSE);
  }
  KSpan k(p, MS_K_PAD_CROP);
  launch_crop_batch<R>(jd, njobs, (const R*)p->psi, p->N, p->Ng, p->ps);
}

// One step of the method (as run_step) for several channels at once: the
// major cycles' residuals through residual_batch, every minor cycle through
// the batched FISTA loop.  low_images: i^_L of each job (FULL); out: each
// job's final image.
template <typename R>
void run_step_batch(ms_plan* p, int step, int njobs, const int32_t* chans,
                    const void* const* vis, const ms_recon_opts& o,
                    const void* const* low_images, void* const* out, ms_stats* stats) {
  FistaBatch& F = p->fb;
  const int N = p->N;
  const int64_t n2 = (int64_t)N * N, nspec = (int64_t)N * (N / 2 + 1);
  const int part = step_part(step);
  const std::vector<int32_t> parts(njobs, part);
  const bool full = step == MS_STEP_FULL;
  R* model = (R*)F.model;
  R* res = (R*)F.res;
  R* l = (R*)F.l;
  ck(cudaMemsetAsync(model, 0, sizeof(R) * n2 * njobs, p->ps), "memset");
  const double coef = step == MS_STEP_LOW ? o.lambda_low
                      : full ? o.lambda_full : o.lambda_single;
  std::vector<FistaCtl> h(njobs);
  for (int n = 1; n <= o.n_major; ++n) {
    residual_batch<R>(p, njobs, chans, parts.data(), vis, model, res);
    for (int j = 0; j < njobs; ++j) {
      FistaCtl* c = F.ctl + j;
      R* rj = res + j * n2;
      PartDev& pd = part_of(p, part, chans[j]);
      launch_image_norms<R>(rj, n2, p->parts, c, p->tickets + 5, p->ps);
      if (n == 1) {
        init_ctl_kernel<<<1, 1, 0, p->ps>>>(
            c, o.fista_iters, o.rel_tol, 0.0, 0, o.sigma2,
            o.sigma2 > 0 && o.eta2 > 0 ? o.eta2 : 1e-3 * o.sigma2, o.sigma2 > 0 ? 1 : 0);
        if (full && !(o.sigma2 > 0)) {
          launch_sigma2_hat<R>(rj, N, p->parts, c, p->tickets + 6, o.eta2 > 0 ? 0 : 1, p->ps);
          if (o.eta2 > 0) set_eta_kernel<<<1, 1, 0, p->ps>>>(c, o.eta2);
        }
        build_normal<R>(p, step, pd, p->d.ell_px, p->d.delta_px, c, (R*)F.Ks + j * nspec);
      }
      init_ctl_kernel<<<1, 1, 0, p->ps>>>(c, o.fista_iters, o.rel_tol, 0.0, 0, 0, 0, 0);
      launch_set_lambda(c, o.lambda_rule, coef, n, n == 1 ? 1 : 0, p->ps);
      if (full) {
        // l = i^_L - sum i_j, and this job's filters for b^
        launch_axpby<R>((const R*)low_images[j], model + j * n2, l + j * n2, 1.0, -1.0, n2,
                        p->ps);
        launch_filters<R>(N, p->d.ell_px, p->d.delta_px, c, (R*)p->gl2, (R*)p->gh2, p->ps);
      }
      build_b<R>(p, step, pd, rj, full ? l + j * n2 : nullptr, c, (C2<R>*)F.Bs + j * nspec);
    }
    run_fista_batch<R>(p, njobs, o.fista_iters, o.rel_tol);
    launch_axpby<R>(model, (const R*)F.x, model, 1.0, 1.0, n2 * njobs, p->ps);   // i^ += W beta
    ck(cudaMemcpyAsync(h.data(), F.ctl, sizeof(FistaCtl) * njobs, cudaMemcpyDeviceToHost, p->ps),
       "read ctl");
    ck(cudaStreamSynchronize(p->ps), "synchronize");
    for (int j = 0; j < njobs; ++j) {
      if (h[j].error)
        throw Fail{(ms_status)h[j].error, "non-finite objective or invalid noise levels"};
      if (stats) {
        stats[j].total_iterations += h[j].k;
        stats[j].gridded_vis += part_of(p, part, chans[j]).n;
      }
    }
  }
  residual_batch<R>(p, njobs, chans, parts.data(), vis, model, res);   // i~_{N+1}
  for (int j = 0; j < njobs; ++j) {
    launch_axpby<R>(res + j * n2, model + j * n2, (R*)out[j], 1.0, 1.0, n2, p->ps);
    if (stats) {
      stats[j].gridded_vis += part_of(p, part, chans[j]).n;
      stats[j].major_cycles += o.n_major;
      stats[j].iterations = h[j].k;
      stats[j].converged = h[j].converged;
      stats[j].objective = h[j].F_cur;
      stats[j].lambda = h[j].lam;
      stats[j].theta = h[j].theta;
      stats[j].sigma2 = h[j].sigma2;
      stats[j].eta2 = h[j].eta2;
    }
  }
}

// The interleaved pipeline on plans the batched form does not serve (the
// linear PSF operator, the IUWT dictionary, N not a power of two): the two
// nodes' minor cycles of a major cycle run one after the other on the plan's
// own minor-cycle state, both reading the models of the previous cycle, so
// the result is the batched form's.  Per node the plan's K^ and step size are
// rebuilt for every minor cycle (one problem of each node at a time); the
// lambda rule must be NORM2_2N.
template <typename R>
void interleaved_seq(ms_plan* p, int chan, const void* vis, const ms_recon_opts* o,
                     void* img_out, void* node_l_out, void* node_h_out, ms_stats* stats) {
  arg(o->lambda_rule == MS_LAMBDA_NORM2_2N,
      "the interleaved pipeline on this plan needs the NORM2_2N lambda rule");
  const int N = p->N;
  const int64_t n2 = (int64_t)N * N;
  if (!p->il_buf) p->il_buf = p->alloc<R>(6 * n2, "interleaved images");
  R* model = (R*)p->il_buf;   // [node L, node H]
  R* res = model + 2 * n2;
  R* l = res + 2 * n2;
  ensure_trace(p, o->fista_iters);
  const int parts[2] = {MS_PART_L, MS_PART_H};
  const double coef[2] = {o->lambda_low, o->lambda_full};
  double s2[2] = {0, 0}, e2[2] = {0, 0};
  int64_t iters[2] = {0, 0};
  FistaCtl h{};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ck(cudaEventCreate(&e0), "event");
  ck(cudaEventCreate(&e1), "event");
  ck(cudaEventRecord(e0, p->ps), "event");
  ck(cudaMemsetAsync(model, 0, sizeof(R) * 2 * n2, p->ps), "memset");
  auto residuals = [&]() {
    for (int j = 0; j < 2; ++j) {
      PartDev& pd = part_of(p, parts[j], chan);
      launch_gather_vis<R>(pd.idx, pd.n, (const C2<R>*)vis, (C2<R>*)p->vis_a, p->ps);
      residual_sorted<R>(p, pd, p->vis_a, model + j * n2, res + j * n2, nullptr);
    }
  };
  for (int n = 1; n <= o->n_major; ++n) {
    residuals();
    if (n >= 2)   // the other node's model minus this one's, both of cycle n - 1
      for (int j = 0; j < 2; ++j)
        launch_axpby<R>(model + (1 - j) * n2, model + j * n2, l + j * n2, 1.0, -1.0, n2, p->ps);
    const int kind[2] = {n == 1 ? MS_STEP_LOW : MS_STEP_FULL_L,
                         n == 1 ? MS_STEP_LOW_H : MS_STEP_FULL};
    for (int j = 0; j < 2; ++j) {
      PartDev& pd = part_of(p, parts[j], chan);
      R* rj = res + j * n2;
      init_ctl_kernel<<<1, 1, 0, p->ps>>>(p->ctl, o->fista_iters, o->rel_tol, 0.0, 0, s2[j],
                                          e2[j], n > 1 ? 1 : 0);
      launch_image_norms<R>(rj, n2, p->parts, p->ctl, p->tickets + 5, p->ps);
      if (n == 1) {   // sigma^2 on the node's first residual, eta^2 = 1e-3 sigma^2
        launch_sigma2_hat<R>(rj, N, p->parts, p->ctl, p->tickets + 6, 1, p->ps);
        ck(cudaMemcpyAsync(&h, p->ctl, sizeof(h), cudaMemcpyDeviceToHost, p->ps), "read ctl");
        ck(cudaStreamSynchronize(p->ps), "synchronize");
        s2[j] = h.sigma2;
        e2[j] = h.eta2;
      }
      launch_set_lambda(p->ctl, o->lambda_rule, coef[j], n, n == 1 ? 1 : 0, p->ps);
      build_normal<R>(p, kind[j], pd, p->d.ell_px, p->d.delta_px);
      run_fista<R>(p, kind[j], pd, rj, n >= 2 ? l + j * n2 : nullptr, nullptr, o->fista_iters,
                   o->rel_tol);
      launch_axpby<R>(model + j * n2, (const R*)p->xwork, model + j * n2, 1.0, 1.0, n2, p->ps);
      ck(cudaMemcpyAsync(&h, p->ctl, sizeof(h), cudaMemcpyDeviceToHost, p->ps), "read ctl");
      ck(cudaStreamSynchronize(p->ps), "synchronize");
      if (h.error) throw Fail{(ms_status)h.error, "non-finite objective or invalid noise levels"};
      iters[j] += h.k;
      if (stats) {
        ms_stats& st = stats[j];
        st.total_iterations = (int32_t)iters[j];
        st.gridded_vis += pd.n;
        st.iterations = h.k;
        st.converged = h.converged;
        st.objective = h.F_cur;
        st.lambda = h.lam;
        st.theta = h.theta;
        st.sigma2 = s2[j];
        st.eta2 = e2[j];
        st.major_cycles = o->n_major;
      }
    }
  }
  residuals();   // i~_{N+1} of both nodes
  R* fin = l;    // the nodes' final images: last residual + model
  launch_axpby<R>(res, model, fin, 1.0, 1.0, 2 * n2, p->ps);
  if (node_l_out)
    ck(cudaMemcpyAsync(node_l_out, fin, sizeof(R) * n2, cudaMemcpyDeviceToDevice, p->ps), "copy");
  if (node_h_out)
    ck(cudaMemcpyAsync(node_h_out, fin + n2, sizeof(R) * n2, cudaMemcpyDeviceToDevice, p->ps),
       "copy");
  // combination with node H's filters
  init_ctl_kernel<<<1, 1, 0, p->ps>>>(p->ctl, 1, 0.0, 0.0, 0, s2[1], e2[1], 1);
  launch_filters<R>(N, p->d.ell_px, p->d.delta_px, p->ctl, (R*)p->gl2, (R*)p->gh2, p->ps);
  fft_r2c<R>(p, fin, p->spec);
  fft_r2c<R>(p, fin + n2, p->spec2);
  launch_combine_spectra<R>((C2<R>*)p->spec, (const C2<R>*)p->spec2, (const R*)p->gl2,
                            (const R*)p->gh2, p->ctl, N, p->ps);
  fft_c2r<R>(p, p->spec, img_out);
  ck(cudaEventRecord(e1, p->ps), "event");
  check_device_error(p);
  float ms = 0;
  ck(cudaEventSynchronize(e1), "event");
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (stats)
    for (int j = 0; j < 2; ++j) {
      stats[j].gridded_vis += part_of(p, parts[j], chan).n;
      stats[j].elapsed_ms = ms;
    }
}

// The interleaved two-image pipeline (ms_reconstruct_interleaved): node L
// (job 0, V_L) and node H (job 1, V_H) of channel `chan`; each major cycle
// one batched residual pass and one batched minor cycle serve both nodes.
template <typename R>
void interleaved(ms_plan* p, int chan, const void* vis, const ms_recon_opts* o, void* img_out,
                 void* node_l_out, void* node_h_out, ms_stats* stats, void* stream) {
  validate_opts(o);
  arg(o->warm_start == nullptr, "the interleaved pipeline takes no warm start network");
  arg(vis && img_out, "vis and img_out are required");
  arg(chan >= 0 && chan < (int)p->ch.size(), "channel out of range");
  arg(p->ch[chan].part[MS_PART_L].n > 0 && p->ch[chan].part[MS_PART_H].n > 0,
      "both partitions need visibilities");
  Scope sc(p, stream);
  if (stats) std::memset(stats, 0, sizeof(ms_stats) * 2);
  const bool batchable =
      p->fused_spec && p->dict == MS_DICT_DAUBECHIES && p->conv == MS_CONV_CIRCULAR;
  if (!batchable) {
    interleaved_seq<R>(p, chan, vis, o, img_out, node_l_out, node_h_out, stats);
    sc.finish();
    return;
  }
  ensure_fista_batch<R>(p, 2, o->fista_iters);
  FistaBatch& F = p->fb;
  const int N = p->N;
  const int64_t n2 = (int64_t)N * N, nspec = (int64_t)N * (N / 2 + 1);
  R* model = (R*)F.model;   // [node L, node H]
  R* res = (R*)F.res;
  R* l = (R*)F.l;
  const int32_t chans[2] = {chan, chan}, parts[2] = {MS_PART_L, MS_PART_H};
  const void* const visv[2] = {vis, vis};
  const double coef[2] = {o->lambda_low, o->lambda_full};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ck(cudaEventCreate(&e0), "event");
  ck(cudaEventCreate(&e1), "event");
  ck(cudaEventRecord(e0, p->ps), "event");
  ck(cudaMemsetAsync(model, 0, sizeof(R) * 2 * n2, p->ps), "memset");
  std::vector<FistaCtl> h(2);
  for (int n = 1; n <= o->n_major; ++n) {
    residual_batch<R>(p, 2, chans, parts, visv, model, res);
    // cycle 1: Eq. LowRes on each node's data; then node L the mirrored
    // FullRes problem, node H Eq. FullRes, each against the other's model
    const int kind[2] = {n == 1 ? MS_STEP_LOW : MS_STEP_FULL_L,
                         n == 1 ? MS_STEP_LOW_H : MS_STEP_FULL};
    for (int j = 0; j < 2; ++j) {
      FistaCtl* c = F.ctl + j;
      R* rj = res + j * n2;
      PartDev& pd = part_of(p, parts[j], chan);
      launch_image_norms<R>(rj, n2, p->parts, c, p->tickets + 5, p->ps);
      if (n == 1) {
        init_ctl_kernel<<<1, 1, 0, p->ps>>>(c, o->fista_iters, o->rel_tol, 0.0, 0, 0, 0, 0);
        // sigma^2 on the node's first residual, eta^2 = 1e-3 sigma^2
        launch_sigma2_hat<R>(rj, N, p->parts, c, p->tickets + 6, 1, p->ps);
      }
      init_ctl_kernel<<<1, 1, 0, p->ps>>>(c, o->fista_iters, o->rel_tol, 0.0, 0, 0, 0, 0);
      if (n <= 2)   // the problem's operator changes once, at cycle 2
        build_normal<R>(p, kind[j], pd, p->d.ell_px, p->d.delta_px, c, (R*)F.Ks + j * nspec);
      launch_set_lambda(c, o->lambda_rule, coef[j], n, n == 1 ? 1 : 0, p->ps);
      R* lj = nullptr;
      if (n >= 2) {
        lj = l + j * n2;   // the other node's model minus this one's
        launch_axpby<R>(model + (1 - j) * n2, model + j * n2, lj, 1.0, -1.0, n2, p->ps);
        launch_filters<R>(N, p->d.ell_px, p->d.delta_px, c, (R*)p->gl2, (R*)p->gh2, p->ps,
                          kind[j] == MS_STEP_FULL_L);
      }
      build_b<R>(p, kind[j], pd, rj, lj, c, (C2<R>*)F.Bs + j * nspec);
    }
    run_fista_batch<R>(p, 2, o->fista_iters, o->rel_tol);
    launch_axpby<R>(model, (const R*)F.x, model, 1.0, 1.0, 2 * n2, p->ps);
    ck(cudaMemcpyAsync(h.data(), F.ctl, sizeof(FistaCtl) * 2, cudaMemcpyDeviceToHost, p->ps),
       "read ctl");
    ck(cudaStreamSynchronize(p->ps), "synchronize");
    for (int j = 0; j < 2; ++j) {
      if (h[j].error)
        throw Fail{(ms_status)h[j].error, "non-finite objective or invalid noise levels"};
      if (stats) {
        stats[j].total_iterations += h[j].k;
        stats[j].gridded_vis += part_of(p, parts[j], chan).n;
      }
    }
  }
  residual_batch<R>(p, 2, chans, parts, visv, model, res);   // i~_{N+1} of both nodes
  R* fin = (R*)F.l;   // the nodes' final images: last residual + model
  launch_axpby<R>(res, model, fin, 1.0, 1.0, 2 * n2, p->ps);
  if (node_l_out)
    ck(cudaMemcpyAsync(node_l_out, fin, sizeof(R) * n2, cudaMemcpyDeviceToDevice, p->ps), "copy");
  if (node_h_out)
    ck(cudaMemcpyAsync(node_h_out, fin + n2, sizeof(R) * n2, cudaMemcpyDeviceToDevice, p->ps),
       "copy");
  // combination with node H's filters: eta^2 g_L^2 F(node L) + sigma^2 g_H^2 F(node H)
  launch_filters<R>(N, p->d.ell_px, p->d.delta_px, F.ctl + 1, (R*)p->gl2, (R*)p->gh2, p->ps);
  fft_r2c<R>(p, fin, p->spec);
  fft_r2c<R>(p, fin + n2, p->spec2);
  launch_combine_spectra<R>((C2<R>*)p->spec, (const C2<R>*)p->spec2, (const R*)p->gl2,
                            (const R*)p->gh2, F.ctl + 1, N, p->ps);
  fft_c2r<R>(p, p->spec, img_out);
  ck(cudaEventRecord(e1, p->ps), "event");
  check_device_error(p);
  float ms = 0;
  ck(cudaEventSynchronize(e1), "event");
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (stats)
    for (int j = 0; j < 2; ++j) {
      ms_stats& st = stats[j];
      st.gridded_vis += part_of(p, parts[j], chan).n;
      st.major_cycles = o->n_major;
      st.iterations = h[j].k;
      st.converged = h[j].converged;
      st.objective = h[j].F_cur;
      st.lambda = h[j].lam;
      st.theta = h[j].theta;
      st.sigma2 = h[j].sigma2;
      st.eta2 = h[j].eta2;
      st.elapsed_ms = ms;
    }
  sc.finish();
}

// ms_reconstruct_two_step_batch / ms_reconstruct_single_step_batch
template <typename R>
void reconstruct_batch(ms_plan* p, bool two, int njobs, const int32_t* chans,
                       const void* const* vis, const ms_recon_opts* o, void* const* low_out,
                       void* const* img_out, ms_stats* stats, void* stream) {
  check_batchable(p);
  validate_opts(o);
  arg(o->warm_start == nullptr, "the batched calls take no warm start network");
  arg(njobs >= 1 && njobs <= 4096, "njobs must be 1..4096");
  arg(chans && vis && img_out && (!two || low_out), "a required array is NULL");
  for (int j = 0; j < njobs; ++j) {
    arg(chans[j] >= 0 && chans[j] < (int)p->ch.size(), "channel out of range");
    arg(vis[j] && img_out[j] && (!two || low_out[j]), "a job's buffer is NULL");
    const ChanDev& c = p->ch[chans[j]];
    if (two)
      arg(c.part[MS_PART_L].n > 0 && c.part[MS_PART_H].n > 0,
          "both partitions need visibilities");
    else
      arg(c.part[MS_PART_ALL].n > 0, "no visibilities");
  }
  Scope sc(p, stream);
  if (stats) std::memset(stats, 0, sizeof(ms_stats) * njobs);
  ensure_fista_batch<R>(p, njobs, o->fista_iters);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ck(cudaEventCreate(&e0), "event");
  ck(cudaEventCreate(&e1), "event");
  ck(cudaEventRecord(e0, p->ps), "event");
  if (two) {
    run_step_batch<R>(p, MS_STEP_LOW, njobs, chans, vis, *o, nullptr, low_out, stats);
    run_step_batch<R>(p, MS_STEP_FULL, njobs, chans, vis, *o, (const void* const*)low_out,
                      img_out, stats);
  } else {
    run_step_batch<R>(p, MS_STEP_SINGLE, njobs, chans, vis, *o, nullptr, img_out, stats);
  }
  ck(cudaEventRecord(e1, p->ps), "event");
  check_device_error(p);
  float ms = 0;
  ck(cudaEventSynchronize(e1), "event");
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (stats)
    for (int j = 0; j < njobs; ++j) stats[j].elapsed_ms = ms;
  sc.finish();
}

}  // namespace

// ====================================================================== ABI
// ------------------------------------------ gridding with static scratch
// ms_grid_static_scratch grids with its per-work-item tiles in this
// fixed-size array instead of the plan's scratch buffer.  The array belongs to
// the library's device image: it is reserved when the module is loaded, so the
// call itself obtains no device memory.  Every tile a call uses is written in
// full by the gridding kernel before the fold reads it, so no part of the
// array has to start at zero.  All plans and streams on a device share the
// one array: calls whose executions overlap on a device race on it.
constexpr size_t kStaticGridScratchBytes = (size_t)64 << 20;   // 64 MiB
static __device__ __align__(256) unsigned char g_grid_scratch[kStaticGridScratchBytes];

namespace {
constexpr int kScratchDevices = 64;
std::mutex g_scratch_mu;
void* g_scratch_addr[kScratchDevices] = {};

// device address of g_grid_scratch on the current device `dev`, looked up
// once per device (the lookup may load the module)
void* static_grid_scratch(int dev) {
  arg(dev >= 0 && dev < kScratchDevices, "device ordinal beyond the static scratch table");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* a = nullptr;
    ck(cudaGetSymbolAddress(&a, g_grid_scratch), "static scratch address");
    g_scratch_addr[dev] = a;
  }
  return g_scratch_addr[dev];
}

}  // namespace

// H2^ of every channel and partition for the linear PSF operator: the real
// spectrum of the PSF on a 2N x 2N field with the same pixel size, from a
// temporary plan of side 2N whose partition bounds are 2 ell, 2 delta (the
// radius r = |uv| N dl doubles with N, exactly, so each row falls in the same
// partitions).  d still carries the caller's u, v and flags.
template <typename R> void build_linear_psf(ms_plan* p, const ms_plan_desc* d) {
  ms_plan_desc d2 = *d;
  d2.npix = 2 * d->npix;
  d2.ell_px = 2.0 * d->ell_px;
  d2.delta_px = 2.0 * d->delta_px;
  d2.levels = 1;
  d2.n_bases = 1;
  d2.dictionary = MS_DICT_DAUBECHIES;
  d2.convolution = MS_CONV_CIRCULAR;
  d2.tile = 0;
  d2.chunk = 0;
  ms_plan* q = nullptr;
  const ms_status st = ms_plan_create(&d2, &q);
  if (st != MS_OK) throw Fail{st, "linear PSF operator: the 2N x 2N plan could not be built"};
  const size_t bytes = sizeof(R) * 2 * p->N * (p->N + 1);
  try {
    ck(cudaSetDevice(q->dev), "set device");
    for (size_t c = 0; c < p->ch.size(); ++c)
      for (int pt = 0; pt < 3; ++pt) {
        PartDev& qd = q->ch[c].part[pt];
        ensure_psf<R>(q, qd);
        PartDev& pd = p->ch[c].part[pt];
        pd.Hhat2 = p->alloc<R>(bytes / sizeof(R), "linear PSF spectrum");
        ck(cudaMemcpyAsync(pd.Hhat2, qd.Hhat, bytes, cudaMemcpyDeviceToDevice, q->ps), "copy");
        ck(cudaStreamSynchronize(q->ps), "synchronize");
      }
  } catch (...) {
    destroy(q);
    throw;
  }
  destroy(q);
}

extern "C" {

ms_status ms_plan_create(const ms_plan_desc* d, ms_plan** out) {
  if (!out) return MS_ERR_ARG;
  *out = nullptr;
  if (!d) return MS_ERR_ARG;
  ms_plan* p = new (std::nothrow) ms_plan();
  if (!p) return MS_ERR_OOM;
  ms_status st = guarded(p, [&] {
    arg(d->u && d->v, "u and v are required");
    arg(d->nvis >= 1 && d->nvis < (int64_t)INT32_MAX, "nvis must be 1 .. 2^31-1");
    arg(d->nchan >= 1, "nchan must be >= 1");
    arg(d->kernel_width == 7, "only kernel_width = 7 is supported");
    arg(d->oversample == 2, "only oversample = 2 is supported");
    arg(d->dictionary == MS_DICT_DAUBECHIES || d->dictionary == MS_DICT_IUWT,
        "unknown dictionary");
    arg(d->dictionary == MS_DICT_IUWT || (d->n_bases >= 1 && d->n_bases <= kMaxBases),
        "n_bases must be 1..8");
    arg(d->levels >= 1 && d->levels <= kMaxLevels, "levels must be 1..8");
    arg(d->npix >= 16 && d->npix % 16 == 0 && d->npix <= 16384, "npix must be a multiple of 16");
    arg(d->npix % (1 << d->levels) == 0 && (d->npix >> d->levels) >= 1,
        "npix must be divisible by 2^levels");
    arg(d->pixel_size > 0 && std::isfinite(d->pixel_size), "pixel_size must be > 0");
    arg(d->delta_px > 0 && std::isfinite(d->ell_px), "delta must be > 0 and ell finite");
    arg(d->precision >= MS_FP64 && d->precision <= MS_FP32_KAHAN, "unknown precision");
    arg(d->convolution == MS_CONV_CIRCULAR || d->convolution == MS_CONV_LINEAR,
        "unknown convolution");
    arg(d->convolution == MS_CONV_CIRCULAR ||
            (d->dictionary == MS_DICT_DAUBECHIES && d->npix <= 8192),
        "the linear PSF operator needs the Daubechies dictionary and npix <= 8192");
    p->d = *d;
    p->d.u = p->d.v = nullptr;
    p->d.flags = nullptr;
    p->dev = d->device;
    DeviceGuard guard;   // the caller's device is current again on every exit
    ck(cudaSetDevice(p->dev), "set device");
    p->N = d->npix;
    p->Ng = 2 * d->npix;
    // default tile side 16: the gridder's warp-private sub-tiles are then a
    // third the size, so several times more warps fit per SM (measured at
    // 1024^2, 9.27M rows, FP32: grid 334 vs 460 us, fold 84 vs 115 us)
    p->T = d->tile ? d->tile : 16;
    arg(p->T == 16 || p->T == 32, "tile must be 16 or 32");
    arg(p->Ng % p->T == 0, "grid side must be a multiple of the tile");
    p->S = p->T + kW - 1;
    p->ntx = p->Ng / p->T;
    p->ntiles = p->ntx * p->ntx;
    p->J = d->levels;
    p->dict = d->dictionary;
    p->M = p->dict == MS_DICT_IUWT ? d->levels + 1 : d->n_bases;   // coefficient planes
    p->prec = d->precision;
    p->conv = d->convolution;
    p->rsz = p->prec == MS_FP64 ? 8 : 4;
    p->beta = d->es_beta > 0 ? d->es_beta : 2.30 * kW;
    if (d->chunk > 0) {
      p->chunk = d->chunk;
    } else {
      const int64_t per = (int64_t)sm_count() * 8;   // about 8 work items per SM
      int64_t c = (d->nvis + per - 1) / per;
      p->chunk = (int)std::min<int64_t>(std::max<int64_t>(c, 512), 8192);
    }
    ck(cudaStreamCreateWithFlags(&p->ps, cudaStreamNonBlocking), "stream");
    ck(cudaEventCreateWithFlags(&p->ev_in, cudaEventDisableTiming), "event");
    ck(cudaEventCreateWithFlags(&p->ev_out, cudaEventDisableTiming), "event");
    DISPATCH(p, build_plan<R>(p, d));
    if (p->conv == MS_CONV_LINEAR) DISPATCH(p, build_linear_psf<R>(p, d));
  });
  if (st != MS_OK) {
    fprintf(stderr, "ms_plan_create: %s\n", p->msg.c_str());
    destroy(p);
    return st;
  }
  *out = p;
  return MS_OK;
}

ms_status ms_plan_destroy(ms_plan* plan) {
  if (!plan) return MS_ERR_ARG;
  destroy(plan);
  return MS_OK;
}

const char* ms_last_error(const ms_plan* plan) { return plan ? plan->msg.c_str() : "no plan"; }

ms_status ms_partition_counts(ms_plan* p, int32_t chan, int64_t out[4]) {
  return guarded(p, [&] {
    arg(out != nullptr, "out is NULL");
    arg(chan >= 0 && chan < (int)p->ch.size(), "channel out of range");
    for (int i = 0; i < 4; ++i) out[i] = p->ch[chan].counts[i];
  });
}

ms_status ms_partition_layout(ms_plan* p, int32_t part, int32_t chan, int64_t out[3]) {
  return guarded(p, [&] {
    arg(out != nullptr, "out is NULL");
    PartDev& pd = part_of(p, part, chan);
    out[0] = pd.nitems;
    out[1] = (int64_t)p->S * p->S;
    out[2] = (int64_t)grid_scratch_cell_bytes(p->prec);
  });
}

ms_status ms_partition_rows(ms_plan* p, int32_t part, int32_t chan, int32_t* rows) {
  return guarded(p, [&] {
    PartDev& pd = part_of(p, part, chan);
    arg(rows != nullptr || pd.n == 0, "rows is NULL");
    DeviceGuard guard;
    ck(cudaSetDevice(p->dev), "set device");
    if (pd.n) ck(cudaMemcpy(rows, pd.idx, sizeof(int32_t) * pd.n, cudaMemcpyDeviceToHost), "copy");
  });
}

ms_status ms_degrid(ms_plan* p, int32_t part, int32_t chan, const void* image,
                    const void* vis_obs, void* vis_out, void* stream) {
  return guarded(p, [&] {
    PartDev& pd = part_of(p, part, chan);
    arg(image && vis_out, "image and vis_out are required");
    Scope sc(p, stream);
    DISPATCH(p, {
      if (vis_obs)
        launch_gather_vis<R>(pd.idx, pd.n, (const C2<R>*)vis_obs, (C2<R>*)p->vis_a, p->ps);
      image_to_grid<R>(p, image, nullptr);
      degrid_sorted<R>(p, pd, vis_obs ? p->vis_a : nullptr, p->vis_b, nullptr);
      launch_scatter_vis<R>(pd.idx, pd.n, (const C2<R>*)p->vis_b, (C2<R>*)vis_out, p->ps);
    });
    check_device_error(p);
    sc.finish();
  });
}

ms_status ms_grid(ms_plan* p, int32_t part, int32_t chan, const void* vis, void* dirty,
                  void* stream) {
  return guarded(p, [&] {
    PartDev& pd = part_of(p, part, chan);
    arg(vis && dirty, "vis and dirty are required");
    Scope sc(p, stream);
    DISPATCH(p, {
      launch_gather_vis<R>(pd.idx, pd.n, (const C2<R>*)vis, (C2<R>*)p->vis_a, p->ps);
      grid_sorted<R>(p, pd, p->vis_a, dirty, nullptr);
    });
    sc.finish();
  });
}

ms_status ms_residual_image(ms_plan* p, int32_t part, int32_t chan, const void* vis_obs,
                            const void* model, void* out, void* stream) {
  return guarded(p, [&] {
    PartDev& pd = part_of(p, part, chan);
    arg(vis_obs && model && out, "vis_obs, model and out are required");
    Scope sc(p, stream);
    DISPATCH(p, {
      launch_gather_vis<R>(pd.idx, pd.n, (const C2<R>*)vis_obs, (C2<R>*)p->vis_a, p->ps);
      residual_sorted<R>(p, pd, p->vis_a, model, out, nullptr);
    });
    check_device_error(p);
    sc.finish();
  });
}

ms_status ms_psf(ms_plan* p, int32_t part, int32_t chan, void* psf, void* stream) {
  return guarded(p, [&] {
    PartDev& pd = part_of(p, part, chan);
    arg(psf != nullptr, "psf is NULL");
    Scope sc(p, stream);
    DISPATCH(p, psf_image<R>(p, pd, psf));
    check_device_error(p);
    sc.finish();
  });
}

ms_status ms_dictionary_synthesis(ms_plan* p, const void* alpha, void* x, void* stream) {
  return guarded(p, [&] {
    arg(alpha && x, "alpha and x are required");
    Scope sc(p, stream);
    DISPATCH(p, dict_synthesis<R>(p, (const R*)alpha, (R*)x));
    sc.finish();
  });
}

ms_status ms_dictionary_analysis(ms_plan* p, const void* x, void* alpha, void* stream) {
  return guarded(p, [&] {
    arg(alpha && x, "alpha and x are required");
    Scope sc(p, stream);
    DISPATCH(p, dict_analysis<R>(p, (const R*)x, (R*)alpha));
    sc.finish();
  });
}

ms_status ms_sigma2_hat(ms_plan* p, const void* image, double* sigma2, void* stream) {
  return guarded(p, [&] {
    arg(image && sigma2, "image and sigma2 are required");
    Scope sc(p, stream);
    DISPATCH(p, launch_sigma2_hat<R>((const R*)image, p->N, p->parts, p->ctl, p->tickets + 6, 1,
                                     p->ps));
    FistaCtl h{};
    ck(cudaMemcpyAsync(&h, p->ctl, sizeof(h), cudaMemcpyDeviceToHost, p->ps), "read ctl");
    ck(cudaStreamSynchronize(p->ps), "synchronize");
    *sigma2 = h.sigma2;
    sc.finish();
  });
}

ms_status ms_lipschitz(ms_plan* p, int32_t step, int32_t chan, double sigma2, double eta2,
                       int32_t power_iters, double* theta_closed, double* theta_power,
                       void* stream) {
  return guarded(p, [&] {
    arg(step >= MS_STEP_LOW && step <= MS_STEP_FULL_L, "unknown step");
    arg(!step_full(step) || (sigma2 > 0 && eta2 > 0), "FULL needs sigma2, eta2 > 0");
    Scope sc(p, stream);
    DISPATCH(p, lipschitz<R>(p, step, chan, sigma2, eta2, power_iters, theta_closed,
                             theta_power));
    sc.finish();
  });
}

ms_status ms_minor_cycle(ms_plan* p, int32_t step, int32_t chan, const void* residual,
                         const void* l_low, double sigma2, double eta2, double lambda,
                         int32_t max_iters, double rel_tol, void* beta_inout, void* model_out,
                         ms_stats* st, void* stream) {
  return guarded(p, [&] {
    arg(step >= MS_STEP_LOW && step <= MS_STEP_FULL_L, "unknown step");
    arg(!step_full(step) || (sigma2 > 0 && eta2 > 0), "FULL needs sigma2, eta2 > 0");
    arg(rel_tol >= 0, "rel_tol must be >= 0");
    if (st) std::memset(st, 0, sizeof(*st));
    Scope sc(p, stream);
    DISPATCH(p, minor_cycle<R>(p, step, chan, residual, l_low, sigma2, eta2, lambda, max_iters,
                               rel_tol, beta_inout, model_out, st));
    sc.finish();
  });
}

ms_status ms_reconstruct_two_step(ms_plan* p, int32_t chan, const void* vis,
                                  const ms_recon_opts* o, void* low_out, void* img_out,
                                  void* model_out, ms_stats* st, void* stream) {
  return guarded(p, [&] {
    validate_opts(o);
    arg(vis && low_out && img_out, "vis, img_low_out and img_out are required");
    arg(chan >= 0 && chan < (int)p->ch.size(), "channel out of range");
    arg(p->ch[chan].part[MS_PART_L].n > 0 && p->ch[chan].part[MS_PART_H].n > 0,
        "both partitions need visibilities");
    DISPATCH(p, two_step<R>(p, chan, vis, o, low_out, img_out, model_out, st, stream));
  });
}

ms_status ms_reconstruct_step(ms_plan* p, int32_t step, int32_t chan, const void* vis,
                              const ms_recon_opts* o, const void* low_image, void* img_out,
                              void* model_out, ms_stats* st, void* stream) {
  return guarded(p, [&] {
    validate_opts(o);
    arg(step == MS_STEP_LOW || step == MS_STEP_FULL || step == MS_STEP_SINGLE,
        "step must be LOW, FULL or SINGLE");
    arg(vis && img_out, "vis and img_out are required");
    arg(step != MS_STEP_FULL || low_image != nullptr, "FULL needs the previous step's image");
    arg(o->warm_start == nullptr, "the warm start belongs to ms_reconstruct_two_step");
    arg(chan >= 0 && chan < (int)p->ch.size(), "channel out of range");
    arg(p->ch[chan].part[step_part(step)].n > 0, "the step's partition has no visibilities");
    DISPATCH(p, one_step<R>(p, step, chan, vis, o, low_image, img_out, model_out, st, stream));
  });
}

ms_status ms_reconstruct_single_step(ms_plan* p, int32_t chan, const void* vis,
                                     const ms_recon_opts* o, void* img_out, void* model_out,
                                     ms_stats* st, void* stream) {
  return guarded(p, [&] {
    validate_opts(o);
    arg(vis && img_out, "vis and img_out are required");
    arg(chan >= 0 && chan < (int)p->ch.size(), "channel out of range");
    arg(p->ch[chan].part[MS_PART_ALL].n > 0, "no visibilities");
    DISPATCH(p, single_step<R>(p, chan, vis, o, img_out, model_out, st, stream));
  });
}

ms_status ms_lambda(ms_plan* p, int32_t rule, double coef, int32_t n, const void* residual,
                    double* lambda, void* stream) {
  return guarded(p, [&] {
    arg(residual && lambda, "residual and lambda are required");
    arg(rule == MS_LAMBDA_NORM2_2N || rule == MS_LAMBDA_MAX_FIXED, "unknown lambda rule");
    arg(n >= 1 && n <= 1000, "n must be 1..1000");
    arg(std::isfinite(coef), "coef must be finite");
    Scope sc(p, stream);
    const int64_t n2 = (int64_t)p->N * p->N;
    DISPATCH(p, launch_image_norms<R>((const R*)residual, n2, p->parts, p->ctl, p->tickets + 5,
                                      p->ps));
    launch_set_lambda(p->ctl, rule, coef, n, 1, p->ps);
    ck(cudaMemcpyAsync(lambda, &p->ctl->lam, sizeof(double), cudaMemcpyDeviceToHost, p->ps),
       "read lambda");
    ck(cudaStreamSynchronize(p->ps), "synchronize");
    sc.finish();
  });
}

ms_status ms_warm_start_coefficients(ms_plan* p, ms_unet* net, const void* low_image,
                                     const void* residual_h1, void* beta_out, void* x0_out,
                                     void* stream) {
  return guarded(p, [&] {
    arg(low_image && residual_h1 && beta_out, "low_image, residual_h1 and beta_out are required");
    Scope sc(p, stream);
    DISPATCH(p, warm_start_beta<R>(p, net, low_image, residual_h1, beta_out, x0_out));
    sc.finish();
  });
}

ms_status ms_set_objective_target(ms_plan* p, double target) {
  return guarded(p, [&] {
    arg(!std::isnan(target), "target must not be NaN (use -inf to turn it off)");
    p->obj_target = std::isfinite(target) ? target : -INFINITY;
  });
}

ms_status ms_set_profiling(ms_plan* p, int32_t on) {
  return guarded(p, [&] {
    DeviceGuard guard;
    ck(cudaSetDevice(p->dev), "set device");
    harvest(p);
    p->prof = on != 0;
  });
}

ms_status ms_get_kernel_profile(ms_plan* p, ms_kernel_profile* out, int32_t reset) {
  return guarded(p, [&] {
    arg(out != nullptr, "out is NULL");
    DeviceGuard guard;
    ck(cudaSetDevice(p->dev), "set device");
    ck(cudaStreamSynchronize(p->ps), "synchronize");
    harvest(p);
    std::memset(out, 0, sizeof(*out));
    for (int i = 0; i < MS_K_COUNT; ++i) {
      out->launches[i] = p->k_launch[i];
      out->total_ms[i] = p->k_ms[i];
    }
    if (reset)
      for (int i = 0; i < 16; ++i) {
        p->k_launch[i] = 0;
        p->k_ms[i] = 0;
      }
  });
}

ms_status ms_grid_static_scratch(ms_plan* p, int32_t part, int32_t chan, const void* vis,
                                 void* dirty, void* stream) {
  return guarded(p, [&] {
    PartDev& pd = part_of(p, part, chan);
    arg(vis && dirty, "vis and dirty are required");
    const size_t need =
        (size_t)pd.nitems * p->S * p->S * grid_scratch_cell_bytes(p->prec);
    if (need > kStaticGridScratchBytes) {
      char buf[192];
      std::snprintf(buf, sizeof(buf),
                    "the partition needs %zu bytes of gridding scratch; the static scratch "
                    "holds %zu bytes (use ms_grid)",
                    need, kStaticGridScratchBytes);
      throw Fail{MS_ERR_ARG, buf};
    }
    Scope sc(p, stream);
    void* scratch = static_grid_scratch(p->dev);
    DISPATCH(p, {
      launch_gather_vis<R>(pd.idx, pd.n, (const C2<R>*)vis, (C2<R>*)p->vis_a, p->ps);
      grid_sorted<R>(p, pd, p->vis_a, dirty, nullptr, scratch);
    });
    sc.finish();
  });
}

ms_status ms_grid_batch(ms_plan* p, int32_t njobs, const int32_t* chans, const int32_t* parts,
                        const void* const* vis, void* const* dirty, void* stream) {
  return guarded(p, [&] {
    Scope sc(p, stream);
    DISPATCH(p, grid_batch<R>(p, njobs, chans, parts, vis, dirty));
    sc.finish();
  });
}

ms_status ms_minor_cycle_batch(ms_plan* p, int32_t njobs, const int32_t* steps,
                               const int32_t* chans, const void* const* residuals,
                               const void* const* l_lows, const double* lambdas,
                               const double* sigma2s, const double* eta2s, int32_t max_iters,
                               double rel_tol, void* const* models_out, ms_stats* stats,
                               double* traces, void* stream) {
  return guarded(p, [&] {
    arg(rel_tol >= 0, "rel_tol must be >= 0");
    if (stats && njobs > 0) std::memset(stats, 0, sizeof(ms_stats) * njobs);
    Scope sc(p, stream);
    DISPATCH(p, minor_cycle_batch<R>(p, njobs, steps, chans, residuals, l_lows, lambdas, sigma2s,
                                     eta2s, max_iters, rel_tol, models_out, stats, traces));
    sc.finish();
  });
}

ms_status ms_reconstruct_two_step_batch(ms_plan* p, int32_t njobs, const int32_t* chans,
                                        const void* const* vis, const ms_recon_opts* o,
                                        void* const* low_out, void* const* img_out,
                                        ms_stats* stats, void* stream) {
  return guarded(p, [&] {
    DISPATCH(p, reconstruct_batch<R>(p, true, njobs, chans, vis, o, low_out, img_out, stats,
                                     stream));
  });
}

ms_status ms_reconstruct_interleaved(ms_plan* p, int32_t chan, const void* vis,
                                     const ms_recon_opts* o, void* img_out, void* node_l_out,
                                     void* node_h_out, ms_stats* stats, void* stream) {
  return guarded(p, [&] {
    DISPATCH(p, interleaved<R>(p, chan, vis, o, img_out, node_l_out, node_h_out, stats, stream));
  });
}

ms_status ms_reconstruct_single_step_batch(ms_plan* p, int32_t njobs, const int32_t* chans,
                                           const void* const* vis, const ms_recon_opts* o,
                                           void* const* img_out, ms_stats* stats,
                                           void* stream) {
  return guarded(p, [&] {
    DISPATCH(p, reconstruct_batch<R>(p, false, njobs, chans, vis, o, nullptr, img_out, stats,
                                     stream));
  });
}

ms_status ms_degrid_batch(ms_plan* p, int32_t njobs, const int32_t* chans, const int32_t* parts,
                          const void* const* images, const void* const* vis_obs,
                          void* const* vis_out, void* stream) {
  return guarded(p, [&] {
    Scope sc(p, stream);
    DISPATCH(p, degrid_batch<R>(p, njobs, chans, parts, images, vis_obs, vis_out));
    check_device_error(p);
    sc.finish();
  });
}

ms_status ms_plan_autotune(const ms_plan_desc* desc, int32_t chan, int32_t reps,
                           int32_t* best_tile, int32_t* best_chunk, double* best_ms) {
  if (!desc || !best_tile || !best_chunk || chan < 0 || chan >= desc->nchan || reps < 1)
    return MS_ERR_ARG;
  const int tiles[2] = {16, 32};
  const int chunks[5] = {512, 1024, 2048, 4096, 8192};
  double best = 1e300;
  int bt = 0, bc = 0;
  void* vis = nullptr;
  void* img = nullptr;
  void* out = nullptr;
  ms_status st = MS_OK;
  for (int ti = 0; ti < 2 && st == MS_OK; ++ti) {
    if ((2 * desc->npix) % tiles[ti]) continue;
    for (int ci = 0; ci < 5 && st == MS_OK; ++ci) {
      ms_plan_desc d = *desc;
      d.tile = tiles[ti];
      d.chunk = chunks[ci];
      d.convolution = MS_CONV_CIRCULAR;   // the gridding layout only
      ms_plan* q = nullptr;
      st = ms_plan_create(&d, &q);
      if (st != MS_OK) break;
      const size_t rsz = q->rsz;
      if (!vis) {
        if (cudaMalloc(&vis, 2 * rsz * std::max<int64_t>(desc->nvis, 1)) != cudaSuccess ||
            cudaMalloc(&out, 2 * rsz * std::max<int64_t>(desc->nvis, 1)) != cudaSuccess ||
            cudaMalloc(&img, rsz * desc->npix * desc->npix) != cudaSuccess) {
          ms_plan_destroy(q);
          st = MS_ERR_OOM;
          break;
        }
        if (rsz == 8) {
          launch_hash_fill<double>((double*)vis, 2 * desc->nvis, 7, q->ps);
          launch_hash_fill<double>((double*)img, (int64_t)desc->npix * desc->npix, 8, q->ps);
        } else {
          launch_hash_fill<float>((float*)vis, 2 * desc->nvis, 7, q->ps);
          launch_hash_fill<float>((float*)img, (int64_t)desc->npix * desc->npix, 8, q->ps);
        }
        cudaStreamSynchronize(q->ps);
      }
      // one untimed pair, then `reps` timed degrid + grid pairs
      cudaEvent_t e0, e1;
      cudaEventCreate(&e0);
      cudaEventCreate(&e1);
      for (int r = 0; r <= reps && st == MS_OK; ++r) {
        if (r == 1) cudaEventRecord(e0, q->ps);
        st = ms_degrid(q, MS_PART_ALL, chan, img, nullptr, out, q->ps);
        if (st == MS_OK) st = ms_grid(q, MS_PART_ALL, chan, vis, img, q->ps);
      }
      cudaEventRecord(e1, q->ps);
      cudaEventSynchronize(e1);
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      ms_plan_destroy(q);
      if (st == MS_OK && ms / reps < best) {
        best = ms / reps;
        bt = tiles[ti];
        bc = chunks[ci];
      }
    }
  }
  for (void* a : {vis, img, out})
    if (a) cudaFree(a);
  if (st != MS_OK) return st;
  *best_tile = bt;
  *best_chunk = bc;
  if (best_ms) *best_ms = best;
  return MS_OK;
}

}  // extern "C"
