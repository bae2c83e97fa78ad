// Fourier-domain pieces of the minor cycle and the FP64 reductions.
//
// Both problems are quadratic in x = W alpha (Sect. 3.2, 3.3):
//   f(alpha) = <x, K x> - 2 <b, x> + c0,
//   LOW / SINGLE (Eq. LowRes):  K^ = |H^|^2,              B^ = H^ I^,
//                               c0 = ||i~||^2
//   FULL (Eq. FullRes):         K^ = g_H^2 |H^|^2 + g_L^2, B^ = g_H^2 H^ I^ + g_L^2 L^,
//                               c0 = ||G_H i~||^2 + ||G_L l||^2
// with H^ the (real) PSF spectrum and I^, L^ the spectra of i~ and l_L, so the
// gradient of Eqs. GradL / GradH is 2 W^H (K x - b) and the Lipschitz constant
// of Sect. 3.4 is 2 M max K^.  Inner products use Parseval on the rfft
// half-plane (columns 0 and N/2 once, the others twice).  Reductions sum
// compensated working-precision pairs within warps; across warps and blocks
// they sum FP64 partials (or, in the fused spectral step, FP32 (hi, lo)
// pairs, since the FP64 pipe is slow) in a fixed order.
//
// For N a power of two the FISTA pass's spectral step is three kernels of
// this file: real row transforms, the column transforms fused with the
// spectral multiply and the objective terms, and the inverse row transforms
// (whose extra block runs the iteration control); other N use 2-D cuFFT
// transforms around spec_mul_kernel.
#include "common.cuh"

namespace ms {

namespace {
constexpr int kThreads = 256;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return v;
}

// block reduction of NV doubles (sum or max per slot); result in thread 0
// (blockDim.x a multiple of 32)
template <int NV>
__device__ void block_reduce(double (&v)[NV], const bool (&is_max)[NV]) {
  __shared__ double red[NV][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = is_max[i] ? warp_max(v[i]) : warp_sum(v[i]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) red[i][warp] = v[i];
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      double s = is_max[i] ? -INFINITY : 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w)
        s = is_max[i] ? fmax(s, red[i][w]) : s + red[i][w];
      v[i] = s;
    }
  }
}

// write this block's partials; returns true in every thread of the last block
template <int NV>
__device__ bool publish_partials(const double (&v)[NV], double* parts, int32_t* ticket) {
  __shared__ int last;
  if (threadIdx.x == 0) {
#pragma unroll
    for (int i = 0; i < NV; ++i) parts[(int64_t)i * gridDim.x + blockIdx.x] = v[i];
    __threadfence();
    int prior = atomicAdd(ticket, 1);
    last = (prior == (int)gridDim.x - 1);
  }
  __syncthreads();
  return last != 0;
}

// the last block combines all partials: thread t takes blocks t, t+256, ...
// then a fixed shuffle tree; the result is valid in thread 0
template <int NV>
__device__ void gather_partials(double (&out)[NV], const double* parts, const bool (&is_max)[NV],
                                int32_t* ticket) {
  __threadfence();
  // L2-coherent loads (the writers fenced before taking their ticket); they
  // are independent, so a thread keeps all of them in flight at once
  double v[NV];
#pragma unroll
  for (int i = 0; i < NV; ++i) v[i] = is_max[i] ? -INFINITY : 0.0;
  const int G = (int)gridDim.x;
  for (int b0 = threadIdx.x; b0 < G; b0 += 4 * blockDim.x) {
    double x[NV][4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int b = b0 + u * blockDim.x;
#pragma unroll
      for (int i = 0; i < NV; ++i)
        x[i][u] = b < G ? __ldcg(parts + (int64_t)i * G + b) : (is_max[i] ? -INFINITY : 0.0);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int i = 0; i < NV; ++i) v[i] = is_max[i] ? fmax(v[i], x[i][u]) : v[i] + x[i][u];
  }
  block_reduce<NV>(v, is_max);
#pragma unroll
  for (int i = 0; i < NV; ++i) out[i] = v[i];
  if (threadIdx.x == 0) *ticket = 0;
}

__device__ __forceinline__ double half_plane_weight(int col, int N) {
  return (col == 0 || col == N / 2) ? 1.0 : 2.0;
}

int nparts_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b > sm_count() * 4) b = sm_count() * 4;
  if (b < 1) b = 1;
  return (int)b;
}
}  // namespace

int spectral_partials(int N) { return nparts_for((int64_t)N * (N / 2 + 1)); }

// ------------------------------------------------------------- PSF spectrum
template <typename R>
__global__ void ifftshift_kernel(const R* __restrict__ in, R* __restrict__ out, int N) {
  int64_t total = (int64_t)N * N;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int p = (int)(k / N), q = (int)(k % N);
    int sp = p + N / 2, sq = q + N / 2;
    sp -= sp >= N ? N : 0;
    sq -= sq >= N ? N : 0;
    out[k] = in[(int64_t)sp * N + sq];
  }
}

template <typename R>
void launch_ifftshift_real(const R* in, R* out, int N, cudaStream_t s) {
  ifftshift_kernel<R><<<nparts_for((int64_t)N * N), kThreads, 0, s>>>(in, out, N);
}

template <typename R>
__global__ void real_part_kernel(const C2<R>* __restrict__ in, R* __restrict__ out, int n) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x)
    out[k] = in[k].x;
}

template <typename R>
void launch_real_part_spectrum(const C2<R>* in, R* out, int n, cudaStream_t s) {
  real_part_kernel<R><<<nparts_for(n), kThreads, 0, s>>>(in, out, n);
}

// ------------------------------------------------------------- filters
// Sect. 3.3: |g_H|^2 = 1/sigma^2 above ell + delta, 0 below ell - delta;
// |g_L|^2 = 1/eta^2 below, 0 above; in the band g_L = a (1 - s), g_H = a (1 + s),
// s = sin(pi (r - ell) / (2 delta)), a = 1/sqrt(eta^2 (1-s)^2 + sigma^2 (1+s)^2).
// r = sqrt(kx^2 + ky^2) on the rfft half-plane, pixel units.  Squares stored.
template <typename R>
__global__ void filters_kernel(int N, double ell, double delta, const FistaCtl* __restrict__ ctl,
                               R* __restrict__ gl2, R* __restrict__ gh2, int mirror) {
  const int nc = N / 2 + 1;
  const int64_t total = (int64_t)N * nc;
  // mirror: the sides exchanged (sigma^2 and eta^2 swapped, data weights on
  // the low side into gh2, prior weights on the high side into gl2)
  const double s2 = mirror ? ctl->eta2 : ctl->sigma2, e2 = mirror ? ctl->sigma2 : ctl->eta2;
  const double pi = 3.141592653589793238462643383279502884;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int row = (int)(k / nc), col = (int)(k % nc);
    double ky = row < N / 2 ? row : row - N;
    double r = sqrt(ky * ky + (double)col * col);
    double l2, h2;
    if (r > ell + delta) {
      l2 = 0.0;
      h2 = 1.0 / s2;
    } else if (r < ell - delta) {
      l2 = 1.0 / e2;
      h2 = 0.0;
    } else {
      double sn = sin(pi * (r - ell) / (2.0 * delta));
      double a2 = 1.0 / (e2 * (1.0 - sn) * (1.0 - sn) + s2 * (1.0 + sn) * (1.0 + sn));
      l2 = a2 * (1.0 - sn) * (1.0 - sn);
      h2 = a2 * (1.0 + sn) * (1.0 + sn);
    }
    gl2[k] = (R)(mirror ? h2 : l2);
    gh2[k] = (R)(mirror ? l2 : h2);
  }
}

template <typename R>
void launch_filters(int N, double ell, double delta, const FistaCtl* ctl, R* gl2, R* gh2,
                    cudaStream_t s, int mirror) {
  filters_kernel<R><<<spectral_partials(N), kThreads, 0, s>>>(N, ell, delta, ctl, gl2, gh2,
                                                              mirror);
}

// a = (eta^2 g_L^2 a + sigma^2 g_H^2 b) / N^2 on the half-plane (sigma^2, eta^2
// from ctl, g_L^2, g_H^2 the unscaled filters of launch_filters): the
// interleaved pipeline's combination of its two nodes' images
template <typename R>
__global__ void combine_spectra_kernel(C2<R>* __restrict__ a, const C2<R>* __restrict__ b,
                                       const R* __restrict__ gl2, const R* __restrict__ gh2,
                                       const FistaCtl* __restrict__ ctl, int N) {
  const int64_t total = (int64_t)N * (N / 2 + 1);
  const double inv = 1.0 / ((double)N * N);
  const R cl = (R)(ctl->eta2 * inv), ch = (R)(ctl->sigma2 * inv);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const R wl = cl * gl2[k], wh = ch * gh2[k];
    const C2<R> x = a[k], y = b[k];
    C2<R> o;
    o.x = wl * x.x + wh * y.x;
    o.y = wl * x.y + wh * y.y;
    a[k] = o;
  }
}

template <typename R>
void launch_combine_spectra(C2<R>* a, const C2<R>* b, const R* gl2, const R* gh2,
                            const FistaCtl* ctl, int N, cudaStream_t s) {
  combine_spectra_kernel<R><<<spectral_partials(N), kThreads, 0, s>>>(a, b, gl2, gh2, ctl, N);
}

// ------------------------------------------------------------- K^ and theta
template <typename R>
__global__ void normal_spectrum_kernel(const R* __restrict__ Hhat, const R* __restrict__ gl2,
                                       const R* __restrict__ gh2, int N, int M,
                                       R* __restrict__ Ks, double* __restrict__ parts,
                                       FistaCtl* __restrict__ ctl, int32_t* ticket) {
  const int64_t total = (int64_t)N * (N / 2 + 1);
  const double inv = 1.0 / ((double)N * N);
  double v[1] = {0.0};
  const bool mx[1] = {true};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    double h = (double)Hhat[k];
    double kk = h * h;
    if (gl2) kk = (double)gh2[k] * kk + (double)gl2[k];
    Ks[k] = (R)(kk * inv);
    v[0] = fmax(v[0], kk);
  }
  block_reduce<1>(v, mx);
  if (publish_partials<1>(v, parts, ticket)) {
    double o[1];
    gather_partials<1>(o, parts, mx, ticket);
    if (threadIdx.x == 0) {
      ctl->kmax = o[0];
      ctl->theta = 2.0 * M * o[0];
      ctl->inv_theta = o[0] > 0 ? 1.0 / (2.0 * M * o[0]) : 0.0;
    }
  }
}

template <typename R>
void launch_normal_spectrum(const R* Hhat, const R* gl2, const R* gh2, int N, int M, R* Ks,
                            double* parts, FistaCtl* ctl, int32_t* ticket, cudaStream_t s) {
  normal_spectrum_kernel<R><<<spectral_partials(N), kThreads, 0, s>>>(Hhat, gl2, gh2, N, M, Ks,
                                                                      parts, ctl, ticket);
}

// ------------------------------------------------------------- b and c0
template <typename R>
__global__ void b_spectrum_kernel(const C2<R>* __restrict__ Ihat, const C2<R>* __restrict__ Lhat,
                                  const R* __restrict__ Hhat, const R* __restrict__ gl2,
                                  const R* __restrict__ gh2, int N, C2<R>* __restrict__ Bs,
                                  double* __restrict__ parts, FistaCtl* __restrict__ ctl,
                                  int32_t* ticket) {
  const int nc = N / 2 + 1;
  const int64_t total = (int64_t)N * nc;
  const double inv = 1.0 / ((double)N * N);
  double v[1] = {0.0};
  const bool mx[1] = {false};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double w = half_plane_weight((int)(k % nc), N);
    C2<R> I = Ihat[k];
    double h = (double)Hhat[k];
    double br, bi, c;
    if (gl2) {
      C2<R> Lv = Lhat[k];
      double gh = (double)gh2[k], gl = (double)gl2[k];
      br = gh * h * I.x + gl * Lv.x;
      bi = gh * h * I.y + gl * Lv.y;
      c = gh * ((double)I.x * I.x + (double)I.y * I.y) + gl * ((double)Lv.x * Lv.x + (double)Lv.y * Lv.y);
    } else {
      br = h * I.x;
      bi = h * I.y;
      c = (double)I.x * I.x + (double)I.y * I.y;
    }
    C2<R> o;
    o.x = (R)(br * inv);
    o.y = (R)(bi * inv);
    Bs[k] = o;
    v[0] += w * c;
  }
  block_reduce<1>(v, mx);
  if (publish_partials<1>(v, parts, ticket)) {
    double o[1];
    gather_partials<1>(o, parts, mx, ticket);
    if (threadIdx.x == 0) {
      ctl->c0 = o[0] * inv;
    }
  }
}

template <typename R>
void launch_b_spectrum(const C2<R>* Ihat, const C2<R>* Lhat, const R* Hhat, const R* gl2,
                       const R* gh2, int N, C2<R>* Bs, double* parts, FistaCtl* ctl,
                       int32_t* ticket, cudaStream_t s) {
  b_spectrum_kernel<R><<<spectral_partials(N), kThreads, 0, s>>>(Ihat, Lhat, Hhat, gl2, gh2, N,
                                                                 Bs, parts, ctl, ticket);
}

// ------------------------------------------------------------- FISTA spectrum
// One pass of the minor cycle in the Fourier domain.  X^_k = rfft(W B_k) gives
// <x_k, K x_k> and <b, x_k> (Parseval) for the objective of B_k; FISTA's
// extrapolation alpha_k = B_k + t_k (B_k - B_{k-1}) is linear, so its gradient
// image 2 (K W alpha_k - b) is the inverse transform of
//   S^ = 2 (K^/N^2 ((1 + t_k) X^_k - t_k X^_{k-1}) - B^/N^2),
// which this kernel writes over X^_{k-1} (no longer needed).  The last block
// assembles F(B_k) = <x,Kx> - 2<b,x> + c0 + lambda ||B_k||_1 (the l1 norm
// from the n_l1 per-block partials the previous analysis pass left), appends
// it to the trace, raises `done` on convergence or at the iteration budget,
// and otherwise advances the iteration index to k + 1 for the analysis pass
// that builds B_{k+1}.
// Block sums of a spectral step (blockDim.x a multiple of 32): the
// objective's two quadratic terms (working-precision pairs (s, -c), combined
// error-free within each warp, FP64 once per warp) and the l1 partials the
// previous analysis pass left (only the first blocks hold some; has_l1 is
// uniform over the block); the result is valid in thread 0.
template <typename R>
__device__ void spec_block_sums(R s0, R c0, R s1, R c1, double l1s, bool has_l1,
                                double (&v)[3]) {
  __shared__ double red3[3][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  R lo0 = -c0, lo1 = -c1;
  warp_sum_comp<R>(s0, lo0);
  warp_sum_comp<R>(s1, lo1);
  double w2 = 0.0;
  if (has_l1) w2 = warp_sum(l1s);
  if (lane == 0) {
    red3[0][warp] = (double)s0 + (double)lo0;
    red3[1][warp] = (double)s1 + (double)lo1;
    red3[2][warp] = w2;
  }
  __syncthreads();
  v[0] = v[1] = v[2] = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
      v[0] += red3[0][q];
      v[1] += red3[1][q];
      v[2] += red3[2][q];
    }
}

// Iteration control from the summed terms o = (<x,Kx>, <b,x>, ||B_k||_1)
// (one thread): F(B_k) = <x,Kx> - 2<b,x> + c0 + lambda ||B_k||_1 goes to the
// trace; `done` rises on a non-finite F, on convergence (relative change, or
// F at or below the objective target), or at the iteration budget, else the
// iteration index, the momentum t_(k+1) and the step scalars advance.
__device__ void spec_control(const double (&o)[3], FistaCtl* ctl, double* trace) {
  const int k = ctl->k;
  const double lam = ctl->lam, Fprev = ctl->F_cur, rtol = ctl->rel_tol;
  const double inv_theta = ctl->inv_theta;
  const double l1 = o[2];
  double F = o[0] - 2.0 * o[1] + ctl->c0 + lam * l1;
  ctl->l1_cur = l1;
  ctl->xkx = o[0];
  ctl->bx = o[1];
  ctl->F_prev = Fprev;
  ctl->F_cur = F;
  trace[k] = F;
  if (!isfinite(F)) {
    ctl->error = 4;
    ctl->done = 1;
  } else if (k >= 1 && rtol > 0.0 && fabs(F - Fprev) <= rtol * fabs(F)) {
    ctl->converged = 1;
    ctl->done = 1;
  } else if (F <= ctl->F_target) {
    ctl->converged = 1;
    ctl->done = 1;
  } else if (k >= ctl->max_iters) {
    ctl->done = 1;
  } else {
    ctl->k = k + 1;
    const double tn = k + 1 >= 2 ? (double)k / (double)(k + 3) : 0.0;   // t_{k+1}
    ctl->td[(k + 1) & 1] = tn;
    ctl->tf[(k + 1) & 1] = (float)tn;
  }
  ctl->mud = inv_theta;
  ctl->thrd = lam * inv_theta;
  ctl->muf = (float)inv_theta;
  ctl->thrf = (float)(lam * inv_theta);
  __threadfence();
}

// End of the unfused spectral step: block sums, then the last block to
// finish gathers every block's sums (fixed order) and runs the iteration
// control.
template <typename R>
__device__ void spec_finish(R s0, R c0, R s1, R c1, double l1s, bool has_l1, double* parts,
                            FistaCtl* ctl, double* trace, int32_t* ticket) {
  double v[3];
  spec_block_sums<R>(s0, c0, s1, c1, l1s, has_l1, v);
  const bool mx[3] = {false, false, false};
  if (publish_partials<3>(v, parts, ticket)) {
    double o[3];
    gather_partials<3>(o, parts, mx, ticket);
    if (threadIdx.x == 0) spec_control(o, ctl, trace);
  }
}


template <typename R>
__global__ void __launch_bounds__(kThreads, 4) spec_mul_kernel(const C2<R>* __restrict__ Xk, C2<R>* __restrict__ Xprev,
                                const R* __restrict__ Ks, const C2<R>* __restrict__ Bs, int N,
                                double* __restrict__ parts, FistaCtl* __restrict__ ctl,
                                double* __restrict__ trace, int32_t* ticket,
                                const double* __restrict__ l1_parts, int n_l1) {
  pdl_wait();
  pdl_trigger();
  if (ctl->done) return;
  const int nc = N / 2 + 1;
  const int64_t total = (int64_t)N * nc;
  const int kit = ctl->k;
  const R t = ctl_t<R>(ctl, kit & 1);
  const R a = (R)1 + t;
  const float inv_nc = 1.0f / (float)nc;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // this thread's share of the l1 partials of the previous analysis pass
  double l1s = 0.0;
  for (int64_t i = first; i < n_l1; i += stride) l1s += __ldcg(l1_parts + i);
  // per-thread compensated sums in the working precision, combined in FP64
  R s0 = 0, c0 = 0, s1 = 0, c1 = 0;
  constexpr int U = 2;   // elements per thread and round, loads issued together
  for (int64_t k0 = first; k0 < total; k0 += U * stride) {
    C2<R> X[U], P[U], B[U];
    R kk[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t k = k0 + u * stride;
      if (k < total) {
        X[u] = Xk[k];
        P[u] = Xprev[k];
        kk[u] = Ks[k];
        B[u] = Bs[k];
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t k = k0 + u * stride;
      if (k >= total) break;
      // column of the half-plane (exact: the quotient stays 0.5/nc from an integer)
      const int row = __float2int_rz(((float)k + 0.5f) * inv_nc);
      const int col = (int)(k - (int64_t)row * nc);
      const R w = (col == 0 || col == N / 2) ? (R)1 : (R)2;
      R y0 = w * kk[u] * (X[u].x * X[u].x + X[u].y * X[u].y) - c0;
      R t0 = s0 + y0;
      c0 = (t0 - s0) - y0;
      s0 = t0;
      R y1 = w * (B[u].x * X[u].x + B[u].y * X[u].y) - c1;
      R t1 = s1 + y1;
      c1 = (t1 - s1) - y1;
      s1 = t1;
      C2<R> S;
      S.x = (R)2 * (kk[u] * (a * X[u].x - t * P[u].x) - B[u].x);
      S.y = (R)2 * (kk[u] * (a * X[u].y - t * P[u].y) - B[u].y);
      Xprev[k] = S;
    }
  }
  spec_finish<R>(s0, c0, s1, c1, l1s, (int64_t)blockIdx.x * blockDim.x < n_l1, parts, ctl, trace,
                 ticket);
}

// ------------------------------------------------- shared-memory transforms
// Complex FFTs of length N = 2^LOGN (a compile-time constant) held in shared
// memory, one sequence per N/8 threads, as a mixed-radix Stockham autosort
// transform (natural order in and out, ping-pong between two buffers):
// radix-8 stages, then one radix-2 or radix-4 stage for what is left.  Stage
// with radix Rd after sub-transforms of size Ns: for j < N/Rd, the Rd inputs
// a[j + r N/Rd] are twiddled by W_N^(r (j mod Ns) N/(Ns Rd)), transformed by
// an Rd-point DFT in registers and written to
// b[(j - j mod Ns) Rd + j mod Ns + r Ns].  Every 16th element is followed by
// one pad element (index i lives at i + i/16), in the data and in the
// twiddle table tw[pad(m)] = W_N^m (m < N), which keeps the strided accesses
// of every stage within a few shared-memory wavefronts.

// cos(2 pi k / 16), k < 8
__device__ __forceinline__ double c16(int k) {
  switch (k) {
    case 0: return 1.0;
    case 1: return 0.92387953251128674;
    case 2: return 0.70710678118654752;
    case 3: return 0.38268343236508977;
    case 4: return 0.0;
    case 5: return -0.38268343236508977;
    case 6: return -0.70710678118654752;
    default: return -0.92387953251128674;
  }
}
// sin(t) = cos(pi/2 - t), and cos is even
__device__ __forceinline__ double s16(int k) { return c16(k <= 4 ? 4 - k : k - 4); }

__host__ __device__ constexpr int padi(int i) { return i + (i >> 4); }

// x * W_16^k (forward: W = exp(-2 pi i / 16); inverse: its conjugate), k < 8
// a compile-time constant after unrolling
template <typename R, bool INV>
__device__ __forceinline__ C2<R> mul_w16(C2<R> x, int k) {
  if (k == 0) return x;
  C2<R> y;
  if (k == 4) {   // -i (forward) or +i (inverse)
    y.x = INV ? -x.y : x.y;
    y.y = INV ? x.x : -x.x;
    return y;
  }
  const R c = (R)c16(k), sn = (R)s16(k);
  y.x = INV ? x.x * c - x.y * sn : x.x * c + x.y * sn;
  y.y = INV ? x.y * c + x.x * sn : x.y * c - x.x * sn;
  return y;
}

template <int LOG> __host__ __device__ constexpr int brev_c(int i) {
  int r = 0;
  for (int bit = 0; bit < LOG; ++bit) r |= ((i >> bit) & 1) << (LOG - 1 - bit);
  return r;
}
template <typename R, bool INV>
__device__ __forceinline__ void bfly(C2<R>& a, C2<R>& b, int k) {
  const C2<R> bq = mul_w16<R, INV>(b, k);
  const C2<R> aq = a;
  a.x = aq.x + bq.x;
  a.y = aq.y + bq.y;
  b.x = aq.x - bq.x;
  b.y = aq.y - bq.y;
}
// Rd-point DFT (Rd = 2, 4, 8) of v in registers: bit-reversed copy, then
// log2(Rd) radix-2 decimation-in-time stages; butterfly q of stage st pairs
// i0 = (q / h) 2h + q mod h with i0 + h (h = 2^st) under the twiddle
// W_2h^(q mod h) = W_16^((q mod h) 16 / 2h)
template <typename R, int Rd, bool INV>
__device__ __forceinline__ void dft_reg(C2<R> (&v)[Rd]) {
  constexpr int LOG = Rd == 2 ? 1 : (Rd == 4 ? 2 : 3);
  C2<R> t[Rd];
#pragma unroll
  for (int i = 0; i < Rd; ++i) t[i] = v[brev_c<LOG>(i)];
#pragma unroll
  for (int st = 0; st < LOG; ++st) {
#pragma unroll
    for (int q = 0; q < Rd / 2; ++q) {
      const int h = 1 << st;
      const int j = q & (h - 1);
      const int i0 = ((q >> st) << (st + 1)) + j;
      bfly<R, INV>(t[i0], t[i0 + h], j * (16 / (2 * h)));
    }
  }
#pragma unroll
  for (int i = 0; i < Rd; ++i) v[i] = t[i];
}

// one Stockham stage (radix Rd after sub-transforms of size NS) of the
// calling thread's sequence; src / dst already offset to the sequence
template <typename R, int LOGN, int Rd, int NS, bool INV>
__device__ __forceinline__ void stage_ct(const C2<R>* src, C2<R>* dst, const C2<R>* tw, int tid) {
  constexpr int N = 1 << LOGN, nj = N / Rd, TPS = N / 8;
#pragma unroll
  for (int j0 = 0; j0 < nj; j0 += TPS) {
    const int j = j0 + tid;
    C2<R> v[Rd];
#pragma unroll
    for (int r = 0; r < Rd; ++r) v[r] = src[padi(j + r * nj)];
    const int js = j & (NS - 1);
    if (NS > 1) {
      const int unit = js * (N / (NS * Rd));
#pragma unroll
      for (int r = 1; r < Rd; ++r) {
        C2<R> w = tw[padi(r * unit)];
        if (INV) w.y = -w.y;
        const C2<R> x = v[r];
        v[r].x = x.x * w.x - x.y * w.y;
        v[r].y = x.x * w.y + x.y * w.x;
      }
    }
    dft_reg<R, Rd, INV>(v);
    const int d0 = (j - js) * Rd + js;
#pragma unroll
    for (int r = 0; r < Rd; ++r) dst[padi(d0 + r * NS)] = v[r];
  }
}

// the stages from sub-transform size 2^DONE on; data in (cur ? b1 : b0),
// result in (cur ? b1 : b0) on return; a block barrier after every stage
template <typename R, int LOGN, int DONE, bool INV>
__device__ __forceinline__ void stages_ct(C2<R>* b0, C2<R>* b1, int& cur, const C2<R>* tw, int tid,
                                          bool active) {
  if constexpr (DONE < LOGN) {
    constexpr int LR = LOGN - DONE >= 3 ? 3 : LOGN - DONE;
    if (active)
      stage_ct<R, LOGN, 1 << LR, 1 << DONE, INV>(cur ? b1 : b0, cur ? b0 : b1, tw, tid);
    __syncthreads();
    cur ^= 1;
    stages_ct<R, LOGN, DONE + LR, INV>(b0, b1, cur, tw, tid, active);
  }
}

// data stride of one sequence in shared memory: padded length + 8, so that
// the sequences of one row fall in different banks
__host__ __device__ constexpr int seq_pitch(int n) { return padi(n) + 8; }

// Column-kernel configuration for transform length 2^LOGN and complex size
// CBYTES: CB columns per block (one 32-byte sector of each row, fewer when
// the shared memory would pass kColSmemCap) and PF, the prefetch of the
// block's X^_{k-1}, B^ and K^ when it fits.
constexpr size_t kColSmemCap = 200 * 1024;
#ifndef MS_COL_ROW_BYTES
#define MS_COL_ROW_BYTES 32
#endif
constexpr size_t col_smem_c(int n, int cb, size_t cbytes, bool pf) {
  return (2 * (size_t)cb * seq_pitch(n) + padi(n) + 1) * cbytes +
         (pf ? (size_t)cb * seq_pitch(n) * (2 * cbytes + cbytes / 2) : 0);
}
constexpr int col_cb_c(int n, size_t cbytes, bool pf) {
  int cb = (int)(MS_COL_ROW_BYTES / cbytes) > 4 ? 4 : (int)(MS_COL_ROW_BYTES / cbytes);
  if (cb < 1) cb = 1;
  while (cb > 1 && col_smem_c(n, cb, cbytes, pf) > kColSmemCap) cb /= 2;
  return cb;
}
template <typename R, int LOGN> struct ColCfg {
  static constexpr int N = 1 << LOGN;
  static constexpr size_t CBY = sizeof(C2<R>);
  static constexpr bool PF = col_smem_c(N, col_cb_c(N, CBY, true), CBY, true) <= kColSmemCap;
  static constexpr int CB = col_cb_c(N, CBY, PF);
  static constexpr int TPS = N / 8;
  static constexpr int THREADS = CB * TPS < 32 ? 32 : CB * TPS;
  static constexpr size_t SMEM = col_smem_c(N, CB, CBY, PF);
  static_assert(THREADS <= 1024 && THREADS % 32 == 0, "column block");
};

// A compensated sum hi + lo as an FP32 pair (hi, lo) (exact for FP32 input;
// about 48 significant bits for FP64).
template <typename R> __device__ __forceinline__ float2 fp32_pair(R hi, R lo) {
  if constexpr (sizeof(R) == 4) {
    float s, e;
    two_sum<float>(hi, lo, s, e);
    return make_float2(s, e);
  } else {
    const double v = hi + lo;
    const float h = __double2float_rn(v);
    return make_float2(h, __double2float_rn(v - (double)h));
  }
}

// The spectral step with the column transforms fused in, for N = 2^LOGN.
// Z holds the row transforms of x_k ([N][N/2+1], the half-plane layout);
// each block takes CB columns: the column FFT gives X^_k (the 2-D transform
// of x_k, kept in Xk for the next pass's momentum), the step of
// spec_mul_kernel forms S = 2 (K^((1 + t) X^_k - t X^_{k-1}) - B^) and the
// objective partials, and the inverse column FFT of S goes back into Z,
// whose inverse row transforms then give the gradient image.  Global accesses
// take one row's CB columns per lane group (coalesced) and are asynchronous
// copies issued at the start: the columns of Z, and (PF) the block's
// X^_{k-1}, K^ and B^, which arrive while the forward transforms run.  Each
// warp leaves its sums of the objective terms in parts[i W + warp] (W warps
// in all; i = <x,Kx>, <b,x>, the l1 partials); the inverse row transform
// kernel gathers them and runs the iteration control, so this kernel has no
// grid-wide tail.
template <typename R, int LOGN>
__global__ void __launch_bounds__(ColCfg<R, LOGN>::THREADS, 1) spec_col_kernel(
    C2<R>* __restrict__ Z, C2<R>* __restrict__ Xk, const C2<R>* __restrict__ Xprev,
    const R* __restrict__ Ks, const C2<R>* __restrict__ Bs, const C2<R>* __restrict__ tw_g,
    double* __restrict__ parts, const FistaCtl* __restrict__ ctl,
    const double* __restrict__ l1_parts, int n_l1, JobStride js) {
  using Cfg = ColCfg<R, LOGN>;
  if (blockIdx.z != 0) {   // this block's job (batched form)
    const int64_t z = blockIdx.z;
    Z += z * js.spec;
    Xk += z * js.spec;
    Xprev += z * js.spec;
    Ks += z * js.spec;
    Bs += z * js.spec;
    parts += z * js.parts;
    ctl += z;
    l1_parts += z * js.l1;
  }
  constexpr int N = Cfg::N, CB = Cfg::CB, T = Cfg::THREADS, P = seq_pitch(N);
  constexpr bool PF = Cfg::PF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* b0 = reinterpret_cast<C2<R>*>(smem_raw);   // [CB][P]
  C2<R>* b1 = b0 + CB * P;                           // [CB][P]
  C2<R>* tw = b1 + CB * P;                           // [pad(N) + 1]
  // the twiddle table is written once per plan: staged while the
  // predecessor kernel finishes
  for (int m = threadIdx.x; m < N; m += T) cp_async<sizeof(C2<R>)>(tw + padi(m), tw_g + m);
  cp_async_commit();
  pdl_wait();
  pdl_trigger();
  C2<R>* sP = tw + padi(N) + 1;                      // PF: [CB][P] X^_{k-1}
  C2<R>* sB = sP + CB * P;                           // PF: [CB][P] B^
  R* sK = reinterpret_cast<R*>(sB + CB * P);         // PF: [CB][P] K^
  constexpr int nc = N / 2 + 1;
  const int c0 = blockIdx.x * CB;
  const int ccol = threadIdx.x / Cfg::TPS, tcol = threadIdx.x - ccol * Cfg::TPS;
  const bool active = ccol < CB;
  // element e = (row e / CB, column e mod CB); lanes cover whole rows
  for (int e = threadIdx.x; e < N * CB; e += T) {
    const int r = e / CB, c = e - r * CB;
    C2<R>* d = b0 + c * P + padi(r);
    if (c0 + c < nc) {
      cp_async<sizeof(C2<R>)>(d, Z + (int64_t)r * nc + c0 + c);
    } else {
      d->x = (R)0;
      d->y = (R)0;
    }
  }
  cp_async_commit();
  if (PF) {
    for (int e = threadIdx.x; e < N * CB; e += T) {
      const int r = e / CB, c = e - r * CB;
      if (c0 + c < nc) {
        const int64_t k = (int64_t)r * nc + c0 + c;
        const int o = c * P + padi(r);
        cp_async<sizeof(C2<R>)>(sP + o, Xprev + k);
        cp_async<sizeof(C2<R>)>(sB + o, Bs + k);
        cp_async<sizeof(R)>(sK + o, Ks + k);
      }
    }
    cp_async_commit();
  }
  // the control block and the l1 partials load while the copies run (the
  // copies were issued before `done` is known: when it is set, they are
  // waited for and the block returns)
  const int done = ctl->done;
  const int kit = ctl->k;
  const R t = ctl_t<R>(ctl, kit & 1);
  const R a = (R)1 + t;
  double l1s = 0.0;
  const int64_t first = blockIdx.x * (int64_t)T + threadIdx.x;
  for (int64_t i = first; i < n_l1; i += (int64_t)gridDim.x * T) l1s += __ldcg(l1_parts + i);
  if (done) {
    cp_async_wait<0>();
    return;
  }
  if (PF) cp_async_wait<1>();   // twiddles and the columns of Z (the prefetch may still run)
  else cp_async_wait<0>();
  __syncthreads();
  int cur = 0;
  C2<R>* c_b0 = b0 + (active ? ccol : 0) * P;
  C2<R>* c_b1 = b1 + (active ? ccol : 0) * P;
  stages_ct<R, LOGN, 0, false>(c_b0, c_b1, cur, tw, tcol, active);
  if (PF) cp_async_wait<0>();   // this thread's own prefetched elements
  C2<R>* X = cur ? b1 : b0;
  R s0 = 0, cc0 = 0, s1 = 0, cc1 = 0;
  auto step = [&](int r, int c, const C2<R>& Pv, R kk, const C2<R>& Bv) {
    const int col = c0 + c;
    C2<R>* xp = X + c * P + padi(r);
    const C2<R> Xv = *xp;
    const R w = (col == 0 || col == N / 2) ? (R)1 : (R)2;
    R y0 = w * kk * (Xv.x * Xv.x + Xv.y * Xv.y) - cc0;
    R t0 = s0 + y0;
    cc0 = (t0 - s0) - y0;
    s0 = t0;
    R y1 = w * (Bv.x * Xv.x + Bv.y * Xv.y) - cc1;
    R t1 = s1 + y1;
    cc1 = (t1 - s1) - y1;
    s1 = t1;
    C2<R> S;
    S.x = (R)2 * (kk * (a * Xv.x - t * Pv.x) - Bv.x);
    S.y = (R)2 * (kk * (a * Xv.y - t * Pv.y) - Bv.y);
    Xk[(int64_t)r * nc + col] = Xv;
    *xp = S;   // same element, same thread: no barrier needed before
  };
  if (PF) {
    for (int e = threadIdx.x; e < N * CB; e += T) {
      const int r = e / CB, c = e - r * CB;
      const int o = c * P + padi(r);
      if (c0 + c < nc) {
        step(r, c, sP[o], sK[o], sB[o]);
      } else {
        X[o].x = (R)0;
        X[o].y = (R)0;
      }
    }
  } else {
    // direct loads, four elements' loads in flight at a time
    constexpr int U = 4;
    for (int e0 = threadIdx.x; e0 < N * CB; e0 += U * T) {
      C2<R> Pv[U], Bv[U];
      R kk[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * T, r = e / CB, c = e - r * CB;
        if (e < N * CB && c0 + c < nc) {
          const int64_t k = (int64_t)r * nc + c0 + c;
          Pv[u] = Xprev[k];
          kk[u] = Ks[k];
          Bv[u] = Bs[k];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * T, r = e / CB, c = e - r * CB;
        if (e >= N * CB) break;
        if (c0 + c < nc) {
          step(r, c, Pv[u], kk[u], Bv[u]);
        } else {
          X[c * P + padi(r)].x = (R)0;
          X[c * P + padi(r)].y = (R)0;
        }
      }
    }
  }
  __syncthreads();
  stages_ct<R, LOGN, 0, true>(c_b0, c_b1, cur, tw, tcol, active);
  const C2<R>* Y = cur ? b1 : b0;
  for (int e = threadIdx.x; e < N * CB; e += T) {
    const int r = e / CB, c = e - r * CB;
    if (c0 + c < nc) Z[(int64_t)r * nc + c0 + c] = Y[c * P + padi(r)];
  }
  // this warp's sums (no block barrier at the end): the inverse row
  // transform kernel that follows gathers them and runs the iteration
  // control
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (T / 32);
  const int64_t wi = (int64_t)blockIdx.x * (T / 32) + (threadIdx.x >> 5);
  R lo0 = -cc0, lo1 = -cc1;
  warp_sum_comp<R>(s0, lo0);
  warp_sum_comp<R>(s1, lo1);
  double w2 = 0.0;
  if ((int64_t)blockIdx.x * T < n_l1) w2 = warp_sum(l1s);   // uniform over the block
  if (lane == 0) {
    // as FP32 (hi, lo) pairs, which the control block adds in FP32
    float2* pp = reinterpret_cast<float2*>(parts);
    pp[wi] = fp32_pair<R>(s0, lo0);
    pp[nw + wi] = fp32_pair<R>(s1, lo1);
    pp[2 * nw + wi] = fp32_pair<double>(w2, 0.0);
  }
}

// ------------------------------------------------------------ row transforms
// Real transforms of the N rows of length N = 2^LOGN through complex
// transforms of length M = N/2 (the standard packing of a real sequence):
// z_n = x_2n + i x_2n+1, Z = FFT_M(z), and for k = 0..M, with Z_M = Z_0,
//   E_k = (Z_k + conj Z_(M-k)) / 2,  O_k = -i (Z_k - conj Z_(M-k)) / 2,
//   X_k = E_k + W_N^k O_k.
// The inverse (unnormalized, the imaginary parts of X_0 and X_M ignored)
// forms Z'_k = (X_k + conj X_(M-k)) + i W_N^-k (X_k - conj X_(M-k)), k < M,
// and x_2n + i x_2n+1 = sum_k Z'_k W_M^-kn.  One row per M/8 threads, RB
// rows per block.
#ifndef MS_ROW_THREADS
#define MS_ROW_THREADS 512   // threads per block of the row transforms (rows x N/16)
#endif
template <typename R, int LOGN> struct RowCfg {
  static constexpr int N = 1 << LOGN, M = N / 2;
  static constexpr int TPS = M / 8 > 0 ? M / 8 : 1;
  static constexpr int RB = MS_ROW_THREADS / TPS < 1
                                ? 1
                                : (MS_ROW_THREADS / TPS > N ? N : MS_ROW_THREADS / TPS);
  static constexpr int THREADS = RB * TPS < 32 ? 32 : RB * TPS;
  // two buffers of RB rows, the M-point twiddle table W_M^m = W_N^2m
  // (padded) and W_N^k, k <= M, for the packing step
  static constexpr size_t SMEM =
      (2 * (size_t)RB * seq_pitch(M) + padi(M) + 1 + M + 1) * sizeof(C2<R>);
  static_assert(THREADS <= 1024 && THREADS % 32 == 0, "row block");
};

template <typename R, int LOGN>
__global__ void __launch_bounds__(RowCfg<R, LOGN>::THREADS) row_r2c_kernel(
    const R* __restrict__ x, C2<R>* __restrict__ Z, const C2<R>* __restrict__ tw_g,
    const FistaCtl* __restrict__ ctl, JobStride js) {
  using Cfg = RowCfg<R, LOGN>;
  if (blockIdx.z != 0) {   // this block's job (batched form)
    const int64_t z = blockIdx.z;
    x += z * js.img;
    Z += z * js.spec;
    ctl += z;
  }
  constexpr int M = Cfg::M, RB = Cfg::RB, P = seq_pitch(M), nc = M + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* b0 = reinterpret_cast<C2<R>*>(smem_raw);   // [RB][P]
  C2<R>* b1 = b0 + RB * P;                           // [RB][P]
  C2<R>* tw = b1 + RB * P;                           // [pad(M) + 1]
  C2<R>* twn = tw + padi(M) + 1;                     // [M + 1]
  // twiddles (written once per plan) staged while the predecessor finishes
  for (int m = threadIdx.x; m < M; m += Cfg::THREADS)
    cp_async<sizeof(C2<R>)>(tw + padi(m), tw_g + 2 * m);
  for (int k = threadIdx.x; k <= M; k += Cfg::THREADS) cp_async<sizeof(C2<R>)>(twn + k, tw_g + k);
  cp_async_commit();
  pdl_wait();
  pdl_trigger();
  if (ctl->done) {
    cp_async_wait<0>();
    return;
  }
  const int rr = threadIdx.x / Cfg::TPS, t = threadIdx.x - rr * Cfg::TPS;
  const bool active = rr < RB;
  const int row0 = blockIdx.x * RB;
  const C2<R>* xin = reinterpret_cast<const C2<R>*>(x) + (int64_t)row0 * M;   // pairs
  for (int e = threadIdx.x; e < RB * M; e += Cfg::THREADS) {
    const int q = e / M, n = e - q * M;
    cp_async<sizeof(C2<R>)>(b0 + q * P + padi(n), xin + e);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  int cur = 0;
  stages_ct<R, LOGN - 1, 0, false>(b0 + (active ? rr : 0) * P, b1 + (active ? rr : 0) * P, cur,
                                   tw, t, active);
  if (!active) return;
  const C2<R>* Zs = (cur ? b1 : b0) + rr * P;
  C2<R>* out = Z + (int64_t)(row0 + rr) * nc;
  for (int k = t; k <= M; k += Cfg::TPS) {
    const C2<R> zk = Zs[padi(k == M ? 0 : k)], zm = Zs[padi(k == 0 ? 0 : M - k)];
    const R ex = (R)0.5 * (zk.x + zm.x), ey = (R)0.5 * (zk.y - zm.y);
    const R ox = (R)0.5 * (zk.y + zm.y), oy = (R)-0.5 * (zk.x - zm.x);
    const C2<R> w = twn[k];   // W_N^k, k <= N/2
    C2<R> X;
    X.x = ex + (w.x * ox - w.y * oy);
    X.y = ey + (w.x * oy + w.y * ox);
    out[k] = X;
  }
}

template <typename R, int LOGN>
__global__ void __launch_bounds__(RowCfg<R, LOGN>::THREADS) row_c2r_kernel(
    const C2<R>* __restrict__ Z, R* __restrict__ x, const C2<R>* __restrict__ tw_g,
    FistaCtl* __restrict__ ctl, const double* __restrict__ parts, int G,
    double* __restrict__ trace, JobStride js) {
  using Cfg = RowCfg<R, LOGN>;
  if (blockIdx.z != 0) {   // this block's job (batched form)
    const int64_t z = blockIdx.z;
    Z += z * js.spec;
    x += z * js.img;
    ctl += z;
    if (parts) parts += z * js.parts;
    trace += z * js.trace;
  }
  constexpr int M = Cfg::M, RB = Cfg::RB, P = seq_pitch(M), nc = M + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C2<R>* b0 = reinterpret_cast<C2<R>*>(smem_raw);   // [RB][P]
  C2<R>* b1 = b0 + RB * P;                           // [RB][P]
  C2<R>* tw = b1 + RB * P;                           // [pad(M) + 1]
  C2<R>* twn = tw + padi(M) + 1;                     // [M + 1]
  if (!(parts && blockIdx.x == 0)) {   // (the control block needs no twiddles)
    for (int m = threadIdx.x; m < M; m += Cfg::THREADS)
      cp_async<sizeof(C2<R>)>(tw + padi(m), tw_g + 2 * m);
    for (int k = threadIdx.x; k <= M; k += Cfg::THREADS)
      cp_async<sizeof(C2<R>)>(twn + k, tw_g + k);
  }
  cp_async_commit();
  pdl_wait();
  pdl_trigger();
  if (ctl->done) {
    cp_async_wait<0>();
    return;
  }
  if (parts && blockIdx.x == 0) {
    // the spectral step (the predecessor, complete) left G warp sums of
    // each objective term as FP32 (hi, lo) pairs: add them in a fixed order
    // with error-free FP32 additions (the FP64 pipe is slow) and run the
    // iteration control, beside the blocks that transform the rows
    __shared__ float2 wred[3][32];
    const float2* pp = reinterpret_cast<const float2*>(parts);
    float hi[3] = {0.f, 0.f, 0.f}, lo[3] = {0.f, 0.f, 0.f};
    constexpr int U = 8;   // a thread's loads of U pairs per term in flight together
    for (int b0 = threadIdx.x; b0 < G; b0 += U * blockDim.x) {
      float2 x[3][U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int b = b0 + u * blockDim.x;
#pragma unroll
        for (int i = 0; i < 3; ++i)
          x[i][u] = b < G ? __ldcg(pp + (int64_t)i * G + b) : make_float2(0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < U; ++u)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          float sm, e;
          two_sum<float>(hi[i], x[i][u].x, sm, e);
          hi[i] = sm;
          lo[i] += x[i][u].y + e;
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      warp_sum_comp<float>(hi[i], lo[i]);
      if (lane == 0) wred[i][warp] = make_float2(hi[i], lo[i]);
    }
    __syncthreads();
    if (warp == 0) {
      double o[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float h = 0.f, l = 0.f;
        if (lane < nw) {
          h = wred[i][lane].x;
          l = wred[i][lane].y;
        }
        warp_sum_comp<float>(h, l);
        o[i] = (double)h + (double)l;
      }
      if (lane == 0) spec_control(o, ctl, trace);
    }
    return;
  }
  const int rr = threadIdx.x / Cfg::TPS, t = threadIdx.x - rr * Cfg::TPS;
  const bool active = rr < RB;
  const int row0 = (blockIdx.x - (parts ? 1 : 0)) * RB;
  // the rows' M + 1 spectrum values into b1 (pad(M) < P)
  for (int e = threadIdx.x; e < RB * nc; e += Cfg::THREADS) {
    const int q = e / nc, k = e - q * nc;
    cp_async<sizeof(C2<R>)>(b1 + q * P + padi(k), Z + (int64_t)row0 * nc + e);
  }
  cp_async_commit();
  cp_async_wait<0>();
  __syncthreads();
  if (active) {
    const C2<R>* Y = b1 + rr * P;
    C2<R>* Zp = b0 + rr * P;
    for (int k = t; k < M; k += Cfg::TPS) {
      C2<R> a = Y[padi(k)], b = Y[padi(M - k)];
      if (k == 0) {
        a.y = (R)0;
        b.y = (R)0;
      }
      const R sx = a.x + b.x, sy = a.y - b.y;   // X_k + conj X_(M-k)
      const R dx = a.x - b.x, dy = a.y + b.y;   // X_k - conj X_(M-k)
      const C2<R> w = twn[k];                   // W_N^k; times its conjugate below
      const R fx = w.x * dx + w.y * dy, fy = w.x * dy - w.y * dx;
      C2<R> zp;
      zp.x = sx - fy;   // + i (fx + i fy)
      zp.y = sy + fx;
      Zp[padi(k)] = zp;
    }
  }
  __syncthreads();
  int cur = 0;
  stages_ct<R, LOGN - 1, 0, true>(b0 + (active ? rr : 0) * P, b1 + (active ? rr : 0) * P, cur,
                                  tw, t, active);
  if (!active) return;
  const C2<R>* zs = (cur ? b1 : b0) + rr * P;
  C2<R>* xo = reinterpret_cast<C2<R>*>(x) + (int64_t)(row0 + rr) * M;
  for (int n = t; n < M; n += Cfg::TPS) xo[n] = zs[padi(n)];
}

namespace {
// dispatch over the supported transform lengths 2^4 .. 2^13
template <template <int> class F, typename... A> cudaError_t by_logn(int logN, A... args) {
  switch (logN) {
    case 4: return F<4>::go(args...);
    case 5: return F<5>::go(args...);
    case 6: return F<6>::go(args...);
    case 7: return F<7>::go(args...);
    case 8: return F<8>::go(args...);
    case 9: return F<9>::go(args...);
    case 10: return F<10>::go(args...);
    case 11: return F<11>::go(args...);
    case 12: return F<12>::go(args...);
    case 13: return F<13>::go(args...);
    default: return cudaErrorInvalidValue;
  }
}
int log2_exact(int N) {
  int l = 0;
  while ((1 << l) < N) ++l;
  return (1 << l) == N ? l : -1;
}
// The kernels of the fused step run with plain launches: with programmatic
// dependent launch their early-launched successors measured slower at
// N = 1024 (10 us per FISTA iteration for the row kernels).
#ifndef MS_FFT_PDL
#define MS_FFT_PDL 0
#endif
template <typename... KArgs, typename... Args>
cudaError_t launch_fft(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                       cudaStream_t s, Args... args) {
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (MS_FFT_PDL) return launch_pdl(kernel, grid, block, smem, s, args...);
  kernel<<<grid, block, smem, s>>>(args...);
  return cudaGetLastError();
}
template <typename R> struct ColLaunch {
  template <int LOGN> struct At {
    static cudaError_t go(C2<R>* Z, C2<R>* Xk, const C2<R>* Xprev, const R* Ks, const C2<R>* Bs,
                          const C2<R>* tw, double* parts, const FistaCtl* ctl,
                          const double* l1_parts, int n_l1, cudaStream_t s, JobStride js) {
      using Cfg = ColCfg<R, LOGN>;
      return launch_fft(spec_col_kernel<R, LOGN>,
                        dim3((Cfg::N / 2 + 1 + Cfg::CB - 1) / Cfg::CB, 1, js.jobs),
                        dim3(Cfg::THREADS), Cfg::SMEM, s, Z, Xk, Xprev, Ks, Bs, tw, parts, ctl,
                        l1_parts, n_l1, js);
    }
  };
  template <int LOGN> struct Info {
    static cudaError_t go(int* blocks, size_t* smem, int* warps) {
      using Cfg = ColCfg<R, LOGN>;
      *blocks = (Cfg::N / 2 + 1 + Cfg::CB - 1) / Cfg::CB;
      *smem = Cfg::SMEM;
      *warps = Cfg::THREADS / 32;
      return cudaSuccess;
    }
  };
};
template <typename R> struct RowLaunch {
  template <int LOGN> struct R2C {
    static cudaError_t go(const R* x, C2<R>* Z, const C2<R>* tw, const FistaCtl* ctl,
                          cudaStream_t s, JobStride js) {
      using Cfg = RowCfg<R, LOGN>;
      return launch_fft(row_r2c_kernel<R, LOGN>, dim3(Cfg::N / Cfg::RB, 1, js.jobs),
                        dim3(Cfg::THREADS), Cfg::SMEM, s, x, Z, tw, ctl, js);
    }
  };
  template <int LOGN> struct C2R {
    static cudaError_t go(const C2<R>* Z, R* x, const C2<R>* tw, FistaCtl* ctl,
                          const double* parts, int G, double* trace, cudaStream_t s,
                          JobStride js) {
      using Cfg = RowCfg<R, LOGN>;
      return launch_fft(row_c2r_kernel<R, LOGN>,
                        dim3(Cfg::N / Cfg::RB + (parts ? 1 : 0), 1, js.jobs), dim3(Cfg::THREADS),
                        Cfg::SMEM, s, Z, x, tw, ctl, parts, G, trace, js);
    }
  };
  template <int LOGN> struct Info {
    static cudaError_t go(size_t* smem) {
      *smem = RowCfg<R, LOGN>::SMEM;
      return cudaSuccess;
    }
  };
};
}  // namespace

// sizes of the fused step's kernels; 0 / SIZE_MAX when N is not supported
int spec_col_warps(int N, size_t complex_bytes) {
  int b = 0, w = 0;
  size_t sm = 0;
  const int l = log2_exact(N);
  if (complex_bytes == 8) by_logn<ColLaunch<float>::Info>(l, &b, &sm, &w);
  else by_logn<ColLaunch<double>::Info>(l, &b, &sm, &w);
  return b * w;
}
int spec_col_blocks(int N, size_t complex_bytes) {
  int b = 0, w = 0;
  size_t sm = 0;
  const int l = log2_exact(N);
  if (complex_bytes == 8) by_logn<ColLaunch<float>::Info>(l, &b, &sm, &w);
  else by_logn<ColLaunch<double>::Info>(l, &b, &sm, &w);
  return b;
}
size_t spec_col_smem(int N, size_t complex_bytes) {
  int b = 0, w = 0;
  size_t sm = SIZE_MAX;
  const int l = log2_exact(N);
  if (complex_bytes == 8) by_logn<ColLaunch<float>::Info>(l, &b, &sm, &w);
  else by_logn<ColLaunch<double>::Info>(l, &b, &sm, &w);
  return sm;
}
size_t row_fft_smem(int N, size_t complex_bytes) {
  size_t sm = SIZE_MAX;
  const int l = log2_exact(N);
  if (complex_bytes == 8) by_logn<RowLaunch<float>::Info>(l, &sm);
  else by_logn<RowLaunch<double>::Info>(l, &sm);
  return sm;
}

template <typename R>
cudaError_t launch_spec_col(C2<R>* Z, C2<R>* Xk, const C2<R>* Xprev, const R* Ks,
                            const C2<R>* Bs, const C2<R>* tw, int N, double* parts,
                            const FistaCtl* ctl, const double* l1_parts, int n_l1,
                            cudaStream_t s, const JobStride& js) {
  return by_logn<ColLaunch<R>::template At>(log2_exact(N), Z, Xk, Xprev, Ks, Bs, tw, parts,
                                            ctl, l1_parts, n_l1, s, js);
}
template <typename R>
cudaError_t launch_row_r2c(const R* x, C2<R>* Z, const C2<R>* tw, int N, const FistaCtl* ctl,
                           cudaStream_t s, const JobStride& js) {
  return by_logn<RowLaunch<R>::template R2C>(log2_exact(N), x, Z, tw, ctl, s, js);
}
template <typename R>
cudaError_t launch_row_c2r(const C2<R>* Z, R* x, const C2<R>* tw, int N, FistaCtl* ctl,
                           const double* parts, int G, double* trace, cudaStream_t s,
                           const JobStride& js) {
  return by_logn<RowLaunch<R>::template C2R>(log2_exact(N), Z, x, tw, ctl, parts, G, trace, s,
                                             js);
}

template <typename R>
void launch_spec_mul(const C2<R>* Xk, C2<R>* Xprev, const R* Ks, const C2<R>* Bs, int N,
                     double* parts, FistaCtl* ctl, double* trace, int32_t* ticket,
                     const double* l1_parts, int n_l1, cudaStream_t s) {
  launch_pdl(spec_mul_kernel<R>, dim3(spectral_partials(N)), dim3(kThreads), 0, s, Xk, Xprev, Ks,
             Bs, N, parts, ctl, trace, ticket, l1_parts, n_l1);
}

template <typename R>
__global__ void spec_apply_kernel(C2<R>* __restrict__ spec, const R* __restrict__ Ks, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    C2<R> X = spec[k];
    R kk = Ks[k];
    X.x *= kk;
    X.y *= kk;
    spec[k] = X;
  }
}

template <typename R>
void launch_spec_apply(C2<R>* spec, const R* Ks, int N, cudaStream_t s) {
  int64_t n = (int64_t)N * (N / 2 + 1);
  spec_apply_kernel<R><<<nparts_for(n), kThreads, 0, s>>>(spec, Ks, n);
}

// ------------------------------------------------------------- image stats
// ||x||_2^2 and max |x| of an image -> ctl->norm2, ctl->absmax
template <typename R>
__global__ void image_norms_kernel(const R* __restrict__ img, int64_t n, double* parts,
                                   FistaCtl* ctl, int32_t* ticket) {
  double v[2] = {0.0, 0.0};
  const bool mx[2] = {false, true};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    double x = (double)img[k];
    v[0] += x * x;
    v[1] = fmax(v[1], fabs(x));
  }
  block_reduce<2>(v, mx);
  if (publish_partials<2>(v, parts, ticket)) {
    double o[2];
    gather_partials<2>(o, parts, mx, ticket);
    if (threadIdx.x == 0) {
      ctl->norm2 = o[0];
      ctl->absmax = o[1];
    }
  }
}

template <typename R>
void launch_image_norms(const R* img, int64_t n, double* parts, FistaCtl* ctl, int32_t* ticket,
                        cudaStream_t s) {
  image_norms_kernel<R><<<nparts_for(n), kThreads, 0, s>>>(img, n, parts, ctl, ticket);
}

// Sect. 4.3: mean over all inside 5x5 windows of the population variance.
template <typename R>
__global__ void sigma2_kernel(const R* __restrict__ img, int N, double* parts, FistaCtl* ctl,
                              int32_t* ticket, int set_eta) {
  const int nw = N - 4;
  const int64_t total = (int64_t)nw * nw;
  double v[1] = {0.0};
  const bool mx[1] = {false};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int p = (int)(k / nw), q = (int)(k % nw);
    double s = 0.0, s2 = 0.0;
    for (int a = 0; a < 5; ++a)
      for (int b = 0; b < 5; ++b) {
        double x = (double)img[(int64_t)(p + a) * N + q + b];
        s += x;
        s2 += x * x;
      }
    double mean = s / 25.0;
    double var = s2 / 25.0 - mean * mean;
    v[0] += var > 0.0 ? var : 0.0;
  }
  block_reduce<1>(v, mx);
  if (publish_partials<1>(v, parts, ticket)) {
    double o[1];
    gather_partials<1>(o, parts, mx, ticket);
    if (threadIdx.x == 0) {
      double s2 = o[0] / (double)total;
      ctl->sigma2 = s2;
      if (set_eta) ctl->eta2 = 1e-3 * s2;
    }
  }
}

template <typename R>
void launch_sigma2_hat(const R* img, int N, double* parts, FistaCtl* ctl, int32_t* ticket,
                       int set_eta, cudaStream_t s) {
  sigma2_kernel<R><<<nparts_for((int64_t)(N - 4) * (N - 4)), kThreads, 0, s>>>(
      img, N, parts, ctl, ticket, set_eta);
}

// lambda of major cycle n (1-based): rule 0: c ||i~_n||_2 2^n; rule 1: c max|i~_1|
__global__ void set_lambda_kernel(FistaCtl* ctl, int rule, double coef, int n, int first) {
  if (first) ctl->absmax_first = ctl->absmax;
  if (rule == 0)
    ctl->lam = coef * sqrt(ctl->norm2) * ldexp(1.0, n);
  else
    ctl->lam = coef * ctl->absmax_first;
}

// ------------------------------------------------------------- small vector ops
template <typename R>
__global__ void axpby_kernel(const R* __restrict__ x, const R* __restrict__ y, R* __restrict__ o,
                             R a, R b, int64_t n) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    o[k] = a * x[k] + (y ? b * y[k] : (R)0);
}

template <typename R>
void launch_axpby(const R* x, const R* y, R* out, double a, double b, int64_t n, cudaStream_t s) {
  axpby_kernel<R><<<nparts_for(n), kThreads, 0, s>>>(x, y, out, (R)a, (R)b, n);
}

// sum |x| (OP 0) or <x, y> (OP 1) in FP64 -> *out
template <typename R, int OP>
__global__ void reduce_kernel(const R* __restrict__ x, const R* __restrict__ y, int64_t n,
                              double* parts, double* out, int32_t* ticket) {
  double v[1] = {0.0};
  const bool mx[1] = {false};
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    v[0] += OP == 0 ? fabs((double)x[k]) : (double)x[k] * (double)y[k];
  block_reduce<1>(v, mx);
  if (publish_partials<1>(v, parts, ticket)) {
    double o[1];
    gather_partials<1>(o, parts, mx, ticket);
    if (threadIdx.x == 0) {
      *out = o[0];
    }
  }
}

template <typename R>
void launch_l1(const R* x, int64_t n, double* parts, double* out, int32_t* ticket,
               cudaStream_t s) {
  reduce_kernel<R, 0><<<nparts_for(n), kThreads, 0, s>>>(x, nullptr, n, parts, out, ticket);
}

template <typename R>
void launch_dot(const R* x, const R* y, int64_t n, double* parts, double* out, int32_t* ticket,
                cudaStream_t s) {
  reduce_kernel<R, 1><<<nparts_for(n), kThreads, 0, s>>>(x, y, n, parts, out, ticket);
}

// x <- x / sqrt(*den)
template <typename R>
__global__ void normalize_kernel(R* __restrict__ x, int64_t n, const double* __restrict__ den) {
  const double sc = 1.0 / sqrt(*den);
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    x[k] = (R)((double)x[k] * sc);
}

template <typename R>
void launch_normalize(R* x, int64_t n, const double* den, cudaStream_t s) {
  normalize_kernel<R><<<nparts_for(n), kThreads, 0, s>>>(x, n, den);
}

// deterministic pseudo-random start vector in [-1, 1] (splitmix64 of the index)
template <typename R>
__global__ void hash_fill_kernel(R* __restrict__ x, int64_t n, uint64_t seed) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(k + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    x[k] = (R)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
  }
}

template <typename R>
void launch_hash_fill(R* x, int64_t n, uint64_t seed, cudaStream_t s) {
  hash_fill_kernel<R><<<nparts_for(n), kThreads, 0, s>>>(x, n, seed);
}

void launch_set_lambda(FistaCtl* ctl, int rule, double coef, int n, int first, cudaStream_t s) {
  set_lambda_kernel<<<1, 1, 0, s>>>(ctl, rule, coef, n, first);
}

// ------------------------------------------------- linear PSF operator
// The minor cycle's PSF operator read as the linear convolution that
// A^H A / sum(w) is on images of the N x N field:
//   H x = P F2^-1( H2^ . F2( P^T x ) ),
// P^T the zero padding to 2N x 2N, P the restriction to the first N x N,
// F2 the 2N x 2N DFT and H2^ the real spectrum of the PSF on the 2N x 2N
// field (offsets up to +-N, so no product wraps).  The transforms are
// cuFFT's; these kernels pad, multiply, restrict and run the iteration
// control.  With it the smooth parts are no longer diagonal in the N x N
// Fourier basis, so a FISTA pass evaluates them in the image domain:
//   LOW:  y_k = H x_k, f = ||y_k - i~||^2, gradient image 2 H r,
//         r = (1 + t_k) y_k - t_k y_k-1 - i~ (= H z - i~ at the extrapolated
//         point z, H being linear);
//   FULL: D_k = y_k - i~, E_k = x_k - l, f = ||G_H D_k||^2 + ||G_L E_k||^2
//         (Parseval on the N x N half-plane), gradient image
//         2 (H G_H^2 D_z + G_L^2 E_z) with D_z, E_z the momentum combinations
//         of the last two spectra.
// Kernels given a control block return once `done` is set (uniform early
// exit); with ctl == nullptr they always run (plain operator calls).
// Row loops: one block per row (grid-stride), threads across the row.

template <typename R>
__global__ void lin_pad_kernel(const R* __restrict__ x, R* __restrict__ xp, int N,
                               const FistaCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  const int N2 = 2 * N;
  for (int row = blockIdx.x; row < N2; row += gridDim.x) {
    R* out = xp + (int64_t)row * N2;
    const R* in = x + (int64_t)row * N;
    for (int c = threadIdx.x; c < N2; c += blockDim.x)
      out[c] = (row < N && c < N) ? in[c] : (R)0;
  }
}

// S *= H2^ / (2N)^2 (the inverse transform is unnormalized)
template <typename R>
__global__ void lin_mul_kernel(C2<R>* __restrict__ S, const R* __restrict__ H2, int64_t n, R inv,
                               const FistaCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const R h = H2[k] * inv;
    C2<R> v = S[k];
    v.x *= h;
    v.y *= h;
    S[k] = v;
  }
}

// out = scale (P q + add), q a 2N x 2N image, add an N x N image or null
template <typename R>
__global__ void lin_crop_kernel(const R* __restrict__ q, const R* __restrict__ add,
                                R* __restrict__ out, int N, R scale,
                                const FistaCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  const int N2 = 2 * N;
  for (int row = blockIdx.x; row < N; row += gridDim.x) {
    const R* qr = q + (int64_t)row * N2;
    const int64_t o = (int64_t)row * N;
    for (int c = threadIdx.x; c < N; c += blockDim.x)
      out[o + c] = scale * (qr[c] + (add ? add[o + c] : (R)0));
  }
}

// this thread's share of the |B_k| partials left by the previous analysis
__device__ __forceinline__ double lin_l1_share(const double* __restrict__ l1_parts, int n_l1) {
  double l1s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_l1;
       i += (int64_t)gridDim.x * blockDim.x)
    l1s += __ldcg(l1_parts + i);
  return l1s;
}

template <typename R> __device__ __forceinline__ void kahan_add(R& s, R& c, R y) {
  y -= c;
  const R t = s + y;
  c = (t - s) - y;
  s = t;
}

// LOW / SINGLE: y_k = P q into ycur, f = ||y_k - i~||^2 (with ||B_k||_1 the
// iteration control, in the last block), and r = (1 + t_k) y_k - t_k y_k-1 - i~
// zero-padded into rp
template <typename R>
__global__ void lin_low_step_kernel(const R* __restrict__ q, const R* __restrict__ res,
                                    R* __restrict__ ycur, const R* __restrict__ yprev,
                                    R* __restrict__ rp, int N, double* __restrict__ parts,
                                    FistaCtl* __restrict__ ctl, double* __restrict__ trace,
                                    int32_t* ticket, const double* __restrict__ l1_parts,
                                    int n_l1) {
  if (ctl->done) return;   // uniform: `done` changes only in this kernel's last block
  const int kit = ctl->k;
  const R t = ctl_t<R>(ctl, kit & 1);
  const R a = (R)1 + t;
  const int N2 = 2 * N;
  const double l1s = lin_l1_share(l1_parts, n_l1);
  R s0 = 0, c0 = 0;
  for (int row = blockIdx.x; row < N2; row += gridDim.x) {
    R* out = rp + (int64_t)row * N2;
    if (row >= N) {
      for (int c = threadIdx.x; c < N2; c += blockDim.x) out[c] = (R)0;
      continue;
    }
    const R* qr = q + (int64_t)row * N2;
    const int64_t o = (int64_t)row * N;
    for (int c = threadIdx.x; c < N2; c += blockDim.x) {
      if (c >= N) {
        out[c] = (R)0;
        continue;
      }
      const R y = qr[c];
      const R b = res[o + c];
      const R d = y - b;
      kahan_add<R>(s0, c0, d * d);
      out[c] = a * y - t * yprev[o + c] - b;
      ycur[o + c] = y;
    }
  }
  double v[3];
  spec_block_sums<R>(s0, c0, (R)0, (R)0, l1s, (int64_t)blockIdx.x * blockDim.x < n_l1, v);
  const bool mx[3] = {false, false, false};
  if (publish_partials<3>(v, parts, ticket)) {
    double o[3];
    gather_partials<3>(o, parts, mx, ticket);
    if (threadIdx.x == 0) {
      const double oo[3] = {o[0], 0.0, o[2]};
      spec_control(oo, ctl, trace);
    }
  }
}

// FULL: D_k = P q - i~ and E_k = x_k - l, stacked [D; E] (N x N each)
template <typename R>
__global__ void lin_full_diff_kernel(const R* __restrict__ q, const R* __restrict__ res,
                                     const R* __restrict__ x, const R* __restrict__ l,
                                     R* __restrict__ de, int N, const FistaCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  const int N2 = 2 * N;
  const int64_t n2 = (int64_t)N * N;
  for (int row = blockIdx.x; row < N; row += gridDim.x) {
    const R* qr = q + (int64_t)row * N2;
    const int64_t o = (int64_t)row * N;
    for (int c = threadIdx.x; c < N; c += blockDim.x) {
      de[o + c] = qr[c] - res[o + c];
      de[n2 + o + c] = x[o + c] - l[o + c];
    }
  }
}

// FULL, on the N x N half-plane: f = (sum w g_H^2 |D^_k|^2 + w g_L^2 |E^_k|^2) / N^2
// (w = 1 on columns 0 and N/2, else 2) with the control, and the filtered
// momentum spectra U^ = g_H^2 ((1 + t) D^_k - t D^_k-1) / N^2,
// V^ = g_L^2 ((1 + t) E^_k - t E^_k-1) / N^2, stacked [U^; V^].  With ctl ==
// nullptr (the plain normal operator) t = 0 and no objective.
template <typename R>
__global__ void lin_full_spec_kernel(const C2<R>* __restrict__ dek, const C2<R>* __restrict__ dep,
                                     const R* __restrict__ gl2, const R* __restrict__ gh2,
                                     C2<R>* __restrict__ uv, int N, double* __restrict__ parts,
                                     FistaCtl* __restrict__ ctl, double* __restrict__ trace,
                                     int32_t* ticket, const double* __restrict__ l1_parts,
                                     int n_l1) {
  if (ctl && ctl->done) return;
  const R t = ctl ? ctl_t<R>(ctl, ctl->k & 1) : (R)0;
  const R a = (R)1 + t;
  const int nc = N / 2 + 1;
  const int64_t total = (int64_t)N * nc;
  const R inv = (R)(1.0 / ((double)N * N));
  const double l1s = ctl ? lin_l1_share(l1_parts, n_l1) : 0.0;
  R s0 = 0, c0 = 0, s1 = 0, c1 = 0;
  for (int row = blockIdx.x; row < N; row += gridDim.x) {
    for (int col = threadIdx.x; col < nc; col += blockDim.x) {
      const int64_t k = (int64_t)row * nc + col;
      const C2<R> D = dek[k], E = dek[total + k];
      const R gh = gh2[k], gl = gl2[k];
      C2<R> U, V;
      if (ctl) {
        const R w = (col == 0 || col == N / 2) ? (R)1 : (R)2;
        kahan_add<R>(s0, c0, w * gh * (D.x * D.x + D.y * D.y));
        kahan_add<R>(s1, c1, w * gl * (E.x * E.x + E.y * E.y));
        const C2<R> Dp = dep[k], Ep = dep[total + k];
        U.x = gh * inv * (a * D.x - t * Dp.x);
        U.y = gh * inv * (a * D.y - t * Dp.y);
        V.x = gl * inv * (a * E.x - t * Ep.x);
        V.y = gl * inv * (a * E.y - t * Ep.y);
      } else {
        U.x = gh * inv * D.x;
        U.y = gh * inv * D.y;
        V.x = gl * inv * E.x;
        V.y = gl * inv * E.y;
      }
      uv[k] = U;
      uv[total + k] = V;
    }
  }
  if (!ctl) return;
  double v[3];
  spec_block_sums<R>(s0, c0, s1, c1, l1s, (int64_t)blockIdx.x * blockDim.x < n_l1, v);
  const bool mx[3] = {false, false, false};
  if (publish_partials<3>(v, parts, ticket)) {
    double o[3];
    gather_partials<3>(o, parts, mx, ticket);
    if (threadIdx.x == 0) {
      const double oo[3] = {(o[0] + o[1]) / ((double)N * N), 0.0, o[2]};
      spec_control(oo, ctl, trace);
    }
  }
}

// Step size for the linear operator (an upper bound of 2 lambda_max):
// ||P H P^T|| <= max |H2^|, so theta = 2 M max H2^2 (LOW / SINGLE) or
// 2 M (max g_H^2 max H2^2 + max g_L^2) (FULL).  Also c0 = 0 (the objective
// is evaluated directly in the image domain).
template <typename R>
__global__ void lin_theta_kernel(const R* __restrict__ H2, int64_t n2, const R* __restrict__ gl2,
                                 const R* __restrict__ gh2, int64_t nspec, int M,
                                 double* __restrict__ parts, FistaCtl* __restrict__ ctl,
                                 int32_t* ticket) {
  double v[3] = {0.0, 0.0, 0.0};
  const bool mx[3] = {true, true, true};
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t first = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  for (int64_t k = first; k < n2; k += stride) {
    const double h = (double)H2[k];
    v[0] = fmax(v[0], h * h);
  }
  if (gl2)
    for (int64_t k = first; k < nspec; k += stride) {
      v[1] = fmax(v[1], (double)gh2[k]);
      v[2] = fmax(v[2], (double)gl2[k]);
    }
  block_reduce<3>(v, mx);
  if (publish_partials<3>(v, parts, ticket)) {
    double o[3];
    gather_partials<3>(o, parts, mx, ticket);
    if (threadIdx.x == 0) {
      const double kmax = gl2 ? o[1] * o[0] + o[2] : o[0];
      ctl->kmax = kmax;
      ctl->theta = 2.0 * M * kmax;
      ctl->inv_theta = kmax > 0 ? 1.0 / (2.0 * M * kmax) : 0.0;
      ctl->c0 = 0.0;
    }
  }
}

namespace {
int lin_rows_grid(int rows) { return std::max(1, std::min(rows, sm_count() * 8)); }
}  // namespace

template <typename R>
void launch_lin_pad(const R* x, R* xp, int N, const FistaCtl* ctl, cudaStream_t s) {
  lin_pad_kernel<R><<<lin_rows_grid(2 * N), kThreads, 0, s>>>(x, xp, N, ctl);
}
template <typename R>
void launch_lin_mul(C2<R>* S, const R* H2, int N, const FistaCtl* ctl, cudaStream_t s) {
  const int64_t n = (int64_t)2 * N * (N + 1);
  const R inv = (R)(1.0 / (4.0 * (double)N * N));
  lin_mul_kernel<R><<<nparts_for(n), kThreads, 0, s>>>(S, H2, n, inv, ctl);
}
template <typename R>
void launch_lin_crop(const R* q, const R* add, R* out, int N, double scale, const FistaCtl* ctl,
                     cudaStream_t s) {
  lin_crop_kernel<R><<<lin_rows_grid(N), kThreads, 0, s>>>(q, add, out, N, (R)scale, ctl);
}
template <typename R>
void launch_lin_low_step(const R* q, const R* res, R* ycur, const R* yprev, R* rp, int N,
                         double* parts, FistaCtl* ctl, double* trace, int32_t* ticket,
                         const double* l1_parts, int n_l1, cudaStream_t s) {
  lin_low_step_kernel<R><<<std::min(2 * N, sm_count() * 4), kThreads, 0, s>>>(
      q, res, ycur, yprev, rp, N, parts, ctl, trace, ticket, l1_parts, n_l1);
}
template <typename R>
void launch_lin_full_diff(const R* q, const R* res, const R* x, const R* l, R* de, int N,
                          const FistaCtl* ctl, cudaStream_t s) {
  lin_full_diff_kernel<R><<<lin_rows_grid(N), kThreads, 0, s>>>(q, res, x, l, de, N, ctl);
}
template <typename R>
void launch_lin_full_spec(const C2<R>* dek, const C2<R>* dep, const R* gl2, const R* gh2,
                          C2<R>* uv, int N, double* parts, FistaCtl* ctl, double* trace,
                          int32_t* ticket, const double* l1_parts, int n_l1, cudaStream_t s) {
  lin_full_spec_kernel<R><<<std::min(N, sm_count() * 4), kThreads, 0, s>>>(
      dek, dep, gl2, gh2, uv, N, parts, ctl, trace, ticket, l1_parts, n_l1);
}
template <typename R>
void launch_lin_theta(const R* H2, int N, const R* gl2, const R* gh2, int M, double* parts,
                      FistaCtl* ctl, int32_t* ticket, cudaStream_t s) {
  const int64_t n2 = (int64_t)2 * N * (N + 1);
  lin_theta_kernel<R><<<nparts_for(n2), kThreads, 0, s>>>(
      H2, n2, gl2, gh2, (int64_t)N * (N / 2 + 1), M, parts, ctl, ticket);
}

#define MS_INST(R)                                                                               \
  template void launch_ifftshift_real<R>(const R*, R*, int, cudaStream_t);                       \
  template void launch_real_part_spectrum<R>(const C2<R>*, R*, int, cudaStream_t);               \
  template void launch_filters<R>(int, double, double, const FistaCtl*, R*, R*, cudaStream_t,    \
                                  int);                                                          \
  template void launch_combine_spectra<R>(C2<R>*, const C2<R>*, const R*, const R*,              \
                                          const FistaCtl*, int, cudaStream_t);                   \
  template void launch_normal_spectrum<R>(const R*, const R*, const R*, int, int, R*, double*,   \
                                          FistaCtl*, int32_t*, cudaStream_t);                    \
  template void launch_b_spectrum<R>(const C2<R>*, const C2<R>*, const R*, const R*, const R*,   \
                                     int, C2<R>*, double*, FistaCtl*, int32_t*, cudaStream_t);   \
  template cudaError_t launch_row_r2c<R>(const R*, C2<R>*, const C2<R>*, int,                \
                                         const FistaCtl*, cudaStream_t, const JobStride&);       \
  template cudaError_t launch_row_c2r<R>(const C2<R>*, R*, const C2<R>*, int, FistaCtl*,      \
                                         const double*, int, double*, cudaStream_t,              \
                                         const JobStride&);                                      \
  template cudaError_t launch_spec_col<R>(C2<R>*, C2<R>*, const C2<R>*, const R*,             \
                                          const C2<R>*, const C2<R>*, int, double*,              \
                                          const FistaCtl*, const double*, int, cudaStream_t,     \
                                          const JobStride&);                                     \
  template void launch_spec_mul<R>(const C2<R>*, C2<R>*, const R*, const C2<R>*, int, double*,  \
                                   FistaCtl*,                                                    \
                                   double*, int32_t*, const double*, int, cudaStream_t);         \
  template void launch_spec_apply<R>(C2<R>*, const R*, int, cudaStream_t);                       \
  template void launch_image_norms<R>(const R*, int64_t, double*, FistaCtl*, int32_t*,           \
                                      cudaStream_t);                                             \
  template void launch_sigma2_hat<R>(const R*, int, double*, FistaCtl*, int32_t*, int,           \
                                     cudaStream_t);                                              \
  template void launch_axpby<R>(const R*, const R*, R*, double, double, int64_t, cudaStream_t);  \
  template void launch_l1<R>(const R*, int64_t, double*, double*, int32_t*, cudaStream_t);       \
  template void launch_dot<R>(const R*, const R*, int64_t, double*, double*, int32_t*,           \
                              cudaStream_t);                                                     \
  template void launch_normalize<R>(R*, int64_t, const double*, cudaStream_t);                   \
  template void launch_hash_fill<R>(R*, int64_t, uint64_t, cudaStream_t);                       \
  template void launch_lin_pad<R>(const R*, R*, int, const FistaCtl*, cudaStream_t);            \
  template void launch_lin_mul<R>(C2<R>*, const R*, int, const FistaCtl*, cudaStream_t);        \
  template void launch_lin_crop<R>(const R*, const R*, R*, int, double, const FistaCtl*,        \
                                   cudaStream_t);                                                \
  template void launch_lin_low_step<R>(const R*, const R*, R*, const R*, R*, int, double*,      \
                                       FistaCtl*, double*, int32_t*, const double*, int,         \
                                       cudaStream_t);                                            \
  template void launch_lin_full_diff<R>(const R*, const R*, const R*, const R*, R*, int,        \
                                        const FistaCtl*, cudaStream_t);                          \
  template void launch_lin_full_spec<R>(const C2<R>*, const C2<R>*, const R*, const R*, C2<R>*, \
                                        int, double*, FistaCtl*, double*, int32_t*,              \
                                        const double*, int, cudaStream_t);                       \
  template void launch_lin_theta<R>(const R*, int, const R*, const R*, int, double*, FistaCtl*, \
                                    int32_t*, cudaStream_t);

MS_INST(float)
MS_INST(double)

}  // namespace ms
