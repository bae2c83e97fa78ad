// The isotropic undecimated wavelet transform (IUWT, "a trous" B3-spline
// starlet) as the minor cycle's dictionary: the alternative the paper
// compares with its Daubechies dictionary (App. A.1), whose step size has no
// closed form (Sect. 3.4: power iteration).
//
// Analysis T: c_0 = x, c_j = h_j * c_{j-1}, w_j = c_{j-1} - c_j (j = 1..J),
// coefficient planes [w_1 .. w_J, c_J]; h_j is the separable B3 filter
// (1, 4, 6, 4, 1) / 16 with taps 2^(j-1) apart, periodic.  The dictionary
// is W = T^H, computed by the recursion y_J = a_{J+1} - a_J,
// y_{j-1} = (a_j - a_{j-1}) + h_j * y_j, W a = a_1 + h_1 * y_1.
//
// Every level is two launches: the column pass (5 taps down the image) into
// a scratch image, then the row pass, which also forms the level's planes
// (and, in the minor cycle, applies FISTA's step to them).  The taps are
// exact binary fractions, so FP32 and FP64 differ only in the sums.
#include "common.cuh"

namespace ms {

namespace {
constexpr int kIThreads = 256;

// per-thread compensated sum of |B_k+1| in the working precision
template <typename R> struct CompSum {
  R s = 0, c = 0;
  __device__ __forceinline__ void add(R v) {
    const R y = v - c;
    const R t = s + y;
    c = (t - s) - y;
    s = t;
  }
};
__host__ __device__ constexpr double b3(int t) {
  return t == 2 ? 6.0 / 16.0 : (t == 1 || t == 3 ? 4.0 / 16.0 : 1.0 / 16.0);
}

// The coefficient set of the minor cycle's pass: B_k (synthesis) or, for
// the analysis of pass k (ctl->k already advanced), B_k, B_k-1 and B_k+1.
template <typename R>
__device__ __forceinline__ const R* ring(const FistaPass<R>& f, int i) {
  i %= 3;
  return i == 0 ? f.B0 : (i == 1 ? f.B1 : f.B2);
}

// column pass: out = h_j (down the columns) applied to src, where src is
// the image `img` or the difference of two coefficient planes pa - pb of
// `coef` (pb < 0: plane pa alone); with a control block the coefficient
// set is the minor cycle's B_k and the kernel skips a finished cycle
template <typename R>
__global__ void __launch_bounds__(kIThreads)
    iuwt_col_kernel(FistaPass<R> f, const R* __restrict__ coef, const R* __restrict__ img,
                    int pa, int pb, R* __restrict__ out, int N, int d) {
  pdl_wait();
  pdl_trigger();
  if (f.ctl) {
    if (f.ctl->done) return;   // uniform
    coef = ring(f, f.ctl->k);
  }
  const int64_t n2 = (int64_t)N * N;
  const R* A = img ? img : coef + (int64_t)pa * n2;
  const R* B = (img || pb < 0) ? nullptr : coef + (int64_t)pb * n2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / N), q = (int)(e - (int64_t)p * N);
    R s = 0;
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      int r = p + (t - 2) * d;
      r = r < 0 ? r + N : (r >= N ? r - N : r);
      const int64_t o = (int64_t)r * N + q;
      const R v = B ? A[o] - B[o] : A[o];
      s = fma((R)b3(t), v, s);
    }
    out[e] = s;
  }
}

// row pass of the synthesis: y = h_j (along the rows) applied to tmp, plus
// planes pa - pb of the coefficient set (pb < 0: plane pa alone)
template <typename R>
__global__ void __launch_bounds__(kIThreads)
    iuwt_row_synth_kernel(FistaPass<R> f, const R* __restrict__ coef, const R* __restrict__ tmp,
                          int pa, int pb, R* __restrict__ out, int N, int d) {
  pdl_wait();
  pdl_trigger();
  if (f.ctl) {
    if (f.ctl->done) return;
    coef = ring(f, f.ctl->k);
  }
  const int64_t n2 = (int64_t)N * N;
  const R* A = coef + (int64_t)pa * n2;
  const R* B = pb < 0 ? nullptr : coef + (int64_t)pb * n2;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / N), q = (int)(e - (int64_t)p * N);
    R s = 0;
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      int c = q + (t - 2) * d;
      c = c < 0 ? c + N : (c >= N ? c - N : c);
      s = fma((R)b3(t), tmp[(int64_t)p * N + c], s);
    }
    out[e] = s + (B ? A[e] - B[e] : A[e]);
  }
}

// row pass of the analysis at level j: c_j = h_j (along the rows) applied to
// tmp (the column pass of c_{j-1}); plane j - 1 receives w_j = c_{j-1} - c_j
// and, at the last level, plane j receives c_j; c_j goes to c_out for the
// next level.  MODE 0 writes the planes to `coef`; MODE 1 (minor cycle)
// applies FISTA's step to them instead: alpha = B_k + t (B_k - B_k-1),
// B_k+1 = soft(alpha - mu g, lambda mu), and leaves the block's sum of
// |B_k+1| in l1_parts[part + blockIdx.x].
template <typename R, int MODE>
__global__ void __launch_bounds__(kIThreads)
    iuwt_row_analysis_kernel(FistaPass<R> f, R* __restrict__ coef, const R* __restrict__ tmp,
                             const R* __restrict__ c_prev, R* __restrict__ c_out, int plane,
                             int last, int N, int d, int part) {
  pdl_wait();
  pdl_trigger();
  __shared__ double red[kIThreads / 32];
  const R* cur = nullptr;
  const R* prev = nullptr;
  R* next = coef;
  R t = 0, mu = 0, thr = 0;
  if (MODE == 1) {
    if (f.ctl->done) return;   // uniform
    const int k = f.ctl->k - 1;
    cur = ring(f, k);
    prev = ring(f, k + 2);
    next = const_cast<R*>(ring(f, k + 1));
    t = ctl_t<R>(f.ctl, k & 1);
    mu = ctl_mu<R>(f.ctl);
    thr = ctl_thr<R>(f.ctl);
  }
  const int64_t n2 = (int64_t)N * N;
  CompSum<R> l1;
  auto put = [&](int pl, int64_t e, R g) {
    const int64_t o = (int64_t)pl * n2 + e;
    if (MODE == 0) {
      next[o] = g;
    } else {
      const R bc = cur[o], bp = prev[o];
      const R alpha = bc + t * (bc - bp);
      const R z = alpha - mu * g;
      const R az = fabs(z) - thr;
      const R nb = az > (R)0 ? copysign(az, z) : (R)0;
      l1.add(fabs(nb));
      next[o] = nb;
    }
  };
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n2;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int p = (int)(e / N), q = (int)(e - (int64_t)p * N);
    R s = 0;
#pragma unroll
    for (int t5 = 0; t5 < 5; ++t5) {
      int c = q + (t5 - 2) * d;
      c = c < 0 ? c + N : (c >= N ? c - N : c);
      s = fma((R)b3(t5), tmp[(int64_t)p * N + c], s);
    }
    put(plane, e, c_prev[e] - s);
    if (last) put(plane + 1, e, s);
    else c_out[e] = s;
  }
  if (MODE == 1) {
    R hi = l1.s, lo = -l1.c;
    warp_sum_comp<R>(hi, lo);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)hi + (double)lo;
    __syncthreads();
    if (threadIdx.x == 0) {
      double sum = 0.0;
      for (int w = 0; w < kIThreads / 32; ++w) sum += red[w];
      f.l1_parts[part + blockIdx.x] = sum;
    }
  }
}

int iuwt_blocks() { return sm_count() * 4; }

template <typename R> FistaPass<R> plain_pass() {
  FistaPass<R> f{};
  return f;
}
}  // namespace

int iuwt_prox_partials(int J) { return J * iuwt_blocks(); }

// Work images: two N x N buffers (the column pass and the running
// approximation / recursion), `work` [2][N][N].
template <typename R>
cudaError_t launch_iuwt_synthesis(const FistaPass<R>* fp, const R* alpha, R* x, R* work, int N,
                                  int J, cudaStream_t s) {
  const FistaPass<R> f = fp ? *fp : plain_pass<R>();
  const int nb = iuwt_blocks();
  const int64_t n2 = (int64_t)N * N;
  R* tmp = work;
  R* y = work + n2;
  cudaError_t e;
  // y_J = a_{J+1} - a_J: the first column pass reads the planes' difference
  for (int j = J; j >= 1; --j) {
    const int d = 1 << (j - 1);
    if (j == J)
      e = launch_pdl(iuwt_col_kernel<R>, dim3(nb), dim3(kIThreads), 0, s, f, alpha,
                     (const R*)nullptr, J, J - 1, tmp, N, d);
    else
      e = launch_pdl(iuwt_col_kernel<R>, dim3(nb), dim3(kIThreads), 0, s, f, alpha, (const R*)y,
                     0, -1, tmp, N, d);
    if (e != cudaSuccess) return e;
    // y_{j-1} = (a_j - a_{j-1}) + h_j y_j, and W a = a_1 + h_1 y_1
    e = launch_pdl(iuwt_row_synth_kernel<R>, dim3(nb), dim3(kIThreads), 0, s, f, alpha,
                   (const R*)tmp, j - 1, j >= 2 ? j - 2 : -1, j == 1 ? x : y, N, d);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename R>
cudaError_t launch_iuwt_analysis(const FistaPass<R>* fp, const R* img, R* alpha, R* work, int N,
                                 int J, cudaStream_t s) {
  const FistaPass<R> f = fp ? *fp : plain_pass<R>();
  const int nb = iuwt_blocks();
  const int64_t n2 = (int64_t)N * N;
  R* tmp = work;
  R* cbuf[2] = {work + n2, alpha};   // c_j ping-pong: scratch image, then a free plane
  cudaError_t e;
  const R* c = img;
  for (int j = 1; j <= J; ++j) {
    const int d = 1 << (j - 1);
    e = launch_pdl(iuwt_col_kernel<R>, dim3(nb), dim3(kIThreads), 0, s, f, (const R*)nullptr,
                   c, 0, -1, tmp, N, d);
    if (e != cudaSuccess) return e;
    // c_j into the scratch image on odd levels; on even levels into plane
    // J of the output, free until the last level (the minor cycle keeps
    // its own second scratch image there)
    R* c_out = (j & 1) ? cbuf[0] : (fp ? work + 2 * n2 : alpha + (int64_t)J * n2);
    if (fp)
      e = launch_pdl(iuwt_row_analysis_kernel<R, 1>, dim3(nb), dim3(kIThreads), 0, s, f,
                     (R*)nullptr, (const R*)tmp, c, c_out, j - 1, j == J ? 1 : 0, N, d,
                     (j - 1) * nb);
    else
      e = launch_pdl(iuwt_row_analysis_kernel<R, 0>, dim3(nb), dim3(kIThreads), 0, s, f, alpha,
                     (const R*)tmp, c, c_out, j - 1, j == J ? 1 : 0, N, d, 0);
    if (e != cudaSuccess) return e;
    c = c_out;
  }
  return cudaSuccess;
}

#define MS_INST(R)                                                                              \
  template cudaError_t launch_iuwt_synthesis<R>(const FistaPass<R>*, const R*, R*, R*, int, int, \
                                                cudaStream_t);                                   \
  template cudaError_t launch_iuwt_analysis<R>(const FistaPass<R>*, const R*, R*, R*, int, int,  \
                                               cudaStream_t);
MS_INST(float)
MS_INST(double)
#undef MS_INST

}  // namespace ms
