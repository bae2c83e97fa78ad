// Dictionary kernels: W = [Psi_1 .. Psi_M], Psi_m the periodized orthonormal
// 2-D Daubechies db_m transform with J levels (Sect. 4.3, App. A.1; the
// closed-form Lipschitz constant of Sect. 3.4 assumes orthogonal bases with
// circular boundaries).
//
// One analysis level on an n x n block X is Y = T X T^T (rows filtered along x
// first, then columns along y), T the periodized analysis matrix:
//   a_i = sum_k h_k x[(2i + k) mod n],  d_i = sum_k g_k x[(2i + k) mod n],
//   g_k = (-1)^k h_{L-1-k}.
// Mallat layout: [0,h)^2 approximation, rows [0,h) x cols [h,n) low-y/high-x,
// rows [h,n) x cols [0,h) high-y/low-x, [h,n)^2 high/high, h = n/2.
// Synthesis is the transpose X = T^T Y T.
//
// The analysis kernel of the minor cycle also does FISTA's step (Algorithm 1):
// it builds the gradient image 2((1+t) y_k - t y_{k-1} - b) on the fly, and at
// each coefficient forms alpha = B_k + t (B_k - B_{k-1}) and writes
// B_{k+1} = soft(alpha - g / theta, lambda / theta), so the gradient
// coefficients never reach global memory.
#include "common.cuh"

namespace ms {

__constant__ double c_hd[kMaxBases][kMaxTaps];
__constant__ double c_gd[kMaxBases][kMaxTaps];
__constant__ float c_hf[kMaxBases][kMaxTaps];
__constant__ float c_gf[kMaxBases][kMaxTaps];
__constant__ int c_len[kMaxBases];

void set_wavelet_filters(const double* h, const int* len, int nbases) {
  double hd[kMaxBases][kMaxTaps] = {}, gd[kMaxBases][kMaxTaps] = {};
  float hf[kMaxBases][kMaxTaps] = {}, gf[kMaxBases][kMaxTaps] = {};
  int l[kMaxBases] = {};
  for (int m = 0; m < nbases; ++m) {
    l[m] = len[m];
    for (int k = 0; k < len[m]; ++k) {
      hd[m][k] = h[m * kMaxTaps + k];
      gd[m][k] = ((k & 1) ? -1.0 : 1.0) * h[m * kMaxTaps + len[m] - 1 - k];
      hf[m][k] = (float)hd[m][k];
      gf[m][k] = (float)gd[m][k];
    }
  }
  cudaMemcpyToSymbol(c_hd, hd, sizeof(hd));
  cudaMemcpyToSymbol(c_gd, gd, sizeof(gd));
  cudaMemcpyToSymbol(c_hf, hf, sizeof(hf));
  cudaMemcpyToSymbol(c_gf, gf, sizeof(gf));
  cudaMemcpyToSymbol(c_len, l, sizeof(l));
}

namespace {
template <typename R> __device__ __forceinline__ R fh(int m, int k);
template <typename R> __device__ __forceinline__ R fg(int m, int k);
template <> __device__ __forceinline__ float fh<float>(int m, int k) { return c_hf[m][k]; }
template <> __device__ __forceinline__ float fg<float>(int m, int k) { return c_gf[m][k]; }
template <> __device__ __forceinline__ double fh<double>(int m, int k) { return c_hd[m][k]; }
template <> __device__ __forceinline__ double fg<double>(int m, int k) { return c_gd[m][k]; }

constexpr int kSynTile = 64;                      // synthesis output tile side
constexpr int kSynCnt = kSynTile / 2 + kMaxTaps / 2 - 1;   // subband positions needed
constexpr int kAnaTile = 32;                      // analysis output tile side (per subband)
constexpr int kAnaCnt = 2 * kAnaTile + kMaxTaps - 2;       // input positions needed
constexpr int kThreads = 256;

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// deterministic block sum of a double (all threads of the block call it)
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;   // valid in thread 0
}
}  // namespace

// ------------------------------------------------------------------ synthesis
// Level j (h = N >> j subband side, n = 2h output side).  Approximation
// input: level J reads the top-left block of each coefficient plane, other
// levels read the LL buffer written by the level above.  Level 1 sums the M
// bases into x; other levels write LL_{j-1} per basis.
template <typename R>
__global__ void __launch_bounds__(kThreads)
    synthesis_kernel(const R* const* __restrict__ coef3, const R* __restrict__ ll_in,
                     R* __restrict__ ll_out, R* __restrict__ x, int N, int j, int J, int M,
                     const FistaCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sA = reinterpret_cast<R*>(smem_raw);      // [cnt][cnt] approximation
  R* sBx = sA + kSynCnt * kSynCnt;             // low-y / high-x
  R* sBy = sBx + kSynCnt * kSynCnt;            // high-y / low-x
  R* sD = sBy + kSynCnt * kSynCnt;             // high / high
  R* zlo = sD + kSynCnt * kSynCnt;             // [TS][cnt]
  R* zhi = zlo + kSynTile * kSynCnt;

  const R* coef = coef3[ctl ? (ctl->k % 3) : 0];
  const int h = N >> j, n = 2 * h;
  const int TS = n < kSynTile ? n : kSynTile;
  const int cnt = TS / 2 + kMaxTaps / 2 - 1;
  const int tiles_x = n / TS;
  const int r0 = (blockIdx.x / tiles_x) * TS, c0 = (blockIdx.x % tiles_x) * TS;
  const int i0 = r0 / 2 - (kMaxTaps / 2 - 1), j0 = c0 / 2 - (kMaxTaps / 2 - 1);
  const bool sum_bases = (j == 1);
  const int m_lo = sum_bases ? 0 : blockIdx.y, m_hi = sum_bases ? M : blockIdx.y + 1;
  constexpr int kPer = (kSynTile * kSynTile) / kThreads;   // outputs per thread (16)
  R acc[kPer];
#pragma unroll
  for (int q = 0; q < kPer; ++q) acc[q] = (R)0;

  for (int m = m_lo; m < m_hi; ++m) {
    const R* plane = coef + (int64_t)m * N * N;
    const R* llp = (j == J) ? nullptr : ll_in + (int64_t)m * h * h;
    const int L = c_len[m];
    for (int e = threadIdx.x; e < cnt * cnt; e += blockDim.x) {
      int a = e / cnt, b = e - a * cnt;
      int iy = wrap(i0 + a, h), ix = wrap(j0 + b, h);
      sA[a * kSynCnt + b] = llp ? llp[(int64_t)iy * h + ix] : plane[(int64_t)iy * N + ix];
      sBx[a * kSynCnt + b] = plane[(int64_t)iy * N + h + ix];
      sBy[a * kSynCnt + b] = plane[(int64_t)(h + iy) * N + ix];
      sD[a * kSynCnt + b] = plane[(int64_t)(h + iy) * N + h + ix];
    }
    __syncthreads();
    // columns (y): z[r][b] = sum_k h_k S[(r - k)/2] ...   (k = r mod 2, r mod 2 + 2, ...)
    for (int e = threadIdx.x; e < TS * cnt; e += blockDim.x) {
      int r = e / cnt, b = e - r * cnt;
      R lo = 0, hi = 0;
      for (int k = r & 1; k < L; k += 2) {
        int a = ((r - k) >> 1) + (kMaxTaps / 2 - 1);
        R hk = fh<R>(m, k), gk = fg<R>(m, k);
        lo += hk * sA[a * kSynCnt + b] + gk * sBy[a * kSynCnt + b];
        hi += hk * sBx[a * kSynCnt + b] + gk * sD[a * kSynCnt + b];
      }
      zlo[r * kSynCnt + b] = lo;
      zhi[r * kSynCnt + b] = hi;
    }
    __syncthreads();
    // rows (x)
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int e = threadIdx.x + q * kThreads;
      if (e < TS * TS) {
        int r = e / TS, c = e - r * TS;
        R s = 0;
        for (int k = c & 1; k < L; k += 2) {
          int b = ((c - k) >> 1) + (kMaxTaps / 2 - 1);
          s += fh<R>(m, k) * zlo[r * kSynCnt + b] + fg<R>(m, k) * zhi[r * kSynCnt + b];
        }
        if (sum_bases) {
          acc[q] += s;
        } else {
          ll_out[(int64_t)m * n * n + (int64_t)(r0 + r) * n + c0 + c] = s;
        }
      }
    }
    __syncthreads();
  }
  if (sum_bases) {
#pragma unroll
    for (int q = 0; q < kPer; ++q) {
      int e = threadIdx.x + q * kThreads;
      if (e < TS * TS) {
        int r = e / TS, c = e - r * TS;
        x[(int64_t)(r0 + r) * N + c0 + c] = acc[q];
      }
    }
  }
}

template <typename R>
void launch_synthesis3(const R* const* coef3_dev, R* x, R* tmp, WaveletGeom g,
                       const FistaCtl* ctl, cudaStream_t s, int only_level) {
  const size_t smem = (size_t)(4 * kSynCnt * kSynCnt + 2 * kSynTile * kSynCnt) * sizeof(R);
  auto k = synthesis_kernel<R>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t half = (int64_t)g.M * (g.N / 2) * (g.N / 2);
  for (int j = g.J; j >= 1; --j) {
    if (only_level > 0 && j != only_level) continue;
    int h = g.N >> j, n = 2 * h;
    int TS = n < kSynTile ? n : kSynTile;
    int tiles = (n / TS) * (n / TS);
    const R* ll_in = (j == g.J) ? nullptr : tmp + ((j + 1) & 1) * half;
    R* ll_out = tmp + (j & 1) * half;
    dim3 grid(tiles, j == 1 ? 1 : g.M);
    k<<<grid, kThreads, smem, s>>>(coef3_dev, ll_in, ll_out, x, g.N, j, g.J, g.M, ctl);
  }
}

// ------------------------------------------------------------------ analysis
// Level j on an n x n input (n = N >> (j-1)), output subbands of side h = n/2.
// MODE 0: plain analysis (W^H x), input x (level 1) or LL_{j-1}; outputs to
//         coefficient planes, approximation to the LL buffer for j < J.
// MODE 1: FISTA step; level 1 input is the gradient image built from
//         y_k, y_{k-1}, b; detail (and level-J approximation) outputs go
//         through the prox into B_{k+1}.
template <typename R, int MODE>
__global__ void __launch_bounds__(kThreads)
    analysis_kernel(const R* __restrict__ x_in, const R* __restrict__ ll_in,
                    R* __restrict__ ll_out, R* __restrict__ out_plain, ProxArgs pa,
                    R* const* __restrict__ B3, R* const* __restrict__ Yh2, int N, int j,
                    int J, int M, FistaCtl* __restrict__ ctl, double* __restrict__ l1_parts,
                    int part_base, int32_t* __restrict__ ticket, int total_parts) {
  if (MODE == 1 && ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double red[kThreads / 32];
  R* sIn = reinterpret_cast<R*>(smem_raw);     // [kAnaCnt][kAnaCnt]
  R* slo = sIn + kAnaCnt * kAnaCnt;            // [kAnaCnt][TO]
  R* shi = slo + kAnaCnt * kAnaTile;

  const int n = N >> (j - 1), h = n / 2;
  const int TO = h < kAnaTile ? h : kAnaTile;
  const int cnt = 2 * TO + kMaxTaps - 2;
  const int tiles_x = h / TO;
  const int o0y = (blockIdx.x / tiles_x) * TO, o0x = (blockIdx.x % tiles_x) * TO;
  const int p0y = 2 * o0y, p0x = 2 * o0x;
  const bool level1 = (j == 1);
  const int m_lo = level1 ? 0 : blockIdx.y, m_hi = level1 ? M : blockIdx.y + 1;

  R t = 0, mu = 0, thr = 0;
  const R* cur = nullptr;
  const R* prev = nullptr;
  R* next = nullptr;
  const R* ykm = nullptr;
  R* ysave = nullptr;
  if (MODE == 1) {
    const int k = ctl->k;
    ykm = Yh2[k % 2];
    ysave = Yh2[(k + 1) % 2];
    double td = k >= 2 ? (double)(k - 1) / (double)(k + 2) : 0.0;
    t = (R)td;
    mu = (R)ctl->inv_theta;
    thr = (R)(ctl->lam * ctl->inv_theta);
    cur = B3[k % 3];
    prev = B3[(k + 2) % 3];
    next = B3[(k + 1) % 3];
  }
  double l1 = 0.0;

  // level 1: the input is shared by all bases, load it once
  auto load_input = [&](int m) {
    for (int e = threadIdx.x; e < cnt * cnt; e += blockDim.x) {
      int a = e / cnt, b = e - a * cnt;
      int py = wrap(p0y + a, n), px = wrap(p0x + b, n);
      int64_t p = (int64_t)py * n + px;
      R v;
      if (level1) {
        if (MODE == 1) {
          const R* yk = static_cast<const R*>(pa.ywork);
          const R* bb = static_cast<const R*>(pa.b);
          R yc = yk[p];
          v = (R)2 * (((R)1 + t) * yc - t * ykm[p] - bb[p]);
          if (a < 2 * TO && b < 2 * TO) ysave[p] = yc;
        } else {
          v = x_in[p];
        }
      } else {
        v = ll_in[(int64_t)m * n * n + p];
      }
      sIn[a * kAnaCnt + b] = v;
    }
  };
  if (level1) {
    load_input(0);
    __syncthreads();
  }
  for (int m = m_lo; m < m_hi; ++m) {
    if (!level1) {
      load_input(m);
      __syncthreads();
    }
    const int L = c_len[m];
    const int rows = 2 * TO + L - 2;
    // rows: filter along x
    for (int e = threadIdx.x; e < rows * TO; e += blockDim.x) {
      int a = e / TO, c = e - a * TO;
      R lo = 0, hi = 0;
      const R* src = sIn + a * kAnaCnt + 2 * c;
      for (int k = 0; k < L; ++k) {
        R v = src[k];
        lo += fh<R>(m, k) * v;
        hi += fg<R>(m, k) * v;
      }
      slo[a * kAnaTile + c] = lo;
      shi[a * kAnaTile + c] = hi;
    }
    __syncthreads();
    // columns: filter along y, four subbands
    R* plane_out = (MODE == 1 ? next : out_plain) + (int64_t)m * N * N;
    const R* plane_cur = MODE == 1 ? cur + (int64_t)m * N * N : nullptr;
    const R* plane_prev = MODE == 1 ? prev + (int64_t)m * N * N : nullptr;
    for (int e = threadIdx.x; e < TO * TO; e += blockDim.x) {
      int r = e / TO, c = e - r * TO;
      R ll = 0, lh = 0, hl = 0, hh = 0;
      for (int k = 0; k < L; ++k) {
        R hk = fh<R>(m, k), gk = fg<R>(m, k);
        R vl = slo[(2 * r + k) * kAnaTile + c], vh = shi[(2 * r + k) * kAnaTile + c];
        ll += hk * vl;
        lh += hk * vh;
        hl += gk * vl;
        hh += gk * vh;
      }
      const int oy = o0y + r, ox = o0x + c;
      // (value, row, col) of the three detail subbands, plus the approximation
      R vals[4] = {lh, hl, hh, ll};
      int rows_[4] = {oy, h + oy, h + oy, oy};
      int cols_[4] = {h + ox, ox, h + ox, ox};
      const int nsub = (j == J) ? 4 : 3;
      for (int sb = 0; sb < nsub; ++sb) {
        int64_t idx = (int64_t)rows_[sb] * N + cols_[sb];
        if (MODE == 1) {
          R bc = plane_cur[idx], bp = plane_prev[idx];
          R alpha = bc + t * (bc - bp);
          R z = alpha - mu * vals[sb];
          R az = fabs(z) - thr;
          R nb = az > (R)0 ? copysign(az, z) : (R)0;
          plane_out[idx] = nb;
          l1 += fabs((double)nb);
        } else {
          plane_out[idx] = vals[sb];
        }
      }
      if (j < J) ll_out[(int64_t)m * h * h + (int64_t)oy * h + ox] = ll;
    }
    __syncthreads();
  }

  if (MODE == 1) {
    double bsum = block_sum(l1, red);
    const int pid = part_base + blockIdx.y * gridDim.x + blockIdx.x;
    if (threadIdx.x == 0) {
      l1_parts[pid] = bsum;
      __threadfence();
    }
    if (j == J) {
      __shared__ int last;
      if (threadIdx.x == 0) {
        int prior = atomicAdd(ticket, 1);
        last = (prior == (int)(gridDim.x * gridDim.y) - 1);
      }
      __syncthreads();
      if (last && threadIdx.x == 0) {
        __threadfence();
        double s = 0;
        const volatile double* vp = l1_parts;
        for (int i = 0; i < total_parts; ++i) s += vp[i];
        ctl->l1_cur = s;
        ctl->k = ctl->k + 1;
        *ticket = 0;
        __threadfence();
      }
    }
  }
}

namespace {
size_t analysis_smem_bytes(size_t rsz) {
  return (size_t)(kAnaCnt * kAnaCnt + 2 * kAnaCnt * kAnaTile) * rsz;
}
}  // namespace

int analysis_prox_partials(WaveletGeom g) {
  int total = 0;
  for (int j = 1; j <= g.J; ++j) {
    int h = g.N >> j;
    int TO = h < kAnaTile ? h : kAnaTile;
    int tiles = (h / TO) * (h / TO);
    total += tiles * (j == 1 ? 1 : g.M);
  }
  return total;
}

template <typename R>
void launch_analysis(const R* x, R* coef, R* tmp, WaveletGeom g, cudaStream_t s) {
  const size_t smem = analysis_smem_bytes(sizeof(R));
  auto k = analysis_kernel<R, 0>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t half = (int64_t)g.M * (g.N / 2) * (g.N / 2);
  ProxArgs none{};
  for (int j = 1; j <= g.J; ++j) {
    int h = g.N >> j;
    int TO = h < kAnaTile ? h : kAnaTile;
    int tiles = (h / TO) * (h / TO);
    const R* ll_in = (j == 1) ? nullptr : tmp + ((j - 1) & 1) * half;
    R* ll_out = tmp + (j & 1) * half;
    dim3 grid(tiles, j == 1 ? 1 : g.M);
    k<<<grid, kThreads, smem, s>>>(x, ll_in, ll_out, coef, none, nullptr, nullptr, g.N, j,
                                   g.J, g.M, nullptr, nullptr, 0, nullptr, 0);
  }
}

template <typename R>
void launch_analysis_prox3(ProxArgs a, R* const* B3_dev, R* const* Yh2_dev, R* tmp,
                           WaveletGeom g, FistaCtl* ctl, int32_t* ticket, double* l1_parts,
                           cudaStream_t s, int only_level) {
  const size_t smem = analysis_smem_bytes(sizeof(R));
  auto k = analysis_kernel<R, 1>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  const int64_t half = (int64_t)g.M * (g.N / 2) * (g.N / 2);
  const int total = analysis_prox_partials(g);
  int base = 0;
  for (int j = 1; j <= g.J; ++j) {
    int h = g.N >> j;
    int TO = h < kAnaTile ? h : kAnaTile;
    int tiles = (h / TO) * (h / TO);
    const R* ll_in = (j == 1) ? nullptr : tmp + ((j - 1) & 1) * half;
    R* ll_out = tmp + (j & 1) * half;
    dim3 grid(tiles, j == 1 ? 1 : g.M);
    if (only_level <= 0 || j == only_level)
      k<<<grid, kThreads, smem, s>>>(nullptr, ll_in, ll_out, nullptr, a, B3_dev, Yh2_dev, g.N,
                                     j, g.J, g.M, ctl, l1_parts, base, ticket, total);
    base += tiles * (j == 1 ? 1 : g.M);
  }
}

template void launch_synthesis3<float>(const float* const*, float*, float*, WaveletGeom,
                                       const FistaCtl*, cudaStream_t, int);
template void launch_synthesis3<double>(const double* const*, double*, double*, WaveletGeom,
                                        const FistaCtl*, cudaStream_t, int);
template void launch_analysis<float>(const float*, float*, float*, WaveletGeom, cudaStream_t);
template void launch_analysis<double>(const double*, double*, double*, WaveletGeom,
                                      cudaStream_t);
template void launch_analysis_prox3<float>(ProxArgs, float* const*, float* const*, float*,
                                           WaveletGeom, FistaCtl*, int32_t*, double*,
                                           cudaStream_t, int);
template void launch_analysis_prox3<double>(ProxArgs, double* const*, double* const*, double*,
                                            WaveletGeom, FistaCtl*, int32_t*, double*,
                                            cudaStream_t, int);

}  // namespace ms
