// The learned warm start: a small U-Net mapping [step-one image, long-baseline
// dirty image] to a starting image for step two (Sect. 3.3), trained on pairs
// the method itself produces.  Activations and weights are bfloat16, every
// product accumulates in FP32 on the tensor cores (mma.sync m16n8k16), master
// weights and the Adam state are FP32, the loss reduces in FP64.
//
// Every convolution is one GEMM over an im2col matrix:
//   forward        Y[P][Co]   = cols(X)[P][K] . W[Co][K]^T          (+ bias, ReLU)
//   data gradient  dcols[P][K] = dZ[P][Co] . Wt[K][Co]^T, then col2im
//   weight grad.   dW[Co][K]  = dZt[Co][P] . colsT(X)[K][P]^T
// with K = 9 Ci (padded to a multiple of 16 with zeros), so a single
// "A[M][K] . B[N][K]^T" kernel (both operands K-contiguous) serves all three.
// Rounding points match the oracle: inputs, weights and stored activations
// (after ReLU, after pooling) are rounded to bfloat16, and so is every
// pre-activation gradient before it enters a product.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "mstep.h"

namespace ms {
namespace {
using bf16 = __nv_bfloat16;
constexpr int kT = 256;

int blocks(int64_t n, int cap = 0) {
  if (cap <= 0) cap = sm_count() * 16;
  int64_t b = (n + kT - 1) / kT;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}
int pad16(int x) { return (x + 15) / 16 * 16; }

__device__ __forceinline__ unsigned su32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

// ------------------------------------------------------------------ GEMM
// C[M][N] = A[M][K] . Bt[N][K]^T (+ bias[n]) (ReLU), bf16 operands, FP32
// accumulation; K a multiple of 16, M and N arbitrary.  Block tile 64 x 64,
// four warps of 32 x 32, k-tiles of 32 staged by cp.async (zero-filled past
// the matrix edges), double-buffered.  Split over K: block z takes the k in
// [z kchunk, (z + 1) kchunk) (kchunk a multiple of 32) and writes its
// partial product to C + z M ldc (FP32 output, no bias or ReLU).
constexpr int GT = 64, GK = 32, GS = 40;   // tile, k-tile, padded smem row (bf16)

__device__ __forceinline__ void cp16(void* dst, const void* src, bool ok) {
  const int n = ok ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(su32(dst)), "l"(src), "r"(n)
               : "memory");
}

template <bool OUT_BF16>
__global__ void __launch_bounds__(128) gemm_tn_kernel(const bf16* __restrict__ A, int lda,
                                                      const bf16* __restrict__ Bt, int ldb,
                                                      void* __restrict__ C, int ldc, int M, int N,
                                                      int K, const float* __restrict__ bias,
                                                      int relu, int kchunk) {
  __shared__ __align__(16) bf16 sA[2][GT][GS];
  __shared__ __align__(16) bf16 sB[2][GT][GS];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int gid = lane >> 2, tig = lane & 3;
  const int m0 = blockIdx.y * GT, n0 = blockIdx.x * GT;
  const int kbeg = blockIdx.z * kchunk;
  const int kend = min(K, kbeg + kchunk);
  if (!OUT_BF16 && gridDim.z > 1) C = static_cast<float*>(C) + (size_t)blockIdx.z * M * ldc;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.0f;

  auto load = [&](int buf, int k0) {
#pragma unroll
    for (int c = tid; c < GT * (GK / 8); c += 128) {
      const int r = c >> 2, kc = (c & 3) * 8;
      const bool kok = k0 + kc < kend;
      const int gm = m0 + r, gn = n0 + r;
      const bool aok = kok && gm < M, bok = kok && gn < N;
      cp16(&sA[buf][r][kc], aok ? A + (size_t)gm * lda + k0 + kc : A, aok);
      cp16(&sB[buf][r][kc], bok ? Bt + (size_t)gn * ldb + k0 + kc : Bt, bok);
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const int nk = kend > kbeg ? (kend - kbeg + GK - 1) / GK : 0;
  if (nk > 0) load(0, kbeg);
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < nk) {
      load(buf ^ 1, kbeg + (kt + 1) * GK);
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; kk += 16) {
      unsigned a[2][4], b[4][2];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int r = wm + mi * 16 + gid;
        a[mi][0] = *reinterpret_cast<const unsigned*>(&sA[buf][r][kk + tig * 2]);
        a[mi][1] = *reinterpret_cast<const unsigned*>(&sA[buf][r + 8][kk + tig * 2]);
        a[mi][2] = *reinterpret_cast<const unsigned*>(&sA[buf][r][kk + 8 + tig * 2]);
        a[mi][3] = *reinterpret_cast<const unsigned*>(&sA[buf][r + 8][kk + 8 + tig * 2]);
      }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int cn = wn + ni * 8 + gid;
        b[ni][0] = *reinterpret_cast<const unsigned*>(&sB[buf][cn][kk + tig * 2]);
        b[ni][1] = *reinterpret_cast<const unsigned*>(&sB[buf][cn][kk + 8 + tig * 2]);
      }
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni)
          asm volatile(
              "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
              "{%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
              : "+f"(acc[mi][ni][0]), "+f"(acc[mi][ni][1]), "+f"(acc[mi][ni][2]),
                "+f"(acc[mi][ni][3])
              : "r"(a[mi][0]), "r"(a[mi][1]), "r"(a[mi][2]), "r"(a[mi][3]), "r"(b[ni][0]),
                "r"(b[ni][1]));
    }
    __syncthreads();
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = m0 + wm + mi * 16 + gid + (q >= 2 ? 8 : 0);
        const int c = n0 + wn + ni * 8 + tig * 2 + (q & 1);
        if (r >= M || c >= N) continue;
        float v = acc[mi][ni][q] + (bias ? bias[c] : 0.0f);
        if (relu) v = fmaxf(v, 0.0f);
        if (OUT_BF16)
          static_cast<bf16*>(C)[(size_t)r * ldc + c] = __float2bfloat16_rn(v);
        else
          static_cast<float*>(C)[(size_t)r * ldc + c] = v;
      }
}

void gemm_tn(const bf16* A, int lda, const bf16* Bt, int ldb, void* C, int ldc, int M, int N,
             int K, const float* bias, bool relu, bool out_bf16, cudaStream_t s) {
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT);
  if (out_bf16)
    gemm_tn_kernel<true><<<grid, 128, 0, s>>>(A, lda, Bt, ldb, C, ldc, M, N, K, bias, relu, K);
  else
    gemm_tn_kernel<false><<<grid, 128, 0, s>>>(A, lda, Bt, ldb, C, ldc, M, N, K, bias, relu, K);
}

// out[i] = sum over z of part[z n + i], z in order (a fixed summation order)
__global__ void sum_splits_kernel(const float* __restrict__ part, int splits, int64_t n,
                                  float* __restrict__ out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float a = 0.0f;
    for (int z = 0; z < splits; ++z) a += part[(int64_t)z * n + i];
    out[i] = a;
  }
}

// K (pixels) per split of the weight-gradient products, and the most splits
constexpr int kSplitRows = 4096, kMaxSplits = 64;
int splits_for(int64_t K) {
  return (int)std::min<int64_t>(kMaxSplits, std::max<int64_t>(1, K / kSplitRows));
}

// C[M][N] (ldc = N) as gemm_tn's FP32 form, with K split over `splits`
// blocks in z whose partial products go to `part` (splits M N floats) and
// are then summed in split order.
void gemm_tn_splitk(const bf16* A, int lda, const bf16* Bt, int ldb, float* part, float* C,
                    int M, int N, int K, int splits, cudaStream_t s) {
  if (splits <= 1) {
    gemm_tn(A, lda, Bt, ldb, C, N, M, N, K, nullptr, false, false, s);
    return;
  }
  const int kchunk = ((K + splits - 1) / splits + GK - 1) / GK * GK;
  const int z = (K + kchunk - 1) / kchunk;
  dim3 grid((N + GT - 1) / GT, (M + GT - 1) / GT, z);
  gemm_tn_kernel<false><<<grid, 128, 0, s>>>(A, lda, Bt, ldb, part, N, M, N, K, nullptr, 0,
                                             kchunk);
  const int64_t n = (int64_t)M * N;
  sum_splits_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, s>>>(part, z, n, C);
}

// ------------------------------------------------------------------ layers
// im2col of a 3x3 'same' window: cols[p][k], k = tap * C + c (tap = ky * 3 + kx),
// zero outside the image and for k >= 9 C (up to Kp).
__global__ void im2col_kernel(const bf16* __restrict__ x, int H, int W, int C, int Kp,
                              bf16* __restrict__ cols) {
  const int64_t total = (int64_t)H * W * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / Kp;
    const int k = (int)(e - p * Kp);
    bf16 v = __float2bfloat16_rn(0.0f);
    if (k < 9 * C) {
      const int tap = k / C, c = k - tap * C;
      const int py = (int)(p / W) + tap / 3 - 1, px = (int)(p % W) + tap % 3 - 1;
      if (py >= 0 && py < H && px >= 0 && px < W) v = x[((int64_t)py * W + px) * C + c];
    }
    cols[e] = v;
  }
}

// transposed im2col: colsT[k][p]
__global__ void im2col_t_kernel(const bf16* __restrict__ x, int H, int W, int C, int Kp,
                                bf16* __restrict__ colsT) {
  const int64_t P = (int64_t)H * W, total = P * Kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / P);
    const int64_t p = e - (int64_t)k * P;
    bf16 v = __float2bfloat16_rn(0.0f);
    if (k < 9 * C) {
      const int tap = k / C, c = k - tap * C;
      const int py = (int)(p / W) + tap / 3 - 1, px = (int)(p % W) + tap % 3 - 1;
      if (py >= 0 && py < H && px >= 0 && px < W) v = x[((int64_t)py * W + px) * C + c];
    }
    colsT[e] = v;
  }
}

// col2im (adjoint of im2col): dx[p][c] = sum_taps dcols[p - tap offset][tap * C + c]
__global__ void col2im_kernel(const float* __restrict__ dcols, int H, int W, int C, int Kp,
                              float* __restrict__ dx) {
  const int64_t total = (int64_t)H * W * C;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / C;
    const int c = (int)(e - p * C);
    const int y = (int)(p / W), x = (int)(p % W);
    float s = 0.0f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int qy = y - (tap / 3 - 1), qx = x - (tap % 3 - 1);
      if (qy >= 0 && qy < H && qx >= 0 && qx < W)
        s += dcols[((int64_t)qy * W + qx) * Kp + tap * C + c];
    }
    dx[e] = s;
  }
}

__global__ void to_bf16_kernel(const float* __restrict__ in, int64_t n, bf16* __restrict__ out) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x)
    out[e] = __float2bfloat16_rn(in[e]);
}

// weights: master [Co][9 Ci] (FP32) -> W [Co][Kp] and Wt [Kp][Cop] (bf16, zero padded)
__global__ void pack_weights_kernel(const float* __restrict__ w, int Co, int Ci, int Kp, int Cop,
                                    bf16* __restrict__ Wb, bf16* __restrict__ Wt) {
  const int64_t total = (int64_t)Kp * Cop;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / Cop), co = (int)(e - (int64_t)k * Cop);
    const bf16 v =
        __float2bfloat16_rn(co < Co && k < 9 * Ci ? w[(int64_t)co * 9 * Ci + k] : 0.0f);
    Wt[e] = v;
    if (co < Co) Wb[(int64_t)co * Kp + k] = v;
  }
}

// 2x2 average pooling of bf16 [H][W][C] -> bf16 [H/2][W/2][C]
__global__ void avgpool_kernel(const bf16* __restrict__ x, int H, int W, int C,
                               bf16* __restrict__ y) {
  const int Ho = H / 2, Wo = W / 2;
  const int64_t total = (int64_t)Ho * Wo * C;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / C;
    const int c = (int)(e - q * C);
    const int oy = (int)(q / Wo), ox = (int)(q % Wo);
    const int64_t b = ((int64_t)(2 * oy) * W + 2 * ox) * C + c;
    const float s = __bfloat162float(x[b]) + __bfloat162float(x[b + C]) +
                    __bfloat162float(x[b + (int64_t)W * C]) +
                    __bfloat162float(x[b + (int64_t)W * C + C]);
    y[e] = __float2bfloat16_rn(0.25f * s);
  }
}

// concatenation [nearest 2x upsampling of lo (Cl channels), skip (Cs)] -> cat
__global__ void upcat_kernel(const bf16* __restrict__ lo, int Cl, const bf16* __restrict__ skip,
                             int Cs, int H, int W, bf16* __restrict__ cat) {
  const int Cc = Cl + Cs;
  const int64_t total = (int64_t)H * W * Cc;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / Cc;
    const int c = (int)(e - p * Cc);
    const int y = (int)(p / W), x = (int)(p % W);
    cat[e] = c < Cl ? lo[((int64_t)(y / 2) * (W / 2) + x / 2) * Cl + c] : skip[p * Cs + c - Cl];
  }
}

// pre-activation gradient: dz = bf16(g * relu'(out)) into [P][Cop] (zero padded)
__global__ void relu_grad_kernel(const float* __restrict__ g, int ldg, const bf16* __restrict__ out,
                                 int64_t P, int Co, int Cop, bf16* __restrict__ dz) {
  const int64_t total = P * Cop;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / Cop;
    const int c = (int)(e - p * Cop);
    float v = 0.0f;
    if (c < Co) {
      v = g[p * ldg + c];
      if (out && !(__bfloat162float(out[p * Co + c]) > 0.0f)) v = 0.0f;
    }
    dz[e] = __float2bfloat16_rn(v);
  }
}

// dzT[c][p] = dz[p][c]
__global__ void transpose_kernel(const bf16* __restrict__ dz, int64_t P, int Cop,
                                 bf16* __restrict__ dzT) {
  const int64_t total = P * Cop;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(e / P);
    const int64_t p = e - (int64_t)c * P;
    dzT[e] = dz[p * Cop + c];
  }
}

// bias gradient: db[c] = sum_p dz[p][c], one block per channel, fixed order
__global__ void colsum_kernel(const bf16* __restrict__ dz, int64_t P, int Cop, float* __restrict__ db) {
  __shared__ float red[kT / 32];
  const int c = blockIdx.x;
  float s = 0.0f;
  for (int64_t p = threadIdx.x; p < P; p += blockDim.x) s += __bfloat162float(dz[p * Cop + c]);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < kT / 32; ++w) t += red[w];
    db[c] = t;
  }
}

// gradient through 2x2 average pooling, added to the skip gradient:
// ds[p][c] += dpool[p / 2][c] / 4
__global__ void avgpool_grad_kernel(const float* __restrict__ dpool, int H, int W, int C,
                                    float* __restrict__ ds) {
  const int64_t total = (int64_t)H * W * C;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / C;
    const int c = (int)(e - p * C);
    const int y = (int)(p / W), x = (int)(p % W);
    ds[e] += 0.25f * dpool[((int64_t)(y / 2) * (W / 2) + x / 2) * C + c];
  }
}

// split the concatenation's gradient: dlo[q][c] = sum of the 2x2 block of
// dcat[.][c] (c < Cl); dskip[p][c] = dcat[p][Cl + c]
__global__ void upcat_grad_kernel(const float* __restrict__ dcat, int Cl, int Cs, int H, int W,
                                  float* __restrict__ dlo, float* __restrict__ dskip) {
  const int Cc = Cl + Cs;
  const int64_t total = (int64_t)H * W * Cs;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = e / Cs;
    const int c = (int)(e - p * Cs);
    dskip[e] = dcat[p * Cc + Cl + c];
  }
  const int Wo = W / 2;
  const int64_t tlo = (int64_t)(H / 2) * Wo * Cl;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tlo;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / Cl;
    const int c = (int)(e - q * Cl);
    const int y = 2 * (int)(q / Wo), x = 2 * (int)(q % Wo);
    const int64_t b = ((int64_t)y * W + x) * Cc + c;
    dlo[e] = dcat[b] + dcat[b + Cc] + dcat[b + (int64_t)W * Cc] + dcat[b + (int64_t)W * Cc + Cc];
  }
}

// head output (FP32 GEMM result + bias) plus the step-one image channel
__global__ void head_out_kernel(const float* __restrict__ h, const float* __restrict__ in,
                                int64_t P, float* __restrict__ out) {
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x)
    out[p] = h[p] + in[2 * p];
}

// g = 2 (y - t) / P and per-block partial sums of (y - t)^2 in FP64
__global__ void mse_kernel(const float* __restrict__ y, const float* __restrict__ t, int64_t P,
                           float* __restrict__ g, double* __restrict__ parts) {
  __shared__ double red[kT / 32];
  double s = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
       p += (int64_t)gridDim.x * blockDim.x) {
    const float d = y[p] - t[p];
    g[p] = 2.0f * d / (float)P;
    s += (double)d * (double)d;
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < kT / 32; ++w) a += red[w];
    parts[blockIdx.x] = a;
  }
}

// Adam (Kingma and Ba 2015) on the FP32 master weights; the gradient of a
// weight matrix is read from its [Co][Kp] GEMM result
__global__ void adam_kernel(float* __restrict__ w, const float* __restrict__ gw, int Co, int K9,
                            int Kp, float* __restrict__ m, float* __restrict__ v, float lr,
                            float b1, float b2, float c1, float c2, float eps) {
  const int64_t total = (int64_t)Co * K9;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int co = (int)(e / K9), k = (int)(e - (int64_t)co * K9);
    const float g = gw[(int64_t)co * Kp + k];
    const float mm = b1 * m[e] + (1.0f - b1) * g;
    const float vv = b2 * v[e] + (1.0f - b2) * g * g;
    m[e] = mm;
    v[e] = vv;
    w[e] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
  }
}

// copies the weight gradient [Co][Kp] to a dense [Co][9 Ci] array
__global__ void unpad_kernel(const float* __restrict__ gw, int Co, int K9, int Kp,
                             float* __restrict__ out) {
  const int64_t total = (int64_t)Co * K9;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int co = (int)(e / K9), k = (int)(e - (int64_t)co * K9);
    out[e] = gw[(int64_t)co * Kp + k];
  }
}
}  // namespace
}  // namespace ms

// ====================================================================== host
using namespace ms;

namespace {
struct Layer {
  int ci, co, kp, cop, level;   // input / output channels, padded K and Co, resolution level
  bool relu;
  size_t woff;                  // offset of the weights in the master array (bias after)
  float *gw = nullptr, *gb = nullptr;        // gradients
  float *mw = nullptr, *vw = nullptr, *mb = nullptr, *vb = nullptr;   // Adam state
  bf16 *Wb = nullptr, *Wt = nullptr;         // packed bf16 weights
  const bf16* in = nullptr;                  // forward input (bf16 [P][ci])
  bf16* out = nullptr;                       // forward output (bf16 [P][co]) (not the head)
  bf16* dz_keep = nullptr;                   // kept pre-activation gradient [P][cop]
};

struct Fail {
  ms_status st;
  std::string msg;
};
void ck(cudaError_t e, const char* what) {
  if (e != cudaSuccess)
    throw Fail{e == cudaErrorMemoryAllocation ? MS_ERR_OOM : MS_ERR_CUDA,
               std::string(what) + ": " + cudaGetErrorString(e)};
}
}  // namespace

struct ms_unet {
  int levels = 0, width = 0, max_side = 0, dev = 0;
  std::vector<Layer> L;
  size_t nparams = 0;
  float* master = nullptr;   // FP32 weights and biases, conv after conv
  std::vector<void*> allocs;
  // activations (bf16): x, per encoder level a and skip, pooled, bottom, per
  // decoder level cat, a, b
  bf16* xin = nullptr;
  std::vector<bf16*> enc_a, skip, pooled, dec_cat, dec_a, dec_b;
  bf16 *bot_a = nullptr, *bot_b = nullptr;
  bf16 *cols = nullptr, *colsT = nullptr, *dz = nullptr, *dzT = nullptr;
  float *head = nullptr, *g = nullptr, *dcols = nullptr, *dA = nullptr, *dB = nullptr;
  float* wsplit = nullptr;   // split-K partial products of the weight gradients
  std::vector<float*> dskip;
  double* parts = nullptr;
  int adam_t = 0;
  bool keep = false;         // keep every layer's pre-activation gradient
  int last_h = 0, last_w = 0;   // image size of the last forward pass
  std::string msg;
  template <typename T> T* alloc(size_t n) {
    void* p = nullptr;
    ck(cudaMalloc(&p, sizeof(T) * (n ? n : 1)), "allocation");
    allocs.push_back(p);
    return (T*)p;
  }
  ~ms_unet() {
    for (void* p : allocs) cudaFree(p);
  }
};

int ms_unet_device_of(const ms_unet* net) { return net ? net->dev : -1; }

namespace {
template <typename F> ms_status guard(ms_unet* u, F&& f) {
  if (!u) return MS_ERR_ARG;
  try {
    u->msg.clear();
    f();
    return MS_OK;
  } catch (const Fail& e) {
    u->msg = e.msg;
    return e.st;
  }
}

void arg(bool ok, const char* what) {
  if (!ok) throw Fail{MS_ERR_ARG, what};
}

// one convolution: Y = act(cols(X) . W^T + b); the head writes FP32 to u->head
void conv_forward(ms_unet* u, Layer& l, const bf16* x, int H, int W, cudaStream_t s) {
  const int64_t P = (int64_t)H * W;
  l.in = x;
  im2col_kernel<<<blocks(P * l.kp), kT, 0, s>>>(x, H, W, l.ci, l.kp, u->cols);
  const float* bias = u->master + l.woff + (size_t)l.co * 9 * l.ci;
  if (l.out)
    gemm_tn(u->cols, l.kp, l.Wb, l.kp, l.out, l.co, (int)P, l.co, l.kp, bias, l.relu, true, s);
  else
    gemm_tn(u->cols, l.kp, l.Wb, l.kp, u->head, 1, (int)P, 1, l.kp, bias, false, false, s);
}

// backward of one convolution: g = dL/d(output) (FP32, [P][ldg]); writes the
// weight and bias gradients and, if dx, dL/d(input) (FP32 [P][ci])
void conv_backward(ms_unet* u, Layer& l, const float* g, int ldg, int H, int W, float* dx,
                   cudaStream_t s) {
  const int64_t P = (int64_t)H * W;
  relu_grad_kernel<<<blocks(P * l.cop), kT, 0, s>>>(g, ldg, l.relu ? l.out : nullptr, P, l.co,
                                                    l.cop, u->dz);
  if (u->keep)
    ck(cudaMemcpyAsync(l.dz_keep, u->dz, sizeof(bf16) * P * l.cop, cudaMemcpyDeviceToDevice, s),
       "keep gradient");
  colsum_kernel<<<l.co, kT, 0, s>>>(u->dz, P, l.cop, l.gb);
  transpose_kernel<<<blocks(P * l.cop), kT, 0, s>>>(u->dz, P, l.cop, u->dzT);
  im2col_t_kernel<<<blocks(P * l.kp), kT, 0, s>>>(l.in, H, W, l.ci, l.kp, u->colsT);
  gemm_tn_splitk(u->dzT, (int)P, u->colsT, (int)P, u->wsplit, l.gw, l.co, l.kp, (int)P,
                 splits_for(P), s);
  if (dx) {
    gemm_tn(u->dz, l.cop, l.Wt, l.cop, u->dcols, l.kp, (int)P, l.kp, l.cop, nullptr, false,
            false, s);
    col2im_kernel<<<blocks(P * l.ci), kT, 0, s>>>(u->dcols, H, W, l.ci, l.kp, dx);
  }
}

void pack(ms_unet* u, cudaStream_t s) {
  for (Layer& l : u->L)
    pack_weights_kernel<<<blocks((int64_t)l.kp * l.cop), kT, 0, s>>>(
        u->master + l.woff, l.co, l.ci, l.kp, l.cop, l.Wb, l.Wt);
}

void forward(ms_unet* u, const float* in, int H, int W, cudaStream_t s) {
  arg(H >= 4 && W >= 4 && H <= u->max_side && W <= u->max_side, "image side out of range");
  arg(H % (4 << (u->levels - 1)) == 0 && W % (4 << (u->levels - 1)) == 0,
      "image sides must be divisible by 4 * 2^(levels-1)");
  pack(u, s);
  u->last_h = H;
  u->last_w = W;
  const int Lv = u->levels;
  to_bf16_kernel<<<blocks((int64_t)H * W * 2), kT, 0, s>>>(in, (int64_t)H * W * 2, u->xin);
  size_t li = 0;
  const bf16* x = u->xin;
  int h = H, w = W;
  for (int lv = 0; lv < Lv; ++lv) {
    Layer& l0 = u->L[li++];
    conv_forward(u, l0, x, h, w, s);
    Layer& l1 = u->L[li++];
    conv_forward(u, l1, l0.out, h, w, s);
    if (lv < Lv - 1) {
      avgpool_kernel<<<blocks((int64_t)h * w * l1.co / 4), kT, 0, s>>>(l1.out, h, w, l1.co,
                                                                        u->pooled[lv]);
      x = u->pooled[lv];
      h /= 2;
      w /= 2;
    }
  }
  const bf16* lo = u->L[li - 1].out;
  int clo = u->L[li - 1].co;
  for (int lv = Lv - 2; lv >= 0; --lv) {
    h *= 2;
    w *= 2;
    const int cs = u->width << lv;
    upcat_kernel<<<blocks((int64_t)h * w * (clo + cs)), kT, 0, s>>>(lo, clo, u->skip[lv], cs, h,
                                                                     w, u->dec_cat[lv]);
    Layer& l0 = u->L[li++];
    conv_forward(u, l0, u->dec_cat[lv], h, w, s);
    Layer& l1 = u->L[li++];
    conv_forward(u, l1, l0.out, h, w, s);
    lo = l1.out;
    clo = l1.co;
  }
  conv_forward(u, u->L[li], lo, h, w, s);
}

// gradients of the mean squared error of the output against target
double backward(ms_unet* u, const float* in, const float* target, int H, int W, float* out,
                cudaStream_t s) {
  const int64_t P = (int64_t)H * W;
  head_out_kernel<<<blocks(P), kT, 0, s>>>(u->head, in, P, out);
  const int nb = blocks(P, 1024);
  mse_kernel<<<nb, kT, 0, s>>>(out, target, P, u->g, u->parts);
  const int Lv = u->levels;
  int li = (int)u->L.size() - 1;
  // head
  conv_backward(u, u->L[li--], u->g, 1, H, W, u->dA, s);
  float* ga = u->dA;   // gradient of the current activation
  float* gb = u->dB;
  int h = H, w = W;
  for (int lv = 0; lv <= Lv - 2; ++lv) {   // decoder, finest level first
    Layer& l1 = u->L[li--];
    conv_backward(u, l1, ga, l1.co, h, w, gb, s);
    Layer& l0 = u->L[li--];
    conv_backward(u, l0, gb, l0.co, h, w, ga, s);   // ga = d(cat)
    const int cs = u->width << lv, clo = l0.ci - cs;
    upcat_grad_kernel<<<blocks(P), kT, 0, s>>>(ga, clo, cs, h, w, gb, u->dskip[lv]);
    std::swap(ga, gb);   // ga = d(lower level output)
    h /= 2;
    w /= 2;
  }
  for (int lv = Lv - 1; lv >= 0; --lv) {   // bottom and encoder; h, w: level lv
    if (lv < Lv - 1) {
      // ga = d(pooled output of level lv) at half resolution: through the
      // pooling, added to the skip gradient the decoder left in dskip[lv]
      const int c = u->width << lv;
      avgpool_grad_kernel<<<blocks((int64_t)h * w * c), kT, 0, s>>>(ga, h, w, c, u->dskip[lv]);
      ga = u->dskip[lv];
    }
    float* t1 = (ga == u->dA) ? u->dB : u->dA;
    float* t0 = (t1 == u->dA) ? u->dB : u->dA;
    Layer& l1 = u->L[li--];
    conv_backward(u, l1, ga, l1.co, h, w, t1, s);
    Layer& l0 = u->L[li--];
    conv_backward(u, l0, t1, l0.co, h, w, lv > 0 ? t0 : nullptr, s);
    ga = t0;
    h *= 2;
    w *= 2;
  }
  std::vector<double> hp(nb);
  ck(cudaMemcpyAsync(hp.data(), u->parts, sizeof(double) * nb, cudaMemcpyDeviceToHost, s),
     "loss");
  ck(cudaStreamSynchronize(s), "synchronize");
  double sum = 0.0;
  for (double v : hp) sum += v;
  return sum / (double)P;
}
}  // namespace

extern "C" {

ms_status ms_unet_create(int32_t levels, int32_t width, int32_t max_side, uint64_t seed,
                         int32_t device, ms_unet** out) {
  if (!out || levels < 2 || levels > 6 || width < 1 || width > 256 || max_side < 8 ||
      max_side > 8192)
    return MS_ERR_ARG;
  *out = nullptr;
  ms_unet* u = new ms_unet();
  ms_status st = guard(u, [&] {
    u->levels = levels;
    u->width = width;
    u->max_side = max_side;
    u->dev = device;
    ck(cudaSetDevice(device), "set device");
    // layers in execution order: encoder + bottom, decoder, head
    auto add = [&](int co, int ci, int level, bool relu) {
      Layer l{};
      l.ci = ci;
      l.co = co;
      l.kp = pad16(9 * ci);
      l.cop = pad16(co);
      l.level = level;
      l.relu = relu;
      l.woff = u->nparams;
      u->nparams += (size_t)co * 9 * ci + co;
      u->L.push_back(l);
    };
    int cin = 2;
    for (int lv = 0; lv < levels; ++lv) {
      const int c = width << lv;
      add(c, cin, lv, true);
      add(c, c, lv, true);
      cin = c;
    }
    for (int lv = levels - 2; lv >= 0; --lv) {
      const int c = width << lv;
      add(c, (width << (lv + 1)) + c, lv, true);
      add(c, c, lv, true);
    }
    add(1, width, 0, false);
    u->master = u->alloc<float>(u->nparams);
    // He-normal initialization on the host (Box-Muller on a 64-bit LCG)
    std::vector<float> h(u->nparams, 0.0f);
    uint64_t st64 = seed * 6364136223846793005ULL + 1442695040888963407ULL;
    auto uni = [&]() {
      st64 = st64 * 6364136223846793005ULL + 1442695040888963407ULL;
      return ((st64 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    for (Layer& l : u->L) {
      // the head starts at zero: the untrained network returns its first
      // input channel (the step-one image) unchanged, and training learns a
      // correction to it
      if (!l.relu) continue;
      const double sd = std::sqrt(2.0 / (9.0 * l.ci));
      for (size_t i = 0; i < (size_t)l.co * 9 * l.ci; ++i) {
        const double r = std::sqrt(-2.0 * std::log(uni())), t = 6.283185307179586 * uni();
        h[l.woff + i] = (float)(sd * r * std::cos(t));
      }
    }
    ck(cudaMemcpy(u->master, h.data(), sizeof(float) * u->nparams, cudaMemcpyHostToDevice),
       "init");
    const int64_t P0 = (int64_t)max_side * max_side;
    int kmax = 0, cmax = 16;
    size_t wsplit_n = 1;
    for (Layer& l : u->L) {
      l.gw = u->alloc<float>((size_t)l.co * l.kp);
      l.gb = u->alloc<float>(l.co);
      const size_t nw = (size_t)l.co * 9 * l.ci;
      l.mw = u->alloc<float>(nw);
      l.vw = u->alloc<float>(nw);
      l.mb = u->alloc<float>(l.co);
      l.vb = u->alloc<float>(l.co);
      ck(cudaMemset(l.mw, 0, sizeof(float) * nw), "memset");
      ck(cudaMemset(l.vw, 0, sizeof(float) * nw), "memset");
      ck(cudaMemset(l.mb, 0, sizeof(float) * l.co), "memset");
      ck(cudaMemset(l.vb, 0, sizeof(float) * l.co), "memset");
      l.Wb = u->alloc<bf16>((size_t)l.co * l.kp);
      l.Wt = u->alloc<bf16>((size_t)l.kp * l.cop);
      const int64_t Pl = P0 >> (2 * l.level);
      if (l.relu) l.out = u->alloc<bf16>((size_t)Pl * l.co);
      kmax = std::max(kmax, l.kp);
      cmax = std::max(cmax, std::max(l.cop, l.ci));
      wsplit_n = std::max(wsplit_n, (size_t)splits_for(Pl) * l.co * l.kp);
    }
    u->wsplit = u->alloc<float>(wsplit_n);
    u->xin = u->alloc<bf16>((size_t)P0 * 2);
    for (int lv = 0; lv < levels - 1; ++lv) {
      const int64_t Pl = P0 >> (2 * lv);
      const int c = width << lv;
      u->skip.push_back(u->L[2 * lv + 1].out);
      u->pooled.push_back(u->alloc<bf16>((size_t)(Pl / 4) * c));
      u->dec_cat.push_back(u->alloc<bf16>((size_t)Pl * (c + (width << (lv + 1)))));
      u->dskip.push_back(u->alloc<float>((size_t)Pl * c));
    }
    u->cols = u->alloc<bf16>((size_t)P0 * kmax);
    u->colsT = u->alloc<bf16>((size_t)P0 * kmax);
    u->dz = u->alloc<bf16>((size_t)P0 * cmax);
    u->dzT = u->alloc<bf16>((size_t)P0 * cmax);
    u->dcols = u->alloc<float>((size_t)P0 * kmax);
    u->dA = u->alloc<float>((size_t)P0 * cmax);
    u->dB = u->alloc<float>((size_t)P0 * cmax);
    u->head = u->alloc<float>((size_t)P0);
    u->g = u->alloc<float>((size_t)P0);
    u->parts = u->alloc<double>(1024);
    ck(cudaDeviceSynchronize(), "create");
  });
  if (st != MS_OK) {
    delete u;
    return st;
  }
  *out = u;
  return MS_OK;
}

ms_status ms_unet_destroy(ms_unet* u) {
  if (!u) return MS_ERR_ARG;
  cudaSetDevice(u->dev);
  delete u;
  return MS_OK;
}

const char* ms_unet_last_error(const ms_unet* u) { return u ? u->msg.c_str() : "no network"; }

ms_status ms_unet_param_count(const ms_unet* u, int64_t* n) {
  if (!u || !n) return MS_ERR_ARG;
  *n = (int64_t)u->nparams;
  return MS_OK;
}

ms_status ms_unet_get_params(ms_unet* u, float* host, int64_t n) {
  return guard(u, [&] {
    arg(host && n == (int64_t)u->nparams, "host buffer of param_count floats required");
    ck(cudaSetDevice(u->dev), "set device");
    ck(cudaMemcpy(host, u->master, sizeof(float) * n, cudaMemcpyDeviceToHost), "copy");
  });
}

ms_status ms_unet_set_params(ms_unet* u, const float* host, int64_t n) {
  return guard(u, [&] {
    arg(host && n == (int64_t)u->nparams, "host buffer of param_count floats required");
    ck(cudaSetDevice(u->dev), "set device");
    ck(cudaMemcpy(u->master, host, sizeof(float) * n, cudaMemcpyHostToDevice), "copy");
    u->adam_t = 0;
    for (Layer& l : u->L) {
      const size_t nw = (size_t)l.co * 9 * l.ci;
      ck(cudaMemset(l.mw, 0, sizeof(float) * nw), "memset");
      ck(cudaMemset(l.vw, 0, sizeof(float) * nw), "memset");
      ck(cudaMemset(l.mb, 0, sizeof(float) * l.co), "memset");
      ck(cudaMemset(l.vb, 0, sizeof(float) * l.co), "memset");
    }
  });
}

ms_status ms_unet_forward(ms_unet* u, const float* in, int32_t H, int32_t W, float* out,
                          void* stream) {
  return guard(u, [&] {
    arg(in && out, "in and out are required");
    ck(cudaSetDevice(u->dev), "set device");
    cudaStream_t s = (cudaStream_t)stream;
    forward(u, in, H, W, s);
    head_out_kernel<<<blocks((int64_t)H * W), kT, 0, s>>>(u->head, in, (int64_t)H * W, out);
    ck(cudaGetLastError(), "kernel launch");
  });
}

ms_status ms_unet_gradients(ms_unet* u, const float* in, const float* target, int32_t H,
                            int32_t W, float* out, float* grads_host, double* loss,
                            void* stream) {
  return guard(u, [&] {
    arg(in && target && out, "in, target and out are required");
    ck(cudaSetDevice(u->dev), "set device");
    cudaStream_t s = (cudaStream_t)stream;
    forward(u, in, H, W, s);
    const double l = backward(u, in, target, H, W, out, s);
    if (loss) *loss = l;
    if (grads_host) {
      float* tmp = nullptr;
      ck(cudaMalloc(&tmp, sizeof(float) * u->nparams), "allocation");
      for (Layer& lay : u->L) {
        const int K9 = 9 * lay.ci;
        unpad_kernel<<<blocks((int64_t)lay.co * K9), kT, 0, s>>>(lay.gw, lay.co, K9, lay.kp,
                                                                 tmp + lay.woff);
        cudaMemcpyAsync(tmp + lay.woff + (size_t)lay.co * K9, lay.gb, sizeof(float) * lay.co,
                        cudaMemcpyDeviceToDevice, s);
      }
      cudaError_t e = cudaMemcpyAsync(grads_host, tmp, sizeof(float) * u->nparams,
                                      cudaMemcpyDeviceToHost, s);
      cudaStreamSynchronize(s);
      cudaFree(tmp);
      ck(e, "copy gradients");
    }
    ck(cudaGetLastError(), "kernel launch");
  });
}

ms_status ms_unet_keep_intermediates(ms_unet* u, int32_t keep) {
  return guard(u, [&] {
    ck(cudaSetDevice(u->dev), "set device");
    if (keep && !u->keep) {
      const int64_t P0 = (int64_t)u->max_side * u->max_side;
      for (Layer& l : u->L)
        if (!l.dz_keep) l.dz_keep = u->alloc<bf16>((size_t)(P0 >> (2 * l.level)) * l.cop);
    }
    u->keep = keep != 0;
  });
}

ms_status ms_unet_layer_tensor(ms_unet* u, int32_t layer, int32_t which, float* host, int64_t n) {
  return guard(u, [&] {
    arg(layer >= 0 && layer < (int)u->L.size(), "layer out of range");
    arg(which >= 0 && which <= 2, "which must be 0 (input), 1 (output) or 2 (gradient)");
    arg(u->last_h > 0, "no forward pass yet");
    const Layer& l = u->L[layer];
    const int64_t P = (int64_t)(u->last_h >> l.level) * (u->last_w >> l.level);
    const int c = which == 0 ? l.ci : l.co;
    arg(host && n == P * c, "host buffer of H_l W_l channels floats required");
    const bf16* src = which == 0 ? l.in : (which == 1 ? l.out : l.dz_keep);
    arg(src != nullptr, which == 1 ? "the head keeps no bfloat16 output"
                                   : "no kept gradient: enable ms_unet_keep_intermediates "
                                     "before ms_unet_gradients");
    const int ld = which == 2 ? l.cop : c;   // row length of the stored array
    ck(cudaSetDevice(u->dev), "set device");
    std::vector<bf16> h((size_t)P * ld);
    ck(cudaMemcpy(h.data(), src, sizeof(bf16) * h.size(), cudaMemcpyDeviceToHost), "copy");
    for (int64_t p = 0; p < P; ++p)
      for (int k = 0; k < c; ++k) host[p * c + k] = __bfloat162float(h[(size_t)p * ld + k]);
  });
}

ms_status ms_unet_train_step(ms_unet* u, const float* in, const float* target, int32_t H,
                             int32_t W, float lr, double* loss, void* stream) {
  return guard(u, [&] {
    arg(in && target, "in and target are required");
    ck(cudaSetDevice(u->dev), "set device");
    cudaStream_t s = (cudaStream_t)stream;
    forward(u, in, H, W, s);
    const double l = backward(u, in, target, H, W, u->g, s);
    if (loss) *loss = l;
    u->adam_t += 1;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)u->adam_t);
    const float c2 = 1.0f - std::pow(b2, (float)u->adam_t);
    for (Layer& lay : u->L) {
      const int K9 = 9 * lay.ci;
      adam_kernel<<<blocks((int64_t)lay.co * K9), kT, 0, s>>>(
          u->master + lay.woff, lay.gw, lay.co, K9, lay.kp, lay.mw, lay.vw, lr, b1, b2, c1, c2,
          1e-8f);
      adam_kernel<<<1, kT, 0, s>>>(u->master + lay.woff + (size_t)lay.co * K9, lay.gb, 1,
                                   lay.co, lay.co, lay.mb, lay.vb, lr, b1, b2, c1, c2, 1e-8f);
    }
    ck(cudaGetLastError(), "kernel launch");
  });
}

}  // extern "C"
