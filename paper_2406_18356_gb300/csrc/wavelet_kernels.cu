// Dictionary kernels: W = [Psi_1 .. Psi_M], Psi_m the periodized orthonormal
// 2-D Daubechies db_m transform with J levels (Sect. 4.3, App. A.1; the
// closed-form Lipschitz constant of Sect. 3.4 assumes orthogonal bases with
// circular boundaries).
//
// One analysis level on an n x n block X is Y = T X T^T, T the periodized
// analysis matrix:
//   a_i = sum_k h_k x[(2i + k) mod n],  d_i = sum_k g_k x[(2i + k) mod n],
//   g_k = (-1)^k h_{L-1-k}.
// Mallat layout: [0,h)^2 approximation, rows [0,h) x cols [h,n) low-y/high-x,
// rows [h,n) x cols [0,h) high-y/low-x, [h,n)^2 high/high, h = n/2.
// Synthesis is the transpose X = T^T Y T.
//
// Both directions are register-blocked: a thread slides over 8 outputs of one
// row or column with its inputs held in registers, and each basis is a
// separate template instance so the filter taps are compile-time constant-bank
// operands.  Global traffic goes through shared memory in whole rows: input
// windows arrive by TMA (level-1 analysis) or cp.async (the next basis's
// subband windows are prefetched while the current one is filtered), and
// results leave as 16-byte vector stores.
//
// The analysis kernel of the minor cycle also does FISTA's step (Algorithm 1):
// its level-1 input is the gradient image 2 (K W alpha_k - b) of the
// extrapolated point, and at each coefficient it forms
// alpha = B_k + t (B_k - B_{k-1}) and writes
// B_{k+1} = soft(alpha - g/theta, lambda/theta), so gradient coefficients
// never reach global memory.

#include <algorithm>
#include <type_traits>

#include "common.cuh"

namespace ms {

__constant__ double c_hd[kMaxBases][kMaxTaps];
__constant__ double c_gd[kMaxBases][kMaxTaps];
__constant__ float c_hf[kMaxBases][kMaxTaps];
__constant__ float c_gf[kMaxBases][kMaxTaps];
// FP32 coefficient pairs for the packed filters: (h_k, g_k) of the analysis
// tap k, (h_2m, h_2m+1) and (g_2m, g_2m+1) of the synthesis output pair
__constant__ float2 c_hg2[kMaxBases][kMaxTaps];
__constant__ float2 c_hh2[kMaxBases][kMaxTaps / 2];
__constant__ float2 c_gg2[kMaxBases][kMaxTaps / 2];

void set_wavelet_filters(const double* h, const int* len, int nbases) {
  double hd[kMaxBases][kMaxTaps] = {}, gd[kMaxBases][kMaxTaps] = {};
  float hf[kMaxBases][kMaxTaps] = {}, gf[kMaxBases][kMaxTaps] = {};
  for (int m = 0; m < nbases; ++m) {
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
  float2 hg[kMaxBases][kMaxTaps] = {}, hh[kMaxBases][kMaxTaps / 2] = {},
         gg[kMaxBases][kMaxTaps / 2] = {};
  for (int m = 0; m < kMaxBases; ++m)
    for (int k = 0; k < kMaxTaps; ++k) {
      hg[m][k] = make_float2(hf[m][k], gf[m][k]);
      if (k % 2 == 0) {
        hh[m][k / 2] = make_float2(hf[m][k], hf[m][k + 1]);
        gg[m][k / 2] = make_float2(gf[m][k], gf[m][k + 1]);
      }
    }
  cudaMemcpyToSymbol(c_hg2, hg, sizeof(hg));
  cudaMemcpyToSymbol(c_hh2, hh, sizeof(hh));
  cudaMemcpyToSymbol(c_gg2, gg, sizeof(gg));
}

namespace {
template <typename R> __device__ __forceinline__ R fh(int m, int k);
template <typename R> __device__ __forceinline__ R fg(int m, int k);
template <> __device__ __forceinline__ float fh<float>(int m, int k) { return c_hf[m][k]; }
template <> __device__ __forceinline__ float fg<float>(int m, int k) { return c_gf[m][k]; }
template <> __device__ __forceinline__ double fh<double>(int m, int k) { return c_hd[m][k]; }
template <> __device__ __forceinline__ double fg<double>(int m, int k) { return c_gd[m][k]; }

// Filter pairs on the FP32 pipe's packed form (fma.rn.f32x2: two lanes of
// FP32 fused multiply-add per instruction, each lane rounded as fmaf): the
// two outputs of a filter step that share their input (analysis: the low and
// high band of tap k; synthesis: outputs 2m and 2m + 1), in the same order of
// operations as the scalar chains, so results are bit-identical.  The
// coefficient pairs come from constant memory as one 64-bit operand.
// Measured at 1024^2 (FP32, M = 8, J = 4), per FISTA iteration: synthesis
// levels 4..2 29.8 -> 26.8 us, level 1 36.0 -> 33.3 us, analysis levels 2..4
// 35.5 -> 33.6 us, level 1 37.1 -> 35.1 us (144.9 -> 136.0 us in all).
#ifndef MS_PACKED_F32
#define MS_PACKED_F32 1
#endif
// (d.x, d.y) = (c.x x + acc.x, c.y x + acc.y), c a coefficient pair read from
// constant memory as one 64-bit operand
__device__ __forceinline__ float2 ffma2_cx(const float2& c, float x, float2 acc) {
  float2 d;
  const unsigned long long cc = *reinterpret_cast<const unsigned long long*>(&c);
  asm("{\n\t.reg .b64 rx, ra, rd;\n\t"
      "mov.b64 rx, {%3, %3};\n\tmov.b64 ra, {%4, %5};\n\t"
      "fma.rn.f32x2 rd, %2, rx, ra;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "l"(cc), "f"(x), "f"(acc.x), "f"(acc.y));
  return d;
}
// analysis tap k of basis MB on input x: (a, d) += (h_k, g_k) x
template <typename R, int MB, bool PACK>
__device__ __forceinline__ void tap_hg(int k, R x, R& a, R& d) {
  if constexpr (sizeof(R) == 4 && MS_PACKED_F32 && PACK) {
    const float2 r = ffma2_cx(c_hg2[MB][k], x, make_float2(a, d));
    a = r.x;
    d = r.y;
  } else {
    a = fma(fh<R>(MB, k), x, a);
    d = fma(fg<R>(MB, k), x, d);
  }
}
// synthesis taps 2m, 2m + 1 of basis MB on low input x and high input y:
// (e, o) += (h_2m, h_2m+1) x, then (e, o) += (g_2m, g_2m+1) y
template <typename R, int MB>
__device__ __forceinline__ void tap_syn(int m, R x, R y, R& e, R& o) {
  if constexpr (sizeof(R) == 4 && MS_PACKED_F32) {
    float2 r = ffma2_cx(c_hh2[MB][m], x, make_float2(e, o));
    r = ffma2_cx(c_gg2[MB][m], y, r);
    e = r.x;
    o = r.y;
  } else {
    e = fma(fh<R>(MB, 2 * m), x, e);
    e = fma(fg<R>(MB, 2 * m), y, e);
    o = fma(fh<R>(MB, 2 * m + 1), x, o);
    o = fma(fg<R>(MB, 2 * m + 1), y, o);
  }
}
#ifndef MS_PACKED_ANALYSIS
#define MS_PACKED_ANALYSIS 1
#endif

constexpr int kP = 8;   // outputs per thread and direction

__host__ __device__ constexpr int round4(int x) { return (x + 3) / 4 * 4; }

// Analysis geometry for subband tiles of side AT (per block and basis): the
// staged input window, the column-filtered rows ylo / yhi and the four output
// subbands, which alias the window.  Region sizes are multiples of 4 elements
// so every region starts 16-byte aligned.  Every geometry keeps 256 threads:
// the small levels run in one wave, and there the per-block critical path
// (not occupancy) sets the time, so more threads per tile is better.
template <int AT> struct AG {
  static constexpr int T = AT;
  static constexpr int In = 2 * AT + kMaxTaps - 2;   // window side: 78, 46, 30
  static constexpr int InS = round4(In + 2);         // window row stride: 80, 48, 32
  static constexpr int YS = In + 1;                  // odd row stride of ylo / yhi
  static constexpr int GS = AT + 4;                  // 16-byte row stride of the outputs
  static constexpr int InSz = round4(In * InS);
  static constexpr int YSz = round4(AT * YS);
#ifndef MS_ANA_SMALL_THREADS
  static constexpr int Threads = 256;
#else
  static constexpr int Threads = AT >= 32 ? 256 : MS_ANA_SMALL_THREADS;
#endif
  static_assert(4 * AT * GS <= InSz, "the outputs alias the input window");
  static_assert(2 * AT * (AT / kP) <= Threads, "one thread per row unit");
};
// Synthesis geometry for output tiles of side ST: four staged subband windows
// per basis (double-buffered over the bases) and the column-filtered rows.
template <int ST> struct SG {
  static constexpr int T = ST;
  static constexpr int In = ST / 2 + kMaxTaps / 2 - 1;   // window side: 39, 23, 15
  static constexpr int SubS = round4(In + 1);            // staged row stride: 40, 24, 16
  static constexpr int ZS = In + 2;                      // odd row stride of zlo / zhi
  static constexpr int SubSz = 4 * In * SubS;            // one staged basis
#ifndef MS_SYN_SMALL_THREADS
  static constexpr int Threads = 256;
#else
  static constexpr int Threads = ST >= 64 ? 256 : MS_SYN_SMALL_THREADS;
#endif
  static constexpr int Q = (ST * (ST / kP) + Threads - 1) / Threads;   // row units per thread
};
// Staging table of a synthesis block that sums all M bases (level 1): the
// 16-byte chunks a thread copies, and their source offsets from the basis's
// plane (or LL buffer), are the same for every basis, so an interior tile
// computes them once.  K slots per thread.
template <typename R, class G> struct SynTab {
  static constexpr int V = 16 / (int)sizeof(R);
  static constexpr int K = (4 * G::In * ((G::In + 1 + V - 1) / V) + G::Threads - 1) / G::Threads;
};
// the widest tiles (level 1 at N >= 512); the TMA box of the level-1 window
constexpr int kAT = 32;
constexpr int kST = 64;

// Tile sides (compile-time tunables; the defaults are the measured best on
// GB300): large levels use wide tiles (less halo), small levels narrow ones
// with small blocks so that they still fill the SMs.
#ifndef MS_SYN_T1
#define MS_SYN_T1 64   // synthesis output tile for n >= 512 (<= kST)
#endif
#ifndef MS_SYN_T2
#define MS_SYN_T2 32   // synthesis output tile for 256 <= n < 512
#endif
#ifndef MS_SYN_T3
#define MS_SYN_T3 16   // synthesis output tile for 16 <= n < 256
#endif
#ifndef MS_ANA_L1_TILE
#define MS_ANA_L1_TILE 1   // level-1 analysis: one block per tile over all bases
#endif
#ifndef MS_ANA_T1
#define MS_ANA_T1 32   // analysis subband tile for h >= 256 (<= kAT)
#endif
#ifndef MS_ANA_T2
#define MS_ANA_T2 16   // analysis subband tile for 128 <= h < 256
#endif
static_assert(MS_SYN_T1 <= kST && MS_SYN_T2 <= kST && MS_SYN_T3 <= kST, "synthesis tile");
static_assert(MS_ANA_T1 <= kAT && MS_ANA_T2 <= kAT, "analysis tile");
// The largest power of two <= the preferred side that divides the level's
// side (sides need not be powers of two: N = 48 gives 48, 24, 12, 6).
__host__ __device__ __forceinline__ int fit_tile(int t, int n) {
  int p = 1;
  while (2 * p <= t && n % (2 * p) == 0) p *= 2;
  return p;
}
#ifndef MS_SYN_T1B
#define MS_SYN_T1B MS_SYN_T1   // synthesis output tile for 512 <= n < 1024
#endif
// wide: the batched minor cycles, whose launches have blocks to spare (the
// jobs multiply them), take the widest tiles at every level: the per-tile
// staging and set-up dominate the narrow tiles of the coarse levels.
__host__ __device__ __forceinline__ int syn_tile(int n, bool wide = false) {   // output side
  if (wide) return fit_tile(kST, n);
  return fit_tile(n >= 1024 ? MS_SYN_T1 : (n >= 512 ? MS_SYN_T1B : (n >= 256 ? MS_SYN_T2 : MS_SYN_T3)),
                  n);
}
__host__ __device__ __forceinline__ int ana_tile(int h, bool wide = false) {   // subband side
  if (wide) return fit_tile(kAT, h);
  return fit_tile(h >= 256 ? MS_ANA_T1 : (h >= 128 ? MS_ANA_T2 : 16), h);
}
// geometry (template argument) serving a tile side
__host__ __device__ __forceinline__ int syn_geom(int TS) { return TS >= 64 ? 64 : (TS >= 32 ? 32 : 16); }
__host__ __device__ __forceinline__ int ana_geom(int TO) { return TO >= 32 ? 32 : (TO >= 16 ? 16 : 8); }

__device__ __forceinline__ int wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}
// periodic index for i in [-n, 2n)
__device__ __forceinline__ int wrapc(int i, int n) {
  return i < 0 ? i + n : (i >= n ? i - n : i);
}

// u / d (integer quotient) for 0 <= u < 2^22, d >= 1, through the FP32
// reciprocal inv = 1 / d: (u + 0.5) / d lies at least 0.5 / d from an
// integer, and the two roundings move it by at most (u / d) 2^-23 < 0.5 / d,
// so truncation gives the quotient (a few instructions instead of an integer
// division)
__device__ __forceinline__ int div_small(int u, float inv) {
  return (int)(((float)u + 0.5f) * inv);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(bar)),
               "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                   (unsigned)__cvta_generic_to_shared(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned phase) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(bar);
  for (int it = 0; it < (1 << 22); ++it) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(a), "r"(phase)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y),
      "r"((unsigned)__cvta_generic_to_shared(bar))
      : "memory");
}

// first 128-byte-aligned shared address at or after p
__device__ __forceinline__ unsigned char* smem_align128(unsigned char* p) {
  const unsigned pad = (128u - (saddr(p) & 127u)) & 127u;
  return p + pad;
}

// Tile sides up to MS_COMPACT_T use the compact filters (below).
#ifndef MS_COMPACT_T
#define MS_COMPACT_T 16   // tile sides up to this use the compact filters
#endif
template <int T> constexpr bool kCompact = T <= MS_COMPACT_T;

// 8 decimated outputs from 2*8 + L - 2 inputs held in registers
template <typename R, int MB>
__device__ __forceinline__ void fir_down8(const R* x, R* lo, R* hi) {
  constexpr int L = 2 * (MB + 1);
#pragma unroll
  for (int j = 0; j < kP; ++j) {
    R a = 0, d = 0;
#pragma unroll
    for (int k = 0; k < L; ++k) tap_hg<R, MB, MS_PACKED_ANALYSIS>(k, x[2 * j + k], a, d);
    lo[j] = a;
    hi[j] = d;
  }
}

// 8 upsampled outputs r = 0..7 from L/2 + 3 low and high inputs:
// out[r] = sum_{k = r mod 2, step 2} h_k lo[(r - k)/2 + L/2 - 1] + g_k hi[...]
template <typename R, int MB>
__device__ __forceinline__ void fir_up8(const R* lo, const R* hi, R* out) {
  constexpr int L = 2 * (MB + 1);
  // one fused multiply-add per tap and band (a chain, no separate product
  // and sum); outputs 2m and 2m + 1 read the same inputs (with the even and
  // the odd taps), so they run as one pair
#pragma unroll
  for (int r = 0; r < kP; r += 2) {
    R e = 0, o = 0;
#pragma unroll
    for (int m = 0; m < L / 2; ++m) {
      const int i = r / 2 - m + L / 2 - 1;
      tap_syn<R, MB>(m, lo[i], hi[i], e, o);
    }
    out[r] = e;
    out[r + 1] = o;
  }
}

// per-thread compensated sum of |x| in the working precision (Kahan), so the
// FP64 unit only sees one value per thread
template <typename R> struct KSum {
  R s = 0, c = 0;
  __device__ __forceinline__ void add(R v) {
    R y = v - c;
    R t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <typename R> struct Vec;
template <> struct Vec<float> { using T = float4; static constexpr int N = 4; };
template <> struct Vec<double> { using T = double2; static constexpr int N = 2; };
}  // namespace

// ------------------------------------------------------------------ synthesis
// Level j: subbands of side h = N >> j -> output side n = 2h.  Level J reads
// its approximation from the coefficient planes, lower levels from the LL
// buffer written by the level above.  Level 1 sums the M bases into x, with
// the next basis's windows prefetched by cp.async while the current one is
// filtered.  G = SG<ST> is the geometry serving the level's tile side.

// Stages the four subband windows of one basis: rows from r0/2 - 7, columns
// from c0/2 - 8 (one column before the filter's first, so that in the image's
// interior each window row starts on a 16-byte boundary and is copied in
// whole 16-byte chunks); rows always, columns near the edges, wrap
// periodically.  Window element (a, b) of subband s is at sub[s][a][b] with
// b = column - (c0/2 - 8).
template <typename R, class G>
__device__ __forceinline__ void synth_stage(const R* plane, const R* llp, int N, int h, int r0,
                                            int c0, int cnt, R* sub) {
  const int base_r = r0 / 2 - (kMaxTaps / 2 - 1), base_c = c0 / 2 - kMaxTaps / 2;
  const int ncol = cnt + 1;
  constexpr int V = 16 / (int)sizeof(R);
  const int nch = (ncol + V - 1) / V;
  // rows lie in [-7, h), columns in [-8, h): one conditional wrap when h >= 8
  const bool cheap = h >= kMaxTaps / 2;
  if (base_c >= 0 && base_c + nch * V <= h) {
    const int per_sub = cnt * nch;
    for (int e = threadIdx.x; e < 4 * per_sub; e += G::Threads) {
      const int sb = e / per_sub, rem = e - sb * per_sub;
      const int a = rem / nch, c = rem - a * nch;
      const int iy = cheap ? wrapc(base_r + a, h) : wrap(base_r + a, h);
      const int ix = base_c + c * V;
      const R* src;
      if (sb == 0)
        src = llp ? llp + (int64_t)iy * h + ix : plane + (int64_t)iy * N + ix;
      else if (sb == 1)
        src = plane + (int64_t)iy * N + h + ix;
      else if (sb == 2)
        src = plane + (int64_t)(h + iy) * N + ix;
      else
        src = plane + (int64_t)(h + iy) * N + h + ix;
      cp_async<16>(sub + (sb * G::In + a) * G::SubS + c * V, src);
    }
    return;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int NW = G::Threads / 32;
  for (int a = warp; a < cnt; a += NW) {
    const int iy = cheap ? wrapc(base_r + a, h) : wrap(base_r + a, h);
    for (int b = lane; b < ncol; b += 32) {
      const int ix = cheap ? wrapc(base_c + b, h) : wrap(base_c + b, h);
      R* d = sub + a * G::SubS + b;
      cp_async<sizeof(R)>(d, llp ? llp + (int64_t)iy * h + ix : plane + (int64_t)iy * N + ix);
      cp_async<sizeof(R)>(d + G::In * G::SubS, plane + (int64_t)iy * N + h + ix);
      cp_async<sizeof(R)>(d + 2 * G::In * G::SubS, plane + (int64_t)(h + iy) * N + ix);
      cp_async<sizeof(R)>(d + 3 * G::In * G::SubS, plane + (int64_t)(h + iy) * N + h + ix);
    }
  }
}

// The compact synthesis filter (see analysis_filter_compact): output pairs
// (2 rr, 2 rr + 1) of a unit both read inputs rr - kk + L/2 - 1, kk < L/2,
// with the even and the odd taps; same summation order as fir_up8.  Used
// for the levels that write an LL buffer (not the basis sum of level 1).
template <typename R, int MB, class G>
__device__ __forceinline__ void synth_basis_compact(int TS, int lts, int cnt, int r0, int c0,
                                                    const R* sub, R* zlo, R* zhi, R* ll_out,
                                                    int n) {
  constexpr int L = 2 * (MB + 1);
  const int tid = threadIdx.x;
  const int nseg = TS / kP > 0 ? TS / kP : 1;
  const int units_a = cnt * 2 * nseg;
  const float inv_cnt = 1.0f / (float)cnt;
  for (int u = tid; u < units_a; u += G::Threads) {
    int rest = div_small(u, inv_cnt);
    int b = u - rest * cnt;
    int pair = rest & 1, seg = rest >> 1;
    const R* s0 = sub + (pair ? 1 : 0) * G::In * G::SubS + 1 + b;
    const R* s1 = sub + (pair ? 3 : 2) * G::In * G::SubS + 1 + b;
    const int first = 4 * seg + 8 - L / 2;
    R* z = (pair ? zhi : zlo) + (kP * seg) * G::ZS + b;
#pragma unroll 1
    for (int rr = 0; rr < kP / 2; ++rr) {
      R e = 0, o = 0;
#pragma unroll
      for (int kk = 0; kk < L / 2; ++kk) {
        const int i = first + rr - kk + L / 2 - 1;
        const R x = s0[i * G::SubS], y = s1[i * G::SubS];
        tap_syn<R, MB>(kk, x, y, e, o);
      }
      z[(2 * rr) * G::ZS] = e;
      z[(2 * rr + 1) * G::ZS] = o;
    }
  }
  __syncthreads();
  for (int q = 0; q < G::Q; ++q) {
    int u = tid + q * G::Threads;
    int r = u & (TS - 1), seg = u >> lts;
    if (seg >= nseg) continue;
    const int first = 4 * seg + 8 - L / 2;
    const R* lr = zlo + r * G::ZS + first;
    const R* hr = zhi + r * G::ZS + first;
    R* dst = ll_out + (int64_t)(r0 + r) * n + c0 + kP * seg;
#pragma unroll 1
    for (int rr = 0; rr < kP / 2; ++rr) {
      R e = 0, o = 0;
#pragma unroll
      for (int kk = 0; kk < L / 2; ++kk) {
        const int i = rr - kk + L / 2 - 1;
        tap_syn<R, MB>(kk, lr[i], hr[i], e, o);
      }
      if (kP * seg + 2 * rr < TS) dst[2 * rr] = e;
      if (kP * seg + 2 * rr + 1 < TS) dst[2 * rr + 1] = o;
    }
  }
}

template <typename R, int MB, class G>
__device__ __forceinline__ void synth_basis(int TS, int lts, int cnt, int r0, int c0,
                                            const R* sub, R* zlo, R* zhi, R (&acc)[G::Q][kP],
                                            bool sum_bases, R* ll_out, int n) {
  constexpr int L = 2 * (MB + 1);
  constexpr int NI = L / 2 + 3;
  const int tid = threadIdx.x;
  if constexpr (kCompact<G::T>) {
    if (!sum_bases) {
      synth_basis_compact<R, MB, G>(TS, lts, cnt, r0, c0, sub, zlo, zhi, ll_out, n);
      return;
    }
  }
  // columns (y): units (b, pair, seg); pair 0 -> zlo from (approximation,
  // high-y/low-x), pair 1 -> zhi from (low-y/high-x, high/high)
  const int nseg = TS / kP > 0 ? TS / kP : 1;
  const int units_a = cnt * 2 * nseg;
  const float inv_cnt = 1.0f / (float)cnt;
  for (int u = tid; u < units_a; u += G::Threads) {
    int rest = div_small(u, inv_cnt);
    int b = u - rest * cnt;
    int pair = rest & 1, seg = rest >> 1;
    // window column b + 1 is filter column b (the window starts one early)
    const R* s0 = sub + (pair ? 1 : 0) * G::In * G::SubS + 1;
    const R* s1 = sub + (pair ? 3 : 2) * G::In * G::SubS + 1;
    const int first = 4 * seg + 8 - L / 2;
    R lo[NI], hi[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      lo[i] = s0[(first + i) * G::SubS + b];
      hi[i] = s1[(first + i) * G::SubS + b];
    }
    R out[kP];
    fir_up8<R, MB>(lo, hi, out);
    R* z = pair ? zhi : zlo;
#pragma unroll
    for (int r = 0; r < kP; ++r) z[(kP * seg + r) * G::ZS + b] = out[r];
  }
  __syncthreads();
  // rows (x): units (r, seg), a warp takes consecutive rows of one segment
#pragma unroll
  for (int q = 0; q < G::Q; ++q) {
    int u = tid + q * G::Threads;
    int r = u & (TS - 1), seg = u >> lts;
    if (seg >= nseg) continue;
    const int first = 4 * seg + 8 - L / 2;
    R lo[NI], hi[NI];
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      lo[i] = zlo[r * G::ZS + first + i];
      hi[i] = zhi[r * G::ZS + first + i];
    }
    R out[kP];
    fir_up8<R, MB>(lo, hi, out);
    if (sum_bases) {
#pragma unroll
      for (int cc = 0; cc < kP; ++cc) acc[q][cc] += out[cc];
    } else {
      R* dst = ll_out + (int64_t)(r0 + r) * n + c0 + kP * seg;
#pragma unroll
      for (int cc = 0; cc < kP; ++cc)
        if (kP * seg + cc < TS) dst[cc] = out[cc];
    }
  }
}

// One synthesis work item: output tile `tile` of level j for basis mb
// (level 1: all bases summed into x).  Ends with a block barrier, so the
// caller may reuse the shared buffers.
template <typename R, class G>
__device__ __forceinline__ void synth_item(unsigned char* smem_raw, const R* __restrict__ coef,
                                           const R* __restrict__ ll_in, R* __restrict__ ll_out,
                                           R* __restrict__ x, int N, int j, int J, int M,
                                           int tile, int mb, bool wide = false) {
  R* subs = reinterpret_cast<R*>(smem_raw);          // [2][4][G::In][G::SubS]
  R* zlo = subs + 2 * G::SubSz;                       // [G::T][G::ZS]
  R* zhi = zlo + G::T * G::ZS;
  int2* tab = reinterpret_cast<int2*>(zhi + G::T * G::ZS);   // [K][G::Threads]
  const int h = N >> j, n = 2 * h;
  const int TS = syn_tile(n, wide);
  const int lts = 31 - __clz(TS);
  const int cnt = TS / 2 + kMaxTaps / 2 - 1;
  const int tiles_x = n / TS;
  const int r0 = (tile / tiles_x) * TS, c0 = (tile % tiles_x) * TS;
  const bool sum_bases = (j == 1);
  const int m_lo = sum_bases ? 0 : mb, m_hi = sum_bases ? M : mb + 1;
  R acc[G::Q][kP];
#pragma unroll
  for (int q = 0; q < G::Q; ++q)
#pragma unroll
    for (int cc = 0; cc < kP; ++cc) acc[q][cc] = (R)0;
  // interior tiles of a level summing several bases stage through the table:
  // entry = {source offset, shared offset | 1 << 30 for the LL buffer}, or
  // y = -1 for an unused slot; each thread reads back only its own entries
  using Tab = SynTab<R, G>;
  constexpr int V = Tab::V;
  const int nch = (cnt + 1 + V - 1) / V;
  const int base_r = r0 / 2 - (kMaxTaps / 2 - 1), base_c = c0 / 2 - kMaxTaps / 2;
  const bool table = sum_bases && m_hi - m_lo > 1 && base_c >= 0 && base_c + nch * V <= h;
  if (table) {
    const int per_sub = cnt * nch;
    const bool cheap = h >= kMaxTaps / 2;
    const bool from_ll = j != J;
#pragma unroll
    for (int k = 0; k < Tab::K; ++k) {
      const int e = threadIdx.x + k * G::Threads;
      int2 t = make_int2(0, -1);
      if (e < 4 * per_sub) {
        const int sb = e / per_sub, rem = e - sb * per_sub;
        const int a = rem / nch, c = rem - a * nch;
        const int iy = cheap ? wrapc(base_r + a, h) : wrap(base_r + a, h);
        const int ix = base_c + c * V;
        int off;
        if (sb == 0)
          off = from_ll ? iy * h + ix : iy * N + ix;
        else if (sb == 1)
          off = iy * N + h + ix;
        else if (sb == 2)
          off = (h + iy) * N + ix;
        else
          off = (h + iy) * N + h + ix;
        t.x = off;
        t.y = ((sb * G::In + a) * G::SubS + c * V) | ((sb == 0 && from_ll) ? 1 << 30 : 0);
      }
      tab[k * G::Threads + threadIdx.x] = t;
    }
  }
  auto stage = [&](int m) {
    const R* plane = coef + (int64_t)m * N * N;
    const R* llp = (j == J) ? nullptr : ll_in + (int64_t)m * h * h;
    R* dst = subs + (m & 1) * G::SubSz;
    if (table) {
#pragma unroll
      for (int k = 0; k < Tab::K; ++k) {
        const int2 t = tab[k * G::Threads + threadIdx.x];
        if (t.y >= 0) cp_async<16>(dst + (t.y & ((1 << 30) - 1)), ((t.y >> 30) ? llp : plane) + t.x);
      }
    } else {
      synth_stage<R, G>(plane, llp, N, h, r0, c0, cnt, dst);
    }
    cp_async_commit();
  };
  stage(m_lo);
  for (int m = m_lo; m < m_hi; ++m) {
    if (m + 1 < m_hi) {
      stage(m + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const R* sub = subs + (m & 1) * G::SubSz;
    R* llo = sum_bases ? nullptr : ll_out + (int64_t)m * n * n;
    switch (m) {
#define MS_SYN(MBV)                                                                       \
  case MBV:                                                                               \
    synth_basis<R, MBV, G>(TS, lts, cnt, r0, c0, sub, zlo, zhi, acc, sum_bases, llo, n);  \
    break;
      MS_SYN(0) MS_SYN(1) MS_SYN(2) MS_SYN(3) MS_SYN(4) MS_SYN(5) MS_SYN(6) MS_SYN(7)
#undef MS_SYN
    }
    __syncthreads();
  }
  if (sum_bases) {
    const int nseg = TS / kP > 0 ? TS / kP : 1;
#pragma unroll
    for (int q = 0; q < G::Q; ++q) {
      int u = threadIdx.x + q * G::Threads;
      int r = u & (TS - 1), seg = u >> lts;
      if (seg >= nseg) continue;
      R* dst = x + (int64_t)(r0 + r) * N + c0 + kP * seg;
      if (TS % kP == 0) {
        using V = typename Vec<R>::T;
        constexpr int NV = Vec<R>::N;
#pragma unroll
        for (int cc = 0; cc < kP; cc += NV) {
          V v;
          R* vp = reinterpret_cast<R*>(&v);
#pragma unroll
          for (int e = 0; e < NV; ++e) vp[e] = acc[q][cc + e];
          *reinterpret_cast<V*>(dst + cc) = v;
        }
      } else {
#pragma unroll
        for (int cc = 0; cc < kP; ++cc)
          if (kP * seg + cc < TS) dst[cc] = acc[q][cc];
      }
    }
  }
}

// one level per launch (dictionary synthesis of the API and the power
// iteration): blockIdx.x = tile, blockIdx.y = basis
template <typename R, int ST>
__global__ void __launch_bounds__(SG<ST>::Threads, 512 / SG<ST>::Threads)
    synthesis_kernel(const R* const* __restrict__ coef3, const R* __restrict__ ll_in,
                     R* __restrict__ ll_out, R* __restrict__ x, int N, int j, int J, int M,
                     const FistaCtl* __restrict__ ctl) {
  if (ctl && ctl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const R* coef = coef3[ctl ? (ctl->k % 3) : 0];
  synth_item<R, SG<ST>>(smem_raw, coef, ll_in, ll_out, x, N, j, J, M, blockIdx.x, blockIdx.y);
}

// Level j of the minor cycle's synthesis x = W B_k: blockIdx.x = output
// tile, blockIdx.y = basis (level 1: one block per tile sums all bases).  The
// buffers come by value and B_k is picked by k % 3, so no pointer table is
// read before the first load.
template <typename R, int ST>
__global__ void __launch_bounds__(SG<ST>::Threads, 512 / SG<ST>::Threads)
    synthesis_level_kernel(FistaPass<R> a_, int j) {
  const FistaPass<R> a = job_slice(a_);   // blockIdx.z: the job (batched form)
  pdl_wait();
  pdl_trigger();
  const int done = a.ctl->done;
  const int k = a.ctl->k;
  if (done) return;   // uniform: `done` does not change during this kernel
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const R* coef = k % 3 == 0 ? a.B0 : (k % 3 == 1 ? a.B1 : a.B2);
  const int64_t half = (int64_t)a.M * (a.N / 2) * (a.N / 2);
  const R* ll_in = (j == a.J) ? nullptr : a.tmp + ((j + 1) & 1) * half;
  R* ll_out = a.tmp + (j & 1) * half;
  synth_item<R, SG<ST>>(smem_raw, coef, ll_in, ll_out, a.x, a.N, j, a.J, a.M, blockIdx.x,
                        blockIdx.y, a.js.jobs > 1);
}

namespace {
// staged windows, column-filtered rows and the staging table
template <int ST> size_t synthesis_smem_bytes(size_t rsz) {
  const size_t tab = rsz == 4 ? SynTab<float, SG<ST>>::K : SynTab<double, SG<ST>>::K;
  return (size_t)(2 * SG<ST>::SubSz + 2 * SG<ST>::T * SG<ST>::ZS) * rsz +
         tab * SG<ST>::Threads * sizeof(int2);
}
// the four output subbands alias the input window; + alignment slack,
// block-sum scratch, mbarrier and flags
template <int AT> size_t analysis_smem_bytes(size_t rsz) {
  return (size_t)(AG<AT>::InSz + 2 * AG<AT>::YSz) * rsz + 128 +
         (AG<AT>::Threads / 32) * sizeof(double) + sizeof(uint64_t) + 2 * sizeof(int);
}
}  // namespace

template <typename R>
void launch_synthesis3(const R* const* coef3_dev, R* x, R* tmp, WaveletGeom g,
                       const FistaCtl* ctl, cudaStream_t s, int only_level) {
  const int64_t half = (int64_t)g.M * (g.N / 2) * (g.N / 2);
  for (int j = g.J; j >= 1; --j) {
    if (only_level > 0 && j != only_level) continue;
    int h = g.N >> j, n = 2 * h;
    int TS = syn_tile(n);
    int tiles = (n / TS) * (n / TS);
    const R* ll_in = (j == g.J) ? nullptr : tmp + ((j + 1) & 1) * half;
    R* ll_out = tmp + (j & 1) * half;
    dim3 grid(tiles, j == 1 ? 1 : g.M);
    auto go = [&](auto kern, int threads, size_t smem) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kern<<<grid, threads, smem, s>>>(coef3_dev, ll_in, ll_out, x, g.N, j, g.J, g.M, ctl);
    };
    switch (syn_geom(TS)) {
      case 64: go(synthesis_kernel<R, 64>, SG<64>::Threads, synthesis_smem_bytes<64>(sizeof(R))); break;
      case 32: go(synthesis_kernel<R, 32>, SG<32>::Threads, synthesis_smem_bytes<32>(sizeof(R))); break;
      default: go(synthesis_kernel<R, 16>, SG<16>::Threads, synthesis_smem_bytes<16>(sizeof(R))); break;
    }
  }
}

// ------------------------------------------------------------------ analysis
// Small tiles (the coarse levels) run the same filters with the output loop
// rolled and the inputs read from shared memory per tap: a few times more
// shared-memory loads, a fraction of the code.  A coarse level's blocks each
// execute one basis's filter once, so its time is set by the instruction
// fetch of that code, not by the loads.  The sums are formed in the same
// order as the register-blocked versions, so results are identical.

template <typename R, int MB, class G>
__device__ __forceinline__ void analysis_filter_compact(const R* sIn, R* ylo, R* yhi, R* gout,
                                                        int TOe, int lt) {
  constexpr int L = 2 * (MB + 1);
  const int tid = threadIdx.x;
  const int nparts = TOe >> 3;
  const int cols = 2 * TOe + L - 2;
  const float inv_cols = 1.0f / (float)cols;
  for (int u = tid; u < nparts * cols; u += G::Threads) {
    const int part = div_small(u, inv_cols);
    const int col = u - part * cols;
    const R* xc = sIn + (2 * kP * part) * G::InS + col;
#pragma unroll 1
    for (int r = 0; r < kP; ++r) {
      R a = 0, d = 0;
#pragma unroll
      for (int k = 0; k < L; ++k) {
        tap_hg<R, MB, MS_PACKED_ANALYSIS>(k, xc[(2 * r + k) * G::InS], a, d);
      }
      ylo[(kP * part + r) * G::YS + col] = a;
      yhi[(kP * part + r) * G::YS + col] = d;
    }
  }
  __syncthreads();
  const int lp = lt - 3;
  const int r = tid & (TOe - 1), seg = (tid >> lt) & (nparts - 1), src = tid >> (lt + lp);
  __syncthreads();   // (the barrier pair of the register-blocked version)
  if (src >= 2) return;
  const R* yrow = (src ? yhi : ylo) + r * G::YS + 2 * kP * seg;
  R* o_lo = gout + (src ? 2 : 0) * G::T * G::GS + r * G::GS + kP * seg;
  R* o_hi = gout + (src ? 3 : 1) * G::T * G::GS + r * G::GS + kP * seg;
#pragma unroll 1
  for (int q = 0; q < kP; ++q) {
    R a = 0, d = 0;
#pragma unroll
    for (int k = 0; k < L; ++k) {
      tap_hg<R, MB, MS_PACKED_ANALYSIS>(k, yrow[2 * q + k], a, d);
    }
    o_lo[q] = a;
    o_hi[q] = d;
  }
}

// Filtering of one basis on the staged input tile: columns (y) into
// ylo / yhi, then rows (x) into the four subbands gout[0..3] =
// (approximation, low-y/high-x, high-y/low-x, high/high), G::T x G::GS each.
// TOe (a power of two, 8..G::T) outputs per subband side, lt = log2(TOe).
// (ROWS_IN_REGS: the register-blocked version whatever the tile side, for
// callers whose outputs alias the column-filtered rows)
template <typename R, int MB, class G, bool ROWS_IN_REGS = false>
__device__ __forceinline__ void analysis_filter(const R* sIn, R* ylo, R* yhi, R* gout, int TOe,
                                                int lt) {
  constexpr int L = 2 * (MB + 1);
  constexpr int NI = 2 * kP + L - 2;
  const int tid = threadIdx.x;
  const int nparts = TOe >> 3;
  const int cols = 2 * TOe + L - 2;
  if constexpr (kCompact<G::T> && !ROWS_IN_REGS) {
    analysis_filter_compact<R, MB, G>(sIn, ylo, yhi, gout, TOe, lt);
  } else {
    const float inv_cols = 1.0f / (float)cols;
    for (int u = tid; u < nparts * cols; u += G::Threads) {
      int part = div_small(u, inv_cols);
      int col = u - part * cols;
      R xin[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) xin[i] = sIn[(2 * kP * part + i) * G::InS + col];
      R lo[kP], hi[kP];
      fir_down8<R, MB>(xin, lo, hi);
#pragma unroll
      for (int r = 0; r < kP; ++r) {
        ylo[(kP * part + r) * G::YS + col] = lo[r];
        yhi[(kP * part + r) * G::YS + col] = hi[r];
      }
    }
    __syncthreads();
    // rows: unit = (row r, segment, source); a warp takes consecutive rows of
    // one segment
    const int lp = lt - 3;   // log2(nparts)
    const int r = tid & (TOe - 1), seg = (tid >> lt) & (nparts - 1), src = tid >> (lt + lp);
    const bool active = src < 2;
    R xin[NI];
    if (active) {
      const R* yrow = (src ? yhi : ylo) + r * G::YS + 2 * kP * seg;
#pragma unroll
      for (int i = 0; i < NI; ++i) xin[i] = yrow[i];
    }
    __syncthreads();   // the outputs overwrite the input tile
    if (!active) return;
    R lo[kP], hi[kP];
    fir_down8<R, MB>(xin, lo, hi);
    R* o_lo = gout + (src ? 2 : 0) * G::T * G::GS + r * G::GS + kP * seg;
    R* o_hi = gout + (src ? 3 : 1) * G::T * G::GS + r * G::GS + kP * seg;
    using V = typename Vec<R>::T;
    constexpr int NV = Vec<R>::N;
#pragma unroll
    for (int q = 0; q < kP; q += NV) {
      *reinterpret_cast<V*>(o_lo + q) = *reinterpret_cast<const V*>(lo + q);
      *reinterpret_cast<V*>(o_hi + q) = *reinterpret_cast<const V*>(hi + q);
    }
  }
}

// shared-memory layout of an analysis block (after the 128-byte alignment)
template <typename R, class G> struct AnaSmem {
  R* sIn;        // [G::In][G::InS]; later the outputs [4][G::T][G::GS]
  R* ylo;        // [G::T][G::YS]
  R* yhi;
  double* red;   // [G::Threads / 32]
  uint64_t* bar;
  int* flags;    // [2]
  __device__ __forceinline__ explicit AnaSmem(unsigned char* base) {
    sIn = reinterpret_cast<R*>(base);
    ylo = sIn + G::InSz;
    yhi = ylo + G::YSz;
    red = reinterpret_cast<double*>(yhi + G::YSz);
    bar = reinterpret_cast<uint64_t*>(red + G::Threads / 32);
    flags = reinterpret_cast<int*>(bar + 1);
  }
};

// One analysis work item: subband tile `tile` (of side TO <= G::T) of level
// j for basis MB.  n = N >> (j-1) is the input side, h = n/2 the subband side.
// MODE 0: plain analysis (W^H x); input x (level 1) or LL_{j-1}.
// MODE 1: FISTA step; level 1 input is the gradient image 2 (K W alpha_k - b);
//         detail (and level-J approximation) outputs go through the prox into
//         B_{k+1} and |B_{k+1}| accumulates into l1.
// With the widest geometry, level 1 stages its 78 x 78 input window by one
// TMA tensor copy when the window lies inside the image (the caller has
// initialized the mbarrier and tracks its phase); other windows are staged by
// cp.async with periodic wrap.  Ends with a block barrier, so the caller may
// reuse the shared buffers.
template <typename R, int MODE, int MB, class G>
__device__ __forceinline__ void analysis_item(unsigned char* base, const CUtensorMap* xmap,
                                              bool use_tma, unsigned& phase, const R* x_in,
                                              const R* ll_in, R* ll_out, R* out_plain,
                                              const R* cur, const R* prev, R* next, R t, R mu,
                                              R thr, int N, int j, int J, int tile,
                                              FistaCtl* ctl, KSum<R>& l1, int tma_y0 = 0,
                                              bool wide = false) {
  constexpr int m = MB;
  const AnaSmem<R, G> sm(base);
  R* sIn = sm.sIn;
  R* gout = sIn;

  const int n = N >> (j - 1), h = n / 2;
  const int TO = ana_tile(h, wide);
  const int TOe = TO < kP ? kP : TO;             // outputs computed per side
  const int lt = 31 - __clz(TOe);
  const int lto = 31 - __clz(TO);
  const int ext = 2 * TOe + kMaxTaps - 2;        // staged input window side
  const int tiles_x = h / TO;
  const int o0y = (tile / tiles_x) * TO, o0x = (tile % tiles_x) * TO;
  const int p0y = 2 * o0y, p0x = 2 * o0x;
  constexpr int NV = Vec<R>::N;
  constexpr int LNV = NV == 4 ? 2 : 1;
  using V = typename Vec<R>::T;
  const bool vec = (TO % NV) == 0;
  const int64_t plane = (int64_t)m * N * N;
  // coefficient-plane offset of (subband s = 1..3, row, col) of this tile
  auto coef_off = [&](int s, int row, int col) -> int64_t {
    int rr = (s >= 2 ? h : 0) + o0y + row;
    int cc = (s & 1 ? h : 0) + o0x + col;
    return plane + (int64_t)rr * N + cc;
  };

  // The TMA copy is issued only after checking its alignment rules (128-byte
  // shared destination, 64-byte descriptor, 16-byte start column); a
  // violation is recorded in ctl->error (MS_ERR_UNSUPPORTED) and the window
  // is staged by cp.async instead.
  bool tma = G::T == kAT && use_tma && j == 1 && TO == kAT && p0x + G::InS <= n &&
             p0y + G::In <= n;
  if (tma) {
    if (threadIdx.x == 0) {
      const bool aligned = (saddr(sIn) & 127u) == 0 &&
                           (reinterpret_cast<uintptr_t>(xmap) & 63u) == 0 &&
                           ((p0x * (int)sizeof(R)) & 15) == 0;
      sm.flags[1] = aligned ? 1 : 0;
      if (aligned) {
        // order the block's earlier generic accesses of the window before
        // the asynchronous copy overwrites it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(sm.bar, (unsigned)(G::In * G::InS * sizeof(R)));
        tma_load_2d(sIn, xmap, p0x, p0y + tma_y0, sm.bar);
      } else if (ctl) {
        atomicExch(&ctl->error, 8);
      }
    }
    __syncthreads();
    tma = sm.flags[1] != 0;
  }

  if (!tma) {
    // stage the input window with periodic wrap
    const R* src = (j == 1) ? x_in : ll_in + (int64_t)m * n * n;
    const bool cheap = n >= ext;   // positions lie in [0, n + ext)
    constexpr int V16 = 16 / (int)sizeof(R);
    const int nch = (ext + V16 - 1) / V16;
    if (p0x + nch * V16 <= n && (n % V16) == 0) {
      // the window's columns need no wrap: whole 16-byte chunks per row
      // (p0x = 2 o0x is a multiple of 16), rows wrap
      for (int e = threadIdx.x; e < ext * nch; e += G::Threads) {
        const int a = e / nch, c = e - a * nch;
        const int py = cheap ? wrapc(p0y + a, n) : wrap(p0y + a, n);
        cp_async<16>(sIn + a * G::InS + c * V16, src + (int64_t)py * n + p0x + c * V16);
      }
    } else {
      const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
      constexpr int NW = G::Threads / 32;
      for (int a = warp; a < ext; a += NW) {
        const int py = cheap ? wrapc(p0y + a, n) : wrap(p0y + a, n);
        const R* row = src + (int64_t)py * n;
        for (int b = lane; b < ext; b += 32) {
          const int px = cheap ? wrapc(p0x + b, n) : wrap(p0x + b, n);
          cp_async<sizeof(R)>(sIn + a * G::InS + b, row + px);
        }
      }
    }
    cp_async_commit();
  }

  bool skip = false;
  if (tma) {
    // bounded wait for the window; on time-out the tile is skipped (the
    // error is recorded) but every barrier is still passed
    const bool ok = mbar_wait_bounded(sm.bar, phase);
    phase ^= 1u;
    skip = __syncthreads_or(!ok) != 0;
    if (skip && threadIdx.x == 0 && ctl) atomicExch(&ctl->error, 5);
  } else {
    cp_async_wait<0>();
  }
  __syncthreads();
  if (!skip) {
    analysis_filter<R, MB, G>(sIn, sm.ylo, sm.yhi, gout, TOe, lt);
  } else {
    __syncthreads();   // the filter's two barriers
    __syncthreads();
  }
  __syncthreads();

  // write / update the tile's coefficients
  auto prox = [&](R g, R bc, R bp) -> R {
    R alpha = bc + t * (bc - bp);
    R z = alpha - mu * g;
    R az = fabs(z) - thr;
    R nb = az > (R)0 ? copysign(az, z) : (R)0;
    l1.add(fabs(nb));
    return nb;
  };
  if (skip) {
    // nothing is written for a tile whose window never arrived
  } else if (vec) {
    const int lpr = lto - LNV;    // log2(vectors per tile row)
    const int s_first = (j == J) ? 0 : 1;
    const int lsub = lto + lpr;   // log2(vectors per subband tile)
    const int items = (4 - s_first) << lsub;
    for (int e = threadIdx.x; e < items; e += G::Threads) {
      int s = s_first + (e >> lsub);
      int rem = e & ((1 << lsub) - 1);
      int row = rem >> lpr, c4 = (rem & ((1 << lpr) - 1)) << LNV;
      V gv = *reinterpret_cast<const V*>(gout + (s * G::T + row) * G::GS + c4);
      int64_t off = s ? coef_off(s, row, c4) : plane + (int64_t)(o0y + row) * N + o0x + c4;
      if (MODE == 0) {
        *reinterpret_cast<V*>(out_plain + off) = gv;
      } else {
        V cv = *reinterpret_cast<const V*>(cur + off);
        V pv = *reinterpret_cast<const V*>(prev + off);
        V nv;
        R* np = reinterpret_cast<R*>(&nv);
        const R* gp = reinterpret_cast<const R*>(&gv);
        const R* cp = reinterpret_cast<const R*>(&cv);
        const R* pp = reinterpret_cast<const R*>(&pv);
#pragma unroll
        for (int q = 0; q < NV; ++q) np[q] = prox(gp[q], cp[q], pp[q]);
        *reinterpret_cast<V*>(next + off) = nv;
      }
    }
    if (j < J) {   // approximation feeds the next level
      for (int e = threadIdx.x; e < (1 << lsub); e += G::Threads) {
        int row = e >> lpr, c4 = (e & ((1 << lpr) - 1)) << LNV;
        *reinterpret_cast<V*>(ll_out + (int64_t)m * h * h + (int64_t)(o0y + row) * h + o0x + c4) =
            *reinterpret_cast<const V*>(gout + row * G::GS + c4);
      }
    }
  } else {   // tiny levels: scalar path
    const int s_first = (j == J) ? 0 : 1;
    for (int e = threadIdx.x; e < 4 * TO * TO; e += G::Threads) {
      int s = e / (TO * TO);
      int row = (e / TO) % TO, col = e % TO;
      R gval = gout[(s * G::T + row) * G::GS + col];
      if (s == 0 && j < J) {
        ll_out[(int64_t)m * h * h + (int64_t)(o0y + row) * h + o0x + col] = gval;
        continue;
      }
      if (s < s_first) continue;
      int64_t off = s ? coef_off(s, row, col) : plane + (int64_t)(o0y + row) * N + o0x + col;
      if (MODE == 0)
        out_plain[off] = gval;
      else
        next[off] = prox(gval, cur[off], prev[off]);
    }
  }
  __syncthreads();
}

// one level per launch (dictionary analysis of the API and the power
// iteration): blockIdx.x = tile, blockIdx.y = basis
template <typename R, int AT>
__global__ void __launch_bounds__(AG<AT>::Threads, 512 / AG<AT>::Threads)
    analysis_kernel(const R* __restrict__ x_in, const R* __restrict__ ll_in,
                    R* __restrict__ ll_out, R* __restrict__ out_plain, int N, int j, int J) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_align128(smem_raw);
  unsigned phase = 0;
  KSum<R> l1;
  switch (blockIdx.y) {
#define MS_ANA(MBV)                                                                             \
  case MBV:                                                                                     \
    analysis_item<R, 0, MBV, AG<AT>>(base, nullptr, false, phase, x_in, ll_in, ll_out,          \
                                     out_plain, nullptr, nullptr, nullptr, (R)0, (R)0, (R)0, N, \
                                     j, J, blockIdx.x, nullptr, l1);                            \
    break;
    MS_ANA(0) MS_ANA(1) MS_ANA(2) MS_ANA(3) MS_ANA(4) MS_ANA(5) MS_ANA(6) MS_ANA(7)
#undef MS_ANA
  }
}

// Level j of the minor cycle's analysis + FISTA update: blockIdx.x = subband
// tile, blockIdx.y = basis.  The spectral kernel of this pass has already
// advanced ctl->k, so this builds B_{k+1} with k = ctl->k - 1.  Each block
// leaves its sum of |B_{k+1}| over its tile in l1_parts[part_base + block];
// the next spectral kernel adds them up (fixed order).
template <typename R, int AT>
__global__ void __launch_bounds__(AG<AT>::Threads, 512 / AG<AT>::Threads)
    analysis_level_kernel(const __grid_constant__ CUtensorMap xmap, FistaPass<R> a_, int j,
                          int use_tma, int part_base) {
  using G = AG<AT>;
  const FistaPass<R> a = job_slice(a_);   // blockIdx.z: the job (batched form)
  pdl_wait();
  pdl_trigger();
  const int done = a.ctl->done;
  const int kc = a.ctl->k;
  if (done) return;   // uniform: `done` does not change during this kernel
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_align128(smem_raw);
  const AnaSmem<R, G> sm(base);
  const int k = kc - 1;
  const R t = ctl_t<R>(a.ctl, k & 1);   // momentum t_k
  const R mu = ctl_mu<R>(a.ctl);        // 1 / theta
  const R thr = ctl_thr<R>(a.ctl);      // lambda / theta
  const R* cur = k % 3 == 0 ? a.B0 : (k % 3 == 1 ? a.B1 : a.B2);
  const R* prev = k % 3 == 0 ? a.B2 : (k % 3 == 1 ? a.B0 : a.B1);
  R* next = k % 3 == 0 ? a.B1 : (k % 3 == 1 ? a.B2 : a.B0);
  const bool tma = G::T == kAT && use_tma != 0 && j == 1;
  if (tma && threadIdx.x == 0) mbar_init(sm.bar, 1);
  __syncthreads();
  unsigned phase = 0;
  KSum<R> l1;
  const int64_t half = (int64_t)a.M * (a.N / 2) * (a.N / 2);
  const R* ll_in = (j == 1) ? nullptr : a.tmp + ((j - 1) & 1) * half;
  R* ll_out = a.tmp + (j & 1) * half;
  switch (blockIdx.y) {
#define MS_ANA(MBV)                                                                          \
  case MBV:                                                                                  \
    analysis_item<R, 1, MBV, G>(base, &xmap, tma, phase, a.grad, ll_in, ll_out, nullptr, cur, \
                                prev, next, t, mu, thr, a.N, j, a.J, blockIdx.x, a.ctl, l1,   \
                                (int)blockIdx.z * a.N, a.js.jobs > 1);                        \
    break;
    MS_ANA(0) MS_ANA(1) MS_ANA(2) MS_ANA(3) MS_ANA(4) MS_ANA(5) MS_ANA(6) MS_ANA(7)
#undef MS_ANA
  }
  // block sum of |B_{k+1}|: error-free working-precision warp sums, FP64
  // once per warp
  R hi = l1.s, lo = -l1.c;
  warp_sum_comp<R>(hi, lo);
  if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = (double)hi + (double)lo;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int q = 0; q < G::Threads / 32; ++q) sum += sm.red[q];
    a.l1_parts[part_base + (int64_t)blockIdx.y * gridDim.x + blockIdx.x] = sum;
  }
}

// Level 1 of the minor cycle's analysis + FISTA step with one block per
// subband tile looping over the M bases (for the widest geometry, 1 < J):
// the gradient window is staged once (TMA, or cp.async with wrap at the
// image edge) and serves every basis, and the tiles of B_k and B_{k-1} of the
// next basis arrive by cp.async (double-buffered) while the current basis is
// filtered.  The filter's outputs alias its column-filtered rows (both are
// dead / rewritten only after the block barriers that separate them), so
// the window survives.  The block's sum of |B_{k+1}| over all bases goes to
// l1_parts[part_base + tile]; it zeroes the other M - 1 slots of its tile.
template <typename R> struct AnaTile {
  using G = AG<kAT>;
  static constexpr int T = G::T;
  static constexpr int PF = 2 * 2 * 3 * T * T;   // [buffer][B_k, B_k-1][subband 1..3][T][T]
  static constexpr size_t bytes() {
    return (size_t)(G::InSz + 2 * G::YSz + PF) * sizeof(R) + 128 +
           (G::Threads / 32) * sizeof(double) + sizeof(uint64_t) + 2 * sizeof(int);
  }
  static_assert(4 * T * G::GS <= 2 * G::YSz, "the outputs alias the filtered rows");
};

template <typename R>
__global__ void __launch_bounds__(AG<kAT>::Threads, 2)
    analysis_l1_tile_kernel(const __grid_constant__ CUtensorMap xmap, FistaPass<R> a_,
                            int use_tma, int part_base, int split) {
  using A = AnaTile<R>;
  const FistaPass<R> a = job_slice(a_);   // blockIdx.z: the job (batched form)
  // blockIdx.y: the basis group, bases [0, split) or [split, M) (split = M:
  // one group)
  const int m_lo = blockIdx.y == 0 ? 0 : split, m_hi = blockIdx.y == 0 ? split : a.M;
  using G = typename A::G;
  constexpr int T = A::T;
  pdl_wait();
  pdl_trigger();
  const int done = a.ctl->done;
  const int kc = a.ctl->k;
  if (done) return;   // uniform: `done` does not change during this kernel
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = smem_align128(smem_raw);
  R* sIn = reinterpret_cast<R*>(base);   // [G::In][G::InS]
  R* ylo = sIn + G::InSz;                // [T][G::YS]; also the outputs [4][T][G::GS]
  R* yhi = ylo + G::YSz;
  R* gout = ylo;
  R* pf = yhi + G::YSz;                  // [2][2][3][T][T]
  double* red = reinterpret_cast<double*>(pf + A::PF);
  uint64_t* bar = reinterpret_cast<uint64_t*>(red + G::Threads / 32);
  int* flags = reinterpret_cast<int*>(bar + 1);

  const int k = kc - 1;
  const R t = ctl_t<R>(a.ctl, k & 1);   // momentum t_k
  const R mu = ctl_mu<R>(a.ctl);        // 1 / theta
  const R thr = ctl_thr<R>(a.ctl);      // lambda / theta
  const R* cur = k % 3 == 0 ? a.B0 : (k % 3 == 1 ? a.B1 : a.B2);
  const R* prev = k % 3 == 0 ? a.B2 : (k % 3 == 1 ? a.B0 : a.B1);
  R* next = k % 3 == 0 ? a.B1 : (k % 3 == 1 ? a.B2 : a.B0);
  const int N = a.N, n = N, h = N / 2;
  const int tile = blockIdx.x;
  const int tiles_x = h / T;
  const int o0y = (tile / tiles_x) * T, o0x = (tile % tiles_x) * T;
  const int p0y = 2 * o0y, p0x = 2 * o0x;
  constexpr int ext = G::In;   // 2 T + 14
  constexpr int NV = Vec<R>::N;
  constexpr int LNV = NV == 4 ? 2 : 1;
  using V = typename Vec<R>::T;
  const int64_t half = (int64_t)a.M * (N / 2) * (N / 2);
  R* ll_out = a.tmp + half;   // level 1 writes LL buffer (1 & 1)

  // coefficient offset of (subband s = 1..3, row, col) of this tile in basis m
  auto coef_off = [&](int m, int s, int row, int col) -> int64_t {
    return (int64_t)m * N * N + (int64_t)((s >= 2 ? h : 0) + o0y + row) * N + (s & 1 ? h : 0) +
           o0x + col;
  };
  // prefetch of basis m's B_k and B_k-1 tiles into buffer m & 1
  auto prefetch = [&](int m) {
    constexpr int V16 = 16 / (int)sizeof(R);
    constexpr int CPR = T / V16;   // 16-byte chunks per tile row
    R* dst = pf + (m & 1) * (2 * 3 * T * T);
    for (int e = threadIdx.x; e < 2 * 3 * T * CPR; e += G::Threads) {
      const int arr = e / (3 * T * CPR), r = e - arr * (3 * T * CPR);
      const int sb = r / (T * CPR), r2 = r - sb * (T * CPR);
      const int row = r2 / CPR, ch = r2 - row * CPR;
      cp_async<16>(dst + ((arr * 3 + sb) * T + row) * T + ch * V16,
                   (arr ? prev : cur) + coef_off(m, sb + 1, row, ch * V16));
    }
    cp_async_commit();
  };

  // the window: TMA when interior and aligned, else cp.async with wrap
  if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  bool tma = use_tma != 0 && p0x + G::InS <= n && p0y + G::In <= n;
  if (tma) {
    if (threadIdx.x == 0) {
      const bool aligned = (saddr(sIn) & 127u) == 0 &&
                           (reinterpret_cast<uintptr_t>(&xmap) & 63u) == 0 &&
                           ((p0x * (int)sizeof(R)) & 15) == 0;
      flags[1] = aligned ? 1 : 0;
      if (aligned) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, (unsigned)(G::In * G::InS * sizeof(R)));
        tma_load_2d(sIn, &xmap, p0x, p0y + (int)blockIdx.z * N, bar);
      } else {
        atomicExch(&a.ctl->error, 8);
      }
    }
    __syncthreads();
    tma = flags[1] != 0;
  }
  if (!tma) {
    const R* src = a.grad;
    const bool cheap = n >= ext;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int NW = G::Threads / 32;
    for (int r = warp; r < ext; r += NW) {
      const int py = cheap ? wrapc(p0y + r, n) : wrap(p0y + r, n);
      const R* row = src + (int64_t)py * n;
      for (int b = lane; b < ext; b += 32) {
        const int px = cheap ? wrapc(p0x + b, n) : wrap(p0x + b, n);
        cp_async<sizeof(R)>(sIn + r * G::InS + b, row + px);
      }
    }
  }
  cp_async_commit();   // (empty on the TMA path)
  prefetch(m_lo);
  bool skip = false;
  if (tma) {
    unsigned phase = 0;
    const bool ok = mbar_wait_bounded(bar, phase);
    skip = __syncthreads_or(!ok) != 0;
    if (skip && threadIdx.x == 0) atomicExch(&a.ctl->error, 5);
  }
  cp_async_wait<1>();   // the window's copies (the first prefetch may still run)
  __syncthreads();
  if (skip) {
    cp_async_wait<0>();
    return;   // uniform: nothing is written for a tile whose window never arrived
  }

  KSum<R> l1;
  constexpr int lto = 5, lpr = lto - LNV, lsub = lto + lpr;   // T = 32
  static_assert(T == 32, "level-1 tile side");
  constexpr int items = 3 << lsub;
  // the bases in sequence, each a straight-line step (a loop around a
  // switch over the bases raised register pressure into spills)
  auto step = [&](auto mb) {
    constexpr int m = decltype(mb)::value;
    if (m < m_lo || m >= m_hi) return;   // uniform over the block
    if (m + 1 < m_hi) prefetch(m + 1);
    analysis_filter<R, m, G, true>(sIn, ylo, yhi, gout, T, lto);
    if (m + 1 < m_hi) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();   // the filter's outputs and basis m's prefetch are visible
    const R* pc = pf + (m & 1) * (2 * 3 * T * T);
    const R* pp = pc + 3 * T * T;
    for (int e = threadIdx.x; e < items; e += G::Threads) {
      const int sb = e >> lsub;   // subband 1..3 is sb + 1
      const int rem = e & ((1 << lsub) - 1);
      const int row = rem >> lpr, c4 = (rem & ((1 << lpr) - 1)) << LNV;
      const V gv = *reinterpret_cast<const V*>(gout + ((sb + 1) * T + row) * G::GS + c4);
      const V cv = *reinterpret_cast<const V*>(pc + (sb * T + row) * T + c4);
      const V qv = *reinterpret_cast<const V*>(pp + (sb * T + row) * T + c4);
      V nv;
      R* np = reinterpret_cast<R*>(&nv);
      const R* gp = reinterpret_cast<const R*>(&gv);
      const R* cp = reinterpret_cast<const R*>(&cv);
      const R* qp = reinterpret_cast<const R*>(&qv);
#pragma unroll
      for (int q = 0; q < NV; ++q) {
        const R alpha = cp[q] + t * (cp[q] - qp[q]);
        const R z = alpha - mu * gp[q];
        const R az = fabs(z) - thr;
        const R nb = az > (R)0 ? copysign(az, z) : (R)0;
        l1.add(fabs(nb));
        np[q] = nb;
      }
      *reinterpret_cast<V*>(next + coef_off(m, sb + 1, row, c4)) = nv;
    }
    // the approximation feeds level 2
    for (int e = threadIdx.x; e < (1 << lsub); e += G::Threads) {
      const int row = e >> lpr, c4 = (e & ((1 << lpr) - 1)) << LNV;
      *reinterpret_cast<V*>(ll_out + (int64_t)m * h * h + (int64_t)(o0y + row) * h + o0x + c4) =
          *reinterpret_cast<const V*>(gout + row * G::GS + c4);
    }
    __syncthreads();   // gout and prefetch buffer m & 1 are reused
  };
  step(std::integral_constant<int, 0>{});
  step(std::integral_constant<int, 1>{});
  step(std::integral_constant<int, 2>{});
  step(std::integral_constant<int, 3>{});
  step(std::integral_constant<int, 4>{});
  step(std::integral_constant<int, 5>{});
  step(std::integral_constant<int, 6>{});
  step(std::integral_constant<int, 7>{});
  static_assert(kMaxBases == 8, "one step per basis");
  R hi = l1.s, lo = -l1.c;
  warp_sum_comp<R>(hi, lo);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)hi + (double)lo;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int q = 0; q < G::Threads / 32; ++q) sum += red[q];
    // slot (group, tile); the first group also zeroes the slots no group uses
    a.l1_parts[part_base + (int64_t)blockIdx.y * gridDim.x + tile] = sum;
    if (blockIdx.y == 0)
      for (int m = gridDim.y; m < a.M; ++m)
        a.l1_parts[part_base + (int64_t)m * gridDim.x + tile] = 0.0;
  }
}

#include "coarse_levels.cuh"

// CTAs per SM of the one-launch coarse levels and their shared-memory
// budget per CTA (compile-time tunables; the defaults are the measured best)
#ifndef MS_COARSE_CTAS_PER_SM
#define MS_COARSE_CTAS_PER_SM 1
#endif
#ifndef MS_COARSE_BUDGET_KB
#define MS_COARSE_BUDGET_KB 200
#endif
#ifndef MS_COARSE_WOFF
#define MS_COARSE_WOFF 24   // fixed share of a basis's work per row, in taps / 2 (measured best)
#endif

namespace {
template <typename R>
size_t coarse_smem(bool analysis, WaveletGeom g, const CoarseGroups& gr, int budget) {
  int cs_min = 1 << 30;
  for (int m = 0; m < g.M; ++m) cs_min = std::min(cs_min, gr.first[m + 1] - gr.first[m]);
  return strip_smem_bytes(analysis, g.N, g.J, cs_min, sizeof(R), (size_t)budget);
}

// The level-1 analysis tile kernel's basis groups: bases [0, split) and
// [split, M), split where the work (2 (m + 1) taps + MS_L1_WFIX per basis)
// is closest to half; split = M (one group) when MS_L1_GROUPS is 1.
#ifndef MS_L1_GROUPS
#define MS_L1_GROUPS 1   // 2 measured no faster at 1024^2 (37.4 vs 37.2 us)
#endif
#ifndef MS_L1_WFIX
#define MS_L1_WFIX 10
#endif
int l1_basis_split(int M) {
  if (MS_L1_GROUPS < 2 || M < 2) return M;
  double total = 0.0;
  for (int m = 0; m < M; ++m) total += 2.0 * (m + 1) + MS_L1_WFIX;
  double acc = 0.0;
  int best = 1;
  double best_d = 1e30;
  for (int sp = 1; sp < M; ++sp) {
    acc += 2.0 * sp + MS_L1_WFIX;   // work of bases 0..sp-1
    const double d = std::fabs(2.0 * acc - total);
    if (d < best_d) {
      best_d = d;
      best = sp;
    }
  }
  return best;
}

// l1 partial slots of level 1 (the per-tile kernel's share) and in all
int level1_partials(WaveletGeom g) {
  const int h = g.N >> 1, TO = ana_tile(h);
  return (h / TO) * (h / TO) * g.M;
}

template <typename R>
cudaError_t launch_coarse(const FistaPass<R>& a, bool analysis, int part_base, int part_end,
                          cudaStream_t s) {
  const WaveletGeom g{a.N, a.J, a.M};
  const size_t smem = coarse_smem<R>(analysis, g, a.coarse_groups, a.coarse_budget);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(a.coarse_ctas);
  cfg.blockDim = dim3(kStripThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;   // every group resident at once
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (analysis) {
    auto kern = coarse_analysis_kernel<R>;
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return cudaLaunchKernelEx(&cfg, kern, a, a.coarse_groups, a.coarse_bar, part_base, part_end,
                              a.coarse_budget);
  }
  auto kern = coarse_synthesis_kernel<R>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  return cudaLaunchKernelEx(&cfg, kern, a, a.coarse_groups, a.coarse_bar, a.coarse_budget);
}

// CTAs of both strip kernels resident per SM with `budget` bytes of shared
// memory per CTA
template <typename R> int coarse_per_sm(WaveletGeom g, const CoarseGroups& gr, int budget) {
  int per = 1 << 30;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  for (int an = 0; an < 2; ++an) {
    const size_t smem = coarse_smem<R>(an != 0, g, gr, budget);
    if (smem == 0 || smem > (size_t)optin) return 0;   // strips too wide for shared memory
    int blocks = 0;
    cudaError_t e;
    if (an) {
      auto kern = coarse_analysis_kernel<R>;
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, kStripThreads, smem);
    } else {
      auto kern = coarse_synthesis_kernel<R>;
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kern, kStripThreads, smem);
    }
    if (e != cudaSuccess) {
      cudaGetLastError();   // clear: "does not fit" is an answer here, not an error
      return 0;
    }
    per = std::min(per, blocks);
  }
  return per;
}
}  // namespace

int coarse_groups(WaveletGeom g, size_t rsz, CoarseGroups* gr, int* budget) {
#ifdef MS_NO_COARSE_GROUPS
  return 0;
#endif
  const bool pow2 = g.N > 0 && (g.N & (g.N - 1)) == 0;
  if (!pow2 || g.N < 256 || g.J < 2 || (g.N >> g.J) < 8 || g.M < 1) return 0;
  int dev = 0, coop = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop)
    return 0;
  const int span = analysis_prox_partials(g) - level1_partials(g);
  // one CTA per SM; group m gets CTAs in proportion to its work per row:
  // the filters' 2 (m + 1) taps plus a share that does not grow with them
  // (staging, stores, the prox), measured at about 4 taps' worth
  auto weight = [](int m) { return m + 1 + MS_COARSE_WOFF; };
  int total_w = 0;
  for (int m = 0; m < g.M; ++m) total_w += weight(m);
  // one l1 partial per CTA in the coarse share
  const int ctas = std::min(MS_COARSE_CTAS_PER_SM * sm_count(), span);
  if (ctas < g.M) return 0;
  gr->first[0] = 0;
  for (int m = 0; m < g.M; ++m)
    gr->first[m + 1] = gr->first[m] + std::max(1, ctas * weight(m) / total_w);
  for (int m = g.M + 1; m <= kMaxBases; ++m) gr->first[m] = gr->first[g.M];
  const int used = gr->first[g.M];
  if (used > ctas) return 0;
  for (int b : {MS_COARSE_BUDGET_KB * 1024, MS_COARSE_BUDGET_KB * 1024 * 4 / 5}) {
    const int per = rsz == 4 ? coarse_per_sm<float>(g, *gr, b) : coarse_per_sm<double>(g, *gr, b);
    if (per >= 1 && per * sm_count() >= used) {
      *budget = b;
      return used;
    }
  }
  return 0;
}

#ifdef MS_COARSE_PROBE
}  // namespace ms
extern "C" int ms_coarse_probe_read(unsigned long long* host) {
  return (int)cudaMemcpyFromSymbol(host, ms::g_coarse_probe, sizeof(ms::g_coarse_probe));
}
namespace ms {
#endif

int analysis_prox_partials(WaveletGeom g) {
  int total = 0;
  for (int j = 1; j <= g.J; ++j) {
    int h = g.N >> j;
    int TO = ana_tile(h);
    int tiles = (h / TO) * (h / TO);
    total += tiles * g.M;
  }
  return total;
}

template <typename R>
void launch_analysis(const R* x, R* coef, R* tmp, WaveletGeom g, cudaStream_t s) {
  const int64_t half = (int64_t)g.M * (g.N / 2) * (g.N / 2);
  for (int j = 1; j <= g.J; ++j) {
    int h = g.N >> j;
    int TO = ana_tile(h);
    int tiles = (h / TO) * (h / TO);
    const R* ll_in = (j == 1) ? nullptr : tmp + ((j - 1) & 1) * half;
    R* ll_out = tmp + (j & 1) * half;
    dim3 grid(tiles, g.M);
    auto go = [&](auto kern, int threads, size_t smem) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      kern<<<grid, threads, smem, s>>>(x, ll_in, ll_out, coef, g.N, j, g.J);
    };
    switch (ana_geom(TO)) {
      case 32: go(analysis_kernel<R, 32>, AG<32>::Threads, analysis_smem_bytes<32>(sizeof(R))); break;
      case 16: go(analysis_kernel<R, 16>, AG<16>::Threads, analysis_smem_bytes<16>(sizeof(R))); break;
      default: go(analysis_kernel<R, 8>, AG<8>::Threads, analysis_smem_bytes<8>(sizeof(R))); break;
    }
  }
}

// TMA box of the level-1 input window: {80 columns, 78 rows}
void analysis_window_box(unsigned* cols, unsigned* rows) {
  *cols = AG<kAT>::InS;
  *rows = AG<kAT>::In;
}

template <typename R>
cudaError_t launch_synthesis_pass(const FistaPass<R>& a, cudaStream_t s, int only_level) {
  if (only_level < 0 && a.coarse_ctas > 0 && a.js.jobs == 1)   // levels J..2, one cooperative launch
    return launch_coarse<R>(a, false, 0, 0, s);
  for (int j = a.J; j >= 1; --j) {
    if (only_level > 0 && j != only_level) continue;
    if (only_level < 0 && j == 1) continue;
    int n = 2 * (a.N >> j), TS = syn_tile(n, a.js.jobs > 1);
    dim3 grid((n / TS) * (n / TS), j == 1 ? 1 : a.M, a.js.jobs);
    auto go = [&](auto kern, int threads, size_t smem) {
      cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      return launch_pdl(kern, grid, dim3(threads), smem, s, a, j);
    };
    cudaError_t e;
    switch (syn_geom(TS)) {
      case 64: e = go(synthesis_level_kernel<R, 64>, SG<64>::Threads, synthesis_smem_bytes<64>(sizeof(R))); break;
      case 32: e = go(synthesis_level_kernel<R, 32>, SG<32>::Threads, synthesis_smem_bytes<32>(sizeof(R))); break;
      default: e = go(synthesis_level_kernel<R, 16>, SG<16>::Threads, synthesis_smem_bytes<16>(sizeof(R))); break;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename R>
cudaError_t launch_analysis_pass(const FistaPass<R>& a, const CUtensorMap* grad_map,
                                 cudaStream_t s, int only_level) {
  const CUtensorMap m = grad_map ? *grad_map : CUtensorMap{};
  if (only_level < 0 && a.coarse_ctas > 0 && a.js.jobs == 1) {   // levels 2..J, one cooperative launch
    const WaveletGeom g{a.N, a.J, a.M};
    return launch_coarse<R>(a, true, level1_partials(g), analysis_prox_partials(g), s);
  }
  int part_base = 0;
  for (int j = 1; j <= a.J; ++j) {
    const int h = a.N >> j, TO = ana_tile(h, a.js.jobs > 1);
    const int tiles = (h / TO) * (h / TO);
    const bool run = only_level == 0 || j == only_level || (only_level < 0 && j > 1);
    bool done_here = false;
    if constexpr (sizeof(R) == 4) {
      if (run && MS_ANA_L1_TILE && j == 1 && a.J > 1 && TO == kAT && grad_map) {
        const size_t smem = AnaTile<R>::bytes();
        auto kern = analysis_l1_tile_kernel<R>;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        // two block groups over the bases, split where the filter work
        // (taps plus a fixed per-basis share) is about equal
        const int split = l1_basis_split(a.M);
        const cudaError_t e =
            launch_pdl(kern, dim3(tiles, split < a.M ? 2 : 1, a.js.jobs), dim3(AG<kAT>::Threads),
                       smem, s, m, a, 1, part_base, split);
        if (e != cudaSuccess) return e;
        done_here = true;
      }
    }
    if (run && !done_here) {
      dim3 grid(tiles, a.M, a.js.jobs);
      auto go = [&](auto kern, int threads, size_t smem) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return launch_pdl(kern, grid, dim3(threads), smem, s, m, a, j, grad_map ? 1 : 0,
                          part_base);
      };
      cudaError_t e;
      switch (ana_geom(TO)) {
        case 32: e = go(analysis_level_kernel<R, 32>, AG<32>::Threads, analysis_smem_bytes<32>(sizeof(R))); break;
        case 16: e = go(analysis_level_kernel<R, 16>, AG<16>::Threads, analysis_smem_bytes<16>(sizeof(R))); break;
        default: e = go(analysis_level_kernel<R, 8>, AG<8>::Threads, analysis_smem_bytes<8>(sizeof(R))); break;
      }
      if (e != cudaSuccess) return e;
    }
    part_base += tiles * a.M;
  }
  return cudaSuccess;
}

template void launch_synthesis3<float>(const float* const*, float*, float*, WaveletGeom,
                                       const FistaCtl*, cudaStream_t, int);
template void launch_synthesis3<double>(const double* const*, double*, double*, WaveletGeom,
                                        const FistaCtl*, cudaStream_t, int);
template void launch_analysis<float>(const float*, float*, float*, WaveletGeom, cudaStream_t);
template void launch_analysis<double>(const double*, double*, double*, WaveletGeom,
                                      cudaStream_t);
template cudaError_t launch_synthesis_pass<float>(const FistaPass<float>&, cudaStream_t, int);
template cudaError_t launch_synthesis_pass<double>(const FistaPass<double>&, cudaStream_t, int);
template cudaError_t launch_analysis_pass<float>(const FistaPass<float>&, const CUtensorMap*,
                                                 cudaStream_t, int);
template cudaError_t launch_analysis_pass<double>(const FistaPass<double>&, const CUtensorMap*,
                                                  cudaStream_t, int);

}  // namespace ms
