// Coarse wavelet levels (2..J) of the minor cycle in one launch (App. A.1's
// multilevel transform; Algorithm 1's prox on the coarse coefficients).
// Included by wavelet_kernels.cu, whose filters (constant bank), FIR helpers
// and geometry it uses.
//
// Layout.  Every basis gets its own group of CTAs, sized in proportion to
// its work per row (db_m's 2m taps plus a fixed share, so that the groups
// finish together); the
// launch is cooperative, so all groups are resident at once, and the CTAs of
// a group meet at a software barrier between levels (a counter and a
// generation word per basis in global memory, with a bounded wait).  The
// CTAs of a group split each level's rows into contiguous strips (full image
// width, so the row filter wraps inside the strip); a strip's column filter
// needs up to 14 rows past it (analysis) or 7 rows before it (synthesis),
// which come from the neighbours' strips of the level before, read through
// L2 after the barrier.  Approximations between levels live in per-basis
// regions of the approximation ping-pong (basis m at m (N/2)^2 of either
// half), so groups never share a region.
//
// Per level a CTA stages its input rows (own strip and the rows around it,
// wrapped) by cp.async into shared memory, filters the columns (8 outputs
// per thread from registers), then the rows, in chunks of rows sized to the
// shared-memory budget.  The analysis applies FISTA's step to every detail
// coefficient (and the level-J approximation) as it is produced, exactly as
// the per-level kernels do; the synthesis writes the approximation of the
// level below, level 2 the one that level-1 synthesis reads.

constexpr int kStripThreads = 512;
constexpr int kStripHalo = kMaxTaps - 2;     // analysis: input rows past a strip
// Filtered-row strides: odd, so that a warp reading one column of 32 rows
// hits 32 banks.  Analysis rows hold n values plus 14 wrapped ones (n + 15);
// synthesis rows hold h values after 8 wrapped ones (h + 9).
constexpr int kYPad = 15;
constexpr int kZPad = 9;
constexpr int kBarrierSpins = 1 << 22;        // bounded wait of the group barrier

// Group barrier: count[0] counts arrivals, count[1] is the generation.  The
// last CTA to arrive resets the count and advances the generation; the
// others wait (bounded) for the generation to change.  Global writes before
// the barrier are visible to every CTA of the group after it (device-scope
// fences around the counter; the data is read through L2).  A wait that runs
// out records MS_ERR_TIMEOUT in ctl->error and returns; the caller goes on
// (its results are then void) so the kernel always ends.
__device__ __forceinline__ void group_barrier(int* count, int n, FistaCtl* ctl) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile int* gen = count + 1;
    const int g = *gen;
    __threadfence();
    if (atomicAdd(count, 1) == n - 1) {
      atomicExch(count, 0);
      __threadfence();
      atomicAdd(count + 1, 1);
    } else {
      int it = 0;
      while (*gen == g && ++it < kBarrierSpins) __nanosleep(32);
      if (*gen == g) atomicExch(&ctl->error, 5);
    }
    __threadfence();
  }
  __syncthreads();
}

// rows of a strip: CTA `rank` of `cs` owns [begin, end) of `rows` (multiples
// of 8 per CTA, so some CTAs of a small level own none)
__host__ __device__ __forceinline__ void strip_rows(int rows, int cs, int rank, int& begin,
                                                    int& end) {
  const int per = ((rows + cs - 1) / cs + 7) / 8 * 8;
  begin = min(rows, rank * per);
  end = min(rows, begin + per);
}

// Shared memory of a chunk of RC output rows.  Analysis, input side n:
// (2 RC + 14) n staged + 2 RC (n + 15) filtered.  Synthesis, output side n
// (subband side n / 2): 4 (RC / 2 + 8) (n / 2) staged + 2 RC (n / 2 + 9)
// filtered.
__host__ __device__ __forceinline__ size_t strip_chunk_bytes(bool analysis, int n, int rc,
                                                             size_t rsz) {
  return analysis
             ? ((size_t)(2 * rc + kStripHalo) * n + (size_t)2 * rc * (n + kYPad)) * rsz
             : ((size_t)4 * (rc / 2 + 8) * (n / 2) + (size_t)2 * rc * (n / 2 + kZPad)) * rsz;
}
// Output rows per chunk (a multiple of 8) that fit `budget` bytes.
__host__ __device__ __forceinline__ int strip_chunk_rows(bool analysis, int n, size_t rsz,
                                                         size_t budget, int rows_per_cta) {
  int best = 8;
  for (int rc = 8; rc <= rows_per_cta; rc += 8)
    if (strip_chunk_bytes(analysis, n, rc, rsz) <= budget) best = rc;
  return best;
}

// Bytes of shared memory a strip launch needs (the largest level, for the
// smallest group of `cs_min` CTAs), or 0 when even the smallest chunk of 8
// rows of some level exceeds the budget (full-width strips of wide images).
inline size_t strip_smem_bytes(bool analysis, int N, int J, int cs_min, size_t rsz,
                               size_t budget) {
  size_t most = 0;
  for (int j = 2; j <= J; ++j) {
    const int n = N >> (j - 1);                          // analysis input / synthesis output side
    const int rows = analysis ? n / 2 : n;               // output rows of the level
    int b, e;
    strip_rows(rows, cs_min, 0, b, e);
    const int rc = strip_chunk_rows(analysis, n, rsz, budget, e - b);
    const size_t need = strip_chunk_bytes(analysis, n, rc, rsz);
    if (need > budget) return 0;
    most = need > most ? need : most;
  }
  return most + 64 * sizeof(double);
}

// One analysis level of basis MB for the CTA's strip: input LL_{j-1}
// (n x n, row stride n) -> subbands of side h = n / 2; details (and at level
// J the approximation) through the prox into `next`, the approximation of
// j < J into ll_out (h x h).
template <typename R, int MB>
__device__ __forceinline__ void strip_analysis_level(
    const R* __restrict__ in, R* __restrict__ ll_out, int n, bool last, int i0, int i1,
    int rc_max, R* smem, const R* __restrict__ cur, const R* __restrict__ prev,
    R* __restrict__ next, int64_t plane, int N, R t, R mu, R thr, KSum<R>& l1) {
  constexpr int L = 2 * (MB + 1);
  constexpr int NI = 2 * kP + L - 2;
  constexpr int V = 16 / (int)sizeof(R);
  const int h = n / 2;
  const int YS = n + kYPad;        // filtered-row stride (wrap copies at n .. n + 13)
  const int tid = threadIdx.x;
  for (int c0 = i0; c0 < i1; c0 += rc_max) {
    const int rc = min(rc_max, i1 - c0);
    const int groups = (rc + kP - 1) / kP;
    const int rows_in = 2 * groups * kP + kStripHalo;
    R* sin = smem;                                     // [rows_in][n]
    R* ylo = smem + (size_t)(2 * rc_max + kStripHalo) * n;   // [rc_max][YS]
    R* yhi = ylo + (size_t)rc_max * YS;
    // stage input rows 2 c0 .. 2 c0 + rows_in - 1 (wrapped)
    const int vpr = n / V;
    for (int e = tid; e < rows_in * vpr; e += kStripThreads) {
      const int q = e / vpr, c = e - q * vpr;
      const int row = (2 * c0 + q) % n;
      cp_async<16>(sin + (size_t)q * n + c * V, in + (size_t)row * n + c * V);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    // columns: unit = (column x, group of 8 output rows)
    for (int u = tid; u < groups * n; u += kStripThreads) {
      const int g = u / n, x = u - g * n;
      R xin[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) xin[i] = sin[(size_t)(2 * kP * g + i) * n + x];
      R lo[kP], hi[kP];
      fir_down8<R, MB>(xin, lo, hi);
#pragma unroll
      for (int r = 0; r < kP; ++r) {
        ylo[(kP * g + r) * YS + x] = lo[r];
        yhi[(kP * g + r) * YS + x] = hi[r];
        if (x < kStripHalo) {   // wrapped copy for the row filter
          ylo[(kP * g + r) * YS + n + x] = lo[r];
          yhi[(kP * g + r) * YS + n + x] = hi[r];
        }
      }
    }
    __syncthreads();
    // rows: unit = (row r, segment of 8 outputs, source lo / hi), r fastest
    const int segs = h / kP;
    for (int u = tid; u < rc * segs * 2; u += kStripThreads) {
      const int r = u % rc, rest = u / rc;
      const int seg = rest % segs, src = rest / segs;
      const R* yrow = (src ? yhi : ylo) + r * YS + 2 * kP * seg;
      const int gi = c0 + r, u0 = kP * seg;
      // src 0: approximation (a) and low-y/high-x (d); src 1: high-y/low-x
      // (a) and high/high (d).  The prox operands B_k, B_k-1 of d are
      // loaded before the filter runs, so their latency hides behind it.
      const bool a_prox = src == 1 || last;
      const int64_t off_a = src ? plane + (int64_t)(h + gi) * N + u0 : plane + (int64_t)gi * N + u0;
      const int64_t off_d = off_a + h;
      using Vt = typename Vec<R>::T;
      constexpr int NV = Vec<R>::N;
      Vt ca[kP / NV], pa[kP / NV], cd[kP / NV], pd[kP / NV];
#pragma unroll
      for (int q = 0; q < kP / NV; ++q) {
        cd[q] = *reinterpret_cast<const Vt*>(cur + off_d + q * NV);
        pd[q] = *reinterpret_cast<const Vt*>(prev + off_d + q * NV);
      }
      R xin[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) xin[i] = yrow[i];
      R a[kP], d[kP];
      fir_down8<R, MB>(xin, a, d);
      auto prox8 = [&](const R* g8, const Vt* cv, const Vt* pv, int64_t off) {
#pragma unroll
        for (int q = 0; q < kP / NV; ++q) {
          const R* cp = reinterpret_cast<const R*>(&cv[q]);
          const R* pp = reinterpret_cast<const R*>(&pv[q]);
          Vt nv;
          R* np = reinterpret_cast<R*>(&nv);
#pragma unroll
          for (int e = 0; e < NV; ++e) {
            const R alpha = cp[e] + t * (cp[e] - pp[e]);
            const R z = alpha - mu * g8[q * NV + e];
            const R az = fabs(z) - thr;
            const R nb = az > (R)0 ? copysign(az, z) : (R)0;
            l1.add(fabs(nb));
            np[e] = nb;
          }
          *reinterpret_cast<Vt*>(next + off + q * NV) = nv;
        }
      };
      if (a_prox) {
#pragma unroll
        for (int q = 0; q < kP / NV; ++q) {
          ca[q] = *reinterpret_cast<const Vt*>(cur + off_a + q * NV);
          pa[q] = *reinterpret_cast<const Vt*>(prev + off_a + q * NV);
        }
        prox8(a, ca, pa, off_a);
      } else {
#pragma unroll
        for (int q0 = 0; q0 < kP; q0 += NV) {
          Vt v;
          R* vp = reinterpret_cast<R*>(&v);
#pragma unroll
          for (int e = 0; e < NV; ++e) vp[e] = a[q0 + e];
          *reinterpret_cast<Vt*>(ll_out + (size_t)gi * h + u0 + q0) = v;
        }
      }
      prox8(d, cd, pd, off_d);
    }
    __syncthreads();   // the chunk's buffers are reused
  }
}

// One synthesis level of basis MB for the CTA's strip: subbands of side h
// (approximation from `ap` with row stride `aps`, details from the basis's
// plane) -> output rows [t0, t1) of the n x n approximation of the level
// below (row stride n).
template <typename R, int MB>
__device__ __forceinline__ void strip_synthesis_level(const R* __restrict__ ap, int aps,
                                                      const R* __restrict__ plane, int N, int h,
                                                      R* __restrict__ out, int t0, int t1,
                                                      int rc_max, R* smem) {
  constexpr int L = 2 * (MB + 1);
  constexpr int NI = L / 2 + 3;
  constexpr int V = 16 / (int)sizeof(R);
  const int n = 2 * h;
  const int ZS = h + kZPad;        // z rows: column u at u + 8, wrapped copies before
  const int tid = threadIdx.x;
  for (int c0 = t0; c0 < t1; c0 += rc_max) {
    const int rc = min(rc_max, t1 - c0);
    const int groups = (rc + kP - 1) / kP;
    const int rows_in = groups * kP / 2 + 8;
    const int SR = rc_max / 2 + 8;   // staged rows per subband
    R* sub = smem;                   // [4][SR][h]
    R* zlo = smem + (size_t)4 * SR * h;   // [rc_max][ZS]
    R* zhi = zlo + (size_t)rc_max * ZS;
    // stage subband rows c0/2 - 7 .. (wrapped), 4 subbands
    const int vpr = h / V;
    for (int e = tid; e < 4 * rows_in * vpr; e += kStripThreads) {
      const int s = e / (rows_in * vpr), rem = e - s * (rows_in * vpr);
      const int q = rem / vpr, c = rem - q * vpr;
      const int row = (c0 / 2 - (kMaxTaps / 2 - 1) + q + h) % h;
      const R* src;
      if (s == 0)
        src = ap + (size_t)row * aps;
      else if (s == 1)
        src = plane + (size_t)row * N + h;
      else if (s == 2)
        src = plane + (size_t)(h + row) * N;
      else
        src = plane + (size_t)(h + row) * N + h;
      cp_async<16>(sub + ((size_t)s * SR + q) * h + c * V, src + c * V);
    }
    cp_async_commit();
    cp_async_wait<0>();
    __syncthreads();
    // columns: unit = (column x, group of 8 output rows, pair); pair 0 ->
    // zlo from (approximation, high-y/low-x), pair 1 -> zhi from
    // (low-y/high-x, high/high)
    for (int u = tid; u < groups * h * 2; u += kStripThreads) {
      const int x = u % h, rest = u / h;
      const int g = rest % groups, pair = rest / groups;
      const R* s0 = sub + (size_t)(pair ? 1 : 0) * SR * h + x;
      const R* s1 = sub + (size_t)(pair ? 3 : 2) * SR * h + x;
      const int first = 4 * g + 8 - L / 2;   // staged row of lo[0]
      R lo[NI], hi[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        lo[i] = s0[(size_t)(first + i) * h];
        hi[i] = s1[(size_t)(first + i) * h];
      }
      R o[kP];
      fir_up8<R, MB>(lo, hi, o);
      R* z = pair ? zhi : zlo;
#pragma unroll
      for (int r = 0; r < kP; ++r) {
        z[(kP * g + r) * ZS + 8 + x] = o[r];
        if (x >= h - 8) z[(kP * g + r) * ZS + x - (h - 8)] = o[r];   // wrapped copy
      }
    }
    __syncthreads();
    // rows: unit = (row r, segment of 8 outputs), r fastest
    const int segs = n / kP;
    for (int u = tid; u < rc * segs; u += kStripThreads) {
      const int r = u % rc, seg = u / rc;
      const int first = 4 * seg + 8 - L / 2 + 1;   // z column of lo[0]
      R lo[NI], hi[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        lo[i] = zlo[r * ZS + first + i];
        hi[i] = zhi[r * ZS + first + i];
      }
      R o[kP];
      fir_up8<R, MB>(lo, hi, o);
      R* dst = out + (size_t)(c0 + r) * n + kP * seg;
      using Vt = typename Vec<R>::T;
      constexpr int NV = Vec<R>::N;
#pragma unroll
      for (int q = 0; q < kP; q += NV) {
        Vt v;
        R* vp = reinterpret_cast<R*>(&v);
#pragma unroll
        for (int e = 0; e < NV; ++e) vp[e] = o[q + e];
        *reinterpret_cast<Vt*>(dst + q) = v;
      }
    }
    __syncthreads();
  }
}

#ifdef MS_COARSE_PROBE
// per-CTA timestamps of the coarse kernels (timing experiments only)
__device__ unsigned long long g_coarse_probe[2][512][8];
__device__ __forceinline__ void probe(int kind, int slot) {
  if (threadIdx.x == 0 && blockIdx.x < 512) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    g_coarse_probe[kind][blockIdx.x][slot] = t;
  }
}
#else
__device__ __forceinline__ void probe(int, int) {}
#endif

// the CTA's basis and its rank in the basis's group
__device__ __forceinline__ void group_of(const CoarseGroups& gr, int M, int& m, int& rank,
                                         int& cs) {
  // unrolled (no dynamic index into the parameter array)
  const int b = (int)blockIdx.x;
  m = 0;
  int lo = gr.first[0], hi = gr.first[1];
#pragma unroll
  for (int q = 1; q < kMaxBases; ++q) {
    if (q < M && b >= gr.first[q]) {
      m = q;
      lo = gr.first[q];
      hi = gr.first[q + 1];
    }
  }
  rank = b - lo;
  cs = hi - lo;
}

// Synthesis levels J..2, one basis per group: LL_{j-1} of basis m at
// tmp + (j & 1) half + m (N/2)^2 (level 2: the buffer level-1 synthesis
// reads).  bar: two ints per basis (group barrier state).
template <typename R>
__global__ void __launch_bounds__(kStripThreads, 1)
    coarse_synthesis_kernel(FistaPass<R> a, CoarseGroups gr, int* bar, int rc_budget_bytes) {
  const int done = a.ctl->done;
  const int k = a.ctl->k;
  if (done) return;   // uniform over the grid
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* smem = reinterpret_cast<R*>(smem_raw);
  int m, rank, cs;
  group_of(gr, a.M, m, rank, cs);
  const R* coef = k % 3 == 0 ? a.B0 : (k % 3 == 1 ? a.B1 : a.B2);
  const int N = a.N, J = a.J;
  const int64_t half = (int64_t)a.M * (N / 2) * (N / 2);
  const int64_t region = (int64_t)m * (N / 2) * (N / 2);
  const R* plane = coef + (int64_t)m * N * N;
  probe(0, 0);
  for (int j = J; j >= 2; --j) {
    const int h = N >> j, n = 2 * h;
    const R* ap = (j == J) ? plane : a.tmp + ((j + 1) & 1) * half + region;
    const int aps = (j == J) ? N : h;   // row stride of the approximation
    R* out = a.tmp + (j & 1) * half + region;
    int t0, t1;
    strip_rows(n, cs, rank, t0, t1);
    const int rc = strip_chunk_rows(false, n, sizeof(R), (size_t)rc_budget_bytes, t1 - t0);
    switch (m) {
#define MS_SS(MBV) \
  case MBV: strip_synthesis_level<R, MBV>(ap, aps, plane, N, h, out, t0, t1, rc, smem); break;
      MS_SS(0) MS_SS(1) MS_SS(2) MS_SS(3) MS_SS(4) MS_SS(5) MS_SS(6) MS_SS(7)
#undef MS_SS
    }
    probe(0, 1 + 2 * (J - j));
    if (j > 2) group_barrier(bar + 2 * m, cs, a.ctl);   // LL_{j-1} complete for level j - 1
    probe(0, 2 + 2 * (J - j));
  }
}

// Analysis + FISTA step of levels 2..J, one basis per group, from LL_1 at
// tmp + half + m (N/2)^2 (written by level 1).  Each CTA leaves its sum of
// |B_{k+1}| in l1_parts[part_base + blockIdx.x] and zeroes the slots up to
// part_end (the per-level kernels' share of the partials).
template <typename R>
__global__ void __launch_bounds__(kStripThreads, 1)
    coarse_analysis_kernel(FistaPass<R> a, CoarseGroups gr, int* bar, int part_base,
                           int part_end, int rc_budget_bytes) {
  const int done = a.ctl->done;
  const int kc = a.ctl->k;
  if (done) return;   // uniform over the grid
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* smem = reinterpret_cast<R*>(smem_raw);
  int m, rank, cs;
  group_of(gr, a.M, m, rank, cs);
  const int k = kc - 1;
  const R t = ctl_t<R>(a.ctl, k & 1);   // momentum t_k
  const R mu = ctl_mu<R>(a.ctl);        // 1 / theta
  const R thr = ctl_thr<R>(a.ctl);      // lambda / theta
  const R* cur = k % 3 == 0 ? a.B0 : (k % 3 == 1 ? a.B1 : a.B2);
  const R* prev = k % 3 == 0 ? a.B2 : (k % 3 == 1 ? a.B0 : a.B1);
  R* next = k % 3 == 0 ? a.B1 : (k % 3 == 1 ? a.B2 : a.B0);
  const int N = a.N, J = a.J;
  const int64_t half = (int64_t)a.M * (N / 2) * (N / 2);
  const int64_t region = (int64_t)m * (N / 2) * (N / 2);
  const int64_t plane = (int64_t)m * N * N;
  KSum<R> l1;
  probe(1, 0);
  for (int j = 2; j <= J; ++j) {
    const int n = N >> (j - 1), h = n / 2;
    const R* in = a.tmp + ((j - 1) & 1) * half + region;
    R* ll_out = a.tmp + (j & 1) * half + region;
    int i0, i1;
    strip_rows(h, cs, rank, i0, i1);
    const int rc = strip_chunk_rows(true, n, sizeof(R), (size_t)rc_budget_bytes, i1 - i0);
    switch (m) {
#define MS_SA(MBV)                                                                            \
  case MBV:                                                                                   \
    strip_analysis_level<R, MBV>(in, ll_out, n, j == J, i0, i1, rc, smem, cur, prev, next,    \
                                 plane, N, t, mu, thr, l1);                                    \
    break;
      MS_SA(0) MS_SA(1) MS_SA(2) MS_SA(3) MS_SA(4) MS_SA(5) MS_SA(6) MS_SA(7)
#undef MS_SA
    }
    probe(1, 1 + 2 * (j - 2));
    if (j < J) group_barrier(bar + 2 * m, cs, a.ctl);   // LL_j complete for level j + 1
    probe(1, 2 + 2 * (j - 2));
  }
  // block sum of |B_{k+1}| (working-precision pairs within a warp, FP64 once
  // per warp), in a fixed order
  double* red = reinterpret_cast<double*>(smem_raw);
  R hi = l1.s, lo = -l1.c;
  warp_sum_comp<R>(hi, lo);
  __syncthreads();   // the staging buffers are dead
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)hi + (double)lo;
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum = 0.0;
    for (int q = 0; q < kStripThreads / 32; ++q) sum += red[q];
    a.l1_parts[part_base + blockIdx.x] = sum;
  }
  for (int q = part_base + (int)gridDim.x + blockIdx.x * kStripThreads + threadIdx.x; q < part_end;
       q += (int)gridDim.x * kStripThreads)
    a.l1_parts[q] = 0.0;
}
