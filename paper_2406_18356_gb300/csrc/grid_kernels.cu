// Measurement operator kernels (Sect. 2: i~ = F^H G^H (v - G F x)):
//   pad   : D Z   (deapodize, zero-pad N -> Ng, checkerboard so the FFT is centred)
//   crop  : Z^H D^H (real part of the centred inverse FFT, deapodize, 1/sum w)
//   degrid: G     (TMA-staged grid tile, W x W ES taps per visibility)
//   grid  : G^H   (register sums per anchor run, warp-private shared-memory
//                  sub-tiles, no global atomics)
//   fold  : sums the per-work-item tiles (with their halos) into the grid.
#include "common.cuh"

namespace ms {

namespace {
constexpr int kThreads = 256;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ unsigned mbar_try_wait(uint64_t* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(phase)
      : "memory");
  return ok;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

// bounded wait on an mbarrier phase; false if it ran out
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, unsigned phase) {
  for (int it = 0; it < (1 << 22); ++it)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

// ES weights of the W taps along one axis, from the centre offset f of the
// footprint: tap i is at distance t = f + (W-1)/2 - i cells from the sample.
// phi = exp(beta (sqrt(1 - z^2) - 1)) is evaluated as
// exp(-beta z^2 / (1 + sqrt(1 - z^2))) so the centre taps keep full precision.
// FP64: correctly rounded library sqrt / exp and an IEEE division.  FP32:
// the SFU's approximate square root, reciprocal and base-2 exponential
// (relative errors near 2^-22 each, far inside the FP32 form's 1e-5 bar),
// with exp(x) = 2^(x log2 e).
__device__ __forceinline__ float sqrt_approx(float x) {
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ float exp2_approx(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
// packed FP32 pair FMA (fma.rn.f32x2): d = a b + c in both lanes, each
// rounded as fmaf
__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) {
  float2 d;
  asm("{\n\t.reg .b64 ra, rb, rc, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\tmov.b64 rc, {%6, %7};\n\t"
      "fma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d.x), "=f"(d.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
  return d;
}
#ifndef MS_DEGRID_PACKED
#define MS_DEGRID_PACKED 1
#endif

template <typename R>
__device__ __forceinline__ void es_weights(R f, R beta, R* w) {
  const R c = (R)(4.0 / (kW * kW));
#pragma unroll
  for (int i = 0; i < kW; ++i) {
    R t = f + (R)(kHalfW - i);
    R z2 = t * t * c;
    R s = (R)1 - z2;
    s = s > (R)0 ? s : (R)0;
    w[i] = exp(-beta * z2 / ((R)1 + sqrt(s)));
  }
}
template <>
__device__ __forceinline__ void es_weights<float>(float f, float beta, float* w) {
  const float c = 4.0f / (kW * kW);
  const float nb = -beta * 1.4426950408889634f;   // -beta log2(e)
#pragma unroll
  for (int i = 0; i < kW; ++i) {
    const float t = f + (float)(kHalfW - i);
    const float z2 = t * t * c;
    const float s = fmaxf(1.0f - z2, 0.0f);
    w[i] = exp2_approx(nb * z2 * rcp_approx(1.0f + sqrt_approx(s)));
  }
}
}  // namespace

// ------------------------------------------------------------------ pad / crop
template <typename R>
__global__ void pad_kernel(const R* __restrict__ image, const R* __restrict__ psi, int npix,
                           int Ng, C2<R>* __restrict__ grid) {
  int64_t total = (int64_t)Ng * Ng;
  const int h = npix / 2;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int rr = (int)(k / Ng), cc = (int)(k % Ng);
    int a = cc < h ? cc : (cc >= Ng - h ? cc - Ng : INT32_MAX);
    int b = rr < h ? rr : (rr >= Ng - h ? rr - Ng : INT32_MAX);
    C2<R> o;
    o.x = (R)0;
    o.y = (R)0;
    if (a != INT32_MAX && b != INT32_MAX) {
      int q = a + h, p = b + h;
      R val = image[(int64_t)p * npix + q] / (psi[p] * psi[q]);
      o.x = ((a + b) & 1) ? -val : val;
    }
    grid[k] = o;
  }
}

template <typename R>
__global__ void crop_kernel(const C2<R>* __restrict__ grid, const R* __restrict__ psi,
                            int npix, int Ng, R scale, R* __restrict__ image) {
  int64_t total = (int64_t)npix * npix;
  const int h = npix / 2;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int p = (int)(k / npix), q = (int)(k % npix);
    int a = q - h, b = p - h;
    int cc = a < 0 ? a + Ng : a;
    int rr = b < 0 ? b + Ng : b;
    R val = grid[(int64_t)rr * Ng + cc].x * scale / (psi[p] * psi[q]);
    image[k] = ((a + b) & 1) ? -val : val;
  }
}

template <typename R>
void launch_pad(const R* image, const R* psi, int npix, int Ng, C2<R>* grid, cudaStream_t s) {
  int64_t total = (int64_t)Ng * Ng;
  int blocks = (int)((total + kThreads - 1) / kThreads);
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  pad_kernel<R><<<blocks, kThreads, 0, s>>>(image, psi, npix, Ng, grid);
}

template <typename R>
void launch_crop(const C2<R>* grid, const R* psi, int npix, int Ng, double scale, R* image,
                 cudaStream_t s) {
  int64_t total = (int64_t)npix * npix;
  int blocks = (int)((total + kThreads - 1) / kThreads);
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  crop_kernel<R><<<blocks, kThreads, 0, s>>>(grid, psi, npix, Ng, (R)scale, image);
}

// ------------------------------------------------------------------ degrid
// One CTA per work item.  The (T + W - 1)^2 grid region that the item's
// footprints cover is staged in shared memory by one TMA tensor copy (plain
// loads with periodic wrap for tiles on the grid's last row/column), then each
// thread interpolates visibilities: V = sum_j phi_v[j] sum_i phi_u[i] G[..].
// One degridding work item `it` of a grid whose TMA descriptor row of the
// grid's first row is tma_y0 (0 for one grid; job * Ng for stacked grids).
template <typename R, bool HAS_OBS>
__device__ __forceinline__ void degrid_item(const CUtensorMap* tmap, int tma_y0,
                                            const C2<R>* __restrict__ grid, const WorkItem it,
                                            const uint32_t* __restrict__ cell,
                                            const C2<R>* __restrict__ frac,
                                            const C2<R>* __restrict__ obs,
                                            C2<R>* __restrict__ out, int Ng, int T, int ntx,
                                            R beta, int32_t* __restrict__ err) {
  // the tile sits at a 128-byte-aligned shared address (TMA destination rule),
  // the mbarrier and a flag after it, all in the dynamic allocation
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const unsigned pad = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
  C2<R>* tile = reinterpret_cast<C2<R>*>(smem_raw + pad);
  const int S = T + kW - 1;
  uint64_t& bar = *reinterpret_cast<uint64_t*>(tile + S * S);
  int& use_tma = *reinterpret_cast<int*>(&bar + 1);
  const int tx = it.tile % ntx, ty = it.tile / ntx;
  const int ox = tx * T, oy = ty * T;
  bool edge = (ox + S > Ng) || (oy + S > Ng);
  bool ok = true;
  if (!edge) {
    if (threadIdx.x == 0) {
      // alignment rules of the copy, checked before it is issued
      const bool aligned = (smem_addr(tile) & 127u) == 0 &&
                           (reinterpret_cast<uintptr_t>(tmap) & 63u) == 0 &&
                           ((2 * ox * (int)sizeof(R)) & 15) == 0;
      use_tma = aligned ? 1 : 0;
      if (aligned) {
        mbar_init(&bar, 1);
        fence_mbar_init();
      } else {
        atomicExch(err, 8);
      }
    }
    __syncthreads();
    edge = use_tma == 0;
  }
  if (!edge) {
    if (threadIdx.x == 0) {
      mbar_expect_tx(&bar, (unsigned)(S * S * sizeof(C2<R>)));
      tma_load_2d(tile, tmap, 2 * ox, tma_y0 + oy, &bar);
    }
    ok = mbar_wait_bounded(&bar, 0);
    if (!ok) {
      if (threadIdx.x == 0) atomicExch(err, 5);
      mbar_wait_bounded(&bar, 0);   // give the copy in flight a second bounded chance
      return;
    }
  } else {
    for (int c = threadIdx.x; c < S * S; c += blockDim.x) {
      int lv = c / S, lu = c - lv * S;
      int gy = oy + lv, gx = ox + lu;
      gy -= gy >= Ng ? Ng : 0;
      gx -= gx >= Ng ? Ng : 0;
      tile[c] = grid[(int64_t)gy * Ng + gx];
    }
    __syncthreads();
  }
  const int end = it.start + it.count;
  for (int k = it.start + threadIdx.x; k < end; k += blockDim.x) {
    uint32_t pc = cell[k];
    int lu = (int)(pc & 0xffffu) - ox;
    int lv = (int)(pc >> 16) - oy;
    C2<R> f = frac[k];
    R wu[kW], wv[kW];
    es_weights<R>(f.x, beta, wu);
    es_weights<R>(f.y, beta, wv);
    R accr = 0, acci = 0;
    if constexpr (sizeof(R) == 4 && MS_DEGRID_PACKED) {
      // the real and imaginary chains as packed FP32 pairs (same operations)
      float2 acc = make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < kW; ++j) {
        const float2* row = reinterpret_cast<const float2*>(tile + (lv + j) * S + lu);
        float2 r = make_float2(0.f, 0.f);
#pragma unroll
        for (int i = 0; i < kW; ++i) r = ffma2(make_float2(wu[i], wu[i]), row[i], r);
        acc = ffma2(make_float2(wv[j], wv[j]), r, acc);
      }
      accr = acc.x;
      acci = acc.y;
    } else {
#pragma unroll
      for (int j = 0; j < kW; ++j) {
        const C2<R>* row = tile + (lv + j) * S + lu;
        R rr = 0, ri = 0;
#pragma unroll
        for (int i = 0; i < kW; ++i) {
          C2<R> g = row[i];
          rr = fma(wu[i], g.x, rr);
          ri = fma(wu[i], g.y, ri);
        }
        accr = fma(wv[j], rr, accr);
        acci = fma(wv[j], ri, acci);
      }
    }
    C2<R> o;
    if (HAS_OBS) {
      C2<R> v = obs[k];
      o.x = v.x - accr;
      o.y = v.y - acci;
    } else {
      o.x = accr;
      o.y = acci;
    }
    out[k] = o;
  }
}


template <typename R, bool HAS_OBS>
__global__ void __launch_bounds__(kThreads)
    degrid_kernel(const __grid_constant__ CUtensorMap tmap, const C2<R>* __restrict__ grid,
                  const WorkItem* __restrict__ items, const uint32_t* __restrict__ cell,
                  const C2<R>* __restrict__ frac, const C2<R>* __restrict__ obs,
                  C2<R>* __restrict__ out, int Ng, int T, int ntx, R beta,
                  int32_t* __restrict__ err) {
  degrid_item<R, HAS_OBS>(&tmap, 0, grid, items[blockIdx.x], cell, frac, obs, out, Ng, T, ntx,
                          beta, err);
}

// Stacked form: one block per work item of all jobs; job_of[item] names the
// job, whose grid is row block job * Ng of the stacked TMA descriptor.
template <typename R, bool HAS_OBS>
__global__ void __launch_bounds__(kThreads)
    degrid_batch_kernel(const __grid_constant__ CUtensorMap tmap,
                        const BatchJob<R>* __restrict__ jobs, const int32_t* __restrict__ job_of,
                        int Ng, int T, int ntx, R beta, int32_t* __restrict__ err) {
  const int j = job_of[blockIdx.x];
  const BatchJob<R> jb = jobs[j];
  const WorkItem it = jb.items[blockIdx.x - jb.item_base];
  degrid_item<R, HAS_OBS>(&tmap, j * Ng, jb.grid, it, jb.cell, jb.frac, jb.sorted_in,
                          jb.sorted_out, Ng, T, ntx, beta, err);
}

template <typename R>
void launch_degrid(const CUtensorMap* tmap, const C2<R>* grid, const WorkItem* items,
                   int nitems, const uint32_t* cell, const C2<R>* frac, const C2<R>* obs,
                   C2<R>* out, int Ng, int tile, int ntx, double beta, int32_t* err,
                   cudaStream_t s) {
  if (nitems <= 0) return;
  const int S = tile + kW - 1;
  // tile + alignment slack + mbarrier + flag
  size_t smem = (size_t)S * S * sizeof(C2<R>) + 128 + sizeof(uint64_t) + sizeof(int) + 4;
  if (obs) {
    auto k = degrid_kernel<R, true>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<nitems, kThreads, smem, s>>>(*tmap, grid, items, cell, frac, obs, out, Ng, tile, ntx,
                                     (R)beta, err);
  } else {
    auto k = degrid_kernel<R, false>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<nitems, kThreads, smem, s>>>(*tmap, grid, items, cell, frac, obs, out, Ng, tile, ntx,
                                     (R)beta, err);
  }
}

// ------------------------------------------------------------------ grid
// Scratch holds one (T + W - 1)^2 tile per work item: float2 for the plain
// FP32 form, double2 for FP64 and for the compensated FP32 form.
template <typename R, bool KAHAN> struct ScratchOf { using T = double2; };
template <> struct ScratchOf<float, false> { using T = float2; };

size_t grid_scratch_cell_bytes(int precision) { return precision == 1 ? 8 : 16; }

template <typename R, bool KAHAN> __host__ __device__ constexpr int grid_warps() {
  return (KAHAN || sizeof(R) == 8) ? 4 : 8;
}

// Adds v (and, compensated, its correction) to a tile cell.
template <typename R, bool KAHAN>
__device__ __forceinline__ void cell_add(C2<R>* my, C2<R>* myc, int c, C2<R> v) {
  C2<R> a = my[c];
  if (KAHAN) {
    C2<R> cp = myc[c];
    const R yr = v.x - cp.x, yi = v.y - cp.y;
    const R tr = a.x + yr, ti = a.y + yi;
    cp.x = (tr - a.x) - yr;
    cp.y = (ti - a.y) - yi;
    a.x = tr;
    a.y = ti;
    myc[c] = cp;
  } else {
    a.x += v.x;
    a.y += v.y;
  }
  my[c] = a;
}

// Register sum of one tap over a run of visibilities (compensated for the
// Kahan form).
template <typename R, bool KAHAN> struct TapSum {
  R sr = 0, si = 0, cr = 0, ci = 0;
  __device__ __forceinline__ void add(R w, C2<R> v) {
    if (KAHAN) {
      const R yr = w * v.x - cr, yi = w * v.y - ci;
      const R tr = sr + yr, ti = si + yi;
      cr = (tr - sr) - yr;
      ci = (ti - si) - yi;
      sr = tr;
      si = ti;
    } else {
      sr = fma(w, v.x, sr);
      si = fma(w, v.y, si);
    }
  }
  __device__ __forceinline__ C2<R> value() const {
    C2<R> o;
    o.x = sr - cr;
    o.y = si - ci;
    return o;
  }
  __device__ __forceinline__ void clear() { sr = si = cr = ci = (R)0; }
};

// FP64 and compensated FP32 forms (the plain FP32 form: grid_item_lanes).
// A warp grids its share of the work item's rows, which the plan sorts by
// anchor cell inside the tile: lane t takes tap t (t < 32) and lanes 0..16
// also tap t + 32 (tap (i, j) = (t mod 7, t div 7)).  While consecutive rows
// share an anchor cell, every lane sums its taps' contributions in registers;
// when the anchor changes, the lanes add their sums to the 49 distinct cells
// of the footprint in the warp's own sub-tile (no atomics) and __syncwarp
// orders that update before the next.  The rows' ES weights, values and
// anchors are staged 32 at a time in shared memory.  The compensated form
// sums each run with Kahan compensation and adds it into compensated cells.
// At the end the warps' sub-tiles are summed in a fixed order into the
// item's scratch tile.
// One gridding work item `it`; its tile goes to scratch tile `scratch_tile`.
template <typename R, bool KAHAN>
__device__ __forceinline__ void grid_item(const WorkItem it, const uint32_t* __restrict__ cell,
                                          const C2<R>* __restrict__ frac,
                                          const C2<R>* __restrict__ vis,
                                          typename ScratchOf<R, KAHAN>::T* __restrict__ scratch,
                                          int64_t scratch_tile, int T, int ntx, R beta) {
  using Acc = typename ScratchOf<R, KAHAN>::T;
  constexpr int NW = grid_warps<R, KAHAN>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int S = T + kW - 1;
  const int cells = S * S;
  C2<R>* tiles = reinterpret_cast<C2<R>*>(smem_raw);                  // [NW][cells]
  C2<R>* comps = tiles + (KAHAN ? NW * cells : 0);                     // [NW][cells]
  R* stage_w = reinterpret_cast<R*>(tiles + (KAHAN ? 2 : 1) * NW * cells);  // [NW][32][14]
  C2<R>* stage_v = reinterpret_cast<C2<R>*>(stage_w + NW * 32 * 2 * kW);     // [NW][32]
  int* stage_c = reinterpret_cast<int*>(stage_v + NW * 32);                  // [NW][32]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ox = (it.tile % ntx) * T, oy = (it.tile / ntx) * T;

  for (int c = threadIdx.x; c < NW * cells; c += blockDim.x) {
    C2<R> z;
    z.x = (R)0;
    z.y = (R)0;
    tiles[c] = z;
    if (KAHAN) comps[c] = z;
  }
  __syncthreads();

  C2<R>* my = tiles + warp * cells;
  C2<R>* myc = comps + warp * cells;
  R* sw = stage_w + warp * 32 * 2 * kW;
  C2<R>* sv = stage_v + warp * 32;
  int* sc = stage_c + warp * 32;
  const int i1 = lane % kW, j1 = lane / kW;
  const int i2 = (lane + 32) % kW, j2 = (lane + 32) / kW;
  const bool two = lane + 32 < kW * kW;
  const int off1 = j1 * S + i1, off2 = j2 * S + i2;

  const int per = (it.count + NW - 1) / NW;
  const int ws = it.start + warp * per;
  int we = ws + per;
  if (we > it.start + it.count) we = it.start + it.count;
  TapSum<R, KAHAN> t1, t2;
  int run = -1;   // anchor (tile-local cell index) of the current run
  for (int base = ws; base < we; base += 32) {
    int k = base + lane;
    if (k < we) {
      uint32_t pc = cell[k];
      int lu = (int)(pc & 0xffffu) - ox;
      int lv = (int)(pc >> 16) - oy;
      C2<R> f = frac[k];
      es_weights<R>(f.x, beta, sw + lane * 2 * kW);
      es_weights<R>(f.y, beta, sw + lane * 2 * kW + kW);
      sv[lane] = vis[k];
      sc[lane] = lv * S + lu;
    }
    __syncwarp();
    int nb = we - base < 32 ? we - base : 32;
    for (int sidx = 0; sidx < nb; ++sidx) {
      const int c0 = sc[sidx];   // uniform over the warp
      if (c0 != run) {
        if (run >= 0) {
          cell_add<R, KAHAN>(my, myc, run + off1, t1.value());
          if (two) cell_add<R, KAHAN>(my, myc, run + off2, t2.value());
          __syncwarp();   // this run's cells before the next run's
        }
        run = c0;
        t1.clear();
        t2.clear();
      }
      const R* w = sw + sidx * 2 * kW;
      const C2<R> val = sv[sidx];
      t1.add(w[i1] * w[kW + j1], val);
      if (two) t2.add(w[i2] * w[kW + j2], val);
    }
    __syncwarp();   // the staging buffers are rewritten
  }
  if (run >= 0) {
    cell_add<R, KAHAN>(my, myc, run + off1, t1.value());
    if (two) cell_add<R, KAHAN>(my, myc, run + off2, t2.value());
  }
  __syncthreads();
  Acc* dst = scratch + scratch_tile * cells;
  for (int c = threadIdx.x; c < cells; c += blockDim.x) {
    Acc s;
    s.x = 0;
    s.y = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      C2<R> a = tiles[w * cells + c];
      if (KAHAN) {
        C2<R> cp = comps[w * cells + c];
        s.x += (double)a.x - (double)cp.x;
        s.y += (double)a.y - (double)cp.y;
      } else {
        s.x += a.x;
        s.y += a.y;
      }
    }
    dst[c] = s;
  }
}


// Plain FP32 form: a lane per row instead of a lane per tap.  A warp's rows
// are cut into 32 contiguous slots, one per lane.  A lane walks its slot and
// sums in registers the 49 taps' contributions wu_i (wv_j v) of the rows that
// share its current anchor cell (packed FP32 pairs, real and imaginary part
// together); the next row's cell, offsets and value are loaded a step ahead.
// When its anchor changes, and after its slot's last row, the lane's sums
// are flushed: the flushing lanes of a step, up to kStageRows at a time in
// ascending lane order, write their sums to rows of the warp's staging
// buffer, and the warp adds each staged row, lane per tap, into its sub-tile
// (one fixed order, so the result does not depend on timing).  Per row a
// lane issues its 14 ES weights and 56 packed multiply-adds, against the
// lane-per-tap form's staging, broadcast reads and unpacked FMAs of every
// tap.
#ifndef MS_GRID_LANE_ROWS
#define MS_GRID_LANE_ROWS 1
#endif
#ifndef MS_GRID_STAGE_ROWS
#define MS_GRID_STAGE_ROWS 8
#endif
constexpr int kLaneWarps = 4;          // warps per block of the lane-per-row form
constexpr int kStageQuads = 25;        // float4 per staging row: 49 taps + 1 pad
constexpr int kStageRows = MS_GRID_STAGE_ROWS;   // staging rows per warp (<= 32)
static_assert(kStageRows >= 1 && kStageRows <= 32, "staging rows per warp");

__host__ __device__ constexpr size_t grid_lanes_smem(int S) {
  return (size_t)kLaneWarps * kStageRows * kStageQuads * 16 +
         (size_t)kLaneWarps * kStageRows * 4 + (size_t)kLaneWarps * S * S * 8;
}

// One walk of a warp's slots for the tap rows j in [J0, J0 + NJ) of the
// footprint (all seven taps i of each): register sums, flushes through the
// staging rows, lane-per-tap adds into the warp's sub-tile `my`.
template <int J0, int NJ>
__device__ __forceinline__ void grid_lanes_pass(const uint32_t* __restrict__ cell,
                                                const float2* __restrict__ frac,
                                                const float2* __restrict__ vis, float2* my,
                                                float4* st, int* sa, int lane, int ms, int me,
                                                int PL, int ox, int oy, int S, float beta) {
  constexpr int NT = NJ * kW;            // taps of this walk
  constexpr int NQ = (NT + 1) / 2;       // float4 per staging row
  // lane-per-tap cells of the adds: tap t = (i, j) = (t mod 7, J0 + t div 7)
  const bool one = lane < NT;
  const int off1 = (J0 + lane / kW) * S + lane % kW;
  const bool two = lane + 32 < NT;
  const int off2 = (J0 + (lane + 32) / kW) * S + (lane + 32) % kW;

  float2 acc[2 * NQ];   // NT taps; an odd count leaves the last entry zero (staging pad)
#pragma unroll
  for (int t = 0; t < 2 * NQ; ++t) acc[t] = make_float2(0.f, 0.f);
  int cur = -1;   // anchor (tile-local cell index) of the sums held
  uint32_t pc_n = 0;
  float2 f_n = make_float2(0.f, 0.f), v_n = make_float2(0.f, 0.f);
  if (ms < me) {
    pc_n = cell[ms];
    f_n = frac[ms];
    v_n = vis[ms];
  }
  for (int m = 0; m <= PL; ++m) {   // the extra step flushes the slots' last sums
    const int k = ms + m;
    const bool valid = k < me;
    const int a = valid ? ((int)(pc_n >> 16) - oy) * S + (int)(pc_n & 0xffffu) - ox : -1;
    const float2 f = f_n, v = v_n;
    if (k + 1 < me) {
      pc_n = cell[k + 1];
      f_n = frac[k + 1];
      v_n = vis[k + 1];
    }
    const bool fl = cur >= 0 && a != cur;
    const unsigned fm = __ballot_sync(0xffffffffu, fl);
    for (unsigned todo = fm; todo;) {
      // the next (up to) kStageRows flushing lanes, lowest lanes first
      unsigned later = todo;
#pragma unroll
      for (int c = 0; c < kStageRows; ++c) later &= later - 1;
      const unsigned batch = todo ^ later;
      todo = later;
      if ((batch >> lane) & 1u) {
        const int r = __popc(batch & ((1u << lane) - 1u));
#pragma unroll
        for (int q = 0; q < NQ; ++q)
          st[r * kStageQuads + q] =
              make_float4(acc[2 * q].x, acc[2 * q].y, acc[2 * q + 1].x, acc[2 * q + 1].y);
        sa[r] = cur;
      }
      __syncwarp();
      const int nb = __popc(batch);
      for (int r = 0; r < nb; ++r) {
        const float2* row = reinterpret_cast<const float2*>(st + r * kStageQuads);
        const int c0 = sa[r];
        if (one) {
          float2 s1 = row[lane];
          float2 o1 = my[c0 + off1];
          o1.x += s1.x;
          o1.y += s1.y;
          my[c0 + off1] = o1;
        }
        if (two) {
          float2 s2 = row[lane + 32];
          float2 o2 = my[c0 + off2];
          o2.x += s2.x;
          o2.y += s2.y;
          my[c0 + off2] = o2;
        }
        __syncwarp();   // this row's cells (and staging reads) before the next
      }
    }
    if (fl) {
#pragma unroll
      for (int t = 0; t < NT; ++t) acc[t] = make_float2(0.f, 0.f);
    }
    cur = a;
    if (valid) {
      float wu[kW], wv[kW];
      es_weights<float>(f.x, beta, wu);
      es_weights<float>(f.y, beta, wv);
#pragma unroll
      for (int j = 0; j < NJ; ++j) {
        const float2 wvv = make_float2(wv[J0 + j] * v.x, wv[J0 + j] * v.y);
#pragma unroll
        for (int i = 0; i < kW; ++i)
          acc[j * kW + i] = ffma2(make_float2(wu[i], wu[i]), wvv, acc[j * kW + i]);
      }
    }
  }
}

__device__ __forceinline__ void grid_item_lanes(const WorkItem it,
                                                const uint32_t* __restrict__ cell,
                                                const float2* __restrict__ frac,
                                                const float2* __restrict__ vis,
                                                float2* __restrict__ scratch,
                                                int64_t scratch_tile, int T, int ntx,
                                                float beta) {
  constexpr int NW = kLaneWarps;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int S = T + kW - 1;
  const int cells = S * S;
  float4* stage = reinterpret_cast<float4*>(smem_raw);   // [NW][kStageRows][25]
  int* stage_a = reinterpret_cast<int*>(stage + NW * kStageRows * kStageQuads);
  float2* tiles = reinterpret_cast<float2*>(stage_a + NW * kStageRows);   // [NW][cells]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ox = (it.tile % ntx) * T, oy = (it.tile / ntx) * T;
  for (int c = threadIdx.x; c < NW * cells; c += blockDim.x) tiles[c] = make_float2(0.f, 0.f);
  __syncthreads();

  float2* my = tiles + warp * cells;
  float4* st = stage + warp * kStageRows * kStageQuads;
  int* sa = stage_a + warp * kStageRows;

  const int per = (it.count + NW - 1) / NW;
  const int ws = it.start + warp * per;
  int we = ws + per;
  if (we > it.start + it.count) we = it.start + it.count;
  const int len = we - ws;
  const int PL = len > 0 ? (len + 31) / 32 : 0;   // rows per lane slot
  const int ms = ws + lane * PL;
  const int me = ms + PL < we ? ms + PL : we;     // this lane's slot [ms, me)
  grid_lanes_pass<0, kW>(cell, frac, vis, my, st, sa, lane, ms, me, PL, ox, oy, S, beta);
  __syncthreads();
  float2* dst = scratch + scratch_tile * cells;
  for (int c = threadIdx.x; c < cells; c += blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const float2 a = tiles[w * cells + c];
      s.x += a.x;
      s.y += a.y;
    }
    dst[c] = s;
  }
}

// the plain FP32 form takes the lane-per-row item when it is enabled
template <typename R, bool KAHAN> __host__ __device__ constexpr bool grid_lane_rows() {
  return MS_GRID_LANE_ROWS && sizeof(R) == 4 && !KAHAN;
}
template <typename R, bool KAHAN> __host__ __device__ constexpr int grid_block_threads() {
  return grid_lane_rows<R, KAHAN>() ? 32 * kLaneWarps : 32 * grid_warps<R, KAHAN>();
}
// Resident blocks per SM the lane-per-row form is compiled for: 3, so up to
// 170 registers a thread (the tap sums take 98), 12 warps.  Measured at
// 1024 px, 9.27M rows: 215 us, against 242 us with 4 blocks (128
// registers, 16 warps): more independent weight and multiply-add chains per
// warp pay more than the extra warps.
#ifndef MS_GRID_LANE_MINB
#define MS_GRID_LANE_MINB 3
#endif
template <typename R, bool KAHAN> __host__ __device__ constexpr int grid_min_blocks() {
  return grid_lane_rows<R, KAHAN>() ? MS_GRID_LANE_MINB : 1;
}
template <typename R, bool KAHAN> size_t grid_smem_bytes(int tile) {
  const int S = tile + kW - 1;
  if (grid_lane_rows<R, KAHAN>()) return grid_lanes_smem(S);
  constexpr int NW = grid_warps<R, KAHAN>();
  return (size_t)NW * S * S * sizeof(C2<R>) * (KAHAN ? 2 : 1) +
         (size_t)NW * 32 * (2 * kW * sizeof(R) + sizeof(C2<R>) + sizeof(int));
}

template <typename R, bool KAHAN>
__device__ __forceinline__ void grid_any_item(const WorkItem it, const uint32_t* cell,
                                              const C2<R>* frac, const C2<R>* vis,
                                              typename ScratchOf<R, KAHAN>::T* scratch,
                                              int64_t scratch_tile, int T, int ntx, R beta) {
  if constexpr (grid_lane_rows<R, KAHAN>())
    grid_item_lanes(it, cell, reinterpret_cast<const float2*>(frac),
                    reinterpret_cast<const float2*>(vis), reinterpret_cast<float2*>(scratch),
                    scratch_tile, T, ntx, (float)beta);
  else
    grid_item<R, KAHAN>(it, cell, frac, vis, scratch, scratch_tile, T, ntx, beta);
}

template <typename R, bool KAHAN>
__global__ void __launch_bounds__(grid_block_threads<R, KAHAN>(), grid_min_blocks<R, KAHAN>())
    grid_kernel(const WorkItem* __restrict__ items, const uint32_t* __restrict__ cell,
                const C2<R>* __restrict__ frac, const C2<R>* __restrict__ vis,
                typename ScratchOf<R, KAHAN>::T* __restrict__ scratch, int Ng, int T, int ntx,
                R beta) {
  grid_any_item<R, KAHAN>(items[blockIdx.x], cell, frac, vis, scratch, blockIdx.x, T, ntx, beta);
}

// Stacked form: one block per work item of all jobs (scratch tile = the
// item's index over all jobs).
template <typename R, bool KAHAN>
__global__ void __launch_bounds__(grid_block_threads<R, KAHAN>(), grid_min_blocks<R, KAHAN>())
    grid_batch_kernel(const BatchJob<R>* __restrict__ jobs, const int32_t* __restrict__ job_of,
                      typename ScratchOf<R, KAHAN>::T* __restrict__ scratch, int T, int ntx,
                      R beta) {
  const BatchJob<R> jb = jobs[job_of[blockIdx.x]];
  grid_any_item<R, KAHAN>(jb.items[blockIdx.x - jb.item_base], jb.cell, jb.frac, jb.sorted_in,
                      scratch, blockIdx.x, T, ntx, beta);
}

template <typename R, bool KAHAN>
void launch_grid(const WorkItem* items, int nitems, const uint32_t* cell, const C2<R>* frac,
                 const C2<R>* vis, void* scratch, int Ng, int tile, int ntx, double beta,
                 cudaStream_t s) {
  if (nitems <= 0) return;
  const size_t smem = grid_smem_bytes<R, KAHAN>(tile);
  auto k = grid_kernel<R, KAHAN>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<nitems, grid_block_threads<R, KAHAN>(), smem, s>>>(items, cell, frac, vis,
                                 reinterpret_cast<typename ScratchOf<R, KAHAN>::T*>(scratch),
                                 Ng, tile, ntx, (R)beta);
}

// Cells are walked x-stride over the whole grid (dense tiles, with many
// items, spread over all blocks); a cell's items are read four at a time
// (independent loads in flight) and added in item order.
template <typename R, bool KAHAN>
__device__ __forceinline__ void fold_cells(const typename ScratchOf<R, KAHAN>::T* __restrict__ scratch,
                                           const int32_t* __restrict__ tile_items, int Ng, int T,
                                           int ntx, C2<R>* __restrict__ grid) {
  using Acc = typename ScratchOf<R, KAHAN>::T;
  const int S = T + kW - 1;
  const int cells = S * S;
  const int lt = __ffs(T) - 1;   // T is a power of two
  const int total = Ng * Ng;     // < 2^31 (Ng <= 32768)
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
    const int cv = k / Ng, cu = k - cv * Ng;
    const int tx = cu >> lt, ty = cv >> lt, ou = cu & (T - 1), ov = cv & (T - 1);
    Acc sum;
    sum.x = 0;
    sum.y = 0;
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      if (dy && ov >= kW - 1) break;
#pragma unroll
      for (int dx = 0; dx < 2; ++dx) {
        if (dx && ou >= kW - 1) break;
        int stx = tx - dx, sty = ty - dy;
        stx += stx < 0 ? ntx : 0;
        sty += sty < 0 ? ntx : 0;
        const int t = sty * ntx + stx;
        const int off = (ov + dy * T) * S + (ou + dx * T);
        const int e = tile_items[t + 1];
        int i = tile_items[t];
        for (; i + 4 <= e; i += 4) {
          Acc a[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) a[u] = scratch[(int64_t)(i + u) * cells + off];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            sum.x += a[u].x;
            sum.y += a[u].y;
          }
        }
        for (; i < e; ++i) {
          const Acc a = scratch[(int64_t)i * cells + off];
          sum.x += a.x;
          sum.y += a.y;
        }
      }
    }
    C2<R> o;
    o.x = (R)sum.x;
    o.y = (R)sum.y;
    grid[k] = o;
  }
}

// Every grid cell sums, in a fixed order, the scratch tiles of all work items
// of the (up to four) tiles whose footprint region covers it: its own tile
// and, within W - 1 cells of a tile edge, the tiles to the left and above
// (periodically).  Each cell is written once, so the grid needs no clearing.
template <typename R, bool KAHAN>
__global__ void fold_kernel(const typename ScratchOf<R, KAHAN>::T* __restrict__ scratch,
                            const int32_t* __restrict__ tile_items, int Ng, int T, int ntx,
                            C2<R>* __restrict__ grid) {
  fold_cells<R, KAHAN>(scratch, tile_items, Ng, T, ntx, grid);
}

// stacked form: blockIdx.y = job (its tiles start at its first item)
template <typename R, bool KAHAN>
__global__ void fold_batch_kernel(const BatchJob<R>* __restrict__ jobs,
                                  const typename ScratchOf<R, KAHAN>::T* __restrict__ scratch,
                                  int Ng, int T, int ntx) {
  const BatchJob<R> jb = jobs[blockIdx.y];
  const int S = T + kW - 1;
  fold_cells<R, KAHAN>(scratch + jb.item_base * (int64_t)(S * S), jb.tile_items, Ng, T, ntx,
                       jb.grid);
}

template <typename R, bool KAHAN>
void launch_fold(const void* scratch, const int32_t* tile_items, int Ng, int tile, int ntx,
                 C2<R>* grid, cudaStream_t s) {
  int64_t total = (int64_t)Ng * Ng;
  int blocks = (int)((total + kThreads - 1) / kThreads);
  if (blocks > sm_count() * 32) blocks = sm_count() * 32;
  fold_kernel<R, KAHAN><<<blocks, kThreads, 0, s>>>(
      reinterpret_cast<const typename ScratchOf<R, KAHAN>::T*>(scratch), tile_items, Ng, tile,
      ntx, grid);
}

// ---------------------------------------------------------------- instances
// ------------------------------------------------------------ batched form
// Every job's rows / cells are walked by blockIdx.x, x-stride; blockIdx.y = job.
template <typename R>
__global__ void job_of_kernel(const BatchJob<R>* __restrict__ jobs, int32_t* __restrict__ job_of) {
  const BatchJob<R> jb = jobs[blockIdx.y];
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < jb.nitems; i += gridDim.x * blockDim.x)
    job_of[jb.item_base + i] = (int32_t)blockIdx.y;
}

template <typename R>
__global__ void batch_gather_kernel(const BatchJob<R>* __restrict__ jobs) {
  const BatchJob<R> jb = jobs[blockIdx.y];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < jb.n;
       k += (int64_t)gridDim.x * blockDim.x)
    jb.sorted_in[k] = jb.user_in[jb.idx[k]];
}

template <typename R>
__global__ void batch_scatter_kernel(const BatchJob<R>* __restrict__ jobs) {
  const BatchJob<R> jb = jobs[blockIdx.y];
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < jb.n;
       k += (int64_t)gridDim.x * blockDim.x)
    jb.user_out[jb.idx[k]] = jb.sorted_out[k];
}

template <typename R>
__global__ void pad_batch_kernel(const BatchJob<R>* __restrict__ jobs, const R* __restrict__ psi,
                                 int npix, int Ng) {
  const BatchJob<R> jb = jobs[blockIdx.y];
  int64_t total = (int64_t)Ng * Ng;
  const int h = npix / 2;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int rr = (int)(k / Ng), cc = (int)(k % Ng);
    int a = cc < h ? cc : (cc >= Ng - h ? cc - Ng : INT32_MAX);
    int b = rr < h ? rr : (rr >= Ng - h ? rr - Ng : INT32_MAX);
    C2<R> o;
    o.x = (R)0;
    o.y = (R)0;
    if (a != INT32_MAX && b != INT32_MAX) {
      int q = a + h, p = b + h;
      R val = jb.image_in[(int64_t)p * npix + q] / (psi[p] * psi[q]);
      o.x = ((a + b) & 1) ? -val : val;
    }
    jb.grid[k] = o;
  }
}

template <typename R>
__global__ void crop_batch_kernel(const BatchJob<R>* __restrict__ jobs, const R* __restrict__ psi,
                                  int npix, int Ng) {
  const BatchJob<R> jb = jobs[blockIdx.y];
  const R scale = (R)jb.inv_n;
  int64_t total = (int64_t)npix * npix;
  const int h = npix / 2;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total;
       k += (int64_t)gridDim.x * blockDim.x) {
    int p = (int)(k / npix), q = (int)(k % npix);
    int a = q - h, b = p - h;
    int cc = a < 0 ? a + Ng : a;
    int rr = b < 0 ? b + Ng : b;
    R val = jb.grid[(int64_t)rr * Ng + cc].x * scale / (psi[p] * psi[q]);
    jb.image_out[k] = ((a + b) & 1) ? -val : val;
  }
}

namespace {
int blocks_for(int64_t n, int cap) {
  int64_t b = (n + kThreads - 1) / kThreads;
  if (b > cap) b = cap;
  return b < 1 ? 1 : (int)b;
}
}  // namespace

template <typename R>
void launch_job_of(const BatchJob<R>* jobs, int njobs, int max_items, int32_t* job_of,
                   cudaStream_t s) {
  job_of_kernel<R><<<dim3(blocks_for(max_items, sm_count()), njobs), kThreads, 0, s>>>(jobs, job_of);
}

template <typename R>
void launch_batch_gather(const BatchJob<R>* jobs, int njobs, int64_t max_n, cudaStream_t s) {
  batch_gather_kernel<R><<<dim3(blocks_for(max_n, sm_count() * 4), njobs), kThreads, 0, s>>>(jobs);
}

template <typename R>
void launch_batch_scatter(const BatchJob<R>* jobs, int njobs, int64_t max_n, cudaStream_t s) {
  batch_scatter_kernel<R><<<dim3(blocks_for(max_n, sm_count() * 4), njobs), kThreads, 0, s>>>(jobs);
}

template <typename R, bool KAHAN>
void launch_grid_batch(const BatchJob<R>* jobs, const int32_t* job_of, int total_items,
                       void* scratch, int tile, int ntx, double beta, cudaStream_t s) {
  if (total_items <= 0) return;
  const size_t smem = grid_smem_bytes<R, KAHAN>(tile);
  auto k = grid_batch_kernel<R, KAHAN>;
  cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k<<<total_items, grid_block_threads<R, KAHAN>(), smem, s>>>(
      jobs, job_of, reinterpret_cast<typename ScratchOf<R, KAHAN>::T*>(scratch), tile, ntx,
      (R)beta);
}

template <typename R, bool KAHAN>
void launch_fold_batch(const BatchJob<R>* jobs, int njobs, const void* scratch, int Ng,
                       int tile, int ntx, cudaStream_t s) {
  fold_batch_kernel<R, KAHAN><<<dim3(blocks_for((int64_t)Ng * Ng, sm_count() * 8), njobs), kThreads, 0,
                                s>>>(
      jobs, reinterpret_cast<const typename ScratchOf<R, KAHAN>::T*>(scratch), Ng, tile, ntx);
}

template <typename R>
void launch_degrid_batch(const CUtensorMap* tmap, const BatchJob<R>* jobs,
                         const int32_t* job_of, int total_items, bool has_obs, int Ng, int tile,
                         int ntx, double beta, int32_t* err, cudaStream_t s) {
  if (total_items <= 0) return;
  const int S = tile + kW - 1;
  size_t smem = (size_t)S * S * sizeof(C2<R>) + 128 + sizeof(uint64_t) + sizeof(int) + 4;
  if (has_obs) {
    auto k = degrid_batch_kernel<R, true>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<total_items, kThreads, smem, s>>>(*tmap, jobs, job_of, Ng, tile, ntx, (R)beta, err);
  } else {
    auto k = degrid_batch_kernel<R, false>;
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k<<<total_items, kThreads, smem, s>>>(*tmap, jobs, job_of, Ng, tile, ntx, (R)beta, err);
  }
}

template <typename R>
void launch_pad_batch(const BatchJob<R>* jobs, int njobs, const R* psi, int npix, int Ng,
                      cudaStream_t s) {
  pad_batch_kernel<R><<<dim3(blocks_for((int64_t)Ng * Ng, sm_count() * 8), njobs), kThreads, 0, s>>>(
      jobs, psi, npix, Ng);
}

template <typename R>
void launch_crop_batch(const BatchJob<R>* jobs, int njobs, const R* psi, int npix, int Ng,
                       cudaStream_t s) {
  crop_batch_kernel<R><<<dim3(blocks_for((int64_t)npix * npix, sm_count() * 8), njobs), kThreads, 0,
                         s>>>(jobs, psi, npix, Ng);
}

#define MS_BATCH_INST(R)                                                                         \
  template void launch_job_of<R>(const BatchJob<R>*, int, int, int32_t*, cudaStream_t);         \
  template void launch_batch_gather<R>(const BatchJob<R>*, int, int64_t, cudaStream_t);         \
  template void launch_batch_scatter<R>(const BatchJob<R>*, int, int64_t, cudaStream_t);        \
  template void launch_degrid_batch<R>(const CUtensorMap*, const BatchJob<R>*, const int32_t*,  \
                                       int, bool, int, int, int, double, int32_t*,             \
                                       cudaStream_t);                                           \
  template void launch_pad_batch<R>(const BatchJob<R>*, int, const R*, int, int, cudaStream_t); \
  template void launch_crop_batch<R>(const BatchJob<R>*, int, const R*, int, int, cudaStream_t);
MS_BATCH_INST(float)
MS_BATCH_INST(double)
#undef MS_BATCH_INST
template void launch_grid_batch<float, false>(const BatchJob<float>*, const int32_t*, int, void*,
                                              int, int, double, cudaStream_t);
template void launch_grid_batch<float, true>(const BatchJob<float>*, const int32_t*, int, void*,
                                             int, int, double, cudaStream_t);
template void launch_grid_batch<double, false>(const BatchJob<double>*, const int32_t*, int,
                                               void*, int, int, double, cudaStream_t);
template void launch_fold_batch<float, false>(const BatchJob<float>*, int, const void*, int, int,
                                              int, cudaStream_t);
template void launch_fold_batch<float, true>(const BatchJob<float>*, int, const void*, int, int,
                                             int, cudaStream_t);
template void launch_fold_batch<double, false>(const BatchJob<double>*, int, const void*, int,
                                               int, int, cudaStream_t);

template void launch_pad<float>(const float*, const float*, int, int, float2*, cudaStream_t);
template void launch_pad<double>(const double*, const double*, int, int, double2*,
                                 cudaStream_t);
template void launch_crop<float>(const float2*, const float*, int, int, double, float*,
                                 cudaStream_t);
template void launch_crop<double>(const double2*, const double*, int, int, double, double*,
                                  cudaStream_t);
template void launch_degrid<float>(const CUtensorMap*, const float2*, const WorkItem*, int,
                                   const uint32_t*, const float2*, const float2*, float2*, int,
                                   int, int, double, int32_t*, cudaStream_t);
template void launch_degrid<double>(const CUtensorMap*, const double2*, const WorkItem*, int,
                                    const uint32_t*, const double2*, const double2*, double2*,
                                    int, int, int, double, int32_t*, cudaStream_t);
template void launch_grid<float, false>(const WorkItem*, int, const uint32_t*, const float2*,
                                        const float2*, void*, int, int, int, double,
                                        cudaStream_t);
template void launch_grid<float, true>(const WorkItem*, int, const uint32_t*, const float2*,
                                       const float2*, void*, int, int, int, double,
                                       cudaStream_t);
template void launch_grid<double, false>(const WorkItem*, int, const uint32_t*, const double2*,
                                         const double2*, void*, int, int, int, double,
                                         cudaStream_t);
template void launch_fold<float, false>(const void*, const int32_t*, int, int, int, float2*,
                                        cudaStream_t);
template void launch_fold<float, true>(const void*, const int32_t*, int, int, int, float2*,
                                       cudaStream_t);
template void launch_fold<double, false>(const void*, const int32_t*, int, int, int, double2*,
                                         cudaStream_t);

}  // namespace ms
