// Plan-time kernels: classify rows into the baseline partitions (Sect. 3.1),
// place each row's ES footprint on the oversampled grid, sort each partition
// by grid tile (stable LSD radix sort), build work items, gather per-row
// geometry into sorted order, and tabulate the deapodization correction.
#include "common.cuh"

namespace ms {

namespace {
constexpr int kRadixBlock = 256;
constexpr int kRadixRounds = 16;
constexpr int kRadixChunk = kRadixBlock * kRadixRounds;   // rows per sort block

int grid_for(int64_t n, int block) {
  int64_t g = (n + block - 1) / block;
  const int64_t cap = (int64_t)sm_count() * 64;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}
}  // namespace

int sm_count() {
  constexpr int kDevices = 64;
  static int cache[kDevices] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevices) return 152;
  if (!cache[dev]) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 152;   // the attribute query cannot fail on a live device; GB300's count
    cache[dev] = n;
  }
  return cache[dev];
}

// Row k: grid coordinate g = u Ng dl (uv origin at 0), first footprint cell
// c0 = floor(g - W/2) + 1, centre offset f = (g - c0) - (W-1)/2 in (-0.5, 0.5].
// The centred grid stores frequency c at index (c + Ng/2) mod Ng.
__global__ void classify_kernel(const double* __restrict__ u, const double* __restrict__ v,
                                const uint8_t* __restrict__ flags, int64_t n, int Ng,
                                int npix, double dl, double ell, double delta, int tile,
                                int ntx, uint32_t* __restrict__ cell,
                                double2* __restrict__ frac, uint32_t* __restrict__ tile_id,
                                uint8_t* __restrict__ member) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    double uu = u[i], vv = v[i];
    double gu = (uu * (double)Ng) * dl;
    double gv = (vv * (double)Ng) * dl;
    double c0u = floor(gu - 0.5 * kW) + 1.0;
    double c0v = floor(gv - 0.5 * kW) + 1.0;
    frac[i] = make_double2((gu - c0u) - (double)kHalfW, (gv - c0v) - (double)kHalfW);
    long long iu = (long long)c0u + Ng / 2;
    long long iv = (long long)c0v + Ng / 2;
    iu %= Ng; if (iu < 0) iu += Ng;
    iv %= Ng; if (iv < 0) iv += Ng;
    cell[i] = (uint32_t)iu | ((uint32_t)iv << 16);
    tile_id[i] = (uint32_t)((iv / tile) * ntx + (iu / tile));
    double r = hypot(uu, vv) * (double)npix * dl;
    uint8_t m = 0;
    bool ok = flags == nullptr || flags[i] == 0;
    bool finite = isfinite(gu) && isfinite(gv);
    if (ok && finite) {
      m |= 4;
      if (r <= ell + delta) m |= 1;
      if (r >= ell - delta) m |= 2;
    }
    member[i] = m;
  }
}

void launch_classify(const double* u, const double* v, const uint8_t* flags, int64_t n,
                     int Ng, int npix, double dl, double ell, double delta, int tile,
                     int ntx, uint32_t* cell, double2* frac, uint32_t* tile_id,
                     uint8_t* member, cudaStream_t s) {
  classify_kernel<<<grid_for(n, 256), 256, 0, s>>>(u, v, flags, n, Ng, npix, dl, ell, delta,
                                                    tile, ntx, cell, frac, tile_id, member);
}

// Sort key of a row: its tile, then its anchor cell inside the tile (row v,
// then column u), so that rows sharing an anchor are adjacent in plan order;
// rows outside the partition get the sentinel (after every tile).
__global__ void make_keys_kernel(const uint32_t* __restrict__ tile_id,
                                 const uint32_t* __restrict__ cell,
                                 const uint8_t* __restrict__ member, int64_t n, uint8_t mask,
                                 int log2_tile, uint32_t sentinel, uint32_t* __restrict__ keys,
                                 int32_t* __restrict__ vals) {
  const uint32_t tmask = (1u << log2_tile) - 1u;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = cell[i];
    const uint32_t lu = (c & 0xffffu) & tmask, lv = (c >> 16) & tmask;
    keys[i] = (member[i] & mask) == mask
                  ? (tile_id[i] << (2 * log2_tile)) | (lv << log2_tile) | lu
                  : sentinel;
    vals[i] = (int32_t)i;
  }
}

void launch_make_keys(const uint32_t* tile_id, const uint32_t* cell, const uint8_t* member,
                      int64_t n, uint8_t mask, int log2_tile, uint32_t sentinel, uint32_t* keys,
                      int32_t* vals, cudaStream_t s) {
  make_keys_kernel<<<grid_for(n, 256), 256, 0, s>>>(tile_id, cell, member, n, mask, log2_tile,
                                                     sentinel, keys, vals);
}

// ---------------------------------------------------------------- radix sort
__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                  int32_t* __restrict__ hist, int nblocks) {
  __shared__ int32_t cnt[256];
  cnt[threadIdx.x] = 0;
  __syncthreads();
  int64_t lo = (int64_t)blockIdx.x * kRadixChunk;
  int64_t hi = lo + kRadixChunk < n ? lo + kRadixChunk : n;
  for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
    atomicAdd(&cnt[(keys[i] >> shift) & 255u], 1);
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

// Stable scatter: a block walks its chunk in order, 256 rows per round; inside
// a round, rows of equal digit keep their order through warp match masks and
// per-warp prefix counts.
__global__ void radix_scatter_kernel(const uint32_t* __restrict__ kin,
                                     const int32_t* __restrict__ vin, int64_t n, int shift,
                                     const int32_t* __restrict__ offs, int nblocks,
                                     uint32_t* __restrict__ kout, int32_t* __restrict__ vout) {
  __shared__ int32_t base[256];
  __shared__ int32_t wcnt[kRadixBlock / 32][256];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  base[tid] = offs[(int64_t)tid * nblocks + blockIdx.x];
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int r = 0; r < kRadixRounds; ++r) {
    int64_t i = (int64_t)blockIdx.x * kRadixChunk + (int64_t)r * kRadixBlock + tid;
    bool valid = i < n;
    uint32_t key = valid ? kin[i] : 0u;
    int digit = valid ? (int)((key >> shift) & 255u) : 256;
#pragma unroll
    for (int w = 0; w < kRadixBlock / 32; ++w) wcnt[w][tid] = 0;
    __syncthreads();
    unsigned peers = __match_any_sync(0xffffffffu, digit);
    int rank = __popc(peers & lt_mask);
    if (valid && lane == __ffs(peers) - 1) wcnt[warp][digit] = __popc(peers);
    __syncthreads();
    int run = 0;
#pragma unroll
    for (int w = 0; w < kRadixBlock / 32; ++w) {
      int c = wcnt[w][tid];
      wcnt[w][tid] = run;
      run += c;
    }
    __syncthreads();
    if (valid) {
      int pos = base[digit] + wcnt[warp][digit] + rank;
      kout[pos] = key;
      vout[pos] = vin[i];
    }
    __syncthreads();
    base[tid] += run;
    __syncthreads();
  }
}

// Single-block exclusive scan, out has n + 1 entries (out[n] = total).
__global__ void scan_single_block_kernel(const int32_t* __restrict__ in,
                                         int32_t* __restrict__ out, int n) {
  __shared__ int32_t sums[1024];
  const int tid = threadIdx.x;
  int seg = (n + 1023) / 1024;
  int lo = tid * seg;
  int hi = lo + seg < n ? lo + seg : n;
  int s = 0;
  for (int i = lo; i < hi; ++i) s += in[i];
  sums[tid] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int t = tid >= off ? sums[tid - off] : 0;
    __syncthreads();
    sums[tid] += t;
    __syncthreads();
  }
  int run = sums[tid] - s;
  for (int i = lo; i < hi; ++i) {
    out[i] = run;
    run += in[i];
  }
  if (tid == 1023) out[n] = sums[1023];
}

void launch_exclusive_scan(const int32_t* in, int32_t* out, int n, cudaStream_t s) {
  scan_single_block_kernel<<<1, 1024, 0, s>>>(in, out, n);
}

int64_t radix_hist_size(int64_t n) {
  int64_t nb = (n + kRadixChunk - 1) / kRadixChunk;
  if (nb < 1) nb = 1;
  return 2 * (nb * 256 + 1);   // histogram + its scan
}

void radix_sort(uint32_t** keys, int32_t** vals, uint32_t* ktmp, int32_t* vtmp, int64_t n,
                int bits, int32_t* hist, int64_t hist_cap, cudaStream_t s) {
  int nblocks = (int)((n + kRadixChunk - 1) / kRadixChunk);
  if (nblocks < 1) return;
  (void)hist_cap;
  int32_t* offs = hist + (int64_t)nblocks * 256 + 1;   // second half of the buffer
  uint32_t* ka = *keys;
  int32_t* va = *vals;
  uint32_t* kb = ktmp;
  int32_t* vb = vtmp;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist_kernel<<<nblocks, 256, 0, s>>>(ka, n, shift, hist, nblocks);
    scan_single_block_kernel<<<1, 1024, 0, s>>>(hist, offs, nblocks * 256);
    radix_scatter_kernel<<<nblocks, kRadixBlock, 0, s>>>(ka, va, n, shift, offs, nblocks, kb,
                                                         vb);
    uint32_t* tk = ka; ka = kb; kb = tk;
    int32_t* tv = va; va = vb; vb = tv;
  }
  *keys = ka;
  *vals = va;
}

__global__ void count_tiles_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                   int32_t* __restrict__ counts) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&counts[keys[i] >> shift], 1);
}

void launch_count_tiles(const uint32_t* keys, int64_t n, int shift, int32_t* counts,
                        cudaStream_t s) {
  if (n > 0) count_tiles_kernel<<<grid_for(n, 256), 256, 0, s>>>(keys, n, shift, counts);
}

__global__ void chunks_kernel(const int32_t* __restrict__ counts, int ntiles, int chunk,
                              int32_t* __restrict__ nchunks) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < ntiles) nchunks[t] = (counts[t] + chunk - 1) / chunk;
}

void launch_chunks_per_tile(const int32_t* counts, int ntiles, int chunk, int32_t* nchunks,
                            cudaStream_t s) {
  chunks_kernel<<<(ntiles + 255) / 256, 256, 0, s>>>(counts, ntiles, chunk, nchunks);
}

__global__ void make_items_kernel(const int32_t* __restrict__ counts,
                                  const int32_t* __restrict__ tile_start,
                                  const int32_t* __restrict__ item_start, int ntiles, int chunk,
                                  WorkItem* __restrict__ items) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntiles) return;
  int c = counts[t];
  int it = item_start[t];
  for (int off = 0; off < c; off += chunk, ++it) {
    WorkItem w;
    w.tile = t;
    w.start = tile_start[t] + off;
    w.count = c - off < chunk ? c - off : chunk;
    w.pad = 0;
    items[it] = w;
  }
}

void launch_make_items(const int32_t* counts, const int32_t* tile_start,
                       const int32_t* item_start, int ntiles, int chunk, WorkItem* items,
                       cudaStream_t s) {
  make_items_kernel<<<(ntiles + 255) / 256, 256, 0, s>>>(counts, tile_start, item_start, ntiles,
                                                          chunk, items);
}

template <typename R>
__global__ void gather_geometry_kernel(const int32_t* __restrict__ idx, int64_t n,
                                       const uint32_t* __restrict__ cell_all,
                                       const double2* __restrict__ frac_all,
                                       uint32_t* __restrict__ cell, C2<R>* __restrict__ frac) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = idx[k];
    cell[k] = cell_all[r];
    double2 f = frac_all[r];
    C2<R> o;
    o.x = (R)f.x;
    o.y = (R)f.y;
    frac[k] = o;
  }
}

template <typename R>
void launch_gather_geometry(const int32_t* idx, int64_t n, const uint32_t* cell_all,
                            const double2* frac_all, uint32_t* cell, C2<R>* frac,
                            cudaStream_t s) {
  if (n > 0)
    gather_geometry_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(idx, n, cell_all, frac_all,
                                                               cell, frac);
}

template <typename R>
__global__ void gather_vis_kernel(const int32_t* __restrict__ idx, int64_t n,
                                  const C2<R>* __restrict__ src, C2<R>* __restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[k] = src[idx[k]];
}

template <typename R>
__global__ void scatter_vis_kernel(const int32_t* __restrict__ idx, int64_t n,
                                   const C2<R>* __restrict__ src, C2<R>* __restrict__ dst) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x)
    dst[idx[k]] = src[k];
}

template <typename R>
void launch_gather_vis(const int32_t* idx, int64_t n, const C2<R>* src, C2<R>* dst,
                       cudaStream_t s) {
  if (n > 0) gather_vis_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(idx, n, src, dst);
}

template <typename R>
void launch_scatter_vis(const int32_t* idx, int64_t n, const C2<R>* src, C2<R>* dst,
                        cudaStream_t s) {
  if (n > 0) scatter_vis_kernel<R><<<grid_for(n, 256), 256, 0, s>>>(idx, n, src, dst);
}

// psi(a) = int phi(t) cos(2 pi a t / Ng) dt over |t| <= W/2.  With
// t = (W/2) sin(theta) the ES kernel becomes exp(beta (cos theta - 1)) and the
// integrand is smooth, so Gauss-Legendre in theta converges fast.
__global__ void deapod_kernel(int npix, int ngrid, double beta, const double* __restrict__ x,
                              const double* __restrict__ w, int nq, double* __restrict__ psi) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npix) return;
  const double half = 0.5 * kW;
  const double pi = 3.141592653589793238462643383279502884;
  double a = (double)(p - npix / 2);
  double acc = 0.0;
  for (int q = 0; q < nq; ++q) {
    double th = 0.5 * pi * x[q];
    double st, ct;
    sincos(th, &st, &ct);
    double t = half * st;
    acc += (0.5 * pi * w[q]) * half * ct * exp(beta * (ct - 1.0)) *
           cos(2.0 * pi * a * t / (double)ngrid);
  }
  psi[p] = acc;
}

void launch_deapodization(int npix, int ngrid, double beta, const double* nodes,
                          const double* weights, int nq, double* psi, cudaStream_t s) {
  deapod_kernel<<<(npix + 127) / 128, 128, 0, s>>>(npix, ngrid, beta, nodes, weights, nq, psi);
}

template void launch_gather_geometry<float>(const int32_t*, int64_t, const uint32_t*,
                                            const double2*, uint32_t*, float2*, cudaStream_t);
template void launch_gather_geometry<double>(const int32_t*, int64_t, const uint32_t*,
                                             const double2*, uint32_t*, double2*, cudaStream_t);
template void launch_gather_vis<float>(const int32_t*, int64_t, const float2*, float2*,
                                       cudaStream_t);
template void launch_gather_vis<double>(const int32_t*, int64_t, const double2*, double2*,
                                        cudaStream_t);
template void launch_scatter_vis<float>(const int32_t*, int64_t, const float2*, float2*,
                                        cudaStream_t);
template void launch_scatter_vis<double>(const int32_t*, int64_t, const double2*, double2*,
                                         cudaStream_t);

}  // namespace ms
