// lgs_bin.cu -- preprocess, angular-tile binning, radix sorts and tile ranges.
//
// Pipeline of one lgs_bin_sort (all on the caller's stream, no host sync):
//   k_tables      per frame: binary32 sine / direction tables of the tile
//                 rows and columns (pixel-centre extremes of each tile)
//   k_preprocess  per (frame, surfel) item: 64 B compositing record, depth
//                 key = bits of binary32 |mu_sensor|, tile count
//   depth sort    stable LSD radix sort of (key, item) over the items that
//                 cover at least one tile (4 passes of 8 bits; the first pass
//                 also compacts)
//   scan + emit   exclusive scan of tile counts in depth order, then each item
//                 writes (global tile id, item) pairs at its offset
//   tile sort     stable LSD radix sort of the pairs by tile id
//                 (ceil(log2 tiles / 8) passes)
//   k_ranges      [start, end) of every tile's run
// The result is the LSD sort of the 64-bit key (tile << 32 | depth) with ties
// broken by item index: the depth digits are sorted once per item instead of
// once per pair, because every pair of an item shares the item's depth key.
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {

// ---------------------------------------------------------------------------
// Descriptors and tables
// ---------------------------------------------------------------------------
__global__ void k_write_desc(const __grid_constant__ Desc h, Desc* __restrict__ d) {
  const int nw = static_cast<int>(sizeof(Desc) / 4);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(&h);
  uint32_t* dst = reinterpret_cast<uint32_t*>(d);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nw; i += gridDim.x * blockDim.x) dst[i] = src[i];
}

cudaError_t launch_write_desc(const Desc& h, Desc* d, Status*, cudaStream_t s) {
  k_write_desc<<<4, 256, 0, s>>>(h, d);
  return cudaGetLastError();
}

__global__ void k_tables(const Desc* __restrict__ D, float* __restrict__ tab, Status* __restrict__ st) {
  const FrameDev& F = D->f[blockIdx.x];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->required_pairs = 0;
    st->n_pairs = 0;
    st->n_vis = 0;
    st->overflow = 0;
    st->timeout = 0;
    st->check = 0;
    st->work_counter = 0;
    st->work_counter2 = 0;
    st->evals_fwd = 0;
    st->evals_bwd = 0;
    st->contrib_fwd = 0;
    st->contrib_bwd = 0;
  }
  for (int i = threadIdx.x; i < F.ntr; i += blockDim.x) {
    const int r0 = i * F.th;
    const int r1 = ((i + 1) * F.th < F.H ? (i + 1) * F.th : F.H) - 1;
    tab[F.row_tab + 2 * i] = bin_sin(bin_row_elev(r0, F.H, F.emin, F.emax));
    tab[F.row_tab + 2 * i + 1] = bin_sin(bin_row_elev(r1, F.H, F.emin, F.emax));
  }
  for (int j = threadIdx.x; j < F.ntc; j += blockDim.x) {
    const int c0 = j * F.tw;
    const int c1 = ((j + 1) * F.tw < F.W ? (j + 1) * F.tw : F.W) - 1;
    float cs, sn;
    bin_col_dir(c0, F.W, cs, sn);
    tab[F.col_tab + 4 * j] = cs;
    tab[F.col_tab + 4 * j + 1] = sn;
    bin_col_dir(c1, F.W, cs, sn);
    tab[F.col_tab + 4 * j + 2] = cs;
    tab[F.col_tab + 4 * j + 3] = sn;
  }
}

// Number of tiles the item covers (rows x columns), using the tables.
__device__ __forceinline__ uint32_t count_tiles(const BinGeom& g, const FrameDev& F, const float* __restrict__ tab) {
  int nr = 0;
  for (int i = 0; i < F.ntr; ++i) nr += bin_row_hit(g, tab[F.row_tab + 2 * i], tab[F.row_tab + 2 * i + 1]);
  if (nr == 0) return 0;
  const float4* ct = reinterpret_cast<const float4*>(tab + F.col_tab);
  ColWin w;
  bin_col_window(g, F, w);
  int nc = 0;
  for (int j = w.a0; j <= w.a1; ++j) nc += bin_col_hit(g, ct[j]);
  for (int j = w.b0; j <= w.b1; ++j) nc += bin_col_hit(g, ct[j]);
  return static_cast<uint32_t>(nr * nc);
}

// ---------------------------------------------------------------------------
// Preprocess: record + key + count per (frame, surfel) item
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_preprocess(const Desc* __restrict__ D, const float* __restrict__ tab,
                                                     float4* __restrict__ rec, float4* __restrict__ box,
                                                     uint32_t* __restrict__ key, uint32_t* __restrict__ cnt) {
  const int64_t item = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (item >= D->n_items) return;
  const int f = frame_of_item(*D, item);
  const FrameDev& F = D->f[f];
  const MapDev& M = D->m[F.map];
  const int64_t i = item - F.item_base;
  BinGeom g;
  bin_geom(M.mean + 3 * i, M.ls + 2 * i, F, g);
  key[item] = __float_as_uint(g.r);
  cnt[item] = count_tiles(g, F, tab);
  box[item] = pixel_box(g, F);

  // compositing record (accuracy only): rotation of the unit quaternion,
  // axes to the sensor frame, activations
  const float4 q = reinterpret_cast<const float4*>(M.quat)[i];
  const float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w);
  const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  // world-frame columns of R(q)
  const float c0x = 1.f - 2.f * (y * y + z * z), c0y = 2.f * (x * y + w * z), c0z = 2.f * (x * z - w * y);
  const float c1x = 2.f * (x * y - w * z), c1y = 1.f - 2.f * (x * x + z * z), c1z = 2.f * (y * z + w * x);
  const float c2x = 2.f * (x * z + w * y), c2y = 2.f * (y * z - w * x), c2z = 1.f - 2.f * (x * x + y * y);
  const float* R = F.R;
  // sensor frame: v_s = R^T v_w
  const float tux = R[0] * c0x + R[3] * c0y + R[6] * c0z, tuy = R[1] * c0x + R[4] * c0y + R[7] * c0z,
              tuz = R[2] * c0x + R[5] * c0y + R[8] * c0z;
  const float tvx = R[0] * c1x + R[3] * c1y + R[6] * c1z, tvy = R[1] * c1x + R[4] * c1y + R[7] * c1z,
              tvz = R[2] * c1x + R[5] * c1y + R[8] * c1z;
  const float nx = R[0] * c2x + R[3] * c2y + R[6] * c2z, ny = R[1] * c2x + R[4] * c2y + R[7] * c2z,
              nz = R[2] * c2x + R[5] * c2y + R[8] * c2z;
  const float isu = expf(-M.ls[2 * i]), isv = expf(-M.ls[2 * i + 1]);
  const float alpha = 1.0f / (1.0f + expf(-M.logit[i]));
  const float mx = g.x, my = g.y, mz = g.z;
  float4* out = rec + 4 * item;
  out[0] = make_float4(nx, ny, nz, nx * mx + ny * my + nz * mz);
  out[1] = make_float4(tux * isu, tuy * isu, tuz * isu, (tux * mx + tuy * my + tuz * mz) * isu);
  out[2] = make_float4(tvx * isv, tvy * isv, tvz * isv, (tvx * mx + tvy * my + tvz * mz) * isv);
  out[3] = make_float4(alpha, expf(M.ls[2 * i]), expf(M.ls[2 * i + 1]), 0.f);
}

// ---------------------------------------------------------------------------
// Stable LSD radix pass on (u32 key, u32 value), 8-bit digit at `shift`.
// Three kernels: per-CTA digit histograms, per-digit scan over CTAs, and a
// scatter that ranks stably inside the CTA (warp match + per-warp digit
// counts), reorders the chunk in shared memory and writes each digit's run
// contiguously.  MODE 0: keys/values from the ping-pong arrays, count from
// *n_dev.  MODE 1 (first depth pass): key = key[i], value = i, and items with
// cnt[i] == 0 are dropped (compaction), count = n_static.
// ---------------------------------------------------------------------------
struct PassIn {
  const uint32_t* k;
  const uint32_t* v;
  const uint32_t* cnt;       // MODE 1 only
  const unsigned long long* n64;   // MODE 0: count from a 64-bit status word
  const unsigned int* n32;   // MODE 0: count from a 32-bit status word
  int64_t n_static;
};

template <int MODE>
__device__ __forceinline__ int64_t pass_n(const PassIn& in) {
  if (MODE == 1) return in.n_static;
  if (in.n64) return static_cast<int64_t>(*in.n64);
  return static_cast<int64_t>(*in.n32);
}

template <int MODE>
__device__ __forceinline__ bool pass_load(const PassIn& in, int64_t idx, int64_t n, uint32_t& k, uint32_t& v) {
  if (idx >= n) return false;
  if (MODE == 1) {
    if (in.cnt[idx] == 0) return false;
    k = in.k[idx];
    v = static_cast<uint32_t>(idx);
    return true;
  }
  k = in.k[idx];
  v = in.v[idx];
  return true;
}

template <int MODE>
__global__ void __launch_bounds__(kSortThreads) k_radix_hist(PassIn in, int shift, uint32_t* __restrict__ hist,
                                                               uint32_t* __restrict__ dtot, int G) {
  __shared__ uint32_t s_h[256];
  const int tid = threadIdx.x;
  s_h[tid] = 0;
  __syncthreads();
  const int64_t n = pass_n<MODE>(in);
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortChunk;
  if (base < n) {
#pragma unroll 4
    for (int j = 0; j < kSortItems; ++j) {
      uint32_t k, v;
      if (pass_load<MODE>(in, base + j * kSortThreads + tid, n, k, v)) atomicAdd(&s_h[(k >> shift) & 255u], 1u);
    }
  }
  __syncthreads();
  const uint32_t c = s_h[tid];
  hist[static_cast<int64_t>(tid) * G + blockIdx.x] = c;
  if (c) atomicAdd(&dtot[tid], c);
}

// CTA d scans digit d's counts over all CTAs: offset = (sum of the totals of
// smaller digits) + (counts of digit d in earlier CTAs).  The last CTA also
// publishes the number of keys of the pass when n_out != nullptr.
__global__ void __launch_bounds__(256) k_radix_digit_scan(uint32_t* __restrict__ hist,
                                                           const uint32_t* __restrict__ dtot, int G,
                                                           unsigned int* __restrict__ n_out) {
  __shared__ uint32_t s_w[8];
  __shared__ uint32_t s_carry;
  const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // base = sum_{d' < d} dtot[d']
  uint32_t v = (tid < d) ? dtot[tid] : 0u;
  uint32_t all = dtot[tid];
  for (int o = 16; o > 0; o >>= 1) {
    v += __shfl_xor_sync(0xffffffffu, v, o);
    all += __shfl_xor_sync(0xffffffffu, all, o);
  }
  if (lane == 0) s_w[wid] = v;
  __syncthreads();
  uint32_t base = 0;
  for (int i = 0; i < 8; ++i) base += s_w[i];
  __syncthreads();
  if (n_out && d == 255) {
    if (lane == 0) s_w[wid] = all;
    __syncthreads();
    if (tid == 0) {
      uint32_t t = 0;
      for (int i = 0; i < 8; ++i) t += s_w[i];
      *n_out = t;
    }
    __syncthreads();
  }
  if (tid == 0) s_carry = base;
  __syncthreads();
  uint32_t* row = hist + static_cast<int64_t>(d) * G;
  for (int b0 = 0; b0 < G; b0 += 256) {
    const int b = b0 + tid;
    const uint32_t x = b < G ? row[b] : 0u;
    // inclusive block scan
    uint32_t s = x;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane == 31) s_w[wid] = s;
    __syncthreads();
    uint32_t wpre = 0;
    for (int i = 0; i < wid; ++i) wpre += s_w[i];
    uint32_t tot = 0;
    for (int i = 0; i < 8; ++i) tot += s_w[i];
    const uint32_t carry = s_carry;
    if (b < G) row[b] = carry + wpre + s - x;
    __syncthreads();
    if (tid == 0) s_carry = carry + tot;
    __syncthreads();
  }
}

template <int MODE>
__global__ void __launch_bounds__(kSortThreads) k_radix_scatter(PassIn in, int shift, const uint32_t* __restrict__ offs,
                                                                  int G, uint32_t* __restrict__ ko,
                                                                  uint32_t* __restrict__ vo) {
  __shared__ uint32_t s_k[kSortChunk];
  __shared__ uint32_t s_v[kSortChunk];
  __shared__ uint32_t s_wc[8][256];
  __shared__ uint32_t s_run[256];
  __shared__ uint32_t s_loc[256];
  __shared__ uint32_t s_glob[256];
  __shared__ uint32_t s_ws[8];
  const int64_t n = pass_n<MODE>(in);
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortChunk;
  if (base >= n) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const uint32_t lt_mask = (1u << lane) - 1u;
  s_run[tid] = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) s_wc[w][tid] = 0;
  s_glob[tid] = offs[static_cast<int64_t>(tid) * G + blockIdx.x];
  __syncthreads();
  uint32_t mk[kSortItems], mv[kSortItems], mr[kSortItems];
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    uint32_t k = 0, v = 0;
    const bool ok = pass_load<MODE>(in, base + j * kSortThreads + tid, n, k, v);
    const uint32_t d = ok ? ((k >> shift) & 255u) : (256u + lane);
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t lr = __popc(peers & lt_mask);
    if (ok && lane == __ffs(peers) - 1) s_wc[wid][d] = __popc(peers);
    __syncthreads();
    uint32_t r = 0xffffffffu;
    if (ok) {
      r = s_run[d] + lr;
      for (int w = 0; w < wid; ++w) r += s_wc[w][d];
    }
    __syncthreads();
    uint32_t t = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      t += s_wc[w][tid];
      s_wc[w][tid] = 0;
    }
    s_run[tid] += t;
    __syncthreads();
    mk[j] = k;
    mv[j] = v;
    mr[j] = r;
  }
  // exclusive scan of the CTA's digit histogram -> local offsets
  {
    const uint32_t x = s_run[tid];
    uint32_t s = x;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane == 31) s_ws[wid] = s;
    __syncthreads();
    uint32_t wpre = 0;
    for (int i = 0; i < wid; ++i) wpre += s_ws[i];
    s_loc[tid] = wpre + s - x;
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < kSortItems; ++j) {
    if (mr[j] != 0xffffffffu) {
      const uint32_t p = s_loc[(mk[j] >> shift) & 255u] + mr[j];
      s_k[p] = mk[j];
      s_v[p] = mv[j];
    }
  }
  __syncthreads();
  const uint32_t total = s_loc[255] + s_run[255];
  for (uint32_t p = tid; p < total; p += kSortThreads) {
    const uint32_t k = s_k[p];
    const uint32_t d = (k >> shift) & 255u;
    const uint32_t g = s_glob[d] + (p - s_loc[d]);
    ko[g] = k;
    vo[g] = s_v[p];
  }
}

template <int MODE>
static cudaError_t radix_pass(const PassIn& in, int shift, uint32_t* hist, uint32_t* dtot, int G, unsigned int* n_out,
                              uint32_t* ko, uint32_t* vo, cudaStream_t s) {
  k_radix_hist<MODE><<<G, kSortThreads, 0, s>>>(in, shift, hist, dtot, G);
  k_radix_digit_scan<<<256, 256, 0, s>>>(hist, dtot, G, n_out);
  k_radix_scatter<MODE><<<G, kSortThreads, 0, s>>>(in, shift, hist, G, ko, vo);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Scan of tile counts in depth order + pair emission
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t* __restrict__ sorted_item,
                                                               const uint32_t* __restrict__ cnt,
                                                               const Status* __restrict__ st,
                                                               unsigned long long* __restrict__ bsum) {
  __shared__ unsigned long long s_w[8];
  const int64_t n = st->n_vis;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanChunk;
  unsigned long long acc = 0;
  if (base < n) {
    for (int j = 0; j < kScanItems; ++j) {
      const int64_t i = base + j * kScanThreads + threadIdx.x;
      if (i < n) acc += cnt[sorted_item[i]];
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long t = 0;
    for (int i = 0; i < 8; ++i) t += s_w[i];
    bsum[blockIdx.x] = t;
  }
}

// single CTA: exclusive scan of the block sums; publishes the pair count and
// the overflow flag
__global__ void __launch_bounds__(1024) k_scan_top(unsigned long long* __restrict__ bsum, int nb,
                                                   Status* __restrict__ st, int64_t cap) {
  __shared__ unsigned long long s_w[32];
  __shared__ unsigned long long s_carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_carry = 0;
  __syncthreads();
  for (int b0 = 0; b0 < nb; b0 += 1024) {
    const int b = b0 + tid;
    const unsigned long long x = b < nb ? bsum[b] : 0ull;
    unsigned long long s = x;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane == 31) s_w[wid] = s;
    __syncthreads();
    unsigned long long wpre = 0, tot = 0;
    for (int i = 0; i < 32; ++i) {
      if (i < wid) wpre += s_w[i];
      tot += s_w[i];
    }
    const unsigned long long carry = s_carry;
    if (b < nb) bsum[b] = carry + wpre + s - x;
    __syncthreads();
    if (tid == 0) s_carry = carry + tot;
    __syncthreads();
  }
  if (tid == 0) {
    const unsigned long long total = s_carry;
    st->required_pairs = total;
    const bool over = total > static_cast<unsigned long long>(cap);
    st->overflow = over ? 1u : 0u;
    st->n_pairs = over ? 0ull : total;
  }
}

__global__ void __launch_bounds__(kScanThreads) k_scan_emit(const Desc* __restrict__ D, const float* __restrict__ tab,
                                                             const uint32_t* __restrict__ sorted_item,
                                                             const uint32_t* __restrict__ cnt,
                                                             const unsigned long long* __restrict__ bsum,
                                                             Status* __restrict__ st,
                                                             uint32_t* __restrict__ pk, uint32_t* __restrict__ pv) {
  __shared__ uint32_t s_w[8];
  const int64_t n = st->n_vis;
  if (st->overflow) return;
  const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanChunk;
  if (base >= n) return;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  // each thread takes kScanItems consecutive sorted items
  const int64_t i0 = base + static_cast<int64_t>(tid) * kScanItems;
  uint32_t c[kScanItems];
  uint32_t it[kScanItems];
  uint32_t tsum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const int64_t i = i0 + j;
    it[j] = i < n ? sorted_item[i] : 0u;
    c[j] = i < n ? cnt[it[j]] : 0u;
    tsum += c[j];
  }
  uint32_t s = tsum;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
    if (lane >= o) s += y;
  }
  if (lane == 31) s_w[wid] = s;
  __syncthreads();
  uint32_t wpre = 0;
  for (int i = 0; i < wid; ++i) wpre += s_w[i];
  unsigned long long off = bsum[blockIdx.x] + wpre + s - tsum;
#pragma unroll 1
  for (int j = 0; j < kScanItems; ++j) {
    if (i0 + j >= n || c[j] == 0) continue;
    const int64_t item = it[j];
    const int f = frame_of_item(*D, item);
    const FrameDev& F = D->f[f];
    const MapDev& M = D->m[F.map];
    const int64_t i = item - F.item_base;
    BinGeom g;
    bin_geom(M.mean + 3 * i, M.ls + 2 * i, F, g);
    const float4* ct = reinterpret_cast<const float4*>(tab + F.col_tab);
    ColWin w;
    bin_col_window(g, F, w);
    uint32_t left = c[j];
    for (int r = 0; r < F.ntr && left; ++r) {
      if (!bin_row_hit(g, tab[F.row_tab + 2 * r], tab[F.row_tab + 2 * r + 1])) continue;
      const uint32_t rowbase = F.tile_base + static_cast<uint32_t>(r * F.ntc);
      for (int pass = 0; pass < 2; ++pass) {
        const int ja = pass ? w.b0 : w.a0, jb = pass ? w.b1 : w.a1;
        for (int jc = ja; jc <= jb && left; ++jc) {
          if (!bin_col_hit(g, ct[jc])) continue;
          pk[off] = rowbase + static_cast<uint32_t>(jc);
          pv[off] = static_cast<uint32_t>(item);
          ++off;
          --left;
        }
      }
    }
    // The emission repeats the counting pass exactly, so nothing is left; if
    // it ever were, fill the reserved slots with an out-of-range tile (sorted
    // last, ignored by the ranges) and record a device check failure.
    for (; left; --left, ++off) {
      pk[off] = 0xffffffffu;
      pv[off] = 0u;
      st->check = 1u;
    }
  }
}

__global__ void k_ranges(const uint32_t* __restrict__ pk, const Status* __restrict__ st, uint32_t n_tiles,
                         uint2* __restrict__ ranges) {
  const int64_t n = static_cast<int64_t>(st->n_pairs);
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const uint32_t t = pk[i];
    if (t >= n_tiles) continue;
    if (i == 0 || pk[i - 1] != t) ranges[t].x = static_cast<uint32_t>(i);
    if (i == n - 1 || pk[i + 1] != t) ranges[t].y = static_cast<uint32_t>(i + 1);
  }
}

// ---------------------------------------------------------------------------
// Orchestration
// ---------------------------------------------------------------------------
static int tile_passes(uint32_t n_tiles) {
  int bits = 0;
  while (bits < 32 && (1ull << bits) < n_tiles) ++bits;
  const int p = (bits + 7) / 8;
  return p < 1 ? 1 : p;
}

int pair_sort_result_in_b(uint32_t n_tiles) { return tile_passes(n_tiles) & 1; }

// kernels launch_bin enqueues (memsets not counted)
int bin_kernel_count(uint32_t n_tiles) { return 2 + 3 * 4 + 3 + 3 * tile_passes(n_tiles) + 1; }

cudaError_t launch_bin(const Layout& L, const WsPtrs& w, int n_frames, int64_t n_items, uint32_t n_tiles,
                       cudaStream_t s) {
  cudaError_t e;
  e = cudaMemsetAsync(w.dtot, 0, sizeof(uint32_t) * 256 * 8, s);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(w.ranges, 0, sizeof(uint2) * n_tiles, s);
  if (e != cudaSuccess) return e;
  k_tables<<<n_frames, 256, 0, s>>>(w.desc, w.tables, w.st);
  const int64_t ni = n_items > 0 ? n_items : 1;
  k_preprocess<<<static_cast<unsigned>((ni + 255) / 256), 256, 0, s>>>(w.desc, w.tables, w.rec, w.box, w.key,
                                                                       w.cnt);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  // depth sort of the visible items (first pass compacts)
  const int Gi = static_cast<int>((ni + kSortChunk - 1) / kSortChunk);
  {
    PassIn p{w.key, nullptr, w.cnt, nullptr, nullptr, n_items};
    if ((e = radix_pass<1>(p, 0, w.hist, w.dtot, Gi, &w.st->n_vis, w.sk_a, w.sv_a, s)) != cudaSuccess) return e;
  }
  uint32_t *ka = w.sk_a, *va = w.sv_a, *kb = w.sk_b, *vb = w.sv_b;
  for (int pass = 1; pass < 4; ++pass) {
    PassIn p{ka, va, nullptr, nullptr, &w.st->n_vis, 0};
    if ((e = radix_pass<0>(p, 8 * pass, w.hist, w.dtot + 256 * pass, Gi, nullptr, kb, vb, s)) != cudaSuccess)
      return e;
    uint32_t* t;
    t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
  }
  const uint32_t* sorted_items = va;   // after 4 passes: the B buffers

  // scan of tile counts in depth order, then emission of the pairs
  const int nb = static_cast<int>((ni + kScanChunk - 1) / kScanChunk);
  k_scan_reduce<<<nb, kScanThreads, 0, s>>>(sorted_items, w.cnt, w.st, w.bsum);
  k_scan_top<<<1, 1024, 0, s>>>(w.bsum, nb, w.st, L.pairs_cap);
  k_scan_emit<<<nb, kScanThreads, 0, s>>>(w.desc, w.tables, sorted_items, w.cnt, w.bsum, w.st, w.pk_a, w.pv_a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;

  // stable sort of the pairs by tile id
  const int64_t pc = L.pairs_cap > 0 ? L.pairs_cap : 1;
  const int Gp = static_cast<int>((pc + kSortChunk - 1) / kSortChunk);
  const int np = tile_passes(n_tiles);
  ka = w.pk_a; va = w.pv_a; kb = w.pk_b; vb = w.pv_b;
  for (int pass = 0; pass < np; ++pass) {
    PassIn p{ka, va, nullptr, &w.st->n_pairs, nullptr, 0};
    if ((e = radix_pass<0>(p, 8 * pass, w.hist, w.dtot + 256 * (4 + pass), Gp, nullptr, kb, vb, s)) != cudaSuccess)
      return e;
    uint32_t* t;
    t = ka; ka = kb; kb = t;
    t = va; va = vb; vb = t;
  }
  const int64_t rg = (pc + 255) / 256;
  k_ranges<<<static_cast<unsigned>(rg < 2048 ? rg : 2048), 256, 0, s>>>(ka, w.st, n_tiles, w.ranges);
  return cudaGetLastError();
}

}  // namespace lgs
