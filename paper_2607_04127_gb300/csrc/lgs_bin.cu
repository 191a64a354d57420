// lgs_bin.cu -- preprocess, angular-tile binning, per-tile depth sort.
//
// Pipeline of one lgs_bin_sort (all on the caller's stream, no host sync):
//   k_tables      per frame: binary32 sine / direction tables of the tile
//                 rows and columns (pixel-centre extremes of each tile)
//   k_preprocess  per (frame, surfel) item: 64 B compositing record, pixel
//                 box, depth key = bits of binary32 |mu_sensor|; the item's
//                 tiles (a range of tile rows times a circular range of tile
//                 columns, stored per item) and one count per covered tile
//                 (shared-memory counters per CTA, one atomic per tile)
//   k_tile_scan   one CTA: exclusive scan of the tile counts -> every tile's
//                 [start, end) and its fill cursor; capacity check; the
//                 longest-first tile order of the persistent kernels; the
//                 lists of tiles longer than kLongList, 2048 and 1024 keys
//   k_emit        every item appends (depth key << 32 | item) to the bucket
//                 of each tile of its stored set (order inside a bucket
//                 arbitrary)
//   k_tile_sort_all
//                 sort every bucket of up to 2048 keys by the 64-bit key in
//                 one launch: up to 1024 keys by a merge sort on half a CTA,
//                 up to 2048 on a whole CTA; then write the item list
//   k_sort_long   longer buckets, one 1024-thread CTA each, longest first:
//                 8192-key chunks sorted in shared memory, merged pairwise
//                 through global memory; then the item list
// The result is the order of the key (tile, depth, item): per tile, by depth,
// ties by item index.
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

__global__ void k_tables(const Desc* __restrict__ D, float* __restrict__ tab, Status* __restrict__ st,
                         uint32_t* __restrict__ loss_acc, uint32_t loss_words, uint32_t* __restrict__ tcount,
                         uint32_t n_tiles) {
  pdl_wait();               // (launched after a kernel of this chain: wait for it)
  pdl_launch_dependents();  // the next kernel may be dispatched now
  const FrameDev& F = D->f[blockIdx.x];
  // the tile counts start at zero (k_preprocess adds into them)
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_tiles; i += gridDim.x * blockDim.x) tcount[i] = 0u;
  // the loss accumulators start every binning at zero
  if (blockIdx.x == 0)
    for (uint32_t i = threadIdx.x; i < loss_words; i += blockDim.x) loss_acc[i] = 0u;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->required_pairs = 0;
    st->n_pairs = 0;
    st->n_vis = 0;
    st->overflow = 0;
    st->timeout = 0;
    st->check = 0;
    st->work_counter = 0;
    st->work_counter2 = 0;
    for (int c = 0; c < kBwdClasses; ++c) st->bq_count[c] = 0;
    st->evals_fwd = 0;
    st->evals_bwd = 0;
    st->contrib_fwd = 0;
    st->contrib_bwd = 0;
    st->alg_fwd = 0;
    st->loss_ticket = 0;
    st->count_ticket = 0;
    st->n_long = 0;
    st->n_big = 0;
    st->n_mid = 0;
    st->long_sort_counter = 0;
    st->long_counter_fwd = 0;
    st->long_counter_bwd = 0;
    st->long_done_fwd = 0;
    st->long_done_bwd = 0;
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

// Calls fn(global tile id) for every tile the item's bounding cone meets:
// rows ascending, then the candidate column ranges of bin_col_window in order.
// Only the tile rows that hold a pixel row of the item's pixel box (which
// pads the cone's elevation band by a whole pixel row on each side) are
// tested: a tile row the cone meets always holds one.
template <class Fn>
__device__ __forceinline__ uint32_t for_each_tile(const BinGeom& g, const FrameDev& F, const float* __restrict__ tab,
                                                  const float4& pbox, Fn fn) {
  const float4* ct = reinterpret_cast<const float4*>(tab + F.col_tab);
  ColWin w;
  bin_col_window(g, F, w);
  int ra = 0, rb = F.ntr - 1;
  if (!g.all_rows) {
    ra = max(0, static_cast<int>(pbox.x) / F.th);
    rb = min(F.ntr - 1, static_cast<int>(pbox.y) / F.th);
  }
  uint32_t n = 0;
  for (int r = ra; r <= rb; ++r) {
    if (!bin_row_hit(g, tab[F.row_tab + 2 * r], tab[F.row_tab + 2 * r + 1])) continue;
    const uint32_t rowbase = F.tile_base + static_cast<uint32_t>(r * F.ntc);
    for (int pass = 0; pass < 2; ++pass) {
      const int ja = pass ? w.b0 : w.a0, jb = pass ? w.b1 : w.a1;
      for (int jc = ja; jc <= jb; ++jc) {
        if (!bin_col_hit(g, ct[jc])) continue;
        fn(rowbase + static_cast<uint32_t>(jc));
        ++n;
      }
    }
  }
  return n;
}

// The tiles an item's bounding cone meets form a product of tile rows and
// tile columns (the row test depends on the row only, the column test on
// the column only).  The passing rows form one range and the passing columns
// one circular range (the cone is convex in elevation and in azimuth, and a
// tile between two passing tiles lies deep inside the cone), so an item's
// tiles are stored as rows [r0, r1] and nc columns from c0 on, modulo the
// column count.  Should the passing rows or columns not form one range (a
// decision at the binary32 edge of the cone), tile_set returns false and the
// caller enumerates the tiles one by one instead (for_each_tile).
struct TileSet {
  int r0, r1, c0, nc;
};

constexpr uint32_t kTsEnumerate = 0xffffffffu;   // stored tile set: enumerate tile by tile

__device__ __forceinline__ bool tile_set(const BinGeom& g, const FrameDev& F, const float* __restrict__ tab,
                                         const float4& pbox, TileSet& t) {
  const float4* ct = reinterpret_cast<const float4*>(tab + F.col_tab);
  t.r0 = 0;
  t.r1 = -1;
  t.c0 = 0;
  t.nc = 0;
  if (F.ntr >= 0xffff || F.ntc >= 0xffff) return false;
  int ra = 0, rb = F.ntr - 1;
  if (!g.all_rows) {
    ra = max(0, static_cast<int>(pbox.x) / F.th);
    rb = min(F.ntr - 1, static_cast<int>(pbox.y) / F.th);
  }
  int r0 = -1, r1 = -1, nr = 0;
  for (int r = ra; r <= rb; ++r) {
    if (!bin_row_hit(g, tab[F.row_tab + 2 * r], tab[F.row_tab + 2 * r + 1])) continue;
    if (r0 < 0) r0 = r;
    r1 = r;
    ++nr;
  }
  if (nr == 0) return true;
  if (nr != r1 - r0 + 1) return false;
  ColWin w;
  bin_col_window(g, F, w);
  // the candidate columns in circular order (the window's second range
  // continues the first across the azimuth seam)
  int prev = -1, runs = 0, first = 0, second = 0, n = 0;
  for (int pass = 0; pass < 2; ++pass) {
    const int ja = pass ? w.b0 : w.a0, jb = pass ? w.b1 : w.a1;
    for (int jc = ja; jc <= jb; ++jc) {
      if (!bin_col_hit(g, ct[jc])) continue;
      if (prev < 0 || jc != (prev + 1 == F.ntc ? 0 : prev + 1)) {
        ++runs;
        if (runs == 1) first = jc;
        else second = jc;
      }
      prev = jc;
      ++n;
    }
  }
  if (n == 0) return true;
  if (runs == 1) {
    t.c0 = first;
  } else if (runs == 2 && first == 0 && prev == F.ntc - 1) {
    t.c0 = second;        // one range across the seam, seen from column 0
  } else {
    return false;
  }
  t.r0 = r0;
  t.r1 = r1;
  t.nc = n;
  return true;
}

template <class Fn>
__device__ __forceinline__ void for_each_in_set(const TileSet& t, const FrameDev& F, Fn fn) {
  for (int r = t.r0; r <= t.r1; ++r) {
    const uint32_t rowbase = F.tile_base + static_cast<uint32_t>(r * F.ntc);
    for (int k = 0; k < t.nc; ++k) {
      int jc = t.c0 + k;
      if (jc >= F.ntc) jc -= F.ntc;
      fn(rowbase + static_cast<uint32_t>(jc));
    }
  }
}

__device__ __forceinline__ uint2 pack_set(const TileSet& t) {
  return make_uint2(static_cast<uint32_t>(t.r0) | (static_cast<uint32_t>(t.r1 < 0 ? 0 : t.r1) << 16),
                    static_cast<uint32_t>(t.c0) | (static_cast<uint32_t>(t.nc) << 16));
}

__device__ __forceinline__ TileSet unpack_set(uint2 p) {
  TileSet t;
  t.r0 = static_cast<int>(p.x & 0xffffu);
  t.r1 = static_cast<int>(p.x >> 16);
  t.c0 = static_cast<int>(p.y & 0xffffu);
  t.nc = static_cast<int>(p.y >> 16);
  return t;
}

// Per-CTA tile counters in shared memory: when all of a CTA's items belong
// to one frame with at most kAggTiles tiles, its per-tile atomics go to
// shared memory and each tile it touched gets one global atomic (items are
// usually stored in scan order, so a CTA touches few tiles).
constexpr int kAggTiles = 4096;

struct AggWin {
  bool local;
  uint32_t base, n;   // global id of the frame's tile 0, tiles of the frame
};

__device__ __forceinline__ AggWin agg_window(const Desc& D) {
  const int64_t first = static_cast<int64_t>(blockIdx.x) * blockDim.x;
  int64_t last = first + blockDim.x - 1;
  if (last >= D.n_items) last = D.n_items - 1;
  AggWin a;
  a.local = false;
  a.base = 0;
  a.n = 0;
  if (first > last) return a;
  const int f0 = frame_of_item(D, first), f1 = frame_of_item(D, last);
  const FrameDev& F = D.f[f0];
  a.n = static_cast<uint32_t>(F.ntr * F.ntc);
  a.base = F.tile_base;
  a.local = f0 == f1 && a.n <= static_cast<uint32_t>(kAggTiles);
  return a;
}

// ---------------------------------------------------------------------------
// Preprocess: record + key + box per (frame, surfel) item; tile counts
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_preprocess(const Desc* __restrict__ D, const float* __restrict__ tab,
                                                     float4* __restrict__ rec, float4* __restrict__ box,
                                                     uint32_t* __restrict__ key, uint32_t* __restrict__ cnt,
                                                     uint2* __restrict__ tset, uint32_t* __restrict__ tcount,
                                                     Status* __restrict__ st) {
  pdl_wait();               // (launched after a kernel of this chain: wait for it)
  pdl_launch_dependents();  // the next kernel may be dispatched now
  __shared__ uint32_t s_cnt[kAggTiles];
  const int64_t item = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool live = item < D->n_items;
  const AggWin aw = agg_window(*D);
  if (aw.local) {
    for (uint32_t t = threadIdx.x; t < aw.n; t += blockDim.x) s_cnt[t] = 0u;
    __syncthreads();
  }
  uint32_t c = 0;
  if (live) {
    const int f = frame_of_item(*D, item);
    const FrameDev& F = D->f[f];
    const MapDev& M = D->m[F.map];
    const int64_t i = item - F.item_base;
    // every parameter load issued up front (the atomics below would otherwise
    // keep the compiler from hoisting them)
    const float4 q = reinterpret_cast<const float4*>(M.quat)[i];
    const float ls0 = M.ls[2 * i], ls1 = M.ls[2 * i + 1], lg = M.logit[i];
    BinGeom g;
    bin_geom(M.mean + 3 * i, M.ls + 2 * i, F, g);
    key[item] = __float_as_uint(g.r);
    const float4 pb = pixel_box(g, F);
    TileSet ts;
    const auto count = [&](uint32_t t) {
      if (aw.local) atomicAdd(s_cnt + (t - aw.base), 1u);
      else atomicAdd(tcount + t, 1u);
    };
    if (tile_set(g, F, tab, pb, ts)) {
      for_each_in_set(ts, F, count);
      c = static_cast<uint32_t>((ts.r1 - ts.r0 + 1) * ts.nc);
      tset[item] = pack_set(ts);
    } else {
      c = for_each_tile(g, F, tab, pb, count);
      tset[item] = make_uint2(kTsEnumerate, kTsEnumerate);
    }
    cnt[item] = c;

    // compositing record (accuracy only): rotation of the unit quaternion,
    // axes to the sensor frame, activations
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
    const float isu = expf(-ls0), isv = expf(-ls1);
    const float alpha = 1.0f / (1.0f + expf(-lg));
    const float mx = g.x, my = g.y, mz = g.z;
    float4* out = rec + 4 * item;
    out[0] = make_float4(nx, ny, nz, nx * mx + ny * my + nz * mz);
    out[1] = make_float4(tux * isu, tuy * isu, tuz * isu, (tux * mx + tuy * my + tuz * mz) * isu);
    out[2] = make_float4(tvx * isv, tvy * isv, tvz * isv, (tvx * mx + tvy * my + tvz * mz) * isv);
    const float su = expf(ls0), sv = expf(ls1);
    out[3] = make_float4(alpha, su, sv, 0.f);
    box[item] = cull_box(g, F, pb, tux, tuy, tuz, tvx, tvy, tvz, su, sv);
  }
  // visible-item count, one atomic per warp
  const uint32_t vis = __ballot_sync(0xffffffffu, c > 0);
  if ((threadIdx.x & 31) == 0 && vis) atomicAdd(&st->n_vis, static_cast<unsigned int>(__popc(vis)));
  if (aw.local) {
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < aw.n; t += blockDim.x)
      if (s_cnt[t]) atomicAdd(tcount + aw.base + t, s_cnt[t]);
  }
}

// ---------------------------------------------------------------------------
// Tile offsets: one CTA scans the tile counts
// ---------------------------------------------------------------------------
constexpr int kScanCta = 1024;

constexpr uint32_t kLenCache = 4096;   // tiles whose list length the scan keeps in shared memory

// Bucket of a tile list length for the longest-first order: floor(log2(n)) + 1
// (0 for an empty tile), reversed so that bucket 0 holds the longest lists.
// Buckets of up to kMergeMax keys take the merge sort (one CTA per tile, all
// in one launch: a bucket's sort is a long serial chain, so every bucket
// runs concurrently); longer ones k_sort_long, in this longest-first order.
constexpr int kMergeMax = 2048;
constexpr int kMergeSmall = 1024;   // buckets up to this size: the 128-thread merge sort
constexpr int kOrderBuckets = 33;
__device__ __forceinline__ int order_bucket(uint32_t n) { return kOrderBuckets - 1 - (n ? 32 - __clz(n) : 0); }

__global__ void __launch_bounds__(kScanCta) k_tile_scan(uint32_t* __restrict__ tcur, uint32_t n_tiles,
                                                          uint2* __restrict__ ranges, Status* __restrict__ st,
                                                          int64_t cap, uint32_t* __restrict__ order,
                                                          uint32_t* __restrict__ longt, uint32_t* __restrict__ cbase,
                                                          uint32_t* __restrict__ midl) {
  pdl_wait();               // (launched after a kernel of this chain: wait for it)
  pdl_launch_dependents();  // the next kernel may be dispatched now
  __shared__ unsigned long long s_w[32];
  __shared__ uint32_t s_wc[32];
  __shared__ unsigned long long s_carry, s_tot;
  __shared__ uint32_t s_ccarry, s_ctot;
  __shared__ uint32_t s_bucket[kOrderBuckets];
  __shared__ uint32_t s_len[kLenCache];   // list lengths of the first tiles, kept for the order passes
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) {
    s_carry = 0;
    s_ccarry = 0;
  }
  if (tid < kOrderBuckets) s_bucket[tid] = 0;
  __syncthreads();
  for (uint32_t b0 = 0; b0 < n_tiles; b0 += kScanCta) {
    const uint32_t t = b0 + tid;
    const unsigned long long x = t < n_tiles ? tcur[t] : 0ull;
    // backward chunks of the list: ceil(n / kChunk)
    const uint32_t xc = static_cast<uint32_t>((x + kChunk - 1) / kChunk);
    unsigned long long v = x;
    uint32_t vc = xc;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
      const uint32_t yc = __shfl_up_sync(0xffffffffu, vc, o);
      if (lane >= o) {
        v += y;
        vc += yc;
      }
    }
    if (lane == 31) {
      s_w[wid] = v;
      s_wc[wid] = vc;
    }
    __syncthreads();
    // warp 0 turns the 32 warp totals into exclusive prefixes and the pass total
    if (wid == 0) {
      const unsigned long long x0 = s_w[lane];
      const uint32_t c0 = s_wc[lane];
      unsigned long long y = x0;
      uint32_t yc = c0;
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long z = __shfl_up_sync(0xffffffffu, y, o);
        const uint32_t zc = __shfl_up_sync(0xffffffffu, yc, o);
        if (lane >= o) {
          y += z;
          yc += zc;
        }
      }
      s_w[lane] = y - x0;
      s_wc[lane] = yc - c0;
      if (lane == 31) {
        s_tot = y;
        s_ctot = yc;
      }
    }
    __syncthreads();
    const unsigned long long wpre = s_w[wid], tot = s_tot;
    const uint32_t cpre = s_wc[wid], ctot = s_ctot;
    const unsigned long long start = s_carry + wpre + v - x;
    if (t < n_tiles) {
      // offsets past the capacity are never used: the emission is skipped
      const uint32_t s32 = static_cast<uint32_t>(start);
      if (t < kLenCache) s_len[t] = static_cast<uint32_t>(x);
      tcur[t] = s32;
      ranges[t] = x ? make_uint2(s32, static_cast<uint32_t>(start + x)) : make_uint2(0u, 0u);   // empty: (0, 0)
      // first chunk of the tile (non-decreasing over tiles: the chunk of a
      // global chunk index is found by binary search)
      cbase[t] = s_ccarry + cpre + vc - xc;
    }
    __syncthreads();
    if (tid == 0) {
      s_carry += tot;
      s_ccarry += ctot;
    }
    __syncthreads();
  }
  const unsigned long long total = s_carry;
  const bool over = total > static_cast<unsigned long long>(cap);
  if (tid == 0) {
    st->required_pairs = total;
    st->overflow = over ? 1u : 0u;
    st->n_pairs = over ? 0ull : total;
    st->n_chunks = over ? 0u : s_ccarry;   // at most pairs / kChunk + tiles
  }
  if (over) {
    // nothing is emitted: every tile renders empty
    for (uint32_t t = tid; t < n_tiles; t += kScanCta) ranges[t] = make_uint2(0u, 0u);
  }
  // work order of the persistent kernels: tiles by list length, longest
  // power-of-two class first (order inside a class is arbitrary; results do
  // not depend on it).  Both passes read the final ranges.
  __syncthreads();
  // one shared atomic per distinct class in a warp (most tiles of a frame
  // fall in a few classes, so per-tile atomics would serialise)
  // list length of tile t as the ranges now hold it
  const auto tile_len = [&](uint32_t t) -> uint32_t {
    if (over) return 0u;
    if (t < kLenCache) return s_len[t];
    const uint2 rg = ranges[t];
    return rg.y - rg.x;
  };
  for (uint32_t b0 = 0; b0 < n_tiles; b0 += kScanCta) {
    const uint32_t t = b0 + tid;
    const int b = t < n_tiles ? order_bucket(tile_len(t)) : -1;
    const uint32_t peers = __match_any_sync(0xffffffffu, b);
    if (b >= 0 && lane == __ffs(peers) - 1) atomicAdd(&s_bucket[b], static_cast<uint32_t>(__popc(peers)));
  }
  __syncthreads();
  // exclusive prefix of the 33 class counts by one warp (class 32 after the
  // other 32)
  static_assert(kOrderBuckets == 33, "one class per lane plus the last");
  if (wid == 0) {
    const uint32_t c = s_bucket[lane];
    uint32_t y = c;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t z = __shfl_up_sync(0xffffffffu, y, o);
      if (lane >= o) y += z;
    }
    s_bucket[lane] = y - c;
    if (lane == 31) s_bucket[32] = y;
  }
  __syncthreads();
  for (uint32_t b0 = 0; b0 < n_tiles; b0 += kScanCta) {
    const uint32_t t = b0 + tid;
    const uint32_t len = t < n_tiles ? tile_len(t) : 0u;
    const int b = t < n_tiles ? order_bucket(len) : -1;
    const uint32_t peers = __match_any_sync(0xffffffffu, b);
    const int leader = __ffs(peers) - 1;
    uint32_t pos = 0;
    if (b >= 0 && lane == leader) pos = atomicAdd(&s_bucket[b], static_cast<uint32_t>(__popc(peers)));
    pos = __shfl_sync(0xffffffffu, pos, leader) + __popc(peers & ((1u << lane) - 1u));
    if (b >= 0) order[pos] = t;
    if (len > kLongList) longt[atomicAdd(&st->n_long, 1u)] = t;
    // buckets beyond the merge sort (k_sort_long's, found through the
    // order); those beyond the 128-thread merge sort, for its 256-thread form
    if (len > kMergeMax) atomicAdd(&st->n_big, 1u);
    if (len > kMergeSmall && len <= kMergeMax) midl[atomicAdd(&st->n_mid, 1u)] = t;
  }
}

// ---------------------------------------------------------------------------
// Emission into the tile buckets
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_emit(const Desc* __restrict__ D, const float* __restrict__ tab,
                                               const uint32_t* __restrict__ key, const uint32_t* __restrict__ cnt,
                                               const uint2* __restrict__ tset, uint32_t* __restrict__ tcur,
                                               const uint2* __restrict__ ranges, Status* __restrict__ st,
                                               unsigned long long* __restrict__ pkey) {
  pdl_wait();               // (launched after a kernel of this chain: wait for it)
  pdl_launch_dependents();  // the next kernel may be dispatched now
  __shared__ uint32_t s_cnt[kAggTiles], s_base[kAggTiles];
  if (st->overflow) return;
  const int64_t item = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const AggWin aw = agg_window(*D);
  uint32_t c = 0;
  const FrameDev* F = nullptr;
  unsigned long long k = 0;
  // the item's tiles: its stored set, or (a set that is not one range) the
  // counting pass's enumeration repeated from the geometry
  TileSet ts{0, -1, 0, 0};
  bool slow = false;
  BinGeom g;
  float4 pb = make_float4(0.f, 0.f, 0.f, 0.f);
  if (item < D->n_items) {
    c = cnt[item];
    if (c) {
      const int f = frame_of_item(*D, item);
      F = &D->f[f];
      k = (static_cast<unsigned long long>(key[item]) << 32) | static_cast<uint32_t>(item);
      const uint2 packed = tset[item];
      slow = packed.x == kTsEnumerate;
      if (slow) {
        const MapDev& M = D->m[F->map];
        const int64_t i = item - F->item_base;
        bin_geom(M.mean + 3 * i, M.ls + 2 * i, *F, g);
        pb = pixel_box(g, *F);   // the sphere box the counting pass used (the stored box is the culling box)
      } else {
        ts = unpack_set(packed);
      }
    }
  }
  const auto tiles = [&](auto fn) -> uint32_t {
    if (slow) return for_each_tile(g, *F, tab, pb, fn);
    for_each_in_set(ts, *F, fn);
    return static_cast<uint32_t>((ts.r1 - ts.r0 + 1) * ts.nc);
  };
  // the enumeration repeats the counting pass exactly, so every slot lies
  // inside the tile's run; a slot outside it is dropped and recorded
  const auto put = [&](uint32_t t, uint32_t pos) {
    if (pos < ranges[t].y) pkey[pos] = k;
    else st->check = 1u;
  };
  if (!aw.local) {
    if (c) {
      const uint32_t n = tiles([&](uint32_t t) { put(t, atomicAdd(tcur + t, 1u)); });
      if (n != c) st->check = 1u;
    }
    return;
  }
  // shared counters: count, reserve one run per touched tile, then fill it
  for (uint32_t t = threadIdx.x; t < aw.n; t += blockDim.x) s_cnt[t] = 0u;
  __syncthreads();
  if (c) {
    const uint32_t n = tiles([&](uint32_t t) { atomicAdd(s_cnt + (t - aw.base), 1u); });
    if (n != c) st->check = 1u;
  }
  __syncthreads();
  for (uint32_t t = threadIdx.x; t < aw.n; t += blockDim.x) {
    const uint32_t m = s_cnt[t];
    if (m) {
      s_base[t] = atomicAdd(tcur + aw.base + t, m);
      s_cnt[t] = 0u;
    }
  }
  __syncthreads();
  if (c) tiles([&](uint32_t t) {
    const uint32_t lt = t - aw.base;
    put(t, s_base[lt] + atomicAdd(s_cnt + lt, 1u));
  });
}

// ---------------------------------------------------------------------------
// Per-tile sort
// ---------------------------------------------------------------------------
// ---- buckets of at most 2048 keys: merge sort in shared memory -----------
// Every thread sorts 8 keys in registers (a 19-comparator network), then
// runs of 8, 16, ... keys are merged pairwise until one run remains: each
// thread finds where its 8 outputs start in its pair of runs by a binary
// search along the merge path (ties, which only the padding has, go to the
// first run) and merges them sequentially.  The bucket is padded with +inf to
// a whole number N of 8-key rows; a pass's last runs may be shorter than L.

__device__ __forceinline__ void cas_reg(unsigned long long& a, unsigned long long& b) {
  const unsigned long long x = a, y = b;
  const bool sw = x > y;
  a = sw ? y : x;
  b = sw ? x : y;
}

__device__ __forceinline__ void sort8(unsigned long long (&k)[8]) {
  // Batcher's odd-even merge network for 8 inputs (19 comparators)
  cas_reg(k[0], k[1]); cas_reg(k[2], k[3]); cas_reg(k[4], k[5]); cas_reg(k[6], k[7]);
  cas_reg(k[0], k[2]); cas_reg(k[1], k[3]); cas_reg(k[4], k[6]); cas_reg(k[5], k[7]);
  cas_reg(k[1], k[2]); cas_reg(k[5], k[6]);
  cas_reg(k[0], k[4]); cas_reg(k[1], k[5]); cas_reg(k[2], k[6]); cas_reg(k[3], k[7]);
  cas_reg(k[2], k[4]); cas_reg(k[3], k[5]);
  cas_reg(k[1], k[2]); cas_reg(k[3], k[4]); cas_reg(k[5], k[6]);
}

// Shared-memory index of key x: one padding slot after every 8 keys, so the
// 8-key rows of consecutive threads start in different banks.
__device__ __forceinline__ uint32_t pad8(uint32_t x) { return x + (x >> 3); }

// Barrier of the threads sorting one bucket: the whole CTA (id 0), or one
// half of it (ids 1, 2 with 128 threads each), so that the two halves of a
// CTA sort two buckets independently.
template <int ID>
__device__ __forceinline__ void part_sync(uint32_t nthr) {
  if (ID == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"n"(ID), "r"(nthr) : "memory");
}

// The n <= 8 * nthr keys g[0, n) sorted by threads t = 0 .. nthr - 1 of one
// part of a CTA (barrier BAR) in sa / sb (pad8 of 8 * nthr keys each);
// returns the buffer that holds them (key i at pad8(i)), after a barrier.
template <int BAR>
__device__ __forceinline__ unsigned long long* smem_merge_sort(const unsigned long long* __restrict__ g, uint32_t n,
                                                               unsigned long long* sa, unsigned long long* sb,
                                                               uint32_t t, uint32_t nthr) {
  const uint32_t N = n > 8 ? (n + 7u) & ~7u : 8u;   // padded to whole 8-key rows only
  for (uint32_t i = t; i < N; i += nthr) sa[pad8(i)] = i < n ? g[i] : ~0ull;
  part_sync<BAR>(nthr);
  const bool act = 8 * t < N;
  if (act) {
    unsigned long long k[8];
#pragma unroll
    for (int r = 0; r < 8; ++r) k[r] = sa[9 * t + r];
    sort8(k);
#pragma unroll
    for (int r = 0; r < 8; ++r) sa[9 * t + r] = k[r];
  }
  // a pass over runs of L keys reads only the 2 L keys of its thread group's
  // pair of runs: up to L = 128 those are the 256 keys of the thread's own
  // warp, so the passes before it need only a warp barrier
  __syncwarp();
  unsigned long long *src = sa, *dst = sb;
  for (uint32_t L = 8; L < N; L <<= 1) {
    if (act) {
      const uint32_t tpp = L / 4;                  // threads per pair of runs
      const uint32_t pair = t / tpp, d = 8 * (t % tpp);
      // runs A = [a0, a0 + la), B = [b0, b0 + lb): L keys each, the last
      // ones shorter (B empty when A is the last run)
      const uint32_t a0 = 2 * L * pair, b0 = a0 + L;
      const uint32_t la = min(L, N - a0), lb = b0 < N ? min(L, N - b0) : 0u;
      // i = number of the first d outputs taken from A
      uint32_t lo = d > lb ? d - lb : 0, hi = d < la ? d : la;
      while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (src[pad8(a0 + mid)] > src[pad8(b0 + d - mid - 1)]) hi = mid;
        else lo = mid + 1;
      }
      uint32_t i = lo, j = d - lo;
      const uint32_t o = 9 * (a0 / 8 + d / 8);        // pad8 of the 8-aligned output row
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        // ties (only the +inf padding) go to A first, as in the search
        const unsigned long long a = i < la ? src[pad8(a0 + i)] : ~0ull, b = j < lb ? src[pad8(b0 + j)] : ~0ull;
        const bool takeA = j >= lb || (i < la && a <= b);
        dst[o + r] = takeA ? a : b;
        i += takeA;
        j += !takeA;
      }
    }
    if (2 * L <= 128) __syncwarp();
    else part_sync<BAR>(nthr);
    unsigned long long* tmp = src;
    src = dst;
    dst = tmp;
  }
  part_sync<BAR>(nthr);   // the result is read from every warp's keys
  return src;
}

// One bucket of at most 8 * nthr keys: sorted in shared memory, its item list
// written.
template <int BAR>
__device__ __forceinline__ void merge_sort_bucket(uint32_t tile, const uint2* __restrict__ ranges,
                                                  const unsigned long long* __restrict__ pkey,
                                                  uint32_t* __restrict__ pv, unsigned long long* sa,
                                                  unsigned long long* sb, uint32_t t, uint32_t nthr) {
  const uint2 rg = ranges[tile];
  const uint32_t n = rg.y - rg.x;
  const unsigned long long* src = smem_merge_sort<BAR>(pkey + rg.x, n, sa, sb, t, nthr);
  for (uint32_t i = t; i < n; i += nthr) pv[rg.x + i] = static_cast<uint32_t>(src[pad8(i)]);
}

// ---- buckets beyond 2048 keys: one CTA each, merged through global memory --
// A long bucket is sorted by one CTA of kLongSortCta threads: chunks of
// kLongChunk keys in shared memory (smem_merge_sort), then passes that merge
// pairs of sorted runs into runs twice as long, ping-ponging between the key
// array and a second buffer made of the pair-tile and item arrays (high and
// low 32 bits of each key; the pair tiles are rewritten on request only, and
// the item list is the keys' low half, so a result left there is already the
// list).  A pass writes its output in tiles of kLongChunk keys: the tile's
// first and last merge-path diagonals are found by binary searches in global
// memory (one per thread, for up to kLongSortCta tiles at once), its two input
// ranges loaded into shared memory, and every thread merges its 8 outputs.
// O(n log n) per bucket instead of the bitonic network's O(n log^2 n).
constexpr int kLongSortCta = 1024;
constexpr uint32_t kLongChunk = 8 * kLongSortCta;   // 8192 keys
constexpr size_t kLongSortSmem = 2 * sizeof(unsigned long long) * (kLongChunk + kLongChunk / 8) +
                                 sizeof(uint32_t) * (kLongSortCta + 1);   // two key buffers, the diagonals

// A bucket's keys: 64-bit words, or split into high and low 32-bit halves.
struct KeyBuf {
  unsigned long long* k;
  uint32_t *hi, *lo;
  __device__ __forceinline__ unsigned long long get(uint32_t i) const {
    return k ? k[i] : (static_cast<unsigned long long>(hi[i]) << 32) | lo[i];
  }
  __device__ __forceinline__ void put(uint32_t i, unsigned long long v) const {
    if (k) {
      k[i] = v;
    } else {
      hi[i] = static_cast<uint32_t>(v >> 32);
      lo[i] = static_cast<uint32_t>(v);
    }
  }
};

// Merge-path split: how many of the first d outputs of merging A[0, la) and
// B[0, lb) come from A (keys are distinct).
__device__ __forceinline__ uint32_t path_split(const KeyBuf& X, uint32_t a0, uint32_t la, uint32_t b0, uint32_t lb,
                                               uint32_t d) {
  uint32_t lo = d > lb ? d - lb : 0u, hi = d < la ? d : la;
  while (lo < hi) {
    const uint32_t mid = (lo + hi) >> 1;
    if (X.get(a0 + mid) > X.get(b0 + d - mid - 1)) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

__global__ void __launch_bounds__(kLongSortCta) k_sort_long(const uint2* __restrict__ ranges,
                                                             Status* __restrict__ st,
                                                             const uint32_t* __restrict__ order,
                                                             uint32_t n_tiles, unsigned long long* __restrict__ pkey,
                                                             uint32_t* __restrict__ ptile, uint32_t* __restrict__ pv) {
  extern __shared__ __align__(16) unsigned long long s_long[];
  unsigned long long* sa = s_long;
  unsigned long long* sb = s_long + kLongChunk + kLongChunk / 8;
  uint32_t* s_split = reinterpret_cast<uint32_t*>(sb + kLongChunk + kLongChunk / 8);
  __shared__ uint32_t s_claim;
  if (st->overflow || st->n_big == 0) return;
  const uint32_t t = threadIdx.x;
  while (true) {
    // buckets in the tile scan's longest-first order; the long ones come
    // first, so the first list of at most kMergeMax keys ends the work
    __syncthreads();
    if (t == 0) s_claim = atomicAdd(&st->long_sort_counter, 1u);
    __syncthreads();
    const uint32_t k = s_claim;
    if (k >= n_tiles) return;
    const uint32_t tile = order[k];
    const uint2 rg = ranges[tile];
    const uint32_t n = rg.y - rg.x;
    if (order_bucket(n) > order_bucket(kMergeMax + 1)) return;   // a shorter class: no long list follows
    if (n <= kMergeMax) continue;
    KeyBuf X{pkey + rg.x, nullptr, nullptr}, Y{nullptr, ptile + rg.x, pv + rg.x};
    // sorted chunks, in place
    for (uint32_t c0 = 0; c0 < n; c0 += kLongChunk) {
      const uint32_t m = min(kLongChunk, n - c0);
      const unsigned long long* res = smem_merge_sort<0>(X.k + c0, m, sa, sb, t, kLongSortCta);
      for (uint32_t i = t; i < m; i += kLongSortCta) X.k[c0 + i] = res[pad8(i)];
      __syncthreads();
    }
    // merge passes: runs of R keys into runs of 2 R
    bool in_x = true;
    for (uint32_t R = kLongChunk; R < n; R <<= 1) {
      const KeyBuf& S = in_x ? X : Y;
      const KeyBuf& Dst = in_x ? Y : X;
      const uint32_t n_out = (n + kLongChunk - 1) / kLongChunk;   // output tiles (a run pair holds whole tiles)
      for (uint32_t q0 = 0; q0 < n_out; q0 += kLongSortCta) {
        // first diagonal of output tiles q0 + t (and the end of the last one)
        __syncthreads();
        for (uint32_t q = q0 + t; q <= min(q0 + kLongSortCta, n_out); q += kLongSortCta) {
          const uint32_t o = min(q * kLongChunk, n);
          uint32_t p = o / (2 * R);
          if (o == n && o % (2 * R) == 0 && o > 0) --p;   // the end diagonal of the last pair
          const uint32_t a0 = 2 * R * p, la = min(R, n - a0), b0 = a0 + R;
          const uint32_t lb = b0 < n ? min(R, n - b0) : 0u;
          s_split[q - q0] = path_split(S, a0, la, b0, lb, o - a0);
        }
        __syncthreads();
        const uint32_t q1 = min(q0 + kLongSortCta, n_out);
        for (uint32_t q = q0; q < q1; ++q) {
          const uint32_t o = q * kLongChunk, oe = min(o + kLongChunk, n);
          const uint32_t p = o / (2 * R);
          const uint32_t a0 = 2 * R * p, la = min(R, n - a0), b0 = a0 + R;
          const uint32_t d0 = o - a0, d1 = oe - a0;
          const uint32_t i0 = s_split[q - q0];
          // the tile's end diagonal: the next tile's first one, or the whole
          // pair when the tile closes it
          const uint32_t i1 = d1 == la + (b0 < n ? min(R, n - b0) : 0u) ? la : s_split[q + 1 - q0];
          const uint32_t j0 = d0 - i0, j1 = d1 - i1;
          const uint32_t na = i1 - i0, nb = j1 - j0;
          // A's part then B's part, in shared memory
          for (uint32_t i = t; i < na; i += kLongSortCta) sa[i] = S.get(a0 + i0 + i);
          for (uint32_t i = t; i < nb; i += kLongSortCta) sa[na + i] = S.get(b0 + j0 + i);
          __syncthreads();
          const uint32_t d = 8 * t;
          if (d < na + nb) {
            uint32_t lo = d > nb ? d - nb : 0u, hi = d < na ? d : na;
            while (lo < hi) {
              const uint32_t mid = (lo + hi) >> 1;
              if (sa[mid] > sa[na + d - mid - 1]) hi = mid;
              else lo = mid + 1;
            }
            uint32_t i = lo, j = d - lo;
            const uint32_t cnt = min(8u, na + nb - d);
            for (uint32_t r = 0; r < cnt; ++r) {
              const unsigned long long a = i < na ? sa[i] : ~0ull, b = j < nb ? sa[na + j] : ~0ull;
              const bool takeA = j >= nb || (i < na && a < b);
              Dst.put(o + d + r, takeA ? a : b);
              i += takeA;
              j += !takeA;
            }
          }
          __syncthreads();
        }
      }
      in_x = !in_x;
    }
    // the item list: the keys' low halves (already in place when the result
    // is in the split buffer)
    if (in_x)
      for (uint32_t i = t; i < n; i += kLongSortCta) pv[rg.x + i] = static_cast<uint32_t>(X.k[i]);
  }
}

// ---- every bucket of at most 2048 keys in one launch ------------------------
// The first n_lead CTAs take the buckets of 1025..2048 keys from the tile
// scan's list (the merge sort over the whole CTA), looping until it is done;
// every other CTA sorts two buckets of at most 1024 keys, one per half (128
// threads, its own named barrier).  Shared memory: two halves of two
// 1152-key buffers, or one pair of 2304-key buffers.  Longer buckets are
// k_sort_long's.
constexpr int kSortAllCta = 256;
constexpr int kSortAllSmem = 2 * (kMergeMax + kMergeMax / 8);   // 4608 keys, 36 KB
static_assert(kSortAllCta == kMergeMax / 8 && kSortAllCta == 2 * (kMergeSmall / 8), "thread counts");

__global__ void __launch_bounds__(kSortAllCta) k_tile_sort_all(const uint2* __restrict__ ranges,
                                                                const Status* __restrict__ st,
                                                                const uint32_t* __restrict__ midl,
                                                                uint32_t n_tiles, uint32_t n_lead,
                                                                unsigned long long* __restrict__ pkey,
                                                                uint32_t* __restrict__ pv) {
  __shared__ unsigned long long s[kSortAllSmem];
  if (st->overflow) return;
  if (blockIdx.x < n_lead) {
    for (uint32_t k = blockIdx.x; k < st->n_mid; k += n_lead) {
      __syncthreads();
      merge_sort_bucket<0>(midl[k], ranges, pkey, pv, s, s + kMergeMax + kMergeMax / 8, threadIdx.x, kSortAllCta);
    }
    return;
  }
  const uint32_t half = threadIdx.x >> 7;
  const uint32_t tile = 2 * (blockIdx.x - n_lead) + half;
  if (tile >= n_tiles) return;
  const uint2 rg = ranges[tile];
  const uint32_t n = rg.y - rg.x;
  if (n == 0 || n > kMergeSmall) return;   // empty, or a list of the lead CTAs
  unsigned long long* sa = s + half * 2 * (kMergeSmall + kMergeSmall / 8);
  unsigned long long* sb = sa + kMergeSmall + kMergeSmall / 8;
  if (half == 0) merge_sort_bucket<1>(tile, ranges, pkey, pv, sa, sb, threadIdx.x & 127u, 128);
  else merge_sort_bucket<2>(tile, ranges, pkey, pv, sa, sb, threadIdx.x & 127u, 128);
}

// The tile of every pair (sorted order), written only when a caller asks for
// it (the session's bin read-back): one CTA per tile fills its run.
__global__ void k_fill_tile_of_pair(const uint2* __restrict__ ranges, const Status* __restrict__ st,
                                    uint32_t* __restrict__ ptile) {
  if (st->overflow) return;
  const uint2 rg = ranges[blockIdx.x];
  for (uint32_t i = rg.x + threadIdx.x; i < rg.y; i += blockDim.x) ptile[i] = blockIdx.x;
}

cudaError_t launch_fill_tile_of_pair(const WsPtrs& w, uint32_t n_tiles, cudaStream_t s) {
  if (n_tiles) k_fill_tile_of_pair<<<n_tiles, 256, 0, s>>>(w.ranges, w.st, w.ptile);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Orchestration
// ---------------------------------------------------------------------------
// kernels launch_bin enqueues (memsets not counted)
int bin_kernel_count(uint32_t) { return 5; }

cudaError_t launch_bin(const Layout& L, const WsPtrs& w, int n_frames, int64_t n_items, uint32_t n_tiles,
                       const SideStream& side, cudaStream_t s) {
  k_tables<<<n_frames, 256, 0, s>>>(w.desc, w.tables, w.st, reinterpret_cast<uint32_t*>(w.loss_part),
                                    static_cast<uint32_t>(loss_part_bytes() / 4), w.tcur, n_tiles);
  const int64_t ni = n_items > 0 ? n_items : 1;
  const unsigned gi = static_cast<unsigned>((ni + 255) / 256);
  // each of the next three follows a kernel of this chain: dispatched while
  // its predecessor runs, it waits for it in its first instruction
  cudaError_t e0 = launch_dep(k_preprocess, dim3(gi), dim3(256), 0, s, w.desc, w.tables, w.rec, w.box, w.key, w.cnt,
                              w.tset, w.tcur, w.st);
  if (e0 == cudaSuccess)
    e0 = launch_dep(k_tile_scan, dim3(1), dim3(kScanCta), 0, s, w.tcur, n_tiles, w.ranges, w.st, L.pairs_cap, w.work,
                    w.longt, w.cbase, w.midl);
  if (e0 == cudaSuccess)
    e0 = launch_dep(k_emit, dim3(gi), dim3(256), 0, s, w.desc, w.tables, w.key, w.cnt, w.tset, w.tcur, w.ranges, w.st,
                    w.pkey);
  if (e0 != cudaSuccess) return e0;
  if (n_tiles > 0) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned few = static_cast<unsigned>(sms) < n_tiles ? static_cast<unsigned>(sms) : n_tiles;
    const unsigned grid = few + (n_tiles + 1) / 2;
    // the long buckets: one CTA each, longest first (an early exit when the
    // tile scan found none), on the side stream alongside the short buckets
    static bool smem_set[64] = {false};
    if (dev < 64 && !smem_set[dev]) {
      const cudaError_t e = cudaFuncSetAttribute(k_sort_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(kLongSortSmem));
      if (e != cudaSuccess) return e;
      smem_set[dev] = true;
    }
    cudaError_t e = cudaEventRecord(side.fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side.s, side.fork, 0);
    if (e != cudaSuccess) return e;
    k_sort_long<<<sms, kLongSortCta, kLongSortSmem, side.s>>>(w.ranges, w.st, w.work, n_tiles, w.pkey, w.ptile,
                                                               w.pv);
    if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaEventRecord(side.join, side.s)) != cudaSuccess) return e;
    k_tile_sort_all<<<grid, kSortAllCta, 0, s>>>(w.ranges, w.st, w.midl, n_tiles, few, w.pkey, w.pv);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(s, side.join, 0)) != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace lgs
