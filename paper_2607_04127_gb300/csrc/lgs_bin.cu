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
//                 sort every bucket by the 64-bit key in one launch: up to
//                 1024 keys by a merge sort on half a CTA, up to 2048 on a
//                 whole CTA, longer buckets by a bitonic network (up to 4096
//                 in shared memory, beyond that chunks merged through global
//                 memory); then write the item list
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
// runs concurrently); longer ones the bitonic network, over their own list.
constexpr int kMergeMax = 2048;
constexpr int kMergeSmall = 1024;   // buckets up to this size: the 128-thread merge sort
constexpr int kOrderBuckets = 33;
__device__ __forceinline__ int order_bucket(uint32_t n) { return kOrderBuckets - 1 - (n ? 32 - __clz(n) : 0); }

__global__ void __launch_bounds__(kScanCta) k_tile_scan(uint32_t* __restrict__ tcur, uint32_t n_tiles,
                                                          uint2* __restrict__ ranges, Status* __restrict__ st,
                                                          int64_t cap, uint32_t* __restrict__ order,
                                                          uint32_t* __restrict__ longt, uint32_t* __restrict__ cbase,
                                                          uint32_t* __restrict__ sortl, uint32_t* __restrict__ midl) {
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
    // backward chunks of the list: ceil(n / kChunk) for n <= kLongList
    // entries (longer lists have their own kernels)
    const uint32_t xc = x <= kLongList ? static_cast<uint32_t>((x + kChunk - 1) / kChunk) : 0u;
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
    // buckets beyond the merge sort, for the bitonic sort; those beyond the
    // 128-thread merge sort, for its 256-thread form
    if (len > kMergeMax) sortl[atomicAdd(&st->n_big, 1u)] = t;
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
// Bitonic network in its ascending-only form: the first step of every merge
// compares i with its mirror i ^ (k - 1), the later steps are half-cleaners
// (i, i + j).  Every comparator puts the minimum at the lower index, so
// positions past the end of a bucket act as +infinity and are never touched.
constexpr int kSortSmem = 4096;   // keys sorted in shared memory at once

__device__ __forceinline__ void cas(unsigned long long* a, uint32_t i, uint32_t j) {
  const unsigned long long x = a[i], y = a[j];
  if (x > y) {
    a[i] = y;
    a[j] = x;
  }
}

// Comparator p of a step with stride j = 2^lj (half-cleaner) or of the
// mirror step of a merge of blocks k = 2^(lj+1): its lower index.  For
// strides below 64 the 32 comparators of a warp stay inside one 64-key
// block, so those steps need only a warp barrier.
__device__ __forceinline__ uint32_t lower_index(uint32_t p, uint32_t lj) {
  return ((p >> lj) << (lj + 1)) | (p & ((1u << lj) - 1u));
}

// Barrier around a step of the given stride: a step that crosses warps
// (stride >= 64) is fenced by block barriers on both sides; between two
// warp-local steps a warp barrier suffices.
__device__ __forceinline__ void step_sync(uint32_t stride) {
  if (stride >= 64) __syncthreads();
  else __syncwarp();
}

// Full sort of s[0, N) in shared memory (N a power of two <= kSortSmem).
__device__ void smem_sort(unsigned long long* s, uint32_t N) {
  for (uint32_t lk = 1; (1u << lk) <= N; ++lk) {
    const uint32_t k = 1u << lk;
    if ((k >> 1) >= 64) __syncthreads();
    for (uint32_t p = threadIdx.x; p < N / 2; p += blockDim.x) {
      const uint32_t i = lower_index(p, lk - 1);
      cas(s, i, i ^ (k - 1));
    }
    step_sync(k >> 1);
    for (int lj = static_cast<int>(lk) - 2; lj >= 0; --lj) {
      if ((1u << lj) >= 64) __syncthreads();
      for (uint32_t p = threadIdx.x; p < N / 2; p += blockDim.x) {
        const uint32_t i = lower_index(p, lj);
        cas(s, i, i + (1u << lj));
      }
      step_sync(1u << lj);
    }
  }
  __syncthreads();
}

// Half-cleaners j = S/2 .. 1 on s[0, S) (the tail of a merge step).
__device__ void smem_clean(unsigned long long* s, uint32_t S) {
  for (int lj = 31 - __clz(S) - 1; lj >= 0; --lj) {
    if ((1u << lj) >= 64) __syncthreads();
    for (uint32_t p = threadIdx.x; p < S / 2; p += blockDim.x) {
      const uint32_t i = lower_index(p, lj);
      cas(s, i, i + (1u << lj));
    }
    step_sync(1u << lj);
  }
  __syncthreads();
}

__device__ void chunk_load(unsigned long long* s, const unsigned long long* g, uint32_t base, uint32_t n, uint32_t S) {
  for (uint32_t i = threadIdx.x; i < S; i += blockDim.x) s[i] = base + i < n ? g[base + i] : ~0ull;
  __syncthreads();
}

__device__ void chunk_store(const unsigned long long* s, unsigned long long* g, uint32_t base, uint32_t n, uint32_t S) {
  for (uint32_t i = threadIdx.x; i < S; i += blockDim.x)
    if (base + i < n) g[base + i] = s[i];
  __syncthreads();
}

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

// One bucket of at most 8 * nthr keys sorted by threads t = 0 .. nthr - 1 of
// one part of a CTA (barrier BAR), in sa / sb (pad8 of 8 * nthr keys each).
template <int BAR>
__device__ __forceinline__ void merge_sort_bucket(uint32_t tile, const uint2* __restrict__ ranges,
                                                  const unsigned long long* __restrict__ pkey,
                                                  uint32_t* __restrict__ pv, unsigned long long* sa,
                                                  unsigned long long* sb, uint32_t t, uint32_t nthr) {
  const uint2 rg = ranges[tile];
  const uint32_t n = rg.y - rg.x;
  const uint32_t N = n > 8 ? (n + 7u) & ~7u : 8u;   // padded to whole 8-key rows only
  const unsigned long long* g = pkey + rg.x;
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
  part_sync<BAR>(nthr);   // the list is written from every warp's keys
  for (uint32_t i = t; i < n; i += nthr) pv[rg.x + i] = static_cast<uint32_t>(src[pad8(i)]);
}

// ---- buckets beyond 2048 keys: a bitonic network over the whole CTA --------
__device__ void bitonic_bucket(uint32_t tile, const uint2* __restrict__ ranges, unsigned long long* __restrict__ pkey,
                               uint32_t* __restrict__ pv, unsigned long long* s) {
  const uint2 rg = ranges[tile];
  const uint32_t n = rg.y - rg.x;
  unsigned long long* g = pkey + rg.x;
  if (n <= kSortSmem) {
    uint32_t N = 2;
    while (N < n) N <<= 1;
    chunk_load(s, g, 0, n, N);
    smem_sort(s, N);
    for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) pv[rg.x + i] = static_cast<uint32_t>(s[i]);
    return;
  }
  // long bucket: sorted chunks of kSortSmem, then the merge steps whose
  // stride spans chunks run in global memory (this CTA only; __syncthreads
  // orders its global accesses), the rest per chunk in shared memory
  const uint32_t S = kSortSmem;
  uint32_t N = S;
  while (N < n) N <<= 1;
  for (uint32_t b = 0; b < n; b += S) {
    chunk_load(s, g, b, n, S);
    smem_sort(s, S);
    chunk_store(s, g, b, n, S);
  }
  for (uint32_t lk = 31 - __clz(2 * S); (1u << lk) <= N; ++lk) {
    const uint32_t k = 1u << lk;
    for (uint32_t p = threadIdx.x; p < N / 2; p += blockDim.x) {
      const uint32_t i = lower_index(p, lk - 1), j = i ^ (k - 1);
      if (j < n) cas(g, i, j);
    }
    __syncthreads();
    for (uint32_t lj = lk - 2; (1u << lj) >= S; --lj) {
      for (uint32_t p = threadIdx.x; p < N / 2; p += blockDim.x) {
        const uint32_t i = lower_index(p, lj);
        if (i + (1u << lj) < n) cas(g, i, i + (1u << lj));
      }
      __syncthreads();
    }
    for (uint32_t b = 0; b < n; b += S) {
      chunk_load(s, g, b, n, S);
      smem_clean(s, S);
      chunk_store(s, g, b, n, S);
    }
  }
  for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) pv[rg.x + i] = static_cast<uint32_t>(g[i]);
}

// ---- every bucket in one launch ------------------------------------------------
// The first n_lead CTAs take the long buckets, which take longest, from the
// tile scan's lists (beyond 2048 keys the bitonic network, then those of
// 1025..2048 keys the merge sort over the whole CTA), looping until the lists
// are done; every other CTA sorts two buckets of at most 1024 keys, one per
// half (128 threads, its own named barrier).  Shared memory: two halves of
// two 1152-key buffers, or one pair of 2304-key buffers, or 4096 keys of the
// bitonic network.
constexpr int kSortAllCta = 256;
constexpr int kSortAllSmem = 2 * (kMergeMax + kMergeMax / 8);   // 4608 keys, 36 KB
static_assert(kSortAllSmem >= kSortSmem, "the bitonic network fits the merge buffers");
static_assert(kSortAllCta == kMergeMax / 8 && kSortAllCta == 2 * (kMergeSmall / 8), "thread counts");

__global__ void __launch_bounds__(kSortAllCta) k_tile_sort_all(const uint2* __restrict__ ranges,
                                                                const Status* __restrict__ st,
                                                                const uint32_t* __restrict__ sortl,
                                                                const uint32_t* __restrict__ midl,
                                                                uint32_t n_tiles, uint32_t n_lead,
                                                                unsigned long long* __restrict__ pkey,
                                                                uint32_t* __restrict__ pv) {
  __shared__ unsigned long long s[kSortAllSmem];
  if (st->overflow) return;
  if (blockIdx.x < n_lead) {
    for (uint32_t k = blockIdx.x; k < st->n_big; k += n_lead) {
      __syncthreads();   // the previous bucket's readers are done with s
      bitonic_bucket(sortl[k], ranges, pkey, pv, s);
    }
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
                       cudaStream_t s) {
  k_tables<<<n_frames, 256, 0, s>>>(w.desc, w.tables, w.st, reinterpret_cast<uint32_t*>(w.loss_part),
                                    static_cast<uint32_t>(loss_part_bytes() / 4), w.tcur, n_tiles);
  const int64_t ni = n_items > 0 ? n_items : 1;
  const unsigned gi = static_cast<unsigned>((ni + 255) / 256);
  k_preprocess<<<gi, 256, 0, s>>>(w.desc, w.tables, w.rec, w.box, w.key, w.cnt, w.tset, w.tcur, w.st);
  k_tile_scan<<<1, kScanCta, 0, s>>>(w.tcur, n_tiles, w.ranges, w.st, L.pairs_cap, w.work, w.longt, w.cbase,
                                     w.sortl, w.midl);
  k_emit<<<gi, 256, 0, s>>>(w.desc, w.tables, w.key, w.cnt, w.tset, w.tcur, w.ranges, w.st, w.pkey);
  if (n_tiles > 0) {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned few = static_cast<unsigned>(sms) < n_tiles ? static_cast<unsigned>(sms) : n_tiles;
    const unsigned grid = few + (n_tiles + 1) / 2;
    k_tile_sort_all<<<grid, kSortAllCta, 0, s>>>(w.ranges, w.st, w.sortl, w.midl, n_tiles, few, w.pkey, w.pv);
  }
  return cudaGetLastError();
}

}  // namespace lgs
