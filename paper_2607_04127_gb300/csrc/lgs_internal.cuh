// lgs_internal.cuh -- device-side descriptors and shared device functions of
// the GB300 surfel rasterizer (CUDA path only).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/lgs.h"

namespace lgs {

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched with launch_dep may be
// dispatched while the previous kernel on its stream still runs: its CTAs
// become resident and wait in pdl_wait() (griddepcontrol.wait: until that
// kernel has completed and its memory is visible) before touching anything
// it wrote.  A kernel calls pdl_launch_dependents() at its start so that
// its successor's dispatch overlaps its own run; the successor is launched
// only once every CTA of the kernel has started, so waiting CTAs never hold
// the slots the kernel still needs.  Both are no-ops for a kernel launched
// without the attribute.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// ---------------------------------------------------------------------------
// Descriptors (written once per call into the workspace by k_write_desc)
// ---------------------------------------------------------------------------
struct FrameDev {
  int32_t H, W, th, tw, ntr, ntc;
  int32_t map;             // index of the surfel set this frame renders
  uint32_t tile_base;      // global id of the frame's tile 0
  int64_t item_base;       // global id of (this frame, surfel 0)
  int64_t n;               // surfels of the map
  uint32_t row_tab;        // float offset of [2*ntr] (sin_top, sin_bot) in tables
  uint32_t col_tab;        // float offset of [4*ntc] (cos0, sin0, cos1, sin1) in tables
  float emin, emax;
  float R[9];              // sensor -> world rotation, row-major
  float o[3];              // sensor origin (world)
  // per-call pointers (caller-owned device memory)
  float *A, *St, *Sn, *Tf;
  int32_t* nc;
  const float *gA, *gSt, *gSn;
  float *oA, *oSt, *oSn;   // loss: gradient planes to write
  const float *D, *Ng;     // loss: targets
};

struct MapDev {
  const float *mean, *quat, *ls, *logit;
  int64_t n;
  int64_t surf_base;       // first surfel of this map in the flattened surfel range
  float *d_mean, *d_quat, *d_ls, *d_logit;
  int32_t n_frames;        // frames of the call that render this map
  int32_t pad;
};

struct Desc {
  int32_t n_frames, n_maps;
  int32_t th, tw;
  uint32_t n_tiles;        // total over frames
  int64_t n_items;         // total (frame, surfel) items
  int64_t n_surf;          // total surfels over maps
  FrameDev f[LGS_MAX_FRAMES];
  MapDev m[LGS_MAX_MAPS];
};

// Queues of the chunked backward's work items, in the order warps claim
// them: class 0 holds the chunks a warp block walks in full (and every chunk
// of a long list), classes 1 .. kBwdClasses-1 the chunk in which the block's
// last composited entry lies, by decreasing length of its walked part.  The
// costliest items go first, so the backward ends on short ones.  Built at
// the start of every backward from the forward's per-block last entries.
constexpr int kBwdClasses = 9;

// Status words (device, in the workspace).
struct Status {
  unsigned long long required_pairs;  // pairs the last bin_sort needed
  unsigned long long n_pairs;         // pairs actually emitted (0 on overflow)
  unsigned int n_vis;                 // items with at least one tile
  unsigned int overflow;              // 1 if required_pairs > capacity
  unsigned int timeout;               // a bounded wait gave up
  unsigned int check;                 // a checked-build bounds check failed
  unsigned int work_counter;          // persistent scheduler: next work item
  unsigned int work_counter2;
  unsigned int bq_count[kBwdClasses]; // backward items queued per class (zero between backwards)
  unsigned int n_long;                // tiles whose list is longer than kLongList
  unsigned int long_counter_fwd;      // work counters of the long-list kernels (self-resetting)
  unsigned int long_counter_bwd;
  unsigned int long_done_fwd;         // warps of the long-list kernels that have finished
  unsigned int long_done_bwd;
  unsigned long long evals_fwd;       // ray/surfel evaluations (cumulative since bin_sort)
  unsigned long long evals_bwd;
  unsigned long long contrib_fwd;     // composited (fwd) / valid re-evaluated (bwd) pairs
  unsigned long long contrib_bwd;
  unsigned long long alg_fwd;         // list entries up to and including each pixel's stop point
  unsigned int loss_ticket;           // loss CTAs finished (the last one reduces; self-resetting)
  unsigned int n_chunks;              // backward chunks of the last binning (kChunk list entries each)
  unsigned int count_ticket;          // mask-count CTAs finished (the last one adds up; self-resetting)
  unsigned int n_big;                 // buckets of more than 2048 keys (the bitonic sort)
  unsigned int n_mid;                 // buckets of 1025..2048 keys (the wide merge sort)
  unsigned int long_sort_counter;     // tile order positions claimed by the long-bucket sort
};

struct Layout {
  size_t desc, status, tables, rec, box, key, cnt, tset, tcur, pkey, ptile, pv, ranges, g13, work, longt, loss_part,
      cbase, ckpt, csuf, cmask, midl, bwm, bq, total;
  int64_t items_cap, pairs_cap, chunks_cap;
  uint32_t bq_cap0, bq_capk;  // capacity of the backward queue of class 0 and of each other class
  uint32_t tiles_cap;
  uint32_t tables_cap;     // floats
  int32_t loss_blocks;
};

struct WsPtrs {
  Desc* desc;
  Status* st;
  float* tables;
  float4* rec;             // [items][4]
  float4* box;             // [items] conservative pixel box: row_lo, row_hi, col centre, col half-width
  uint32_t* key;           // depth key per item
  uint32_t* cnt;           // tile count per item
  uint2* tset;             // tile set per item: rows (first | last << 16), columns (first | count << 16)
  uint32_t* tcur;          // [tiles] pair counts, then fill cursors
  unsigned long long* pkey;// [pairs] (depth key << 32 | item), bucketed by tile, then sorted
  uint32_t* ptile;         // [pairs] tile of every pair (sorted order)
  uint32_t* pv;            // [pairs] item of every pair (sorted order)
  uint2* ranges;           // [tiles]
  float* g13;              // [items][16]
  uint32_t* work;          // persistent scheduler tile order
  uint32_t* longt;         // tiles with lists longer than kLongList (st->n_long of them)
  double* loss_part;       // loss partial sums and mask counts
  uint32_t* cbase;         // [tiles] first backward chunk of every tile
  float* ckpt;             // [chunks][kCkptSlots][tile pixels] forward checkpoint at every chunk end
  float* csuf;             // [chunks][tile pixels] long lists: the suffix of the later chunks (backward)
  uint32_t* cmask;         // [chunks][4 windows][tile pixels] entries each pixel composited, one bit per entry
  uint32_t* midl;          // [tiles] tiles whose bucket takes the wide merge sort (st->n_mid of them)
  uint32_t* bwm;           // [tiles][warp blocks] the block's largest n_contrib (short lists; written by k_fwd_s)
  uint2* bq;               // backward work queues: (chunk * blocks per tile + block, tile); class 0 first
  uint32_t bq_cap0, bq_capk;
};

inline WsPtrs ws_ptrs(void* base, const Layout& L) {
  char* b = static_cast<char*>(base);
  WsPtrs p;
  p.desc = reinterpret_cast<Desc*>(b + L.desc);
  p.st = reinterpret_cast<Status*>(b + L.status);
  p.tables = reinterpret_cast<float*>(b + L.tables);
  p.rec = reinterpret_cast<float4*>(b + L.rec);
  p.box = reinterpret_cast<float4*>(b + L.box);
  p.key = reinterpret_cast<uint32_t*>(b + L.key);
  p.cnt = reinterpret_cast<uint32_t*>(b + L.cnt);
  p.tset = reinterpret_cast<uint2*>(b + L.tset);
  p.tcur = reinterpret_cast<uint32_t*>(b + L.tcur);
  p.pkey = reinterpret_cast<unsigned long long*>(b + L.pkey);
  p.ptile = reinterpret_cast<uint32_t*>(b + L.ptile);
  p.pv = reinterpret_cast<uint32_t*>(b + L.pv);
  p.ranges = reinterpret_cast<uint2*>(b + L.ranges);
  p.g13 = reinterpret_cast<float*>(b + L.g13);
  p.work = reinterpret_cast<uint32_t*>(b + L.work);
  p.longt = reinterpret_cast<uint32_t*>(b + L.longt);
  p.loss_part = reinterpret_cast<double*>(b + L.loss_part);
  p.cbase = reinterpret_cast<uint32_t*>(b + L.cbase);
  p.ckpt = reinterpret_cast<float*>(b + L.ckpt);
  p.csuf = reinterpret_cast<float*>(b + L.csuf);
  p.cmask = reinterpret_cast<uint32_t*>(b + L.cmask);
  p.midl = reinterpret_cast<uint32_t*>(b + L.midl);
  p.bwm = reinterpret_cast<uint32_t*>(b + L.bwm);
  p.bq = reinterpret_cast<uint2*>(b + L.bq);
  p.bq_cap0 = L.bq_cap0;
  p.bq_capk = L.bq_capk;
  return p;
}

// ---------------------------------------------------------------------------
// Binary32 binning arithmetic.  Every operation below is a single correctly
// rounded IEEE operation (the __f*_rn intrinsics forbid contraction into
// FMA), so the binning decision and the depth key are a fixed function of the
// FP32 inputs.  Transcendentals are replaced by fixed polynomials:
//   exp: x = k ln2 + r (ln2 = 0x1.62e4p-1 + 0x1.7f7d1cp-20), e^r by its
//        Taylor series through r^7, then an exact scaling by 2^k;
//   sin / cos on [-pi/2, pi/2]: Taylor series through x^11 / x^12.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float fsqrt(float a) { return __fsqrt_rn(a); }

__device__ __forceinline__ float bin_exp(float x) {
  if (!(x < 80.0f)) x = 80.0f;
  if (x < -80.0f) x = -80.0f;
  const float kf = rintf(fmul(x, 0x1.715476p+0f));
  float r = fsub(x, fmul(kf, 0x1.62e4p-1f));
  r = fsub(r, fmul(kf, 0x1.7f7d1cp-20f));
  float p = 0x1.a01a02p-13f;
  p = fadd(fmul(p, r), 0x1.6c16c2p-10f);
  p = fadd(fmul(p, r), 0x1.111112p-7f);
  p = fadd(fmul(p, r), 0x1.555556p-5f);
  p = fadd(fmul(p, r), 0x1.555556p-3f);
  p = fadd(fmul(p, r), 0.5f);
  p = fadd(fmul(p, r), 1.0f);
  p = fadd(fmul(p, r), 1.0f);
  const int k = static_cast<int>(kf);
  return fmul(p, __int_as_float((k + 127) << 23));
}

__device__ __forceinline__ float bin_sin(float x) {
  const float x2 = fmul(x, x);
  float p = -0x1.ae6456p-26f;
  p = fadd(fmul(p, x2), 0x1.71de3ap-19f);
  p = fsub(fmul(p, x2), 0x1.a01a02p-13f);
  p = fadd(fmul(p, x2), 0x1.111112p-7f);
  p = fsub(fmul(p, x2), 0x1.555556p-3f);
  p = fmul(p, x2);
  return fadd(fmul(p, x), x);
}

__device__ __forceinline__ float bin_cos(float x) {
  const float x2 = fmul(x, x);
  float p = 0x1.1eed8ep-29f;
  p = fsub(fmul(p, x2), 0x1.27e4fcp-22f);
  p = fadd(fmul(p, x2), 0x1.a01a02p-16f);
  p = fsub(fmul(p, x2), 0x1.6c16c2p-10f);
  p = fadd(fmul(p, x2), 0x1.555556p-5f);
  p = fsub(fmul(p, x2), 0.5f);
  return fadd(fmul(p, x2), 1.0f);
}

// elevation of pixel row r (row 0 at the top)
__device__ __forceinline__ float bin_row_elev(int r, int H, float emin, float emax) {
  const float dth = fdiv(fsub(emax, emin), static_cast<float>(H));
  return fsub(emax, fmul(fadd(static_cast<float>(r), 0.5f), dth));
}

// (cos, sin) of the azimuth 2 pi (2c+1)/(2W) of pixel column c
__device__ __forceinline__ void bin_col_dir(int c, int W, float& cs, float& sn) {
  const float f = fdiv(static_cast<float>(2 * c + 1), static_cast<float>(2 * W));
  int k = static_cast<int>(fmul(f, 4.0f));
  k = k > 3 ? 3 : k;
  const float rq = fsub(f, fmul(static_cast<float>(k), 0.25f));
  const float x = fmul(rq, 0x1.921fb6p+2f);
  const float s0 = bin_sin(x), c0 = bin_cos(x);
  switch (k) {
    case 0: cs = c0; sn = s0; break;
    case 1: cs = -s0; sn = c0; break;
    case 2: cs = -c0; sn = -s0; break;
    default: cs = s0; sn = -c0; break;
  }
}

// Bounding cone of one surfel in one frame.
struct BinGeom {
  float x, y, z, r, h, rho, sin_hi, sin_lo;
  bool all_rows, all_cols;
};

__device__ __forceinline__ void bin_geom(const float* __restrict__ mw, const float* __restrict__ ls,
                                         const FrameDev& F, BinGeom& g) {
  const float dx = fsub(mw[0], F.o[0]), dy = fsub(mw[1], F.o[1]), dz = fsub(mw[2], F.o[2]);
  g.x = fadd(fadd(fmul(F.R[0], dx), fmul(F.R[3], dy)), fmul(F.R[6], dz));
  g.y = fadd(fadd(fmul(F.R[1], dx), fmul(F.R[4], dy)), fmul(F.R[7], dz));
  g.z = fadd(fadd(fmul(F.R[2], dx), fmul(F.R[5], dy)), fmul(F.R[8], dz));
  const float h2 = fadd(fmul(g.x, g.x), fmul(g.y, g.y));
  const float r2 = fadd(h2, fmul(g.z, g.z));
  g.r = fsqrt(r2);
  g.h = fsqrt(h2);
  const float sm = ls[0] >= ls[1] ? ls[0] : ls[1];
  const float s = bin_exp(sm);
  g.rho = fadd(fmul(fmul(3.0f, s), 1.0001f), fmul(1e-5f, fadd(g.r, 1.0f)));
  g.all_rows = false;
  g.all_cols = false;
  g.sin_hi = 2.0f;
  g.sin_lo = -2.0f;
  const float rr = fsub(r2, fmul(g.rho, g.rho));
  if (!(rr > 0.0f)) {
    g.all_rows = true;
    g.all_cols = true;
    return;
  }
  const float c = fsqrt(rr);
  const float hc = fmul(g.h, c), zp = fmul(g.z, g.rho), zc = fmul(g.z, c), hp = fmul(g.h, g.rho);
  const bool north = hc <= zp, south = hc <= -zp;
  g.sin_hi = north ? 2.0f : fdiv(fadd(zc, hp), r2);
  g.sin_lo = south ? -2.0f : fdiv(fsub(zc, hp), r2);
  g.all_cols = north || south;
}

__device__ __forceinline__ bool bin_row_hit(const BinGeom& g, float s_top, float s_bot) {
  return g.all_rows || (s_bot <= g.sin_hi && s_top >= g.sin_lo);
}

__device__ __forceinline__ bool bin_dir_in_cap(const BinGeom& g, float cs, float sn) {
  const float dt = fadd(fmul(g.x, cs), fmul(g.y, sn));
  const float cr = fsub(fmul(g.x, sn), fmul(g.y, cs));
  return dt > 0.0f && fabsf(cr) <= g.rho;
}

__device__ __forceinline__ bool bin_col_hit(const BinGeom& g, float4 c) {
  if (g.all_cols) return true;
  if (bin_dir_in_cap(g, c.x, c.y) || bin_dir_in_cap(g, c.z, c.w)) return true;
  return fsub(fmul(c.x, g.y), fmul(c.y, g.x)) >= 0.0f && fsub(fmul(g.x, c.w), fmul(g.y, c.z)) >= 0.0f;
}

// Candidate tile columns, as up to two inclusive ranges [a0,a1] and [b0,b1]
// (b empty when b0 > b1), guaranteed to contain every column bin_col_hit
// accepts: the cone's azimuth interval widened by two pixel columns on each
// side, split at the azimuth seam.  Not part of the binning definition; it
// only prunes the search.
struct ColWin {
  int a0, a1, b0, b1;
};

__device__ __forceinline__ void bin_col_window(const BinGeom& g, const FrameDev& F, ColWin& w) {
  w.b0 = 1;
  w.b1 = 0;
  w.a0 = 0;
  w.a1 = F.ntc - 1;
  if (g.all_cols) return;
  const float two_pi = 6.283185307f;
  float phic = atan2f(g.y, g.x);
  if (phic < 0.0f) phic += two_pi;
  const float dphi = asinf(fminf(g.rho / g.h, 1.0f));
  const float cpr = static_cast<float>(F.W) / two_pi;  // pixel columns per radian
  const int cl = static_cast<int>(floorf((phic - dphi) * cpr - 0.5f)) - 2;
  const int ch = static_cast<int>(ceilf((phic + dphi) * cpr - 0.5f)) + 2;
  if (ch - cl + 1 >= F.W - 2 * F.tw) return;  // nearly everything: take all columns
  if (cl < 0) {
    w.a0 = (cl + F.W) / F.tw; w.a1 = F.ntc - 1; w.b0 = 0; w.b1 = ch / F.tw;
  } else if (ch >= F.W) {
    w.a0 = cl / F.tw; w.a1 = F.ntc - 1; w.b0 = 0; w.b1 = (ch - F.W) / F.tw;
  } else {
    w.a0 = cl / F.tw; w.a1 = ch / F.tw;
  }
}

// Conservative pixel-space box of the bounding cone: rows [x, y] (floats),
// columns as a circular centre z and half-width w, padded by one pixel.  It
// only prunes searches (a warp skips records that cannot pass the cut-off at
// any of its pixels; the binning tests only the tile rows it spans); results
// never depend on it.
__device__ __forceinline__ float4 pixel_box(const BinGeom& g, const FrameDev& F) {
  float r_lo = 0.f, r_hi = static_cast<float>(F.H - 1);
  if (!g.all_rows) {
    const float dth = (F.emax - F.emin) / static_cast<float>(F.H);
    const float th_hi = asinf(fminf(fmaxf(g.sin_hi, -1.f), 1.f));
    const float th_lo = asinf(fminf(fmaxf(g.sin_lo, -1.f), 1.f));
    r_lo = fmaxf(floorf((F.emax - th_hi) / dth - 0.5f) - 1.f, 0.f);
    r_hi = fminf(ceilf((F.emax - th_lo) / dth - 0.5f) + 1.f, static_cast<float>(F.H - 1));
  }
  float cc = 0.f, chw = static_cast<float>(F.W);
  if (!g.all_cols) {
    const float two_pi = 6.283185307f;
    float phic = atan2f(g.y, g.x);
    if (phic < 0.f) phic += two_pi;
    const float dphi = asinf(fminf(g.rho / g.h, 1.f));
    const float cpr = static_cast<float>(F.W) / two_pi;
    cc = phic * cpr - 0.5f;
    chw = dphi * cpr + 1.5f;
  }
  return make_float4(r_lo, r_hi, cc, chw);
}

// Culling box of the compositing kernels: the pixels whose centre ray can
// meet the surfel's 3-sigma disc {mu + A c + B s : c^2 + s^2 <= 1}, A = 3 s_u
// t_u, B = 3 s_v t_v (sensor frame), intersected with the bounding-sphere box
// sb (same column centre).  Over the disc, sin(elevation) g(p) = p_z / |p|
// and the azimuth phi(p) = atan2(p_y, p_x) are bounded by their first-order
// terms, whose maximum over the disc is |(grad . A, grad . B)|, plus the
// Taylor remainder: |x^T H x| <= 3 |x|^2 / |p|^2 for g and |x|^2 / h^2 for phi
// (h the distance from the z axis), so with rho >= |A c + B s| the remainder
// is at most 1.5 rho^2 / (|mu| - rho)^2, resp. 0.5 rho^2 / (h - rho)^2.  The
// disc is widened by 0.1 % and the pixel bounds by 0.02 pixels for binary32
// rounding.  Only the compositing kernels read this box; binning keeps the
// sphere box.
__device__ __forceinline__ float4 cull_box(const BinGeom& g, const FrameDev& F, const float4& sb, float tux,
                                           float tuy, float tuz, float tvx, float tvy, float tvz, float su,
                                           float sv) {
  float4 b = sb;
  const float ka = 3.003f * su, kb = 3.003f * sv;
  const float Ax = ka * tux, Ay = ka * tuy, Az = ka * tuz;
  const float Bx = kb * tvx, By = kb * tvy, Bz = kb * tvz;
  const float rho = fmaxf(ka, kb) * 1.001f;
  const float r = g.r;
  if (!g.all_rows && r > 1.01f * rho) {
    const float ir = 1.0f / r;
    const float g0 = g.z * ir;
    // grad g = (z_hat - g0 p_hat) / |p|
    const float gx = -g0 * g.x * ir * ir, gy = -g0 * g.y * ir * ir, gz = (1.0f - g0 * g.z * ir) * ir;
    const float la = gx * Ax + gy * Ay + gz * Az, lb = gx * Bx + gy * By + gz * Bz;
    const float d = r - rho;
    const float ext = sqrtf(la * la + lb * lb) * 1.001f + 1.5f * rho * rho / (d * d);
    const float s_hi = g0 + ext, s_lo = g0 - ext;
    const float dth = (F.emax - F.emin) / static_cast<float>(F.H);
    if (s_hi < 1.0f && s_lo > -1.0f) {
      // rows whose centre elevation emax - (r + 1/2) dth lies in the band
      const float rl = ceilf((F.emax - asinf(s_hi)) / dth - 0.52f);
      const float rh = floorf((F.emax - asinf(s_lo)) / dth - 0.48f);
      b.x = fmaxf(b.x, rl);
      b.y = fminf(b.y, rh);
    }
  }
  if (!g.all_cols && g.h > 1.01f * rho) {
    const float ih2 = 1.0f / (g.h * g.h);
    // grad phi = (-y, x, 0) / h^2
    const float la = (g.x * Ay - g.y * Ax) * ih2, lb = (g.x * By - g.y * Bx) * ih2;
    const float d = g.h - rho;
    const float half = sqrtf(la * la + lb * lb) * 1.001f + 0.5f * rho * rho / (d * d);
    if (half < 3.0f) {
      const float cpr = static_cast<float>(F.W) / 6.283185307f;
      b.w = fminf(b.w, half * cpr + 0.02f);
    }
  }
  return b;
}

// Pixel of a thread inside its tile: 4 x 8 pixel blocks per warp when the
// tile shape allows, row-major otherwise.
__device__ __forceinline__ void pixel_of_thread(const FrameDev& F, int tid, int& lr, int& lc) {
  if ((F.tw & 7) == 0 && (F.th & 3) == 0) {
    const int w = tid >> 5, lane = tid & 31, wpr = F.tw >> 3;
    lr = (w / wpr) * 4 + (lane >> 3);
    lc = (w % wpr) * 8 + (lane & 7);
  } else {
    lr = tid / F.tw;
    lc = tid % F.tw;
  }
}

// The pixel block of a warp: rows [r0, r1], columns centred on cmid with
// half-width chalf (an empty block when no lane is inside the frame).
struct WarpBox {
  float r0, r1, cmid, chalf, W;
};

__device__ __forceinline__ WarpBox warp_box(bool inside, int r, int c, int W) {
  const int rmin = __reduce_min_sync(0xffffffffu, inside ? r : 0x7fffffff);
  const int rmax = __reduce_max_sync(0xffffffffu, inside ? r : -1);
  const int cmin = __reduce_min_sync(0xffffffffu, inside ? c : 0x7fffffff);
  const int cmax = __reduce_max_sync(0xffffffffu, inside ? c : -1);
  WarpBox b;
  b.r0 = static_cast<float>(rmin);
  b.r1 = static_cast<float>(rmax);
  b.cmid = 0.5f * (static_cast<float>(cmin) + static_cast<float>(cmax));
  b.chalf = 0.5f * (static_cast<float>(cmax) - static_cast<float>(cmin));
  b.W = static_cast<float>(W);
  return b;
}

__device__ __forceinline__ bool box_hits(const float4& b, const WarpBox& w) {
  if (b.x > w.r1 || b.y < w.r0) return false;
  float d = b.z - w.cmid;
  d -= w.W * rintf(d / w.W);
  return fabsf(d) <= b.w + w.chalf;
}

// ---------------------------------------------------------------------------
// Compositing record (4 x float4 = 64 B per item):
//   r0 = (n, h = n.mu), r1 = (a_u = t_u/s_u, b_u = t_u.mu/s_u),
//   r2 = (a_v, b_v), r3 = (alpha, s_u, s_v, 0); sensor frame.
// Then for a unit ray d: den = n.d, t = h/den, u = t (a_u.d) - b_u,
// v = t (a_v.d) - b_v.
// ---------------------------------------------------------------------------
// Tiles whose list is longer than this are composited by the entry-parallel
// per-pixel kernels instead of the per-tile ones (their pixels would walk the
// whole list one entry at a time).
constexpr uint32_t kLongList = 4096;

// Backward work unit of the chunked walk: kChunk consecutive entries of a
// tile list.  The forward records, per pixel, at the end of every chunk the
// transmittance and the chunk's own sums of w, w t and w n' (a checkpoint of
// six floats), so every chunk's reverse walk can start on its own.
constexpr uint32_t kChunk = 128;
// Floats of a checkpoint per (chunk, pixel): T at the chunk end and the
// chunk's own sums of w, w t and w n.
constexpr int kCkptSlots = 6;

struct Eval {
  float den, rden, t, ud, vd, u, v, q, G, araw, a;
  bool valid;
};

// Hardware reciprocal and base-2 exponential (PTX rcp.approx.ftz.f32,
// ex2.approx.ftz.f32).  The flush-to-zero forms map to one MUFU instruction
// each; the IEEE-denormal forms add range fix-ups around it.  No input of
// the compositing arithmetic is near the denormal range (|n.d| >= 1e-6 on
// every accepted pair, exponents >= -4.5 log2 e).
__device__ __forceinline__ float rcp_ftz(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ float ex2_ftz(float x) {
  float r;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// exp(-q / 2) = 2^(q * (-log2(e) / 2)); -log2(e) / 2 = -1 / (2 ln 2).
constexpr float kNegHalfLog2e = -0.72134752044448170368f;

// One ray / surfel evaluation, arithmetic pinned (explicit fma / rounded mul)
// so the forward and backward kernels take identical skip decisions.
__device__ __forceinline__ void eval_pair(const float4& r0, const float4& r1, const float4& r2,
                                          float alpha, float dx, float dy, float dz, Eval& e) {
  e.den = __fmaf_rn(r0.z, dz, __fmaf_rn(r0.y, dy, __fmul_rn(r0.x, dx)));
  e.rden = rcp_ftz(e.den);
  e.t = __fmul_rn(r0.w, e.rden);
  e.ud = __fmaf_rn(r1.z, dz, __fmaf_rn(r1.y, dy, __fmul_rn(r1.x, dx)));
  e.vd = __fmaf_rn(r2.z, dz, __fmaf_rn(r2.y, dy, __fmul_rn(r2.x, dx)));
  e.u = __fmaf_rn(e.t, e.ud, -r1.w);
  e.v = __fmaf_rn(e.t, e.vd, -r2.w);
  e.q = __fmaf_rn(e.u, e.u, __fmul_rn(e.v, e.v));
  e.G = ex2_ftz(__fmul_rn(kNegHalfLog2e, e.q));
  e.araw = __fmul_rn(alpha, e.G);
  e.a = fminf(e.araw, 0.99f);
  e.valid = (fabsf(e.den) >= 1e-6f) && (e.t > 0.2f) && (e.q <= 9.0f) && (e.a >= (1.0f / 255.0f));
}

// Unit ray of pixel (r, c) (accuracy only, not part of any bit-exact contract).
__device__ __forceinline__ void pixel_ray(const FrameDev& F, int r, int c, float& dx, float& dy, float& dz) {
  const float th = F.emax - (static_cast<float>(r) + 0.5f) * ((F.emax - F.emin) / static_cast<float>(F.H));
  float st, ct, sp, cp;
  sincosf(th, &st, &ct);
  sincospif((2.0f * static_cast<float>(c) + 1.0f) / static_cast<float>(F.W), &sp, &cp);
  dx = ct * cp;
  dy = ct * sp;
  dz = st;
}

// Loss sums in 64-bit fixed point.  Every per-pixel (or per-surfel) term is
// rounded once to a fixed grid and the sums are integer additions, exact in
// any order: CTAs accumulate with atomics and the result is still
// deterministic, and no FP64 arithmetic is involved (FP64 is slow on this
// part).  Grids: depth L1 and the scale regulariser in 2^-32 m (the sum of a
// 262,144-pixel frame holds a mean error of 8 km per pixel; the regulariser
// is summed with at most 1 km per surfel), the opacity and normal terms in
// 2^-40 (at most 13.8 and 2 per pixel).
constexpr float kFixD = 4294967296.0f;        // 2^32
constexpr float kFixU = 1099511627776.0f;     // 2^40

__device__ __forceinline__ long long to_fix(float v, float grid) { return __float2ll_rn(v * grid); }

// Mean of a loss term from its fixed-point sum over n pixels (0 for an
// empty mask), in binary32.
__device__ __forceinline__ float fix_mean(long long sum, float grid, int n) {
  return n ? (static_cast<float>(sum) / grid) / static_cast<float>(n) : 0.0f;
}

// Image terms of one pixel (Eqs. depthloss and normalloss without the N_surf
// term, Eq. totalloss weights): masked L1 depth, positive BCE opacity,
// cosine normal against N_gicp.  Adds the terms' fixed-point values to ld,
// la, ln and returns dL/d(A, S_t, S_n) (scaled by `scale` = 1 / frames of the
// map) in g.  Every loss path (the loss kernel, the forward epilogues, the
// allocation-free loss) calls this one function, so their bits agree.
__device__ __forceinline__ void pixel_image_loss(float Dm, float A, float St, float nx, float ny, float nz, float sx,
                                                 float sy, float sz, float scale, float ind, float inn,
                                                 const lgs_loss_params& P, float (&g)[5], long long& ld,
                                                 long long& la, long long& ln) {
  g[0] = g[1] = g[2] = g[3] = g[4] = 0.f;
  if (!(Dm > 0.f)) return;
  const float a = A + 1e-6f;
  const float Dh = St / a;
  const float diff = Dh - Dm;
  ld += to_fix(fabsf(diff), kFixD);
  const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
  const float gDh = sgn * ind;
  g[1] = scale * gDh / a;
  g[0] = scale * (-gDh * St / (a * a));
  // log(A + 1e-6): for A >= 1/2 as log1p((A - 1) + 1e-6), where A - 1 is
  // exact, so opacities near 1 keep their precision; below 1/2 directly,
  // where A + 1e-6 is exact to half an ulp
  la += to_fix(-(A >= 0.5f ? log1pf((A - 1.0f) + 1e-6f) : logf(A + 1e-6f)), kFixU);
  g[0] -= scale * P.lambda_alpha * ind / (A + 1e-6f);
  if (nx * nx + ny * ny + nz * nz > 0.f) {
    const float m = sqrtf(sx * sx + sy * sy + sz * sz + 1e-12f);
    const float im = 1.f / m;
    ln += to_fix(1.0f - (sx * nx + sy * ny + sz * nz) * im, kFixU);
    const float k = -P.lambda_n * P.lambda_ng * inn;
    const float g0 = k * nx, g1 = k * ny, g2 = k * nz;
    const float sg = (sx * g0 + sy * g1 + sz * g2) * im * im * im;
    g[2] = scale * (g0 * im - sx * sg);
    g[3] = scale * (g1 * im - sy * sg);
    g[4] = scale * (g2 * im - sz * sg);
  }
}

// Sum of v over the CTA (any order), then one atomic add into acc by
// thread 0.  Every thread of the CTA calls it; s_ll holds a value per warp.
__device__ __forceinline__ void cta_add_fix(long long v, unsigned long long* acc, long long* s_ll) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_ll[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += s_ll[w];
    if (t) atomicAdd(acc, static_cast<unsigned long long>(t));
  }
}

// Loss vector (Eq. totalloss) from the fixed-point totals of a loss call:
// per frame the means of its terms, per map the frames' image terms over its
// frame count plus lambda_s times its regulariser sum, and the total; then
// the totals, the mask counts and the ticket are cleared for the next call.
// Run by the first warp of the CTA that finished last (after a fence).
__device__ __forceinline__ void finish_loss_vector(const Desc& D, const lgs_loss_params& P, int* ctot,
                                                   unsigned long long* acc, float* out, Status* st) {
  __shared__ float s_fr[LGS_MAX_FRAMES];
  const int lane = threadIdx.x & 31;
  __threadfence();
  if (lane == 0) st->loss_ticket = 0;
  const int nf = D.n_frames, nmap = D.n_maps;
  for (int f = lane; f < nf; f += 32) {
    const int nd = __ldcg(ctot + 2 * f), nn = __ldcg(ctot + 2 * f + 1);
    const unsigned long long* a = acc + 4 * f;
    const float Ld = fix_mean(static_cast<long long>(__ldcg(a)), kFixD, nd);
    const float La = fix_mean(static_cast<long long>(__ldcg(a + 1)), kFixU, nd);
    const float Ln = fix_mean(static_cast<long long>(__ldcg(a + 2)), kFixU, nn);
    const float Ls = fix_mean(static_cast<long long>(__ldcg(a + 3)), kFixU, nd);
    float* o = out + 1 + LGS_LOSS_TERMS * f;
    o[0] = Ld;
    o[1] = La;
    o[2] = Ln;
    o[3] = Ls;
    s_fr[f] = (Ld + P.lambda_alpha * La + P.lambda_n * P.lambda_ng * Ln + P.lambda_n * P.lambda_ns * Ls) /
              static_cast<float>(D.m[D.f[f].map].n_frames);
  }
  __syncwarp();
  if (lane == 0) {
    float Lmap[LGS_MAX_MAPS];
    for (int m = 0; m < nmap; ++m) Lmap[m] = 0.0f;
    for (int f = 0; f < nf; ++f) Lmap[D.f[f].map] += s_fr[f];
    float L = 0.0f;
    for (int m = 0; m < nmap; ++m) {
      const long long sr = static_cast<long long>(__ldcg(acc + 4 * LGS_MAX_FRAMES + m));
      Lmap[m] += P.lambda_s * (static_cast<float>(sr) / kFixD);
      out[1 + LGS_LOSS_TERMS * nf + m] = Lmap[m];
      L += Lmap[m];
    }
    out[0] = L;
  }
  __syncwarp();
  for (int f = lane; f < nf; f += 32) {
    ctot[2 * f] = 0;
    ctot[2 * f + 1] = 0;
    for (int k = 0; k < 4; ++k) acc[4 * f + k] = 0ull;
  }
  for (int m = lane; m < nmap; m += 32) acc[4 * LGS_MAX_FRAMES + m] = 0ull;
}

// Frame of a global tile id (binary search over the frames' tile bases).
__device__ __forceinline__ int frame_of_tile(const Desc& D, uint32_t tile) {
  int lo = 0, hi = D.n_frames - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (D.f[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int frame_of_item(const Desc& D, int64_t item) {
  int lo = 0, hi = D.n_frames - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (D.f[mid].item_base <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Host-side launchers (one per translation unit).
// ---------------------------------------------------------------------------
cudaError_t launch_write_desc(const Desc& h, Desc* d, Status* st, cudaStream_t s);
// A second stream with its fork and join events (owned by a session).
struct SideStream {
  cudaStream_t s;
  cudaEvent_t fork, join;
};
cudaError_t launch_bin(const Layout& L, const WsPtrs& w, int n_frames, int64_t n_items, uint32_t n_tiles,
                       const SideStream& side, cudaStream_t s);
int bin_kernel_count(uint32_t n_tiles);
// the tile of every pair of the last binning into w.ptile (on request only)
cudaError_t launch_fill_tile_of_pair(const WsPtrs& w, uint32_t n_tiles, cudaStream_t s);
cudaError_t launch_raster_fwd(const Layout& L, const WsPtrs& w, const Desc& h, const uint32_t* pv, int batch, int group,
                              int persistent, cudaStream_t s);
// chunked: the forward was the shared-memory walk, which wrote the chunk
// checkpoints the chunked backward starts from.
cudaError_t launch_raster_bwd(const Layout& L, const WsPtrs& w, const Desc& h, const uint32_t* pv, int batch, int group,
                              int persistent, bool chunked, cudaStream_t s);
size_t loss_part_bytes();
// mask counts [frame][2] inside the loss accumulators
inline int* loss_counts_ptr(const WsPtrs& w) {
  return reinterpret_cast<int*>(reinterpret_cast<unsigned long long*>(w.loss_part) + 4 * LGS_MAX_FRAMES +
                                LGS_MAX_MAPS);
}
// map management (lgs_manage.cu)
struct MgHostParams {
  lgs_manage_params p;
  float logit_prune, logit_min;   // binary32 logits of alpha_prune, alpha_min
};
size_t manage_scratch_bytes(int64_t n);
int manage_kernel_count(int n_passes);
cudaError_t launch_manage(const lgs_surfels& M, const float* lam, const float* res, const MgHostParams& H,
                          void* scratch, float* score, const lgs_surfel_params_out& out, int64_t capacity,
                          int32_t* src, uint8_t* role, int64_t* counts, cudaStream_t s);
cudaError_t launch_manage_gather(const int32_t* src, const uint8_t* role, const int64_t* counts, int64_t capacity,
                                 const void* in, void* out, int words, int zero_children, cudaStream_t s);

// exclusive scan of uint32 (out[len] = total; in may equal out; part holds
// scan_partials_bytes(len) bytes), defined in lgs_manage.cu
size_t scan_partials_bytes(uint64_t len);
void exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint32_t len, uint32_t* part, cudaStream_t s);

// keyframe initialisation (lgs_init.cu)
size_t init_scratch_bytes(int64_t n);
int64_t init_max_points();
int init_launches();
cudaError_t launch_keyframe_init(const float* pts, int64_t n, const float pose[12], const lgs_init_params& p,
                                 void* scratch, int32_t* knn, const lgs_surfel_params_out& out, float* lam,
                                 float* conf, int64_t* pairs, cudaStream_t s);

size_t trackable_scratch_bytes(int64_t n);
cudaError_t launch_trackable(const lgs_surfels& M, const uint8_t* mask, const int32_t* last_kf, int32_t k_min,
                             float logit_min, float thick, float eps, float w_max, void* scratch, int32_t* index,
                             float* mean, float* cov, float* weight, int64_t* count, cudaStream_t s);
cudaError_t launch_raster_fwd_loss(const WsPtrs& w, const Desc& h, const uint32_t* pv, int persistent,
                                   const lgs_loss_params& p, float* loss_out, cudaStream_t s);
cudaError_t launch_loss_counts(const WsPtrs& w, const Desc& h, const lgs_loss_params& p, bool scale_grad,
                               cudaStream_t s);
size_t noalloc_scratch_bytes();
cudaError_t noalloc_scratch(void** out);
cudaError_t launch_image_loss_noalloc(void* scratch, int n_frames, const int32_t* H, const int32_t* W,
                                      const lgs_fwd_out* fwd, const lgs_target* targets,
                                      const lgs_loss_params& P, const lgs_fwd_grad_out* grads_out, float* loss_out,
                                      cudaStream_t s);
cudaError_t launch_preprocess_bwd(const Layout& L, const WsPtrs& w, const Desc& h, cudaStream_t s);
cudaError_t launch_loss(const Layout& L, const WsPtrs& w, const Desc& h, const lgs_loss_params& p,
                        bool scale_grad, float* loss_out, cudaStream_t s);
cudaError_t launch_adam_batch(const lgs_adam_map* maps, int n_maps, float b1, float b2, float eps, int zero_grad,
                              cudaStream_t s);
cudaError_t launch_adam(float* p[4], float* g[4], float* m[4], float* v[4], const int64_t cnt[4],
                        int64_t step, const float lr[4], float b1, float b2, float eps, int zero_grad,
                        cudaStream_t s);

}  // namespace lgs
