// lgs_manage.cu -- map management on the device: the control score (paper
// Sec. 3.3, Eq. controlscore), opacity pruning (the baseline of Table 4), the
// multi-pass planar cover-and-prune and the structure-aware adaptive split
// (Sec. 3.5, "Real-time Map Budget Control for Long Sequences").
//
// Every decision is an integer outcome of floating point, so it is specified
// in binary32: each operation a single correctly rounded IEEE operation in a
// fixed order (the f* helpers forbid FMA contraction) and the scales through
// the fixed polynomial exponential of binning.  The result is then a fixed
// function of the inputs, whatever the launch shape or the order of atomics.
//
// Quantiles (the lower order statistic sorted[floor(q (n - 1))]) and caps (the
// first k of an order) are exact: an 8-bit radix select over 64-bit keys
// finds the k-th smallest key, one histogram launch and one one-CTA pick per
// digit.  Groups of a cover-and-prune pass live in an open-addressing hash
// table keyed by the biased 2D voxel; the representative (largest logit,
// then lowest index) is an atomicMax over a packed key; members scatter their
// squared cover radii into per-group buckets, and each member decides alone
// whether it is inside its group's cover region by counting its bucket's
// strictly smaller radii (the decision equals "radius <= the k-th smallest").
//
// Launches (one stream, no host synchronisation, counts written on the
// device): init; residual quantile; score and opacity prune; per pass: the
// survivors' score quantile, table clear, insert, measure, bucket scan,
// scatter, decide, cap select, apply; then the split quantile, split keys,
// split cap select, weights, output scan, write.
#include <cuda_runtime.h>

#include <cmath>

#include "lgs_internal.cuh"

namespace lgs {
namespace {

constexpr int kMgCta = 256;
constexpr unsigned long long kNoKey = ~0ull;
constexpr int kScanCta = 1024;
constexpr int kScanItems = 4;
constexpr uint32_t kScanBlock = kScanCta * kScanItems;
// groups up to this many members decide by counting; larger ones get the
// k-th smallest radius from a one-CTA radix select
constexpr uint32_t kSmallGroup = 256;

enum : uint32_t { kAlive = 1u, kCand = 2u, kMember = 4u, kFlag = 8u, kSplit = 16u };
enum : uint32_t { kSelNone = 0u, kSelAll = 1u, kSelKth = 2u };

// State of one radix select.  count accumulates the keys taking part (reset
// by the setup kernel that reads it); base is the number of survivors a cap is
// a fraction of; after the last digit prefix is the selected key.
struct Sel {
  unsigned long long prefix;
  uint32_t count;
  uint32_t k;
  uint32_t kind;
  uint32_t base;
  uint32_t n_big;              // groups of the current pass with more than kSmallGroup members
  uint32_t hist[256];
};

struct MgScratch {
  Sel* sel;
  uint32_t* flags;             // [n] kAlive | kCand | kMember | kFlag | kSplit
  unsigned long long* key;     // [n] select keys (kNoKey: not taking part)
  uint32_t* slot;              // [n] hash slot of a candidate's group
  uint32_t* r2;                // [n] a member's squared cover radius (float bits)
  uint32_t* pos;               // [n + 1] output weights, then their exclusive scan
  uint32_t* bucket;            // [n] members' radii grouped by slot
  unsigned long long* htab;    // [T] voxel keys (kNoKey: empty)
  unsigned long long* rep;     // [T] packed representative: order key of the logit << 32 | ~index
  uint32_t* cnt;               // [T] members per slot
  uint32_t* off;               // [T + 1] exclusive scan of cnt
  uint32_t* big;               // [n / kSmallGroup + 1] slots of the large groups
  uint32_t* part;              // scan partials
  uint32_t T;                  // table capacity (power of two >= 2 n)
};

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

uint32_t table_capacity(int64_t n) {
  uint64_t t = 1024;
  while (t < static_cast<uint64_t>(2 * n)) t <<= 1;
  return static_cast<uint32_t>(t);
}

uint32_t scan_blocks(uint64_t len) { return static_cast<uint32_t>((len + kScanBlock - 1) / kScanBlock); }

// Byte offsets of the scratch arrays; the total is the size.
struct MgLayout {
  size_t sel, flags, key, slot, r2, pos, bucket, htab, rep, cnt, off, big, part, total;
  uint32_t T;
};

MgLayout mg_layout(int64_t n) {
  MgLayout L{};
  const size_t N = static_cast<size_t>(n > 0 ? n : 1);
  L.T = table_capacity(n);
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = align_up(o + bytes, 256); return at; };
  L.sel = take(sizeof(Sel));
  L.flags = take(4 * N);
  L.key = take(8 * N);
  L.slot = take(4 * N);
  L.r2 = take(4 * N);
  L.pos = take(4 * (N + 1));
  L.bucket = take(4 * N);
  L.htab = take(8 * static_cast<size_t>(L.T));
  L.rep = take(8 * static_cast<size_t>(L.T));
  L.cnt = take(4 * static_cast<size_t>(L.T));
  L.off = take(4 * (static_cast<size_t>(L.T) + 1));
  L.big = take(4 * (N / kSmallGroup + 1));
  const uint64_t longest = static_cast<uint64_t>(L.T) + 1 > N + 1 ? static_cast<uint64_t>(L.T) + 1 : N + 1;
  L.part = take(4 * (static_cast<size_t>(scan_blocks(longest)) + 1));
  L.total = o;
  return L;
}

MgScratch mg_scratch(void* base, int64_t n) {
  const MgLayout L = mg_layout(n);
  char* b = static_cast<char*>(base);
  MgScratch s;
  s.sel = reinterpret_cast<Sel*>(b + L.sel);
  s.flags = reinterpret_cast<uint32_t*>(b + L.flags);
  s.key = reinterpret_cast<unsigned long long*>(b + L.key);
  s.slot = reinterpret_cast<uint32_t*>(b + L.slot);
  s.r2 = reinterpret_cast<uint32_t*>(b + L.r2);
  s.pos = reinterpret_cast<uint32_t*>(b + L.pos);
  s.bucket = reinterpret_cast<uint32_t*>(b + L.bucket);
  s.htab = reinterpret_cast<unsigned long long*>(b + L.htab);
  s.rep = reinterpret_cast<unsigned long long*>(b + L.rep);
  s.cnt = reinterpret_cast<uint32_t*>(b + L.cnt);
  s.off = reinterpret_cast<uint32_t*>(b + L.off);
  s.big = reinterpret_cast<uint32_t*>(b + L.big);
  s.part = reinterpret_cast<uint32_t*>(b + L.part);
  s.T = L.T;
  return s;
}

// Parameters as the kernels use them (thresholds already as binary32 logits).
struct MgParams {
  float logit_prune, logit_min;
  float w_l, w_c, w_r, q_res, eps;
  float q_plane, voxel, q_cover, slab, prune_cap;
  float q_split, split_cap, split_shift, split_dlog;
};

// ---------------------------------------------------------------------------
// binary32 helpers
// ---------------------------------------------------------------------------
// total-order key of a binary32 value (ascending with the value; -0 < +0)
__device__ __forceinline__ uint32_t okey(float x) {
  const uint32_t b = __float_as_uint(x);
  return (b >> 31) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float okey_inv(uint32_t k) {
  return __uint_as_float((k >> 31) ? (k & 0x7fffffffu) : ~k);
}

// columns of R(q) for the normalised quaternion (w, x, y, z): t_u = R e0,
// t_v = R e1, n = R e2
__device__ __forceinline__ void quat_axes(const float* q, float3& tu, float3& tv, float3& nn) {
  float w = q[0], x = q[1], y = q[2], z = q[3];
  const float r = fsqrt(fadd(fadd(fadd(fmul(w, w), fmul(x, x)), fmul(y, y)), fmul(z, z)));
  w = fdiv(w, r);
  x = fdiv(x, r);
  y = fdiv(y, r);
  z = fdiv(z, r);
  tu = make_float3(fsub(1.f, fmul(2.f, fadd(fmul(y, y), fmul(z, z)))), fmul(2.f, fadd(fmul(x, y), fmul(w, z))),
                   fmul(2.f, fsub(fmul(x, z), fmul(w, y))));
  tv = make_float3(fmul(2.f, fsub(fmul(x, y), fmul(w, z))), fsub(1.f, fmul(2.f, fadd(fmul(x, x), fmul(z, z)))),
                   fmul(2.f, fadd(fmul(y, z), fmul(w, x))));
  nn = make_float3(fmul(2.f, fadd(fmul(x, z), fmul(w, y))), fmul(2.f, fsub(fmul(y, z), fmul(w, x))),
                   fsub(1.f, fmul(2.f, fadd(fmul(x, x), fmul(y, y)))));
}

__device__ __forceinline__ float dot3(float3 a, float3 b) {
  return fadd(fadd(fmul(a.x, b.x), fmul(a.y, b.y)), fmul(a.z, b.z));
}

__device__ __forceinline__ uint32_t voxel_index(float m, float voxel) {
  float g = floorf(fdiv(m, voxel));
  g = g < -1073741824.f ? -1073741824.f : (g > 1073741824.f ? 1073741824.f : g);
  return static_cast<uint32_t>(static_cast<int>(g) + (1 << 30));   // biased into [0, 2^31]
}

__device__ __forceinline__ unsigned long long mix64(unsigned long long x) {
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// warp-aggregated count into a 32-bit or 64-bit counter
__device__ __forceinline__ void warp_count(bool pred, uint32_t* ctr) {
  const uint32_t b = __ballot_sync(0xffffffffu, pred);
  if ((threadIdx.x & 31) == 0 && b) atomicAdd(ctr, static_cast<uint32_t>(__popc(b)));
}
__device__ __forceinline__ void warp_count64(bool pred, int64_t* ctr) {
  const uint32_t b = __ballot_sync(0xffffffffu, pred);
  if ((threadIdx.x & 31) == 0 && b)
    atomicAdd(reinterpret_cast<unsigned long long*>(ctr), static_cast<unsigned long long>(__popc(b)));
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 (out[len] = total; in may equal out)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* s_warp, uint32_t& total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) s_warp[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    uint32_t w = lane < nw ? s_warp[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < nw) s_warp[lane] = w;
  }
  __syncthreads();
  total = s_warp[(blockDim.x >> 5) - 1];
  const uint32_t before = wid ? s_warp[wid - 1] : 0u;
  __syncthreads();   // s_warp may be reused by the caller
  return before + inc - v;
}

__global__ void __launch_bounds__(kScanCta) k_scan_blocks(const uint32_t* in, uint32_t* out, uint32_t len,
                                                          uint32_t* __restrict__ part) {
  __shared__ uint32_t s_warp[32];
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanBlock + static_cast<uint64_t>(threadIdx.x) * kScanItems;
  uint32_t v[kScanItems], sum = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    v[j] = base + j < len ? in[base + j] : 0u;
    sum += v[j];
  }
  uint32_t total;
  uint32_t run = block_exclusive_scan(sum, s_warp, total);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    if (base + j < len) out[base + j] = run;
    run += v[j];
  }
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanCta) k_scan_top(uint32_t* __restrict__ part, uint32_t nb,
                                                       uint32_t* __restrict__ out, uint32_t len) {
  __shared__ uint32_t s_warp[32];
  uint32_t carry = 0;
  for (uint32_t b0 = 0; b0 < nb; b0 += kScanCta) {
    const uint32_t b = b0 + threadIdx.x;
    const uint32_t v = b < nb ? part[b] : 0u;
    uint32_t total;
    const uint32_t ex = block_exclusive_scan(v, s_warp, total);
    if (b < nb) part[b] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) out[len] = carry;
}

__global__ void __launch_bounds__(kScanCta) k_scan_add(uint32_t* __restrict__ out, uint32_t len,
                                                       const uint32_t* __restrict__ part) {
  const uint32_t add = part[blockIdx.x];
  const uint64_t base = static_cast<uint64_t>(blockIdx.x) * kScanBlock;
  for (uint32_t j = threadIdx.x; j < kScanBlock; j += kScanCta)
    if (base + j < len) out[base + j] += add;
}

void launch_scan(const uint32_t* in, uint32_t* out, uint32_t len, uint32_t* part, cudaStream_t s) {
  const uint32_t nb = scan_blocks(len);
  if (nb) k_scan_blocks<<<nb, kScanCta, 0, s>>>(in, out, len, part);
  k_scan_top<<<1, kScanCta, 0, s>>>(part, nb, out, len);
  if (nb) k_scan_add<<<nb, kScanCta, 0, s>>>(out, len, part);
}

// ---------------------------------------------------------------------------
// radix select of the k-th smallest 64-bit key
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMgCta) k_sel_hist(const unsigned long long* __restrict__ key, uint32_t n,
                                                     Sel* __restrict__ sel, int shift) {
  if (sel->kind != kSelKth) return;
  __shared__ uint32_t h[256];
  for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
  __syncthreads();
  const unsigned long long pre = sel->prefix;
  const unsigned long long hi = shift >= 56 ? 0ull : (~0ull << (shift + 8));
  const int lane = threadIdx.x & 31;
  // warp-uniform loop: every lane reaches the match; lanes with equal digits
  // add once (long runs of equal keys are common: planar scores of 0)
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    uint32_t bin = 256u;
    if (i < n) {
      const unsigned long long k = key[i];
      if (k != kNoKey && !((k ^ pre) & hi)) bin = static_cast<uint32_t>((k >> shift) & 255u);
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, bin);
    if (bin < 256u && lane == __ffs(peers) - 1) atomicAdd(&h[bin], static_cast<uint32_t>(__popc(peers)));
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += blockDim.x)
    if (h[t]) atomicAdd(&sel->hist[t], h[t]);
}

__global__ void __launch_bounds__(256) k_sel_pick(Sel* __restrict__ sel, int shift) {
  if (sel->kind != kSelKth) return;
  __shared__ uint32_t s_warp[32];
  const uint32_t k = sel->k;
  const uint32_t v = sel->hist[threadIdx.x];
  uint32_t total;
  const uint32_t ex = block_exclusive_scan(v, s_warp, total);
  if (ex <= k && k < ex + v) {
    sel->prefix |= static_cast<unsigned long long>(threadIdx.x) << shift;
    sel->k = k - ex;
  }
  sel->hist[threadIdx.x] = 0;
}

// quantile: the floor(q (count - 1))-th smallest of the keys counted
__global__ void k_sel_quantile(Sel* __restrict__ sel, float q) {
  const uint32_t c = sel->count;
  sel->base = c;
  sel->count = 0;
  sel->prefix = 0;
  if (c == 0) {
    sel->kind = kSelNone;
    return;
  }
  sel->kind = kSelKth;
  sel->k = static_cast<uint32_t>(floor(static_cast<double>(q) * static_cast<double>(c - 1)));
}

// cap: at most floor(frac * base) of the keys counted, the smallest first
__global__ void k_sel_cap(Sel* __restrict__ sel, float frac) {
  const uint32_t c = sel->count;
  const double cap = floor(static_cast<double>(frac) * static_cast<double>(sel->base));
  sel->count = 0;
  sel->prefix = 0;
  if (static_cast<double>(c) <= cap) {
    sel->kind = kSelAll;
  } else if (cap < 1.0) {
    sel->kind = kSelNone;
  } else {
    sel->kind = kSelKth;
    sel->k = static_cast<uint32_t>(cap) - 1u;
  }
}

void launch_select(const unsigned long long* key, uint32_t n, Sel* sel, int digits, int grid, cudaStream_t s) {
  for (int d = 0; d < digits; ++d) {
    const int shift = 56 - 8 * d;
    k_sel_hist<<<grid, kMgCta, 0, s>>>(key, n, sel, shift);
    k_sel_pick<<<1, 256, 0, s>>>(sel, shift);
  }
}

// selected if the select takes every key, or the key is at most the k-th
__device__ __forceinline__ bool sel_takes(uint32_t kind, unsigned long long prefix, unsigned long long k) {
  return kind == kSelAll || (kind == kSelKth && k <= prefix);
}

// ---------------------------------------------------------------------------
// kernels of the step
// ---------------------------------------------------------------------------
__global__ void k_mg_init(Sel* __restrict__ sel, uint32_t n, int64_t* __restrict__ counts) {
  for (int t = threadIdx.x; t < 256; t += blockDim.x) sel->hist[t] = 0;
  if (threadIdx.x == 0) {
    sel->prefix = 0;
    sel->count = n;      // the residual quantile takes every surfel
    sel->k = 0;
    sel->kind = kSelNone;
    sel->base = 0;
    sel->n_big = 0;
  }
  if (threadIdx.x < 6) counts[threadIdx.x] = 0;
}

__global__ void __launch_bounds__(kMgCta) k_mg_res_keys(const float* __restrict__ res, uint32_t n,
                                                        unsigned long long* __restrict__ key) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    key[i] = static_cast<unsigned long long>(okey(res[i])) << 32;
}

// Control score (Eq. controlscore) with the residual normalised by its
// quantile, and the opacity prune.
__global__ void __launch_bounds__(kMgCta) k_mg_score(const float* __restrict__ lam, const float* __restrict__ res,
                                                     const float* __restrict__ logit, uint32_t n,
                                                     const Sel* __restrict__ sel, MgParams P,
                                                     float* __restrict__ score, uint32_t* __restrict__ flags,
                                                     int64_t* __restrict__ counts) {
  const float rq = okey_inv(static_cast<uint32_t>(sel->prefix >> 32));
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const uint32_t i = i0 + threadIdx.x;
    bool dead = false;
    if (i < n) {
      float a = lam[3 * i], b = lam[3 * i + 1], c = lam[3 * i + 2];
      // descending order by compare-exchange
      if (a < b) { const float t = a; a = b; b = t; }
      if (b < c) { const float t = b; b = c; c = t; }
      if (a < b) { const float t = a; a = b; b = t; }
      const float lin = fdiv(fsub(a, b), fadd(a, P.eps));
      const float cur = fdiv(c, fadd(fadd(fadd(a, b), c), P.eps));
      float cv = fmul(3.f, cur);
      cv = cv < 1.f ? cv : 1.f;
      float rn = fdiv(res[i], fadd(rq, P.eps));
      rn = rn < 1.f ? rn : 1.f;
      float s = fadd(fadd(fmul(P.w_l, lin), fmul(P.w_c, cv)), fmul(P.w_r, rn));
      s = s < 1.f ? s : 1.f;
      s = s > 0.f ? s : 0.f;
      score[i] = s;
      const bool alive = logit[i] >= P.logit_prune;
      flags[i] = alive ? kAlive : 0u;
      dead = !alive;
    }
    warp_count64(dead, &counts[1]);
  }
}

// select keys of the survivors' scores (and the start of a pass: per-pass
// flags cleared)
__global__ void __launch_bounds__(kMgCta) k_mg_alive_keys(const float* __restrict__ score, uint32_t n,
                                                          uint32_t* __restrict__ flags,
                                                          unsigned long long* __restrict__ key, Sel* __restrict__ sel) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const uint32_t i = i0 + threadIdx.x;
    bool alive = false;
    if (i < n) {
      const uint32_t f = flags[i] & kAlive;
      flags[i] = f;
      alive = f != 0;
      key[i] = alive ? static_cast<unsigned long long>(__float_as_uint(score[i])) << 32 : kNoKey;
    }
    warp_count(alive, &sel->count);
  }
}

__global__ void __launch_bounds__(kMgCta) k_mg_clear(unsigned long long* __restrict__ htab,
                                                     unsigned long long* __restrict__ rep, uint32_t* __restrict__ cnt,
                                                     uint32_t T, Sel* __restrict__ sel) {
  if (blockIdx.x == 0 && threadIdx.x == 0) sel->n_big = 0;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < T; i += gridDim.x * blockDim.x) {
    htab[i] = kNoKey;
    rep[i] = 0ull;
    cnt[i] = 0u;
  }
}

// Planar candidates of the pass join their voxel's group; the group's
// representative is the largest (order key of the logit, then ~index).
__global__ void __launch_bounds__(kMgCta) k_mg_insert(const float* __restrict__ mean, const float* __restrict__ logit,
                                                      const float* __restrict__ score, uint32_t n,
                                                      const Sel* __restrict__ sel, MgParams P, int ax, int bx,
                                                      MgScratch S) {
  const bool any = sel->kind != kSelNone;
  const float qp = __uint_as_float(static_cast<uint32_t>(sel->prefix >> 32));
  const uint32_t mask = S.T - 1;
  const int lane = threadIdx.x & 31;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    uint32_t h = 0xffffffffu;   // no group
    unsigned long long v = 0ull;
    if (i < n) {
      S.key[i] = kNoKey;
      const float lg = logit[i];
      if (any && (S.flags[i] & kAlive) && score[i] <= qp && lg >= P.logit_min) {
        const unsigned long long hk =
            (static_cast<unsigned long long>(voxel_index(mean[3 * i + ax], P.voxel)) << 32) |
            voxel_index(mean[3 * i + bx], P.voxel);
        h = static_cast<uint32_t>(mix64(hk)) & mask;
        // the table has at least twice as many slots as surfels: a free or
        // matching slot is always found within T probes
        for (uint32_t it = 0; it < S.T; ++it) {
          const unsigned long long cur = S.htab[h];
          if (cur == hk) break;
          if (cur == kNoKey) {
            const unsigned long long prev = atomicCAS(&S.htab[h], kNoKey, hk);
            if (prev == kNoKey || prev == hk) break;
          }
          h = (h + 1) & mask;
        }
        S.slot[i] = h;
        S.flags[i] |= kCand;
        v = (static_cast<unsigned long long>(okey(lg)) << 32) | (0xffffffffu - i);
      }
    }
    // lanes of one group combine their maximum first (long planar runs put
    // thousands of surfels into one group)
    const uint32_t peers = __match_any_sync(0xffffffffu, h);
    if (h != 0xffffffffu) {
      for (uint32_t m = peers; m; m &= m - 1) {
        const unsigned long long o = __shfl_sync(peers, v, __ffs(m) - 1);
        v = o > v ? o : v;
      }
      if (lane == __ffs(peers) - 1) atomicMax(&S.rep[h], v);
    }
  }
}

// Each candidate other than its group's representative, in the
// representative's tangent frame: inside the slab it is a member with
// squared cover radius u^2 + v^2.
__global__ void __launch_bounds__(kMgCta) k_mg_measure(const float* __restrict__ mean, const float* __restrict__ quat,
                                                       const float* __restrict__ log_scale, uint32_t n, MgParams P,
                                                       MgScratch S) {
  const int lane = threadIdx.x & 31;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    uint32_t member_of = 0xffffffffu;
    if (i < n && (S.flags[i] & kCand)) {
      const uint32_t h = S.slot[i];
      const uint32_t r = 0xffffffffu - static_cast<uint32_t>(S.rep[h]);
      if (r != i) {
        float3 tu, tv, nn;
        quat_axes(quat + 4 * static_cast<size_t>(r), tu, tv, nn);
        const float su = bin_exp(log_scale[2 * r]), sv = bin_exp(log_scale[2 * r + 1]);
        const float3 d = make_float3(fsub(mean[3 * i], mean[3 * r]), fsub(mean[3 * i + 1], mean[3 * r + 1]),
                                     fsub(mean[3 * i + 2], mean[3 * r + 2]));
        const float u = fdiv(dot3(tu, d), su), v = fdiv(dot3(tv, d), sv);
        if (fabsf(dot3(nn, d)) <= P.slab) {
          S.flags[i] |= kMember;
          S.r2[i] = __float_as_uint(fadd(fmul(u, u), fmul(v, v)));
          member_of = h;
        }
      }
    }
    const uint32_t peers = __match_any_sync(0xffffffffu, member_of);
    if (member_of != 0xffffffffu && lane == __ffs(peers) - 1)
      atomicAdd(&S.cnt[member_of], static_cast<uint32_t>(__popc(peers)));
  }
}

__global__ void __launch_bounds__(kMgCta) k_mg_scatter(uint32_t n, MgScratch S) {
  const int lane = threadIdx.x & 31;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += gridDim.x * blockDim.x) {
    const uint32_t i = i0 + threadIdx.x;
    const uint32_t h = (i < n && (S.flags[i] & kMember)) ? S.slot[i] : 0xffffffffu;
    const uint32_t peers = __match_any_sync(0xffffffffu, h);
    if (h == 0xffffffffu) continue;
    const uint32_t b = S.off[h], m = S.off[h + 1] - b;
    const int lead = __ffs(peers) - 1;
    uint32_t old = 0;
    if (lane == lead) old = atomicSub(&S.cnt[h], static_cast<uint32_t>(__popc(peers)));
    old = __shfl_sync(peers, old, lead);
    // the peers take slots old-1, old-2, ... of the group's bucket
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    S.bucket[b + old - 1u - rank] = S.r2[i];
    // the first decrement of a large group lists it for the radix select
    if (lane == lead && old == m && m > kSmallGroup) S.big[atomicAdd(&S.sel->n_big, 1u)] = h;
  }
}

// k-th smallest radius of each large group by a one-CTA radix select over
// its bucket (4 digits of 8 bits); the result goes to cnt[h] (all zero after
// the scatter), read by the members in k_mg_decide.
__global__ void __launch_bounds__(kMgCta) k_mg_big_select(MgScratch S, MgParams P) {
  __shared__ uint32_t h[256];
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_pre, s_k;
  const uint32_t nb = S.sel->n_big;
  for (uint32_t g = blockIdx.x; g < nb; g += gridDim.x) {
    const uint32_t slot = S.big[g];
    const uint32_t b = S.off[slot], e = S.off[slot + 1];
    const uint32_t k = static_cast<uint32_t>(ceil(static_cast<double>(P.q_cover) * static_cast<double>(e - b)));
    if (threadIdx.x == 0) {
      s_pre = 0;
      s_k = k - 1u;
    }
    if (k == 0) {   // uniform across the CTA
      if (threadIdx.x == 0) S.cnt[slot] = 0u;   // unused: no member is covered
      __syncthreads();
      continue;
    }
    for (int shift = 24; shift >= 0; shift -= 8) {
      h[threadIdx.x] = 0;
      __syncthreads();
      const uint32_t pre = s_pre;
      const uint32_t hi = shift == 24 ? 0u : (~0u << (shift + 8));
      for (uint32_t j = b + threadIdx.x; j < e; j += blockDim.x) {
        const uint32_t x = S.bucket[j];
        if ((x ^ pre) & hi) continue;
        atomicAdd(&h[(x >> shift) & 255u], 1u);
      }
      __syncthreads();
      const uint32_t v = h[threadIdx.x];
      const uint32_t kk = s_k;
      uint32_t total;
      const uint32_t ex = block_exclusive_scan(v, s_warp, total);
      if (ex <= kk && kk < ex + v) {
        s_pre = pre | (threadIdx.x << shift);
        s_k = kk - ex;
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) S.cnt[slot] = s_pre;
    __syncthreads();
  }
}

// A member is covered when fewer than k = ceil(q_cover m) members of its
// group are strictly closer (its radius is then at most the k-th smallest).
__global__ void __launch_bounds__(kMgCta) k_mg_decide(const float* __restrict__ score, uint32_t n, MgParams P,
                                                      MgScratch S) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const uint32_t i = i0 + threadIdx.x;
    bool flagged = false;
    if (i < n && (S.flags[i] & kMember)) {
      const uint32_t h = S.slot[i];
      const uint32_t b = S.off[h], e = S.off[h + 1];
      const uint32_t k = static_cast<uint32_t>(ceil(static_cast<double>(P.q_cover) * static_cast<double>(e - b)));
      const uint32_t x = S.r2[i];
      bool covered;
      if (e - b > kSmallGroup) {
        covered = k > 0 && x <= S.cnt[h];   // the k-th smallest from k_mg_big_select
      } else {
        uint32_t less = 0;
        for (uint32_t j = b; j < e && less < k; ++j) less += S.bucket[j] < x ? 1u : 0u;
        covered = less < k;
      }
      if (covered) {
        flagged = true;
        S.flags[i] |= kFlag;
        S.key[i] = (static_cast<unsigned long long>(__float_as_uint(score[i])) << 32) | i;
      }
    }
    warp_count(flagged, &S.sel->count);
  }
}

__global__ void __launch_bounds__(kMgCta) k_mg_apply_prune(uint32_t n, MgScratch S, int64_t* __restrict__ removed) {
  const uint32_t kind = S.sel->kind;
  const unsigned long long prefix = S.sel->prefix;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const uint32_t i = i0 + threadIdx.x;
    bool rm = false;
    if (i < n && (S.flags[i] & kFlag) && sel_takes(kind, prefix, S.key[i])) {
      rm = true;
      S.flags[i] &= ~kAlive;
    }
    warp_count64(rm, removed);
  }
}

// split candidates: survivors with c >= Q_{q_split} and alpha >= alpha_min,
// keyed for "largest score first, then lowest index"
__global__ void __launch_bounds__(kMgCta) k_mg_split_keys(const float* __restrict__ logit,
                                                          const float* __restrict__ score, uint32_t n, MgParams P,
                                                          MgScratch S) {
  const bool any = S.sel->kind != kSelNone;
  const float qs = __uint_as_float(static_cast<uint32_t>(S.sel->prefix >> 32));
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const uint32_t i = i0 + threadIdx.x;
    bool cand = false;
    if (i < n) {
      const float c = score[i];
      cand = any && (S.flags[i] & kAlive) && c >= qs && logit[i] >= P.logit_min;
      S.key[i] = cand ? ((static_cast<unsigned long long>(~__float_as_uint(c)) << 32) | i) : kNoKey;
    }
    warp_count(cand, &S.sel->count);
  }
}

__global__ void __launch_bounds__(kMgCta) k_mg_weights(uint32_t n, MgScratch S) {
  const uint32_t kind = S.sel->kind;
  const unsigned long long prefix = S.sel->prefix;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint32_t f = S.flags[i];
    const bool split = (f & kAlive) && S.key[i] != kNoKey && sel_takes(kind, prefix, S.key[i]);
    if (split) f |= kSplit;
    S.flags[i] = f;
    S.pos[i] = (f & kAlive) ? (split ? 2u : 1u) : 0u;
  }
}

// The new map: survivors in ascending index, a split surfel replaced at its
// place by its children mu +- split_shift s_0 a_i (a_i = R(q_i) e0) with
// s~_0 + split_dlog.
__global__ void __launch_bounds__(kMgCta) k_mg_write(const float* __restrict__ mean, const float* __restrict__ quat,
                                                     const float* __restrict__ log_scale,
                                                     const float* __restrict__ logit, uint32_t n, MgParams P,
                                                     MgScratch S, lgs_surfel_params_out out, int64_t capacity,
                                                     int32_t* __restrict__ src, uint8_t* __restrict__ role,
                                                     int64_t* __restrict__ counts) {
  const uint32_t stride = gridDim.x * blockDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) counts[0] = S.pos[n];
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const uint32_t i = i0 + threadIdx.x;
    bool split = false;
    if (i < n && (S.flags[i] & kAlive)) {
      const uint32_t p = S.pos[i];
      split = (S.flags[i] & kSplit) != 0;
      const int copies = split ? 2 : 1;
      float3 off = make_float3(0.f, 0.f, 0.f);
      if (split) {
        float3 tu, tv, nn;
        quat_axes(quat + 4 * static_cast<size_t>(i), tu, tv, nn);
        const float a = fmul(P.split_shift, bin_exp(log_scale[2 * i]));
        off = make_float3(fmul(a, tu.x), fmul(a, tu.y), fmul(a, tu.z));
      }
      for (int c = 0; c < copies; ++c) {
        const int64_t o = static_cast<int64_t>(p) + c;
        if (o >= capacity) break;   // cannot happen for a capacity of n + floor(split_cap n)
        const float m0 = mean[3 * i], m1 = mean[3 * i + 1], m2 = mean[3 * i + 2];
        if (!split) {
          out.mean[3 * o] = m0;
          out.mean[3 * o + 1] = m1;
          out.mean[3 * o + 2] = m2;
        } else if (c == 0) {
          out.mean[3 * o] = fadd(m0, off.x);
          out.mean[3 * o + 1] = fadd(m1, off.y);
          out.mean[3 * o + 2] = fadd(m2, off.z);
        } else {
          out.mean[3 * o] = fsub(m0, off.x);
          out.mean[3 * o + 1] = fsub(m1, off.y);
          out.mean[3 * o + 2] = fsub(m2, off.z);
        }
        for (int k = 0; k < 4; ++k) out.quat[4 * o + k] = quat[4 * static_cast<size_t>(i) + k];
        out.log_scale[2 * o] = split ? fadd(log_scale[2 * i], P.split_dlog) : log_scale[2 * i];
        out.log_scale[2 * o + 1] = log_scale[2 * i + 1];
        out.opacity_logit[o] = logit[i];
        src[o] = static_cast<int32_t>(i);
        role[o] = static_cast<uint8_t>(split ? 1 + c : 0);
      }
    }
    warp_count64(split, &counts[5]);
  }
}

__global__ void __launch_bounds__(kMgCta) k_mg_gather(const int32_t* __restrict__ src, const uint8_t* __restrict__ role,
                                                      const int64_t* __restrict__ counts, int64_t capacity,
                                                      const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                      int words, int zero_children) {
  const int64_t n_out = counts[0] < capacity ? counts[0] : capacity;
  const int64_t total = n_out * words;
  for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < total;
       j += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const int64_t row = j / words;
    const int w = static_cast<int>(j - row * words);
    out[j] = (zero_children && role[row]) ? 0u : in[static_cast<int64_t>(src[row]) * words + w];
  }
}

int grid_for(uint64_t n, int sms) {
  const uint64_t want = (n + kMgCta - 1) / kMgCta;
  const uint64_t cap = static_cast<uint64_t>(sms) * 8;
  return static_cast<int>(want < 1 ? 1 : (want > cap ? cap : want));
}

int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

}  // namespace

size_t manage_scratch_bytes(int64_t n) { return mg_layout(n).total; }

int manage_kernel_count(int n_passes) {
  // init, residual keys + 4 digits, score; per pass: keys, quantile + 4
  // digits, clear, insert, measure, scan (3), scatter, large-group select,
  // decide, cap + 8 digits, apply; split: keys, quantile + 4 digits, split keys, cap + 8
  // digits, weights, scan (3), write
  return 1 + (1 + 8) + 1 + 1 + n_passes * (1 + 1 + 8 + 1 + 1 + 1 + 3 + 1 + 1 + 1 + 1 + 16 + 1) +
         (1 + 1 + 8 + 1 + 1 + 16 + 1 + 3 + 1);
}

cudaError_t launch_manage(const lgs_surfels& M, const float* lam, const float* res, const MgHostParams& H,
                          void* scratch, float* score, const lgs_surfel_params_out& out, int64_t capacity,
                          int32_t* src, uint8_t* role, int64_t* counts, cudaStream_t s) {
  const uint32_t n = static_cast<uint32_t>(M.n);
  const MgScratch S = mg_scratch(scratch, M.n);
  const int sms = sm_count();
  const int g = grid_for(n, sms);
  const int gT = grid_for(S.T, sms);
  MgParams P;
  P.logit_prune = H.logit_prune;
  P.logit_min = H.logit_min;
  P.w_l = H.p.w_l;
  P.w_c = H.p.w_c;
  P.w_r = H.p.w_r;
  P.q_res = H.p.q_res;
  P.eps = H.p.eps;
  P.q_plane = H.p.q_plane;
  P.voxel = H.p.voxel;
  P.q_cover = H.p.q_cover;
  P.slab = H.p.slab;
  P.prune_cap = H.p.prune_cap;
  P.q_split = H.p.q_split;
  P.split_cap = H.p.split_cap;
  P.split_shift = H.p.split_shift;
  P.split_dlog = H.p.split_dlog;
  static const int planes[3][2] = {{0, 1}, {1, 2}, {2, 0}};

  k_mg_init<<<1, 256, 0, s>>>(S.sel, n, counts);
  k_mg_res_keys<<<g, kMgCta, 0, s>>>(res, n, S.key);
  k_sel_quantile<<<1, 1, 0, s>>>(S.sel, P.q_res);
  launch_select(S.key, n, S.sel, 4, g, s);
  k_mg_score<<<g, kMgCta, 0, s>>>(lam, res, M.opacity_logit, n, S.sel, P, score, S.flags, counts);
  for (int p = 0; p < H.p.n_passes; ++p) {
    k_mg_alive_keys<<<g, kMgCta, 0, s>>>(score, n, S.flags, S.key, S.sel);
    k_sel_quantile<<<1, 1, 0, s>>>(S.sel, P.q_plane);
    launch_select(S.key, n, S.sel, 4, g, s);
    k_mg_clear<<<gT, kMgCta, 0, s>>>(S.htab, S.rep, S.cnt, S.T, S.sel);
    k_mg_insert<<<g, kMgCta, 0, s>>>(M.mean, M.opacity_logit, score, n, S.sel, P, planes[p][0], planes[p][1], S);
    k_mg_measure<<<g, kMgCta, 0, s>>>(M.mean, M.quat, M.log_scale, n, P, S);
    launch_scan(S.cnt, S.off, S.T, S.part, s);
    k_mg_scatter<<<g, kMgCta, 0, s>>>(n, S);
    k_mg_big_select<<<sms * 4, kMgCta, 0, s>>>(S, P);
    k_mg_decide<<<g, kMgCta, 0, s>>>(score, n, P, S);
    k_sel_cap<<<1, 1, 0, s>>>(S.sel, P.prune_cap);
    launch_select(S.key, n, S.sel, 8, g, s);
    k_mg_apply_prune<<<g, kMgCta, 0, s>>>(n, S, counts + 2 + p);
  }
  k_mg_alive_keys<<<g, kMgCta, 0, s>>>(score, n, S.flags, S.key, S.sel);
  k_sel_quantile<<<1, 1, 0, s>>>(S.sel, P.q_split);
  launch_select(S.key, n, S.sel, 4, g, s);
  k_mg_split_keys<<<g, kMgCta, 0, s>>>(M.opacity_logit, score, n, P, S);
  k_sel_cap<<<1, 1, 0, s>>>(S.sel, P.split_cap);
  launch_select(S.key, n, S.sel, 8, g, s);
  k_mg_weights<<<g, kMgCta, 0, s>>>(n, S);
  launch_scan(S.pos, S.pos, n, S.part, s);
  k_mg_write<<<g, kMgCta, 0, s>>>(M.mean, M.quat, M.log_scale, M.opacity_logit, n, P, S, out, capacity, src, role,
                                  counts);
  return cudaGetLastError();
}

cudaError_t launch_manage_gather(const int32_t* src, const uint8_t* role, const int64_t* counts, int64_t capacity,
                                 const void* in, void* out, int words, int zero_children, cudaStream_t s) {
  const int g = grid_for(static_cast<uint64_t>(capacity) * static_cast<uint64_t>(words), sm_count());
  k_mg_gather<<<g, kMgCta, 0, s>>>(src, role, counts, capacity, static_cast<const uint32_t*>(in),
                                   static_cast<uint32_t*>(out), words, zero_children);
  return cudaGetLastError();
}

}  // namespace lgs
