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
// first k of an order) are exact: a radix select over 64-bit keys in 11-bit
// digits finds the k-th smallest key, one kernel per digit whose last CTA to
// finish picks the bin; from the second digit on, the keys still matching
// the prefix go to a compaction buffer that the next digit reads instead of
// the full array.  Groups of a cover-and-prune pass live in an
// open-addressing hash table keyed by the biased 2D voxel; the representative
// (largest logit, then lowest index) is an atomicMax over a packed key;
// members scatter (squared cover radius, index) pairs into per-group
// buckets.  A member is covered when its radius is at most the group's k-th
// smallest: small groups decide one warp per group by counting strictly
// smaller radii staged in shared memory, large groups find the k-th smallest
// by a one-CTA radix select over the bucket.
//
// Launches (one stream, no host synchronisation, counts written on the
// device; 71 with three passes): residual keys (and the select's reset),
// residual quantile; score, opacity prune, the survivors' keys and the table
// clear; per pass: the survivors' score quantile, insert, measure, bucket
// scan, scatter, decide, cap select, apply (which also writes the next
// quantile's keys and clears the table); then the split quantile, split keys,
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
// by the first digit, which reads it); base is the number of survivors a cap
// is a fraction of; after the last digit prefix is the selected key.
struct Sel {
  unsigned long long prefix;
  uint32_t count;
  uint32_t k;
  uint32_t kind;
  uint32_t base;
  uint32_t n_big;              // groups of the current pass with more than kSmallGroup members
  uint32_t n_small;            // the other groups with members
  uint32_t ticket;             // CTAs of the current digit done (the last one picks)
  uint32_t ccount[2];          // keys in the two compaction buffers
  uint32_t hist[2048];
};

struct MgScratch {
  Sel* sel;
  uint32_t* flags;             // [n] kAlive | kCand | kMember | kFlag | kSplit
  unsigned long long* key;     // [n] select keys (kNoKey: not taking part)
  uint32_t* slot;              // [n] hash slot of a candidate's group
  uint32_t* r2;                // [n] a member's squared cover radius (float bits)
  uint32_t* pos;               // [n + 1] output weights, then their exclusive scan
  unsigned long long* bucket;  // [n] members (radius bits << 32 | index) grouped by slot
  unsigned long long* cbuf[2]; // [n] each: keys still matching the select's prefix
  uint32_t* small;             // [n] slots of the groups with 1..kSmallGroup members
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
  size_t sel, flags, key, slot, r2, pos, bucket, cbuf0, cbuf1, small, htab, rep, cnt, off, big, part, total;
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
  L.bucket = take(8 * N);
  L.cbuf0 = take(8 * N);
  L.cbuf1 = take(8 * N);
  L.small = take(4 * N);
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
  s.bucket = reinterpret_cast<unsigned long long*>(b + L.bucket);
  s.cbuf[0] = reinterpret_cast<unsigned long long*>(b + L.cbuf0);
  s.cbuf[1] = reinterpret_cast<unsigned long long*>(b + L.cbuf1);
  s.small = reinterpret_cast<uint32_t*>(b + L.small);
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

// One atomic per CTA: the CTA's sum of v into a 32-bit or 64-bit counter
// (every thread of the CTA calls it, after its grid-stride loop).
__device__ __forceinline__ uint32_t block_sum(uint32_t v) {
  __shared__ uint32_t s_sum;
  if (threadIdx.x == 0) s_sum = 0;
  __syncthreads();
  v = __reduce_add_sync(0xffffffffu, v);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(&s_sum, v);
  __syncthreads();
  const uint32_t t = s_sum;
  __syncthreads();   // read by all before a second call resets it
  return t;
}
__device__ __forceinline__ void block_count(uint32_t v, uint32_t* ctr) {
  const uint32_t t = block_sum(v);
  if (threadIdx.x == 0 && t) atomicAdd(ctr, t);
}
__device__ __forceinline__ void block_count64(uint32_t v, int64_t* ctr) {
  const uint32_t t = block_sum(v);
  if (threadIdx.x == 0 && t) atomicAdd(reinterpret_cast<unsigned long long*>(ctr), static_cast<unsigned long long>(t));
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
// Digits of the select, most significant first: 11 bits each, so a quantile
// (keys significant in their upper 32 bits) takes 3 digits and a cap (all 64
// bits) 6.
struct Digit {
  int shift, width;
};
constexpr Digit kDigits64[6] = {{53, 11}, {42, 11}, {31, 11}, {20, 11}, {9, 11}, {0, 9}};
constexpr Digit kDigits32[3] = {{53, 11}, {42, 11}, {32, 10}};
constexpr uint32_t kBins = 2048;

enum : int { kSetupNone = 0, kSetupQuantile = 1, kSetupCap = 2 };

// The select's kind and rank from the counted keys.  Quantile: the
// floor(q (count - 1))-th smallest; cap: at most floor(q base) keys, the
// smallest first (every key when count <= cap).
__device__ void sel_setup(const Sel* sel, int mode, float q, uint32_t& kind, uint32_t& k, uint32_t& base) {
  const uint32_t c = sel->count;
  k = 0;
  if (mode == kSetupQuantile) {
    base = c;
    if (c == 0) {
      kind = kSelNone;
    } else {
      kind = kSelKth;
      k = static_cast<uint32_t>(floor(static_cast<double>(q) * static_cast<double>(c - 1)));
    }
  } else {
    base = sel->base;
    const double cap = floor(static_cast<double>(q) * static_cast<double>(base));
    if (static_cast<double>(c) <= cap) {
      kind = kSelAll;
    } else if (cap < 1.0) {
      kind = kSelNone;
    } else {
      kind = kSelKth;
      k = static_cast<uint32_t>(cap) - 1u;
    }
  }
}

constexpr uint32_t kStage = 256;   // keys a warp stages before it appends them

__device__ __forceinline__ void flush_stage(const unsigned long long* stage, uint32_t sc, unsigned long long* dst,
                                            uint32_t* dcount, int lane) {
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(dcount, sc);
  base = __shfl_sync(0xffffffffu, base, 0);
  for (uint32_t t = lane; t < sc; t += 32) dst[base + t] = stage[t];
  __syncwarp();   // the stage is rewritten only after every lane has copied out
}

// One digit of the radix select: every CTA histograms its share of the keys
// that match the prefix so far; the last CTA to finish (ticket) picks the bin
// holding rank k, extends the prefix and clears the histogram.  The first
// digit also sets the select up from the counted keys (mode != kSetupNone).
// Digit 0 and 1 read every key; digit 1 and later also copy the keys that
// match the prefix into a compaction buffer, which the next digit reads
// instead (keys never leave the prefix's range once they fall out of it).
__global__ void __launch_bounds__(kMgCta) k_sel_digit(const unsigned long long* __restrict__ key, uint32_t n,
                                                      Sel* __restrict__ sel, unsigned long long* cbuf0,
                                                      unsigned long long* cbuf1, int d, int last, int shift,
                                                      int width, int mode, float q) {
  __shared__ uint32_t h[kBins];
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_kind, s_k, s_base, s_last;
  __shared__ unsigned long long s_pre;
  __shared__ unsigned long long s_stage[kMgCta / 32][kStage];
  if (threadIdx.x == 0) {
    if (mode != kSetupNone) {
      sel_setup(sel, mode, q, s_kind, s_k, s_base);
      s_pre = 0ull;
    } else {
      s_kind = sel->kind;
      s_k = sel->k;
      s_pre = sel->prefix;
    }
  }
  for (uint32_t t = threadIdx.x; t < kBins; t += blockDim.x) h[t] = 0;
  __syncthreads();
  const bool active = s_kind == kSelKth;
  if (active) {
    // digit d >= 2 reads the buffer digit d - 1 wrote; digit d >= 1 writes
    // the other one (unless it is the last digit)
    const unsigned long long* src = key;
    uint32_t len = n;
    if (d >= 2) {
      src = ((d - 2) & 1) ? cbuf1 : cbuf0;
      len = sel->ccount[(d - 2) & 1];
    }
    unsigned long long* dst = ((d - 1) & 1) ? cbuf1 : cbuf0;
    uint32_t* dcount = &sel->ccount[(d - 1) & 1];
    const bool compact = d >= 1 && !last;
    unsigned long long* stage = s_stage[threadIdx.x >> 5];
    uint32_t sc = 0;   // keys staged by this warp (warp-uniform)
    const unsigned long long pre = s_pre;
    const unsigned long long hi = shift + width >= 64 ? 0ull : (~0ull << (shift + width));
    const uint32_t dmask = (1u << width) - 1u;
    const int lane = threadIdx.x & 31;
    // kUnroll keys per thread per round, loaded before use (the loop is
    // latency-bound otherwise); warp-uniform rounds
    constexpr int kUnroll = 4;
    const uint32_t step = gridDim.x * blockDim.x * kUnroll;
    for (uint32_t i0 = blockIdx.x * blockDim.x * kUnroll; i0 < len; i0 += step) {
      unsigned long long kk[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const uint32_t i = i0 + u * blockDim.x + threadIdx.x;
        kk[u] = i < len ? src[i] : kNoKey;
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const unsigned long long k = kk[u];
        const uint32_t bin =
            (k != kNoKey && !((k ^ pre) & hi)) ? (static_cast<uint32_t>(k >> shift) & dmask) : kBins;
        // a warp whose keys share one bin adds once; otherwise each lane adds
        const uint32_t b0 = __shfl_sync(0xffffffffu, bin, 0);
        if (__all_sync(0xffffffffu, bin == b0)) {
          if (lane == 0 && b0 < kBins) atomicAdd(&h[b0], 32u);
        } else if (bin < kBins) {
          atomicAdd(&h[bin], 1u);
        }
        if (compact) {
          // staged per warp, flushed with one atomic per ~224 keys
          const uint32_t m = __ballot_sync(0xffffffffu, bin < kBins);
          if (bin < kBins) stage[sc + __popc(m & ((1u << lane) - 1u))] = k;
          sc += __popc(m);
          if (sc > kStage - 32) {
            __syncwarp();
            flush_stage(stage, sc, dst, dcount, lane);
            sc = 0;
          }
        }
      }
    }
    if (compact && sc) {
      __syncwarp();
      flush_stage(stage, sc, dst, dcount, lane);
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < kBins; t += blockDim.x)
      if (h[t]) atomicAdd(&sel->hist[t], h[t]);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&sel->ticket, 1u) == gridDim.x - 1 ? 1u : 0u;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  if (threadIdx.x == 0) {
    sel->ticket = 0;
    sel->ccount[d & 1] = 0;   // the buffer digit d + 1 writes (digit d read it, or nobody did)
    if (mode != kSetupNone) {
      sel->kind = s_kind;
      sel->k = s_k;
      sel->base = s_base;
      sel->count = 0;
      sel->prefix = 0ull;
    }
  }
  if (!active) return;
  // pick: each of the 256 threads owns 8 consecutive bins
  constexpr int kPer = kBins / kMgCta;
  volatile uint32_t* vh = sel->hist;
  uint32_t v[kPer], sum = 0;
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    v[j] = vh[threadIdx.x * kPer + j];
    sum += v[j];
  }
  const uint32_t kk = s_k;
  uint32_t total;
  uint32_t ex = block_exclusive_scan(sum, s_warp, total);
#pragma unroll
  for (int j = 0; j < kPer; ++j) {
    if (ex <= kk && kk < ex + v[j]) {
      sel->prefix = s_pre | (static_cast<unsigned long long>(threadIdx.x * kPer + j) << shift);
      sel->k = kk - ex;
    }
    ex += v[j];
    vh[threadIdx.x * kPer + j] = 0u;
  }
}

template <int D>
void launch_select(const unsigned long long* key, uint32_t n, Sel* sel, unsigned long long* const (&cbuf)[2],
                   const Digit (&digits)[D], int mode, float q, int grid, cudaStream_t s) {
  for (int d = 0; d < D; ++d)
    k_sel_digit<<<grid, kMgCta, 0, s>>>(key, n, sel, cbuf[0], cbuf[1], d, d == D - 1 ? 1 : 0, digits[d].shift,
                                        digits[d].width, d == 0 ? mode : kSetupNone, q);
}

// selected if the select takes every key, or the key is at most the k-th
__device__ __forceinline__ bool sel_takes(uint32_t kind, unsigned long long prefix, unsigned long long k) {
  return kind == kSelAll || (kind == kSelKth && k <= prefix);
}

// ---------------------------------------------------------------------------
// kernels of the step
// ---------------------------------------------------------------------------
// Residual keys for its quantile; CTA 0 also resets the select and the counts.
__global__ void __launch_bounds__(kMgCta) k_mg_res_keys(const float* __restrict__ res, uint32_t n,
                                                        unsigned long long* __restrict__ key, Sel* __restrict__ sel,
                                                        int64_t* __restrict__ counts) {
  if (blockIdx.x == 0) {
    for (uint32_t t = threadIdx.x; t < kBins; t += blockDim.x) sel->hist[t] = 0;
    if (threadIdx.x == 0) {
      sel->prefix = 0;
      sel->count = n;      // the residual quantile takes every surfel
      sel->k = 0;
      sel->kind = kSelNone;
      sel->base = 0;
      sel->n_big = 0;
      sel->n_small = 0;
      sel->ticket = 0;
      sel->ccount[0] = 0;
      sel->ccount[1] = 0;
    }
    if (threadIdx.x < 6) counts[threadIdx.x] = 0;
  }
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    key[i] = static_cast<unsigned long long>(okey(res[i])) << 32;
}

// Clears the hash table of a pass (and its large-group list).
__device__ __forceinline__ void clear_table(const MgScratch& S) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    S.sel->n_big = 0;
    S.sel->n_small = 0;
  }
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < S.T; i += gridDim.x * blockDim.x) {
    S.htab[i] = kNoKey;
    S.rep[i] = 0ull;
    S.cnt[i] = 0u;
  }
}

// Control score (Eq. controlscore) with the residual normalised by its
// quantile, and the opacity prune.
__global__ void __launch_bounds__(kMgCta) k_mg_score(const float* __restrict__ lam, const float* __restrict__ res,
                                                     const float* __restrict__ logit, uint32_t n, MgParams P,
                                                     float* __restrict__ score, MgScratch S,
                                                     int64_t* __restrict__ counts) {
  const float rq = okey_inv(static_cast<uint32_t>(S.sel->prefix >> 32));
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t n_dead = 0, n_alive = 0;
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
      S.flags[i] = alive ? kAlive : 0u;
      // the survivors' scores are the keys of the next quantile
      S.key[i] = alive ? static_cast<unsigned long long>(__float_as_uint(s)) << 32 : kNoKey;
      dead = !alive;
    }
    n_dead += dead ? 1u : 0u;
    n_alive += (i < n && !dead) ? 1u : 0u;
  }
  block_count64(n_dead, &counts[1]);
  block_count(n_alive, &S.sel->count);
  clear_table(S);
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
    S.bucket[b + old - 1u - rank] = (static_cast<unsigned long long>(S.r2[i]) << 32) | i;
    // the first decrement lists the group for k_mg_decide
    if (lane == lead && old == m) {
      if (m > kSmallGroup) S.big[atomicAdd(&S.sel->n_big, 1u)] = h;
      else S.small[atomicAdd(&S.sel->n_small, 1u)] = h;
    }
  }
}

// Marks a member covered: the cap select takes its key (score, index).
__device__ __forceinline__ void cover(const float* __restrict__ score, const MgScratch& S, uint32_t i) {
  S.flags[i] |= kFlag;
  S.key[i] = (static_cast<unsigned long long>(__float_as_uint(score[i])) << 32) | i;
}

// A member is covered when its radius is at most the k-th smallest of its
// group, k = ceil(q_cover m).  Large groups (more than kSmallGroup members):
// one CTA finds the k-th smallest by a radix select over the bucket (4
// digits of 8 bits) and flags; the others: one warp per group stages the
// radii in shared memory and each member counts the strictly smaller ones
// (fewer than k: covered).
__global__ void __launch_bounds__(kMgCta) k_mg_decide(const float* __restrict__ score, MgParams P, MgScratch S) {
  __shared__ uint32_t h[kBins];
  __shared__ uint32_t s_warp[32];
  __shared__ uint32_t s_pre, s_k, s_cov;
  __shared__ uint4 s_r2[kMgCta / 32][kSmallGroup / 4];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t nb = S.sel->n_big, ns = S.sel->n_small;
  for (uint32_t g = blockIdx.x; g < nb; g += gridDim.x) {
    const uint32_t slot = S.big[g];
    const uint32_t b = S.off[slot], e = S.off[slot + 1];
    const uint32_t k = static_cast<uint32_t>(ceil(static_cast<double>(P.q_cover) * static_cast<double>(e - b)));
    if (k == 0) continue;   // uniform across the CTA
    if (threadIdx.x == 0) {
      s_pre = 0;
      s_k = k - 1u;
      s_cov = 0;
    }
    // digits of 11, 11 and 10 bits over the 32-bit radii
    for (int d = 0; d < 3; ++d) {
      const int shift = d == 0 ? 21 : (d == 1 ? 10 : 0);
      const int width = d == 2 ? 10 : 11;
      for (uint32_t t = threadIdx.x; t < kBins; t += blockDim.x) h[t] = 0;
      __syncthreads();
      const uint32_t pre = s_pre;
      const uint32_t hi = d == 0 ? 0u : (~0u << (shift + width));
      const uint32_t dmask = (1u << width) - 1u;
      constexpr int kUnroll = 4;
      for (uint32_t j0 = b + threadIdx.x; j0 < e; j0 += blockDim.x * kUnroll) {
        uint32_t x[kUnroll];
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const uint32_t j = j0 + u * blockDim.x;
          x[u] = j < e ? static_cast<uint32_t>(S.bucket[j] >> 32) : 0u;
        }
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
          if (j0 + u * blockDim.x < e && !((x[u] ^ pre) & hi)) atomicAdd(&h[(x[u] >> shift) & dmask], 1u);
      }
      __syncthreads();
      constexpr int kPer = kBins / kMgCta;
      uint32_t v[kPer], sum = 0;
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        v[j] = h[threadIdx.x * kPer + j];
        sum += v[j];
      }
      const uint32_t kk = s_k;
      uint32_t total;
      uint32_t ex = block_exclusive_scan(sum, s_warp, total);
#pragma unroll
      for (int j = 0; j < kPer; ++j) {
        if (ex <= kk && kk < ex + v[j]) {
          s_pre = pre | ((threadIdx.x * kPer + j) << shift);
          s_k = kk - ex;
        }
        ex += v[j];
      }
      __syncthreads();
    }
    const uint32_t beta2 = s_pre;
    uint32_t mine = 0;
    for (uint32_t j = b + threadIdx.x; j < e; j += blockDim.x) {
      const unsigned long long bj = S.bucket[j];
      if (static_cast<uint32_t>(bj >> 32) <= beta2) {
        cover(score, S, static_cast<uint32_t>(bj));
        ++mine;
      }
    }
    atomicAdd(&s_cov, mine);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&S.sel->count, s_cov);
    __syncthreads();
  }
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  uint4* r4 = s_r2[wid];
  uint32_t* r2 = reinterpret_cast<uint32_t*>(r4);
  for (uint32_t g = blockIdx.x * (blockDim.x >> 5) + wid; g < ns; g += warps) {
    const uint32_t slot = S.small[g];
    const uint32_t b = S.off[slot], m = S.off[slot + 1] - b;
    const uint32_t k = static_cast<uint32_t>(ceil(static_cast<double>(P.q_cover) * static_cast<double>(m)));
    const uint32_t m4 = (m + 3) / 4;
    // radii staged in shared memory, the tail padded with the largest key
    // (never strictly smaller than a radius)
    for (uint32_t j = lane; j < 4 * m4; j += 32) r2[j] = j < m ? static_cast<uint32_t>(S.bucket[b + j] >> 32) : ~0u;
    __syncwarp();
    uint32_t cov = 0;
    for (uint32_t j0 = 0; j0 < m; j0 += 32) {
      const uint32_t j = j0 + lane;
      const uint32_t x = j < m ? r2[j] : 0u;
      // strictly smaller radii of the group: every lane reads the same
      // 16-byte words (broadcast); four independent partial counts
      uint32_t l0 = 0, l1 = 0, l2 = 0, l3 = 0;
      for (uint32_t t = 0; t < m4; ++t) {
        const uint4 v = r4[t];
        l0 += v.x < x;
        l1 += v.y < x;
        l2 += v.z < x;
        l3 += v.w < x;
      }
      const bool covered = j < m && (l0 + l1) + (l2 + l3) < k;
      if (covered) cover(score, S, static_cast<uint32_t>(S.bucket[b + j]));
      cov += __popc(__ballot_sync(0xffffffffu, covered));
    }
    if (lane == 0 && cov) atomicAdd(&S.sel->count, cov);
    __syncwarp();   // the staged radii are read before the next group overwrites them
  }
}

// Removes the covered members the cap admits; writes the survivors' score
// keys for the next quantile (counted into the select) and clears the table.
__global__ void __launch_bounds__(kMgCta) k_mg_apply_prune(const float* __restrict__ score, uint32_t n, MgScratch S,
                                                           int64_t* __restrict__ removed) {
  const uint32_t kind = S.sel->kind;
  const unsigned long long prefix = S.sel->prefix;
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t n_rm = 0, n_alive = 0;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const uint32_t i = i0 + threadIdx.x;
    bool rm = false, alive = false;
    if (i < n) {
      uint32_t f = S.flags[i];
      if ((f & kFlag) && sel_takes(kind, prefix, S.key[i])) {
        rm = true;
        f &= ~kAlive;
      }
      f &= kAlive;
      S.flags[i] = f;
      alive = f != 0;
      S.key[i] = alive ? static_cast<unsigned long long>(__float_as_uint(score[i])) << 32 : kNoKey;
    }
    n_rm += rm ? 1u : 0u;
    n_alive += alive ? 1u : 0u;
  }
  block_count64(n_rm, removed);
  block_count(n_alive, &S.sel->count);
  clear_table(S);
}

// split candidates: survivors with c >= Q_{q_split} and alpha >= alpha_min,
// keyed for "largest score first, then lowest index"
__global__ void __launch_bounds__(kMgCta) k_mg_split_keys(const float* __restrict__ logit,
                                                          const float* __restrict__ score, uint32_t n, MgParams P,
                                                          MgScratch S) {
  const bool any = S.sel->kind != kSelNone;
  const float qs = __uint_as_float(static_cast<uint32_t>(S.sel->prefix >> 32));
  const uint32_t stride = gridDim.x * blockDim.x;
  uint32_t n_cand = 0;
  for (uint32_t i0 = blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
    const uint32_t i = i0 + threadIdx.x;
    bool cand = false;
    if (i < n) {
      const float c = score[i];
      cand = any && (S.flags[i] & kAlive) && c >= qs && logit[i] >= P.logit_min;
      S.key[i] = cand ? ((static_cast<unsigned long long>(~__float_as_uint(c)) << 32) | i) : kNoKey;
    }
    n_cand += cand ? 1u : 0u;
  }
  block_count(n_cand, &S.sel->count);
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
  uint32_t n_split = 0;
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
    n_split += split ? 1u : 0u;
  }
  block_count64(n_split, &counts[5]);
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

size_t scan_partials_bytes(uint64_t len) { return 4 * (static_cast<size_t>(scan_blocks(len)) + 1); }

void exclusive_scan_u32(const uint32_t* in, uint32_t* out, uint32_t len, uint32_t* part, cudaStream_t s) {
  launch_scan(in, out, len, part, s);
}

int manage_kernel_count(int n_passes) {
  // residual keys, 3 digits, score; per pass: 3 digits, insert, measure,
  // scan (3), scatter, decide, 6 digits, apply; split: 3 digits, split keys,
  // 6 digits, weights, scan (3), write
  return 1 + 3 + 1 + n_passes * (3 + 1 + 1 + 3 + 1 + 1 + 6 + 1) + (3 + 1 + 6 + 1 + 3 + 1);
}

cudaError_t launch_manage(const lgs_surfels& M, const float* lam, const float* res, const MgHostParams& H,
                          void* scratch, float* score, const lgs_surfel_params_out& out, int64_t capacity,
                          int32_t* src, uint8_t* role, int64_t* counts, cudaStream_t s) {
  const uint32_t n = static_cast<uint32_t>(M.n);
  const MgScratch S = mg_scratch(scratch, M.n);
  const int sms = sm_count();
  const int g = grid_for(n, sms);
  const int gc = grid_for(n > S.T ? n : S.T, sms);   // kernels that also clear the table
  const int gs = grid_for(n, sms) < 2 * sms ? grid_for(n, sms) : 2 * sms;   // select digits
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

  k_mg_res_keys<<<g, kMgCta, 0, s>>>(res, n, S.key, S.sel, counts);
  launch_select(S.key, n, S.sel, S.cbuf, kDigits32, kSetupQuantile, P.q_res, gs, s);
  k_mg_score<<<gc, kMgCta, 0, s>>>(lam, res, M.opacity_logit, n, P, score, S, counts);
  for (int p = 0; p < H.p.n_passes; ++p) {
    launch_select(S.key, n, S.sel, S.cbuf, kDigits32, kSetupQuantile, P.q_plane, gs, s);
    k_mg_insert<<<g, kMgCta, 0, s>>>(M.mean, M.opacity_logit, score, n, S.sel, P, planes[p][0], planes[p][1], S);
    k_mg_measure<<<g, kMgCta, 0, s>>>(M.mean, M.quat, M.log_scale, n, P, S);
    launch_scan(S.cnt, S.off, S.T, S.part, s);
    k_mg_scatter<<<g, kMgCta, 0, s>>>(n, S);
    k_mg_decide<<<sms * 4, kMgCta, 0, s>>>(score, P, S);
    launch_select(S.key, n, S.sel, S.cbuf, kDigits64, kSetupCap, P.prune_cap, gs, s);
    k_mg_apply_prune<<<gc, kMgCta, 0, s>>>(score, n, S, counts + 2 + p);
  }
  launch_select(S.key, n, S.sel, S.cbuf, kDigits32, kSetupQuantile, P.q_split, gs, s);
  k_mg_split_keys<<<g, kMgCta, 0, s>>>(M.opacity_logit, score, n, P, S);
  launch_select(S.key, n, S.sel, S.cbuf, kDigits64, kSetupCap, P.split_cap, gs, s);
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
