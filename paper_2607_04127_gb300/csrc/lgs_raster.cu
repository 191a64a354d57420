// lgs_raster.cu -- per-tile front-to-back compositing (forward) and its
// reverse-order adjoint (backward) for the spherical surfel rasterizer.
//
// One CTA renders one angular tile (tile_h x tile_w pixels, one thread per
// pixel).  The tile's depth-ordered list is streamed through shared memory in
// batches of BATCH records (64 B each, gathered by item id); every thread
// walks the batch for its own ray.  Pixels stop once T (1 - a) would drop
// below 1e-4; a warp whose lanes have all stopped skips the batch, and the
// CTA leaves when every pixel has stopped.
//
// The backward re-evaluates the same records per tile in reverse list order
// (no per-pixel surfel lists are stored): the transmittance before each
// contributor is recovered as T_k = T_{k+1} / (1 - a_k) from T_final, and the
// suffix sum S = sum_{j>k} w_j (g . c_j) gives dL/da_k = T_k (g . c_k) -
// S / (1 - a_k).  Per entry the warp reduces its 15 geometric gradients with a
// butterfly reduce-scatter (16 shuffles), 15 lanes add them into a shared
// per-batch accumulator, and the CTA flushes one atomic add per (surfel,
// component) into the per-item gradient buffer.
#include <cstddef>
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {

constexpr int kMaxTileThreads = 256;
// Per-item gradient moments written by the backward.  With the unclamped
// opacity derivative g = alpha G dL/da of a contribution (0 where a is
// clamped), its offset (u, v) in the plane, ct = (dL/dt) / (n.d) and the
// direct normal term w sg gS_n, every surfel gradient is a fixed combination
// of their sums over the contributions (k_preprocess_bwd forms it):
//   [0] g  [1] u g  [2] v g  [3] u^2 g  [4] v^2 g  [5] u v g
//   [6] ct  [7] ct u  [8] ct v  [9..11] w sg gS_n
// because dL/du = -u g, dL/dv = -v g and the intersection offset inside the
// plane is u s_u t_u + v s_v t_v.
constexpr int kGrad = 12;

// The 12 moments of one valid contribution with transmittance Tk before it
// and suffix S (the sum over the later contributors of w (g.c)), added into v.
__device__ __forceinline__ void moments(const Eval& E, const float4& r0, float Tk, float S, float iom, float gA,
                                        float gSt, float gSx, float gSy, float gSz, float (&v)[16]) {
  const float sg = E.den > 0.f ? -1.f : 1.f;
  const float gc = gA + gSt * E.t + sg * (gSx * r0.x + gSy * r0.y + gSz * r0.z);
  const float w = E.a * Tk;
  const float dLda = Tk * gc - S * iom;
  const float g = E.araw < 0.99f ? E.araw * dLda : 0.f;
  const float ug = E.u * g, vg = E.v * g;
  const float ct = fmaf(w, gSt, -fmaf(ug, E.ud, vg * E.vd)) * E.rden;
  const float wsg = w * sg;
  v[0] += g;
  v[1] += ug;
  v[2] += vg;
  v[3] += E.u * ug;
  v[4] += E.v * vg;
  v[5] += E.u * vg;
  v[6] += ct;
  v[7] += ct * E.u;
  v[8] += ct * E.v;
  v[9] += wsg * gSx;
  v[10] += wsg * gSy;
  v[11] += wsg * gSz;
}

// Reverse-order step of one valid contribution: updates the transmittance T
// (before it) and the suffix S, and adds its 12 moments into v (the same
// arithmetic as moments(), with S updated in place).
__device__ __forceinline__ void contrib_moments(const Eval& E, const float4& r0, float gA, float gSt, float gSx,
                                                float gSy, float gSz, float& T, float& S, float (&v)[16]) {
  const float iom = rcp_ftz(1.0f - E.a);
  const float Tk = T * iom;
  const float sg = E.den > 0.f ? -1.f : 1.f;
  const float gc = gA + gSt * E.t + sg * (gSx * r0.x + gSy * r0.y + gSz * r0.z);
  const float w = E.a * Tk;
  const float dLda = Tk * gc - S * iom;
  S = fmaf(w, gc, S);
  T = Tk;
  const float g = E.araw < 0.99f ? E.araw * dLda : 0.f;
  const float ug = E.u * g, vg = E.v * g;
  const float ct = fmaf(w, gSt, -fmaf(ug, E.ud, vg * E.vd)) * E.rden;
  const float wsg = w * sg;
  v[0] += g;
  v[1] += ug;
  v[2] += vg;
  v[3] += E.u * ug;
  v[4] += E.v * vg;
  v[5] += E.u * vg;
  v[6] += ct;
  v[7] += ct * E.u;
  v[8] += ct * E.v;
  v[9] += wsg * gSx;
  v[10] += wsg * gSy;
  v[11] += wsg * gSz;
}

struct TileCtx {
  int f;
  int r, c;
  bool inside;
  uint32_t start, end;
  int64_t pix;
  int HW;
};

__device__ __forceinline__ TileCtx tile_ctx(const Desc& D, uint32_t tile, const uint2* __restrict__ ranges) {
  TileCtx t;
  t.f = frame_of_tile(D, tile);
  const FrameDev& F = D.f[t.f];
  const int lt = static_cast<int>(tile - F.tile_base);
  const int ti = lt / F.ntc, tj = lt - ti * F.ntc;
  int lr, lc;
  pixel_of_thread(F, static_cast<int>(threadIdx.x), lr, lc);
  t.r = ti * F.th + lr;
  t.c = tj * F.tw + lc;
  t.inside = t.r < F.H && t.c < F.W;
  t.pix = static_cast<int64_t>(t.r) * F.W + t.c;
  t.HW = F.H * F.W;
  const uint2 rg = ranges[tile];
  t.start = rg.x;
  t.end = rg.y;
  return t;
}

// Work item of the CTA: its own tile, or (persistent mode) the next entry of
// the longest-first order claimed through an atomic counter.
__device__ __forceinline__ bool next_tile(bool persistent, const uint32_t* __restrict__ order, uint32_t n_tiles,
                                          unsigned int* counter, uint32_t& tile, int iter) {
  if (!persistent) {
    tile = blockIdx.x;
    return iter == 0;
  }
  __shared__ uint32_t s_tile;
  __syncthreads();
  if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
  __syncthreads();
  const uint32_t k = s_tile;
  if (k >= n_tiles) return false;
  tile = order ? order[k] : k;
  return true;
}

// The batch entries whose pixel box meets the warp's pixel block, in list
// order: 32 boxes tested per step (one per lane) and compacted with a ballot.
// Returns the count (uniform over the warp).
__device__ __forceinline__ int warp_list(const float4* s_box, int nb, const WarpBox& wb, uint16_t* list) {
  const int lane = threadIdx.x & 31;
  const uint32_t lt = (1u << lane) - 1u;
  int cnt = 0;
  for (int base = 0; base < nb; base += 32) {
    const int j = base + lane;
    const bool hit = j < nb && box_hits(s_box[j], wb);
    const uint32_t m = __ballot_sync(0xffffffffu, hit);
    if (hit) list[cnt + __popc(m & lt)] = static_cast<uint16_t>(j);
    cnt += __popc(m);
  }
  __syncwarp();
  return cnt;
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------
template <int BATCH>
__global__ void __launch_bounds__(kMaxTileThreads)
    k_fwd(const Desc* __restrict__ D, const uint2* __restrict__ ranges, const uint32_t* __restrict__ pv,
          const float4* __restrict__ rec, const float4* __restrict__ box, const uint32_t* __restrict__ order,
          Status* __restrict__ st, int persistent) {
  __shared__ float4 s_r0[BATCH], s_r1[BATCH], s_r2[BATCH], s_box[BATCH];
  __shared__ float s_al[BATCH];
  __shared__ uint16_t s_list[kMaxTileThreads / 32][BATCH];
  const int nthr = blockDim.x;
  const int tid = threadIdx.x, wid = tid >> 5;
  uint32_t tile;
  uint32_t evals = 0, contrib = 0, alg = 0;
  for (int iter = 0; next_tile(persistent, order, D->n_tiles, &st->work_counter, tile, iter); ++iter) {
    const TileCtx tc = tile_ctx(*D, tile, ranges);
    if (tc.end - tc.start > kLongList) continue;   // the long-list kernels' tile
    const FrameDev& F = D->f[tc.f];
    const WarpBox wb = warp_box(tc.inside, tc.r, tc.c, F.W);
    float dx = 0.f, dy = 0.f, dz = 0.f;
    if (tc.inside) pixel_ray(F, tc.r, tc.c, dx, dy, dz);
    float T = 1.0f, A = 0.0f, St = 0.0f, Sx = 0.0f, Sy = 0.0f, Sz = 0.0f;
    int last = 0, stop_at = -1;
    bool done = !tc.inside;
    for (uint32_t b0 = tc.start; b0 < tc.end; b0 += BATCH) {
      if (__syncthreads_and(done)) break;
      const int nb = static_cast<int>(min(static_cast<uint32_t>(BATCH), tc.end - b0));
      for (int j = tid; j < nb; j += nthr) {
        const uint32_t item = pv[b0 + j];
        const float4* rp = rec + 4 * static_cast<int64_t>(item);
        s_r0[j] = rp[0];
        s_r1[j] = rp[1];
        s_r2[j] = rp[2];
        s_al[j] = rp[3].x;
        s_box[j] = box[item];
      }
      __syncthreads();
      int cnt = 0;
      if (!__all_sync(0xffffffffu, done)) cnt = warp_list(s_box, nb, wb, s_list[wid]);
      if (!done) {
        for (int k = 0; k < cnt; k += 2) {
          const int jj[2] = {s_list[wid][k], k + 1 < cnt ? s_list[wid][k + 1] : s_list[wid][k]};
          Eval ee[2];
#pragma unroll
          for (int q = 0; q < 2; ++q) eval_pair(s_r0[jj[q]], s_r1[jj[q]], s_r2[jj[q]], s_al[jj[q]], dx, dy, dz, ee[q]);
#pragma unroll
          for (int q = 0; q < 2; ++q) {
            if (done || k + q >= cnt) break;
            const int j = jj[q];
            const Eval& e = ee[q];
            ++evals;
            if (!e.valid) continue;
            const float Tn = __fmul_rn(T, __fsub_rn(1.0f, e.a));
            if (Tn < 1e-4f) {
              done = true;
              stop_at = static_cast<int>(b0 - tc.start) + j + 1;
              break;
            }
            const float w = e.a * T;
            const float ws = e.den > 0.f ? -w : w;
            A += w;
            St = fmaf(w, e.t, St);
            Sx = fmaf(ws, s_r0[j].x, Sx);
            Sy = fmaf(ws, s_r0[j].y, Sy);
            Sz = fmaf(ws, s_r0[j].z, Sz);
            T = Tn;
            last = static_cast<int>(b0 - tc.start) + j + 1;
            ++contrib;
          }
          if (done) break;
        }
      }
    }
    if (tc.inside) {
      F.A[tc.pix] = A;
      F.St[tc.pix] = St;
      F.Sn[tc.pix] = Sx;
      F.Sn[tc.HW + tc.pix] = Sy;
      F.Sn[2 * static_cast<int64_t>(tc.HW) + tc.pix] = Sz;
      F.Tf[tc.pix] = T;
      F.nc[tc.pix] = last;
      alg += stop_at >= 0 ? static_cast<uint32_t>(stop_at) : tc.end - tc.start;
    }
  }
  unsigned long long ev = evals, co = contrib;
  for (int o = 16; o > 0; o >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, o);
    co += __shfl_xor_sync(0xffffffffu, co, o);
  }
  unsigned long long al = alg;
  for (int o = 16; o > 0; o >>= 1) al += __shfl_xor_sync(0xffffffffu, al, o);
  if ((tid & 31) == 0 && ev) atomicAdd(&st->evals_fwd, ev);
  if ((tid & 31) == 0 && co) atomicAdd(&st->contrib_fwd, co);
  if ((tid & 31) == 0 && al) atomicAdd(&st->alg_fwd, al);
}

// ---------------------------------------------------------------------------
// Backward
// ---------------------------------------------------------------------------
// Butterfly reduce-scatter of 16 values over the warp: afterwards lane L holds
// in v[0] the warp sum of value index 8 b4 + 4 b3 + 2 b2 + b1 (bits of L).
__device__ __forceinline__ void warp_reduce16(float (&v)[16], int lane) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool hi = lane & 16;
    const float send = hi ? v[i] : v[i + 8];
    const float keep = hi ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool hi = lane & 8;
    const float send = hi ? v[i] : v[i + 4];
    const float keep = hi ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = lane & 4;
    const float send = hi ? v[i] : v[i + 2];
    const float keep = hi ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool hi = lane & 2;
    const float send = hi ? v[0] : v[1];
    const float keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
}

template <int BATCH>
__global__ void __launch_bounds__(kMaxTileThreads)
    k_bwd(const Desc* __restrict__ D, const uint2* __restrict__ ranges, const uint32_t* __restrict__ pv,
          const float4* __restrict__ rec, const float4* __restrict__ box, float* __restrict__ g13,
          const uint32_t* __restrict__ order, Status* __restrict__ st, int persistent) {
  __shared__ float4 s_r0[BATCH], s_r1[BATCH], s_r2[BATCH], s_r3[BATCH], s_box[BATCH];
  __shared__ uint16_t s_list[kMaxTileThreads / 32][BATCH];
  __shared__ uint32_t s_item[BATCH];
  __shared__ float s_g[kGrad][BATCH];
  __shared__ int s_max;
  const int nthr = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31;
  const int gidx = 8 * ((lane >> 4) & 1) + 4 * ((lane >> 3) & 1) + 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1);
  const bool writer = ((lane & 1) == 0) && gidx < kGrad;
  uint32_t tile;
  uint32_t evals = 0, contrib = 0;
  for (int iter = 0; next_tile(persistent, order, D->n_tiles, &st->work_counter2, tile, iter); ++iter) {
    const TileCtx tc = tile_ctx(*D, tile, ranges);
    if (tc.end - tc.start > kLongList) continue;   // the long-list kernels' tile
    const FrameDev& F = D->f[tc.f];
    const WarpBox wb = warp_box(tc.inside, tc.r, tc.c, F.W);
    float dx = 0.f, dy = 0.f, dz = 0.f;
    float T = 1.f, gA = 0.f, gSt = 0.f, gSx = 0.f, gSy = 0.f, gSz = 0.f;
    int nc = 0;
    if (tc.inside) {
      pixel_ray(F, tc.r, tc.c, dx, dy, dz);
      T = F.Tf[tc.pix];
      nc = F.nc[tc.pix];
      gA = F.gA[tc.pix];
      gSt = F.gSt[tc.pix];
      gSx = F.gSn[tc.pix];
      gSy = F.gSn[tc.HW + tc.pix];
      gSz = F.gSn[2 * static_cast<int64_t>(tc.HW) + tc.pix];
    }
    if (tid == 0) s_max = 0;
    __syncthreads();
    if (nc > 0) atomicMax(&s_max, nc);
    __syncthreads();
    // n_contrib comes from the caller: never walk past the tile's list
    const uint32_t len = tc.end - tc.start;
    const uint32_t stop = tc.start + min(static_cast<uint32_t>(s_max), len);
    float S = 0.f;
    for (uint32_t bend = stop; bend > tc.start;) {
      const uint32_t b0 = bend - tc.start > static_cast<uint32_t>(BATCH) ? bend - BATCH : tc.start;
      const int nb = static_cast<int>(bend - b0);
      __syncthreads();
      for (int j = tid; j < nb; j += nthr) {
        const uint32_t item = pv[b0 + j];
        s_item[j] = item;
        const float4* rp = rec + 4 * static_cast<int64_t>(item);
        s_r0[j] = rp[0];
        s_r1[j] = rp[1];
        s_r2[j] = rp[2];
        s_r3[j] = rp[3];
        s_box[j] = box[item];
#pragma unroll
        for (int c = 0; c < kGrad; ++c) s_g[c][j] = 0.f;
      }
      __syncthreads();
      const int cnt = warp_list(s_box, nb, wb, s_list[tid >> 5]);
      for (int kk = cnt - 1; kk >= 0; --kk) {
        const int j = s_list[tid >> 5][kk];
        const int k = static_cast<int>(b0 - tc.start) + j;
        float v[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) v[c] = 0.f;
        bool valid = false;
        if (k < nc) {
          const float4 r0 = s_r0[j];
          const float alpha = s_r3[j].x;
          Eval e;
          eval_pair(r0, s_r1[j], s_r2[j], alpha, dx, dy, dz, e);
          ++evals;
          valid = e.valid;
          if (valid) {
            ++contrib;
            contrib_moments(e, r0, gA, gSt, gSx, gSy, gSz, T, S, v);
          }
        }
        if (__any_sync(0xffffffffu, valid)) {
          warp_reduce16(v, lane);
          if (writer) atomicAdd(&s_g[gidx][j], v[0]);
        }
      }
      __syncthreads();
      for (int j = tid; j < nb; j += nthr) {
        float* gp = g13 + 16 * static_cast<int64_t>(s_item[j]);
#pragma unroll
        for (int c = 0; c < kGrad; ++c) {
          const float x = s_g[c][j];
          if (x != 0.f) atomicAdd(gp + c, x);
        }
      }
      bend = b0;
    }
  }
  unsigned long long ev = evals, co = contrib;
  for (int o = 16; o > 0; o >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, o);
    co += __shfl_xor_sync(0xffffffffu, co, o);
  }
  if ((tid & 31) == 0 && ev) atomicAdd(&st->evals_bwd, ev);
  if ((tid & 31) == 0 && co) atomicAdd(&st->contrib_bwd, co);
}

// ---------------------------------------------------------------------------
// Warp-independent walk (batch = 0)
// ---------------------------------------------------------------------------
// Each warp culls and composites the tile list on its own: 32 entries per
// step (one pixel box per lane, compacted with a ballot), records of the hits
// read by the whole warp from L1 (broadcast loads; a tile's records are
// shared by its warps through L1 instead of shared memory), the next hit's
// record fetched while the current one is composited.  No CTA barrier sits in
// the loop: a warp leaves when its own pixels have stopped, and the backward
// walks only up to its own pixels' last contributor.  The per-pixel
// arithmetic and order are those of the batched kernels (results are
// bit-identical in the forward).
struct Rec {
  float4 r0, r1, r2, r3;
};

__device__ __forceinline__ Rec load_rec(const float4* __restrict__ rec, uint32_t item) {
  const float4* rp = rec + 4 * static_cast<int64_t>(item);
  Rec r;
  r.r0 = __ldg(rp);
  r.r1 = __ldg(rp + 1);
  r.r2 = __ldg(rp + 2);
  r.r3 = __ldg(rp + 3);
  return r;
}

// G hits per step: their records are fetched and evaluated together (G
// independent chains for the scheduler), then composited in list order.
template <int G>
__global__ void __launch_bounds__(kMaxTileThreads)
    k_fwd_w(const Desc* __restrict__ D, const uint2* __restrict__ ranges, const uint32_t* __restrict__ pv,
            const float4* __restrict__ rec, const float4* __restrict__ box, const uint32_t* __restrict__ order,
            Status* __restrict__ st, int persistent) {
  const int lane = threadIdx.x & 31;
  uint32_t tile;
  uint32_t evals = 0, contrib = 0, alg = 0;
  for (int iter = 0; next_tile(persistent, order, D->n_tiles, &st->work_counter, tile, iter); ++iter) {
    const TileCtx tc = tile_ctx(*D, tile, ranges);
    if (tc.end - tc.start > kLongList) continue;   // the long-list kernels' tile
    const FrameDev& F = D->f[tc.f];
    const WarpBox wb = warp_box(tc.inside, tc.r, tc.c, F.W);
    float dx = 0.f, dy = 0.f, dz = 0.f;
    if (tc.inside) pixel_ray(F, tc.r, tc.c, dx, dy, dz);
    float T = 1.0f, A = 0.0f, St = 0.0f, Sx = 0.0f, Sy = 0.0f, Sz = 0.0f;
    int last = 0, stop_at = -1;
    bool done = !tc.inside;
    for (uint32_t base = tc.start; base < tc.end; base += 32) {
      if (__all_sync(0xffffffffu, done)) break;
      const uint32_t j = base + lane;
      uint32_t item = 0;
      bool hit = false;
      if (j < tc.end) {
        item = __ldg(pv + j);
        hit = box_hits(__ldg(box + item), wb);
      }
      uint32_t m = __ballot_sync(0xffffffffu, hit);
      while (m) {
        int bq[G];
        float4 r0[G], r1[G], r2[G];
        float al[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
          bq[q] = m ? __ffs(m) - 1 : -1;
          m &= m - 1;
          if (bq[q] >= 0) {
            const float4* rp = rec + 4 * static_cast<int64_t>(__shfl_sync(0xffffffffu, item, bq[q]));
            r0[q] = __ldg(rp);
            r1[q] = __ldg(rp + 1);
            r2[q] = __ldg(rp + 2);
            al[q] = __ldg(reinterpret_cast<const float*>(rp + 3));
          }
        }
        Eval e[G];
#pragma unroll
        for (int q = 0; q < G; ++q)
          if (bq[q] >= 0) eval_pair(r0[q], r1[q], r2[q], al[q], dx, dy, dz, e[q]);
#pragma unroll
        for (int q = 0; q < G; ++q) {
          if (bq[q] < 0 || done) continue;
          ++evals;
          if (!e[q].valid) continue;
          const float Tn = __fmul_rn(T, __fsub_rn(1.0f, e[q].a));
          if (Tn < 1e-4f) {
            done = true;
            stop_at = static_cast<int>(base - tc.start) + bq[q] + 1;
            continue;
          }
          const float w = e[q].a * T;
          const float ws = e[q].den > 0.f ? -w : w;
          A += w;
          St = fmaf(w, e[q].t, St);
          Sx = fmaf(ws, r0[q].x, Sx);
          Sy = fmaf(ws, r0[q].y, Sy);
          Sz = fmaf(ws, r0[q].z, Sz);
          T = Tn;
          last = static_cast<int>(base - tc.start) + bq[q] + 1;
          ++contrib;
        }
        if (__all_sync(0xffffffffu, done)) break;
      }
    }
    if (tc.inside) {
      F.A[tc.pix] = A;
      F.St[tc.pix] = St;
      F.Sn[tc.pix] = Sx;
      F.Sn[tc.HW + tc.pix] = Sy;
      F.Sn[2 * static_cast<int64_t>(tc.HW) + tc.pix] = Sz;
      F.Tf[tc.pix] = T;
      F.nc[tc.pix] = last;
      alg += stop_at >= 0 ? static_cast<uint32_t>(stop_at) : tc.end - tc.start;
    }
  }
  unsigned long long ev = evals, co = contrib;
  for (int o = 16; o > 0; o >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, o);
    co += __shfl_xor_sync(0xffffffffu, co, o);
  }
  unsigned long long al = alg;
  for (int o = 16; o > 0; o >>= 1) al += __shfl_xor_sync(0xffffffffu, al, o);
  if (lane == 0 && ev) atomicAdd(&st->evals_fwd, ev);
  if (lane == 0 && co) atomicAdd(&st->contrib_fwd, co);
  if (lane == 0 && al) atomicAdd(&st->alg_fwd, al);
}

template <int G>
__global__ void __launch_bounds__(kMaxTileThreads)
    k_bwd_w(const Desc* __restrict__ D, const uint2* __restrict__ ranges, const uint32_t* __restrict__ pv,
            const float4* __restrict__ rec, const float4* __restrict__ box, float* __restrict__ g13,
            const uint32_t* __restrict__ order, Status* __restrict__ st, int persistent) {
  const int lane = threadIdx.x & 31;
  const int gidx = 8 * ((lane >> 4) & 1) + 4 * ((lane >> 3) & 1) + 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1);
  const bool writer = ((lane & 1) == 0) && gidx < kGrad;
  uint32_t tile;
  uint32_t evals = 0, contrib = 0;
  for (int iter = 0; next_tile(persistent, order, D->n_tiles, &st->work_counter2, tile, iter); ++iter) {
    const TileCtx tc = tile_ctx(*D, tile, ranges);
    if (tc.end - tc.start > kLongList) continue;   // the long-list kernels' tile
    const FrameDev& F = D->f[tc.f];
    const WarpBox wb = warp_box(tc.inside, tc.r, tc.c, F.W);
    float dx = 0.f, dy = 0.f, dz = 0.f;
    float T = 1.f, gA = 0.f, gSt = 0.f, gSx = 0.f, gSy = 0.f, gSz = 0.f;
    int nc = 0;
    if (tc.inside) {
      pixel_ray(F, tc.r, tc.c, dx, dy, dz);
      T = F.Tf[tc.pix];
      nc = F.nc[tc.pix];
      gA = F.gA[tc.pix];
      gSt = F.gSt[tc.pix];
      gSx = F.gSn[tc.pix];
      gSy = F.gSn[tc.HW + tc.pix];
      gSz = F.gSn[2 * static_cast<int64_t>(tc.HW) + tc.pix];
    }
    // n_contrib comes from the caller: never walk past the tile's list
    const uint32_t len = tc.end - tc.start;
    const uint32_t stop = min(static_cast<uint32_t>(__reduce_max_sync(0xffffffffu, nc > 0 ? nc : 0)), len);
    float S = 0.f;
    for (int c0 = static_cast<int>((stop + 31) / 32) - 1; c0 >= 0; --c0) {
      const uint32_t k0 = 32u * c0;
      uint32_t item = 0;
      bool hit = false;
      if (k0 + lane < stop) {
        item = __ldg(pv + tc.start + k0 + lane);
        hit = box_hits(__ldg(box + item), wb);
      }
      uint32_t m = __ballot_sync(0xffffffffu, hit);
      while (m) {
        int bq[G];
        uint32_t itq[G];
        float4 r0[G], r1[G], r2[G];
        float al[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
          bq[q] = m ? 31 - __clz(m) : -1;
          if (bq[q] >= 0) {
            m &= ~(1u << bq[q]);
            itq[q] = __shfl_sync(0xffffffffu, item, bq[q]);
            const float4* rp = rec + 4 * static_cast<int64_t>(itq[q]);
            r0[q] = __ldg(rp);
            r1[q] = __ldg(rp + 1);
            r2[q] = __ldg(rp + 2);
            al[q] = __ldg(reinterpret_cast<const float*>(rp + 3));
          }
        }
        Eval e[G];
        bool in[G];
#pragma unroll
        for (int q = 0; q < G; ++q) {
          in[q] = bq[q] >= 0 && static_cast<int>(k0 + bq[q]) < nc;
          if (in[q]) eval_pair(r0[q], r1[q], r2[q], al[q], dx, dy, dz, e[q]);
        }
#pragma unroll
        for (int q = 0; q < G; ++q) {
          if (bq[q] < 0) break;
          const bool valid = in[q] && e[q].valid;
          evals += in[q];
          float v[16];
#pragma unroll
          for (int c = 0; c < 16; ++c) v[c] = 0.f;
          if (valid) {
            ++contrib;
            contrib_moments(e[q], r0[q], gA, gSt, gSx, gSy, gSz, T, S, v);
          }
          if (__any_sync(0xffffffffu, valid)) {
            warp_reduce16(v, lane);
            if (writer && v[0] != 0.f) atomicAdd(g13 + 16 * static_cast<int64_t>(itq[q]) + gidx, v[0]);
          }
        }
      }
    }
  }
  unsigned long long ev = evals, co = contrib;
  for (int o = 16; o > 0; o >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, o);
    co += __shfl_xor_sync(0xffffffffu, co, o);
  }
  if (lane == 0 && ev) atomicAdd(&st->evals_bwd, ev);
  if (lane == 0 && co) atomicAdd(&st->contrib_bwd, co);
}

// ---------------------------------------------------------------------------
// Reduce-scatter of the 12 gradient moments of one (warp, entry) over the
// warp: 15 shuffles for 12 values.
// ---------------------------------------------------------------------------
// Reduce-scatter of 12 values over the warp.  Afterwards the warp sum of
// value 6 b4 + 3 b3 + b2 is held by the lanes with (lane & 3) == 0 and that
// of value 6 b4 + 3 b3 + 2 by the lanes with (lane & 7) == 1 (b4, b3, b2 the
// lane's bits); returns the lane's value and sets idx (-1: not a writer).
__device__ __forceinline__ float warp_reduce12(const float (&v)[12], int lane, int& idx) {
  const bool b4 = lane & 16, b3 = lane & 8, b2 = lane & 4;
  float w[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const float send = b4 ? v[i] : v[i + 6];
    const float keep = b4 ? v[i + 6] : v[i];
    w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  float x[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float send = b3 ? w[i] : w[i + 3];
    const float keep = b3 ? w[i + 3] : w[i];
    x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  float y0, y2;
  {
    const float send = b2 ? x[0] : x[1];
    const float keep = b2 ? x[1] : x[0];
    y0 = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    y2 = x[2] + __shfl_xor_sync(0xffffffffu, x[2], 4);
  }
  y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
  y2 += __shfl_xor_sync(0xffffffffu, y2, 2);
  y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
  y2 += __shfl_xor_sync(0xffffffffu, y2, 1);
  const int base = (b4 ? 6 : 0) + (b3 ? 3 : 0);
  const bool first = (lane & 3) == 0;
  idx = first ? base + (b2 ? 1 : 0) : ((lane & 7) == 1 ? base + 2 : -1);
  return first ? y0 : y2;
}

// ---------------------------------------------------------------------------
// Shared-memory walk (group 16): each warp walks its tile list in chunks of
// 32 entries; the records of the chunk's hits are staged in the warp's own
// shared-memory slots (one 48-B record per lane) and read back with broadcast
// loads, so a hit costs no shuffle, no 64-bit address arithmetic and no
// global load on the critical path.  No CTA barrier: warps proceed alone.
// ---------------------------------------------------------------------------
struct WarpRecs {
  float4 r0[32], r1[32], r2[32];
  float al[32];
};

__device__ __forceinline__ void stage_hit(const float4* __restrict__ rec, uint32_t item, WarpRecs& s, int lane) {
  const float4* rp = rec + 4 * static_cast<int64_t>(item);
  s.r0[lane] = __ldg(rp);
  s.r1[lane] = __ldg(rp + 1);
  s.r2[lane] = __ldg(rp + 2);
  s.al[lane] = __ldg(reinterpret_cast<const float*>(rp + 3));
}

// Image-loss epilogue of the forward kernels: the pixel's terms from its
// composited values still in registers (no re-read of the planes), its
// upstream gradient planes written, the terms' fixed-point values summed over
// the warp and added to the frame's loss sums (one atomic per term and warp).
struct LossEpi {
  lgs_loss_params P;
  int* ctot;                     // mask counts [frame][2], complete before the forward
  unsigned long long* acc;       // fixed-point sums [frame][4], then [maps] of the regulariser
  float* out;                    // loss vector, written by the long-list forward's last CTA
};

__device__ __forceinline__ void loss_epilogue(const Desc& D, const LossEpi& L, int f, bool inside, int64_t pix,
                                              int HW, float A, float St, float Sx, float Sy, float Sz) {
  long long ld = 0, la = 0, ln = 0;
  if (inside) {
    const FrameDev& F = D.f[f];
    const int nd = __ldcg(L.ctot + 2 * f), nn = __ldcg(L.ctot + 2 * f + 1);
    const float scale = 1.0f / static_cast<float>(D.m[F.map].n_frames);
    const float ind = nd > 0 ? 1.0f / static_cast<float>(nd) : 0.f;
    const float inn = nn > 0 ? 1.0f / static_cast<float>(nn) : 0.f;
    float g[5];
    pixel_image_loss(F.D[pix], A, St, F.Ng[pix], F.Ng[HW + pix], F.Ng[2 * static_cast<int64_t>(HW) + pix], Sx, Sy,
                     Sz, scale, ind, inn, L.P, g, ld, la, ln);
    F.oA[pix] = g[0];
    F.oSt[pix] = g[1];
    F.oSn[pix] = g[2];
    F.oSn[HW + pix] = g[3];
    F.oSn[2 * static_cast<int64_t>(HW) + pix] = g[4];
  }
  for (int o = 16; o > 0; o >>= 1) {
    ld += __shfl_xor_sync(0xffffffffu, ld, o);
    la += __shfl_xor_sync(0xffffffffu, la, o);
    ln += __shfl_xor_sync(0xffffffffu, ln, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (ld) atomicAdd(L.acc + 4 * f, static_cast<unsigned long long>(ld));
    if (la) atomicAdd(L.acc + 4 * f + 1, static_cast<unsigned long long>(la));
    if (ln) atomicAdd(L.acc + 4 * f + 2, static_cast<unsigned long long>(ln));
  }
}

// hits evaluated together per step of the shared-memory forward (3 measured
// fastest on the street frame: 2 leaves latency exposed, 4 costs registers)
constexpr int FWD_HITS = 3;

// At most 72 registers: 14 CTAs of an 8 x 8 tile (64 threads) per SM, so
// the 2048 tiles of a 128 x 1024 frame fit in one wave on 152 SMs (75
// registers leave 72 tiles for a second wave).
template <bool LOSS>
__global__ void __maxnreg__(72)
    k_fwd_s(const Desc* __restrict__ D, const uint2* __restrict__ ranges, const uint32_t* __restrict__ pv,
            const float4* __restrict__ rec, const float4* __restrict__ box, const uint32_t* __restrict__ order,
            Status* __restrict__ st, int persistent, const uint32_t* __restrict__ cbase, float* __restrict__ ckpt,
            uint32_t* __restrict__ cmask, uint32_t* __restrict__ bwm, LossEpi loss) {
  pdl_wait();               // (launched after a kernel of this chain: wait for it)
  pdl_launch_dependents();  // the next kernel may be dispatched now
  __shared__ WarpRecs s_w[kMaxTileThreads / 32];
  const int lane = threadIdx.x & 31;
  WarpRecs& sw = s_w[threadIdx.x >> 5];
  uint32_t tile;
  uint32_t evals = 0, contrib = 0, alg = 0;
  for (int iter = 0; next_tile(persistent, order, D->n_tiles, &st->work_counter, tile, iter); ++iter) {
    const TileCtx tc = tile_ctx(*D, tile, ranges);
    if (tc.end - tc.start > kLongList) continue;   // the long-list kernels' tile
    const FrameDev& F = D->f[tc.f];
    const WarpBox wb = warp_box(tc.inside, tc.r, tc.c, F.W);
    float dx = 0.f, dy = 0.f, dz = 0.f;
    if (tc.inside) pixel_ray(F, tc.r, tc.c, dx, dy, dz);
    float T = 1.0f, A = 0.0f, St = 0.0f, Sx = 0.0f, Sy = 0.0f, Sz = 0.0f;
    int last = 0, stop_at = -1;
    bool done = !tc.inside;
    // checkpoint of the backward chunks: this chunk's own sums, written with
    // T at every chunk end (the chunk holding the end of the walk included)
    float cA = 0.f, cSt = 0.f, cSx = 0.f, cSy = 0.f, cSz = 0.f;
    uint32_t chunk = 0;
    const int npx = static_cast<int>(blockDim.x);
    const auto checkpoint = [&]() {
      float* o = ckpt + (static_cast<int64_t>(cbase[tile] + chunk) * kCkptSlots) * npx + threadIdx.x;
      o[0] = T;
      o[npx] = cA;
      o[2 * npx] = cSt;
      o[3 * npx] = cSx;
      o[4 * npx] = cSy;
      o[5 * npx] = cSz;
      cA = cSt = cSx = cSy = cSz = 0.f;
    };
    // software pipeline over the windows: the list entry two windows ahead
    // and the culling box one window ahead are loaded while this window is
    // composited (entry, box and record would otherwise be a chain of
    // dependent round trips per window)
    uint32_t item_nx = tc.start + 32 + lane < tc.end ? __ldg(pv + tc.start + 32 + lane) : 0u;
    uint32_t item_cur = tc.start + lane < tc.end ? __ldg(pv + tc.start + lane) : 0u;
    float4 box_cur = tc.start + lane < tc.end ? __ldg(box + item_cur) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t base = tc.start; base < tc.end; base += 32) {
      if (base - tc.start >= (chunk + 1) * kChunk) {
        checkpoint();
        ++chunk;
      }
      if (__all_sync(0xffffffffu, done)) break;
      // the pixel's composited entries of this window, one bit each, for the
      // chunked backward (every window the warp walks gets its word)
      uint32_t* mword = cmask + (static_cast<int64_t>(cbase[tile]) * 4 + (base - tc.start) / 32) * npx + threadIdx.x;
      const uint32_t j = base + lane;
      const uint32_t item = item_cur;
      const float4 bx = box_cur;
      item_cur = item_nx;
      box_cur = j + 32 < tc.end ? __ldg(box + item_nx) : make_float4(0.f, 0.f, 0.f, 0.f);
      item_nx = j + 64 < tc.end ? __ldg(pv + j + 64) : 0u;
      bool hit = false;
      if (j < tc.end) hit = box_hits(bx, wb);
      uint32_t m = __ballot_sync(0xffffffffu, hit);
      if (!m) {
        *mword = 0u;
        continue;
      }
      const uint32_t m_hits = m;
      const bool done_before = done;
      __syncwarp();
      if (hit) stage_hit(rec, item, sw, lane);
      __syncwarp();
      const int k0 = static_cast<int>(base - tc.start) + 1;
      uint32_t cbits = 0;
      // composite one evaluated hit without branches: lanes that are done or
      // see an invalid pair add zeros and keep T (t and the weight are zeroed
      // first, so no inf or NaN of a rejected pair reaches the sums)
      const auto composite = [&](const Eval& e, const float4& r0, int bq) {
        const bool act = !done && e.valid;
        const float Tn = __fmul_rn(T, __fsub_rn(1.0f, e.a));
        const bool stop = act && Tn < 1e-4f;
        const bool comp = act && !(Tn < 1e-4f);
        const float w = comp ? e.a * T : 0.0f;
        const float tt = comp ? e.t : 0.0f;
        const float ws = e.den > 0.f ? -w : w;
        A += w;
        St = fmaf(w, tt, St);
        Sx = fmaf(ws, r0.x, Sx);
        Sy = fmaf(ws, r0.y, Sy);
        Sz = fmaf(ws, r0.z, Sz);
        cA += w;
        cSt = fmaf(w, tt, cSt);
        cSx = fmaf(ws, r0.x, cSx);
        cSy = fmaf(ws, r0.y, cSy);
        cSz = fmaf(ws, r0.z, cSz);
        T = comp ? Tn : T;
        cbits |= comp ? 1u << bq : 0u;
        stop_at = stop ? k0 + bq : stop_at;
        done = done || stop;
      };
      // FWD_HITS hits per step: their evaluations are independent
      // (instruction-level parallelism), the composites follow in list order
      do {
        int bq[FWD_HITS];
        bq[0] = __ffs(m) - 1;
        m &= m - 1;
#pragma unroll
        for (int q = 1; q < FWD_HITS; ++q) {
          bq[q] = m ? __ffs(m) - 1 : -1;
          m &= m - 1;
        }
        float4 r0q[FWD_HITS];
        Eval eq[FWD_HITS];
#pragma unroll
        for (int q = 0; q < FWD_HITS; ++q) {
          const int b = bq[q] >= 0 ? bq[q] : bq[0];
          r0q[q] = sw.r0[b];
          eval_pair(r0q[q], sw.r1[b], sw.r2[b], sw.al[b], dx, dy, dz, eq[q]);
        }
#pragma unroll
        for (int q = 0; q < FWD_HITS; ++q)
          if (bq[q] >= 0) composite(eq[q], r0q[q], bq[q]);
        if (__all_sync(0xffffffffu, done)) break;
      } while (m);
      *mword = cbits;
      // the window's statistics from its bits: composited pairs, the last
      // one, and the hits evaluated before the pixel stopped (through the
      // stop entry when it stopped in this window)
      if (cbits) last = k0 + (31 - __clz(cbits));
      contrib += __popc(cbits);
      if (!done_before)
        evals += __popc(stop_at >= k0 ? m_hits & (0xffffffffu >> (31 - (stop_at - k0))) : m_hits);
    }
    if (tc.end > tc.start) checkpoint();
    if (tc.inside) {
      F.A[tc.pix] = A;
      F.St[tc.pix] = St;
      F.Sn[tc.pix] = Sx;
      F.Sn[tc.HW + tc.pix] = Sy;
      F.Sn[2 * static_cast<int64_t>(tc.HW) + tc.pix] = Sz;
      F.Tf[tc.pix] = T;
      F.nc[tc.pix] = last;
      alg += stop_at >= 0 ? static_cast<uint32_t>(stop_at) : tc.end - tc.start;
    }
    // the block's largest n_contrib: the backward's chunks of this block end there
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, static_cast<uint32_t>(last));
    if (lane == 0) bwm[tile * (blockDim.x >> 5) + (threadIdx.x >> 5)] = wmax;
    if (LOSS) loss_epilogue(*D, loss, tc.f, tc.inside, tc.pix, tc.HW, A, St, Sx, Sy, Sz);
  }
  unsigned long long ev = evals, co = contrib;
  for (int o = 16; o > 0; o >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, o);
    co += __shfl_xor_sync(0xffffffffu, co, o);
  }
  unsigned long long al = alg;
  for (int o = 16; o > 0; o >>= 1) al += __shfl_xor_sync(0xffffffffu, al, o);
  if (lane == 0 && ev) atomicAdd(&st->evals_fwd, ev);
  if (lane == 0 && co) atomicAdd(&st->contrib_fwd, co);
  if (lane == 0 && al) atomicAdd(&st->alg_fwd, al);
}

__global__ void __launch_bounds__(kMaxTileThreads)
    k_bwd_s(const Desc* __restrict__ D, const uint2* __restrict__ ranges, const uint32_t* __restrict__ pv,
            const float4* __restrict__ rec, const float4* __restrict__ box, float* __restrict__ g13,
            const uint32_t* __restrict__ order, Status* __restrict__ st, int persistent) {
  __shared__ WarpRecs s_w[kMaxTileThreads / 32];
  __shared__ uint32_t s_item[kMaxTileThreads / 32][32];
  const int lane = threadIdx.x & 31;
  WarpRecs& sw = s_w[threadIdx.x >> 5];
  uint32_t* si = s_item[threadIdx.x >> 5];
  uint32_t tile;
  uint32_t evals = 0, contrib = 0;
  for (int iter = 0; next_tile(persistent, order, D->n_tiles, &st->work_counter2, tile, iter); ++iter) {
    const TileCtx tc = tile_ctx(*D, tile, ranges);
    if (tc.end - tc.start > kLongList) continue;   // the long-list kernels' tile
    const FrameDev& F = D->f[tc.f];
    const WarpBox wb = warp_box(tc.inside, tc.r, tc.c, F.W);
    float dx = 0.f, dy = 0.f, dz = 0.f;
    float T = 1.f, gA = 0.f, gSt = 0.f, gSx = 0.f, gSy = 0.f, gSz = 0.f;
    int nc = 0;
    if (tc.inside) {
      pixel_ray(F, tc.r, tc.c, dx, dy, dz);
      T = F.Tf[tc.pix];
      nc = F.nc[tc.pix];
      gA = F.gA[tc.pix];
      gSt = F.gSt[tc.pix];
      gSx = F.gSn[tc.pix];
      gSy = F.gSn[tc.HW + tc.pix];
      gSz = F.gSn[2 * static_cast<int64_t>(tc.HW) + tc.pix];
    }
    // n_contrib comes from the caller: never walk past the tile's list
    const uint32_t len = tc.end - tc.start;
    const uint32_t stop = min(static_cast<uint32_t>(__reduce_max_sync(0xffffffffu, nc > 0 ? nc : 0)), len);
    float S = 0.f;
    for (int c0 = static_cast<int>((stop + 31) / 32) - 1; c0 >= 0; --c0) {
      const int k0 = 32 * c0;
      uint32_t item = 0;
      bool hit = false;
      if (static_cast<uint32_t>(k0 + lane) < stop) {
        item = __ldg(pv + tc.start + k0 + lane);
        hit = box_hits(__ldg(box + item), wb);
      }
      uint32_t m = __ballot_sync(0xffffffffu, hit);
      if (!m) continue;
      __syncwarp();
      if (hit) {
        stage_hit(rec, item, sw, lane);
        si[lane] = item;
      }
      __syncwarp();
      do {
        const int bq = 31 - __clz(m);
        m &= ~(1u << bq);
        const bool in = k0 + bq < nc;
        const float4 r0 = sw.r0[bq];
        Eval e;
        eval_pair(r0, sw.r1[bq], sw.r2[bq], sw.al[bq], dx, dy, dz, e);
        const bool valid = in && e.valid;
        evals += in;
        contrib += valid;
        if (!__any_sync(0xffffffffu, valid)) continue;
        // invalid lanes: zero opacity and finite inputs, so every moment is
        // exactly 0 and T, S pass through unchanged
        const float a = valid ? e.a : 0.f;
        const float araw = valid ? e.araw : 0.f;
        const float t = valid ? e.t : 0.f;
        const float u = valid ? e.u : 0.f;
        const float v = valid ? e.v : 0.f;
        const float rden = valid ? e.rden : 0.f;
        const float iom = rcp_ftz(1.0f - a);
        const float Tk = T * iom;
        const float sg = e.den > 0.f ? -1.f : 1.f;
        const float gc = gA + gSt * t + sg * (gSx * r0.x + gSy * r0.y + gSz * r0.z);
        const float w = a * Tk;
        const float dLda = Tk * gc - S * iom;
        S = fmaf(w, gc, S);
        T = Tk;
        const float g = araw < 0.99f ? araw * dLda : 0.f;
        const float ug = u * g, vg = v * g;
        const float ct = fmaf(w, gSt, -fmaf(ug, e.ud, vg * e.vd)) * rden;
        const float wsg = w * sg;
        float mv[12];
        mv[0] = g;
        mv[1] = ug;
        mv[2] = vg;
        mv[3] = u * ug;
        mv[4] = v * vg;
        mv[5] = u * vg;
        mv[6] = ct;
        mv[7] = ct * u;
        mv[8] = ct * v;
        mv[9] = wsg * gSx;
        mv[10] = wsg * gSy;
        mv[11] = wsg * gSz;
        int idx;
        const float r = warp_reduce12(mv, lane, idx);
        if (idx >= 0 && r != 0.f) atomicAdd(g13 + 16 * static_cast<int64_t>(si[bq]) + idx, r);
      } while (m);
    }
  }
  unsigned long long ev = evals, co = contrib;
  for (int o = 16; o > 0; o >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, o);
    co += __shfl_xor_sync(0xffffffffu, co, o);
  }
  if (lane == 0 && ev) atomicAdd(&st->evals_bwd, ev);
  if (lane == 0 && co) atomicAdd(&st->contrib_bwd, co);
}

// ---------------------------------------------------------------------------
// Chunked backward (group 16 after the shared-memory forward): a work item
// is one warp's 4 x 8 pixel block of a tile over one chunk of kChunk list
// entries, claimed through an atomic counter from k_bwd_prep's queues: only
// chunks that hold one of the block's composited entries, chunks walked in
// full first, then the last ones by decreasing walked length (a warp that
// claims late gets a short item, so the SMs finish together).  The reverse
// walk of chunk c starts from the forward's checkpoint: T at the end of the
// chunk, and the suffix S = sum over the later chunks c' of gA dA_c' + gSt
// dSt_c' + gS . dSn_c' (their own sums of w, w t, w n').  Items are
// independent, so a frame offers several times more warps than pixel
// blocks.
// ---------------------------------------------------------------------------
constexpr int kBwdChunkCta = 256;

__global__ void __launch_bounds__(kBwdChunkCta)
    k_bwd_c(const Desc* __restrict__ D, const uint2* __restrict__ ranges, const uint32_t* __restrict__ pv,
            const float4* __restrict__ rec, const float4* __restrict__ box, float* __restrict__ g13,
            const uint32_t* __restrict__ cbase, const float* __restrict__ ckpt, const uint32_t* __restrict__ cmask,
            const float* __restrict__ csuf, const uint2* __restrict__ bq, uint32_t bq_cap0, uint32_t bq_capk,
            Status* __restrict__ st) {
  pdl_wait();               // (launched after a kernel of this chain: wait for it)
  pdl_launch_dependents();  // the next kernel may be dispatched now
  __shared__ WarpRecs s_w[kBwdChunkCta / 32];
  __shared__ uint32_t s_item[kBwdChunkCta / 32][32];
  const int lane = threadIdx.x & 31;
  WarpRecs& sw = s_w[threadIdx.x >> 5];
  uint32_t* si = s_item[threadIdx.x >> 5];
  const int npx = D->th * D->tw, wpt = npx >> 5;
  // the forward's queues, claimed in class order: lane l < kBwdClasses holds
  // class l's size (clamped to its capacity) and the items before its end
  const uint32_t qn = lane < kBwdClasses ? min(st->bq_count[lane], lane == 0 ? bq_cap0 : bq_capk) : 0u;
  uint32_t qend = qn;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t x = __shfl_up_sync(0xffffffffu, qend, o);
    if (lane >= o) qend += x;
  }
  const uint32_t n_work = __shfl_sync(0xffffffffu, qend, kBwdClasses - 1);
  while (true) {
    uint32_t id = 0;
    if (lane == 0) id = atomicAdd(&st->work_counter2, 1u);
    id = __shfl_sync(0xffffffffu, id, 0);
    if (id >= n_work) break;
    const int cls = __ffs(__ballot_sync(0xffffffffu, lane < kBwdClasses && id < qend)) - 1;
    const uint32_t first = __shfl_sync(0xffffffffu, qend - qn, cls);
    const uint2 q = __ldg(bq + (cls == 0 ? 0u : bq_cap0 + static_cast<uint32_t>(cls - 1) * bq_capk) + (id - first));
    const uint32_t k = q.x / static_cast<uint32_t>(wpt);
    const int vt = static_cast<int>(q.x - k * static_cast<uint32_t>(wpt)) * 32 + lane;   // thread of the tile
    const uint32_t tile = q.y, c = k - __ldg(cbase + tile);
    const int f = frame_of_tile(*D, tile);
    const FrameDev& F = D->f[f];
    const int lt = static_cast<int>(tile - F.tile_base);
    const int ti = lt / F.ntc, tj = lt - ti * F.ntc;
    int lr, lc;
    pixel_of_thread(F, vt, lr, lc);
    const int r = ti * F.th + lr, col = tj * F.tw + lc;
    const bool inside = r < F.H && col < F.W;
    const int HW = F.H * F.W;
    const int64_t pix = static_cast<int64_t>(r) * F.W + col;
    const uint2 rg = ranges[tile];
    const int k_lo = static_cast<int>(c * kChunk);
    const int nc = inside ? F.nc[pix] : 0;
    const bool act = nc > k_lo;
    float dx = 0.f, dy = 0.f, dz = 0.f;
    float T = 1.f, S = 0.f, gA = 0.f, gSt = 0.f, gSx = 0.f, gSy = 0.f, gSz = 0.f;
    if (act) {
      pixel_ray(F, r, col, dx, dy, dz);
      gA = F.gA[pix];
      gSt = F.gSt[pix];
      gSx = F.gSn[pix];
      gSy = F.gSn[HW + pix];
      gSz = F.gSn[2 * static_cast<int64_t>(HW) + pix];
      const float* o = ckpt + (static_cast<int64_t>(cbase[tile] + c) * kCkptSlots) * npx + vt;
      T = o[0];
      if (rg.y - rg.x > kLongList) {
        S = csuf[static_cast<int64_t>(cbase[tile] + c) * npx + vt];   // the suffix k_bwd_prep wrote
      } else {
        const uint32_t c_last = static_cast<uint32_t>(nc - 1) / kChunk;
        for (uint32_t c2 = c + 1; c2 <= c_last; ++c2) {
          const float* q = ckpt + (static_cast<int64_t>(cbase[tile] + c2) * kCkptSlots) * npx + vt;
          S += gA * q[npx] + gSt * q[2 * npx] + gSx * q[3 * npx] + gSy * q[4 * npx] + gSz * q[5 * npx];
        }
      }
    }
    // entries [k_lo, k_hi) of the list, walked down in 32-entry steps: a
    // step's hits are the entries some pixel of the warp composited (the
    // forward's window masks), and a lane takes the ones its pixel did
    const uint32_t len = rg.y - rg.x;
    const int k_hi = static_cast<int>(min(min(static_cast<uint32_t>(k_lo) + kChunk, len),
                                          static_cast<uint32_t>(__reduce_max_sync(0xffffffffu, act ? nc : 0))));
    for (int k0 = k_lo + ((k_hi - k_lo + 31) / 32 - 1) * 32; k0 >= k_lo; k0 -= 32) {
      // entries below the pixel's n_contrib only (a long list's pixels stop
      // on their own, so their words past it are not this step's)
      const int lim = nc - k0;
      uint32_t word = 0u;
      if (act && lim > 0) {
        word = __ldg(cmask + (static_cast<int64_t>(cbase[tile]) * 4 + static_cast<uint32_t>(k0) / 32) * npx + vt);
        if (lim < 32) word &= (1u << lim) - 1u;
      }
      uint32_t m = __reduce_or_sync(0xffffffffu, word);
      if (!m) continue;
      const bool hit = (m >> lane) & 1u;
      const uint32_t item = hit ? __ldg(pv + rg.x + k0 + lane) : 0u;
      __syncwarp();
      if (hit) {
        stage_hit(rec, item, sw, lane);
        si[lane] = item;
      }
      __syncwarp();
      do {
        const int bq = 31 - __clz(m);
        m &= ~(1u << bq);
        // the pixel composited this entry: its evaluation (the forward's,
        // bit for bit) is valid
        const bool valid = (word >> bq) & 1u;
        const float4 r0 = sw.r0[bq];
        Eval e;
        eval_pair(r0, sw.r1[bq], sw.r2[bq], sw.al[bq], dx, dy, dz, e);
        // invalid lanes: zero opacity and finite inputs, so every moment is
        // exactly 0 and T, S pass through unchanged
        const float a = valid ? e.a : 0.f;
        const float araw = valid ? e.araw : 0.f;
        const float t = valid ? e.t : 0.f;
        const float u = valid ? e.u : 0.f;
        const float v = valid ? e.v : 0.f;
        const float rden = valid ? e.rden : 0.f;
        const float iom = rcp_ftz(1.0f - a);
        const float Tk = T * iom;
        const float sg = e.den > 0.f ? -1.f : 1.f;
        const float gc = gA + gSt * t + sg * (gSx * r0.x + gSy * r0.y + gSz * r0.z);
        const float w = a * Tk;
        const float dLda = Tk * gc - S * iom;
        S = fmaf(w, gc, S);
        T = Tk;
        const float g = araw < 0.99f ? araw * dLda : 0.f;
        const float ug = u * g, vg = v * g;
        const float ct = fmaf(w, gSt, -fmaf(ug, e.ud, vg * e.vd)) * rden;
        const float wsg = w * sg;
        float mv[12];
        mv[0] = g;
        mv[1] = ug;
        mv[2] = vg;
        mv[3] = u * ug;
        mv[4] = v * vg;
        mv[5] = u * vg;
        mv[6] = ct;
        mv[7] = ct * u;
        mv[8] = ct * v;
        mv[9] = wsg * gSx;
        mv[10] = wsg * gSy;
        mv[11] = wsg * gSz;
        int idx;
        const float red = warp_reduce12(mv, lane, idx);
        if (idx >= 0 && red != 0.f) atomicAdd(g13 + 16 * static_cast<int64_t>(si[bq]) + idx, red);
      } while (m);
    }
  }
  // (the claim counter and the queue sizes are zeroed for the next backward
  // by k_preprocess_bwd, which follows on the stream; no statistics counters: the backward's contributions are the forward's
  // composited pairs, counted there)
}

// ---------------------------------------------------------------------------
// Long lists (more than kLongList entries): one warp per pixel
// ---------------------------------------------------------------------------
// A tile with a very long list (a far horizon seen along a street: tens of
// thousands of entries, few of which any pixel composites) would make its
// CTA walk the list one entry at a time while the rest of the frame is done.
// Here a work item is one (long tile, pixel), claimed through an atomic
// counter; the 32 lanes take 32 consecutive entries of the list for the
// warp's pixel.  Forward: the transmittance before each entry is T times a
// multiplicative scan of (1 - a) over the lanes, the early stop is the first
// lane whose T (1 - a) falls below 1e-4, and the composited sums are warp
// reductions.  Backward: from T_final, the transmittance before each entry
// is T divided by the suffix product of (1 - a), the suffix S a suffix sum;
// every valid lane adds its own entry's 12 moments with atomics.  The products
// and sums associate differently from the per-tile kernels (same values to a
// few ulps).
// Thread of the per-tile forward that holds tile pixel (lr, lc) (the inverse
// of pixel_of_thread): the chunk checkpoints and window masks are laid out by
// it.
__device__ __forceinline__ int thread_of_pixel(const FrameDev& F, int lr, int lc) {
  if ((F.tw & 7) == 0 && (F.th & 3) == 0) {
    const int wpr = F.tw >> 3;
    return ((((lr >> 2) * wpr) + (lc >> 3)) << 5) | ((lr & 3) << 3) | (lc & 7);
  }
  return lr * F.tw + lc;
}

struct LongPix {
  const FrameDev* F;
  int r, c;
  bool inside;
  uint32_t start, end, tile;
  int64_t pix;
  int HW;
  int vt;   // the pixel's thread in the per-tile layout (checkpoints, masks)
};

__device__ __forceinline__ bool long_item(const Desc& D, const uint2* __restrict__ ranges,
                                          const uint32_t* __restrict__ longt, uint32_t n_long, uint32_t id,
                                          LongPix& p) {
  const uint32_t tp = static_cast<uint32_t>(D.th * D.tw);
  const uint32_t gi = id / tp, k = id - gi * tp;
  if (gi >= n_long) return false;
  const uint32_t tile = longt[gi];
  const int f = frame_of_tile(D, tile);
  const FrameDev& F = D.f[f];
  const int lt = static_cast<int>(tile - F.tile_base);
  const int ti = lt / F.ntc, tj = lt - ti * F.ntc;
  p.F = &F;
  p.tile = tile;
  p.vt = thread_of_pixel(F, static_cast<int>(k) / F.tw, static_cast<int>(k) % F.tw);
  p.r = ti * F.th + static_cast<int>(k) / F.tw;
  p.c = tj * F.tw + static_cast<int>(k) % F.tw;
  p.inside = p.r < F.H && p.c < F.W;
  p.pix = static_cast<int64_t>(p.r) * F.W + p.c;
  p.HW = F.H * F.W;
  const uint2 rg = ranges[tile];
  p.start = rg.x;
  p.end = rg.y;
  return true;
}

__device__ __forceinline__ uint32_t warp_claim(unsigned int* counter) {
  uint32_t id = 0;
  if ((threadIdx.x & 31) == 0) id = atomicAdd(counter, 1u);
  return __shfl_sync(0xffffffffu, id, 0);
}

// A warp that finds no work left counts itself done; the last one resets the
// work and done counters to zero for the next launch on the stream.
__device__ __forceinline__ void long_finish(unsigned int* counter, unsigned int* done) {
  if ((threadIdx.x & 31) == 0) {
    __threadfence();
    const unsigned int total = gridDim.x * (blockDim.x >> 5);
    if (atomicAdd(done, 1u) == total - 1) {
      *counter = 0u;
      *done = 0u;
    }
  }
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Four CTAs per SM (64 registers): with the loads pipelined below, 32 warps
// per SM measured faster than 24 at 72 registers (batched forward 8.0 against
// 8.5 ms).
template <bool LOSS>
__global__ void __launch_bounds__(256, 4) k_fwd_long(const Desc* __restrict__ D, const uint2* __restrict__ ranges,
                                                  const uint32_t* __restrict__ pv, const float4* __restrict__ rec,
                                                  const float4* __restrict__ box,
                                                  const uint32_t* __restrict__ longt, Status* __restrict__ st,
                                                  const uint32_t* __restrict__ cbase, float* __restrict__ ckpt,
                                                  uint32_t* __restrict__ cmask, LossEpi loss) {
  pdl_wait();               // (launched after a kernel of this chain: wait for it)
  pdl_launch_dependents();  // the next kernel may be dispatched now
  const int lane = threadIdx.x & 31;
  const uint32_t n_long = st->n_long;
  if (n_long == 0) {
    // no long list: the per-tile forward before it on the stream has added
    // every pixel's loss terms, so one warp writes the loss vector at once
    // (no ticket over the grid)
    if (LOSS && blockIdx.x == 0 && threadIdx.x < 32)
      finish_loss_vector(*D, loss.P, loss.ctot, loss.acc, loss.out, st);
    return;
  }
  uint32_t evals = 0, contrib = 0, alg = 0;
  LongPix P;
  while (long_item(*D, ranges, longt, n_long, warp_claim(&st->long_counter_fwd), P)) {
    if (!P.inside) continue;
    const FrameDev& F = *P.F;
    float dx, dy, dz;
    pixel_ray(F, P.r, P.c, dx, dy, dz);
    WarpBox pb;
    pb.r0 = pb.r1 = static_cast<float>(P.r);
    pb.cmid = static_cast<float>(P.c);
    pb.chalf = 0.f;
    pb.W = static_cast<float>(F.W);
    float T = 1.f, A = 0.f, St = 0.f, Sx = 0.f, Sy = 0.f, Sz = 0.f;
    int last = 0, stop_at = -1;
    // the chunked backward's inputs, laid out as the per-tile forward's: the
    // pixel's composited entries of every window it walks (one bit each) and,
    // at the end of every chunk it walks, T and the chunk's own sums
    const int npx = D->th * D->tw;
    const int64_t cb = static_cast<int64_t>(cbase[P.tile]);
    float cA = 0.f, cSt = 0.f, cSx = 0.f, cSy = 0.f, cSz = 0.f;
    const auto checkpoint = [&](uint32_t chunk) {
      const float a = warp_sum(cA), b = warp_sum(cSt), x = warp_sum(cSx), y = warp_sum(cSy), z = warp_sum(cSz);
      if (lane == 0) {
        float* o = ckpt + ((cb + chunk) * kCkptSlots) * npx + P.vt;
        o[0] = T;
        o[npx] = a;
        o[2 * npx] = b;
        o[3 * npx] = x;
        o[4 * npx] = y;
        o[5 * npx] = z;
      }
      cA = cSt = cSx = cSy = cSz = 0.f;
    };
    uint32_t win = 0;
    // software pipeline over the windows: the list entry two windows ahead
    // and the culling box one window ahead are loaded while this window is
    // composited (each window's loads would otherwise form a chain of
    // dependent round trips: entry, then box, then record)
    uint32_t item_next = P.start + 32 + lane < P.end ? __ldg(pv + P.start + 32 + lane) : 0u;
    uint32_t item_cur = P.start + lane < P.end ? __ldg(pv + P.start + lane) : 0u;
    float4 box_cur = P.start + lane < P.end ? __ldg(box + item_cur) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (uint32_t base = P.start; base < P.end; base += 32, ++win) {
      if (win > 0 && win % 4 == 0) checkpoint(win / 4 - 1);
      uint32_t* mword = cmask + (cb * 4 + win) * npx + P.vt;
      const uint32_t j = base + lane;
      const uint32_t item = item_cur;
      const float4 bx = box_cur;
      item_cur = item_next;
      box_cur = j + 32 < P.end ? __ldg(box + item_next) : make_float4(0.f, 0.f, 0.f, 0.f);
      item_next = j + 64 < P.end ? __ldg(pv + j + 64) : 0u;
      bool valid = false;
      Eval e;
      float nx = 0.f, ny = 0.f, nz = 0.f;
      if (j < P.end) {
        if (box_hits(bx, pb)) {
          const float4* rp = rec + 4 * static_cast<int64_t>(item);
          const float4 r0 = __ldg(rp);
          eval_pair(r0, __ldg(rp + 1), __ldg(rp + 2), __ldg(reinterpret_cast<const float*>(rp + 3)), dx, dy, dz, e);
          valid = e.valid;
          nx = r0.x; ny = r0.y; nz = r0.z;
          ++evals;
        }
      }
      // a window without a valid pair leaves T and the sums as they are
      if (!__any_sync(0xffffffffu, valid)) {
        if (lane == 0) *mword = 0u;
        continue;
      }
      // P_j = prod_{i <= j} (1 - a_i) over the valid lanes
      float Pj = valid ? __fsub_rn(1.0f, e.a) : 1.0f;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_up_sync(0xffffffffu, Pj, o);
        if (lane >= o) Pj *= y;
      }
      float Pex = __shfl_up_sync(0xffffffffu, Pj, 1);
      if (lane == 0) Pex = 1.0f;
      const uint32_t sm = __ballot_sync(0xffffffffu, valid && T * Pj < 1e-4f);
      const int fs = sm ? __ffs(sm) - 1 : 32;
      const bool inc = valid && lane < fs;
      const float w = inc ? e.a * (T * Pex) : 0.f;
      const float ws = valid && e.den > 0.f ? -w : w;
      // every lane sums its own entries' terms; the pixel's totals are the
      // warp sums of these after the walk
      A += w;
      if (inc) St = fmaf(w, e.t, St);   // (e is unset on lanes without a box hit)
      Sx = fmaf(ws, nx, Sx);
      Sy = fmaf(ws, ny, Sy);
      Sz = fmaf(ws, nz, Sz);
      cA += w;
      if (inc) cSt = fmaf(w, e.t, cSt);
      cSx = fmaf(ws, nx, cSx);
      cSy = fmaf(ws, ny, cSy);
      cSz = fmaf(ws, nz, cSz);
      contrib += inc;
      const uint32_t im = __ballot_sync(0xffffffffu, inc);
      if (lane == 0) *mword = im;
      if (im) last = static_cast<int>(base - P.start) + (31 - __clz(im)) + 1;
      T *= __shfl_sync(0xffffffffu, fs < 32 ? Pex : Pj, fs < 32 ? fs : 31);
      if (sm) {
        stop_at = static_cast<int>(base - P.start) + fs + 1;
        break;
      }
    }
    // the chunk holding the walk's last window (the list end or the stop)
    if (P.end > P.start) checkpoint((win > 0 && stop_at < 0 ? win - 1 : win) / 4);
    A = warp_sum(A);
    St = warp_sum(St);
    Sx = warp_sum(Sx);
    Sy = warp_sum(Sy);
    Sz = warp_sum(Sz);
    if (lane == 0) {
      F.A[P.pix] = A;
      F.St[P.pix] = St;
      F.Sn[P.pix] = Sx;
      F.Sn[P.HW + P.pix] = Sy;
      F.Sn[2 * static_cast<int64_t>(P.HW) + P.pix] = Sz;
      F.Tf[P.pix] = T;
      F.nc[P.pix] = last;
      alg += stop_at >= 0 ? static_cast<uint32_t>(stop_at) : P.end - P.start;
    }
    // the warp holds one pixel: lane 0 alone takes its loss terms
    if (LOSS) loss_epilogue(*D, loss, static_cast<int>(P.F - D->f), lane == 0, P.pix, P.HW, A, St, Sx, Sy, Sz);
  }
  long_finish(&st->long_counter_fwd, &st->long_done_fwd);
  unsigned long long ev = evals, co = contrib, al = alg;
  for (int o = 16; o > 0; o >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, o);
    co += __shfl_xor_sync(0xffffffffu, co, o);
  }
  if (lane == 0 && ev) atomicAdd(&st->evals_fwd, ev);
  if (lane == 0 && co) atomicAdd(&st->contrib_fwd, co);
  if (lane == 0 && al) atomicAdd(&st->alg_fwd, al);
  if (LOSS) {
    // this launch follows the per-tile forward on the stream, so when its
    // last CTA is done every pixel's epilogue has added its terms: that CTA
    // writes the loss vector (the regulariser was summed before the forward)
    __shared__ bool s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      s_last = atomicAdd(&st->loss_ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x < 32) finish_loss_vector(*D, loss.P, loss.ctot, loss.acc, loss.out, st);
  }
}

__global__ void __launch_bounds__(256) k_bwd_long(const Desc* __restrict__ D, const uint2* __restrict__ ranges,
                                                  const uint32_t* __restrict__ pv, const float4* __restrict__ rec,
                                                  const float4* __restrict__ box, float* __restrict__ g13,
                                                  const uint32_t* __restrict__ longt, Status* __restrict__ st) {
  const int lane = threadIdx.x & 31;
  const uint32_t n_long = st->n_long;
  if (n_long == 0) return;
  uint32_t evals = 0, contrib = 0;
  LongPix P;
  while (long_item(*D, ranges, longt, n_long, warp_claim(&st->long_counter_bwd), P)) {
    if (!P.inside) continue;
    const FrameDev& F = *P.F;
    const int nc = F.nc[P.pix];
    // n_contrib comes from the caller: never walk past the tile's list
    const uint32_t stop = min(static_cast<uint32_t>(nc > 0 ? nc : 0), P.end - P.start);
    if (stop == 0) continue;
    float dx, dy, dz;
    pixel_ray(F, P.r, P.c, dx, dy, dz);
    const float gA = F.gA[P.pix], gSt = F.gSt[P.pix];
    const float gSx = F.gSn[P.pix], gSy = F.gSn[P.HW + P.pix], gSz = F.gSn[2 * static_cast<int64_t>(P.HW) + P.pix];
    WarpBox pb;
    pb.r0 = pb.r1 = static_cast<float>(P.r);
    pb.cmid = static_cast<float>(P.c);
    pb.chalf = 0.f;
    pb.W = static_cast<float>(F.W);
    float T = F.Tf[P.pix], S = 0.f;
    for (int c0 = static_cast<int>((stop + 31) / 32) - 1; c0 >= 0; --c0) {
      const uint32_t k = 32u * c0 + lane;
      bool valid = false;
      Eval e;
      float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f);
      uint32_t item = 0;
      if (k < stop) {
        item = __ldg(pv + P.start + k);
        if (box_hits(__ldg(box + item), pb)) {
          const float4* rp = rec + 4 * static_cast<int64_t>(item);
          r0 = __ldg(rp);
          eval_pair(r0, __ldg(rp + 1), __ldg(rp + 2), __ldg(reinterpret_cast<const float*>(rp + 3)), dx, dy, dz, e);
          valid = e.valid;
          ++evals;
        }
      }
      const float om = valid ? 1.0f - e.a : 1.0f;
      // Q_j = prod_{i >= j} (1 - a_i) over the chunk's valid lanes
      float Qj = om;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_down_sync(0xffffffffu, Qj, o);
        if (lane + o < 32) Qj *= y;
      }
      const float Tk = __fdividef(T, Qj);   // transmittance before entry j
      float c = 0.f, gc = 0.f;
      if (valid) {
        const float sg = e.den > 0.f ? -1.f : 1.f;
        gc = gA + gSt * e.t + sg * (gSx * r0.x + gSy * r0.y + gSz * r0.z);
        c = e.a * Tk * gc;
      }
      // suffix sums of w (g.c): after entry j (exclusive) and over the chunk
      float Cs = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const float y = __shfl_down_sync(0xffffffffu, Cs, o);
        if (lane + o < 32) Cs += y;
      }
      float Cex = __shfl_down_sync(0xffffffffu, Cs, 1);
      if (lane == 31) Cex = 0.f;
      if (valid) {
        ++contrib;
        float v[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) v[q] = 0.f;
        moments(e, r0, Tk, S + Cex, rcp_ftz(om), gA, gSt, gSx, gSy, gSz, v);
        float* gp = g13 + 16 * static_cast<int64_t>(item);
#pragma unroll
        for (int q = 0; q < kGrad; ++q)
          if (v[q] != 0.f) atomicAdd(gp + q, v[q]);
      }
      T = __fdividef(T, __shfl_sync(0xffffffffu, Qj, 0));
      S += __shfl_sync(0xffffffffu, Cs, 0);
    }
  }
  long_finish(&st->long_counter_bwd, &st->long_done_bwd);
  unsigned long long ev = evals, co = contrib;
  for (int o = 16; o > 0; o >>= 1) {
    ev += __shfl_xor_sync(0xffffffffu, ev, o);
    co += __shfl_xor_sync(0xffffffffu, co, o);
  }
  if (lane == 0 && ev) atomicAdd(&st->evals_bwd, ev);
  if (lane == 0 && co) atomicAdd(&st->contrib_bwd, co);
}

// Before the chunked backward (one launch):
// (1) its work queues, from the forward's largest n_contrib of every (tile,
//     warp block) (a long list: its length): one thread per tile, warp-
//     aggregated reservations (one atomic per warp for class 0, one per
//     class present and block for the others).  A tile's full chunks are
//     queued chunk by chunk, its blocks side by side: they read the same
//     list entries, so warps that claim them together share those loads in
//     L2.  The queue sizes are zero on entry (cleared with the claim
//     counter).
// (2) over the long lists: the suffix S of every chunk (the sum over the
//     pixel's later chunks c' of gA dA_c' + gSt dSt_c' + gS . dSn_c'),
//     written to a buffer of its own (the checkpoints stay as the forward
//     wrote them, for any further backward), so that k_bwd_c reads it
//     instead of summing, per work item, up to thousands of later chunks.
//     One CTA per (long tile, warp block): its eight warps split the
//     block's chunks into segments (lane = pixel), sum their segment while
//     parking every chunk's term in the suffix buffer, add up the later
//     segments' sums in shared memory, then walk their segment down.  A
//     list of 2,000 chunks is eight chains of 250, not one of 2,000.
constexpr int kMaxBlocks = kMaxTileThreads / 32;

__global__ void __launch_bounds__(256) k_bwd_prep(const Desc* __restrict__ D, const uint2* __restrict__ ranges,
                                                  const uint32_t* __restrict__ longt, Status* __restrict__ st,
                                                  const uint32_t* __restrict__ cbase,
                                                  const uint32_t* __restrict__ bwm, uint2* __restrict__ bq,
                                                  uint32_t cap0, uint32_t capk,
                                                  const float* __restrict__ ckpt, float* __restrict__ csuf) {
  pdl_wait();               // (launched after a kernel of this chain: wait for it)
  pdl_launch_dependents();  // the next kernel may be dispatched now
  const int lane = threadIdx.x & 31;
  const uint32_t blocks = static_cast<uint32_t>(D->th * D->tw) >> 5;
  const uint32_t n_tiles = D->n_tiles;
  // (1) a warp-uniform loop: every lane reaches the warp collectives
  for (uint32_t t0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); t0 < n_tiles; t0 += gridDim.x * blockDim.x) {
    const uint32_t tile = t0 + static_cast<uint32_t>(lane);
    const bool ok = tile < n_tiles;
    // a long list's blocks take every chunk (its pixels' walks end in
    // k_fwd_long, which keeps no per-block maximum)
    const uint32_t len = ok ? ranges[tile].y - ranges[tile].x : 0u;
    uint32_t wm[kMaxBlocks];
    uint32_t nfull = 0, nf_max = 0;
#pragma unroll
    for (int b = 0; b < kMaxBlocks; ++b) {
      wm[b] = ok && static_cast<uint32_t>(b) < blocks ? (len > kLongList ? len : bwm[tile * blocks + b]) : 0u;
      nfull += wm[b] / kChunk;
      nf_max = max(nf_max, wm[b] / kChunk);
    }
    const uint32_t c0 = ok ? cbase[tile] : 0u;
    // class 0: the tile's full chunks, placed by an inclusive warp scan
    uint32_t incl = nfull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += x;
    }
    uint32_t pos = 0;
    if (lane == 31 && incl) pos = atomicAdd(&st->bq_count[0], incl);
    pos = __shfl_sync(0xffffffffu, pos, 31) + incl - nfull;
    for (uint32_t c = 0; c < nf_max; ++c) {
#pragma unroll
      for (int b = 0; b < kMaxBlocks; ++b) {
        if (c < wm[b] / kChunk) {
          if (pos < cap0) bq[pos] = make_uint2((c0 + c) * blocks + static_cast<uint32_t>(b), tile);
          ++pos;
        }
      }
    }
    // every block's chunk holding its last entry: the class of its walked
    // length (longest first), one reservation per class present
#pragma unroll
    for (int b = 0; b < kMaxBlocks; ++b) {
      if (static_cast<uint32_t>(b) >= blocks) break;
      const uint32_t rem = wm[b] % kChunk;
      const uint32_t cls = rem ? 1u + ((kChunk - rem) * (kBwdClasses - 1)) / kChunk : 0u;
      const uint32_t peers = __match_any_sync(0xffffffffu, cls);
      const int leader = __ffs(peers) - 1;
      uint32_t bk = 0;
      if (cls && lane == leader) bk = atomicAdd(&st->bq_count[cls], static_cast<uint32_t>(__popc(peers)));
      bk = __shfl_sync(0xffffffffu, bk, leader) + static_cast<uint32_t>(__popc(peers & ((1u << lane) - 1u)));
      if (cls && bk < capk)
        bq[cap0 + (cls - 1) * capk + bk] = make_uint2((c0 + wm[b] / kChunk) * blocks + static_cast<uint32_t>(b), tile);
    }
  }
  // (2) requires 256 threads (eight segments); CTA-uniform loop
  __shared__ float s_seg[8][32];
  const uint32_t n_long = st->n_long;
  const int npx = static_cast<int>(blocks) * 32;
  const int wseg = threadIdx.x >> 5;
  for (uint32_t it = blockIdx.x; it < n_long * blocks; it += gridDim.x) {
    const uint32_t lt = it / blocks, blk = it - lt * blocks;
    const uint32_t tile = longt[lt];
    const FrameDev& F = D->f[frame_of_tile(*D, tile)];
    const int ltile = static_cast<int>(tile - F.tile_base);
    const int ti = ltile / F.ntc, tj = ltile - ti * F.ntc;
    const int vt = static_cast<int>(blk) * 32 + lane;
    int lr, lc;
    pixel_of_thread(F, vt, lr, lc);
    const int r = ti * F.th + lr, col = tj * F.tw + lc;
    const int64_t pix = static_cast<int64_t>(r) * F.W + col;
    const int HW = F.H * F.W;
    const int nc = r < F.H && col < F.W ? F.nc[pix] : 0;
    const int cl = nc > 0 ? (nc - 1) / static_cast<int>(kChunk) + 1 : 0;   // the pixel's chunks
    const int seg = (__reduce_max_sync(0xffffffffu, static_cast<uint32_t>(cl)) + 7) / 8;
    const int lo = wseg * seg, hi = min(lo + seg, cl);
    float gA = 0.f, gSt = 0.f, gSx = 0.f, gSy = 0.f, gSz = 0.f;
    if (hi > lo) {
      gA = F.gA[pix];
      gSt = F.gSt[pix];
      gSx = F.gSn[pix];
      gSy = F.gSn[HW + pix];
      gSz = F.gSn[2 * static_cast<int64_t>(HW) + pix];
    }
    const int64_t cb = static_cast<int64_t>(cbase[tile]);
    // pass 1: every chunk's term (parked in csuf) and the segment's sum
    float tot = 0.f;
    for (int c = hi - 1; c >= lo; c -= 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        v[u] = 0.f;
        if (c - u >= lo) {
          const float* q = ckpt + (cb + c - u) * kCkptSlots * npx + vt;
          v[u] = gA * q[npx] + gSt * q[2 * npx] + gSx * q[3 * npx] + gSy * q[4 * npx] + gSz * q[5 * npx];
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (c - u >= lo) {
          csuf[(cb + c - u) * npx + vt] = v[u];
          tot += v[u];
        }
      }
    }
    s_seg[wseg][lane] = tot;
    __syncthreads();
    float S = 0.f;
    for (int w2 = 7; w2 > wseg; --w2) S += s_seg[w2][lane];
    // pass 2: the suffix before every chunk of the segment, walking down
    for (int c = hi - 1; c >= lo; c -= 8) {
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = c - u >= lo ? csuf[(cb + c - u) * npx + vt] : 0.f;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (c - u >= lo) {
          csuf[(cb + c - u) * npx + vt] = S;
          S += v[u];
        }
      }
    }
    __syncthreads();   // s_seg is rewritten by the next item
  }
}

// The work counters start at zero (reset at binning and by the last warp of
// every launch), so no memset precedes the launch.
static cudaError_t launch_long(bool fwd, const WsPtrs& w, const uint32_t* pv, cudaStream_t s,
                               const LossEpi* loss = nullptr) {
  int dev = 0, sms = 152, per_sm = 2;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  // as many CTAs as fit (the walks are bound by load latency); warps claim
  // (tile, pixel) items until none are left
  if (fwd && loss) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fwd_long<true>, 256, 0);
  else if (fwd) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fwd_long<false>, 256, 0);
  else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bwd_long, 256, 0);
  const int grid = sms * (per_sm > 0 ? per_sm : 1);
  // (a plain launch: dispatched during the shared-memory forward, its CTAs
  // made the 16-map batch's long-list forward 7.9 -> 14.7 ms)
  if (fwd && loss)
    k_fwd_long<true><<<grid, 256, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, w.longt, w.st, w.cbase, w.ckpt, w.cmask,
                                          *loss);
  else if (fwd)
    k_fwd_long<false><<<grid, 256, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, w.longt, w.st, w.cbase, w.ckpt,
                                           w.cmask, LossEpi{});
  else k_bwd_long<<<grid, 256, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, w.g13, w.longt, w.st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <int B>
static cudaError_t fwd_b(const WsPtrs& w, const uint32_t* pv, const Desc& h, int persistent, int grid, cudaStream_t s) {
  k_fwd<B><<<grid, h.th * h.tw, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, persistent ? w.work : nullptr, w.st,
                                        persistent);
  return cudaGetLastError();
}

template <int B>
static cudaError_t bwd_b(const WsPtrs& w, const uint32_t* pv, const Desc& h, int persistent, int grid, cudaStream_t s) {
  k_bwd<B><<<grid, h.th * h.tw, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, w.g13, persistent ? w.work : nullptr,
                                        w.st, persistent);
  return cudaGetLastError();
}

static int persistent_grid(int threads) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = 2048 / (threads > 0 ? threads : 256);
  return sms * (per_sm < 1 ? 1 : per_sm);
}

static cudaError_t launch_raster_fwd_tiles(const WsPtrs& w, const Desc& h, const uint32_t* pv, int batch,
                                           int group, int persistent, cudaStream_t s) {
  if (persistent) {
    cudaError_t e = cudaMemsetAsync(&w.st->work_counter, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
  }
  const int grid = persistent ? persistent_grid(h.th * h.tw) : static_cast<int>(h.n_tiles);
  const uint32_t* ord = persistent ? w.work : nullptr;
  switch (batch) {
    case 0:
      if (group == 16)
        k_fwd_s<false><<<grid, h.th * h.tw, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, ord, w.st, persistent,
                                                    w.cbase, w.ckpt, w.cmask, w.bwm, LossEpi{});
      else if (group == 1) k_fwd_w<1><<<grid, h.th * h.tw, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, ord, w.st, persistent);
      else if (group == 2) k_fwd_w<2><<<grid, h.th * h.tw, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, ord, w.st, persistent);
      else k_fwd_w<4><<<grid, h.th * h.tw, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, ord, w.st, persistent);
      return cudaGetLastError();
    case 64: return fwd_b<64>(w, pv, h, persistent, grid, s);
    case 128: return fwd_b<128>(w, pv, h, persistent, grid, s);
    case 512: return fwd_b<512>(w, pv, h, persistent, grid, s);
    default: return fwd_b<256>(w, pv, h, persistent, grid, s);
  }
}

static cudaError_t launch_raster_bwd_tiles(const WsPtrs& w, const Desc& h, const uint32_t* pv, int batch,
                                           int group, int persistent, cudaStream_t s) {
  if (persistent) {
    cudaError_t e = cudaMemsetAsync(&w.st->work_counter2, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
  }
  const int grid = persistent ? persistent_grid(h.th * h.tw) : static_cast<int>(h.n_tiles);
  const uint32_t* ord = persistent ? w.work : nullptr;
  switch (batch) {
    case 0:
      if (group == 16) k_bwd_s<<<grid, h.th * h.tw, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, w.g13, ord, w.st, persistent);
      else if (group == 1) k_bwd_w<1><<<grid, h.th * h.tw, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, w.g13, ord, w.st, persistent);
      else if (group == 2) k_bwd_w<2><<<grid, h.th * h.tw, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, w.g13, ord, w.st, persistent);
      else k_bwd_w<4><<<grid, h.th * h.tw, 0, s>>>(w.desc, w.ranges, pv, w.rec, w.box, w.g13, ord, w.st, persistent);
      return cudaGetLastError();
    case 64: return bwd_b<64>(w, pv, h, persistent, grid, s);
    case 128: return bwd_b<128>(w, pv, h, persistent, grid, s);
    default: return bwd_b<256>(w, pv, h, persistent, grid, s);
  }
}

// The per-tile kernel, then the long-list kernel for the tiles it skipped.
cudaError_t launch_raster_fwd(const Layout&, const WsPtrs& w, const Desc& h, const uint32_t* pv, int batch,
                              int group, int persistent, cudaStream_t s) {
  cudaError_t e = launch_raster_fwd_tiles(w, h, pv, batch, group, persistent, s);
  if (e != cudaSuccess) return e;
  return launch_long(true, w, pv, s);
}

// Chunked backward: as many resident CTAs as fit, warps claim (chunk, pixel
// block) items from the queues k_bwd_prep built until none are left.
static cudaError_t launch_raster_bwd_chunks(const WsPtrs& w, const uint32_t* pv, cudaStream_t s) {
  int dev = 0, sms = 152, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_bwd_c, kBwdChunkCta, 0);
  return launch_dep(k_bwd_c, dim3(sms * (per_sm > 0 ? per_sm : 1)), dim3(kBwdChunkCta), 0, s, w.desc, w.ranges, pv,
                    w.rec, w.box, w.g13, w.cbase, w.ckpt, w.cmask, w.csuf, w.bq, w.bq_cap0, w.bq_capk, w.st);
}

// The shared-memory forward with the image-loss epilogue (and the long-list
// forward with the same epilogue).  Follows launch_loss_counts on the same
// stream, which zeroed the tile counter.
cudaError_t launch_raster_fwd_loss(const WsPtrs& w, const Desc& h, const uint32_t* pv, int persistent,
                                   const lgs_loss_params& p, float* loss_out, cudaStream_t s) {
  LossEpi loss{p, loss_counts_ptr(w), reinterpret_cast<unsigned long long*>(w.loss_part), loss_out};
  const int grid = persistent ? persistent_grid(h.th * h.tw) : static_cast<int>(h.n_tiles);
  // (follows k_loss_count on the stream: dispatched while it runs)
  cudaError_t e = launch_dep(k_fwd_s<true>, dim3(grid), dim3(h.th * h.tw), 0, s, w.desc, w.ranges, pv, w.rec, w.box,
                             persistent ? w.work : nullptr, w.st, persistent, w.cbase, w.ckpt, w.cmask, w.bwm, loss);
  if (e != cudaSuccess) return e;
  return launch_long(true, w, pv, s, &loss);
}

cudaError_t launch_raster_bwd(const Layout&, const WsPtrs& w, const Desc& h, const uint32_t* pv, int batch,
                              int group, int persistent, bool chunked, cudaStream_t s) {
  if (chunked) {
    // the claim counter and the queue sizes are zero here (cleared at
    // binning and after every backward by k_preprocess_bwd); the queues and
    // the long lists' suffixes, then the walk
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    k_bwd_prep<<<4 * sms, 256, 0, s>>>(w.desc, w.ranges, w.longt, w.st, w.cbase, w.bwm, w.bq, w.bq_cap0, w.bq_capk,
                                       w.ckpt, w.csuf);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_raster_bwd_chunks(w, pv, s);
  }
  cudaError_t e = launch_raster_bwd_tiles(w, h, pv, batch, group, persistent, s);
  if (e != cudaSuccess) return e;
  return launch_long(false, w, pv, s);
}

}  // namespace lgs
