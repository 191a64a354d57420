// lgs_track.cu -- the tracking-side view of the map (paper Sec. 3.2, "G-ICP
// Tracking with Trackable Gaussians"): the trackable subset of Eq.
// trackable_select, each member's surfel-like target covariance built in
// O(1) from its own parameters (no map-side k-NN), and its geometry weight
// (Eqs. anisotropy, anisotropy_norm, weight_func).
//
// Three launches over the surfels: select (flag, anisotropy; per CTA the
// count and the minimum / maximum anisotropy as float bits, exact in any
// order), scan (one CTA: first output slot of every CTA, the count, the
// global minimum / maximum), write (stable compaction in ascending surfel
// index: mean, covariance, weight).  No global atomics.  Scratch is the caller's (lgs_trackable_scratch_bytes).
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {
namespace {

constexpr int kTrkCta = 256;
constexpr int kTrkScanCta = 1024;

struct TrkScratch {
  uint32_t* count;      // [ctas] selected surfels per CTA, then their first output slot
  uint32_t* kmin;       // [ctas] smallest anisotropy of the CTA's selection (float bits; all positive)
  uint32_t* kmax;       // [ctas] largest
  uint32_t* kbits;      // [2] min and max over the whole selection
};

__device__ __forceinline__ bool trk_selected(const lgs_surfels& M, const uint8_t* mask, const int32_t* last_kf,
                                             int64_t i, int32_t k_min, float logit_min) {
  return mask[i] != 0 && last_kf[i] >= k_min && M.opacity_logit[i] >= logit_min;
}

__device__ __forceinline__ float trk_kappa(const lgs_surfels& M, int64_t i, float eps) {
  const float s0 = expf(M.log_scale[2 * i]), s1 = expf(M.log_scale[2 * i + 1]);
  return fmaxf(s0, s1) / (fminf(s0, s1) + eps);
}

__global__ void __launch_bounds__(kTrkCta) k_trk_select(lgs_surfels M, const uint8_t* __restrict__ mask,
                                                        const int32_t* __restrict__ last_kf, int32_t k_min,
                                                        float logit_min, float eps, TrkScratch sc) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool sel = i < M.n && trk_selected(M, mask, last_kf, i, k_min, logit_min);
  uint32_t kb_min = 0xffffffffu, kb_max = 0u;
  if (sel) {
    const uint32_t b = __float_as_uint(trk_kappa(M, i, eps));
    kb_min = b;
    kb_max = b;
  }
  const uint32_t bal = __ballot_sync(0xffffffffu, sel);
  kb_min = __reduce_min_sync(0xffffffffu, kb_min);
  kb_max = __reduce_max_sync(0xffffffffu, kb_max);
  // per-CTA totals in the CTA's own slots (no global atomics: the scan
  // reduces them)
  __shared__ uint32_t s_n[kTrkCta / 32], s_lo[kTrkCta / 32], s_hi[kTrkCta / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_n[wid] = __popc(bal);
    s_lo[wid] = kb_min;
    s_hi[wid] = kb_max;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const bool in = lane < kTrkCta / 32;
    const uint32_t n = __reduce_add_sync(0xffffffffu, in ? s_n[lane] : 0u);
    const uint32_t lo = __reduce_min_sync(0xffffffffu, in ? s_lo[lane] : 0xffffffffu);
    const uint32_t hi = __reduce_max_sync(0xffffffffu, in ? s_hi[lane] : 0u);
    if (lane == 0) {
      sc.count[blockIdx.x] = n;
      sc.kmin[blockIdx.x] = lo;
      sc.kmax[blockIdx.x] = hi;
    }
  }
}

// Exclusive scan of the per-CTA counts (in place), the total, and the
// minimum and maximum anisotropy over all CTAs.
__global__ void __launch_bounds__(kTrkScanCta) k_trk_scan(TrkScratch sc, uint32_t ctas,
                                                          int64_t* __restrict__ total) {
  __shared__ uint32_t s_w[32], s_lo[32], s_hi[32];
  __shared__ uint32_t s_carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_carry = 0;
  uint32_t lo = 0xffffffffu, hi = 0u;
  for (uint32_t b = tid; b < ctas; b += kTrkScanCta) {
    lo = min(lo, sc.kmin[b]);
    hi = max(hi, sc.kmax[b]);
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if (lane == 0) {
    s_lo[wid] = lo;
    s_hi[wid] = hi;
  }
  __syncthreads();
  if (tid < 32) {
    lo = __reduce_min_sync(0xffffffffu, s_lo[tid]);
    hi = __reduce_max_sync(0xffffffffu, s_hi[tid]);
    if (tid == 0) {
      sc.kbits[0] = lo;
      sc.kbits[1] = hi;
    }
  }
  for (uint32_t b0 = 0; b0 < ctas; b0 += kTrkScanCta) {
    const uint32_t b = b0 + tid;
    const uint32_t x = b < ctas ? sc.count[b] : 0u;
    uint32_t v = x;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += y;
    }
    if (lane == 31) s_w[wid] = v;
    __syncthreads();
    uint32_t pre = 0, tot = 0;
    for (int w = 0; w < 32; ++w) {
      if (w < wid) pre += s_w[w];
      tot += s_w[w];
    }
    if (b < ctas) sc.count[b] = s_carry + pre + v - x;
    __syncthreads();
    if (tid == 0) s_carry += tot;
    __syncthreads();
  }
  if (tid == 0) *total = static_cast<int64_t>(s_carry);
}

__global__ void __launch_bounds__(kTrkCta) k_trk_write(lgs_surfels M, const uint8_t* __restrict__ mask,
                                                       const int32_t* __restrict__ last_kf, int32_t k_min,
                                                       float logit_min, float thick, float eps, float w_max,
                                                       TrkScratch sc, int32_t* __restrict__ out_index,
                                                       float* __restrict__ out_mean, float* __restrict__ out_cov,
                                                       float* __restrict__ out_w) {
  const int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const bool sel = i < M.n && trk_selected(M, mask, last_kf, i, k_min, logit_min);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint32_t bal = __ballot_sync(0xffffffffu, sel);
  __shared__ uint32_t s_w[kTrkCta / 32];
  if (lane == 0) s_w[wid] = __popc(bal);
  __syncthreads();
  if (!sel) return;
  uint32_t pos = sc.count[blockIdx.x] + __popc(bal & ((1u << lane) - 1u));
  for (int w = 0; w < wid; ++w) pos += s_w[w];
  // rotation of the unit quaternion (w, x, y, z): columns t_u, t_v, n
  const float4 q4 = make_float4(M.quat[4 * i], M.quat[4 * i + 1], M.quat[4 * i + 2], M.quat[4 * i + 3]);
  const float inv = rsqrtf(q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w);
  const float qw = q4.x * inv, qx = q4.y * inv, qy = q4.z * inv, qz = q4.w * inv;
  const float R[3][3] = {{1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - qw * qz), 2.f * (qx * qz + qw * qy)},
                         {2.f * (qx * qy + qw * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - qw * qx)},
                         {2.f * (qx * qz - qw * qy), 2.f * (qy * qz + qw * qx), 1.f - 2.f * (qx * qx + qy * qy)}};
  const float s0 = expf(M.log_scale[2 * i]), s1 = expf(M.log_scale[2 * i + 1]);
  const float lam[3] = {s0 * s0, s1 * s1, thick * thick};
  float C[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) C[a][b] = R[a][0] * lam[0] * R[b][0] + R[a][1] * lam[1] * R[b][1] + R[a][2] * lam[2] * R[b][2];
  const float kmin = __uint_as_float(__ldcg(sc.kbits)), kmax = __uint_as_float(__ldcg(sc.kbits + 1));
  const float kap = trk_kappa(M, i, eps);
  const float kb = kmax > kmin ? (kap - kmin) / (kmax - kmin) : 0.f;
  out_index[pos] = static_cast<int32_t>(i);
  out_mean[3 * pos] = M.mean[3 * i];
  out_mean[3 * pos + 1] = M.mean[3 * i + 1];
  out_mean[3 * pos + 2] = M.mean[3 * i + 2];
  float* c = out_cov + 6 * static_cast<int64_t>(pos);
  c[0] = C[0][0];
  c[1] = C[0][1];
  c[2] = C[0][2];
  c[3] = C[1][1];
  c[4] = C[1][2];
  c[5] = C[2][2];
  out_w[pos] = fminf(1.0f / (kb + eps), w_max);
}

}  // namespace

size_t trackable_scratch_bytes(int64_t n) {
  const int64_t ctas = (n + kTrkCta - 1) / kTrkCta;
  return sizeof(uint32_t) * (3 * static_cast<size_t>(ctas > 0 ? ctas : 1) + 2);
}

cudaError_t launch_trackable(const lgs_surfels& M, const uint8_t* mask, const int32_t* last_kf, int32_t k_min,
                             float logit_min, float thick, float eps, float w_max, void* scratch, int32_t* index,
                             float* mean, float* cov, float* weight, int64_t* count, cudaStream_t s) {
  const int64_t n = M.n;
  const uint32_t ctas = static_cast<uint32_t>(n > 0 ? (n + kTrkCta - 1) / kTrkCta : 0);
  uint32_t* base = static_cast<uint32_t*>(scratch);
  const uint32_t c1 = ctas > 0 ? ctas : 1;
  TrkScratch sc{base, base + c1, base + 2 * c1, base + 3 * c1};
  if (ctas == 0) return cudaMemsetAsync(count, 0, sizeof(int64_t), s);
  k_trk_select<<<ctas, kTrkCta, 0, s>>>(M, mask, last_kf, k_min, logit_min, eps, sc);
  k_trk_scan<<<1, kTrkScanCta, 0, s>>>(sc, ctas, count);
  k_trk_write<<<ctas, kTrkCta, 0, s>>>(M, mask, last_kf, k_min, logit_min, thick, eps, w_max, sc, index, mean, cov,
                                       weight);
  return cudaGetLastError();
}

}  // namespace lgs
