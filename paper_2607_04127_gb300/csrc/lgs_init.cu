// lgs_init.cu -- keyframe initialisation of new surfels from a scan (paper
// Sec. 3.2 "Covariance construction and reuse": the k-NN covariance of each
// point and its eigendecomposition; Sec. 3.3: the range-adaptive scale
// initialisation, the physics-based confidence u of Eq. physconf and the
// opacity of Eq. alpha_init).
//
// Launches: the points go into spatial order first (a counting sort by a
// 21-bit Morton code of a uniform grid over the scan's extent: 7 bits per
// axis), so that a tile of 256 consecutive points is compact; per-tile
// bounding boxes; the k nearest neighbours (one CTA per query tile, an exact
// top-K kept sorted in registers, candidate tiles staged in shared memory;
// the CTA's own and adjacent tiles first, then only tiles whose box can still
// hold a point closer than the CTA's current K-th distance, nearest first;
// each warp skips the tiles provably beyond its own K-th distances); the
// frame of each point (covariance of the neighbourhood, cyclic Jacobi
// eigendecomposition, scales, confidence, opacity, orientation).  Keys carry
// the original index, so the order of the sort never shows in a result.
//
// The neighbour sets are integer outcomes: the squared distance that decides
// them is binary32 ((dx dx + dy dy) + dz dz), each operation correctly
// rounded, ties to the lower index, so the sets are a fixed function of the
// input (and bit-exact against the oracle).  Tile pruning is conservative
// (a margin of 1e-5 on the box distance, far above the few ulps that separate
// the box bound from any binary32 distance), so it never changes a set.
#include <cuda_runtime.h>

#include <cmath>

#include "lgs_internal.cuh"

namespace lgs {
namespace {

constexpr int kIniTile = 256;        // points per tile = queries per CTA
constexpr int kIniWindow = 3;        // tiles visited before pruning: own, +-1
constexpr int kIniMaxTiles = 4096;   // n <= 2^20
constexpr int kIniCellBits = 7;      // Morton grid: 2^7 cells per axis
constexpr uint32_t kIniCells = 1u << (3 * kIniCellBits);
constexpr int kIniSorted = 1024;     // candidate lists up to this long are visited nearest first

struct IniBox {
  float lo[3], hi[3];
};

struct IniParams {
  float R[9], t[3];                  // pose: sensor -> world
  float kappa, s_min, s_max, r0, c0, eps, alpha_min, alpha_max;
  int k;
};

__global__ void __launch_bounds__(kIniTile) k_ini_boxes(const float* __restrict__ pts, uint32_t n,
                                                        IniBox* __restrict__ boxes) {
  __shared__ float s_lo[3][kIniTile / 32], s_hi[3][kIniTile / 32];
  const uint32_t i = blockIdx.x * kIniTile + threadIdx.x;
  const bool ok = i < n;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int a = 0; a < 3; ++a) {
    const float v = ok ? pts[3 * i + a] : 0.f;
    float lo = ok ? v : INFINITY, hi = ok ? v : -INFINITY;
    for (int o = 16; o; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      s_lo[a][wid] = lo;
      s_hi[a][wid] = hi;
    }
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    float lo = INFINITY, hi = -INFINITY;
    for (int w = 0; w < kIniTile / 32; ++w) {
      lo = fminf(lo, s_lo[threadIdx.x][w]);
      hi = fmaxf(hi, s_hi[threadIdx.x][w]);
    }
    boxes[blockIdx.x].lo[threadIdx.x] = lo;
    boxes[blockIdx.x].hi[threadIdx.x] = hi;
  }
}

// The scan's extent from the tile boxes (one CTA) and the grid's cell size.
__global__ void __launch_bounds__(256) k_ini_extent(const IniBox* __restrict__ boxes, uint32_t n_tiles,
                                                    float* __restrict__ ext) {
  __shared__ float s_v[6][8];
  float v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
  for (uint32_t t = threadIdx.x; t < n_tiles; t += blockDim.x)
    for (int a = 0; a < 3; ++a) {
      v[a] = fminf(v[a], boxes[t].lo[a]);
      v[3 + a] = fmaxf(v[3 + a], boxes[t].hi[a]);
    }
  for (int a = 0; a < 6; ++a)
    for (int o = 16; o; o >>= 1) {
      const float w = __shfl_xor_sync(0xffffffffu, v[a], o);
      v[a] = a < 3 ? fminf(v[a], w) : fmaxf(v[a], w);
    }
  if ((threadIdx.x & 31) == 0)
    for (int a = 0; a < 6; ++a) s_v[a][threadIdx.x >> 5] = v[a];
  __syncthreads();
  if (threadIdx.x < 6) {
    float r = s_v[threadIdx.x][0];
    for (int w = 1; w < 8; ++w) r = threadIdx.x < 3 ? fminf(r, s_v[threadIdx.x][w]) : fmaxf(r, s_v[threadIdx.x][w]);
    ext[threadIdx.x] = r;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const float span = fmaxf(fmaxf(ext[3] - ext[0], ext[4] - ext[1]), ext[5] - ext[2]);
    ext[6] = fmaxf(span, 1e-20f) * (1.0001f / static_cast<float>(1 << kIniCellBits));   // cell edge
  }
}

__device__ __forceinline__ uint32_t spread3(uint32_t x) {   // bits b -> 3b
  uint32_t r = 0;
#pragma unroll
  for (int b = 0; b < kIniCellBits; ++b) r |= ((x >> b) & 1u) << (3 * b);
  return r;
}

__global__ void __launch_bounds__(256) k_ini_zero(uint32_t* __restrict__ a, uint32_t len) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) a[i] = 0u;
}

__global__ void __launch_bounds__(256) k_ini_cells(const float* __restrict__ pts, uint32_t n,
                                                   const float* __restrict__ ext, uint32_t* __restrict__ cell,
                                                   uint32_t* __restrict__ cnt) {
  const float h = ext[6];
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t c[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const float q = floorf((pts[3 * i + a] - ext[a]) / h);
    c[a] = static_cast<uint32_t>(fminf(fmaxf(q, 0.f), static_cast<float>((1 << kIniCellBits) - 1)));
  }
  const uint32_t code = spread3(c[0]) | (spread3(c[1]) << 1) | (spread3(c[2]) << 2);
  cell[i] = code;
  atomicAdd(&cnt[code], 1u);
}

// points into cell order (order within a cell arbitrary), with their index
__global__ void __launch_bounds__(256) k_ini_scatter(const float* __restrict__ pts, uint32_t n,
                                                     const uint32_t* __restrict__ cell, const uint32_t* __restrict__ off,
                                                     uint32_t* __restrict__ cnt, float* __restrict__ sp,
                                                     uint32_t* __restrict__ orig) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint32_t c = cell[i];
  const uint32_t pos = off[c] + atomicSub(&cnt[c], 1u) - 1u;
  sp[3 * pos] = pts[3 * i];
  sp[3 * pos + 1] = pts[3 * i + 1];
  sp[3 * pos + 2] = pts[3 * i + 2];
  orig[pos] = i;
}

// binary32 squared distance in the specified order (no contraction)
__device__ __forceinline__ float dist2(float ax, float ay, float az, float bx, float by, float bz) {
  const float dx = fsub(bx, ax), dy = fsub(by, ay), dz = fsub(bz, az);
  return fadd(fadd(fmul(dx, dx), fmul(dy, dy)), fmul(dz, dz));
}

// a lower bound of the squared distance between two boxes (exact arithmetic
// up to a few roundings; callers apply the margin)
__device__ __forceinline__ float box_gap2(const IniBox& a, const IniBox& b) {
  float s = 0.f;
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float g = fmaxf(0.f, fmaxf(b.lo[d] - a.hi[d], a.lo[d] - b.hi[d]));
    s += g * g;
  }
  return s;
}

// Sorted insertion of key into best[0..K) (ascending), dropping the largest.
template <int K>
__device__ __forceinline__ void topk_insert(unsigned long long (&best)[K], unsigned long long key) {
#pragma unroll
  for (int t = K - 1; t > 0; --t) {
    const unsigned long long prev = best[t - 1];
    best[t] = prev > key ? prev : (best[t] > key ? key : best[t]);
  }
  best[0] = best[0] > key ? key : best[0];
}

template <int K>
__global__ void __launch_bounds__(kIniTile) k_ini_knn(const float* __restrict__ pts,
                                                      const uint32_t* __restrict__ orig, uint32_t n,
                                                      const IniBox* __restrict__ boxes, uint32_t n_tiles, int k,
                                                      int32_t* __restrict__ knn, int64_t* __restrict__ pairs) {
  __shared__ float sx[kIniTile], sy[kIniTile], sz[kIniTile];
  __shared__ uint32_t s_id[kIniTile];
  __shared__ uint32_t s_list[kIniMaxTiles];
  __shared__ float s_bd[kIniSorted];          // box distances of the first kIniSorted listed tiles
  __shared__ uint32_t s_st[kIniSorted];       // the listed tiles by ascending (box distance, tile)
  __shared__ float s_sbd[kIniSorted];
  __shared__ uint32_t s_nlist, s_worst;
  __shared__ uint32_t s_wmax[kIniTile / 32];
  const uint32_t qt = blockIdx.x;
  const uint32_t i = qt * kIniTile + threadIdx.x;
  const bool valid = i < n;
  const float qx = valid ? pts[3 * i] : 0.f, qy = valid ? pts[3 * i + 1] : 0.f, qz = valid ? pts[3 * i + 2] : 0.f;
  unsigned long long best[K];
#pragma unroll
  for (int t = 0; t < K; ++t) best[t] = ~0ull;

  unsigned long long evaluated = 0;   // (query, candidate) distances of this warp's lane 0
  // the warp's own query box: a tile whose box is provably beyond every one
  // of the warp's K-th distances is skipped by the warp alone
  IniBox wbox;
  {
    const float v[3] = {qx, qy, qz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      float lo = valid ? v[a] : INFINITY, hi = valid ? v[a] : -INFINITY;
      for (int o = 16; o; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
      }
      wbox.lo[a] = lo;
      wbox.hi[a] = hi;
    }
  }
  const uint32_t w_valid = __popc(__ballot_sync(0xffffffffu, valid));
  auto visit = [&](uint32_t tile) {
    const uint32_t base = tile * kIniTile;
    const uint32_t cnt = n - base < static_cast<uint32_t>(kIniTile) ? n - base : kIniTile;
    __syncthreads();   // the previous tile is no longer read
    if (threadIdx.x < cnt) {
      sx[threadIdx.x] = pts[3 * (base + threadIdx.x)];
      sy[threadIdx.x] = pts[3 * (base + threadIdx.x) + 1];
      sz[threadIdx.x] = pts[3 * (base + threadIdx.x) + 2];
      s_id[threadIdx.x] = orig[base + threadIdx.x];
    }
    __syncthreads();
    if (w_valid == 0) return;   // uniform across the warp
    const uint32_t wworst = __reduce_max_sync(0xffffffffu, valid ? static_cast<uint32_t>(best[K - 1] >> 32) : 0u);
    if (wworst < 0x7f800000u && box_gap2(wbox, boxes[tile]) * 0.99999f > __uint_as_float(wworst)) return;
    evaluated += static_cast<unsigned long long>(cnt) * w_valid;
    if (!valid) return;
    uint32_t worst = static_cast<uint32_t>(best[K - 1] >> 32);
    for (uint32_t j = 0; j < cnt; ++j) {
      const uint32_t d = __float_as_uint(dist2(qx, qy, qz, sx[j], sy[j], sz[j]));
      if (d > worst) continue;
      const unsigned long long key = (static_cast<unsigned long long>(d) << 32) | s_id[j];
      if (key < best[K - 1]) {
        topk_insert<K>(best, key);
        worst = static_cast<uint32_t>(best[K - 1] >> 32);
      }
    }
  };

  // the own tile and its neighbours in index order (a scan's consecutive
  // points are neighbours in space)
  for (int w = 0; w < kIniWindow; ++w) {
    const int off = (w & 1) ? (w + 1) / 2 : -(w / 2);
    const long long t = static_cast<long long>(qt) + off;
    if (t < 0 || t >= static_cast<long long>(n_tiles)) continue;   // uniform across the CTA
    visit(static_cast<uint32_t>(t));
  }
  // the CTA's K-th distance: the largest over its queries (bits of a
  // non-negative float; 0xffffffff while some query holds fewer than K)
  auto cta_worst = [&]() -> uint32_t {
    const uint32_t mine = valid ? static_cast<uint32_t>(best[K - 1] >> 32) : 0u;
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, mine);
    __syncthreads();   // s_wmax / s_worst of the previous call are read
    if ((threadIdx.x & 31) == 0) s_wmax[threadIdx.x >> 5] = wmax;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t m = 0;
      for (int w = 0; w < kIniTile / 32; ++w) m = m > s_wmax[w] ? m : s_wmax[w];
      s_worst = m;
    }
    __syncthreads();
    return s_worst;
  };
  // tiles whose box can still hold a point closer than the CTA's K-th
  // distance (a box provably farther cannot; the margin covers rounding)
  auto too_far = [](float bd, uint32_t wb) {
    return wb < 0x7f800000u && bd * 0.99999f > __uint_as_float(wb);
  };
  uint32_t wb = cta_worst();
  if (threadIdx.x == 0) s_nlist = 0;
  __syncthreads();
  const IniBox qb = boxes[qt];
  for (uint32_t t = threadIdx.x; t < n_tiles; t += blockDim.x) {
    const long long d = static_cast<long long>(t) - static_cast<long long>(qt);
    if (d >= -(kIniWindow / 2) && d <= kIniWindow / 2) continue;   // visited
    const float bd = box_gap2(qb, boxes[t]);
    if (too_far(bd, wb)) continue;
    const uint32_t at = atomicAdd(&s_nlist, 1u);
    s_list[at] = t;
    if (at < static_cast<uint32_t>(kIniSorted)) s_bd[at] = bd;
  }
  __syncthreads();
  const uint32_t nl = s_nlist;
  if (nl <= static_cast<uint32_t>(kIniSorted)) {
    // nearest first (rank of each entry by (box distance, tile)); stop at
    // the first box the shrinking K-th distance rules out: every later one
    // is at least as far
    for (uint32_t e = threadIdx.x; e < nl; e += blockDim.x) {
      const float bd = s_bd[e];
      const uint32_t te = s_list[e];
      uint32_t rank = 0;
      for (uint32_t f = 0; f < nl; ++f) {
        const float bf = s_bd[f];
        rank += (bf < bd || (bf == bd && s_list[f] < te)) ? 1u : 0u;
      }
      s_st[rank] = te;
      s_sbd[rank] = bd;
    }
    __syncthreads();
    for (uint32_t l = 0; l < nl; ++l) {
      if (too_far(s_sbd[l], wb)) break;   // uniform: wb is the CTA's
      visit(s_st[l]);
      wb = cta_worst();
    }
  } else {
    for (uint32_t l = 0; l < nl; ++l) visit(s_list[l]);
  }
  if (pairs && (threadIdx.x & 31) == 0 && evaluated)
    atomicAdd(reinterpret_cast<unsigned long long*>(pairs), evaluated);
  if (valid) {
    const size_t row = static_cast<size_t>(orig[i]) * k;
#pragma unroll
    for (int t = 0; t < K; ++t)
      if (t < k) knn[row + t] = static_cast<int32_t>(static_cast<uint32_t>(best[t]));
  }
}

// One cyclic-Jacobi rotation zeroing A[p][q] of the symmetric 3x3 A and
// accumulating it into V (Golub & Van Loan, the symmetric Schur
// decomposition of the 2x2 subproblem): A <- J^T A J, V <- V J.
__device__ __forceinline__ void jacobi_rotate(float (&A)[3][3], float (&V)[3][3], int p, int q) {
  const float apq = A[p][q];
  if (fabsf(apq) < 1e-36f) return;
  const float theta = (A[q][q] - A[p][p]) / (2.f * apq);
  float t;
  if (fabsf(theta) > 1e18f) {
    t = 0.5f / theta;
  } else {
    t = copysignf(1.f, theta) / (fabsf(theta) + sqrtf(theta * theta + 1.f));
  }
  const float c = rsqrtf(t * t + 1.f), s = t * c;
  float B[3][3];
#pragma unroll
  for (int r = 0; r < 3; ++r) {   // B = A J
    B[r][p] = c * A[r][p] - s * A[r][q];
    B[r][q] = s * A[r][p] + c * A[r][q];
    B[r][3 - p - q] = A[r][3 - p - q];
  }
#pragma unroll
  for (int cidx = 0; cidx < 3; ++cidx) {   // A = J^T B
    A[p][cidx] = c * B[p][cidx] - s * B[q][cidx];
    A[q][cidx] = s * B[p][cidx] + c * B[q][cidx];
    A[3 - p - q][cidx] = B[3 - p - q][cidx];
  }
  A[p][q] = 0.f;
  A[q][p] = 0.f;
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const float vp = V[r][p], vq = V[r][q];
    V[r][p] = c * vp - s * vq;
    V[r][q] = s * vp + c * vq;
  }
}

__global__ void __launch_bounds__(256) k_ini_frame(const float* __restrict__ pts, uint32_t n,
                                                   const int32_t* __restrict__ knn, IniParams P,
                                                   lgs_surfel_params_out out, float* __restrict__ lam,
                                                   float* __restrict__ conf) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float px = pts[3 * i], py = pts[3 * i + 1], pz = pts[3 * i + 2];
  const int k = P.k;
  // neighbour offsets from the point (exact for points within a factor of
  // two of each other, Sterbenz), their mean, and the centred second moments
  float mx = 0.f, my = 0.f, mz = 0.f;
  for (int t = 0; t < k; ++t) {
    const int j = knn[static_cast<size_t>(i) * k + t];
    mx += pts[3 * j] - px;
    my += pts[3 * j + 1] - py;
    mz += pts[3 * j + 2] - pz;
  }
  const float ik = 1.f / static_cast<float>(k);
  mx *= ik;
  my *= ik;
  mz *= ik;
  float cxx = 0.f, cxy = 0.f, cxz = 0.f, cyy = 0.f, cyz = 0.f, czz = 0.f;
  for (int t = 0; t < k; ++t) {
    const int j = knn[static_cast<size_t>(i) * k + t];
    const float dx = (pts[3 * j] - px) - mx, dy = (pts[3 * j + 1] - py) - my, dz = (pts[3 * j + 2] - pz) - mz;
    cxx += dx * dx;
    cxy += dx * dy;
    cxz += dx * dz;
    cyy += dy * dy;
    cyz += dy * dz;
    czz += dz * dz;
  }
  float A[3][3] = {{cxx * ik, cxy * ik, cxz * ik}, {cxy * ik, cyy * ik, cyz * ik}, {cxz * ik, cyz * ik, czz * ik}};
  float V[3][3] = {{1.f, 0.f, 0.f}, {0.f, 1.f, 0.f}, {0.f, 0.f, 1.f}};
  for (int sweep = 0; sweep < 6; ++sweep) {
    jacobi_rotate(A, V, 0, 1);
    jacobi_rotate(A, V, 0, 2);
    jacobi_rotate(A, V, 1, 2);
  }
  // eigenpairs in descending order
  float ev[3] = {A[0][0], A[1][1], A[2][2]};
  int o[3] = {0, 1, 2};
  if (ev[o[0]] < ev[o[1]]) { const int x = o[0]; o[0] = o[1]; o[1] = x; }
  if (ev[o[1]] < ev[o[2]]) { const int x = o[1]; o[1] = o[2]; o[2] = x; }
  if (ev[o[0]] < ev[o[1]]) { const int x = o[0]; o[0] = o[1]; o[1] = x; }
  const float l0 = fmaxf(ev[o[0]], 0.f), l1 = fmaxf(ev[o[1]], 0.f), l2 = fmaxf(ev[o[2]], 0.f);
  float3 e0 = make_float3(V[0][o[0]], V[1][o[0]], V[2][o[0]]);
  float3 nn = make_float3(V[0][o[2]], V[1][o[2]], V[2][o[2]]);
  // the normal turned toward the sensor (the origin of the sensor frame)
  if (nn.x * px + nn.y * py + nn.z * pz > 0.f) nn = make_float3(-nn.x, -nn.y, -nn.z);
  float nl = rsqrtf(nn.x * nn.x + nn.y * nn.y + nn.z * nn.z);
  nn = make_float3(nn.x * nl, nn.y * nl, nn.z * nl);
  const float en = e0.x * nn.x + e0.y * nn.y + e0.z * nn.z;
  e0 = make_float3(e0.x - en * nn.x, e0.y - en * nn.y, e0.z - en * nn.z);
  nl = rsqrtf(e0.x * e0.x + e0.y * e0.y + e0.z * e0.z);
  const float3 tu = make_float3(e0.x * nl, e0.y * nl, e0.z * nl);
  const float3 tv = make_float3(nn.y * tu.z - nn.z * tu.y, nn.z * tu.x - nn.x * tu.z, nn.x * tu.y - nn.y * tu.x);
  // range-adaptive scale: clip(kappa max(|p|, 1) sigma_tan, s_min, s_max)
  const float rng = sqrtf(px * px + py * py + pz * pz);
  const float sg0 = sqrtf(l0), sg1 = sqrtf(l1);
  const float t1 = sg0 > 0.f ? sg1 / sg0 : 1.f;   // sigma_tan = (1, sigma_1 / sigma_0)
  const float r = fmaxf(rng, 1.f);
  const float s0 = fminf(fmaxf(P.kappa * r, P.s_min), P.s_max);
  const float s1 = fminf(fmaxf(P.kappa * r * t1, P.s_min), P.s_max);
  // physics-based confidence and opacity
  const float cosv = fabsf(nn.x * px + nn.y * py + nn.z * pz) / rng;
  const float ramp = fminf(fmaxf((cosv - P.c0) / (1.f - P.c0 + P.eps), 0.f), 1.f);
  const float q = rng / P.r0;
  const float u = expf(-q * q) * ramp;
  const float alpha = P.alpha_min + (P.alpha_max - P.alpha_min) * u;
  // world frame: Rw = R [t_u t_v n]; quaternion by the largest of
  // 1 + tr, 1 + 2 R_ii - tr (Shepperd's rule), w >= 0
  float W[3][3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    W[a][0] = P.R[3 * a] * tu.x + P.R[3 * a + 1] * tu.y + P.R[3 * a + 2] * tu.z;
    W[a][1] = P.R[3 * a] * tv.x + P.R[3 * a + 1] * tv.y + P.R[3 * a + 2] * tv.z;
    W[a][2] = P.R[3 * a] * nn.x + P.R[3 * a + 1] * nn.y + P.R[3 * a + 2] * nn.z;
  }
  const float tr = W[0][0] + W[1][1] + W[2][2];
  const float c0 = 1.f + tr, c1 = 1.f + 2.f * W[0][0] - tr, c2 = 1.f + 2.f * W[1][1] - tr,
              c3 = 1.f + 2.f * W[2][2] - tr;
  float qw, qx, qy, qz;
  if (c0 >= c1 && c0 >= c2 && c0 >= c3) {
    const float h = 2.f * sqrtf(c0);
    qw = 0.25f * h; qx = (W[2][1] - W[1][2]) / h; qy = (W[0][2] - W[2][0]) / h; qz = (W[1][0] - W[0][1]) / h;
  } else if (c1 >= c2 && c1 >= c3) {
    const float h = 2.f * sqrtf(c1);
    qw = (W[2][1] - W[1][2]) / h; qx = 0.25f * h; qy = (W[0][1] + W[1][0]) / h; qz = (W[0][2] + W[2][0]) / h;
  } else if (c2 >= c3) {
    const float h = 2.f * sqrtf(c2);
    qw = (W[0][2] - W[2][0]) / h; qx = (W[0][1] + W[1][0]) / h; qy = 0.25f * h; qz = (W[1][2] + W[2][1]) / h;
  } else {
    const float h = 2.f * sqrtf(c3);
    qw = (W[1][0] - W[0][1]) / h; qx = (W[0][2] + W[2][0]) / h; qy = (W[1][2] + W[2][1]) / h; qz = 0.25f * h;
  }
  const float qn = rsqrtf(qw * qw + qx * qx + qy * qy + qz * qz) * (qw < 0.f ? -1.f : 1.f);
  out.quat[4 * i] = qw * qn;
  out.quat[4 * i + 1] = qx * qn;
  out.quat[4 * i + 2] = qy * qn;
  out.quat[4 * i + 3] = qz * qn;
#pragma unroll
  for (int a = 0; a < 3; ++a)
    out.mean[3 * i + a] = P.R[3 * a] * px + P.R[3 * a + 1] * py + P.R[3 * a + 2] * pz + P.t[a];
  out.log_scale[2 * i] = logf(s0);
  out.log_scale[2 * i + 1] = logf(s1);
  out.opacity_logit[i] = logf(alpha / (1.f - alpha));
  lam[3 * i] = l0;
  lam[3 * i + 1] = l1;
  lam[3 * i + 2] = l2;
  conf[i] = u;
}

template <int K>
void launch_knn(const float* sp, const uint32_t* orig, uint32_t n, const IniBox* boxes, uint32_t n_tiles, int k,
                int32_t* knn, int64_t* pairs, cudaStream_t s) {
  k_ini_knn<K><<<n_tiles, kIniTile, 0, s>>>(sp, orig, n, boxes, n_tiles, k, knn, pairs);
}

// Scratch: tile boxes, the extent, cells and their counts / offsets, scan
// partials, the points in cell order and their original indices.
struct IniLayout {
  size_t boxes, ext, cell, cnt, off, part, sp, orig, total;
};

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

IniLayout ini_layout(int64_t n) {
  IniLayout L{};
  const size_t N = static_cast<size_t>(n > 0 ? n : 1);
  const size_t tiles = (N + kIniTile - 1) / kIniTile;
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = o; o = align256(o + bytes); return at; };
  L.boxes = take(tiles * sizeof(IniBox));
  L.ext = take(8 * sizeof(float));
  L.cell = take(4 * N);
  L.cnt = take(4 * static_cast<size_t>(kIniCells));
  L.off = take(4 * (static_cast<size_t>(kIniCells) + 1));
  L.part = take(scan_partials_bytes(kIniCells));
  L.sp = take(12 * N);
  L.orig = take(4 * N);
  L.total = o;
  return L;
}

}  // namespace

size_t init_scratch_bytes(int64_t n) { return ini_layout(n).total; }

int64_t init_max_points() { return static_cast<int64_t>(kIniMaxTiles) * kIniTile; }

// zero, boxes, extent, cells, scan (3), scatter, boxes, k-NN, frame
int init_launches() { return 11; }

cudaError_t launch_keyframe_init(const float* pts, int64_t n64, const float pose[12], const lgs_init_params& p,
                                 void* scratch, int32_t* knn, const lgs_surfel_params_out& out, float* lam,
                                 float* conf, int64_t* pairs, cudaStream_t s) {
  const uint32_t n = static_cast<uint32_t>(n64);
  if (n == 0) return cudaSuccess;
  const uint32_t n_tiles = (n + kIniTile - 1) / kIniTile;
  const IniLayout L = ini_layout(n);
  char* b = static_cast<char*>(scratch);
  IniBox* boxes = reinterpret_cast<IniBox*>(b + L.boxes);
  float* ext = reinterpret_cast<float*>(b + L.ext);
  uint32_t* cell = reinterpret_cast<uint32_t*>(b + L.cell);
  uint32_t* cnt = reinterpret_cast<uint32_t*>(b + L.cnt);
  uint32_t* off = reinterpret_cast<uint32_t*>(b + L.off);
  uint32_t* part = reinterpret_cast<uint32_t*>(b + L.part);
  float* sp = reinterpret_cast<float*>(b + L.sp);
  uint32_t* orig = reinterpret_cast<uint32_t*>(b + L.orig);
  const uint32_t g = (n + 255) / 256;
  k_ini_zero<<<512, 256, 0, s>>>(cnt, kIniCells);
  k_ini_boxes<<<n_tiles, kIniTile, 0, s>>>(pts, n, boxes);
  k_ini_extent<<<1, 256, 0, s>>>(boxes, n_tiles, ext);
  k_ini_cells<<<g, 256, 0, s>>>(pts, n, ext, cell, cnt);
  exclusive_scan_u32(cnt, off, kIniCells, part, s);
  k_ini_scatter<<<g, 256, 0, s>>>(pts, n, cell, off, cnt, sp, orig);
  k_ini_boxes<<<n_tiles, kIniTile, 0, s>>>(sp, n, boxes);
  if (p.k <= 8) launch_knn<8>(sp, orig, n, boxes, n_tiles, p.k, knn, pairs, s);
  else if (p.k <= 16) launch_knn<16>(sp, orig, n, boxes, n_tiles, p.k, knn, pairs, s);
  else if (p.k <= 20) launch_knn<20>(sp, orig, n, boxes, n_tiles, p.k, knn, pairs, s);
  else if (p.k <= 24) launch_knn<24>(sp, orig, n, boxes, n_tiles, p.k, knn, pairs, s);
  else launch_knn<32>(sp, orig, n, boxes, n_tiles, p.k, knn, pairs, s);
  IniParams P;
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) P.R[3 * a + b] = pose[4 * a + b];
    P.t[a] = pose[4 * a + 3];
  }
  P.kappa = p.kappa;
  P.s_min = p.s_min;
  P.s_max = p.s_max;
  P.r0 = p.r0;
  P.c0 = p.c0;
  P.eps = p.eps;
  P.alpha_min = p.alpha_min;
  P.alpha_max = p.alpha_max;
  P.k = p.k;
  k_ini_frame<<<(n + 255) / 256, 256, 0, s>>>(pts, n, knn, P, out, lam, conf);
  return cudaGetLastError();
}

}  // namespace lgs
