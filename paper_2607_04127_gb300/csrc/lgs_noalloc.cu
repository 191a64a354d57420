// lgs_noalloc.cu -- the image terms of the mapping loss without a session or
// workspace (lgs_image_loss_noalloc in include/lgs.h).
//
// For callers that cannot allocate device memory when they need the loss:
// this entry point keeps its scratch (per-CTA partial sums, mask counts, a
// completion counter) in one file-scope static device array of fixed size,
// so neither the library nor the caller allocates anything.  The arithmetic
// and the reduction order are those of the image part of lgs_loss (same CTA
// count per frame, same per-pixel formulas, same fixed-order sums), so both
// give identical bits.
//
// The static scratch is shared by every call on a device: calls that overlap
// in time (other streams, other threads) corrupt each other's sums and must
// be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "lgs_internal.cuh"

namespace lgs {
namespace {

constexpr int kNaBlocks = 256;   // CTAs per frame (as the session loss)
constexpr int kNaThreads = 256;

// scratch layout: partial sums [frame][cta][4] doubles, mask counts
// [frame][cta][2] ints, completion counter
constexpr size_t kPartBytes = sizeof(double) * 4 * LGS_NOALLOC_MAX_FRAMES * kNaBlocks;
constexpr size_t kCountBytes = sizeof(int) * 2 * LGS_NOALLOC_MAX_FRAMES * kNaBlocks;
constexpr size_t kScratchBytes = kPartBytes + kCountBytes + 256;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct NaFrames {
  int n;
  int H[LGS_NOALLOC_MAX_FRAMES], W[LGS_NOALLOC_MAX_FRAMES];
  const float *A[LGS_NOALLOC_MAX_FRAMES], *St[LGS_NOALLOC_MAX_FRAMES], *Sn[LGS_NOALLOC_MAX_FRAMES];
  const float *D[LGS_NOALLOC_MAX_FRAMES], *Ng[LGS_NOALLOC_MAX_FRAMES];
  float *oA[LGS_NOALLOC_MAX_FRAMES], *oSt[LGS_NOALLOC_MAX_FRAMES], *oSn[LGS_NOALLOC_MAX_FRAMES];
};

struct NaScratch {
  double* part;
  int* cpart;
  unsigned int* ticket;
};

__device__ __forceinline__ double na_block_sum(double v, double* s_w) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_w[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) t += s_w[i];
  return t;
}

__device__ __forceinline__ int2 na_counts(const int* __restrict__ cpart, int f, int* s_i) {
  int a = 0, b = 0;
  for (int i = threadIdx.x; i < kNaBlocks; i += blockDim.x) {
    a += cpart[2 * (f * kNaBlocks + i)];
    b += cpart[2 * (f * kNaBlocks + i) + 1];
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = static_cast<int>(blockDim.x >> 5);
  __syncthreads();
  if (lane == 0) {
    s_i[2 * wid] = a;
    s_i[2 * wid + 1] = b;
  }
  __syncthreads();
  int ta = 0, tb = 0;
  for (int i = 0; i < nw; ++i) {
    ta += s_i[2 * i];
    tb += s_i[2 * i + 1];
  }
  return make_int2(ta, tb);
}

// Mask counts per (frame, CTA); CTA (0, 0) also clears the completion counter
// for the kernel that follows on the stream.
__global__ void __launch_bounds__(kNaThreads) k_na_count(NaFrames fr, NaScratch sc) {
  const int f = blockIdx.y;
  const int HW = fr.H[f] * fr.W[f];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *sc.ticket = 0u;
  int md = 0, mn = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    const bool d = fr.D[f][p] > 0.f;
    const float a = fr.Ng[f][p], b = fr.Ng[f][HW + p], c = fr.Ng[f][2 * HW + p];
    md += d;
    mn += d && (a * a + b * b + c * c > 0.f);
  }
  __shared__ int s_c[2][8];
  for (int o = 16; o > 0; o >>= 1) {
    md += __shfl_xor_sync(0xffffffffu, md, o);
    mn += __shfl_xor_sync(0xffffffffu, mn, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    s_c[0][wid] = md;
    s_c[1][wid] = mn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int i = 0; i < static_cast<int>(blockDim.x >> 5); ++i) {
      a += s_c[0][i];
      b += s_c[1][i];
    }
    int* o = sc.cpart + 2 * (static_cast<int64_t>(f) * kNaBlocks + blockIdx.x);
    o[0] = a;
    o[1] = b;
  }
}

// Image terms and upstream planes of every frame (weight 1 / n); the CTA
// that finishes last reduces the partial sums in a fixed order.
__global__ void __launch_bounds__(kNaThreads) k_na_main(NaFrames fr, NaScratch sc, lgs_loss_params P,
                                                         float* __restrict__ out) {
  __shared__ double s_w[8];
  __shared__ int s_i[16];
  __shared__ bool s_last;
  const int f = blockIdx.y;
  const int HW = fr.H[f] * fr.W[f];
  const int2 cnt = na_counts(sc.cpart, f, s_i);
  const int nd = cnt.x, nn = cnt.y;
  const float scale = 1.0f / static_cast<float>(fr.n);
  const float ind = nd > 0 ? 1.0f / static_cast<float>(nd) : 0.f;
  const float inn = nn > 0 ? 1.0f / static_cast<float>(nn) : 0.f;
  double ld = 0.0, la = 0.0, ln = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    float gA = 0.f, gSt = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    const float Dm = fr.D[f][p];
    if (Dm > 0.f) {
      const float A = fr.A[f][p], St = fr.St[f][p];
      const float a = A + 1e-6f;
      const float Dh = St / a;
      const float diff = Dh - Dm;
      ld += fabsf(diff);
      const float sgn = diff > 0.f ? 1.f : (diff < 0.f ? -1.f : 0.f);
      const float gDh = sgn * ind;
      gSt = scale * gDh / a;
      gA = scale * (-gDh * St / (a * a));
      la -= A >= 0.5f ? log1pf((A - 1.0f) + 1e-6f) : logf(A + 1e-6f);
      gA -= scale * P.lambda_alpha * ind / (A + 1e-6f);
      const float nx = fr.Ng[f][p], ny = fr.Ng[f][HW + p], nz = fr.Ng[f][2 * HW + p];
      if (nx * nx + ny * ny + nz * nz > 0.f) {
        const float sx = fr.Sn[f][p], sy = fr.Sn[f][HW + p], sz = fr.Sn[f][2 * HW + p];
        const float m = sqrtf(sx * sx + sy * sy + sz * sz + 1e-12f);
        const float im = 1.f / m;
        ln += 1.0 - static_cast<double>((sx * nx + sy * ny + sz * nz) * im);
        const float k = -P.lambda_n * P.lambda_ng * inn;
        const float g0 = k * nx, g1 = k * ny, g2 = k * nz;
        const float sg = (sx * g0 + sy * g1 + sz * g2) * im * im * im;
        gx = scale * (g0 * im - sx * sg);
        gy = scale * (g1 * im - sy * sg);
        gz = scale * (g2 * im - sz * sg);
      }
    }
    fr.oA[f][p] = gA;
    fr.oSt[f][p] = gSt;
    fr.oSn[f][p] = gx;
    fr.oSn[f][HW + p] = gy;
    fr.oSn[f][2 * HW + p] = gz;
  }
  const double t0 = na_block_sum(ld, s_w);
  const double t1 = na_block_sum(la, s_w);
  const double t2 = na_block_sum(ln, s_w);
  if (threadIdx.x == 0) {
    double* o = sc.part + 4 * (static_cast<int64_t>(f) * kNaBlocks + blockIdx.x);
    o[0] = t0;
    o[1] = t1;
    o[2] = t2;
    __threadfence();
    s_last = atomicAdd(sc.ticket, 1u) == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  __threadfence();
  // the first warp of the last CTA: partial sums in the fixed order of
  // warp_sum_partials (the order the session loss uses), terms per lane
  __shared__ double s_fr[LGS_NOALLOC_MAX_FRAMES][3];
  const int lane = threadIdx.x;
  if (lane == 0) *sc.ticket = 0u;
  for (int g = 0; g < fr.n; ++g) {
    double a[4];
    warp_sum_partials<3>(sc.part + 4 * static_cast<int64_t>(g) * kNaBlocks, kNaBlocks, a);
    if (lane == 0)
      for (int k = 0; k < 3; ++k) s_fr[g][k] = a[k];
  }
  __syncwarp();
  for (int g = lane; g < fr.n; g += 32) {
    int cd = 0, cn = 0;
    for (int b = 0; b < kNaBlocks; ++b) {
      cd += __ldcg(sc.cpart + 2 * (g * kNaBlocks + b));
      cn += __ldcg(sc.cpart + 2 * (g * kNaBlocks + b) + 1);
    }
    const float Ld = loss_mean(s_fr[g][0], cd), La = loss_mean(s_fr[g][1], cd), Ln = loss_mean(s_fr[g][2], cn);
    out[1 + 3 * g] = Ld;
    out[2 + 3 * g] = La;
    out[3 + 3 * g] = Ln;
    s_fr[g][0] = static_cast<double>(Ld + P.lambda_alpha * La + P.lambda_n * P.lambda_ng * Ln) /
                 static_cast<double>(fr.n);
  }
  __syncwarp();
  if (lane == 0) {
    double L = 0.0;
    for (int g = 0; g < fr.n; ++g) L += s_fr[g][0];
    out[0] = static_cast<float>(L);
  }
}

std::mutex g_mu;
void* g_addr[64] = {};

}  // namespace

size_t noalloc_scratch_bytes() { return kScratchBytes; }

// Device address of the static scratch on the current device: looked up
// once per device (with that device current) and cached.
cudaError_t noalloc_scratch(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

cudaError_t launch_image_loss_noalloc(void* scratch, int n_frames, const int32_t* H, const int32_t* W,
                                      const lgs_fwd_out* fwd, const lgs_target* targets,
                                      const lgs_loss_params& P, const lgs_fwd_grad_out* grads_out, float* loss_out,
                                      cudaStream_t s) {
  NaFrames fr{};
  fr.n = n_frames;
  for (int f = 0; f < n_frames; ++f) {
    fr.H[f] = H[f];
    fr.W[f] = W[f];
    fr.A[f] = fwd[f].A;
    fr.St[f] = fwd[f].S_t;
    fr.Sn[f] = fwd[f].S_n;
    fr.D[f] = targets[f].D;
    fr.Ng[f] = targets[f].N_gicp;
    fr.oA[f] = grads_out[f].dA;
    fr.oSt[f] = grads_out[f].dS_t;
    fr.oSn[f] = grads_out[f].dS_n;
  }
  unsigned char* base = static_cast<unsigned char*>(scratch);
  NaScratch sc{reinterpret_cast<double*>(base), reinterpret_cast<int*>(base + kPartBytes),
               reinterpret_cast<unsigned int*>(base + kPartBytes + kCountBytes)};
  k_na_count<<<dim3(kNaBlocks, n_frames), kNaThreads, 0, s>>>(fr, sc);
  k_na_main<<<dim3(kNaBlocks, n_frames), kNaThreads, 0, s>>>(fr, sc, P, loss_out);
  return cudaGetLastError();
}

}  // namespace lgs
