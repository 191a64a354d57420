// lgs_noalloc.cu -- the image terms of the mapping loss without a session or
// workspace (lgs_image_loss_noalloc in include/lgs.h).
//
// For callers that cannot allocate device memory when they need the loss:
// this entry point keeps its scratch (fixed-point loss sums, mask counts, a
// completion counter) in one file-scope static device array of fixed size,
// so neither the library nor the caller allocates anything.  The per-pixel
// arithmetic and the fixed-point sums are those of the image part of
// lgs_loss (integer sums are exact in any order), so both give identical
// bits.  The call leaves the sums and counts at zero for the next one.
//
// The static scratch is shared by every call on a device: calls that overlap
// in time (other streams, other threads) corrupt each other's sums and must
// be serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>

#include "lgs_internal.cuh"

namespace lgs {
namespace {

constexpr int kNaBlocks = 256;   // CTAs per frame (as the session loss)
constexpr int kNaThreads = 256;

// scratch layout: fixed-point sums [frame][3] (L_depth, L_alpha, L_ng), mask
// counts [frame][2], completion counter; all zero between calls
constexpr size_t kAccBytes = sizeof(unsigned long long) * 3 * LGS_NOALLOC_MAX_FRAMES;
constexpr size_t kCountBytes = sizeof(int) * 2 * LGS_NOALLOC_MAX_FRAMES;
constexpr size_t kScratchBytes = kAccBytes + kCountBytes + 256;
static_assert(kScratchBytes == LGS_NOALLOC_SCRATCH_BYTES, "scratch size must match the header");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct NaFrames {
  int n;
  int H[LGS_NOALLOC_MAX_FRAMES], W[LGS_NOALLOC_MAX_FRAMES];
  const float *A[LGS_NOALLOC_MAX_FRAMES], *St[LGS_NOALLOC_MAX_FRAMES], *Sn[LGS_NOALLOC_MAX_FRAMES];
  const float *D[LGS_NOALLOC_MAX_FRAMES], *Ng[LGS_NOALLOC_MAX_FRAMES];
  float *oA[LGS_NOALLOC_MAX_FRAMES], *oSt[LGS_NOALLOC_MAX_FRAMES], *oSn[LGS_NOALLOC_MAX_FRAMES];
};

struct NaScratch {
  unsigned long long* acc;
  int* ctot;
  unsigned int* ticket;
};

// Mask counts of every frame: one integer atomic per warp into ctot[F][2]
// (zero on entry).
__global__ void __launch_bounds__(kNaThreads) k_na_count(NaFrames fr, NaScratch sc) {
  const int f = blockIdx.y;
  const int HW = fr.H[f] * fr.W[f];
  int md = 0, mn = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    const bool d = fr.D[f][p] > 0.f;
    const float a = fr.Ng[f][p], b = fr.Ng[f][HW + p], c = fr.Ng[f][2 * HW + p];
    md += d;
    mn += d && (a * a + b * b + c * c > 0.f);
  }
  for (int o = 16; o > 0; o >>= 1) {
    md += __shfl_xor_sync(0xffffffffu, md, o);
    mn += __shfl_xor_sync(0xffffffffu, mn, o);
  }
  if ((threadIdx.x & 31) == 0) {
    if (md) atomicAdd(sc.ctot + 2 * f, md);
    if (mn) atomicAdd(sc.ctot + 2 * f + 1, mn);
  }
}

// Image terms and upstream planes of every frame (weight 1 / n), summed in
// fixed point; the CTA that finishes last forms the means and clears the
// scratch.
__global__ void __launch_bounds__(kNaThreads) k_na_main(NaFrames fr, NaScratch sc, lgs_loss_params P,
                                                         float* __restrict__ out) {
  __shared__ long long s_ll[8];
  __shared__ bool s_last;
  const int f = blockIdx.y;
  const int HW = fr.H[f] * fr.W[f];
  const int nd = __ldcg(sc.ctot + 2 * f), nn = __ldcg(sc.ctot + 2 * f + 1);
  const float scale = 1.0f / static_cast<float>(fr.n);
  const float ind = nd > 0 ? 1.0f / static_cast<float>(nd) : 0.f;
  const float inn = nn > 0 ? 1.0f / static_cast<float>(nn) : 0.f;
  long long ld = 0, la = 0, ln = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    float gA = 0.f, gSt = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
    const float Dm = fr.D[f][p];
    const float A = fr.A[f][p], St = fr.St[f][p];
    const float nx = fr.Ng[f][p], ny = fr.Ng[f][HW + p], nz = fr.Ng[f][2 * HW + p];
    const float sx = fr.Sn[f][p], sy = fr.Sn[f][HW + p], sz = fr.Sn[f][2 * HW + p];
    float g[5];
    pixel_image_loss(Dm, A, St, nx, ny, nz, sx, sy, sz, scale, ind, inn, P, g, ld, la, ln);
    gA = g[0];
    gSt = g[1];
    gx = g[2];
    gy = g[3];
    gz = g[4];
    fr.oA[f][p] = gA;
    fr.oSt[f][p] = gSt;
    fr.oSn[f][p] = gx;
    fr.oSn[f][HW + p] = gy;
    fr.oSn[f][2 * HW + p] = gz;
  }
  cta_add_fix(ld, sc.acc + 3 * f, s_ll);
  cta_add_fix(la, sc.acc + 3 * f + 1, s_ll);
  cta_add_fix(ln, sc.acc + 3 * f + 2, s_ll);
  if (threadIdx.x == 0) {
    __threadfence();
    s_last = atomicAdd(sc.ticket, 1u) == gridDim.x * gridDim.y - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  __threadfence();
  __shared__ float s_fr[LGS_NOALLOC_MAX_FRAMES];
  const int lane = threadIdx.x;
  for (int g = lane; g < fr.n; g += 32) {
    const int cd = __ldcg(sc.ctot + 2 * g), cn = __ldcg(sc.ctot + 2 * g + 1);
    const float Ld = fix_mean(static_cast<long long>(__ldcg(sc.acc + 3 * g)), kFixD, cd);
    const float La = fix_mean(static_cast<long long>(__ldcg(sc.acc + 3 * g + 1)), kFixU, cd);
    const float Ln = fix_mean(static_cast<long long>(__ldcg(sc.acc + 3 * g + 2)), kFixU, cn);
    out[1 + 3 * g] = Ld;
    out[2 + 3 * g] = La;
    out[3 + 3 * g] = Ln;
    s_fr[g] = (Ld + P.lambda_alpha * La + P.lambda_n * P.lambda_ng * Ln) / static_cast<float>(fr.n);
  }
  __syncwarp();
  if (lane == 0) {
    float L = 0.0f;
    for (int g = 0; g < fr.n; ++g) L += s_fr[g];
    out[0] = L;
    *sc.ticket = 0u;
  }
  for (int g = lane; g < fr.n; g += 32) {
    sc.ctot[2 * g] = 0;
    sc.ctot[2 * g + 1] = 0;
    for (int k = 0; k < 3; ++k) sc.acc[3 * g + k] = 0ull;
  }
}

}  // namespace

size_t noalloc_scratch_bytes() { return kScratchBytes; }

// Device address of the static scratch in the current device's context,
// looked up on every call (with that device current).  Nothing is cached:
// after a device reset, or in a new primary context, the module is loaded
// again at another address, and a cached pointer would be stale.  The first
// lookup in a context may load the library's device code there.
cudaError_t noalloc_scratch(void** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
  if (e != cudaSuccess) return e;
  *out = p;
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
  NaScratch sc{reinterpret_cast<unsigned long long*>(base), reinterpret_cast<int*>(base + kAccBytes),
               reinterpret_cast<unsigned int*>(base + kAccBytes + kCountBytes)};
  k_na_count<<<dim3(kNaBlocks, n_frames), kNaThreads, 0, s>>>(fr, sc);
  k_na_main<<<dim3(kNaBlocks, n_frames), kNaThreads, 0, s>>>(fr, sc, P, loss_out);
  return cudaGetLastError();
}

}  // namespace lgs
