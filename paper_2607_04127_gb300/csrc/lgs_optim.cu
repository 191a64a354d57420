// lgs_optim.cu -- chain of the per-record gradients to the raw surfel
// parameters, the mapping loss (image terms + scale regulariser) with its
// upstream gradients, and a fused Adam step.
#include <algorithm>
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {

// ---------------------------------------------------------------------------
// Preprocess backward: for every surfel, sum over the frames that render its
// map the per-item gradient moments of the backward (see the layout in the
// compositing kernels), form the sensor-frame gradients of one item
//   dL/dmu  = (sum ct) n + (sum u g / s_u) t_u + (sum v g / s_v) t_v
//   dL/dt_u = -(sum u^2 g) t_u - (s_v / s_u)(sum u v g) t_v
//   dL/dt_v = -(s_u / s_v)(sum u v g) t_u - (sum v^2 g) t_v
//   dL/dn   = -s_u (sum ct u) t_u - s_v (sum ct v) t_v + sum w sg gS_n
//   dL/dlog s_u = sum u^2 g,  dL/dlog s_v = sum v^2 g,  dL/dlogit = (1 - alpha) sum g
// (t_u, t_v, n the unit axes; the axes enter at a fixed centre, and the
// intersection offset inside the plane is u s_u t_u + v s_v t_v), chain them
// through mu = R^T (mean - o), [t_u t_v n] = R^T R(q/|q|), then ACCUMULATE
// into the caller's gradient arrays.  The per-item buffer is zeroed as it is
// read, so it is all-zero between backward calls.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int map_of_surfel(const Desc& D, int64_t s) {
  int lo = 0, hi = D.n_maps - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (D.m[mid].surf_base <= s) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_preprocess_bwd(const Desc* __restrict__ D, float* __restrict__ g13,
                                                        Status* __restrict__ st) {
  pdl_wait();               // (launched after a kernel of this chain: wait for it)
  pdl_launch_dependents();  // the next kernel may be dispatched now
  // the backward before it is done: its claim counter and work-queue sizes
  // start the next chunked backward at zero
  if (blockIdx.x == 0 && threadIdx.x <= static_cast<unsigned>(kBwdClasses)) {
    if (threadIdx.x == 0) st->work_counter2 = 0u;
    else st->bq_count[threadIdx.x - 1] = 0u;
  }
  const int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= D->n_surf) return;
  const int m = map_of_surfel(*D, s);
  const MapDev& M = D->m[m];
  const int64_t i = s - M.surf_base;
  if (i >= M.n) return;
  // every load that does not depend on another one is issued here, before
  // the first store (the stores below would keep the compiler from moving
  // them up): the parameters, the gradient sums this surfel adds into, and
  // the moments of the map's first frame; the kernel is bound by the latency
  // of these loads, not by their bytes
  const float4 q = reinterpret_cast<const float4*>(M.quat)[i];
  const float lg = M.logit[i];
  const float ls0 = M.ls[2 * i], ls1 = M.ls[2 * i + 1];
  const float oq0 = M.d_quat[4 * i], oq1 = M.d_quat[4 * i + 1], oq2 = M.d_quat[4 * i + 2], oq3 = M.d_quat[4 * i + 3];
  const float om0 = M.d_mean[3 * i], om1 = M.d_mean[3 * i + 1], om2 = M.d_mean[3 * i + 2];
  const float ol0 = M.d_ls[2 * i], ol1 = M.d_ls[2 * i + 1], olg = M.d_logit[i];
  int f0 = 0;
  while (f0 < D->n_frames && D->f[f0].map != m) ++f0;
  float4 pa = make_float4(0.f, 0.f, 0.f, 0.f), pb = pa, pc = pa;
  if (f0 < D->n_frames) {
    const float4* gp = reinterpret_cast<const float4*>(g13 + 16 * (D->f[f0].item_base + i));
    pa = gp[0];
    pb = gp[1];
    pc = gp[2];
  }
  const float qn2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  const float inv = rsqrtf(qn2);
  const float w = q.x * inv, x = q.y * inv, y = q.z * inv, z = q.w * inv;
  const float c0[3] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y + w * z), 2.f * (x * z - w * y)};
  const float c1[3] = {2.f * (x * y - w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z + w * x)};
  const float c2[3] = {2.f * (x * z + w * y), 2.f * (y * z - w * x), 1.f - 2.f * (x * x + y * y)};
  const float alpha = 1.0f / (1.0f + expf(-lg));
  const float su = expf(ls0), sv = expf(ls1);
  float gm[3] = {0.f, 0.f, 0.f}, G0[3] = {0.f, 0.f, 0.f}, G1[3] = {0.f, 0.f, 0.f}, G2[3] = {0.f, 0.f, 0.f};
  float gls0 = 0.f, gls1 = 0.f, gsum = 0.f;
  bool any = false;
  for (int f = f0; f < D->n_frames; ++f) {
    const FrameDev& F = D->f[f];
    if (F.map != m) continue;
    float4* gp = reinterpret_cast<float4*>(g13 + 16 * (F.item_base + i));
    const float4 a = f == f0 ? pa : gp[0], b = f == f0 ? pb : gp[1], c = f == f0 ? pc : gp[2];
    if (a.x == 0.f && a.y == 0.f && a.z == 0.f && a.w == 0.f && b.x == 0.f && b.y == 0.f && b.z == 0.f &&
        b.w == 0.f && c.x == 0.f && c.y == 0.f && c.z == 0.f && c.w == 0.f)
      continue;
    any = true;
    const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
    gp[0] = zero; gp[1] = zero; gp[2] = zero;
    // moments: a = (g, u g, v g, u^2 g), b = (v^2 g, u v g, ct, ct u), c = (ct v, w sg gS_n)
    const float* R = F.R;
    // sensor-frame axes: v_s = R^T v_w
    float tu[3], tv[3], n[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      tu[k] = R[k] * c0[0] + R[3 + k] * c0[1] + R[6 + k] * c0[2];
      tv[k] = R[k] * c1[0] + R[3 + k] * c1[1] + R[6 + k] * c1[2];
      n[k] = R[k] * c2[0] + R[3 + k] * c2[1] + R[6 + k] * c2[2];
    }
    const float cmu_u = a.y / su, cmu_v = a.z / sv, uv = b.y;
    const float ktu_u = -a.w, ktu_v = -(sv / su) * uv;
    const float ktv_u = -(su / sv) * uv, ktv_v = -b.x;
    const float kn_u = -su * b.w, kn_v = -sv * c.x;
    float gmu[3], gtu[3], gtv[3], gnn[3];
    const float wsn[3] = {c.y, c.z, c.w};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      gmu[k] = b.z * n[k] + cmu_u * tu[k] + cmu_v * tv[k];
      gtu[k] = ktu_u * tu[k] + ktu_v * tv[k];
      gtv[k] = ktv_u * tu[k] + ktv_v * tv[k];
      gnn[k] = kn_u * tu[k] + kn_v * tv[k] + wsn[k];
    }
    gsum += a.x;
    gls0 += a.w;
    gls1 += b.x;
    // back to the world frame: v_w = R v_s
#pragma unroll
    for (int a2 = 0; a2 < 3; ++a2) {
      gm[a2] += R[3 * a2] * gmu[0] + R[3 * a2 + 1] * gmu[1] + R[3 * a2 + 2] * gmu[2];
      G0[a2] += R[3 * a2] * gtu[0] + R[3 * a2 + 1] * gtu[1] + R[3 * a2 + 2] * gtu[2];
      G1[a2] += R[3 * a2] * gtv[0] + R[3 * a2 + 1] * gtv[1] + R[3 * a2 + 2] * gtv[2];
      G2[a2] += R[3 * a2] * gnn[0] + R[3 * a2 + 1] * gnn[1] + R[3 * a2 + 2] * gnn[2];
    }
  }
  if (!any) return;
  // d/dq_hat of the columns of R(q_hat), contracted with (G0, G1, G2)
  const float gw = G0[1] * 2.f * z - G0[2] * 2.f * y - G1[0] * 2.f * z + G1[2] * 2.f * x + G2[0] * 2.f * y -
                   G2[1] * 2.f * x;
  const float gx = G0[1] * 2.f * y + G0[2] * 2.f * z + G1[0] * 2.f * y - G1[1] * 4.f * x + G1[2] * 2.f * w +
                   G2[0] * 2.f * z - G2[1] * 2.f * w - G2[2] * 4.f * x;
  const float gy = -G0[0] * 4.f * y + G0[1] * 2.f * x - G0[2] * 2.f * w + G1[0] * 2.f * x + G1[2] * 2.f * z +
                   G2[0] * 2.f * w + G2[1] * 2.f * z - G2[2] * 4.f * y;
  const float gz = -G0[0] * 4.f * z + G0[1] * 2.f * w + G0[2] * 2.f * x - G1[0] * 2.f * w - G1[1] * 4.f * z +
                   G1[2] * 2.f * y + G2[0] * 2.f * x + G2[1] * 2.f * y;
  // through q_hat = q / |q|
  const float pr = gw * w + gx * x + gy * y + gz * z;
  M.d_quat[4 * i] = oq0 + (gw - w * pr) * inv;
  M.d_quat[4 * i + 1] = oq1 + (gx - x * pr) * inv;
  M.d_quat[4 * i + 2] = oq2 + (gy - y * pr) * inv;
  M.d_quat[4 * i + 3] = oq3 + (gz - z * pr) * inv;
  M.d_mean[3 * i] = om0 + gm[0];
  M.d_mean[3 * i + 1] = om1 + gm[1];
  M.d_mean[3 * i + 2] = om2 + gm[2];
  M.d_ls[2 * i] = ol0 + gls0;
  M.d_ls[2 * i + 1] = ol1 + gls1;
  M.d_logit[i] = olg + gsum * (1.f - alpha);
}

cudaError_t launch_preprocess_bwd(const Layout&, const WsPtrs& w, const Desc& h, cudaStream_t s) {
  const int64_t n = h.n_surf > 0 ? h.n_surf : 1;
  // follows the backward's last kernel on the stream: dispatched while it runs
  return launch_dep(k_preprocess_bwd, dim3(static_cast<unsigned>((n + 255) / 256)), dim3(256), 0, s, w.desc, w.g13,
                    w.st);
}

// ---------------------------------------------------------------------------
// Mapping loss (Eqs. depthloss, normalloss, scaleloss, totalloss)
//   per frame f of map m (F_m frames render map m):
//     L_img,f = L_depth + la L_alpha + ln lng L_ng
//   L = sum_m [ (1/F_m) sum_{f in m} L_img,f + ls L_scale,m ]
// with masked means over M_D = [D > 0] and M_N = M_D [|N_gicp| > 0].
// ---------------------------------------------------------------------------
constexpr int kLossBlocks = 256;  // CTAs per frame and map

// Eq. scaleloss of map mi over this CTA's share of its surfels: sum of
// max(s) - s_max over the surfels above the threshold (fixed point) into the
// map's accumulator, and lambda_s max(s) added to d log s of the larger axis.
__device__ void scale_reg_row(const Desc& D, const lgs_loss_params& P, int write_grad, unsigned long long* acc,
                              int mi, long long* s_ll) {
  const MapDev& M = D.m[mi];
  long long sr = 0;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < M.n;
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float s0 = expf(M.ls[2 * i]), s1 = expf(M.ls[2 * i + 1]);
    const bool first = s0 >= s1;
    const float sm = first ? s0 : s1;
    if (sm > P.s_max) {
      // the sum takes at most 1 km per surfel (the gradient is exact)
      sr += to_fix(fminf(sm - P.s_max, 1e3f), kFixD);
      if (write_grad) M.d_ls[2 * i + (first ? 0 : 1)] += P.lambda_s * sm;
    }
  }
  cta_add_fix(sr, acc + 4 * LGS_MAX_FRAMES + mi, s_ll);
}

// Mask counts |M_D|, |M_N| of every frame: one integer atomic per CTA into
// ctot[F][2] (zero on entry: cleared by the binning and by the loss).  Rows
// y >= n_frames (when launched with them): the scale regulariser of map
// y - n_frames, which needs no rendered value, so a forward with the
// image-loss epilogue leaves only the loss vector for after it.  The first
// CTA also zeroes that forward's counters (`clear`, n_clear words: its tile
// counter), which spares the forward a memset.
__global__ void __launch_bounds__(256) k_loss_count(const Desc* __restrict__ D, int* __restrict__ ctot,
                                                    lgs_loss_params P, int write_grad,
                                                    unsigned long long* __restrict__ acc,
                                                    unsigned int* __restrict__ clear, int n_clear) {
  pdl_wait();               // (launched after a kernel of this chain: wait for it)
  pdl_launch_dependents();  // the next kernel may be dispatched now
  if (blockIdx.x == 0 && blockIdx.y == 0 && static_cast<int>(threadIdx.x) < n_clear) clear[threadIdx.x] = 0u;
  if (blockIdx.y >= static_cast<unsigned>(D->n_frames)) {
    __shared__ long long s_ll[8];
    scale_reg_row(*D, P, write_grad, acc, blockIdx.y - D->n_frames, s_ll);
    return;
  }
  const FrameDev& F = D->f[blockIdx.y];
  const int HW = F.H * F.W;
  int md = 0, mn = 0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
    const bool d = F.D[p] > 0.f;
    const float a = F.Ng[p], b = F.Ng[HW + p], c = F.Ng[2 * HW + p];
    md += d;
    mn += d && (a * a + b * b + c * c > 0.f);
  }
  for (int o = 16; o > 0; o >>= 1) {
    md += __shfl_xor_sync(0xffffffffu, md, o);
    mn += __shfl_xor_sync(0xffffffffu, mn, o);
  }
  // one atomic per CTA and count (every CTA of a frame adds to the same two
  // words, so per-warp atomics would queue at one L2 address)
  __shared__ int s_md[8], s_mn[8];
  const int wid = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) {
    s_md[wid] = md;
    s_mn[wid] = mn;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int a = 0, b = 0;
    for (int k = 0; k < static_cast<int>(blockDim.x >> 5); ++k) {
      a += s_md[k];
      b += s_mn[k];
    }
    if (a) atomicAdd(ctot + 2 * blockIdx.y, a);
    if (b) atomicAdd(ctot + 2 * blockIdx.y + 1, b);
  }
}

// ---- the N_surf term of Eq. normalloss ---------------------------------------
// X = Dh d: the rendered range of pixel (r, c) back-projected along its ray.
__device__ __forceinline__ float3 backproject(const FrameDev& F, int r, int c, float3& d) {
  const int p = r * F.W + c;
  const float Dh = F.St[p] / (F.A[p] + 1e-6f);
  pixel_ray(F, r, c, d.x, d.y, d.z);
  return make_float3(Dh * d.x, Dh * d.y, Dh * d.z);
}

__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 axpy3(float a, float3 x, float3 y) {
  return make_float3(a * x.x + y.x, a * x.y + y.y, a * x.z + y.z);
}

// The term of pixel (r, c): none on the last row, or unless the pixel, its
// next column (wrapping at 2 pi) and its next row all have a return (D > 0)
// and a rendered surface (A > 0: at least one composited surfel; a pixel that
// renders nothing has X = 0, and two such neighbours would make e_c parallel
// to e_r).  Otherwise
// N_surf = normalise(e_c x e_r), e_c = X(r, c+1) - X(r, c), e_r = X(r+1, c) -
// X(r, c); val = 1 - Nh . N_surf, and the gradients of k val w.r.t. X(r, c),
// X(r, c+1), X(r+1, c) and S_n(r, c).
struct NsTerm {
  float val;
  float3 gp, gr, gb, gsn;
};

__device__ bool ns_term(const FrameDev& F, int r, int c, float k, NsTerm& t) {
  if (r < 0 || r + 1 >= F.H) return false;
  const int W = F.W, HW = F.H * F.W;
  const int cr = c + 1 == W ? 0 : c + 1;
  const int p = r * W + c, pr = r * W + cr, pb = p + W;
  if (!(F.D[p] > 0.f && F.D[pr] > 0.f && F.D[pb] > 0.f)) return false;
  if (!(F.A[p] > 0.f && F.A[pr] > 0.f && F.A[pb] > 0.f)) return false;
  float3 d;
  const float3 X = backproject(F, r, c, d), XR = backproject(F, r, cr, d), XB = backproject(F, r + 1, c, d);
  const float3 ec = make_float3(XR.x - X.x, XR.y - X.y, XR.z - X.z);
  const float3 er = make_float3(XB.x - X.x, XB.y - X.y, XB.z - X.z);
  const float3 cx = cross3(ec, er);
  const float imc = 1.f / sqrtf(dot3(cx, cx) + 1e-12f);
  const float3 ns = make_float3(cx.x * imc, cx.y * imc, cx.z * imc);
  const float3 sn = make_float3(F.Sn[p], F.Sn[HW + p], F.Sn[2 * HW + p]);
  const float im = 1.f / sqrtf(dot3(sn, sn) + 1e-12f);
  const float3 nh = make_float3(sn.x * im, sn.y * im, sn.z * im);
  t.val = dot3(nh, ns);   // the caller forms 1 - val in double
  // dL/dNh = -k N_surf through Nh = S_n / |S_n|
  const float3 g = make_float3(-k * ns.x, -k * ns.y, -k * ns.z);
  t.gsn = axpy3(-dot3(sn, g) * im * im * im, sn, make_float3(g.x * im, g.y * im, g.z * im));
  // dL/dN_surf = -k Nh through N_surf = c / |c|, c = e_c x e_r
  const float3 gc = make_float3(-k * nh.x, -k * nh.y, -k * nh.z);
  const float3 gcx = axpy3(-dot3(cx, gc) * imc * imc * imc, cx, make_float3(gc.x * imc, gc.y * imc, gc.z * imc));
  t.gr = cross3(er, gcx);
  t.gb = cross3(gcx, ec);
  t.gp = make_float3(-(t.gr.x + t.gb.x), -(t.gr.y + t.gb.y), -(t.gr.z + t.gb.z));
  return true;
}

// Rows y < n_frames: the image terms of frame y and its upstream gradient
// planes; rows n_frames + m: the scale regulariser of map m.  The CTA that
// finishes last reduces every partial sum in a fixed order (deterministic)
// and writes the loss vector.
// Rows y < nfr: the image terms of frame y and its upstream gradient planes
// (nfr = 0 when a forward epilogue computed them); rows nfr + m: the scale
// regulariser of map m.
__global__ void __launch_bounds__(256) k_loss_main(const Desc* __restrict__ D, Status* __restrict__ st,
                                                    lgs_loss_params P, int write_grad, int* __restrict__ ctot,
                                                    unsigned long long* __restrict__ acc, float* __restrict__ out,
                                                    int nfr) {
  __shared__ long long s_ll[8];
  __shared__ bool s_last;
  if (blockIdx.y < static_cast<unsigned>(nfr)) {
    const int f = blockIdx.y;
    const FrameDev& F = D->f[f];
    const int HW = F.H * F.W;
    const int nd = __ldcg(ctot + 2 * f), nn = __ldcg(ctot + 2 * f + 1);
    const float scale = 1.0f / static_cast<float>(D->m[F.map].n_frames);
    const float ind = nd > 0 ? 1.0f / static_cast<float>(nd) : 0.f;
    const float inn = nn > 0 ? 1.0f / static_cast<float>(nn) : 0.f;
    const float kns = P.lambda_n * P.lambda_ns * ind;
    long long ld = 0, la = 0, ln = 0, ls = 0;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < HW; p += gridDim.x * blockDim.x) {
      float gA = 0.f, gSt = 0.f, gx = 0.f, gy = 0.f, gz = 0.f;
      // every plane of the pixel is loaded before any decision, so the loads
      // of a pixel overlap instead of following the mask test
      const float Dm = F.D[p];
      const float A = F.A[p], St = F.St[p];
      const float nx = F.Ng[p], ny = F.Ng[HW + p], nz = F.Ng[2 * HW + p];
      const float sx = F.Sn[p], sy = F.Sn[HW + p], sz = F.Sn[2 * HW + p];
      float g[5];
      pixel_image_loss(Dm, A, St, nx, ny, nz, sx, sy, sz, scale, ind, inn, P, g, ld, la, ln);
      gA = g[0];
      gSt = g[1];
      gx = g[2];
      gy = g[3];
      gz = g[4];
      if (Dm > 0.f) {
        const float a = A + 1e-6f;
        if (kns != 0.f) {
          // this pixel's own term, and the terms of its left and upper
          // neighbours, in which it is the next column / the next row
          const int r = p / F.W, c = p - r * F.W;
          float3 gX = make_float3(0.f, 0.f, 0.f);
          NsTerm t;
          if (ns_term(F, r, c, kns, t)) {
            ls += to_fix(1.0f - t.val, kFixU);
            gX = t.gp;
            gx += scale * t.gsn.x;
            gy += scale * t.gsn.y;
            gz += scale * t.gsn.z;
          }
          if (ns_term(F, r, c == 0 ? F.W - 1 : c - 1, kns, t)) gX = axpy3(1.f, t.gr, gX);
          if (ns_term(F, r - 1, c, kns, t)) gX = axpy3(1.f, t.gb, gX);
          float3 d;
          pixel_ray(F, r, c, d.x, d.y, d.z);
          const float gD = dot3(gX, d);
          gSt += scale * gD / a;
          gA += scale * (-gD * St / (a * a));
        }
      }
      F.oA[p] = gA;
      F.oSt[p] = gSt;
      F.oSn[p] = gx;
      F.oSn[HW + p] = gy;
      F.oSn[2 * HW + p] = gz;
    }
    cta_add_fix(ld, acc + 4 * f, s_ll);
    cta_add_fix(la, acc + 4 * f + 1, s_ll);
    cta_add_fix(ln, acc + 4 * f + 2, s_ll);
    cta_add_fix(ls, acc + 4 * f + 3, s_ll);
  } else {
    scale_reg_row(*D, P, write_grad, acc, blockIdx.y - nfr, s_ll);
  }

  // last CTA: the means and the loss vector from the fixed-point totals (no
  // reduction left to do), then the totals and counts are cleared for the
  // next call
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned total = gridDim.x * gridDim.y;
    s_last = atomicAdd(&st->loss_ticket, 1u) == total - 1;
  }
  __syncthreads();
  if (!s_last || threadIdx.x >= 32) return;
  finish_loss_vector(*D, P, ctot, acc, out, st);
}

cudaError_t launch_loss(const Layout&, const WsPtrs& w, const Desc& h, const lgs_loss_params& p, bool scale_grad,
                        float* loss_out, cudaStream_t s) {
  unsigned long long* acc = reinterpret_cast<unsigned long long*>(w.loss_part);
  int* ctot = loss_counts_ptr(w);
  // (between a forward and its backward: the forward's queues stay)
  k_loss_count<<<dim3(kLossBlocks, h.n_frames), 256, 0, s>>>(w.desc, ctot, p, 0, acc, nullptr, 0);
  k_loss_main<<<dim3(kLossBlocks, h.n_frames + h.n_maps), 256, 0, s>>>(w.desc, w.st, p, scale_grad ? 1 : 0, ctot,
                                                                        acc, loss_out, h.n_frames);
  return cudaGetLastError();
}

// Before a forward with the image-loss epilogue: the mask counts (the
// epilogue normalises by them) and the scale regulariser; the forward's
// long-list kernel writes the loss vector when every pixel is done.  Also
// zeroes the forward's tile counter.
cudaError_t launch_loss_counts(const WsPtrs& w, const Desc& h, const lgs_loss_params& p, bool scale_grad,
                               cudaStream_t s) {
  // one pixel or surfel per thread where it fits (a grid-stride loop would
  // put a chain of DRAM round trips on every thread) when the call has few
  // rows; kLossBlocks CTAs per row otherwise (more CTAs per row measured
  // slower on a 32-row call: every CTA adds its counts with atomics on a
  // few words).  The counts and the fixed-point sums do not depend on the
  // grid.
  int64_t most = 1;
  for (int f = 0; f < h.n_frames; ++f) most = std::max<int64_t>(most, static_cast<int64_t>(h.f[f].H) * h.f[f].W);
  for (int m = 0; m < h.n_maps; ++m) most = std::max<int64_t>(most, h.m[m].n);
  const int rows = h.n_frames + h.n_maps;
  const int64_t cap = std::max<int64_t>(kLossBlocks, 2048 / std::max(rows, 1));
  const int gx = static_cast<int>(std::min<int64_t>(cap, (most + 255) / 256));
  k_loss_count<<<dim3(gx, h.n_frames + h.n_maps), 256, 0, s>>>(
      w.desc, loss_counts_ptr(w), p, scale_grad ? 1 : 0, reinterpret_cast<unsigned long long*>(w.loss_part),
      &w.st->work_counter, 1);
  return cudaGetLastError();
}

// Loss accumulators: fixed-point sums [frames][4] and [maps], mask counts
// [frames][2].  All zero between calls (the binning clears them, and every
// loss call clears them after use).
size_t loss_part_bytes() {
  return sizeof(unsigned long long) * (4 * static_cast<size_t>(LGS_MAX_FRAMES) + LGS_MAX_MAPS) +
         sizeof(int) * 2 * static_cast<size_t>(LGS_MAX_FRAMES);
}

// ---------------------------------------------------------------------------
// Adam (the paper does not name its optimiser; this is the mapping loop's)
// ---------------------------------------------------------------------------
struct AdamSeg {
  float* p[4];
  float* g[4];
  float* m[4];
  float* v[4];
  int64_t n[4];
  float lr[4];
};

__global__ void __launch_bounds__(256) k_adam(AdamSeg a, float b1, float b2, float eps, float c1, float c2,
                                               int zero_grad) {
  const int sgm = blockIdx.y;
  float* __restrict__ p = a.p[sgm];
  float* __restrict__ g = a.g[sgm];
  float* __restrict__ m = a.m[sgm];
  float* __restrict__ v = a.v[sgm];
  const float lr = a.lr[sgm];
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n[sgm];
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    if (zero_grad) g[i] = 0.f;
  }
}

cudaError_t launch_adam(float* p[4], float* g[4], float* m[4], float* v[4], const int64_t cnt[4], int64_t step,
                        const float lr[4], float b1, float b2, float eps, int zero_grad, cudaStream_t s) {
  AdamSeg a;
  int64_t mx = 1;
  for (int k = 0; k < 4; ++k) {
    a.p[k] = p[k]; a.g[k] = g[k]; a.m[k] = m[k]; a.v[k] = v[k]; a.n[k] = cnt[k]; a.lr[k] = lr[k];
    if (cnt[k] > mx) mx = cnt[k];
  }
  const double c1 = 1.0 / (1.0 - pow(static_cast<double>(b1), static_cast<double>(step)));
  const double c2 = 1.0 / (1.0 - pow(static_cast<double>(b2), static_cast<double>(step)));
  int64_t blocks = (mx + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  k_adam<<<dim3(static_cast<unsigned>(blocks), 4), 256, 0, s>>>(a, b1, b2, eps, static_cast<float>(c1),
                                                                 static_cast<float>(c2), zero_grad);
  return cudaGetLastError();
}

// Batched form: segment 4 k + g is parameter group g of map k, each map with
// its own bias corrections.
struct AdamBatch {
  float* p[4 * LGS_MAX_MAPS];
  float* g[4 * LGS_MAX_MAPS];
  float* m[4 * LGS_MAX_MAPS];
  float* v[4 * LGS_MAX_MAPS];
  int64_t n[4 * LGS_MAX_MAPS];
  float lr[4 * LGS_MAX_MAPS];
  float c1[LGS_MAX_MAPS], c2[LGS_MAX_MAPS];
};

__global__ void __launch_bounds__(256) k_adam_batch(const __grid_constant__ AdamBatch a, float b1, float b2, float eps,
                                                    int zero_grad) {
  const int sgm = blockIdx.y, map = sgm >> 2;
  float* __restrict__ p = a.p[sgm];
  float* __restrict__ g = a.g[sgm];
  float* __restrict__ m = a.m[sgm];
  float* __restrict__ v = a.v[sgm];
  const float lr = a.lr[sgm], c1 = a.c1[map], c2 = a.c2[map];
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < a.n[sgm];
       i += static_cast<int64_t>(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    if (zero_grad) g[i] = 0.f;
  }
}

cudaError_t launch_adam_batch(const lgs_adam_map* maps, int n_maps, float b1, float b2, float eps, int zero_grad,
                              cudaStream_t s) {
  static_assert(sizeof(AdamBatch) < 32000, "kernel parameter size");
  AdamBatch a;
  int64_t mx = 1;
  for (int k = 0; k < n_maps; ++k) {
    const lgs_adam_map& M = maps[k];
    float* p[4] = {M.mean, M.quat, M.log_scale, M.logit};
    float* g[4] = {M.grad.d_mean, M.grad.d_quat, M.grad.d_log_scale, M.grad.d_opacity_logit};
    const int64_t cnt[4] = {3 * M.n, 4 * M.n, 2 * M.n, M.n};
    const int64_t off[4] = {0, 3 * M.n, 7 * M.n, 9 * M.n};
    for (int q = 0; q < 4; ++q) {
      a.p[4 * k + q] = p[q];
      a.g[4 * k + q] = g[q];
      a.m[4 * k + q] = M.m_state + off[q];
      a.v[4 * k + q] = M.v_state + off[q];
      a.n[4 * k + q] = cnt[q];
      a.lr[4 * k + q] = M.lr[q];
      if (cnt[q] > mx) mx = cnt[q];
    }
    a.c1[k] = static_cast<float>(1.0 / (1.0 - pow(static_cast<double>(b1), static_cast<double>(M.step))));
    a.c2[k] = static_cast<float>(1.0 / (1.0 - pow(static_cast<double>(b2), static_cast<double>(M.step))));
  }
  int64_t blocks = (mx + 255) / 256;
  if (blocks > 2048) blocks = 2048;
  k_adam_batch<<<dim3(static_cast<unsigned>(blocks), 4 * n_maps), 256, 0, s>>>(a, b1, b2, eps, zero_grad);
  return cudaGetLastError();
}

}  // namespace lgs
