// lgs_api.cu -- the C ABI (include/lgs.h): sessions, workspace layout,
// argument validation and the launch sequence of every entry point.
#include <cuda_runtime.h>

#include <cstddef>

#include <vector>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>

#include "lgs_internal.cuh"

using lgs::Desc;
using lgs::Layout;
using lgs::Status;
using lgs::WsPtrs;

static_assert(sizeof(Desc) < 32000, "descriptors are passed as one kernel parameter (<= 32764 bytes)");
static_assert(sizeof(Desc) % 4 == 0, "descriptor copy works on 32-bit words");

struct lgs_session_s {
  int device = 0;
  size_t budget = 0;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool binned = false;
  Layout lay{};
  Desc* desc = nullptr;         // host copy of the last bin_sort's descriptors
  Desc* desc_prev = nullptr;    // scratch: the descriptors before a bin_sort rebuilt them
  Desc* desc_dev = nullptr;     // what the workspace's descriptor block holds (when desc_dev_at is set)
  const void* desc_dev_at = nullptr;
  size_t g13_zero_off = 0;      // g13 region known to be all-zero
  int64_t g13_zero_items = -1;
  cudaStream_t last_stream = nullptr;
  lgs_tuning tune{0, 0, 16, 0};
  bool ckpt_valid = false;      // the last forward since binning wrote the backward's chunk checkpoints
  Status* h_status = nullptr;   // pinned
  int64_t launches = 0;         // kernels enqueued by this session
  // optional device timing of kernel groups
  struct Timed {
    int group;
    cudaEvent_t a, b;
  };
  bool timing = false;
  std::vector<Timed> timed;
  std::vector<cudaEvent_t> ev_pool;
  // side stream of the binning: the long-bucket sort runs on it alongside the
  // short buckets' sort, forked from and joined to the caller's stream
  lgs::SideStream side{nullptr, nullptr, nullptr};
};

namespace {

thread_local char g_err[512] = "";

lgs_status fail(lgs_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
lgs_status fail(lgs_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

lgs_status cuda_fail(cudaError_t e, const char* where) {
  return fail(LGS_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

size_t align_up(size_t x, size_t a = 256) { return (x + a - 1) / a * a; }

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// ---------------------------------------------------------------------------
// Validation and descriptor construction
// ---------------------------------------------------------------------------
lgs_status check_frames(const lgs_frame* frames, int n_frames) {
  if (!frames) return fail(LGS_ERR_INVALID_ARG, "frames is NULL");
  if (n_frames < 1 || n_frames > LGS_MAX_FRAMES)
    return fail(LGS_ERR_INVALID_ARG, "n_frames=%d outside [1, %d]", n_frames, LGS_MAX_FRAMES);
  const int th = frames[0].tile_h, tw = frames[0].tile_w;
  for (int f = 0; f < n_frames; ++f) {
    const lgs_frame& F = frames[f];
    if (F.H < 1 || F.W < 1) return fail(LGS_ERR_INVALID_ARG, "frame %d: H=%d W=%d", f, F.H, F.W);
    if (F.H > (1 << 16) || F.W > (1 << 16)) return fail(LGS_ERR_INVALID_ARG, "frame %d too large", f);
    if (F.tile_h < 1 || F.tile_w < 1 || F.tile_h * F.tile_w > LGS_MAX_TILE_PIXELS || (F.tile_h * F.tile_w) % 32)
      return fail(LGS_ERR_INVALID_ARG, "frame %d: tile %dx%d must have a multiple of 32 pixels, at most %d", f,
                  F.tile_h, F.tile_w, LGS_MAX_TILE_PIXELS);
    if (F.tile_h != th || F.tile_w != tw)
      return fail(LGS_ERR_INVALID_ARG, "frame %d: all frames of a call need the same tile shape", f);
    if (!(F.elev_min < F.elev_max) || !(F.elev_min >= -1.5707964f) || !(F.elev_max <= 1.5707964f))
      return fail(LGS_ERR_INVALID_ARG, "frame %d: elevation range [%g, %g] invalid", f, F.elev_min, F.elev_max);
    for (int k = 0; k < 12; ++k)
      if (!std::isfinite(F.pose[k])) return fail(LGS_ERR_INVALID_ARG, "frame %d: pose not finite", f);
  }
  return LGS_OK;
}

lgs_status check_maps(const lgs_surfels* maps, int n_maps, const int32_t* frame_map, int n_frames) {
  if (!maps) return fail(LGS_ERR_INVALID_ARG, "surfels is NULL");
  if (n_maps < 1 || n_maps > LGS_MAX_MAPS)
    return fail(LGS_ERR_INVALID_ARG, "n_maps=%d outside [1, %d]", n_maps, LGS_MAX_MAPS);
  for (int m = 0; m < n_maps; ++m) {
    const lgs_surfels& M = maps[m];
    if (M.n < 0) return fail(LGS_ERR_INVALID_ARG, "map %d: n < 0", m);
    if (M.n > 0 && (!M.mean || !M.quat || !M.log_scale || !M.opacity_logit))
      return fail(LGS_ERR_INVALID_ARG, "map %d: NULL parameter pointer", m);
    if (M.n > 0 && (reinterpret_cast<uintptr_t>(M.quat) & 15))
      return fail(LGS_ERR_INVALID_ARG, "map %d: quat must be 16-byte aligned", m);
  }
  if (frame_map)
    for (int f = 0; f < n_frames; ++f)
      if (frame_map[f] < 0 || frame_map[f] >= n_maps)
        return fail(LGS_ERR_INVALID_ARG, "frame %d: map index %d invalid", f, frame_map[f]);
  return LGS_OK;
}

struct Plan {
  int64_t n_items = 0, n_surf = 0;
  uint32_t n_tiles = 0;
  uint32_t table_floats = 0;
  uint32_t tile_pixels = 0;
};

lgs_status build_desc(const lgs_surfels* maps, int n_maps, const lgs_frame* frames, const int32_t* frame_map,
                      int n_frames, Desc& d, Plan& p) {
  memset(&d, 0, sizeof(Desc));
  d.n_frames = n_frames;
  d.n_maps = n_maps;
  d.th = frames[0].tile_h;
  d.tw = frames[0].tile_w;
  int64_t surf = 0;
  for (int m = 0; m < n_maps; ++m) {
    lgs::MapDev& M = d.m[m];
    M.mean = maps[m].mean;
    M.quat = maps[m].quat;
    M.ls = maps[m].log_scale;
    M.logit = maps[m].opacity_logit;
    M.n = maps[m].n;
    M.surf_base = surf;
    surf += maps[m].n;
  }
  uint64_t tiles = 0, items = 0, tab = 0;
  for (int f = 0; f < n_frames; ++f) {
    const lgs_frame& F = frames[f];
    lgs::FrameDev& D = d.f[f];
    const int m = frame_map ? frame_map[f] : 0;
    D.H = F.H;
    D.W = F.W;
    D.th = F.tile_h;
    D.tw = F.tile_w;
    D.ntr = ceil_div(F.H, F.tile_h);
    D.ntc = ceil_div(F.W, F.tile_w);
    D.map = m;
    D.tile_base = static_cast<uint32_t>(tiles);
    D.item_base = static_cast<int64_t>(items);
    D.n = maps[m].n;
    D.row_tab = static_cast<uint32_t>(tab);
    tab += 2 * static_cast<uint64_t>(D.ntr);
    tab = (tab + 3) & ~3ull;   // column tables are read as float4: 16-byte aligned
    D.col_tab = static_cast<uint32_t>(tab);
    tab += 4 * static_cast<uint64_t>(D.ntc);
    D.emin = F.elev_min;
    D.emax = F.elev_max;
    for (int a = 0; a < 3; ++a) {
      for (int b = 0; b < 3; ++b) D.R[3 * a + b] = F.pose[4 * a + b];
      D.o[a] = F.pose[4 * a + 3];
    }
    tiles += static_cast<uint64_t>(D.ntr) * D.ntc;
    items += static_cast<uint64_t>(maps[m].n);
    d.m[m].n_frames += 1;
  }
  if (tiles >= (1ull << 31)) return fail(LGS_ERR_INVALID_ARG, "too many tiles (%llu)", (unsigned long long)tiles);
  if (items >= 0xffffffffull) return fail(LGS_ERR_INVALID_ARG, "too many (frame, surfel) items");
  d.n_tiles = static_cast<uint32_t>(tiles);
  d.n_items = static_cast<int64_t>(items);
  d.n_surf = surf;
  p.n_items = d.n_items;
  p.n_surf = surf;
  p.n_tiles = d.n_tiles;
  p.table_floats = static_cast<uint32_t>(tab);
  p.tile_pixels = static_cast<uint32_t>(d.th * d.tw);
  return LGS_OK;
}

// Backward chunks that pairs_cap pairs over `tiles` tiles can form: every
// non-empty tile list of n entries has ceil(n / kChunk) <= n / kChunk + 1.
int64_t chunk_cap(int64_t pairs_cap, uint32_t tiles) {
  return (pairs_cap > 0 ? pairs_cap : 0) / lgs::kChunk + static_cast<int64_t>(tiles) + 1;
}

Layout make_layout(int64_t items, uint32_t tiles, int64_t pairs_cap, uint32_t table_floats, uint32_t tile_pixels) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + (bytes ? bytes : 1));
    return o;
  };
  const size_t I = static_cast<size_t>(items > 0 ? items : 1);
  const size_t P = static_cast<size_t>(pairs_cap > 0 ? pairs_cap : 1);
  const size_t T = static_cast<size_t>(tiles > 0 ? tiles : 1);
  L.desc = take(sizeof(Desc));
  L.status = take(sizeof(Status));
  L.tables = take(sizeof(float) * (table_floats + 4));
  L.rec = take(64 * I);
  L.box = take(16 * I);
  L.key = take(4 * I);
  L.cnt = take(4 * I);
  L.tset = take(8 * I);
  L.tcur = take(4 * T);
  L.pkey = take(8 * P);
  L.ptile = take(4 * P);
  L.pv = take(4 * P);
  L.ranges = take(8 * T);
  L.g13 = take(64 * I);
  L.work = take(4 * T);
  L.longt = take(4 * T);
  L.loss_part = take(lgs::loss_part_bytes());
  const int64_t C = chunk_cap(pairs_cap, tiles);
  L.cbase = take(4 * T);
  L.ckpt = take(sizeof(float) * lgs::kCkptSlots * static_cast<size_t>(tile_pixels) * static_cast<size_t>(C));
  L.csuf = take(sizeof(float) * static_cast<size_t>(tile_pixels) * static_cast<size_t>(C));
  L.cmask = take(sizeof(uint32_t) * 4 * static_cast<size_t>(tile_pixels) * static_cast<size_t>(C));
  L.midl = take(4 * T);
  // backward queues: class 0 takes at most every (chunk, warp block) item,
  // every other class at most one item per (tile, warp block)
  const size_t blocks = tile_pixels >= 32 ? tile_pixels / 32 : 1;
  L.bq_cap0 = static_cast<uint32_t>(static_cast<size_t>(C) * blocks);
  L.bq_capk = static_cast<uint32_t>(T * blocks);
  L.bwm = take(sizeof(uint32_t) * T * blocks);
  L.bq = take(sizeof(uint2) * (static_cast<size_t>(L.bq_cap0) + (lgs::kBwdClasses - 1) * static_cast<size_t>(L.bq_capk)));
  L.chunks_cap = C;
  L.total = off;
  L.items_cap = items;
  L.pairs_cap = pairs_cap;
  L.tiles_cap = tiles;
  L.tables_cap = table_floats;
  return L;
}

// Largest pair capacity whose layout fits in `bytes` (-1 if none).
int64_t fit_pairs(size_t bytes, const Plan& p) {
  if (make_layout(p.n_items, p.n_tiles, 0, p.table_floats, p.tile_pixels).total > bytes) return -1;
  int64_t lo = 0, hi = 1;
  while (hi < (1ll << 32) && make_layout(p.n_items, p.n_tiles, hi, p.table_floats, p.tile_pixels).total <= bytes) hi *= 2;
  if (hi > 0xfffffffell) hi = 0xfffffffell;
  while (lo < hi) {
    const int64_t mid = lo + (hi - lo + 1) / 2;
    if (make_layout(p.n_items, p.n_tiles, mid, p.table_floats, p.tile_pixels).total <= bytes) lo = mid; else hi = mid - 1;
  }
  return lo;
}

cudaEvent_t take_event(lgs_session s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Runs launch() between two events on cs when timing is on and cs is not
// capturing.
template <class F>
cudaError_t timed(lgs_session s, int group, cudaStream_t cs, F launch) {
  if (!s->timing) return launch();
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(cs, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone) return launch();
  cudaEvent_t a = take_event(s), b = take_event(s);
  if (!a || !b) return launch();
  cudaEventRecord(a, cs);
  const cudaError_t e = launch();
  cudaEventRecord(b, cs);
  s->timed.push_back({group, a, b});
  return e;
}

void drop_timing(lgs_session s) {
  for (auto& t : s->timed) {
    s->ev_pool.push_back(t.a);
    s->ev_pool.push_back(t.b);
  }
  s->timed.clear();
}

// Copy the descriptors to the workspace unless it already holds exactly
// these.  Calls captured into a CUDA graph always copy (the graph must carry
// its own copy) and make the next call copy again.
cudaError_t write_desc(lgs_session s, const Desc& d, Desc* dev, cudaStream_t cs, int64_t& launches) {
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(cs, &cap);
  if (e != cudaSuccess) return e;
  const bool capturing = cap != cudaStreamCaptureStatusNone;
  if (!capturing && s->desc_dev_at == dev && memcmp(&d, s->desc_dev, sizeof(Desc)) == 0) return cudaSuccess;
  if ((e = timed(s, LGS_TIME_DESC, cs, [&] { return lgs::launch_write_desc(d, dev, nullptr, cs); })) != cudaSuccess)
    return e;
  ++launches;
  if (capturing) {
    s->desc_dev_at = nullptr;
  } else {
    memcpy(s->desc_dev, &d, sizeof(Desc));
    s->desc_dev_at = dev;
  }
  return cudaSuccess;
}

// Keep the per-call pointers of the previous descriptors (a bin_sort
// rebuilds the geometry only; every call sets the pointers it uses), so that
// repeated steps over the same buffers leave the descriptors unchanged.
void keep_call_ptrs(Desc& d, const Desc& prev) {
  for (int f = 0; f < LGS_MAX_FRAMES; ++f) {
    lgs::FrameDev& a = d.f[f];
    const lgs::FrameDev& b = prev.f[f];
    a.A = b.A; a.St = b.St; a.Sn = b.Sn; a.Tf = b.Tf; a.nc = b.nc;
    a.gA = b.gA; a.gSt = b.gSt; a.gSn = b.gSn;
    a.oA = b.oA; a.oSt = b.oSt; a.oSn = b.oSn; a.D = b.D; a.Ng = b.Ng;
  }
  for (int m = 0; m < LGS_MAX_MAPS; ++m) {
    d.m[m].d_mean = prev.m[m].d_mean;
    d.m[m].d_quat = prev.m[m].d_quat;
    d.m[m].d_ls = prev.m[m].d_ls;
    d.m[m].d_logit = prev.m[m].d_logit;
  }
}

lgs_status enter(lgs_session s) {
  if (!s) return fail(LGS_ERR_INVALID_ARG, "session is NULL");
  cudaError_t e = cudaSetDevice(s->device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  return LGS_OK;
}

// The frames of a render call must be those of the last bin_sort.
lgs_status check_same(lgs_session s, const lgs_surfels* maps, int n_maps, const lgs_frame* frames,
                      const int32_t* frame_map, int n_frames) {
  if (!s->binned) return fail(LGS_ERR_STATE, "render before lgs_bin_sort");
  const Desc& d = *s->desc;
  if (n_frames != d.n_frames || n_maps != d.n_maps)
    return fail(LGS_ERR_STATE, "frames / maps differ from the last lgs_bin_sort");
  for (int m = 0; m < n_maps; ++m)
    if (maps[m].n != d.m[m].n) return fail(LGS_ERR_STATE, "map %d size differs from the last lgs_bin_sort", m);
  for (int f = 0; f < n_frames; ++f) {
    const lgs::FrameDev& D = d.f[f];
    const lgs_frame& F = frames[f];
    if (F.H != D.H || F.W != D.W || F.tile_h != D.th || F.tile_w != D.tw || (frame_map ? frame_map[f] : 0) != D.map)
      return fail(LGS_ERR_STATE, "frame %d differs from the last lgs_bin_sort", f);
  }
  return LGS_OK;
}

void set_map_ptrs(Desc& d, const lgs_surfels* maps, int n_maps) {
  for (int m = 0; m < n_maps; ++m) {
    d.m[m].mean = maps[m].mean;
    d.m[m].quat = maps[m].quat;
    d.m[m].ls = maps[m].log_scale;
    d.m[m].logit = maps[m].opacity_logit;
  }
}

lgs_status check_fwd_out(const lgs_fwd_out* o, int n_frames) {
  if (!o) return fail(LGS_ERR_INVALID_ARG, "forward outputs are NULL");
  for (int f = 0; f < n_frames; ++f)
    if (!o[f].A || !o[f].S_t || !o[f].S_n || !o[f].T_final || !o[f].n_contrib)
      return fail(LGS_ERR_INVALID_ARG, "frame %d: NULL forward output", f);
  return LGS_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Entry points
// ---------------------------------------------------------------------------
extern "C" {

const char* lgs_version(void) { return "lgs 0.1 (sm_103a)"; }

const char* lgs_last_error(void) { return g_err; }

const char* lgs_status_string(lgs_status st) {
  switch (st) {
    case LGS_OK: return "ok";
    case LGS_ERR_INVALID_ARG: return "invalid argument";
    case LGS_ERR_CAPACITY: return "pair capacity exceeded";
    case LGS_ERR_BUDGET: return "HBM budget exceeded";
    case LGS_ERR_CUDA: return "CUDA error";
    case LGS_ERR_TIMEOUT: return "device wait timed out";
    case LGS_ERR_DEVICE_CHECK: return "device bounds check failed";
    case LGS_ERR_NO_WORKSPACE: return "no or too small workspace";
    case LGS_ERR_STATE: return "invalid call order";
  }
  return "unknown status";
}

void lgs_constants(float out[16]) {
  for (int i = 0; i < 16; ++i) out[i] = 0.f;
  out[0] = 0.2f;
  out[1] = 9.0f;
  out[2] = 1.0f / 255.0f;
  out[3] = 0.99f;
  out[4] = 1e-4f;
  out[5] = 1e-6f;
  out[6] = 1e-6f;
  out[7] = 1e-6f;
  out[8] = 1e-6f;
  out[9] = 3.0f;
  out[10] = 1.0001f;
  out[11] = 1e-5f;
}

lgs_status lgs_session_create(int device, size_t hbm_budget_bytes, lgs_session* out) {
  if (!out) return fail(LGS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
  if (device < 0 || device >= ndev) return fail(LGS_ERR_INVALID_ARG, "device %d of %d", device, ndev);
  lgs_session s = new (std::nothrow) lgs_session_s;
  if (!s) return fail(LGS_ERR_INVALID_ARG, "out of host memory");
  s->device = device;
  s->budget = hbm_budget_bytes;
  s->desc = new (std::nothrow) Desc;
  s->desc_prev = new (std::nothrow) Desc;
  s->desc_dev = new (std::nothrow) Desc;
  if (!s->desc || !s->desc_prev || !s->desc_dev) {
    delete s->desc;
    delete s->desc_prev;
    delete s->desc_dev;
    delete s;
    return fail(LGS_ERR_INVALID_ARG, "out of host memory");
  }
  memset(s->desc, 0, sizeof(Desc));
  if ((e = cudaSetDevice(device)) != cudaSuccess || (e = cudaMallocHost(&s->h_status, sizeof(Status))) != cudaSuccess) {
    delete s->desc;
    delete s->desc_prev;
    delete s->desc_dev;
    delete s;
    return cuda_fail(e, "session create");
  }
  memset(s->h_status, 0, sizeof(Status));
  if ((e = cudaStreamCreateWithFlags(&s->side.s, cudaStreamNonBlocking)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->side.fork, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventCreateWithFlags(&s->side.join, cudaEventDisableTiming)) != cudaSuccess) {
    lgs_session_destroy(s);
    return cuda_fail(e, "session create");
  }
  *out = s;
  return LGS_OK;
}

lgs_status lgs_session_destroy(lgs_session s) {
  if (!s) return LGS_OK;
  if (s->h_status) {
    cudaSetDevice(s->device);
    cudaFreeHost(s->h_status);
  }
  drop_timing(s);
  if (s->side.s || s->side.fork || s->side.join) {
    cudaSetDevice(s->device);
    if (s->side.fork) cudaEventDestroy(s->side.fork);
    if (s->side.join) cudaEventDestroy(s->side.join);
    if (s->side.s) cudaStreamDestroy(s->side.s);
  }
  if (!s->ev_pool.empty()) {
    cudaSetDevice(s->device);
    for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  }
  delete s->desc;
  delete s->desc_prev;
  delete s->desc_dev;
  delete s;
  return LGS_OK;
}

lgs_status lgs_batch_workspace_size(lgs_session s, const int64_t* map_sizes, int n_maps, const lgs_frame* frames,
                                    const int32_t* frame_map, int n_frames, int64_t max_pairs, size_t* bytes) {
  if (!s || !bytes || !map_sizes) return fail(LGS_ERR_INVALID_ARG, "NULL argument");
  if (max_pairs < 0 || max_pairs >= 0xffffffffll) return fail(LGS_ERR_INVALID_ARG, "max_pairs out of range");
  lgs_status st = check_frames(frames, n_frames);
  if (st != LGS_OK) return st;
  if (n_maps < 1 || n_maps > LGS_MAX_MAPS) return fail(LGS_ERR_INVALID_ARG, "n_maps out of range");
  lgs_surfels tmp[LGS_MAX_MAPS];
  const float dummy[4] __attribute__((aligned(16))) = {0, 0, 0, 0};
  for (int m = 0; m < n_maps; ++m) {
    tmp[m] = lgs_surfels{dummy, dummy, dummy, dummy, map_sizes[m]};
    if (map_sizes[m] < 0) return fail(LGS_ERR_INVALID_ARG, "map %d: negative size", m);
  }
  if (frame_map)
    for (int f = 0; f < n_frames; ++f)
      if (frame_map[f] < 0 || frame_map[f] >= n_maps) return fail(LGS_ERR_INVALID_ARG, "frame_map invalid");
  Desc* d = new (std::nothrow) Desc;
  if (!d) return fail(LGS_ERR_INVALID_ARG, "out of host memory");
  Plan p;
  st = build_desc(tmp, n_maps, frames, frame_map, n_frames, *d, p);
  delete d;
  if (st != LGS_OK) return st;
  *bytes = make_layout(p.n_items, p.n_tiles, max_pairs, p.table_floats, p.tile_pixels).total;
  return LGS_OK;
}

lgs_status lgs_session_workspace_size(lgs_session s, int64_t n_surfels, const lgs_frame* frames, int n_frames,
                                      int64_t max_pairs, size_t* bytes) {
  return lgs_batch_workspace_size(s, &n_surfels, 1, frames, nullptr, n_frames, max_pairs, bytes);
}

lgs_status lgs_session_set_workspace(lgs_session s, void* dev_ptr, size_t bytes) {
  if (!s) return fail(LGS_ERR_INVALID_ARG, "session is NULL");
  if (bytes && !dev_ptr) return fail(LGS_ERR_INVALID_ARG, "workspace pointer is NULL");
  if (reinterpret_cast<uintptr_t>(dev_ptr) & 255) return fail(LGS_ERR_INVALID_ARG, "workspace must be 256-byte aligned");
  if (s->budget && bytes > s->budget)
    return fail(LGS_ERR_BUDGET, "workspace of %zu bytes exceeds the budget of %zu", bytes, s->budget);
  s->ws = dev_ptr;
  s->ws_bytes = bytes;
  s->binned = false;
  s->g13_zero_items = -1;
  s->desc_dev_at = nullptr;   // a new workspace holds no descriptors (even at the old address)
  return LGS_OK;
}

lgs_status lgs_session_set_tuning(lgs_session s, const lgs_tuning* t) {
  if (!s || !t) return fail(LGS_ERR_INVALID_ARG, "NULL argument");
  const auto ok_batch = [](int b, int hi) { return b == 0 || ((b == 64 || b == 128 || b == 256 || b == 512) && b <= hi); };
  if (!ok_batch(t->fwd_batch, 512)) return fail(LGS_ERR_INVALID_ARG, "fwd_batch must be 0, 64, 128, 256 or 512");
  if (!ok_batch(t->bwd_batch, 256)) return fail(LGS_ERR_INVALID_ARG, "bwd_batch must be 0, 64, 128 or 256");
  if (t->group != 1 && t->group != 2 && t->group != 4 && t->group != 16)
    return fail(LGS_ERR_INVALID_ARG, "group must be 1, 2, 4 or 16");
  if (t->persistent != 0 && t->persistent != 1) return fail(LGS_ERR_INVALID_ARG, "persistent must be 0 or 1");
  s->tune = *t;
  return LGS_OK;
}

static lgs_status read_status(lgs_session s) {
  lgs_status st = enter(s);
  if (st != LGS_OK) return st;
  if (!s->ws) return fail(LGS_ERR_NO_WORKSPACE, "no workspace");
  if (!s->binned) return fail(LGS_ERR_STATE, "no lgs_bin_sort yet");
  const WsPtrs w = lgs::ws_ptrs(s->ws, s->lay);
  cudaError_t e = cudaMemcpyAsync(s->h_status, w.st, sizeof(Status), cudaMemcpyDeviceToHost, s->last_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->last_stream);
  if (e != cudaSuccess) return cuda_fail(e, "status read");
  return LGS_OK;
}

lgs_status lgs_session_status(lgs_session s, int64_t* required_pairs) {
  lgs_status st = read_status(s);
  if (st != LGS_OK) return st;
  if (required_pairs) *required_pairs = static_cast<int64_t>(s->h_status->required_pairs);
  if (s->h_status->overflow)
    return fail(LGS_ERR_CAPACITY, "%llu pairs needed, capacity %lld",
                static_cast<unsigned long long>(s->h_status->required_pairs), static_cast<long long>(s->lay.pairs_cap));
  if (s->h_status->timeout) return fail(LGS_ERR_TIMEOUT, "a bounded device wait gave up");
  if (s->h_status->check) return fail(LGS_ERR_DEVICE_CHECK, "device bounds check failed");
  return LGS_OK;
}

// lgs_status_word is the head of the device Status word, copied as bytes
static_assert(offsetof(Status, required_pairs) == offsetof(lgs_status_word, required_pairs), "status layout");
static_assert(offsetof(Status, n_pairs) == offsetof(lgs_status_word, n_pairs), "status layout");
static_assert(offsetof(Status, n_vis) == offsetof(lgs_status_word, n_visible), "status layout");
static_assert(offsetof(Status, overflow) == offsetof(lgs_status_word, overflow), "status layout");
static_assert(offsetof(Status, timeout) == offsetof(lgs_status_word, timeout), "status layout");
static_assert(offsetof(Status, check) == offsetof(lgs_status_word, check), "status layout");

lgs_status lgs_session_status_enqueue(lgs_session s, lgs_status_word* out, void* stream) {
  lgs_status st = enter(s);
  if (st != LGS_OK) return st;
  if (!out) return fail(LGS_ERR_INVALID_ARG, "out is NULL");
  if (!s->ws) return fail(LGS_ERR_NO_WORKSPACE, "no workspace");
  if (!s->binned) return fail(LGS_ERR_STATE, "no lgs_bin_sort yet");
  const WsPtrs w = lgs::ws_ptrs(s->ws, s->lay);
  const cudaError_t e = cudaMemcpyAsync(out, w.st, sizeof(lgs_status_word), cudaMemcpyDeviceToHost,
                                        static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "status copy");
  return LGS_OK;
}

lgs_status lgs_status_of_word(const lgs_status_word* w) {
  if (!w) return fail(LGS_ERR_INVALID_ARG, "word is NULL");
  if (w->overflow)
    return fail(LGS_ERR_CAPACITY, "%llu pairs needed", static_cast<unsigned long long>(w->required_pairs));
  if (w->timeout) return fail(LGS_ERR_TIMEOUT, "a bounded device wait gave up");
  if (w->check) return fail(LGS_ERR_DEVICE_CHECK, "device bounds check failed");
  return LGS_OK;
}

lgs_status lgs_session_pair_count(lgs_session s, int64_t* n_pairs) {
  lgs_status st = read_status(s);
  if (st != LGS_OK) return st;
  if (n_pairs) *n_pairs = static_cast<int64_t>(s->h_status->n_pairs);
  return LGS_OK;
}

lgs_status lgs_session_counters(lgs_session s, int64_t out[8]) {
  if (!out) return fail(LGS_ERR_INVALID_ARG, "out is NULL");
  lgs_status st = read_status(s);
  if (st != LGS_OK) return st;
  out[0] = static_cast<int64_t>(s->h_status->n_pairs);
  out[1] = static_cast<int64_t>(s->h_status->n_vis);
  out[2] = static_cast<int64_t>(s->h_status->evals_fwd);
  out[3] = static_cast<int64_t>(s->h_status->evals_bwd);
  out[4] = static_cast<int64_t>(s->h_status->contrib_fwd);
  out[5] = static_cast<int64_t>(s->h_status->contrib_bwd);
  out[6] = s->launches;
  out[7] = static_cast<int64_t>(s->h_status->alg_fwd);
  return LGS_OK;
}

lgs_status lgs_session_set_timing(lgs_session s, int enable) {
  if (!s) return fail(LGS_ERR_INVALID_ARG, "session is NULL");
  s->timing = enable != 0;
  if (!s->timing) drop_timing(s);
  return LGS_OK;
}

lgs_status lgs_session_kernel_times(lgs_session s, double* ms, int64_t* calls) {
  lgs_status st = enter(s);
  if (st != LGS_OK) return st;
  double t[LGS_TIME_GROUPS] = {0};
  int64_t n[LGS_TIME_GROUPS] = {0};
  cudaError_t err = cudaSuccess;
  for (auto& r : s->timed) {
    float x = 0.f;
    cudaError_t e = cudaEventSynchronize(r.b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&x, r.a, r.b);
    if (e != cudaSuccess) {
      err = e;
      continue;
    }
    t[r.group] += x;
    n[r.group] += 1;
  }
  drop_timing(s);
  if (err != cudaSuccess) return cuda_fail(err, "kernel timing");
  for (int g = 0; g < LGS_TIME_GROUPS; ++g) {
    if (ms) ms[g] = t[g];
    if (calls) calls[g] = n[g];
  }
  return LGS_OK;
}

lgs_status lgs_session_bins(lgs_session s, const uint32_t** tile_of_pair, const uint32_t** item_of_pair,
                            const uint32_t** ranges, const uint32_t** depth_key) {
  if (!s) return fail(LGS_ERR_INVALID_ARG, "session is NULL");
  if (!s->binned) return fail(LGS_ERR_STATE, "no lgs_bin_sort yet");
  const WsPtrs w = lgs::ws_ptrs(s->ws, s->lay);
  if (tile_of_pair) {
    // the binning does not write the tile of each pair; fill it now
    cudaError_t e = lgs::launch_fill_tile_of_pair(w, s->desc->n_tiles, s->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->last_stream);
    if (e != cudaSuccess) return cuda_fail(e, "tile of pair");
    *tile_of_pair = w.ptile;
  }
  if (item_of_pair) *item_of_pair = w.pv;
  if (ranges) *ranges = reinterpret_cast<const uint32_t*>(w.ranges);
  if (depth_key) *depth_key = w.key;
  return LGS_OK;
}

lgs_status lgs_session_read_bins(lgs_session s, uint32_t* tile_of_pair, uint32_t* item_of_pair, uint32_t* ranges,
                                 uint32_t* depth_key, int64_t cap_pairs) {
  lgs_status st = read_status(s);
  if (st != LGS_OK) return st;
  const int64_t np = static_cast<int64_t>(s->h_status->n_pairs);
  if ((tile_of_pair || item_of_pair) && cap_pairs < np)
    return fail(LGS_ERR_CAPACITY, "%lld pairs, buffer holds %lld", static_cast<long long>(np),
                static_cast<long long>(cap_pairs));
  const WsPtrs w = lgs::ws_ptrs(s->ws, s->lay);
  cudaError_t e = cudaSuccess;
  if (tile_of_pair && np) {
    // the binning does not write the tile of each pair; fill it now
    e = lgs::launch_fill_tile_of_pair(w, s->desc->n_tiles, s->last_stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->last_stream);
  }
  if (tile_of_pair && np && e == cudaSuccess)
    e = cudaMemcpy(tile_of_pair, w.ptile, 4 * np, cudaMemcpyDeviceToHost);
  if (item_of_pair && np && e == cudaSuccess)
    e = cudaMemcpy(item_of_pair, w.pv, 4 * np, cudaMemcpyDeviceToHost);
  if (ranges && e == cudaSuccess)
    e = cudaMemcpy(ranges, w.ranges, 8 * static_cast<size_t>(s->desc->n_tiles), cudaMemcpyDeviceToHost);
  if (depth_key && s->desc->n_items && e == cudaSuccess)
    e = cudaMemcpy(depth_key, w.key, 4 * static_cast<size_t>(s->desc->n_items), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "read_bins");
  return LGS_OK;
}

lgs_status lgs_bin_sort_batch(lgs_session s, const lgs_surfels* maps, int n_maps, const lgs_frame* frames,
                              const int32_t* frame_map, int n_frames, void* stream) {
  lgs_status st = enter(s);
  if (st != LGS_OK) return st;
  if ((st = check_frames(frames, n_frames)) != LGS_OK) return st;
  if ((st = check_maps(maps, n_maps, frame_map, n_frames)) != LGS_OK) return st;
  if (!s->ws) return fail(LGS_ERR_NO_WORKSPACE, "no workspace set");
  Plan p;
  memcpy(s->desc_prev, s->desc, sizeof(Desc));
  if ((st = build_desc(maps, n_maps, frames, frame_map, n_frames, *s->desc, p)) != LGS_OK) {
    memcpy(s->desc, s->desc_prev, sizeof(Desc));
    return st;
  }
  keep_call_ptrs(*s->desc, *s->desc_prev);
  const int64_t cap = fit_pairs(s->ws_bytes, p);
  if (cap < 0)
    return fail(LGS_ERR_NO_WORKSPACE, "workspace of %zu bytes too small even without pairs (%zu needed)", s->ws_bytes,
                make_layout(p.n_items, p.n_tiles, 0, p.table_floats, p.tile_pixels).total);
  const Layout L = make_layout(p.n_items, p.n_tiles, cap, p.table_floats, p.tile_pixels);
  const WsPtrs w = lgs::ws_ptrs(s->ws, L);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (s->g13_zero_items != p.n_items || s->g13_zero_off != L.g13) {
    // the per-item gradient buffer must start all-zero (the backward re-zeroes it)
    if ((e = cudaMemsetAsync(w.g13, 0, 64 * static_cast<size_t>(p.n_items > 0 ? p.n_items : 1), cs)) != cudaSuccess)
      return cuda_fail(e, "memset");
    s->g13_zero_items = p.n_items;
    s->g13_zero_off = L.g13;
  }
  if ((e = write_desc(s, *s->desc, w.desc, cs, s->launches)) != cudaSuccess) return cuda_fail(e, "write_desc");
  if ((e = timed(s, LGS_TIME_BIN, cs, [&] { return lgs::launch_bin(L, w, n_frames, p.n_items, p.n_tiles, s->side, cs); })) !=
      cudaSuccess)
    return cuda_fail(e, "bin");
  s->launches += lgs::bin_kernel_count(p.n_tiles);
  s->lay = L;
  s->binned = true;
  s->ckpt_valid = false;
  s->last_stream = cs;
  return LGS_OK;
}

lgs_status lgs_bin_sort(lgs_session s, const lgs_surfels* surfels, const lgs_frame* frames, int n_frames,
                        void* stream) {
  return lgs_bin_sort_batch(s, surfels, 1, frames, nullptr, n_frames, stream);
}

size_t lgs_trackable_scratch_bytes(int64_t n) { return lgs::trackable_scratch_bytes(n); }

lgs_status lgs_trackable_targets(const lgs_surfels* map, const uint8_t* mask, const int32_t* last_kf,
                                 const lgs_track_params* p, void* scratch, size_t scratch_bytes, int32_t* index,
                                 float* mean, float* cov, float* weight, int64_t* count, void* stream) {
  if (!map || !p || !scratch || !count) return fail(LGS_ERR_INVALID_ARG, "NULL argument");
  if (map->n < 0 || map->n > 0x7fffffffll) return fail(LGS_ERR_INVALID_ARG, "n outside [0, 2^31)");
  if (map->n > 0 && (!map->mean || !map->quat || !map->log_scale || !map->opacity_logit || !mask || !last_kf ||
                     !index || !mean || !cov || !weight))
    return fail(LGS_ERR_INVALID_ARG, "NULL array");
  if (!(p->alpha_min > 0.f && p->alpha_min < 1.f)) return fail(LGS_ERR_INVALID_ARG, "alpha_min outside (0, 1)");
  if (!(p->thickness > 0.f && p->eps > 0.f && p->w_max > 0.f))
    return fail(LGS_ERR_INVALID_ARG, "thickness, eps and w_max must be positive");
  if (scratch_bytes < lgs::trackable_scratch_bytes(map->n) || (reinterpret_cast<uintptr_t>(scratch) & 3))
    return fail(LGS_ERR_INVALID_ARG, "scratch too small or not 4-byte aligned");
  const double a = p->alpha_min;
  const float logit_min = static_cast<float>(std::log(a / (1.0 - a)));
  const cudaError_t e = lgs::launch_trackable(*map, mask, last_kf, p->k_min, logit_min, p->thickness, p->eps,
                                              p->w_max, scratch, index, mean, cov, weight, count,
                                              static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? LGS_OK : cuda_fail(e, "trackable targets");
}

void lgs_manage_default_params(lgs_manage_params* p) {
  if (!p) return;
  p->alpha_prune = 0.005f;
  p->alpha_min = 0.1f;
  p->w_l = 0.55f;
  p->w_c = 0.30f;
  p->w_r = 0.15f;
  p->q_res = 0.95f;
  p->eps = 1e-6f;
  p->q_plane = 0.3f;
  p->voxel = 1.0f;
  p->n_passes = 3;
  p->q_cover = 0.5f;
  p->slab = 0.05f;
  p->prune_cap = 0.1f;
  p->q_split = 0.9f;
  p->split_cap = 0.05f;
  p->split_shift = 0.5f;
  p->split_dlog = static_cast<float>(std::log(0.5));
}

size_t lgs_manage_scratch_bytes(int64_t n) { return lgs::manage_scratch_bytes(n < 0 ? 0 : n); }

int32_t lgs_manage_launches(const lgs_manage_params* p) {
  return p && p->n_passes >= 0 && p->n_passes <= 3 ? lgs::manage_kernel_count(p->n_passes) : -1;
}

int64_t lgs_manage_capacity(int64_t n, const lgs_manage_params* p) {
  if (n < 0 || !p || !(p->split_cap >= 0.f && p->split_cap <= 1.f)) return -1;
  return n + static_cast<int64_t>(std::floor(static_cast<double>(p->split_cap) * static_cast<double>(n)));
}

namespace {
bool unit_closed(float v) { return v >= 0.f && v <= 1.f; }
bool unit_open(float v) { return v > 0.f && v < 1.f; }
float logit_f32(float a) { return static_cast<float>(std::log(static_cast<double>(a) / (1.0 - a))); }
}  // namespace

lgs_status lgs_map_manage(const lgs_surfels* map, const float* lam, const float* res, const lgs_manage_params* p,
                          void* scratch, size_t scratch_bytes, float* score, const lgs_surfel_params_out* out,
                          int64_t capacity, int32_t* src, uint8_t* role, int64_t* counts, void* stream) {
  if (!map || !p || !scratch || !out || !counts) return fail(LGS_ERR_INVALID_ARG, "NULL argument");
  if (map->n < 0 || map->n > (1ll << 28)) return fail(LGS_ERR_INVALID_ARG, "n outside [0, 2^28]");
  if (map->n > 0 && (!map->mean || !map->quat || !map->log_scale || !map->opacity_logit || !lam || !res ||
                     !score || !out->mean || !out->quat || !out->log_scale || !out->opacity_logit || !src || !role))
    return fail(LGS_ERR_INVALID_ARG, "NULL array");
  if (!unit_open(p->alpha_prune) || !unit_open(p->alpha_min))
    return fail(LGS_ERR_INVALID_ARG, "alpha_prune and alpha_min must lie in (0, 1)");
  if (!unit_closed(p->q_res) || !unit_closed(p->q_plane) || !unit_closed(p->q_cover) || !unit_closed(p->q_split) ||
      !unit_closed(p->prune_cap) || !unit_closed(p->split_cap))
    return fail(LGS_ERR_INVALID_ARG, "quantiles and caps must lie in [0, 1]");
  if (!(p->eps > 0.f) || !(p->voxel > 0.f) || !std::isfinite(p->voxel) || !(p->slab >= 0.f) ||
      !std::isfinite(p->w_l) || !std::isfinite(p->w_c) || !std::isfinite(p->w_r) ||
      !std::isfinite(p->split_shift) || !std::isfinite(p->split_dlog))
    return fail(LGS_ERR_INVALID_ARG, "eps and voxel must be positive, slab >= 0, weights and split finite");
  if (p->n_passes < 0 || p->n_passes > 3) return fail(LGS_ERR_INVALID_ARG, "n_passes outside [0, 3]");
  if (capacity < lgs_manage_capacity(map->n, p))
    return fail(LGS_ERR_INVALID_ARG, "capacity below n + floor(split_cap n)");
  if (scratch_bytes < lgs::manage_scratch_bytes(map->n) || (reinterpret_cast<uintptr_t>(scratch) & 255))
    return fail(LGS_ERR_INVALID_ARG, "scratch too small or not 256-byte aligned");
  lgs::MgHostParams H;
  H.p = *p;
  H.logit_prune = logit_f32(p->alpha_prune);
  H.logit_min = logit_f32(p->alpha_min);
  const cudaError_t e = lgs::launch_manage(*map, lam, res, H, scratch, score, *out, capacity, src, role, counts,
                                           static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? LGS_OK : cuda_fail(e, "map management");
}

lgs_status lgs_map_gather(const int32_t* src, const uint8_t* role, const int64_t* counts, int64_t capacity,
                          const void* in, void* out, int32_t words_per_row, int32_t zero_children, void* stream) {
  if (!counts || capacity < 0 || words_per_row < 1) return fail(LGS_ERR_INVALID_ARG, "bad counts / capacity / words");
  if (capacity > 0 && (!src || !role || !in || !out)) return fail(LGS_ERR_INVALID_ARG, "NULL array");
  if ((reinterpret_cast<uintptr_t>(in) & 3) || (reinterpret_cast<uintptr_t>(out) & 3))
    return fail(LGS_ERR_INVALID_ARG, "in and out must be 4-byte aligned");
  if (capacity == 0) return LGS_OK;
  const cudaError_t e = lgs::launch_manage_gather(src, role, counts, capacity, in, out, words_per_row, zero_children,
                                                  static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? LGS_OK : cuda_fail(e, "map gather");
}

void lgs_init_default_params(lgs_init_params* p) {
  if (!p) return;
  p->k = 20;
  p->kappa = 0.0184f;
  p->s_min = 1e-3f;
  p->s_max = 1.0f;
  p->r0 = 100.f;
  p->c0 = 0.1f;
  p->eps = 1e-6f;
  p->alpha_min = 0.3f;
  p->alpha_max = 0.9f;
}

size_t lgs_init_scratch_bytes(int64_t n) { return lgs::init_scratch_bytes(n < 0 ? 0 : n); }

int64_t lgs_init_max_points(void) { return lgs::init_max_points(); }

int32_t lgs_init_launches(void) { return lgs::init_launches(); }

lgs_status lgs_keyframe_init(const float* points, int64_t n, const float pose[12], const lgs_init_params* p,
                             void* scratch, size_t scratch_bytes, int32_t* knn, const lgs_surfel_params_out* out,
                             float* lam, float* u, int64_t* pairs, void* stream) {
  if (!pose || !p || !out) return fail(LGS_ERR_INVALID_ARG, "NULL argument");
  if (n < 0 || n > lgs::init_max_points()) return fail(LGS_ERR_INVALID_ARG, "n outside [0, 2^20]");
  if (n > 0 && (!points || !scratch || !knn || !out->mean || !out->quat || !out->log_scale ||
                !out->opacity_logit || !lam || !u))
    return fail(LGS_ERR_INVALID_ARG, "NULL array");
  if (p->k < 3 || p->k > 32 || (n > 0 && p->k > n)) return fail(LGS_ERR_INVALID_ARG, "k outside [3, min(32, n)]");
  if (!(p->kappa > 0.f) || !(p->s_min > 0.f) || !(p->s_max >= p->s_min) || !(p->r0 > 0.f) ||
      !(p->c0 >= 0.f && p->c0 < 1.f) || !(p->eps > 0.f) || !(p->alpha_min > 0.f) ||
      !(p->alpha_max >= p->alpha_min) || !(p->alpha_max < 1.f) || !std::isfinite(p->s_max) ||
      !std::isfinite(p->kappa))
    return fail(LGS_ERR_INVALID_ARG, "initialisation parameters out of range");
  for (int a = 0; a < 12; ++a)
    if (!std::isfinite(pose[a])) return fail(LGS_ERR_INVALID_ARG, "pose not finite");
  if (n > 0 && (scratch_bytes < lgs::init_scratch_bytes(n) || (reinterpret_cast<uintptr_t>(scratch) & 15)))
    return fail(LGS_ERR_INVALID_ARG, "scratch too small or not 16-byte aligned");
  const cudaError_t e = lgs::launch_keyframe_init(points, n, pose, *p, scratch, knn, *out, lam, u, pairs,
                                                  static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? LGS_OK : cuda_fail(e, "keyframe initialisation");
}

lgs_status lgs_render_fwd_loss_batch(lgs_session s, const lgs_surfels* maps, int n_maps, const lgs_frame* frames,
                                     const int32_t* frame_map, int n_frames, const lgs_fwd_out* fwd,
                                     const lgs_target* targets, const lgs_loss_params* params,
                                     const lgs_fwd_grad_out* grads_out, const lgs_surfel_grad* grads,
                                     float* loss_out, void* stream) {
  lgs_status st = enter(s);
  if (st != LGS_OK) return st;
  if (!params) return fail(LGS_ERR_INVALID_ARG, "NULL argument");
  const bool fused = params->lambda_ns == 0.f && s->tune.fwd_batch == 0 && s->tune.group == 16;
  if (!fused) {
    if ((st = lgs_render_fwd_batch(s, maps, n_maps, frames, frame_map, n_frames, fwd, stream)) != LGS_OK) return st;
    return lgs_loss_batch(s, maps, n_maps, frames, frame_map, n_frames, fwd, targets, params, grads_out, grads,
                          loss_out, stream);
  }
  if (!maps || !frames || !targets || !grads_out || !loss_out) return fail(LGS_ERR_INVALID_ARG, "NULL argument");
  if ((st = check_same(s, maps, n_maps, frames, frame_map, n_frames)) != LGS_OK) return st;
  if ((st = check_fwd_out(fwd, n_frames)) != LGS_OK) return st;
  for (int f = 0; f < n_frames; ++f) {
    if (!targets[f].D || !targets[f].N_gicp) return fail(LGS_ERR_INVALID_ARG, "frame %d: NULL target", f);
    if (!grads_out[f].dA || !grads_out[f].dS_t || !grads_out[f].dS_n)
      return fail(LGS_ERR_INVALID_ARG, "frame %d: NULL gradient output", f);
  }
  if (!(params->s_max > 0.f)) return fail(LGS_ERR_INVALID_ARG, "s_max must be positive");
  const bool scale_grad = grads != nullptr;
  if (scale_grad)
    for (int m = 0; m < n_maps; ++m)
      if (maps[m].n > 0 && !grads[m].d_log_scale) return fail(LGS_ERR_INVALID_ARG, "map %d: NULL d_log_scale", m);
  Desc& d = *s->desc;
  set_map_ptrs(d, maps, n_maps);
  for (int f = 0; f < n_frames; ++f) {
    d.f[f].A = fwd[f].A;
    d.f[f].St = fwd[f].S_t;
    d.f[f].Sn = fwd[f].S_n;
    d.f[f].Tf = fwd[f].T_final;
    d.f[f].nc = fwd[f].n_contrib;
    d.f[f].D = targets[f].D;
    d.f[f].Ng = targets[f].N_gicp;
    d.f[f].oA = grads_out[f].dA;
    d.f[f].oSt = grads_out[f].dS_t;
    d.f[f].oSn = grads_out[f].dS_n;
  }
  for (int m = 0; m < n_maps; ++m) d.m[m].d_ls = grads ? grads[m].d_log_scale : nullptr;
  const WsPtrs w = lgs::ws_ptrs(s->ws, s->lay);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = write_desc(s, d, w.desc, cs, s->launches)) != cudaSuccess) return cuda_fail(e, "write_desc");
  if ((e = timed(s, LGS_TIME_LOSS, cs,
                 [&] { return lgs::launch_loss_counts(w, d, *params, scale_grad, cs); })) != cudaSuccess)
    return cuda_fail(e, "loss counts");
  if ((e = timed(s, LGS_TIME_FWD, cs, [&] {
         return lgs::launch_raster_fwd_loss(w, d, w.pv, s->tune.persistent, *params, loss_out, cs);
       })) != cudaSuccess)
    return cuda_fail(e, "raster_fwd_loss");
  s->launches += 3;   // counts and regulariser, per-tile forward, long-list forward (which writes the loss vector)
  s->last_stream = cs;
  s->ckpt_valid = true;
  return LGS_OK;
}

lgs_status lgs_render_fwd_batch(lgs_session s, const lgs_surfels* maps, int n_maps, const lgs_frame* frames,
                                const int32_t* frame_map, int n_frames, const lgs_fwd_out* per_frame, void* stream) {
  lgs_status st = enter(s);
  if (st != LGS_OK) return st;
  if (!maps || !frames) return fail(LGS_ERR_INVALID_ARG, "NULL argument");
  if ((st = check_same(s, maps, n_maps, frames, frame_map, n_frames)) != LGS_OK) return st;
  if ((st = check_fwd_out(per_frame, n_frames)) != LGS_OK) return st;
  Desc& d = *s->desc;
  set_map_ptrs(d, maps, n_maps);
  for (int f = 0; f < n_frames; ++f) {
    d.f[f].A = per_frame[f].A;
    d.f[f].St = per_frame[f].S_t;
    d.f[f].Sn = per_frame[f].S_n;
    d.f[f].Tf = per_frame[f].T_final;
    d.f[f].nc = per_frame[f].n_contrib;
  }
  const WsPtrs w = lgs::ws_ptrs(s->ws, s->lay);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = write_desc(s, d, w.desc, cs, s->launches)) != cudaSuccess) return cuda_fail(e, "write_desc");
  const uint32_t* pv = w.pv;
  if ((e = timed(s, LGS_TIME_FWD, cs, [&] {
         return lgs::launch_raster_fwd(s->lay, w, d, pv, s->tune.fwd_batch, s->tune.group, s->tune.persistent, cs);
       })) != cudaSuccess)
    return cuda_fail(e, "raster_fwd");
  s->launches += 2;   // per-tile and long-list kernels
  s->last_stream = cs;
  s->ckpt_valid = s->tune.fwd_batch == 0 && s->tune.group == 16;
  return LGS_OK;
}

lgs_status lgs_render_fwd(lgs_session s, const lgs_surfels* surfels, const lgs_frame* frames, int n_frames,
                          const lgs_fwd_out* per_frame, void* stream) {
  return lgs_render_fwd_batch(s, surfels, 1, frames, nullptr, n_frames, per_frame, stream);
}

lgs_status lgs_render_bwd_batch(lgs_session s, const lgs_surfels* maps, int n_maps, const lgs_frame* frames,
                                const int32_t* frame_map, int n_frames, const lgs_fwd_out* fwd,
                                const lgs_fwd_grad* upstream, const lgs_surfel_grad* grads, void* stream) {
  lgs_status st = enter(s);
  if (st != LGS_OK) return st;
  if (!maps || !frames || !upstream || !grads) return fail(LGS_ERR_INVALID_ARG, "NULL argument");
  if ((st = check_same(s, maps, n_maps, frames, frame_map, n_frames)) != LGS_OK) return st;
  if ((st = check_fwd_out(fwd, n_frames)) != LGS_OK) return st;
  for (int f = 0; f < n_frames; ++f)
    if (!upstream[f].dA || !upstream[f].dS_t || !upstream[f].dS_n)
      return fail(LGS_ERR_INVALID_ARG, "frame %d: NULL upstream gradient", f);
  for (int m = 0; m < n_maps; ++m)
    if (maps[m].n > 0 && (!grads[m].d_mean || !grads[m].d_quat || !grads[m].d_log_scale || !grads[m].d_opacity_logit))
      return fail(LGS_ERR_INVALID_ARG, "map %d: NULL gradient pointer", m);
  Desc& d = *s->desc;
  set_map_ptrs(d, maps, n_maps);
  for (int f = 0; f < n_frames; ++f) {
    d.f[f].Tf = fwd[f].T_final;
    d.f[f].nc = fwd[f].n_contrib;
    d.f[f].A = fwd[f].A;
    d.f[f].St = fwd[f].S_t;
    d.f[f].Sn = fwd[f].S_n;
    d.f[f].gA = upstream[f].dA;
    d.f[f].gSt = upstream[f].dS_t;
    d.f[f].gSn = upstream[f].dS_n;
  }
  for (int m = 0; m < n_maps; ++m) {
    d.m[m].d_mean = grads[m].d_mean;
    d.m[m].d_quat = grads[m].d_quat;
    d.m[m].d_ls = grads[m].d_log_scale;
    d.m[m].d_logit = grads[m].d_opacity_logit;
  }
  const WsPtrs w = lgs::ws_ptrs(s->ws, s->lay);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = write_desc(s, d, w.desc, cs, s->launches)) != cudaSuccess) return cuda_fail(e, "write_desc");
  const uint32_t* pv = w.pv;
  if ((e = timed(s, LGS_TIME_BWD, cs, [&] {
         const bool chunked = s->ckpt_valid && s->tune.bwd_batch == 0 && s->tune.group == 16;
         return lgs::launch_raster_bwd(s->lay, w, d, pv, s->tune.bwd_batch, s->tune.group, s->tune.persistent,
                                       chunked, cs);
       })) != cudaSuccess)
    return cuda_fail(e, "raster_bwd");
  if ((e = timed(s, LGS_TIME_BWD_CHAIN, cs, [&] { return lgs::launch_preprocess_bwd(s->lay, w, d, cs); })) !=
      cudaSuccess)
    return cuda_fail(e, "preprocess_bwd");
  s->launches += 3;   // per-tile and long-list kernels, chain
  s->last_stream = cs;
  return LGS_OK;
}

lgs_status lgs_render_bwd(lgs_session s, const lgs_surfels* surfels, const lgs_frame* frames, int n_frames,
                          const lgs_fwd_out* fwd, const lgs_fwd_grad* upstream, const lgs_surfel_grad* grad,
                          void* stream) {
  return lgs_render_bwd_batch(s, surfels, 1, frames, nullptr, n_frames, fwd, upstream, grad, stream);
}

lgs_status lgs_loss_batch(lgs_session s, const lgs_surfels* maps, int n_maps, const lgs_frame* frames,
                          const int32_t* frame_map, int n_frames, const lgs_fwd_out* fwd, const lgs_target* targets,
                          const lgs_loss_params* params, const lgs_fwd_grad_out* grads_out,
                          const lgs_surfel_grad* grads, float* loss_out, void* stream) {
  lgs_status st = enter(s);
  if (st != LGS_OK) return st;
  if (!maps || !frames || !targets || !params || !grads_out || !loss_out)
    return fail(LGS_ERR_INVALID_ARG, "NULL argument");
  if ((st = check_same(s, maps, n_maps, frames, frame_map, n_frames)) != LGS_OK) return st;
  if ((st = check_fwd_out(fwd, n_frames)) != LGS_OK) return st;
  for (int f = 0; f < n_frames; ++f) {
    if (!targets[f].D || !targets[f].N_gicp) return fail(LGS_ERR_INVALID_ARG, "frame %d: NULL target", f);
    if (!grads_out[f].dA || !grads_out[f].dS_t || !grads_out[f].dS_n)
      return fail(LGS_ERR_INVALID_ARG, "frame %d: NULL gradient output", f);
  }
  if (!(params->s_max > 0.f)) return fail(LGS_ERR_INVALID_ARG, "s_max must be positive");
  if (!(params->lambda_ns >= 0.f && params->lambda_ns < 1e30f))
    return fail(LGS_ERR_INVALID_ARG, "lambda_ns must be finite and >= 0");
  Desc& d = *s->desc;
  set_map_ptrs(d, maps, n_maps);
  for (int f = 0; f < n_frames; ++f) {
    d.f[f].A = fwd[f].A;
    d.f[f].St = fwd[f].S_t;
    d.f[f].Sn = fwd[f].S_n;
    d.f[f].Tf = fwd[f].T_final;
    d.f[f].nc = fwd[f].n_contrib;
    d.f[f].D = targets[f].D;
    d.f[f].Ng = targets[f].N_gicp;
    d.f[f].oA = grads_out[f].dA;
    d.f[f].oSt = grads_out[f].dS_t;
    d.f[f].oSn = grads_out[f].dS_n;
  }
  for (int m = 0; m < n_maps; ++m) d.m[m].d_ls = grads ? grads[m].d_log_scale : nullptr;
  const bool scale_grad = grads != nullptr;
  if (scale_grad)
    for (int m = 0; m < n_maps; ++m)
      if (maps[m].n > 0 && !grads[m].d_log_scale) return fail(LGS_ERR_INVALID_ARG, "map %d: NULL d_log_scale", m);
  const WsPtrs w = lgs::ws_ptrs(s->ws, s->lay);
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if ((e = write_desc(s, d, w.desc, cs, s->launches)) != cudaSuccess) return cuda_fail(e, "write_desc");
  if ((e = timed(s, LGS_TIME_LOSS, cs,
                 [&] { return lgs::launch_loss(s->lay, w, d, *params, scale_grad, loss_out, cs); })) != cudaSuccess)
    return cuda_fail(e, "loss");
  s->launches += 2;
  s->last_stream = cs;
  return LGS_OK;
}

lgs_status lgs_loss(lgs_session s, const lgs_surfels* surfels, const lgs_frame* frames, int n_frames,
                    const lgs_fwd_out* fwd, const lgs_target* targets, const lgs_loss_params* params,
                    const lgs_fwd_grad_out* grads_out, const lgs_surfel_grad* grad, float* loss_out, void* stream) {
  return lgs_loss_batch(s, surfels, 1, frames, nullptr, n_frames, fwd, targets, params, grads_out, grad, loss_out,
                        stream);
}

lgs_status lgs_image_loss_noalloc(const int32_t* H, const int32_t* W, int n_frames, const lgs_fwd_out* fwd,
                                  const lgs_target* targets, const lgs_loss_params* params,
                                  const lgs_fwd_grad_out* grads_out, float* loss_out, void* stream) {
  static_assert(LGS_NOALLOC_SCRATCH_BYTES >= 0, "scratch size");
  if (!H || !W || !fwd || !targets || !params || !grads_out || !loss_out)
    return fail(LGS_ERR_INVALID_ARG, "NULL argument");
  if (n_frames < 1) return fail(LGS_ERR_INVALID_ARG, "n_frames must be >= 1");
  if (n_frames > LGS_NOALLOC_MAX_FRAMES)
    return fail(LGS_ERR_INVALID_ARG, "n_frames = %d exceeds the static scratch (at most %d frames per call)", n_frames,
                LGS_NOALLOC_MAX_FRAMES);
  if (params->lambda_ns != 0.f)
    return fail(LGS_ERR_INVALID_ARG, "lambda_ns must be 0: this call has no frame geometry for N_surf");
  if (lgs::noalloc_scratch_bytes() != static_cast<size_t>(LGS_NOALLOC_SCRATCH_BYTES))
    return fail(LGS_ERR_INVALID_ARG, "scratch size mismatch between header and library");
  for (int f = 0; f < n_frames; ++f) {
    if (H[f] < 1 || W[f] < 1 || static_cast<int64_t>(H[f]) * W[f] >= (1ll << 31))
      return fail(LGS_ERR_INVALID_ARG, "frame %d: bad size %d x %d", f, H[f], W[f]);
    if (!fwd[f].A || !fwd[f].S_t || !fwd[f].S_n || !targets[f].D || !targets[f].N_gicp || !grads_out[f].dA ||
        !grads_out[f].dS_t || !grads_out[f].dS_n)
      return fail(LGS_ERR_INVALID_ARG, "frame %d: NULL plane", f);
  }
  void* scratch = nullptr;
  cudaError_t e = lgs::noalloc_scratch(&scratch);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the loss scratch");
  e = lgs::launch_image_loss_noalloc(scratch, n_frames, H, W, fwd, targets, *params, grads_out, loss_out,
                                     static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "image loss");
  return LGS_OK;
}

lgs_status lgs_adam_step_batch(const lgs_adam_map* maps, int n_maps, float beta1, float beta2, float eps,
                               int zero_grad, void* stream) {
  if (!maps || n_maps < 1 || n_maps > LGS_MAX_MAPS)
    return fail(LGS_ERR_INVALID_ARG, "n_maps must be 1..%d", LGS_MAX_MAPS);
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f))
    return fail(LGS_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
  for (int k = 0; k < n_maps; ++k) {
    const lgs_adam_map& M = maps[k];
    if (M.n < 0 || M.step < 1) return fail(LGS_ERR_INVALID_ARG, "map %d: bad size or step", k);
    if (M.n > 0 && (!M.mean || !M.quat || !M.log_scale || !M.logit || !M.m_state || !M.v_state ||
                    !M.grad.d_mean || !M.grad.d_quat || !M.grad.d_log_scale || !M.grad.d_opacity_logit))
      return fail(LGS_ERR_INVALID_ARG, "map %d: NULL pointer", k);
  }
  const cudaError_t e = lgs::launch_adam_batch(maps, n_maps, beta1, beta2, eps, zero_grad,
                                               static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "adam_batch");
  return LGS_OK;
}

lgs_status lgs_adam_step(float* mean, float* quat, float* log_scale, float* logit, const lgs_surfel_grad* grad,
                         float* m_state, float* v_state, int64_t n, int64_t step, const float lr[4], float beta1,
                         float beta2, float eps, int zero_grad, void* stream) {
  if (n < 0 || step < 1 || !lr || !grad) return fail(LGS_ERR_INVALID_ARG, "bad Adam arguments");
  if (n == 0) return LGS_OK;
  if (!mean || !quat || !log_scale || !logit || !m_state || !v_state || !grad->d_mean || !grad->d_quat ||
      !grad->d_log_scale || !grad->d_opacity_logit)
    return fail(LGS_ERR_INVALID_ARG, "NULL Adam pointer");
  if (!(beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f && beta2 < 1.f && eps >= 0.f))
    return fail(LGS_ERR_INVALID_ARG, "Adam hyper-parameters out of range");
  float* p[4] = {mean, quat, log_scale, logit};
  float* g[4] = {grad->d_mean, grad->d_quat, grad->d_log_scale, grad->d_opacity_logit};
  const int64_t cnt[4] = {3 * n, 4 * n, 2 * n, n};
  float* m[4] = {m_state, m_state + 3 * n, m_state + 7 * n, m_state + 9 * n};
  float* v[4] = {v_state, v_state + 3 * n, v_state + 7 * n, v_state + 9 * n};
  cudaError_t e = lgs::launch_adam(p, g, m, v, cnt, step, lr, beta1, beta2, eps, zero_grad,
                                   static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "adam");
  return LGS_OK;
}

}  // extern "C"
