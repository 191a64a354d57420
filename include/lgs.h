/*
 * lgs.h -- C ABI of the GB300 differentiable spherical rasterizer of 2D
 * Gaussian surfels into LiDAR range images.
 *
 * The operation (paper Sec. 3.1 "Map Representation" and Sec. 3.4 "Map
 * Optimization"): a map of 2D Gaussian surfels (mean mu, orientation q,
 * in-plane log-scale s~, opacity alpha) is rendered under the spherical
 * projection of a spinning LiDAR into a range image, giving per pixel the
 * accumulated opacity A, the weighted range sum S_t and the weighted normal
 * sum S_n, from which the expected depth D = S_t/(A+1e-6) and the normal
 * N = S_n/|S_n| follow; the mapping losses (Eqs. depthloss, normalloss,
 * scaleloss, totalloss) compare them with the scan and are differentiated
 * back to every surfel parameter.
 *
 * Definitions shared by every entry point
 *  - Frame: H x W pixels, row 0 at the top elevation elev_max, pixel-centre
 *    elevation elev_max - (r + 1/2)(elev_max - elev_min)/H; azimuth
 *    (c + 1/2) 2 pi / W counter-clockwise from the sensor +x axis, full
 *    360 degrees.  pose = sensor-to-world [R | t], 3 x 4 row-major; rays are
 *    unit vectors from the sensor origin.
 *  - Tiles: tile_h x tile_w pixels (the last row/column of tiles may be
 *    ragged); tile_h * tile_w is a multiple of 32 and at most 256 (one CUDA
 *    thread per pixel).  Every frame of one call uses the same tile shape.
 *  - Surfel i: centre mean[3i..3i+2] (world), quaternion quat[4i..4i+3]
 *    = (w,x,y,z) (normalised inside), log_scale[2i..2i+1] (scales
 *    exp(log_scale), tangent axes R(q)e0 and R(q)e1), opacity
 *    sigmoid(opacity_logit[i]); normal R(q)e2.
 *  - Per pixel, the surfels listed for its tile are visited in ascending
 *    (binary32 |mu_sensor| bit pattern, surfel index); each is intersected as
 *    a plane, t = (n.mu)/(n.d), skipped if |n.d| < 1e-6, t <= 0.2 m,
 *    u^2+v^2 > 9 or a = min(alpha exp(-(u^2+v^2)/2), 0.99) < 1/255, and
 *    composited front to back (w = a T, T *= 1-a) until T (1-a) < 1e-4, in
 *    which case that surfel is not composited and the pixel stops.
 *  - Binning (which surfels a tile lists) is a conservative bounding-cone
 *    test in specified binary32 arithmetic; the sorted lists are bit-exact
 *    reproducible (see the design notes for the exact definition).
 *
 * Conventions
 *  - All array pointers are DEVICE pointers owned by the caller, FP32 unless
 *    stated, densely packed.  The library never frees them.
 *  - Per-frame image planes are [H*W] row-major; S_n and the normal targets
 *    are planar [3][H*W].
 *  - A session owns descriptors and a small pinned status buffer only;
 *    all scratch lives in a caller-provided device workspace
 *    (lgs_*_workspace_size / lgs_session_set_workspace).
 *  - Calls enqueue work on `stream` (a cudaStream_t; NULL = legacy default
 *    stream) and return without synchronising, except
 *    lgs_session_status / lgs_session_pair_count, which synchronise.
 *  - Argument errors are returned at once and enqueue nothing.  Conditions
 *    found on the device (pair capacity exceeded, a bounded wait that gave
 *    up, a bounds check in checked builds) are recorded in a device status
 *    word and reported by lgs_session_status.
 *  - A session is used from one host thread and one stream at a time.
 *  - lgs_render_bwd needs the bins of the lgs_bin_sort that preceded the
 *    matching lgs_render_fwd: they stay in the workspace until the next
 *    lgs_bin_sort on the same session.
 *  - No C++ exception crosses this interface.
 */
#ifndef LGS_H
#define LGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define LGS_API __attribute__((visibility("default")))
#else
#define LGS_API
#endif

typedef struct lgs_session_s* lgs_session;

typedef enum {
    LGS_OK = 0,
    LGS_ERR_INVALID_ARG = 1,   /* bad pointer, size, tile shape, elevation range ... */
    LGS_ERR_CAPACITY = 2,      /* more (tile, surfel) pairs than the workspace holds */
    LGS_ERR_BUDGET = 3,        /* workspace larger than the session's HBM budget */
    LGS_ERR_CUDA = 4,          /* a CUDA runtime call failed */
    LGS_ERR_TIMEOUT = 5,       /* a bounded device-side wait gave up */
    LGS_ERR_DEVICE_CHECK = 6,  /* a device-side bounds check failed */
    LGS_ERR_NO_WORKSPACE = 7,  /* no (or too small a) workspace is set */
    LGS_ERR_STATE = 8          /* call order violated (e.g. bwd without bins) */
} lgs_status;

/* Limits of one call. */
#define LGS_MAX_FRAMES 64
#define LGS_MAX_MAPS 64
#define LGS_MAX_TILE_PIXELS 256

typedef struct {
    int32_t H, W, tile_h, tile_w;
    float elev_min, elev_max;   /* radians, -pi/2 <= elev_min < elev_max <= pi/2 */
    float pose[12];             /* sensor -> world [R | t], row-major 3 x 4 */
} lgs_frame;

typedef struct {
    const float* mean;          /* [n,3] */
    const float* quat;          /* [n,4] (w,x,y,z) */
    const float* log_scale;     /* [n,2] */
    const float* opacity_logit; /* [n]   */
    int64_t n;
} lgs_surfels;

/* Forward outputs of one frame (device, caller-owned, overwritten). */
typedef struct {
    float* A;          /* [H*W]   accumulated opacity  sum_k w_k            */
    float* S_t;        /* [H*W]   sum_k w_k t_k (range along the unit ray)   */
    float* S_n;        /* [3,H*W] sum_k w_k n'_k, n' = -sign(n.d) n          */
    float* T_final;    /* [H*W]   transmittance after the last contributor   */
    int32_t* n_contrib;/* [H*W]   list position of the last contributor + 1  */
} lgs_fwd_out;

/* Upstream gradients dL/d(A, S_t, S_n) of one frame (device). */
typedef struct {
    const float* dA;   /* [H*W]   */
    const float* dS_t; /* [H*W]   */
    const float* dS_n; /* [3,H*W] */
} lgs_fwd_grad;

/* Gradients w.r.t. the raw surfel parameters (device); ACCUMULATED (+=). */
typedef struct {
    float* d_mean;          /* [n,3] */
    float* d_quat;          /* [n,4] */
    float* d_log_scale;     /* [n,2] */
    float* d_opacity_logit; /* [n]   */
} lgs_surfel_grad;

/* Writable per-frame gradient planes (device), filled by lgs_loss. */
typedef struct {
    float* dA;         /* [H*W]   */
    float* dS_t;       /* [H*W]   */
    float* dS_n;       /* [3,H*W] */
} lgs_fwd_grad_out;

/* Measured scan of one frame (device). */
typedef struct {
    const float* D;      /* [H*W] range, 0 = no return (mask M_D = [D > 0]) */
    const float* N_gicp; /* [3,H*W] tracking normals, zero = undefined       */
} lgs_target;

/* Loss weights (paper Sec. 4.1 implementation details). */
typedef struct {
    float lambda_alpha;  /* 0.1  */
    float lambda_n;      /* 1.0  */
    float lambda_ng;     /* 0.05 */
    float lambda_s;      /* 10.0 */
    float s_max;         /* 1.0 m, threshold of the scale regulariser */
    float lambda_ns;     /* 0.01 once densification has begun (Sec. 3.4), 0 = the
                            N_surf term is off; must be >= 0 */
} lgs_loss_params;

/* Image terms per frame in a loss vector: L_depth, L_alpha, L_ng, L_ns. */
#define LGS_LOSS_TERMS 4

/* Tuning knobs of the compositing kernels (results do not depend on them). */
typedef struct {
    int32_t fwd_batch;   /* forward compositing: 0 = every warp walks the tile list on
                            its own, 32 entries per ballot; 64, 128, 256, 512 = the
                            CTA stages that many records per shared-memory batch */
    int32_t bwd_batch;   /* backward: the same choice (0, 64, 128 or 256) */
    int32_t group;       /* warp walk only: 16 = the records of a chunk's hits are
                            staged in the warp's own shared memory and read back by
                            broadcast; 1, 2 or 4 = records read through L1, that many
                            hits fetched and evaluated together */
    int32_t persistent;  /* 1: persistent CTAs claim tiles through an atomic counter */
} lgs_tuning;

/* ---- sessions and workspace -------------------------------------------- */

/* Create a session on `device` that will refuse workspaces larger than
 * hbm_budget_bytes (0 = no limit).  *out receives the handle. */
LGS_API lgs_status lgs_session_create(int device, size_t hbm_budget_bytes, lgs_session* out);

/* Destroy a session (does not free the caller's workspace). */
LGS_API lgs_status lgs_session_destroy(lgs_session s);

/* Bytes of workspace needed to bin and render `n_frames` frames of one map
 * of n_surfels surfels with room for max_pairs (tile, surfel) pairs. */
LGS_API lgs_status lgs_session_workspace_size(lgs_session s, int64_t n_surfels, const lgs_frame* frames,
                                      int n_frames, int64_t max_pairs, size_t* bytes);

/* Same for a batch: frame f renders map frame_map[f] (0 <= . < n_maps). */
LGS_API lgs_status lgs_batch_workspace_size(lgs_session s, const int64_t* map_sizes, int n_maps,
                                    const lgs_frame* frames, const int32_t* frame_map, int n_frames,
                                    int64_t max_pairs, size_t* bytes);

/* Hand the session a device workspace (256-byte aligned) of `bytes` bytes.
 * LGS_ERR_BUDGET if bytes exceed the session budget. */
LGS_API lgs_status lgs_session_set_workspace(lgs_session s, void* dev_ptr, size_t bytes);

/* Synchronise with the session's last stream and read the device status:
 * LGS_OK, LGS_ERR_CAPACITY (then *required_pairs is the number needed),
 * LGS_ERR_TIMEOUT or LGS_ERR_DEVICE_CHECK.  required_pairs may be NULL. */
LGS_API lgs_status lgs_session_status(lgs_session s, int64_t* required_pairs);

/* The head of the device status word, as lgs_session_status_enqueue copies
 * it: pairs the last lgs_bin_sort needed and emitted, items covering a tile,
 * and the error flags (nonzero: capacity overflow, a bounded wait that gave
 * up, a failed device bounds check). */
typedef struct {
    uint64_t required_pairs, n_pairs;
    uint32_t n_visible, overflow, timeout, check;
} lgs_status_word;

/* Non-blocking form of lgs_session_status: enqueue on `stream` a copy of the
 * status word as it stands when the stream reaches this point (after the
 * session's last lgs_bin_sort and the calls after it) into *out, which must
 * be pinned host memory of sizeof(lgs_status_word) bytes.  No host
 * synchronisation: the caller decodes *out with lgs_status_of_word once an
 * event recorded after this call has completed (a serving loop keeps
 * several steps in flight this way).  LGS_ERR_STATE before any
 * lgs_bin_sort. */
LGS_API lgs_status lgs_session_status_enqueue(lgs_session s, lgs_status_word* out, void* stream);

/* The status a copied word reports: LGS_OK, LGS_ERR_CAPACITY,
 * LGS_ERR_TIMEOUT or LGS_ERR_DEVICE_CHECK (LGS_ERR_INVALID_ARG if w is
 * NULL).  Pure host function. */
LGS_API lgs_status lgs_status_of_word(const lgs_status_word* w);

/* Synchronise and return the pair count of the last bin_sort. */
LGS_API lgs_status lgs_session_pair_count(lgs_session s, int64_t* n_pairs);

/* Synchronise and read the counters of the last bin_sort: out[0] pairs,
 * out[1] items covering at least one tile, out[2] ray/surfel evaluations of
 * the forward calls since that bin_sort, out[3] the same for the backward,
 * out[4] composited pairs of the forward calls, out[5] valid pairs the
 * backward re-evaluated, out[6] CUDA kernels this session has enqueued since
 * it was created, out[7] the forward's algorithmic evaluations: per pixel,
 * the tile-list entries up to and including its stop point (the whole list
 * when it never stops), summed over the forward calls since that bin_sort. */
LGS_API lgs_status lgs_session_counters(lgs_session s, int64_t out[8]);

/* Kernel groups timed by lgs_session_set_timing. */
enum {
    LGS_TIME_DESC = 0,       /* descriptor copies */
    LGS_TIME_BIN = 1,        /* lgs_bin_sort: preprocess, bucket scan, emission, per-tile sort */
    LGS_TIME_FWD = 2,        /* forward compositing kernel */
    LGS_TIME_LOSS = 3,       /* loss kernels */
    LGS_TIME_BWD = 4,        /* backward compositing kernel */
    LGS_TIME_BWD_CHAIN = 5,  /* chain of the per-item moments to the surfel parameters */
    LGS_TIME_GROUPS = 8
};

/* enable != 0: from now on, every kernel group this session enqueues outside
 * a stream capture is bracketed by CUDA events on its stream (a few
 * microseconds of overhead per call).  enable == 0 stops and discards. */
LGS_API lgs_status lgs_session_set_timing(lgs_session s, int enable);

/* Synchronise on the recorded events and return, per group, the summed
 * device milliseconds and the number of timed calls since the last read
 * (then forget them).  Arrays of LGS_TIME_GROUPS entries; either may be NULL. */
LGS_API lgs_status lgs_session_kernel_times(lgs_session s, double* ms, int64_t* calls);

/* Device pointers into the workspace describing the last bin_sort, valid
 * until the next one: tile_of_pair[P] (global tile id, frame f's tiles start
 * at the sum of the tile counts of frames < f), item_of_pair[P] (frame-major
 * item f*n + surfel for one map), ranges[2*T] (start, end per global tile;
 * (0, 0) for a tile without pairs),
 * depth_key[items] (binary32 bits of |mu_sensor|).  The binning itself does
 * not store the tile of each pair (its ranges give it): when tile_of_pair is
 * requested, this call fills it on the session's last stream and
 * synchronises with that stream. */
LGS_API lgs_status lgs_session_bins(lgs_session s, const uint32_t** tile_of_pair, const uint32_t** item_of_pair,
                            const uint32_t** ranges, const uint32_t** depth_key);

/* Synchronise and copy the last bin_sort's lists to HOST buffers (any may be
 * NULL): tile_of_pair / item_of_pair [n_pairs] (only if cap_pairs >= n_pairs,
 * else LGS_ERR_CAPACITY), ranges [2 * total tiles], depth_key [items]. */
LGS_API lgs_status lgs_session_read_bins(lgs_session s, uint32_t* tile_of_pair, uint32_t* item_of_pair,
                                 uint32_t* ranges, uint32_t* depth_key, int64_t cap_pairs);

/* ---- the hot path -------------------------------------------------------- */

/* Bin and sort: per frame, transform the surfels to the sensor frame, list
 * each surfel under every angular tile its bounding cone meets (azimuth seam
 * handled by circular column ranges), and sort each tile's list by
 * (depth key, surfel index) (paper Sec. 3.1: render under the spherical
 * projection; the sort realises front-to-back order). */
LGS_API lgs_status lgs_bin_sort(lgs_session s, const lgs_surfels* surfels, const lgs_frame* frames,
                        int n_frames, void* stream);

/* Forward compositing of every frame of the last lgs_bin_sort (Sec. 3.4:
 * rasterise the map into (D, A, N)).  per_frame[f] receives frame f. */
LGS_API lgs_status lgs_render_fwd(lgs_session s, const lgs_surfels* surfels, const lgs_frame* frames,
                          int n_frames, const lgs_fwd_out* per_frame, void* stream);

/* Backward: given the forward outputs and upstream gradients of every frame,
 * ACCUMULATE dL/d(mean, quat, log_scale, logit) into *grad (Sec. 3.4:
 * optimise Theta = {mu, q, s~, alpha}).  The forward is recomputed per tile
 * in reverse order; no per-pixel surfel lists are stored. */
LGS_API lgs_status lgs_render_bwd(lgs_session s, const lgs_surfels* surfels, const lgs_frame* frames,
                          int n_frames, const lgs_fwd_out* fwd, const lgs_fwd_grad* upstream,
                          const lgs_surfel_grad* grad, void* stream);

/* Mapping loss of a window of frames (Eqs. depthloss, normalloss, scaleloss,
 * totalloss): L = (1/F) sum_f [L_depth + la L_alpha + ln (lng L_ng + lns L_ns)]_f
 * + ls L_scale.  L_ns, the second term of Eq. normalloss, compares the
 * rendered normal with N_surf, the normal of the rendered depth: with X the
 * rendered range of a pixel back-projected along its ray, N_surf =
 * normalise((X(r, c+1) - X(r, c)) x (X(r+1, c) - X(r, c))), columns wrapping
 * at 2 pi; it is taken at pixels with a return and a rendered surface (A > 0)
 * there and at both neighbours (not on the last row), averaged over the
 * pixels with a return, and
 * differentiated through both normals (into S_n of the pixel and S_t, A of
 * the three pixels).  Writes dL/d(A, S_t, S_n) per frame into grads_out[f]
 * (overwritten), adds ls dL_scale/d(log
 * scale) into grad->d_log_scale (if grad != NULL), and stores on the device
 * loss_out[0] = L, loss_out[1 + 4f .. 4 + 4f] = (L_depth, L_alpha, L_ng,
 * L_ns) of frame f, and loss_out[1 + 4 n_frames + m] = the part of L of map m
 * (loss_out has 1 + LGS_LOSS_TERMS n_frames + n_maps floats; one map for
 * lgs_loss).
 * With several frames per map the image terms of that map are averaged over
 * its frames, so a map's gradient does not depend on the other maps of a
 * batch. */
LGS_API lgs_status lgs_loss(lgs_session s, const lgs_surfels* surfels, const lgs_frame* frames, int n_frames,
                    const lgs_fwd_out* fwd, const lgs_target* targets, const lgs_loss_params* params,
                    const lgs_fwd_grad_out* grads_out, const lgs_surfel_grad* grad, float* loss_out,
                    void* stream);

/* Batched forms: maps[m] for m < n_maps; frame f renders maps[frame_map[f]];
 * grads[m] receives map m's gradient. */
LGS_API lgs_status lgs_bin_sort_batch(lgs_session s, const lgs_surfels* maps, int n_maps,
                              const lgs_frame* frames, const int32_t* frame_map, int n_frames,
                              void* stream);
LGS_API lgs_status lgs_render_fwd_batch(lgs_session s, const lgs_surfels* maps, int n_maps,
                                const lgs_frame* frames, const int32_t* frame_map, int n_frames,
                                const lgs_fwd_out* per_frame, void* stream);
LGS_API lgs_status lgs_render_bwd_batch(lgs_session s, const lgs_surfels* maps, int n_maps,
                                const lgs_frame* frames, const int32_t* frame_map, int n_frames,
                                const lgs_fwd_out* fwd, const lgs_fwd_grad* upstream,
                                const lgs_surfel_grad* grads, void* stream);
LGS_API lgs_status lgs_loss_batch(lgs_session s, const lgs_surfels* maps, int n_maps, const lgs_frame* frames,
                          const int32_t* frame_map, int n_frames, const lgs_fwd_out* fwd,
                          const lgs_target* targets, const lgs_loss_params* params,
                          const lgs_fwd_grad_out* grads_out, const lgs_surfel_grad* grads,
                          float* loss_out, void* stream);

/* Forward and mapping loss in one call (Secs. 3.1 and 3.4: the rendering of
 * Eq. 2 and Eqs. depthloss, normalloss, scaleloss, totalloss): the outputs of
 * lgs_render_fwd_batch and of lgs_loss_batch, bit for bit, with the image
 * terms computed in the compositing kernel's epilogue from the values it
 * just composited (no second pass over the planes).  Arguments as in those
 * two calls (fwd receives the forward planes).  The fused path runs with the
 * shared-memory forward (fwd_batch 0, group 16) and without the N_surf term
 * (lambda_ns == 0; that term needs neighbouring tiles' depths); otherwise the
 * call runs the forward and then the loss. */
LGS_API lgs_status lgs_render_fwd_loss_batch(lgs_session s, const lgs_surfels* maps, int n_maps,
                                     const lgs_frame* frames, const int32_t* frame_map, int n_frames,
                                     const lgs_fwd_out* fwd, const lgs_target* targets,
                                     const lgs_loss_params* params, const lgs_fwd_grad_out* grads_out,
                                     const lgs_surfel_grad* grads, float* loss_out, void* stream);

/* ---- tracking-side targets (Sec. 3.2) -------------------------------------
 * The trackable subset of the map (Eq. trackable_select) and, for each member,
 * what covariance-weighted G-ICP needs from it without any map-side k-NN:
 * the mean, the surfel-like target covariance R(q) diag(s_x^2, s_y^2, t^2)
 * R(q)^T (q normalised; t = thickness along the normal) and the geometry
 * weight w = min(1 / (kappa_bar + eps), w_max) (Eqs. anisotropy,
 * anisotropy_norm, weight_func) with kappa = s_0 / (s_1 + eps) of the sorted
 * in-plane scales, normalised over the selected set by its minimum and
 * maximum (kappa_bar = 0 when they coincide). */
typedef struct {
    int32_t k_min;       /* selected: mask != 0, last_kf >= k_min, ... */
    float alpha_min;     /* ... and opacity >= alpha_min, in (0, 1); decided in
                            binary32 as logit >= log(alpha_min / (1 - alpha_min)) */
    float thickness;     /* t, metres, > 0 (0.01 is the library's reading) */
    float eps;           /* > 0 (1e-6) */
    float w_max;         /* > 0 (10, as the paper sets omega_max) */
} lgs_track_params;

/* Bytes of device scratch lgs_trackable_targets needs for n surfels. */
LGS_API size_t lgs_trackable_scratch_bytes(int64_t n);

/* map: one surfel set (device, as lgs_surfels); mask [n] uint8 and last_kf
 * [n] int32: device arrays (the trackable mask m_i and the last keyframe that
 * updated the surfel, k_i).  Writes, in ascending surfel index, the selected
 * surfels' index [count] int32, mean [count][3], cov [count][6] (xx, xy, xz,
 * yy, yz, zz) and weight [count], all device arrays with room for n entries
 * (caller-owned), and count (one int64 on the device).  scratch: device
 * memory of lgs_trackable_scratch_bytes(n) bytes, 4-byte aligned, its
 * contents irrelevant.  Enqueues on stream without a host sync; argument
 * errors return LGS_ERR_INVALID_ARG. */
LGS_API lgs_status lgs_trackable_targets(const lgs_surfels* map, const uint8_t* mask, const int32_t* last_kf,
                                 const lgs_track_params* params, void* scratch, size_t scratch_bytes,
                                 int32_t* index, float* mean, float* cov, float* weight, int64_t* count,
                                 void* stream);

/* ---- map management (Sec. 3.3 control score, Sec. 3.5 map budget control) --
 * One map-management step over one surfel map, on the device:
 *  1. control score (Eq. controlscore) c_i = clip(w_l lin_i + w_c curv~_i +
 *     w_r res~_i, 0, 1) from the tracking covariance's eigenvalues
 *     lambda_i (any order; sorted descending inside): lin = (l0 - l1) /
 *     (l0 + eps), curv = l2 / (l0 + l1 + l2 + eps), curv~ = min(3 curv, 1)
 *     (curv spans [0, 1/3]); the residual normalised by its own quantile,
 *     res~ = min(res / (Q_{q_res}(res) + eps), 1);
 *  2. opacity prune: alpha < alpha_prune is removed (the Table 4 baseline);
 *  3. n_passes passes of planar cover-and-prune over the planes xy, yz, zx:
 *     candidates are survivors with c <= Q_{q_plane}(survivors' c) and
 *     alpha >= alpha_min; grouped by the 2D voxel (floor(mu_a / voxel),
 *     floor(mu_b / voxel)) of the pass's plane; the representative is the
 *     group's largest alpha (ties: lowest index); the other candidates within
 *     |n_r . (mu_j - mu_r)| <= slab are members, with cover radius
 *     u^2 + v^2 in the representative's tangent frame scaled by its scales;
 *     the cover region is the representative's ellipse enlarged to include a
 *     q_cover fraction of the members (the ceil(q_cover m) closest, ties
 *     included), whose members are removed; at most floor(prune_cap x
 *     survivors) per pass, the lowest c first (then lowest index);
 *  4. structure-aware split: survivors with c >= Q_{q_split}(survivors' c)
 *     and alpha >= alpha_min, at most floor(split_cap x survivors), the
 *     highest c first (then lowest index); each is replaced by two children
 *     at mu +- split_shift s_0 a_i along a_i = R(q_i) e0 with
 *     log-scale s~_0 + split_dlog (orientation, s~_1 and opacity kept).
 * Quantiles are the lower order statistic sorted[floor(q (n - 1))].  Every
 * decision is made in binary32 with correctly rounded operations in a fixed
 * order and the scales through a fixed polynomial exponential, so the result
 * is the same on every run and launch shape. */
typedef struct {
    float alpha_prune;   /* in (0, 1); 0.005 (the paper gives no value) */
    float alpha_min;     /* in (0, 1); 0.1 */
    float w_l, w_c, w_r; /* 0.55, 0.30, 0.15 (the paper's values) */
    float q_res;         /* in [0, 1]; 0.95 */
    float eps;           /* > 0; 1e-6 */
    float q_plane;       /* in [0, 1]; 0.3 */
    float voxel;         /* > 0, metres; 1.0 */
    int32_t n_passes;    /* 0..3; 3 */
    float q_cover;       /* in [0, 1]; 0.5 */
    float slab;          /* >= 0, metres; 0.05 */
    float prune_cap;     /* in [0, 1]; 0.1 */
    float q_split;       /* in [0, 1]; 0.9 */
    float split_cap;     /* in [0, 1]; 0.05 */
    float split_shift;   /* finite; 0.5 */
    float split_dlog;    /* finite; log 0.5 */
} lgs_manage_params;

/* Writable surfel parameters (device, layouts as lgs_surfels). */
typedef struct {
    float *mean, *quat, *log_scale, *opacity_logit;
} lgs_surfel_params_out;

/* The defaults listed above. */
LGS_API void lgs_manage_default_params(lgs_manage_params* p);
/* Bytes of device scratch lgs_map_manage needs for n surfels. */
LGS_API size_t lgs_manage_scratch_bytes(int64_t n);
/* Kernel launches one lgs_map_manage call makes (for launch accounting). */
LGS_API int32_t lgs_manage_launches(const lgs_manage_params* p);
/* Rows the new map may need: n + floor(split_cap n). */
LGS_API int64_t lgs_manage_capacity(int64_t n, const lgs_manage_params* p);

/* map: the surfels (device, n <= 2^28); lam [n][3] and res [n]: device
 * arrays of the tracking covariance's eigenvalues (>= 0) and G-ICP residuals
 * (>= 0), finite.  scratch: lgs_manage_scratch_bytes(n) bytes of device
 * memory, 256-byte aligned, contents irrelevant.  Writes score [n] (c_i),
 * the new map into out (rows [0, n_out), capacity rows of room), src
 * [capacity] int32 (the parent of each new row), role [capacity] uint8 (0
 * copy, 1 child at +shift, 2 child at -shift) and counts [6] int64 (n_out,
 * opacity-pruned, pruned by passes 0, 1, 2, split), all device and
 * caller-owned; out must not overlap map.  Enqueues on stream without a host
 * sync; argument errors return LGS_ERR_INVALID_ARG before anything is
 * enqueued. */
LGS_API lgs_status lgs_map_manage(const lgs_surfels* map, const float* lam, const float* res,
                                  const lgs_manage_params* params, void* scratch, size_t scratch_bytes,
                                  float* score, const lgs_surfel_params_out* out, int64_t capacity, int32_t* src,
                                  uint8_t* role, int64_t* counts, void* stream);

/* Carries a per-surfel array (words_per_row 32-bit words a row, e.g. Adam
 * moments) over to the new map: out[j] = in[src[j]] for j < counts[0]
 * (clamped to capacity); rows of children are zero when zero_children != 0.
 * src, role and counts as written by lgs_map_manage; in and out device,
 * 4-byte aligned, not overlapping. */
LGS_API lgs_status lgs_map_gather(const int32_t* src, const uint8_t* role, const int64_t* counts, int64_t capacity,
                                  const void* in, void* out, int32_t words_per_row, int32_t zero_children,
                                  void* stream);

/* ---- keyframe initialisation (Sec. 3.2 k-NN covariance; Sec. 3.3) ------------
 * New surfels at the points of a keyframe scan: for each point its k nearest
 * neighbours among the scan's points (itself included; binary32 squared
 * distance ((dx dx + dy dy) + dz dz), ties to the lower index), the
 * covariance of the neighbourhood about its mean (1/k) and its
 * eigendecomposition (lambda_0 >= lambda_1 >= lambda_2), then
 *  - orientation: normal = the smallest eigenvector turned toward the sensor,
 *    t_u = the largest (its sign is free), t_v = n x t_u, rotated to the
 *    world by the pose;
 *  - the range-adaptive scale s = clip(kappa max(|p|, 1) sigma_tan, s_min,
 *    s_max) with sigma_tan = (1, sigma_1 / sigma_0), sigma = sqrt(lambda)
 *    (normalised by the largest, as G-ICP normalises its covariances);
 *  - the physics-based confidence u = exp(-(|p| / r0)^2) clip((c - c0) /
 *    (1 - c0 + eps), 0, 1), c = |n . p / |p|| (Eq. physconf);
 *  - the opacity alpha = alpha_min + (alpha_max - alpha_min) u (Eq.
 *    alpha_init), stored as its logit.
 * The eigenvalues are returned for the control score of map management. */
typedef struct {
    int32_t k;           /* neighbours, 3..32, <= n; 20 */
    float kappa;         /* > 0; 0.0184 (1.5 x the pitch of a 128-beam +-45 deg sensor) */
    float s_min, s_max;  /* 0 < s_min <= s_max; 1e-3, 1.0 (metres) */
    float r0;            /* > 0; 100 (metres) */
    float c0;            /* in [0, 1); 0.1 */
    float eps;           /* > 0; 1e-6 */
    float alpha_min, alpha_max;   /* 0 < alpha_min <= alpha_max < 1; 0.3, 0.9 */
} lgs_init_params;

/* The defaults listed above. */
LGS_API void lgs_init_default_params(lgs_init_params* p);
/* Bytes of device scratch lgs_keyframe_init needs for n points. */
LGS_API size_t lgs_init_scratch_bytes(int64_t n);
/* Points per call at most (2^20). */
LGS_API int64_t lgs_init_max_points(void);
/* Kernel launches one lgs_keyframe_init call makes (for launch accounting). */
LGS_API int32_t lgs_init_launches(void);

/* points [n][3]: device, the scan's points in the sensor frame, finite and
 * not at the origin; pose: host, 12 floats (sensor -> world, R row-major |
 * t).  scratch: lgs_init_scratch_bytes(n) bytes of device memory, 16-byte
 * aligned, contents irrelevant.  Writes knn [n][k] int32 (ascending
 * distance), the new surfels into out (n rows, world frame), lam [n][3] and
 * u [n], all device and caller-owned.  pairs: NULL, or a device int64 to
 * which the k-NN adds the number of (query, candidate) distances it
 * evaluated (tiles it could not rule out by their bounding boxes).  Enqueues
 * on stream without a host sync; argument errors return LGS_ERR_INVALID_ARG
 * before anything is enqueued. */
LGS_API lgs_status lgs_keyframe_init(const float* points, int64_t n, const float pose[12],
                                     const lgs_init_params* params, void* scratch, size_t scratch_bytes,
                                     int32_t* knn, const lgs_surfel_params_out* out, float* lam, float* u,
                                     int64_t* pairs, void* stream);

/* ---- image loss without a session or workspace --------------------------
 * The paper has no counterpart to this call; it is an interface for callers
 * that cannot allocate device memory at the point where they evaluate the
 * loss (for instance a mapping thread whose device memory is all reserved up
 * front, or code that holds no lgs workspace) and still need the image terms
 * of the mapping loss (Eqs. depthloss, normalloss) of frames they rendered.
 *
 * Computes, for n_frames frames of one map (each weighted 1 / n_frames), the
 * image terms and their upstream gradient planes with the same arithmetic and
 * reduction order as the image part of lgs_loss: on the device,
 * loss_out[0] = (1/F) sum_f [L_depth + la L_alpha + ln lng L_ng]_f and
 * loss_out[1+3f .. 3+3f] = (L_depth, L_alpha, L_ng) of frame f (1 + 3
 * n_frames floats); grads_out[f] (overwritten) as in lgs_loss.  H[f], W[f]:
 * host arrays of the frames' sizes; fwd, targets, grads_out: host arrays of
 * device pointers as in lgs_loss; params->lambda_s and s_max are unused.
 * The call has no frame geometry (pixel rays), so it has no N_surf term:
 * params->lambda_ns must be 0 (else LGS_ERR_INVALID_ARG).
 *
 * Nothing is allocated, by the library or by the caller: the scratch
 * (fixed-point loss sums and mask counts per frame, a completion counter) is
 * one static device array of LGS_NOALLOC_SCRATCH_BYTES inside the library,
 * sized for at most LGS_NOALLOC_MAX_FRAMES frames per call; more frames are
 * rejected with LGS_ERR_INVALID_ARG.  The caller zeroes nothing: the scratch
 * is zero when the library loads and every call leaves it at zero on the
 * device when it completes.  Every call looks up the scratch's address in
 * the current device's context (cudaGetSymbolAddress, with that device
 * current; nothing is cached, so the address stays right after a device
 * reset or in a new context).  The first call in a context may load the
 * library's device code there, so make one call on each device before any
 * stream capture or timing-critical use.  Every call on a device
 * shares the one scratch: calls that overlap in time (on other streams or
 * from other threads) corrupt each other's results and must be serialised by
 * the caller. */
#define LGS_NOALLOC_MAX_FRAMES 8
#define LGS_NOALLOC_SCRATCH_BYTES (8 * 3 * LGS_NOALLOC_MAX_FRAMES + 4 * 2 * LGS_NOALLOC_MAX_FRAMES + 256)
LGS_API lgs_status lgs_image_loss_noalloc(const int32_t* H, const int32_t* W, int n_frames, const lgs_fwd_out* fwd,
                                          const lgs_target* targets, const lgs_loss_params* params,
                                          const lgs_fwd_grad_out* grads_out, float* loss_out, void* stream);

/* Set the compositing knobs of a session (defaults: fwd_batch 0, bwd_batch 0,
 * group 16, persistent 0).  Every choice gives bit-identical forward outputs. */
LGS_API lgs_status lgs_session_set_tuning(lgs_session s, const lgs_tuning* t);

/* One Adam step over the n surfels' 10 parameters (optimiser of the mapping
 * loop; the paper does not name it): m = b1 m + (1-b1) g,
 * v = b2 v + (1-b2) g^2, p -= lr_group * mhat / (sqrt(vhat) + eps) with bias
 * correction for step `step` (>= 1); lr[0..3] for mean, quat, log_scale,
 * logit.  Zeroes the gradients afterwards when zero_grad != 0.  All pointers
 * device, layouts as lgs_surfels; m and v have the parameters' layout. */
LGS_API lgs_status lgs_adam_step(float* mean, float* quat, float* log_scale, float* logit,
                         const lgs_surfel_grad* grad, float* m_state, float* v_state, int64_t n,
                         int64_t step, const float lr[4], float beta1, float beta2, float eps,
                         int zero_grad, void* stream);

/* One map of a batched Adam step (the arguments of lgs_adam_step). */
typedef struct {
    float *mean, *quat, *log_scale, *logit;
    lgs_surfel_grad grad;
    float *m_state, *v_state;
    int64_t n;
    int64_t step;                /* this map's own step count (>= 1) */
    float lr[4];
} lgs_adam_map;

/* lgs_adam_step for n_maps maps (at most LGS_MAX_MAPS) in one launch, each
 * with its own step count and learning rates. */
LGS_API lgs_status lgs_adam_step_batch(const lgs_adam_map* maps, int n_maps, float beta1, float beta2, float eps,
                                       int zero_grad, void* stream);

/* ---- misc ---------------------------------------------------------------- */
LGS_API const char* lgs_status_string(lgs_status st);

/* Text of the last error recorded on the calling host thread ("" if none). */
LGS_API const char* lgs_last_error(void);

/* The library's constants, for cross-checking with an independent oracle:
 * [0] t_near 0.2, [1] cut-off 9, [2] 1/255, [3] clamp 0.99, [4] T stop 1e-4,
 * [5] grazing 1e-6, [6] eps_A 1e-6, [7] eps_N 1e-6, [8] eps_log 1e-6,
 * [9] binning radius factor 3, [10] radius margin 1.0001, [11] 1e-5 m/m. */
LGS_API void lgs_constants(float out[16]);

/* Library version string. */
LGS_API const char* lgs_version(void);

#ifdef __cplusplus
}
#endif
#endif /* LGS_H */
