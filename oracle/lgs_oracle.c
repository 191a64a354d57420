/*
 * lgs_oracle.c -- plain, slow CPU oracle for the spherical rasterizer of 2D
 * Gaussian surfels into a LiDAR range image (forward, mapping losses and the
 * analytic backward), following the map representation and map optimisation
 * of the paper (Sec. 3.1 "Map Representation", Sec. 3.4 "Map Optimization",
 * Eqs. depthloss / normalloss / scaleloss / totalloss).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  It shares no code,
 * header, table or constant generator with the CUDA library; gcc builds it
 * from this file and lgs_fp32_allowance.c.
 *
 * This file is the method and nothing else.  What a binary32 evaluation of
 * the same inputs may differ by (the allowance the parity tests add to their
 * bars) lives in lgs_fp32_allowance.c, which re-walks the evaluations made
 * here; the method never reads it.
 *
 * Two precisions, on purpose:
 *  (i)  Binning (which surfels are listed for which angular tile) and the
 *       depth sort key are defined in IEEE binary32 with a fixed order of
 *       correctly rounded + - * / sqrt (compiled with -ffp-contract=off), so
 *       that a GPU implementation of the same definition is bit-exact.
 *       Transcendentals inside binning are replaced by the fixed polynomial
 *       definitions f32_exp_spec / f32_sin_spec / f32_cos_spec below.
 *  (ii) Everything else (ray directions, ray/surfel-plane intersection,
 *       Gaussian weights, compositing, losses, reverse mode) is FP64 from the
 *       binary32 inputs.
 *
 * Readings of points the paper leaves open (pixel grid, pose convention,
 * cut-offs, clamps, termination rule, depth order) are listed in the design
 * notes; every constant carries its reading (lgs_oracle_impl.h).
 *
 * Parity pins (tests, not this file): single surfel facing the ray (closed
 * form), coaxial stacks (transmittance = product of (1-a)), tiled == brute
 * force all-pairs (bitwise), sort == comparison sort, 90-degree rotation
 * invariance across the azimuth seam, analytic gradient == central finite
 * differences, hand-computed losses.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "lgs_oracle_impl.h"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

void lgso_constants(double out[16])
{
    memset(out, 0, 16 * sizeof(double));
    out[0] = T_NEAR; out[1] = Q_CUT; out[2] = A_MIN; out[3] = A_MAX;
    out[4] = T_STOP; out[5] = DEN_EPS; out[6] = EPS_A; out[7] = EPS_N;
    out[8] = EPS_LOG;
    out[9] = 3.0;       /* binning radius = 3 x max scale ...           */
    out[10] = 1.0001;   /* ... x (1 + 1e-4) ...                         */
    out[11] = 1e-5;     /* ... + 1e-5 x (range + 1 m)                   */
}

/* ------------------------------------------------------------------------ */
/* Part I: binning in specified binary32 arithmetic                          */
/* ------------------------------------------------------------------------ */
static float f32_from_bits(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static uint32_t f32_bits(float f) { uint32_t u; memcpy(&u, &f, 4); return u; }

/* exp(x) for the binning radius only: Cody-Waite reduction x = k ln2 + r with
 * ln2 split into a 15-bit head and a binary32 tail, then the Taylor series of
 * e^r through r^7 in Horner form; finally an exact scaling by 2^k.  Relative
 * error < 1e-6 on [-80, 80], far inside the 1e-4 radius margin. */
float lgso_f32_exp_spec(float x)
{
    if (!(x < 80.0f)) x = 80.0f;          /* NaN also maps to +80 */
    if (x < -80.0f) x = -80.0f;
    float kf = rintf(x * 0x1.715476p+0f);             /* x / ln2 */
    float r = x - kf * 0x1.62e4p-1f;                  /* ln2 head */
    r = r - kf * 0x1.7f7d1cp-20f;                     /* ln2 tail */
    float p = 0x1.a01a02p-13f;                        /* 1/7! */
    p = p * r + 0x1.6c16c2p-10f;                      /* 1/6! */
    p = p * r + 0x1.111112p-7f;                       /* 1/5! */
    p = p * r + 0x1.555556p-5f;                       /* 1/4! */
    p = p * r + 0x1.555556p-3f;                       /* 1/3! */
    p = p * r + 0.5f;                                 /* 1/2! */
    p = p * r + 1.0f;
    p = p * r + 1.0f;
    int k = (int)kf;
    return p * f32_from_bits((uint32_t)(k + 127) << 23);
}

/* The same, over an array (map management specifies the surfels' scales with
 * it, so that its binary32 decisions are a fixed function of the inputs). */
void lgso_f32_exp_spec_n(const float* x, float* y, int64_t n)
{
    for (int64_t i = 0; i < n; i++) y[i] = lgso_f32_exp_spec(x[i]);
}

/* sin and cos on [-pi/2, pi/2] by their Taylor series (through x^11 and
 * x^12), Horner form in x^2, each operation rounded once. */
float lgso_f32_sin_spec(float x)
{
    float x2 = x * x;
    float p = -0x1.ae6456p-26f;                       /* -1/11! */
    p = p * x2 + 0x1.71de3ap-19f;                     /*  1/9!  */
    p = p * x2 - 0x1.a01a02p-13f;                     /* -1/7!  */
    p = p * x2 + 0x1.111112p-7f;                      /*  1/5!  */
    p = p * x2 - 0x1.555556p-3f;                      /* -1/3!  */
    p = p * x2;
    return p * x + x;
}

float lgso_f32_cos_spec(float x)
{
    float x2 = x * x;
    float p = 0x1.1eed8ep-29f;                        /*  1/12! */
    p = p * x2 - 0x1.27e4fcp-22f;                     /* -1/10! */
    p = p * x2 + 0x1.a01a02p-16f;                     /*  1/8!  */
    p = p * x2 - 0x1.6c16c2p-10f;                     /* -1/6!  */
    p = p * x2 + 0x1.555556p-5f;                      /*  1/4!  */
    p = p * x2 - 0.5f;                                /* -1/2!  */
    return p * x2 + 1.0f;
}

/* Elevation of pixel-row centre r (row 0 at the top), binary32. */
static float f32_row_elev(int r, int H, float emin, float emax)
{
    float dth = (emax - emin) / (float)H;
    return emax - ((float)r + 0.5f) * dth;
}

/* (cos, sin) of the azimuth of pixel-column centre c: phi = 2 pi (2c+1)/(2W).
 * The fraction f = (2c+1)/(2W) is split into its quadrant k = floor(4f) and an
 * exact remainder before the angle is formed, so the series is only used on
 * [0, pi/2). */
void lgso_f32_col_dir(int c, int W, float* cs, float* sn)
{
    float f = (float)(2 * c + 1) / (float)(2 * W);
    int k = (int)(f * 4.0f);
    if (k > 3) k = 3;
    float rq = f - (float)k * 0.25f;
    float x = rq * 0x1.921fb6p+2f;                    /* 2 pi */
    float s0 = lgso_f32_sin_spec(x), c0 = lgso_f32_cos_spec(x);
    switch (k) {
    case 0: *cs = c0;  *sn = s0;  break;
    case 1: *cs = -s0; *sn = c0;  break;
    case 2: *cs = -c0; *sn = -s0; break;
    default: *cs = s0; *sn = -c0; break;
    }
}

/* Per-frame binning tables: for tile row i the sines of the elevations of its
 * top and bottom pixel-centre rows; for tile column j the direction (cos,sin)
 * of its first and last pixel-centre columns. */
void lgso_bin_tables(int H, int W, int th, int tw, float emin, float emax,
                     float* sin_top, float* sin_bot, float* col4)
{
    int ntr = (H + th - 1) / th, ntc = (W + tw - 1) / tw;
    for (int i = 0; i < ntr; ++i) {
        int r0 = i * th, r1 = (i + 1) * th < H ? (i + 1) * th - 1 : H - 1;
        sin_top[i] = lgso_f32_sin_spec(f32_row_elev(r0, H, emin, emax));
        sin_bot[i] = lgso_f32_sin_spec(f32_row_elev(r1, H, emin, emax));
    }
    for (int j = 0; j < ntc; ++j) {
        int c0 = j * tw, c1 = (j + 1) * tw < W ? (j + 1) * tw - 1 : W - 1;
        lgso_f32_col_dir(c0, W, &col4[4 * j + 0], &col4[4 * j + 1]);
        lgso_f32_col_dir(c1, W, &col4[4 * j + 2], &col4[4 * j + 3]);
    }
}

/* Binning geometry of one surfel for one frame (binary32 throughout).
 *  - centre in the sensor frame: p_s = R^T (p_w - o), R row-major;
 *  - depth key = |p_s| (its bit pattern sorts like the value, as it is >= 0);
 *  - bounding sphere radius rho = 3 * exp(max log-scale) * 1.0001
 *                                 + 1e-5 * (|p_s| + 1);
 *  - the cone of rays that meet the sphere: rows whose elevation band meets
 *    [theta_c - beta, theta_c + beta] (compared through sines), columns whose
 *    azimuth interval meets [phi_c - dphi, phi_c + dphi] (compared through dot
 *    and cross products with the column directions).  A sensor inside the
 *    sphere covers every tile; a cone containing a pole covers every column. */
typedef struct {
    float x, y, z, r, h, rho;
    int all_rows, all_cols;
    float sin_hi, sin_lo;
    uint32_t key;
} bin_geom;

static void f32_bin_geom(const float* mw, const float* ls, const float* pose, bin_geom* g)
{
    float dx = mw[0] - pose[3], dy = mw[1] - pose[7], dz = mw[2] - pose[11];
    float x = (pose[0] * dx + pose[4] * dy) + pose[8] * dz;
    float y = (pose[1] * dx + pose[5] * dy) + pose[9] * dz;
    float z = (pose[2] * dx + pose[6] * dy) + pose[10] * dz;
    float h2 = x * x + y * y;
    float r2 = h2 + z * z;
    float r = sqrtf(r2), h = sqrtf(h2);
    float sm = ls[0] >= ls[1] ? ls[0] : ls[1];
    float s = lgso_f32_exp_spec(sm);
    float rho = (3.0f * s) * 1.0001f + 1e-5f * (r + 1.0f);
    g->x = x; g->y = y; g->z = z; g->r = r; g->h = h; g->rho = rho;
    g->key = f32_bits(r);
    g->all_rows = 0; g->all_cols = 0; g->sin_hi = 2.0f; g->sin_lo = -2.0f;
    float rr = r2 - rho * rho;
    if (!(rr > 0.0f)) { g->all_rows = 1; g->all_cols = 1; return; }
    float c = sqrtf(rr);
    float hc = h * c, zp = z * rho, zc = z * c, hp = h * rho;
    int north = hc <= zp, south = hc <= -zp;
    g->sin_hi = north ? 2.0f : (zc + hp) / r2;
    g->sin_lo = south ? -2.0f : (zc - hp) / r2;
    g->all_cols = north || south;
}

static int f32_row_hit(const bin_geom* g, float st, float sb)
{
    return g->all_rows || (sb <= g->sin_hi && st >= g->sin_lo);
}

static int f32_dir_in_cap(const bin_geom* g, float cs, float sn)
{
    float dt = g->x * cs + g->y * sn;
    float cr = g->x * sn - g->y * cs;
    return dt > 0.0f && fabsf(cr) <= g->rho;
}

static int f32_col_hit(const bin_geom* g, const float* c4)
{
    if (g->all_cols) return 1;
    if (f32_dir_in_cap(g, c4[0], c4[1]) || f32_dir_in_cap(g, c4[2], c4[3])) return 1;
    /* centre azimuth between the first and last column directions */
    return (c4[0] * g->y - c4[1] * g->x) >= 0.0f && (g->x * c4[3] - g->y * c4[2]) >= 0.0f;
}

typedef struct { uint64_t key; uint32_t val; } pair_t;

static int cmp_pair(const void* a, const void* b)
{
    const pair_t* p = (const pair_t*)a; const pair_t* q = (const pair_t*)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->val < q->val ? -1 : (p->val > q->val);
}

/* Bin one frame.  Writes the depth key bits and tile count per surfel, and,
 * when keys_sorted != NULL and cap >= pairs, the (tile<<32 | depth_bits, idx)
 * pairs in ascending (key, idx) order -- the order a stable sort of keys
 * emitted in surfel-index order produces -- plus [start,end) per tile.
 * Returns the number of pairs. */
int64_t lgso_bin_frame(const float* mean, const float* log_scale, int64_t n,
                       int H, int W, int th, int tw, float emin, float emax,
                       const float* pose, uint32_t* depth_bits, int32_t* count,
                       uint64_t* keys_sorted, uint32_t* vals_sorted, int64_t cap,
                       int64_t* ranges)
{
    int ntr = (H + th - 1) / th, ntc = (W + tw - 1) / tw;
    float* st = (float*)malloc(sizeof(float) * ntr);
    float* sb = (float*)malloc(sizeof(float) * ntr);
    float* c4 = (float*)malloc(sizeof(float) * 4 * ntc);
    lgso_bin_tables(H, W, th, tw, emin, emax, st, sb, c4);
    int64_t total = 0;
    for (int64_t i = 0; i < n; ++i) {
        bin_geom g;
        f32_bin_geom(mean + 3 * i, log_scale + 2 * i, pose, &g);
        int nr = 0, nc = 0;
        for (int a = 0; a < ntr; ++a) nr += f32_row_hit(&g, st[a], sb[a]);
        for (int b = 0; b < ntc; ++b) nc += f32_col_hit(&g, c4 + 4 * b);
        if (depth_bits) depth_bits[i] = g.key;
        if (count) count[i] = nr * nc;
        total += (int64_t)nr * nc;
    }
    if (keys_sorted && total <= cap) {
        pair_t* pr = (pair_t*)malloc(sizeof(pair_t) * (total > 0 ? total : 1));
        int64_t m = 0;
        for (int64_t i = 0; i < n; ++i) {
            bin_geom g;
            f32_bin_geom(mean + 3 * i, log_scale + 2 * i, pose, &g);
            for (int a = 0; a < ntr; ++a) {
                if (!f32_row_hit(&g, st[a], sb[a])) continue;
                for (int b = 0; b < ntc; ++b) {
                    if (!f32_col_hit(&g, c4 + 4 * b)) continue;
                    pr[m].key = ((uint64_t)(uint32_t)(a * ntc + b) << 32) | g.key;
                    pr[m].val = (uint32_t)i;
                    ++m;
                }
            }
        }
        qsort(pr, (size_t)m, sizeof(pair_t), cmp_pair);
        if (ranges) for (int64_t t = 0; t < 2 * (int64_t)ntr * ntc; ++t) ranges[t] = 0;
        for (int64_t k = 0; k < m; ++k) {
            keys_sorted[k] = pr[k].key; vals_sorted[k] = pr[k].val;
            if (ranges) {
                int64_t t = (int64_t)(pr[k].key >> 32);
                if (k == 0 || (pr[k - 1].key >> 32) != (uint64_t)t) ranges[2 * t] = k;
                ranges[2 * t + 1] = k + 1;
            }
        }
        free(pr);
    }
    free(st); free(sb); free(c4);
    return total;
}

/* ------------------------------------------------------------------------ */
/* Part II: FP64 forward                                                     */
/* ------------------------------------------------------------------------ */
/* Rotation matrix of a unit quaternion (w,x,y,z), row-major; its columns are
 * the tangent axes t_u = R e0, t_v = R e1 and the normal n = R e2. */
static void quat_to_rot(const double* q, double* R)
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

void make_frame(frame64* F, int H, int W, int th, int tw, double emin, double emax, const double* pose)
{
    F->H = H; F->W = W; F->th = th; F->tw = tw;
    F->ntr = (H + th - 1) / th; F->ntc = (W + tw - 1) / tw;
    F->emin = emin; F->emax = emax;
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b) F->R[3 * a + b] = pose[4 * a + b];
        F->o[a] = pose[4 * a + 3];
    }
}

/* Surfel i in the sensor frame: mu_s = R^T (mu_w - o), axes R^T R(q/|q|),
 * scales exp(log-scale), opacity sigmoid(logit). */
static void surf_to_sensor(const double* mean, const double* quat, const double* ls,
                           const double* logit, int64_t i, const frame64* F, surf64* s)
{
    const double* q = quat + 4 * i;
    double qn = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int k = 0; k < 4; ++k) s->qh[k] = q[k] / qn;
    s->qnorm = qn;
    double Rq[9];
    quat_to_rot(s->qh, Rq);
    double d[3] = { mean[3 * i] - F->o[0], mean[3 * i + 1] - F->o[1], mean[3 * i + 2] - F->o[2] };
    for (int a = 0; a < 3; ++a) {
        /* (R^T v)_a = sum_k R[k][a] v_k */
        s->mu[a] = F->R[a] * d[0] + F->R[3 + a] * d[1] + F->R[6 + a] * d[2];
        s->tu[a] = F->R[a] * Rq[0] + F->R[3 + a] * Rq[3] + F->R[6 + a] * Rq[6];
        s->tv[a] = F->R[a] * Rq[1] + F->R[3 + a] * Rq[4] + F->R[6 + a] * Rq[7];
        s->n[a]  = F->R[a] * Rq[2] + F->R[3 + a] * Rq[5] + F->R[6 + a] * Rq[8];
    }
    s->su = exp(ls[2 * i]);
    s->sv = exp(ls[2 * i + 1]);
    s->alpha = 1.0 / (1.0 + exp(-logit[i]));
}

/* Unit ray of pixel (r, c): elevation theta_r = emax - (r + 1/2)(emax-emin)/H
 * (row 0 at the top), azimuth phi_c = (c + 1/2) 2 pi / W counter-clockwise
 * from the sensor +x axis; d = (cos th cos ph, cos th sin ph, sin th). */
void pixel_ray(const frame64* F, int r, int c, double* d)
{
    double th = F->emax - (r + 0.5) * (F->emax - F->emin) / F->H;
    double ph = (c + 0.5) * 2.0 * M_PI / F->W;
    d[0] = cos(th) * cos(ph); d[1] = cos(th) * sin(ph); d[2] = sin(th);
}

/* One ray / surfel evaluation: plane intersection t = (n.mu)/(n.d), local
 * coordinates u = t_u.(t d - mu)/s_u, v = t_v.(t d - mu)/s_v, Gaussian
 * G = exp(-(u^2+v^2)/2), opacity a = min(alpha G, 0.99), with the skip rules
 * |n.d| < 1e-6, t <= t_near, u^2+v^2 > 9, a < 1/255 (valid = 0 when one
 * applies; the quantities after the failing rule are not formed). */
void eval_pair(const surf64* s, const double* d, eval64* e)
{
    e->valid = 0;
    e->den = dot3(s->n, d);
    if (fabs(e->den) < DEN_EPS) return;
    e->t = dot3(s->n, s->mu) / e->den;
    if (e->t <= T_NEAR) return;
    for (int k = 0; k < 3; ++k) e->x[k] = e->t * d[k] - s->mu[k];
    e->u = dot3(s->tu, e->x) / s->su;
    e->v = dot3(s->tv, e->x) / s->sv;
    e->q = e->u * e->u + e->v * e->v;
    if (e->q > Q_CUT) return;
    e->G = exp(-0.5 * e->q);
    e->araw = s->alpha * e->G;
    e->a = e->araw < A_MAX ? e->araw : A_MAX;
    if (e->a < A_MIN) return;
    e->valid = 1;
}

surf64* sensor_surfels(const double* mean, const double* quat, const double* ls,
                       const double* logit, int64_t n, const frame64* F)
{
    surf64* S = (surf64*)malloc(sizeof(surf64) * (n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) surf_to_sensor(mean, quat, ls, logit, i, F, S + i);
    return S;
}

/* Front-to-back compositing of one pixel over list[0..len): for each valid
 * surfel, stop (without compositing it) if T (1 - a) < 1e-4, else
 * w = a T; A += w; S_t += w t; S_n += w (-sign(n.d)) n; T *= 1 - a.
 * Contributors are recorded in ck (list position) with the transmittance
 * before them in cT, when ck != NULL.  Returns their number. */
int composite_pixel(const surf64* S, const uint32_t* list, int64_t len, const double* d,
                    pix_out* o, int64_t* ck, double* cT)
{
    o->A = 0; o->St = 0; o->Sn[0] = o->Sn[1] = o->Sn[2] = 0; o->T = 1.0;
    o->ncontrib = 0; o->neval = 0;
    int nc = 0;
    for (int64_t k = 0; k < len; ++k) {
        const surf64* s = S + list[k];
        eval64 e;
        eval_pair(s, d, &e);
        o->neval++;
        if (!e.valid) continue;
        double Tn = o->T * (1.0 - e.a);
        if (Tn < T_STOP) break;
        double w = e.a * o->T;
        double sg = e.den > 0 ? -1.0 : 1.0;           /* -sign(n.d) */
        o->A += w;
        o->St += w * e.t;
        for (int k3 = 0; k3 < 3; ++k3) o->Sn[k3] += w * sg * s->n[k3];
        if (ck) { ck[nc] = k; cT[nc] = o->T; }
        nc++;
        o->T = Tn;
        o->ncontrib = (int32_t)(k + 1);
    }
    return nc;
}

/* Forward render of one frame.  ranges[2*tile] / ranges[2*tile+1] delimit the
 * tile's list in vals (surfel indices in depth order).  Outputs are planar
 * [H*W] (S_n: [3][H*W]).  When pix_flag, eA and eD are given, the binary32
 * allowance of every pixel is added (lgs_fp32_allowance.c): pix_flag marks
 * pixels where some evaluated quantity lies near a threshold (a binary32
 * evaluation may decide it differently), eA / eD bound the opacity and depth
 * a binary32 evaluation of the same inputs may give. */
void lgso_render_fwd(const double* mean, const double* quat, const double* ls, const double* logit,
                     int64_t n, int H, int W, int th, int tw, double emin, double emax,
                     const double* pose, const int64_t* ranges, const uint32_t* vals,
                     double* A, double* St, double* Sn, double* Tf, int32_t* ncontrib,
                     int64_t* neval, uint8_t* pix_flag, int32_t* nvalid, double* eA, double* eD,
                     int nthreads)
{
    frame64 F;
    make_frame(&F, H, W, th, tw, emin, emax, pose);
    surf64* S = sensor_surfels(mean, quat, ls, logit, n, &F);
    int64_t ntiles = (int64_t)F.ntr * F.ntc;
    int64_t HW = (int64_t)H * W;
    int64_t maxlen = 1;
    for (int64_t t = 0; t < ntiles; ++t)
        if (ranges[2 * t + 1] - ranges[2 * t] > maxlen) maxlen = ranges[2 * t + 1] - ranges[2 * t];
    const int unc = pix_flag && eA && eD;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
    int64_t* ck = (int64_t*)malloc(sizeof(int64_t) * maxlen);
    double* cT = (double*)malloc(sizeof(double) * maxlen);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
    for (int64_t tile = 0; tile < ntiles; ++tile) {
        int ti = (int)(tile / F.ntc), tj = (int)(tile % F.ntc);
        int64_t b = ranges[2 * tile], e = ranges[2 * tile + 1];
        for (int r = ti * th; r < (ti + 1) * th && r < H; ++r)
            for (int c = tj * tw; c < (tj + 1) * tw && c < W; ++c) {
                double d[3];
                pixel_ray(&F, r, c, d);
                pix_out o;
                int nc = composite_pixel(S, vals + b, e - b, d, &o, ck, cT);
                int64_t p = (int64_t)r * W + c;
                if (nvalid) nvalid[p] = nc;
                if (unc) {
                    pix_unc u;
                    fwd_allowance(S, vals + b, d, &o, nc, ck, cT, &u, eA + p, eD + p);
                    pix_flag[p] = (uint8_t)u.flags;
                }
                A[p] = o.A; St[p] = o.St; Tf[p] = o.T;
                Sn[p] = o.Sn[0]; Sn[HW + p] = o.Sn[1]; Sn[2 * HW + p] = o.Sn[2];
                if (ncontrib) ncontrib[p] = o.ncontrib;
                if (neval) neval[p] = o.neval;
            }
    }
    free(ck); free(cT);
    }
    free(S);
}

/* Conservativeness of binning: count the (pixel, surfel) pairs whose FP64
 * evaluation is valid (would be composited if reached) although the surfel is
 * not listed for the pixel's tile.  Brute force over all pairs. */
int64_t lgso_coverage_misses(const double* mean, const double* quat, const double* ls, const double* logit,
                             int64_t n, int H, int W, int th, int tw, double emin, double emax,
                             const double* pose, const int64_t* ranges, const uint32_t* vals)
{
    frame64 F;
    make_frame(&F, H, W, th, tw, emin, emax, pose);
    surf64* S = sensor_surfels(mean, quat, ls, logit, n, &F);
    uint8_t* listed = (uint8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
    int64_t misses = 0;
    for (int64_t tile = 0; tile < (int64_t)F.ntr * F.ntc; ++tile) {
        int ti = (int)(tile / F.ntc), tj = (int)(tile % F.ntc);
        for (int64_t k = ranges[2 * tile]; k < ranges[2 * tile + 1]; ++k) listed[vals[k]] = 1;
        for (int r = ti * th; r < (ti + 1) * th && r < H; ++r)
            for (int c = tj * tw; c < (tj + 1) * tw && c < W; ++c) {
                double d[3];
                pixel_ray(&F, r, c, d);
                for (int64_t i = 0; i < n; ++i) {
                    eval64 e;
                    eval_pair(S + i, d, &e);
                    if (e.valid && !listed[i]) misses++;
                }
            }
        for (int64_t k = ranges[2 * tile]; k < ranges[2 * tile + 1]; ++k) listed[vals[k]] = 0;
    }
    free(listed);
    free(S);
    return misses;
}

/* ------------------------------------------------------------------------ */
/* Part III: FP64 reverse mode                                               */
/* ------------------------------------------------------------------------ */
/* Sensor-frame gradient of one contribution: evaluation e of surfel s at
 * transmittance T (before it), with suffix = sum over the later contributors
 * of w_j (g.c_j).  With c = (1, t, n') and w = a T:
 *   dL/da = T (g.c) - suffix / (1 - a),
 * because every later weight carries the factor (1 - a).  Adds into *g and
 * returns g.c.  use_clamp = 0 differentiates through alpha G even where a is
 * clamped at 0.99 (the size of what a clamp decision switches on or off). */
double contrib_grad(const surf64* s, const eval64* e, const double* d, double T, double suffix,
                    double gA, double gSt, const double* gSn, int use_clamp, sgrad* g)
{
    double sg = e->den > 0 ? -1.0 : 1.0;
    double np[3] = { sg * s->n[0], sg * s->n[1], sg * s->n[2] };
    double gc = gA + gSt * e->t + dot3(gSn, np);
    double w = e->a * T;
    double dLda = T * gc - suffix / (1.0 - e->a);
    /* direct terms of S_t and S_n (the sign flip has zero derivative) */
    double dLdt = w * gSt;
    for (int k = 0; k < 3; ++k) g->n[k] += w * sg * gSn[k];
    /* through a = min(alpha G, 0.99): zero derivative when clamped */
    double dLdu = 0, dLdv = 0;
    if (!use_clamp || e->araw < A_MAX) {
        g->alpha += dLda * e->G;
        double dLdq = dLda * s->alpha * (-0.5 * e->G);
        dLdu = dLdq * 2.0 * e->u;
        dLdv = dLdq * 2.0 * e->v;
    }
    /* u = t_u.(t d - mu)/s_u,  v = t_v.(t d - mu)/s_v */
    dLdt += dLdu * dot3(s->tu, d) / s->su + dLdv * dot3(s->tv, d) / s->sv;
    for (int k = 0; k < 3; ++k) {
        g->tu[k] += dLdu * e->x[k] / s->su;
        g->tv[k] += dLdv * e->x[k] / s->sv;
        g->mu[k] -= dLdu * s->tu[k] / s->su + dLdv * s->tv[k] / s->sv;
    }
    g->su -= dLdu * e->u / s->su;
    g->sv -= dLdv * e->v / s->sv;
    /* t = (n.mu)/(n.d): dt/dmu = n/den, dt/dn = (mu - t d)/den */
    for (int k = 0; k < 3; ++k) {
        g->mu[k] += dLdt * s->n[k] / e->den;
        g->n[k] += dLdt * (s->mu[k] - e->t * d[k]) / e->den;
    }
    return gc;
}

static void sgrad_add(sgrad* a, const sgrad* b)
{
    for (int k = 0; k < 3; ++k) {
        a->mu[k] += b->mu[k]; a->tu[k] += b->tu[k]; a->tv[k] += b->tv[k]; a->n[k] += b->n[k];
    }
    a->su += b->su; a->sv += b->sv; a->alpha += b->alpha;
}

/* Reverse mode through composite_pixel for one pixel with upstream gradients
 * (gA, gSt, gSn) of (A, S_t, S_n): the contributors in reverse order, each
 * with its transmittance cT and the suffix over the later contributors
 * (per-pixel contributor lists are what this oracle stores; the GPU
 * recomputes them). */
static void backward_pixel(const surf64* S, const uint32_t* list, const double* d, int nc,
                           const int64_t* ck, const double* cT, double gA, double gSt,
                           const double* gSn, sgrad* G)
{
    double suffix = 0.0;
    for (int m = nc - 1; m >= 0; --m) {
        uint32_t i = list[ck[m]];
        const surf64* s = S + i;
        eval64 e;
        eval_pair(s, d, &e);                   /* recompute the same evaluation */
        sgrad c;
        memset(&c, 0, sizeof(c));
        double gc = contrib_grad(s, &e, d, cT[m], suffix, gA, gSt, gSn, 1, &c);
        suffix += e.a * cT[m] * gc;
        sgrad_add(G + i, &c);
    }
}

/* d R(q)_{ab} / d q_c for a unit quaternion q = (w,x,y,z); R row-major. */
void rot_jacobian(const double* q, double J[9][4])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    double t[9][4] = {
        { 0,      0,      -4 * y, -4 * z },   /* R00 = 1-2(y2+z2) */
        { -2 * z, 2 * y,  2 * x,  -2 * w },   /* R01 = 2(xy-wz)   */
        { 2 * y,  2 * z,  2 * w,  2 * x  },   /* R02 = 2(xz+wy)   */
        { 2 * z,  2 * y,  2 * x,  2 * w  },   /* R10 = 2(xy+wz)   */
        { 0,      -4 * x, 0,      -4 * z },   /* R11 = 1-2(x2+z2) */
        { -2 * x, -2 * w, 2 * z,  2 * y  },   /* R12 = 2(yz-wx)   */
        { -2 * y, 2 * z,  -2 * w, 2 * x  },   /* R20 = 2(xz-wy)   */
        { 2 * x,  2 * w,  2 * z,  2 * y  },   /* R21 = 2(yz+wx)   */
        { 0,      -4 * x, -4 * y, 0      },   /* R22 = 1-2(x2+y2) */
    };
    memcpy(J, t, sizeof(t));
}

/* Chain the sensor-frame gradient of surfel i to the raw parameters
 * (mean, quaternion, log-scale, logit); accumulates (+=). */
void chain_to_params(const surf64* s, const sgrad* g, const frame64* F,
                            double* dmean, double* dquat, double* dls, double* dlogit)
{
    /* mu_s = R^T (mu_w - o)  =>  d mu_w = R d mu_s; same for the axes */
    double dcol[3][3];   /* world-frame gradient of the columns of R(q) */
    for (int a = 0; a < 3; ++a) {
        double gm = 0, g0 = 0, g1 = 0, g2 = 0;
        for (int k = 0; k < 3; ++k) {
            gm += F->R[3 * a + k] * g->mu[k];
            g0 += F->R[3 * a + k] * g->tu[k];
            g1 += F->R[3 * a + k] * g->tv[k];
            g2 += F->R[3 * a + k] * g->n[k];
        }
        dmean[a] += gm;
        dcol[0][a] = g0; dcol[1][a] = g1; dcol[2][a] = g2;
    }
    double J[9][4];
    rot_jacobian(s->qh, J);
    double dqh[4] = { 0, 0, 0, 0 };
    for (int a = 0; a < 3; ++a)          /* row a */
        for (int b = 0; b < 3; ++b)      /* column b */
            for (int c = 0; c < 4; ++c) dqh[c] += dcol[b][a] * J[3 * a + b][c];
    /* q_hat = q / |q|  =>  dq = (dq_hat - q_hat (q_hat . dq_hat)) / |q| */
    double pr = dqh[0] * s->qh[0] + dqh[1] * s->qh[1] + dqh[2] * s->qh[2] + dqh[3] * s->qh[3];
    for (int c = 0; c < 4; ++c) dquat[c] += (dqh[c] - s->qh[c] * pr) / s->qnorm;
    dls[0] += g->su * s->su;                      /* s = exp(ls) */
    dls[1] += g->sv * s->sv;
    dlogit[0] += g->alpha * s->alpha * (1.0 - s->alpha);   /* sigmoid */
}

/* Backward of one frame: accumulates (+=) dL/d(mean, quat, log_scale, logit)
 * for upstream gradients gA, gSt [H*W], gSn [3][H*W].  When gabs and gflip
 * ([n][10]: mean 3, quat 4, log-scale 2, logit 1) are given, the binary32
 * allowance of the gradient is added (lgs_fp32_allowance.c): per surfel the
 * majorant of its per-pixel contributions and their binary32 uncertainty. */
void lgso_render_bwd(const double* mean, const double* quat, const double* ls, const double* logit,
                     int64_t n, int H, int W, int th, int tw, double emin, double emax,
                     const double* pose, const int64_t* ranges, const uint32_t* vals,
                     const double* gA, const double* gSt, const double* gSn,
                     double* dmean, double* dquat, double* dls, double* dlogit,
                     double* gabs, double* gflip, int nthreads)
{
    frame64 F;
    make_frame(&F, H, W, th, tw, emin, emax, pose);
    surf64* S = sensor_surfels(mean, quat, ls, logit, n, &F);
    int64_t ntiles = (int64_t)F.ntr * F.ntc, HW = (int64_t)H * W;
    int64_t maxlen = 1;
    for (int64_t t = 0; t < ntiles; ++t)
        if (ranges[2 * t + 1] - ranges[2 * t] > maxlen) maxlen = ranges[2 * t + 1] - ranges[2 * t];
    const int unc = gabs && gflip;
    int nth = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
    nth = omp_get_max_threads();
#endif
    sgrad* Gall = (sgrad*)calloc((size_t)nth * (n > 0 ? n : 1), sizeof(sgrad));
#ifdef _OPENMP
#pragma omp parallel
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        sgrad* G = Gall + (size_t)tid * (n > 0 ? n : 1);
        int64_t* ck = (int64_t*)malloc(sizeof(int64_t) * maxlen);
        double* cT = (double*)malloc(sizeof(double) * maxlen);
        double* tmp = unc ? (double*)malloc(sizeof(double) * 10 * maxlen) : NULL;
        double* suf = unc ? (double*)malloc(sizeof(double) * maxlen) : NULL;
        double* et = unc ? (double*)malloc(sizeof(double) * maxlen) : NULL;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t tile = 0; tile < ntiles; ++tile) {
            int ti = (int)(tile / F.ntc), tj = (int)(tile % F.ntc);
            int64_t b = ranges[2 * tile], e = ranges[2 * tile + 1];
            for (int r = ti * th; r < (ti + 1) * th && r < H; ++r)
                for (int c = tj * tw; c < (tj + 1) * tw && c < W; ++c) {
                    double d[3];
                    pixel_ray(&F, r, c, d);
                    pix_out o;
                    int nc = composite_pixel(S, vals + b, e - b, d, &o, ck, cT);
                    int64_t p = (int64_t)r * W + c;
                    double gsn[3] = { gSn[p], gSn[HW + p], gSn[2 * HW + p] };
                    backward_pixel(S, vals + b, d, nc, ck, cT, gA[p], gSt[p], gsn, G);
                    if (unc) {
                        pix_unc u;
                        double ea, ed;
                        fwd_allowance(S, vals + b, d, &o, nc, ck, cT, &u, &ea, &ed);
                        bwd_allowance(S, vals + b, d, nc, ck, cT, &o, &u, gA[p], gSt[p], gsn, &F, gabs, gflip,
                                      tmp, suf, et, NULL);
                    }
                }
        }
        free(ck); free(cT); free(tmp); free(suf); free(et);
    }
    for (int64_t i = 0; i < n; ++i) {
        sgrad acc;
        memset(&acc, 0, sizeof(acc));
        for (int t = 0; t < nth; ++t) sgrad_add(&acc, Gall + (size_t)t * n + i);
        chain_to_params(S + i, &acc, &F, dmean + 3 * i, dquat + 4 * i, dls + 2 * i, dlogit + i);
    }
    free(Gall);
    free(S);
}

/* ------------------------------------------------------------------------ */
/* Part IV: mapping losses (Eqs. depthloss, normalloss, scaleloss, totalloss) */
/* ------------------------------------------------------------------------ */
/* Image terms of one frame.  D[H*W] measured range (0 = no return),
 * Ng[3][H*W] normals from tracking (zero = undefined).  With
 *   M_D = [D > 0], M_N = M_D [|Ng| > 0], Dh = S_t/(A+1e-6),
 *   Nh = S_n / sqrt(|S_n|^2 + 1e-12),
 *   L_depth = mean_{M_D} |Dh - D|,  L_alpha = -mean_{M_D} log(A + 1e-6),
 *   L_ng = mean_{M_N} (1 - Nh.Ng),
 *   L_img = L_depth + lam_alpha L_alpha + lam_n lam_ng L_ng
 * (an empty mask makes its term 0; sign(0) = 0 for the L1 subgradient).
 * Writes dL_img/d(A, S_t, S_n) scaled by `scale` and returns scale * L_img;
 * terms[0..2] receive the unscaled L_depth, L_alpha, L_ng. */
double lgso_loss_image(const double* A, const double* St, const double* Sn, const float* D,
                       const float* Ng, int64_t npix, double lam_alpha, double lam_n, double lam_ng,
                       double scale, double* gA, double* gSt, double* gSn, double* terms)
{
    int64_t nd = 0, nn = 0;
    for (int64_t p = 0; p < npix; ++p) {
        int md = D[p] > 0.0f;
        double ng2 = (double)Ng[p] * Ng[p] + (double)Ng[npix + p] * Ng[npix + p] +
                     (double)Ng[2 * npix + p] * Ng[2 * npix + p];
        nd += md;
        nn += md && ng2 > 0.0;
    }
    double ldep = 0, lal = 0, lng = 0;
    for (int64_t p = 0; p < npix; ++p) {
        gA[p] = 0; gSt[p] = 0; gSn[p] = 0; gSn[npix + p] = 0; gSn[2 * npix + p] = 0;
        if (!(D[p] > 0.0f)) continue;
        double a = A[p] + EPS_A;
        double Dh = St[p] / a;
        double diff = Dh - (double)D[p];
        ldep += fabs(diff);
        double sgn = diff > 0 ? 1.0 : (diff < 0 ? -1.0 : 0.0);
        double gDh = sgn / nd;
        gSt[p] += scale * gDh / a;
        gA[p] += scale * (-gDh * St[p] / (a * a));
        lal += -log(A[p] + EPS_LOG);
        gA[p] += scale * (-lam_alpha / nd / (A[p] + EPS_LOG));
        double ng[3] = { Ng[p], Ng[npix + p], Ng[2 * npix + p] };
        if (ng[0] * ng[0] + ng[1] * ng[1] + ng[2] * ng[2] > 0.0) {
            double sn[3] = { Sn[p], Sn[npix + p], Sn[2 * npix + p] };
            double m = sqrt(sn[0] * sn[0] + sn[1] * sn[1] + sn[2] * sn[2] + EPS_N * EPS_N);
            double nh[3] = { sn[0] / m, sn[1] / m, sn[2] / m };
            lng += 1.0 - dot3(nh, ng);
            /* dL/dNh = -lam_n lam_ng Ng / |Omega_N|;  Nh = S/m:
               dL/dS = g/m - S (S.g)/m^3 */
            double g[3] = { -lam_n * lam_ng * ng[0] / nn, -lam_n * lam_ng * ng[1] / nn,
                            -lam_n * lam_ng * ng[2] / nn };
            double sg = dot3(sn, g);
            for (int k = 0; k < 3; ++k) gSn[k * npix + p] += scale * (g[k] / m - sn[k] * sg / (m * m * m));
        }
    }
    double Ld = nd ? ldep / nd : 0.0, La = nd ? lal / nd : 0.0, Ln = nn ? lng / nn : 0.0;
    if (terms) { terms[0] = Ld; terms[1] = La; terms[2] = Ln; }
    return scale * (Ld + lam_alpha * La + lam_n * lam_ng * Ln);
}

/* Second term of Eq. normalloss: the surface normal N_surf "computed from
 * the rendered depth" (Sec. 3.4), compared with the rendered normal Nh by the
 * cosine loss over Omega_D.  The paper gives no formula for N_surf; the
 * reading taken here:
 *   X_p    = Dh_p d_p, the rendered range of pixel p back-projected along its
 *            ray (sensor frame, Dh = S_t/(A+1e-6));
 *   e_c    = X(r, c+1 mod W) - X(r, c)   azimuth neighbour (the image wraps at
 *                                        2 pi, so column W-1 pairs with 0);
 *   e_r    = X(r+1, c) - X(r, c)         next row (lower elevation);
 *   N_surf = (e_c x e_r) / sqrt(|e_c x e_r|^2 + 1e-12); for a surface seen
 *            from the front this points back at the sensor, like Nh;
 *   L_ns   = (1/|Omega_D|) sum over pixels p with D > 0 and a rendered
 *            surface (A > 0, i.e. at least one composited surfel, so A >=
 *            1/255) at p and at both neighbours (the last row has none) of
 *            (1 - Nh_p . N_surf_p), normalised by |Omega_D| as Eq.
 *            normalloss writes it.  Without the A > 0 condition a pixel
 *            that renders nothing would enter with X = 0, and two such
 *            neighbours make e_c parallel to e_r: N_surf = 0 and a gradient
 *            of order 1/1e-6.
 * The gradient flows into Nh_p and, through N_surf, into the rendered ranges
 * of the three pixels.  Accumulates (+=) scale * lam * dL_ns/d(A, S_t, S_n)
 * (lam = lambda_n lambda_{n,s}) and returns the unscaled L_ns.
 *
 * err (optional, [2 H W + 1]) receives what a binary32 evaluation of the
 * same formulas may be off by (a first-order bound, not part of the loss):
 * with u = 2^-24 and each back-projected X good to 3u |X|, e_c and e_r are
 * off by 3u (|X| + |X'|), so the cross product c = e_c x e_r and N_surf are
 * off relatively by about
 *   rho = u (12 ((|X_p| + |X_R|) |e_r| + |e_c| (|X_p| + |X_B|)) / |c| + 8).
 * The gradients project lam/|Omega_D| Nh (resp. N_surf) orthogonally to
 * N_surf (resp. Nh): where the two normals nearly agree that is a small
 * difference of large terms, so their error scales with the terms, not
 * with the result: rho g0 (|e_c| + |e_r|) on dL/dX of each of the three
 * pixels, g0 = lam / (|Omega_D| |c|), and rho lam / (|Omega_D| |S_n|) on
 * dL/dS_n.  err[p] += scale times the first per term touching pixel p (a
 * bound on the range gradient d.dL/dX_p, before the chain into A and S_t),
 * err[HW + p] = scale times the second, err[2 HW] = (sum of rho over the
 * terms) / |Omega_D| (on L_ns). */
static void cross3(const double* a, const double* b, double* c)
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

double lgso_surf_normal_loss(const double* A, const double* St, const double* Sn, const float* D, int H, int W,
                             double emin, double emax, double lam, double scale, double* gA, double* gSt,
                             double* gSn, double* err)
{
    const int64_t HW = (int64_t)H * W;
    int64_t nd = 0;
    for (int64_t p = 0; p < HW; ++p) nd += D[p] > 0.0f;
    if (nd == 0 || H < 2) return 0.0;
    frame64 F;
    const double ident[12] = { 1, 0, 0, 0, 0, 1, 0, 0, 0, 0, 1, 0 };
    make_frame(&F, H, W, 1, 1, emin, emax, ident);
    double* ray = (double*)malloc(sizeof(double) * 3 * HW);
    double* X = (double*)malloc(sizeof(double) * 3 * HW);
    double* gX = (double*)calloc(3 * HW, sizeof(double));
    double* eX = (double*)calloc(HW, sizeof(double));      /* sum of rho |g| per pixel */
    double rho_sum = 0.0;
    for (int r = 0; r < H; ++r)
        for (int c = 0; c < W; ++c) {
            int64_t p = (int64_t)r * W + c;
            pixel_ray(&F, r, c, ray + 3 * p);
            double Dh = St[p] / (A[p] + EPS_A);
            for (int k = 0; k < 3; ++k) X[3 * p + k] = Dh * ray[3 * p + k];
        }
    const double k = lam / (double)nd;
    double sum = 0.0;
    for (int r = 0; r + 1 < H; ++r)
        for (int c = 0; c < W; ++c) {
            int64_t p = (int64_t)r * W + c, pr = (int64_t)r * W + (c + 1) % W, pb = p + W;
            if (!(D[p] > 0.0f && D[pr] > 0.0f && D[pb] > 0.0f)) continue;
            if (!(A[p] > 0.0 && A[pr] > 0.0 && A[pb] > 0.0)) continue;
            double ec[3], er[3], cr[3];
            for (int q = 0; q < 3; ++q) {
                ec[q] = X[3 * pr + q] - X[3 * p + q];
                er[q] = X[3 * pb + q] - X[3 * p + q];
            }
            cross3(ec, er, cr);
            double mc = sqrt(dot3(cr, cr) + EPS_N * EPS_N);
            double ns[3] = { cr[0] / mc, cr[1] / mc, cr[2] / mc };
            double sn[3] = { Sn[p], Sn[HW + p], Sn[2 * HW + p] };
            double m = sqrt(dot3(sn, sn) + EPS_N * EPS_N);
            double nh[3] = { sn[0] / m, sn[1] / m, sn[2] / m };
            sum += 1.0 - dot3(nh, ns);
            /* dL/dNh = -k N_surf through Nh = S_n/m */
            double g[3] = { -k * ns[0], -k * ns[1], -k * ns[2] };
            double sg = dot3(sn, g);
            for (int q = 0; q < 3; ++q) gSn[q * HW + p] += scale * (g[q] / m - sn[q] * sg / (m * m * m));
            /* dL/dN_surf = -k Nh through N_surf = cr/mc, then cr = e_c x e_r:
               dL/de_c = e_r x gcr, dL/de_r = gcr x e_c */
            double gc[3] = { -k * nh[0], -k * nh[1], -k * nh[2] };
            double cg = dot3(cr, gc);
            double gcr[3] = { gc[0] / mc - cr[0] * cg / (mc * mc * mc), gc[1] / mc - cr[1] * cg / (mc * mc * mc),
                              gc[2] / mc - cr[2] * cg / (mc * mc * mc) };
            double gec[3], ger[3];
            cross3(er, gcr, gec);
            cross3(gcr, ec, ger);
            for (int q = 0; q < 3; ++q) {
                gX[3 * pr + q] += gec[q];
                gX[3 * pb + q] += ger[q];
                gX[3 * p + q] -= gec[q] + ger[q];
            }
            if (err) {
                const double U = 0x1p-24;
                double xp = sqrt(dot3(X + 3 * p, X + 3 * p)), xr = sqrt(dot3(X + 3 * pr, X + 3 * pr));
                double xb = sqrt(dot3(X + 3 * pb, X + 3 * pb));
                double rho = U * (12.0 * ((xp + xr) * sqrt(dot3(er, er)) + sqrt(dot3(ec, ec)) * (xp + xb)) /
                                  sqrt(dot3(cr, cr) + 1e-300) + 8.0);
                double gx = rho * k / mc * (sqrt(dot3(ec, ec)) + sqrt(dot3(er, er)));
                eX[pr] += gx;
                eX[pb] += gx;
                eX[p] += 2.0 * gx;
                err[HW + p] = rho * scale * k / m;
                rho_sum += rho;
            }
        }
    /* X = Dh d, Dh = S_t/(A+eps) */
    for (int64_t p = 0; p < HW; ++p) {
        double gD = dot3(gX + 3 * p, ray + 3 * p);
        if (gD == 0.0) continue;
        double a = A[p] + EPS_A;
        gSt[p] += scale * gD / a;
        gA[p] += scale * (-gD * St[p] / (a * a));
    }
    if (err) {
        for (int64_t p = 0; p < HW; ++p) err[p] = scale * eX[p];
        err[2 * HW] = rho_sum / (double)nd;
    }
    free(ray); free(X); free(gX); free(eX);
    return sum / (double)nd;
}

/* L_scale = sum_i max(0, max(s_i0, s_i1) - s_max), s = exp(log-scale); returns
 * lam_s L_scale and accumulates lam_s dL_scale/d(log-scale) (+=).  For equal
 * scales the subgradient goes to the first component. */
double lgso_scale_reg(const double* ls, int64_t n, double s_max, double lam_s, double* dls)
{
    double L = 0;
    for (int64_t i = 0; i < n; ++i) {
        double s0 = exp(ls[2 * i]), s1 = exp(ls[2 * i + 1]);
        int first = s0 >= s1;
        double sm = first ? s0 : s1;
        if (sm > s_max) {
            L += sm - s_max;
            if (dls) dls[2 * i + (first ? 0 : 1)] += lam_s * sm;
        }
    }
    return lam_s * L;
}
