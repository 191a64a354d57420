/*
 * lgs_oracle_impl.h -- internal types and functions shared by the two
 * translation units of the CPU oracle (TEST INFRASTRUCTURE ONLY):
 *
 *   lgs_oracle.c          the method: binary32 binning, FP64 rendering of the
 *                         surfels (Sec. 3.1), the mapping losses and their
 *                         analytic reverse mode (Sec. 3.4);
 *   lgs_fp32_allowance.c  what a binary32 evaluation of the same inputs may
 *                         differ by (the parity tests' allowance), computed by
 *                         re-walking the method's own evaluations.
 *
 * The method never reads anything the allowance computes.  Nothing here is
 * shared with the CUDA library.
 */
#ifndef LGS_ORACLE_IMPL_H
#define LGS_ORACLE_IMPL_H

#include <stdint.h>

#define OI_INTERNAL __attribute__((visibility("hidden")))

/* The method's constants (readings of the paper listed in the design notes). */
#define T_NEAR   0.2          /* ray parameter must exceed this (m)           */
#define Q_CUT    9.0          /* Gaussian support: u^2+v^2 <= 9 (3 sigma)      */
#define A_MIN    (1.0 / 255.0)/* contributions below this opacity are skipped  */
#define A_MAX    0.99         /* per-surfel opacity clamp                      */
#define T_STOP   1e-4         /* stop before T would drop below this           */
#define DEN_EPS  1e-6         /* grazing rays |n.d| < DEN_EPS are skipped       */
#define EPS_A    1e-6         /* D = S_t / (A + EPS_A)                         */
#define EPS_N    1e-6         /* N = S_n / sqrt(|S_n|^2 + EPS_N^2)             */
#define EPS_LOG  1e-6         /* L_alpha = -mean log(A + EPS_LOG)              */

typedef struct {
    double mu[3], tu[3], tv[3], n[3];   /* sensor frame */
    double su, sv, alpha;
    double qh[4], qnorm;                /* unit quaternion (w,x,y,z), |q| */
} surf64;

typedef struct {
    int H, W, th, tw, ntr, ntc;
    double emin, emax, R[9], o[3];
} frame64;

/* One ray / surfel evaluation (valid = composited if reached). */
typedef struct { int valid; double den, t, x[3], u, v, q, G, araw, a; } eval64;

/* One pixel's compositing: outputs, the list position after its last
 * contributor (ncontrib) and the number of list entries evaluated. */
typedef struct {
    double A, St, Sn[3], T;
    int32_t ncontrib;
    int64_t neval;
} pix_out;

/* gradient w.r.t. the sensor-frame surfel quantities */
typedef struct { double mu[3], tu[3], tv[3], n[3], su, sv, alpha; } sgrad;

static inline double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

/* ---- the method (lgs_oracle.c) ------------------------------------------ */
OI_INTERNAL void make_frame(frame64* F, int H, int W, int th, int tw, double emin, double emax, const double* pose);
OI_INTERNAL surf64* sensor_surfels(const double* mean, const double* quat, const double* ls, const double* logit,
                                   int64_t n, const frame64* F);
OI_INTERNAL void pixel_ray(const frame64* F, int r, int c, double* d);
OI_INTERNAL void eval_pair(const surf64* s, const double* d, eval64* e);
OI_INTERNAL int composite_pixel(const surf64* S, const uint32_t* list, int64_t len, const double* d, pix_out* o,
                                int64_t* ck, double* cT);
OI_INTERNAL double contrib_grad(const surf64* s, const eval64* e, const double* d, double T, double suffix,
                                double gA, double gSt, const double* gSn, int use_clamp, sgrad* g);
OI_INTERNAL void chain_to_params(const surf64* s, const sgrad* g, const frame64* F, double* dmean, double* dquat,
                                 double* dls, double* dlogit);
OI_INTERNAL void rot_jacobian(const double* q, double J[9][4]);

/* ---- the binary32 allowance (lgs_fp32_allowance.c) ---------------------- */
/* Per-pixel state of the allowance: near-threshold flags of the pixel and the
 * opacities (and opacity x depth) whose decision may flip. */
typedef struct {
    int flags;
    double flipA, flipAt, flipa, flipTmax;
} pix_unc;

/* Forward allowance of one pixel, given the method's compositing o (nc
 * contributors at list positions ck[] with transmittance cT[] before each):
 * the pixel's flags and the bounds eA (accumulated opacity), eD (depth). */
OI_INTERNAL void fwd_allowance(const surf64* S, const uint32_t* list, const double* d, const pix_out* o, int nc,
                               const int64_t* ck, const double* cT, pix_unc* u, double* eA, double* eD);

/* Per-contributor record of bwd_allowance, for the tests that pin it (any
 * pointer may be NULL; arrays indexed by contributor m, [m][10] for raw
 * parameters): the contribution's raw-parameter gradient, its contrib_unc
 * and majorant, the transmittance before it and the suffix over the later
 * contributors with their binary32 uncertainties (relative eT, absolute dS). */
typedef struct {
    double *grad, *gunc, *gmaj, *T, *S, *eT, *dS;
} bwd_detail;

/* Gradient allowance of one pixel (upstream gA, gSt, gSn): accumulates per
 * surfel and raw parameter the majorant (gabs) and the binary32 uncertainty
 * (gflip) of its contributions.  Scratch: tmp [10 * maxlen], suf, et [maxlen].
 * det: NULL, or the per-contributor record above. */
OI_INTERNAL void bwd_allowance(const surf64* S, const uint32_t* list, const double* d, int nc, const int64_t* ck,
                               const double* cT, const pix_out* o, const pix_unc* u, double gA, double gSt,
                               const double* gSn, const frame64* F, double* gabs, double* gflip, double* tmp,
                               double* suf, double* et, const bwd_detail* det);

#endif
