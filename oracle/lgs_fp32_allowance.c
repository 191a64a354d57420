/*
 * lgs_fp32_allowance.c -- the binary32 allowance of the oracle's outputs
 * (TEST INFRASTRUCTURE ONLY; not part of the method).
 *
 * The GPU evaluates the method in binary32 from the same binary32 inputs the
 * oracle evaluates in FP64.  A binary32 evaluation sees the sensor-frame
 * geometry and the rays rounded to 24 bits, so it may differ from the FP64
 * value by an amount that depends on the conditioning of each evaluation,
 * and it may take a decision that lies near a threshold (the skip rules, the
 * opacity clamp, the early stop) the other way.  This file bounds both, per
 * pixel (opacity, depth) and per surfel gradient, by re-walking the
 * evaluations the method made (lgs_oracle.c) -- it never changes them.  The
 * parity tests add these bounds to their bars; tests/test_fp32_allowance.py
 * checks them against a plain binary32 restatement of the evaluation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#include "lgs_oracle_impl.h"

#define FLAG_REL 1e-3         /* band around a threshold that flags a pixel    */
#define DEN_FLAG 1e-5         /* |n.d| below this flags a pixel                 */
#define EPS32    5.9604644775390625e-08  /* 2^-24, unit roundoff of binary32  */

/* Planted mistakes (tests only): a factor on one bound, selected at build
 * time, so that a test can show that its pins catch a bound that is too
 * small or too large.  All are 1 in the oracle the tests use. */
#ifndef PLANT_EK
#define PLANT_EK 1.0          /* local-coordinate uncertainties eu, ev         */
#endif
#ifndef PLANT_DT
#define PLANT_DT 1.0          /* ray-parameter uncertainty dt of fp32_unc      */
#endif
#ifndef PLANT_EA
#define PLANT_EA 1.0          /* opacity bound eA of fwd_allowance             */
#endif
#ifndef PLANT_ED
#define PLANT_ED 1.0          /* depth bound eD of fwd_allowance               */
#endif
#ifndef PLANT_OPA
#define PLANT_OPA 1.0         /* opacity_unc                                   */
#endif
#ifndef PLANT_CONTRIB
#define PLANT_CONTRIB 1.0     /* contrib_unc                                   */
#endif
#ifndef PLANT_FLIP
#define PLANT_FLIP 1.0        /* flip_opacity                                  */
#endif
#ifndef PLANT_MAJOR
#define PLANT_MAJOR 1.0       /* the majorant (raw_major)                      */
#endif

enum { FL_DEN = 1, FL_TNEAR = 2, FL_QCUT = 4, FL_AMIN = 8, FL_AMAX = 16, FL_TSTOP = 32 };
/* A grazing decision (|n.d| near 1e-6) may admit a surfel at an unbounded
 * ray parameter: its gradient is undetermined.  The other near-threshold
 * decisions (the near plane, the cut-off, the 1/255 skip) are bounded by the
 * contribution they may add or drop. */
#define FL_HARD FL_DEN
#define FL_SOFT (FL_TNEAR | FL_QCUT | FL_AMIN)

static int near_thr(double v, double thr) { return fabs(v - thr) <= FLAG_REL * fabs(thr); }

/* Binary32 uncertainty of one evaluation.  A binary32 evaluation forms the
 * sensor-frame geometry from binary32 parameters (the axes from a normalised
 * quaternion, the centre and axes through the pose) and the ray from its
 * elevation and azimuth, so each coordinate carries a few roundings: a unit
 * axis about 4 EPS32 per component, the centre about 2 EPS32 |mu|, the ray
 * about 1.5 EPS32.  Then n.d (three products and two sums more) is known to
 * about 7 EPS32, h = n.mu to about 4 EPS32 |mu| (the errors of n and mu
 * partly cancel; a plain binary32 restatement of the pipeline never exceeds
 * 4, tests/test_fp32_allowance.py), and the ray parameter t = h/(n.d) has
 * relative uncertainty
 *   dt/t = EPS32 (1 + 7/|n.d| + 4 |mu|/|h|),
 * and a local coordinate u = t (t_u.d)/s_u - (t_u.mu)/s_u, of terms up to
 * max(t,|mu|)/s_u, absolute uncertainty
 *   eu   = EPS32 max(t, |mu|)/s_u (1 + 7/|n.d| + 4 |mu|/|h|)
 * (ev the same with s_v). */
#define DEN_UNC (7.0 * EPS32)
static void fp32_unc(const surf64* s, double den, double t, double* eu, double* ev, double* dt)
{
    double g = 1.0 / fabs(den);
    double rho = sqrt(dot3(s->mu, s->mu));
    double h = fabs(t * den);
    double hr = rho / (h > 1e-30 ? h : 1e-30);
    double k = 1.0 + 7.0 * g + 4.0 * hr;
    double c = PLANT_EK * EPS32 * (fabs(t) > rho ? fabs(t) : rho) * k;
    *eu = c / s->su;
    *ev = c / s->sv;
    *dt = PLANT_DT * fabs(t) * EPS32 * k;
}

/* Near-threshold flags of the method's evaluation e: a decision is "near"
 * its threshold when it lies within the larger of FLAG_REL and a few times
 * the binary32 uncertainty of the quantity it tests (only the quantities the
 * method formed before a skip are tested). */
static int eval_flags(const surf64* s, const eval64* e)
{
    int f = 0;
    if (fabs(e->den) <= DEN_FLAG) f |= FL_DEN;
    if (fabs(e->den) < DEN_EPS) return f;
    double eu, ev, dt;
    fp32_unc(s, e->den, e->t, &eu, &ev, &dt);
    if (fabs(e->t - T_NEAR) <= FLAG_REL * T_NEAR + 4.0 * dt) f |= FL_TNEAR;
    if (e->t <= T_NEAR) return f;
    double dq = 2.0 * (fabs(e->u) * eu + fabs(e->v) * ev);
    if (fabs(e->q - Q_CUT) <= FLAG_REL * Q_CUT + 4.0 * dq) f |= FL_QCUT;
    if (e->q > Q_CUT) return f;
    double da = e->araw * (2.0 * dq + 4.0 * EPS32);     /* relative error of G is dq/2 */
    if (fabs(e->araw - A_MAX) <= FLAG_REL * A_MAX + da) f |= FL_AMAX;
    if (fabs(e->a - A_MIN) <= FLAG_REL * A_MIN + da) f |= FL_AMIN;
    return f;
}

/* The same quantities as eval_pair with no skip applied (t, u, v, q, G, a
 * computed whatever the thresholds say); used to size the contribution of a
 * near-threshold evaluation that a binary32 evaluation may decide otherwise. */
static void force_eval(const surf64* s, const double* d, eval64* e)
{
    e->den = dot3(s->n, d);
    e->t = dot3(s->n, s->mu) / e->den;
    for (int k = 0; k < 3; ++k) e->x[k] = e->t * d[k] - s->mu[k];
    e->u = dot3(s->tu, e->x) / s->su;
    e->v = dot3(s->tv, e->x) / s->sv;
    e->q = e->u * e->u + e->v * e->v;
    e->G = exp(-0.5 * e->q);
    e->araw = s->alpha * e->G;
    e->a = e->araw < A_MAX ? e->araw : A_MAX;
    e->valid = 1;
}

static double opacity_unc(const surf64* s, const eval64* e);

/* Opacity (and ray parameter) the evaluation would have if its skip decision
 * went the other way: a FP32 evaluation may decide a near-threshold case
 * differently, and this is the size of what then changes (the opacity with
 * its own binary32 uncertainty, since the flipped evaluation sees slightly
 * different u, v).  A grazing decision may admit the surfel at its full
 * opacity. */
static double would_be_a(const surf64* s, const double* d, const eval64* e, int flags, double* t)
{
    if (flags & FL_HARD) {
        *t = fabs(dot3(s->n, s->mu) / e->den);
        return s->alpha < A_MAX ? s->alpha : A_MAX;
    }
    eval64 f;
    force_eval(s, d, &f);
    *t = fabs(f.t);
    double a = f.a + opacity_unc(s, &f);
    return a < A_MAX ? a : A_MAX;
}

/* Error bound of a pixel's outputs implied by binary32 representation of
 * its inputs.  A binary32 evaluation sees every sensor-frame coordinate and
 * ray component rounded to 24 bits; a local coordinate u = t_u.(t d - mu)/s
 * then carries an error of about EPS32 max(t, |mu|)/s, amplified by 1/|n.d|
 * through t = (n.mu)/(n.d).  With e_k that error for contributor k:
 *   da_k = a_k ((|u_k| + |v_k|) e_k + 4 EPS32),  dt_k = t_k EPS32 (2 + 2/|n.d|),
 *   eA   = sum_k T_k da_k                      (|dA/da_k| <= T_k)
 *   eD   = sum_k |dD/da_k| da_k + w_k dt_k / (A + 1e-6),
 *   dD/da_k = [T_k (t_k - D) - sum_{j>k} w_j (t_j - D)/(1 - a_k)] / (A + 1e-6),
 * plus the opacities whose decision lies near a threshold (flipA, flipAt). */
void fwd_allowance(const surf64* S, const uint32_t* list, const double* d, const pix_out* o, int nc,
                   const int64_t* ck, const double* cT, pix_unc* u, double* eA, double* eD)
{
    /* the method's walk again: flags, and the opacity that a near-threshold
     * decision may add or drop, with the transmittance at that point */
    u->flags = 0; u->flipA = 0; u->flipAt = 0; u->flipa = 0; u->flipTmax = 0;
    double T = 1.0;
    for (int64_t k = 0; k < o->neval; ++k) {
        const surf64* s = S + list[k];
        eval64 e;
        eval_pair(s, d, &e);
        int fl = eval_flags(s, &e);
        u->flags |= fl;
        if (fl & (FL_DEN | FL_TNEAR | FL_QCUT | FL_AMIN)) {
            double tw, aw = PLANT_FLIP * would_be_a(s, d, &e, fl, &tw);
            u->flipA += T * aw;
            u->flipAt += T * aw * tw;
            u->flipa += aw;
            if (tw > u->flipTmax) u->flipTmax = tw;
        }
        if (!e.valid) continue;
        double Tn = T * (1.0 - e.a);
        if (near_thr(Tn, T_STOP)) {
            u->flags |= FL_TSTOP;
            u->flipA += T * PLANT_FLIP * e.a;
            u->flipAt += T * PLANT_FLIP * e.a * e.t;
            u->flipa += PLANT_FLIP * e.a;
            if (fabs(e.t) > u->flipTmax) u->flipTmax = fabs(e.t);
        }
        if (Tn < T_STOP) break;
        T = Tn;
    }
    double Dh = o->St / (o->A + EPS_A);
    double ea = 0, ed = 0, suffix = 0;
    for (int m = nc - 1; m >= 0; --m) {
        const surf64* s = S + list[ck[m]];
        eval64 e;
        eval_pair(s, d, &e);
        double Tm = cT[m], w = e.a * Tm;
        double eu, ev, dt;
        fp32_unc(s, e.den, e.t, &eu, &ev, &dt);
        double da = e.a * (fabs(e.u) * eu + fabs(e.v) * ev + 4.0 * EPS32);
        ea += Tm * da;
        double dDda = (Tm * fabs(e.t - Dh) + suffix / (1.0 - e.a)) / (o->A + EPS_A);
        ed += dDda * da + w * dt / (o->A + EPS_A);
        suffix += w * fabs(e.t - Dh);
    }
    /* decisions within FLAG_REL of a threshold: the contribution that may
     * flip; the depth, a weighted mean of the contributors' depths, moves by
     * at most the larger of them and the current one */
    ea += u->flipA;
    if (u->flipA > 0) ed += fmin((u->flipAt + Dh * u->flipA) / (o->A + EPS_A), u->flipTmax + Dh);
    *eA = PLANT_EA * ea;
    *eD = PLANT_ED * ed;
}

/* The sensor-frame chain of contrib_grad (lgs_oracle.c) with every term of
 * g.c and dL/da in absolute value: the magnitudes a binary32 evaluation
 * rounds, whatever cancels.  Adds into *g and returns the majorant of g.c. */
static double contrib_grad_major(const surf64* s, const eval64* e, const double* d, double T, double suffix,
                                 double gA, double gSt, const double* gSn, sgrad* g)
{
    double gc = fabs(gA) + fabs(gSt * e->t) + fabs(gSn[0]) + fabs(gSn[1]) + fabs(gSn[2]);
    double w = e->a * T;
    double dLda = T * gc + fabs(suffix) / (1.0 - e->a);
    double aSt = fabs(gSt);
    double dLdt = w * aSt;
    for (int k = 0; k < 3; ++k) g->n[k] += w * fabs(gSn[k]);
    double dLdu = 0, dLdv = 0;
    if (e->araw < A_MAX) {
        g->alpha += dLda * e->G;
        double dLdq = dLda * s->alpha * (-0.5 * e->G);
        dLdu = dLdq * 2.0 * e->u;
        dLdv = dLdq * 2.0 * e->v;
    }
    dLdt += dLdu * dot3(s->tu, d) / s->su + dLdv * dot3(s->tv, d) / s->sv;
    for (int k = 0; k < 3; ++k) {
        g->tu[k] += dLdu * e->x[k] / s->su;
        g->tv[k] += dLdv * e->x[k] / s->sv;
        g->mu[k] -= dLdu * s->tu[k] / s->su + dLdv * s->tv[k] / s->sv;
    }
    g->su -= dLdu * e->u / s->su;
    g->sv -= dLdv * e->v / s->sv;
    for (int k = 0; k < 3; ++k) {
        g->mu[k] += dLdt * s->n[k] / e->den;
        g->n[k] += dLdt * (s->mu[k] - e->t * d[k]) / e->den;
    }
    return gc;
}

/* |raw-parameter gradient| (mean 3, quat 4, log-scale 2, logit 1) of one contribution */
static void raw_abs(const surf64* s, const sgrad* g, const frame64* F, double* r)
{
    double dm[3] = { 0, 0, 0 }, dq[4] = { 0, 0, 0, 0 }, dl[2] = { 0, 0 }, dg = 0;
    chain_to_params(s, g, F, dm, dq, dl, &dg);
    for (int k = 0; k < 3; ++k) r[k] = fabs(dm[k]);
    for (int k = 0; k < 4; ++k) r[3 + k] = fabs(dq[k]);
    r[7] = fabs(dl[0]); r[8] = fabs(dl[1]); r[9] = fabs(dg);
}


/* Majorant of the raw-parameter gradient of one contribution: the chain of
 * chain_to_params with every product in absolute value, i.e. the sum of the
 * magnitudes that a binary32 evaluation of the chain adds up (a rotation of an
 * isotropic surfel about its normal, for one, cancels exactly in FP64 but not
 * in binary32). */
static void raw_major(const surf64* s, const sgrad* g, const frame64* F, double* r)
{
    double dcol[3][3];
    for (int a = 0; a < 3; ++a) {
        double gm = 0, g0 = 0, g1 = 0, g2 = 0;
        for (int k = 0; k < 3; ++k) {
            double R = fabs(F->R[3 * a + k]);
            gm += R * fabs(g->mu[k]);
            g0 += R * fabs(g->tu[k]);
            g1 += R * fabs(g->tv[k]);
            g2 += R * fabs(g->n[k]);
        }
        r[a] = gm;
        dcol[0][a] = g0; dcol[1][a] = g1; dcol[2][a] = g2;
    }
    double J[9][4];
    rot_jacobian(s->qh, J);
    double dqh[4] = { 0, 0, 0, 0 };
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            for (int c = 0; c < 4; ++c) dqh[c] += dcol[b][a] * fabs(J[3 * a + b][c]);
    double pr = 0;
    for (int c = 0; c < 4; ++c) pr += dqh[c] * fabs(s->qh[c]);
    for (int c = 0; c < 4; ++c) r[3 + c] = (dqh[c] + fabs(s->qh[c]) * pr) / s->qnorm;
    r[7] = fabs(g->su) * s->su;
    r[8] = fabs(g->sv) * s->sv;
    r[9] = fabs(g->alpha) * s->alpha * (1.0 - s->alpha);
    for (int c = 0; c < 10; ++c) r[c] *= PLANT_MAJOR;
}


/* The evaluation e with its local coordinates moved by (du, dv), its depth by
 * dtt and n.d by dden, the skip and clamp decisions kept: the inputs a
 * binary32 evaluation may see instead of e's (u and v are absolute
 * uncertainties, so terms proportional to a small u, v or offset x are
 * covered too). */
static void perturb_eval(const surf64* s, const eval64* e, double du, double dv, double dtt, double dden,
                         eval64* p)
{
    *p = *e;
    p->den = e->den + dden;
    p->t = e->t + dtt;
    p->u = e->u + du;
    p->v = e->v + dv;
    for (int k = 0; k < 3; ++k) p->x[k] = e->x[k] + du * s->su * s->tu[k] + dv * s->sv * s->tv[k];
    p->q = p->u * p->u + p->v * p->v;
    p->G = exp(-0.5 * p->q);
    p->araw = s->alpha * p->G;
    p->a = e->araw < A_MAX ? p->araw : A_MAX;
}


static void add10(double* dst, const double* r, double f)
{
    for (int c = 0; c < 10; ++c) {
#ifdef _OPENMP
#pragma omp atomic
#endif
        dst[c] += f * r[c];
    }
}


/* First-order binary32 uncertainty of the opacity of one evaluation: a
 * re-derived with u, v moved by their uncertainties eu, ev, t by dt and n.d
 * by DEN_UNC, the changes added in absolute value, plus 4 ulp of rounding. */
static double opacity_unc(const surf64* s, const eval64* e)
{
    double eu, ev, dt;
    fp32_unc(s, e->den, e->t, &eu, &ev, &dt);
    const double dden = e->den > 0 ? DEN_UNC : -DEN_UNC;
    const double steps[4][4] = { { eu, 0, 0, 0 }, { 0, ev, 0, 0 }, { 0, 0, dt, 0 }, { 0, 0, 0, dden } };
    double da = 4.0 * EPS32 * e->a;
    for (int k = 0; k < 4; ++k) {
        eval64 p;
        perturb_eval(s, e, steps[k][0], steps[k][1], steps[k][2], steps[k][3], &p);
        da += fabs(p.a - e->a);
    }
    return PLANT_OPA * da;
}


/* First-order binary32 uncertainty of one contribution c0 (into r[10], raw
 * parameters): c0 re-derived with u, v moved by their uncertainties eu, ev, t
 * by dt, n.d by DEN_UNC, the transmittance T by the relative amount eT and the
 * suffix by dS, the six changes added in absolute value.  Propagating the
 * inputs' errors this way (instead of scaling a majorant) keeps the size of
 * cancelling upstream terms out of the bound, and keeps terms proportional to
 * a small u, v or offset x in it. */
static void contrib_unc(const surf64* s, const eval64* e, const double* d, double T, double suffix, double eT,
                        double dS, double gA, double gSt, const double* gSn, const frame64* F, const sgrad* c0,
                        double* r)
{
    double eu, ev, dt;
    fp32_unc(s, e->den, e->t, &eu, &ev, &dt);
    const double dden = e->den > 0 ? DEN_UNC : -DEN_UNC;
    const double steps[4][4] = { { eu, 0, 0, 0 }, { 0, ev, 0, 0 }, { 0, 0, dt, 0 }, { 0, 0, 0, dden } };
    for (int c = 0; c < 10; ++c) r[c] = 0;
    for (int k = 0; k < 6; ++k) {
        eval64 p;
        double Tk = T, Sk = suffix;
        if (k < 4) perturb_eval(s, e, steps[k][0], steps[k][1], steps[k][2], steps[k][3], &p);
        else p = *e;
        if (k == 4) Tk = T * (1.0 + eT);
        if (k == 5) Sk = suffix + dS;
        sgrad g;
        memset(&g, 0, sizeof(g));
        contrib_grad(s, &p, d, Tk, Sk, gA, gSt, gSn, 1, &g);
        for (int j = 0; j < 3; ++j) {
            g.mu[j] -= c0->mu[j]; g.tu[j] -= c0->tu[j]; g.tv[j] -= c0->tv[j]; g.n[j] -= c0->n[j];
        }
        g.su -= c0->su; g.sv -= c0->sv; g.alpha -= c0->alpha;
        double q[10];
        raw_abs(s, &g, F, q);
        for (int c = 0; c < 10; ++c) r[c] += PLANT_CONTRIB * q[c];
    }
}

/* Opacity that a binary32 evaluation may add or drop at a near-threshold
 * decision of evaluated entry k of a pixel (contributor or not; 0 if none):
 * fl are the entry's flags, pflags the pixel's. */
static double flip_opacity(const surf64* s, const double* d, const eval64* e, int fl, int pflags, int is_contrib,
                           int last_contrib, int stop_entry)
{
    int tstop = (pflags & FL_TSTOP) != 0;
    if (is_contrib) {
        if ((fl & FL_SOFT) || (tstop && last_contrib)) return PLANT_FLIP * e->a;
        if (fl & FL_AMAX) return PLANT_FLIP * fabs(e->araw - A_MAX);
        return 0.0;
    }
    if ((fl & FL_SOFT) || (tstop && stop_entry)) {
        eval64 f;
        force_eval(s, d, &f);
        return PLANT_FLIP * f.a;
    }
    return 0.0;
}

/* Gradient allowance of one pixel with upstream gradients (gA, gSt, gSn) of
 * (A, S_t, S_n), re-walking the method's reverse pass (backward_pixel in
 * lgs_oracle.c).  Per surfel and raw parameter it accumulates:
 *   gabs  += a majorant of each contribution (its terms in absolute value:
 *            the conditioning of the sums and of the chain to the raw
 *            parameters);
 *   gflip += twice the first-order change of the contribution under the
 *            binary32 uncertainties of its inputs (contrib_unc: u, v, t, n.d,
 *            the transmittance before it and the suffix after it, where a
 *            near-threshold decision of another entry counts as an
 *            uncertainty of its whole opacity), and
 *   gflip += what a near-threshold decision of the surfel's own can change:
 *            its whole would-be contribution; a grazing or near-plane
 *            decision makes the surfel's value undetermined (gflip = inf). */
void bwd_allowance(const surf64* S, const uint32_t* list, const double* d, int nc, const int64_t* ck,
                   const double* cT, const pix_out* o, const pix_unc* u, double gA, double gSt,
                   const double* gSn, const frame64* F, double* gabs, double* gflip, double* tmp,
                   double* suf, double* et, const bwd_detail* det)
{
    double suffix = 0.0, suffix_abs = 0.0, dS = 0.0;
    /* et[m]: relative uncertainty of the transmittance before contributor m:
     * the earlier opacities' binary32 uncertainties, the opacities that a
     * near-threshold decision may add or drop, and the roundings of the
     * products / quotients that carry it */
    {
        double acc = 2.0 * nc * EPS32;
        int mm = 0;
        for (int64_t k = 0; k < o->neval; ++k) {
            const surf64* s = S + list[k];
            int is_contrib = mm < nc && ck[mm] == k;
            eval64 e;
            eval_pair(s, d, &e);
            int fl = eval_flags(s, &e);
            int stop_entry = (k == o->neval - 1) && !is_contrib && e.valid;
            double fa = flip_opacity(s, d, &e, fl, u->flags, is_contrib, mm == nc - 1, stop_entry);
            if (is_contrib) {
                et[mm++] = acc;
                acc += (opacity_unc(s, &e) + fa) / (1.0 - e.a);
            } else if (fa > 0) {
                acc += fa / (1.0 - fa);
            }
        }
    }
    int mm = nc - 1;
    for (int64_t k = o->neval - 1; k >= 0; --k) {
        uint32_t i = list[k];
        const surf64* s = S + i;
        eval64 e;
        eval_pair(s, d, &e);                   /* the method's evaluation */
        int fl = eval_flags(s, &e);
        if (mm < 0 || ck[mm] != k) {
            /* not composited: a near-threshold entry may still be in binary32,
             * adding its term to the suffix of the contributors before it */
            int stop_entry = (k == o->neval - 1) && e.valid;
            double fa = flip_opacity(s, d, &e, fl, u->flags, 0, 0, stop_entry);
            if (fa > 0) {
                eval64 f;
                force_eval(s, d, &f);
                double np = f.den > 0 ? -1.0 : 1.0;
                double gcw = gA + gSt * f.t + np * dot3(gSn, s->n);
                dS += fa * (mm + 1 < nc ? cT[mm + 1] : o->T) * fabs(gcw);
            }
            continue;
        }
        const int m = mm--;
        double T = cT[m];
        sgrad c;
        memset(&c, 0, sizeof(c));
        double gc = contrib_grad(s, &e, d, T, suffix, gA, gSt, gSn, 1, &c);   /* the method's contribution */
        suffix += e.a * T * gc;
        suf[m] = suffix;                       /* sum over contributors >= m */
        {
            sgrad cm;
            memset(&cm, 0, sizeof(cm));
            double gcm = contrib_grad_major(s, &e, d, T, suffix_abs, gA, gSt, gSn, &cm);
            suffix_abs += e.a * T * gcm;
            raw_major(s, &cm, F, tmp + 10 * m);
            add10(gabs + 10 * (int64_t)i, tmp + 10 * m, 1.0);
        }
        {
            double r[10], eu, ev, dt;
            /* suffix - w gc: the suffix over the later contributors only */
            contrib_unc(s, &e, d, T, suffix - e.a * T * gc, et[m], dS, gA, gSt, gSn, F, &c, r);
            add10(gflip + 10 * (int64_t)i, r, 2.0);
            /* this term's own uncertainty, for the contributors before it */
            if (det) {
                if (det->grad) {
                    double dm[3] = { 0, 0, 0 }, dq[4] = { 0, 0, 0, 0 }, dl[2] = { 0, 0 }, dg = 0;
                    chain_to_params(s, &c, F, dm, dq, dl, &dg);
                    double* gg = det->grad + 10 * m;
                    for (int q = 0; q < 3; ++q) gg[q] = dm[q];
                    for (int q = 0; q < 4; ++q) gg[3 + q] = dq[q];
                    gg[7] = dl[0]; gg[8] = dl[1]; gg[9] = dg;
                }
                if (det->gunc) memcpy(det->gunc + 10 * m, r, sizeof(r));
                if (det->gmaj) memcpy(det->gmaj + 10 * m, tmp + 10 * m, 10 * sizeof(double));
                if (det->T) det->T[m] = T;
                if (det->S) det->S[m] = suffix - e.a * T * gc;
                if (det->eT) det->eT[m] = et[m];
                if (det->dS) det->dS[m] = dS;
            }
            fp32_unc(s, e.den, e.t, &eu, &ev, &dt);
            double w = e.a * T;
            double fa = flip_opacity(s, d, &e, fl, u->flags, 1, m == nc - 1, 0);
            dS += (opacity_unc(s, &e) + fa) * T * fabs(gc) + w * fabs(gSt) * dt + et[m] * fabs(w * gc);
        }
        if (fl & FL_AMAX) {
            sgrad g;
            memset(&g, 0, sizeof(g));
            double r[10];
            contrib_grad(s, &e, d, T, m + 1 < nc ? suf[m + 1] : 0.0, gA, gSt, gSn, 0, &g);
            raw_abs(s, &g, F, r);
            add10(gflip + 10 * (int64_t)i, r, PLANT_FLIP);
        }
    }
    if (!u->flags) return;
    if (u->flags & FL_TSTOP && nc > 0) add10(gflip + 10 * (int64_t)list[ck[nc - 1]], tmp + 10 * (nc - 1), PLANT_FLIP);
    /* the surfels whose own decision is near a threshold */
    mm = 0;
    for (int64_t k = 0; k < o->neval; ++k) {
        while (mm < nc && ck[mm] < k) ++mm;
        int is_contrib = mm < nc && ck[mm] == k;
        uint32_t i = list[k];
        const surf64* s = S + i;
        eval64 e;
        eval_pair(s, d, &e);
        int fl = eval_flags(s, &e);
        if (fl & FL_HARD) {
            for (int c = 0; c < 10; ++c) gflip[10 * (int64_t)i + c] = INFINITY;
            continue;
        }
        int stop_entry = (k == o->neval - 1) && !is_contrib && e.valid;
        if (!(fl & FL_SOFT) && !stop_entry) continue;
        if (is_contrib) {
            add10(gflip + 10 * (int64_t)i, tmp + 10 * mm, PLANT_FLIP);
            continue;
        }
        eval64 f;
        force_eval(s, d, &f);
        double T = mm < nc ? cT[mm] : o->T;
        double sx = mm < nc ? suf[mm] : 0.0;
        sgrad g;
        memset(&g, 0, sizeof(g));
        double r[10];
        contrib_grad(s, &f, d, T, sx, gA, gSt, gSn, 1, &g);
        raw_abs(s, &g, F, r);
        add10(gflip + 10 * (int64_t)i, r, PLANT_FLIP);
    }
}

/* ------------------------------------------------------------------------ */
/* Detail of one pixel, for the tests that pin the allowance                 */
/* ------------------------------------------------------------------------ */
/* For pixel (r, c) of a frame with the given tile lists and upstream
 * gradients (gA, gSt, gSn3) of the pixel: every evaluated list entry k
 * (k < returned count <= cap) with
 *   item[k], valid[k], flags[k] (near-threshold flags of the entry),
 *   contrib[k] (index m of the contributor, -1 if not composited),
 *   ev[k][8]  = den, t, u, v, q, G, a, araw of the method's evaluation
 *               (the quantities after a failed skip rule are those of an
 *               evaluation without skips),
 *   unc[k][4] = eu, ev, dt of fp32_unc and opacity_unc (valid entries),
 *   would[k]  = flip_opacity of the entry (0 if its decisions are calm);
 * per contributor m (< nc): the bwd_detail arrays (grad, gunc, gmaj [m][10],
 * T, S, eT, dS [m]); per pixel pix[8] = A, S_t, S_n (3), T_final, eA, eD and
 * pflags (the pixel's flags), nc_out (contributors).  Returns the number of
 * evaluated entries, or -1 if it exceeds cap. */
int64_t lgso_pixel_detail(const double* mean, const double* quat, const double* ls, const double* logit,
                          int64_t n, int H, int W, int th, int tw, double emin, double emax,
                          const double* pose, const int64_t* ranges, const uint32_t* vals, int r, int c,
                          double gA, double gSt, const double* gSn3, int64_t cap,
                          uint32_t* item, int32_t* valid, int32_t* flags, int32_t* contrib, double* ev,
                          double* unc, double* would, double* grad, double* gunc, double* gmaj, double* cTo,
                          double* So, double* eTo, double* dSo, double* pix, int32_t* pflags, int32_t* nc_out)
{
    frame64 F;
    make_frame(&F, H, W, th, tw, emin, emax, pose);
    surf64* S = sensor_surfels(mean, quat, ls, logit, n, &F);
    int64_t tile = (int64_t)(r / th) * F.ntc + c / tw;
    int64_t b = ranges[2 * tile], len = ranges[2 * tile + 1] - b;
    const uint32_t* list = vals + b;
    int64_t L = len > 0 ? len : 1;
    int64_t* ck = (int64_t*)malloc(sizeof(int64_t) * L);
    double* cT = (double*)malloc(sizeof(double) * L);
    double* tmp = (double*)malloc(sizeof(double) * 10 * L);
    double* suf = (double*)malloc(sizeof(double) * L);
    double* et = (double*)malloc(sizeof(double) * L);
    double* gabs = (double*)calloc((size_t)(n > 0 ? n : 1) * 10, sizeof(double));
    double* gflip = (double*)calloc((size_t)(n > 0 ? n : 1) * 10, sizeof(double));
    double d[3];
    pixel_ray(&F, r, c, d);
    pix_out o;
    int nc = composite_pixel(S, list, len, d, &o, ck, cT);
    int64_t ret = o.neval <= cap ? o.neval : -1;
    if (ret >= 0) {
        pix_unc u;
        double ea, ed;
        fwd_allowance(S, list, d, &o, nc, ck, cT, &u, &ea, &ed);
        bwd_detail det = { grad, gunc, gmaj, cTo, So, eTo, dSo };
        bwd_allowance(S, list, d, nc, ck, cT, &o, &u, gA, gSt, gSn3, &F, gabs, gflip, tmp, suf, et, &det);
        int mm = 0;
        for (int64_t k = 0; k < o.neval; ++k) {
            const surf64* s = S + list[k];
            eval64 e, f;
            eval_pair(s, d, &e);
            force_eval(s, d, &f);
            int fl = eval_flags(s, &e);
            int is_contrib = mm < nc && ck[mm] == k;
            item[k] = list[k];
            valid[k] = e.valid;
            flags[k] = fl;
            contrib[k] = is_contrib ? mm : -1;
            const eval64* q = e.valid ? &e : &f;
            double* o8 = ev + 8 * k;
            o8[0] = q->den; o8[1] = q->t; o8[2] = q->u; o8[3] = q->v; o8[4] = q->q; o8[5] = q->G; o8[6] = q->a;
            o8[7] = q->araw;
            double eu = 0, ev = 0, dt = 0, da = 0;
            if (e.valid) {
                fp32_unc(s, e.den, e.t, &eu, &ev, &dt);
                da = opacity_unc(s, &e);
            }
            unc[4 * k] = eu; unc[4 * k + 1] = ev; unc[4 * k + 2] = dt; unc[4 * k + 3] = da;
            int stop_entry = (k == o.neval - 1) && !is_contrib && e.valid;
            would[k] = flip_opacity(s, d, &e, fl, u.flags, is_contrib, mm == nc - 1, stop_entry);
            if (is_contrib) ++mm;
        }
        pix[0] = o.A; pix[1] = o.St; pix[2] = o.Sn[0]; pix[3] = o.Sn[1]; pix[4] = o.Sn[2]; pix[5] = o.T;
        pix[6] = ea; pix[7] = ed;
        *pflags = u.flags;
        *nc_out = nc;
    }
    free(ck); free(cT); free(tmp); free(suf); free(et); free(gabs); free(gflip); free(S);
    return ret;
}

/* The method's contribution (contrib_grad of lgs_oracle.c chained to the raw
 * parameters) of surfel i at pixel (r, c), evaluated from the GIVEN
 * evaluation quantities (den, t, u, v, G, a, araw: six doubles and araw),
 * transmittance T before it and suffix S over the later contributors, with
 * the in-plane offset x = u s_u t_u + v s_v t_v.  The tests feed it the
 * values of a binary32 evaluation: the difference to the FP64 contribution
 * is then the effect of the binary32 inputs alone, which contrib_unc bounds.
 * out[10]: mean 3, quaternion 4, log-scale 2, logit 1. */
void lgso_contrib_with(const double* mean, const double* quat, const double* ls, const double* logit,
                       int64_t i, int H, int W, double emin, double emax, const double* pose, int r, int c,
                       const double* q7, double T, double suffix, double gA, double gSt, const double* gSn3,
                       double* out)
{
    frame64 F;
    make_frame(&F, H, W, 1, 1, emin, emax, pose);
    surf64* S = sensor_surfels(mean + 3 * i, quat + 4 * i, ls + 2 * i, logit + i, 1, &F);
    double d[3];
    pixel_ray(&F, r, c, d);
    eval64 e;
    e.valid = 1;
    e.den = q7[0]; e.t = q7[1]; e.u = q7[2]; e.v = q7[3]; e.G = q7[4]; e.a = q7[5]; e.araw = q7[6];
    e.q = e.u * e.u + e.v * e.v;
    for (int k = 0; k < 3; ++k) e.x[k] = e.u * S->su * S->tu[k] + e.v * S->sv * S->tv[k];
    sgrad g;
    memset(&g, 0, sizeof(g));
    contrib_grad(S, &e, d, T, suffix, gA, gSt, gSn3, 1, &g);
    double dm[3] = { 0, 0, 0 }, dq[4] = { 0, 0, 0, 0 }, dl[2] = { 0, 0 }, dg = 0;
    chain_to_params(S, &g, &F, dm, dq, dl, &dg);
    for (int k = 0; k < 3; ++k) out[k] = dm[k];
    for (int k = 0; k < 4; ++k) out[3 + k] = dq[k];
    out[7] = dl[0]; out[8] = dl[1]; out[9] = dg;
    free(S);
}
