/*
 * Plain FP64 CPU oracle for the fourth-order Hermite scheme with hierarchical
 * (block) individual timesteps of Tanikawa, Yoshikawa, Okamoto & Nitadori,
 * "N-body simulation for self-gravitating collisional systems with a new SIMD
 * instruction set extension to the x86 architecture, AVX" (arXiv:1104.2700).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never calls it and shares no code with it.
 *
 * Conventions
 *   - Every quantity is IEEE double; build with -ffp-contract=off and without
 *     -ffast-math so each operation is rounded exactly as written.
 *   - Positions, velocities, accelerations and jerks are n x 3 row-major
 *     (particle-major) arrays.
 *   - The j-sum runs over ascending j and excludes j == i by index
 *     (Sec. 3.3, force-loop step 3: the self pair is masked by index).
 *   - The optional OpenMP pragma only distributes the independent i
 *     particles over threads; each i's sum keeps the same j order, so the
 *     result does not depend on the thread count.
 *
 * Readings of the paper that this file fixes (the paper is silent or
 * ambiguous on them):
 *   R1 Eq. timestep is written with "(0)" quantities but is evaluated after
 *      step 7 (a0 <- a1, j0 <- j1).  It is evaluated at the new time with
 *      a = a1, j = j1, s = s0 + c0*dt (snap carried to the new time), c = c0.
 *   R2 The power-of-two rule (Sec. 2, "hierarchical timestep"): with
 *      dt_c = min(dt_aarseth, dt_max): double dt_old if dt_c >= 2 dt_old and
 *      t_next is a multiple of 2 dt_old; else keep dt_old if dt_c >= dt_old;
 *      else halve until dt <= dt_c.  Below dt_min is an error.
 *   R3 The first timestep is eta_start*|a|/|j|, rounded down to a power of
 *      two no larger than dt_max.
 *   R4 The active block is every i with t_i + dt_i == t_next exactly (times
 *      are dyadic, so the comparison is exact), listed by ascending index.
 *   R5 A particle that feels nothing (a system of one particle) has
 *      a = j = s = c = 0, where Eq. timestep and the start rule read 0/0: a
 *      zero denominator means no constraint, so the step is dt_max.
 *
 * The sixth-order variant (orc_*6 below) is adjacent to the paper, which
 * integrates with the fourth-order scheme only: the same block-timestep
 * procedure with the snap of each pair evaluated beside its acceleration
 * and jerk, the predictor carried to crackle, and the corrector taken from
 * the quintic Hermite interpolant of a(t) through a, j, s at both ends of
 * the step (the sixth-order Hermite scheme of Nitadori & Makino 2008).
 * Readings it fixes:
 *   H1 The predictor uses a, j, s and the crackle c at the particle's last
 *      time; a load has no crackle yet (c = 0).
 *   H2 The timestep is Eq. timestep generalised to the derivatives the
 *      scheme has: dt = eta ((|a||s| + |j|^2) / (|c||x| + |d|^2))^(1/6) at
 *      the new time, with c, d, x the third, fourth and fifth derivatives of
 *      the interpolant there (R5 for a zero denominator); then R2.
 *   H3 The first steps follow R3 with a and j; the first snap comes from a
 *      second force pass with the accelerations of the first.
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ENONFINITE 4
#define ORC_EDTMIN 5

/* ------------------------------------------------------------------------ */
/* Eqs. acc, jrk, pot (Sec. 2): acceleration, jerk and potential of the     */
/* listed i particles from every other particle j.                           */
/*   a_i   =  sum_{j != i} G m_j r_ij / rt^3                                 */
/*   j_i   =  sum_{j != i} G m_j [ v_ij / rt^3 - 3 (r_ij . v_ij) r_ij / rt^5 ] */
/*   phi_i = -sum_{j != i} G m_j / rt,  rt^2 = |r_ij|^2 + eps^2             */
/* with r_ij = r_j - r_i and v_ij = v_j - v_i (Eq. eom).                     */
/* ------------------------------------------------------------------------ */
void orc_force(int64_t n, const double *m, const double *r, const double *v,
               double eps, double G, int64_t n_act, const int64_t *idx,
               double *acc, double *jerk, double *pot, int nthreads)
{
    const double eps2 = eps * eps;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 4)
#endif
    for (int64_t k = 0; k < n_act; ++k) {
        const int64_t i = idx[k];
        double ax = 0.0, ay = 0.0, az = 0.0;
        double jx = 0.0, jy = 0.0, jz = 0.0;
        double ph = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue; /* the sum excludes the particle itself */
            const double rx = r[3 * j + 0] - r[3 * i + 0];
            const double ry = r[3 * j + 1] - r[3 * i + 1];
            const double rz = r[3 * j + 2] - r[3 * i + 2];
            const double vx = v[3 * j + 0] - v[3 * i + 0];
            const double vy = v[3 * j + 1] - v[3 * i + 1];
            const double vz = v[3 * j + 2] - v[3 * i + 2];
            const double rt2 = rx * rx + ry * ry + rz * rz + eps2;
            const double rt = sqrt(rt2);
            const double rt3 = rt2 * rt;
            const double gm = G * m[j];
            const double rv = rx * vx + ry * vy + rz * vz;
            ax += gm * rx / rt3;
            ay += gm * ry / rt3;
            az += gm * rz / rt3;
            jx += gm * (vx / rt3 - 3.0 * rv * rx / (rt3 * rt2));
            jy += gm * (vy / rt3 - 3.0 * rv * ry / (rt3 * rt2));
            jz += gm * (vz / rt3 - 3.0 * rv * rz / (rt3 * rt2));
            ph -= gm / rt;
        }
        acc[3 * k + 0] = ax;
        acc[3 * k + 1] = ay;
        acc[3 * k + 2] = az;
        jerk[3 * k + 0] = jx;
        jerk[3 * k + 1] = jy;
        jerk[3 * k + 2] = jz;
        pot[k] = ph;
    }
}

/* ------------------------------------------------------------------------ */
/* Eqs. xpred, vpred (Sec. 2): Taylor predictor to time t, dt = t - t0_i.    */
/* ------------------------------------------------------------------------ */
void orc_predict(int64_t n, const double *r0, const double *v0,
                 const double *a0, const double *j0, const double *t0,
                 double t, double *rp, double *vp)
{
    for (int64_t i = 0; i < n; ++i) {
        const double dt = t - t0[i];
        const double dt2 = dt * dt;
        const double dt3 = dt2 * dt;
        for (int d = 0; d < 3; ++d) {
            const int64_t q = 3 * i + d;
            rp[q] = r0[q] + v0[q] * dt + a0[q] / 2.0 * dt2 + j0[q] / 6.0 * dt3;
            vp[q] = v0[q] + a0[q] * dt + j0[q] / 2.0 * dt2;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2, snap/crackle from the third-order Hermite interpolation and the   */
/* corrector for one particle over a step of length dt.                      */
/*   s0 = 2 [-3 (a0 - a1) - (2 j0 + j1) dt] / dt^2                            */
/*   c0 = 6 [ 2 (a0 - a1) + (j0 + j1) dt] / dt^3                              */
/*   r1 = rp + s0 dt^4 / 24 + c0 dt^5 / 120                                   */
/*   v1 = vp + s0 dt^3 / 6  + c0 dt^4 / 24                                    */
/* ------------------------------------------------------------------------ */
void orc_hermite_correct(const double *rp, const double *vp, const double *a0,
                         const double *j0, const double *a1, const double *j1,
                         double dt, double *r1, double *v1, double *s0,
                         double *c0)
{
    const double dt2 = dt * dt;
    const double dt3 = dt2 * dt;
    const double dt4 = dt3 * dt;
    const double dt5 = dt4 * dt;
    for (int d = 0; d < 3; ++d) {
        const double da = a0[d] - a1[d];
        s0[d] = 2.0 * (-3.0 * da - (2.0 * j0[d] + j1[d]) * dt) / dt2;
        c0[d] = 6.0 * (2.0 * da + (j0[d] + j1[d]) * dt) / dt3;
        r1[d] = rp[d] + s0[d] * dt4 / 24.0 + c0[d] * dt5 / 120.0;
        v1[d] = vp[d] + s0[d] * dt3 / 6.0 + c0[d] * dt4 / 24.0;
    }
}

static double norm3(const double *x)
{
    return sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
}

/* Eq. timestep (Sec. 2, Aarseth's criterion). */
double orc_aarseth_dt(double eta, const double *a, const double *j,
                      const double *s, const double *c)
{
    const double A = norm3(a), J = norm3(j), S = norm3(s), C = norm3(c);
    const double den = J * C + S * S;
    if (den == 0.0) return INFINITY; /* reading R5: no constraint */
    return eta * sqrt((A * S + J * J) / den);
}

/* Largest power of two (2^k, k integer) that is <= x, for x > 0 finite. */
double orc_pow2_floor(double x)
{
    int e;
    const double f = frexp(x, &e); /* x = f * 2^e, f in [0.5, 1) */
    (void)f;
    return ldexp(1.0, e - 1);
}

/* Reading R2: power-of-two timestep update of the hierarchical scheme. */
int orc_quantize_dt(double dt_old, double dt_cand, double t_next,
                    double dt_max, double dt_min, double *dt_new)
{
    if (!(dt_cand == dt_cand)) return ORC_ENONFINITE; /* NaN */
    double c = dt_cand < dt_max ? dt_cand : dt_max;
    double dt = dt_old;
    if (c >= 2.0 * dt_old && fmod(t_next, 2.0 * dt_old) == 0.0) {
        dt = 2.0 * dt_old;
    } else if (c >= dt_old) {
        dt = dt_old;
    } else {
        while (dt > c && dt >= dt_min) dt *= 0.5;
    }
    *dt_new = dt;
    return dt < dt_min ? ORC_EDTMIN : ORC_OK;
}

/* Reading R3: first timestep. */
int orc_initial_dt(double eta_start, const double *a, const double *j,
                   double dt_max, double dt_min, double *dt_out)
{
    const double A = norm3(a), J = norm3(j);
    double raw = J == 0.0 ? INFINITY : eta_start * A / J; /* reading R5 */
    if (!(raw == raw)) return ORC_ENONFINITE;
    if (raw > dt_max) raw = dt_max;
    if (raw <= 0.0) return ORC_EDTMIN;
    const double dt = orc_pow2_floor(raw);
    *dt_out = dt;
    return dt < dt_min ? ORC_EDTMIN : ORC_OK;
}

/* Step 1 and reading R4: next block time and the active list.  Returns the
 * number of active particles; idx receives them in ascending order. */
int64_t orc_select(int64_t n, const double *t, const double *dt,
                   double *t_next, int64_t *idx)
{
    double tmin = INFINITY;
    for (int64_t i = 0; i < n; ++i) {
        const double tn = t[i] + dt[i];
        if (tn < tmin) tmin = tn;
    }
    int64_t k = 0;
    for (int64_t i = 0; i < n; ++i)
        if (t[i] + dt[i] == tmin) idx[k++] = i;
    *t_next = tmin;
    return k;
}

/* Kinetic energy and the potential energy 1/2 sum m_i phi_i (Eq. pot),
 * the diagnostic used for energy conservation (Sec. 2, Sec. 4). */
void orc_energy(int64_t n, const double *m, const double *r, const double *v,
                double eps, double G, double *kin, double *pot, int nthreads)
{
    double K = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        const double v2 = v[3 * i] * v[3 * i] + v[3 * i + 1] * v[3 * i + 1] +
                          v[3 * i + 2] * v[3 * i + 2];
        K += 0.5 * m[i] * v2;
    }
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double *a = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *jk = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    double *ph = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    orc_force(n, m, r, v, eps, G, n, idx, a, jk, ph, nthreads);
    double W = 0.0;
    for (int64_t i = 0; i < n; ++i) W += 0.5 * m[i] * ph[i];
    free(idx);
    free(a);
    free(jk);
    free(ph);
    *kin = K;
    *pot = W;
}

/* Initial a, j (full force at t = 0), t_i = t0 and the first timesteps. */
int orc_init(int64_t n, const double *m, double *r, double *v, double *a,
             double *j, double *t, double *dt, double t0, double eps, double G,
             double eta_start, double dt_max, double dt_min, int nthreads)
{
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double *ph = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    orc_force(n, m, r, v, eps, G, n, idx, a, j, ph, nthreads);
    int st = ORC_OK;
    for (int64_t i = 0; i < n && st == ORC_OK; ++i) {
        t[i] = t0;
        st = orc_initial_dt(eta_start, a + 3 * i, j + 3 * i, dt_max, dt_min,
                            dt + i);
    }
    free(idx);
    free(ph);
    return st;
}

/* The integration procedure of Sec. 2 (steps 1-9), repeated while the next
 * block time does not pass t_end.  With t_end a multiple of dt_max every
 * particle ends exactly at t_end.  Counts block steps and interactions
 * (n_act * n per force call, the self pair included by convention). */
int orc_run(int64_t n, const double *m, double *r, double *v, double *a,
            double *j, double *t, double *dt, double t_end, double eps,
            double G, double eta, double dt_max, double dt_min, int nthreads,
            int64_t max_steps, int64_t *n_steps, double *n_inter)
{
    const size_t n3 = 3 * (size_t)(n > 0 ? n : 1);
    double *rp = (double *)malloc(sizeof(double) * n3);
    double *vp = (double *)malloc(sizeof(double) * n3);
    double *a1 = (double *)malloc(sizeof(double) * n3);
    double *j1 = (double *)malloc(sizeof(double) * n3);
    double *ph = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int st = ORC_OK;
    int64_t steps = 0;
    double inter = 0.0;
    for (;;) {
        /* Step 1: the i block with the earliest next time. */
        double t_next;
        const int64_t n_act = orc_select(n, t, dt, &t_next, idx);
        if (n_act == 0 || t_next > t_end) break;
        if (max_steps > 0 && steps >= max_steps) break;
        /* Steps 2 and 3: predict every particle (i and j) to t_next. */
        orc_predict(n, r, v, a, j, t, t_next, rp, vp);
        /* Step 4: force on the i block from the predicted j particles. */
        orc_force(n, m, rp, vp, eps, G, n_act, idx, a1, j1, ph, nthreads);
        inter += (double)n_act * (double)n;
        for (int64_t k = 0; k < n_act && st == ORC_OK; ++k) {
            const int64_t i = idx[k];
            for (int d = 0; d < 3; ++d)
                if (!isfinite(a1[3 * k + d]) || !isfinite(j1[3 * k + d]))
                    st = ORC_ENONFINITE;
            if (st != ORC_OK) break;
            /* Steps 5 and 6: Hermite interpolation and corrector. */
            double r1[3], v1[3], s0[3], c0[3];
            const double h = dt[i];
            orc_hermite_correct(rp + 3 * i, vp + 3 * i, a + 3 * i, j + 3 * i,
                                a1 + 3 * k, j1 + 3 * k, h, r1, v1, s0, c0);
            /* Step 7: a0 <- a1, j0 <- j1; the particle is now at t_next. */
            for (int d = 0; d < 3; ++d) {
                r[3 * i + d] = r1[d];
                v[3 * i + d] = v1[d];
                a[3 * i + d] = a1[3 * k + d];
                j[3 * i + d] = j1[3 * k + d];
            }
            t[i] = t_next;
            /* Step 8: next timestep (readings R1, R2). */
            double s_new[3];
            for (int d = 0; d < 3; ++d) s_new[d] = s0[d] + c0[d] * h;
            const double dt_a =
                orc_aarseth_dt(eta, a + 3 * i, j + 3 * i, s_new, c0);
            st = orc_quantize_dt(h, dt_a, t_next, dt_max, dt_min, dt + i);
        }
        ++steps;
        if (st != ORC_OK) break;
    }
    free(rp);
    free(vp);
    free(a1);
    free(j1);
    free(ph);
    free(idx);
    *n_steps = steps;
    *n_inter = inter;
    return st;
}

/* ------------------------------------------------------------------------ */
/* Sixth-order variant.                                                      */
/* Snap of Eqs. acc and jrk: the second time derivative of each pair term   */
/* along the predicted trajectories, with r = r_j - r_i, v, a likewise,     */
/* rt^2 = |r|^2 + eps^2, alpha = (r.v)/rt^2, beta = (v.v + r.a)/rt^2 +     */
/* alpha^2, and the pair's acceleration A = G m r / rt^3 and jerk           */
/* J = G m v / rt^3 - 3 alpha A:                                             */
/*   S = G m a / rt^3 - 6 alpha J - 3 beta A.                                */
/* a_in holds the predicted accelerations of all particles.                 */
/* ------------------------------------------------------------------------ */
void orc_force_snap(int64_t n, const double *m, const double *r, const double *v,
                    const double *a_in, double eps, double G, int64_t n_act,
                    const int64_t *idx, double *acc, double *jerk, double *snap,
                    double *pot, int nthreads)
{
    const double eps2 = eps * eps;
    if (nthreads < 1) nthreads = 1;
#ifdef _OPENMP
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 4)
#endif
    for (int64_t k = 0; k < n_act; ++k) {
        const int64_t i = idx[k];
        double A[3] = {0.0, 0.0, 0.0}, J[3] = {0.0, 0.0, 0.0}, S[3] = {0.0, 0.0, 0.0};
        double ph = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double rr[3], vv[3], aa[3];
            for (int d = 0; d < 3; ++d) {
                rr[d] = r[3 * j + d] - r[3 * i + d];
                vv[d] = v[3 * j + d] - v[3 * i + d];
                aa[d] = a_in[3 * j + d] - a_in[3 * i + d];
            }
            const double rt2 = rr[0] * rr[0] + rr[1] * rr[1] + rr[2] * rr[2] + eps2;
            const double rt = sqrt(rt2);
            const double rt3 = rt2 * rt;
            const double gm = G * m[j];
            const double alpha = (rr[0] * vv[0] + rr[1] * vv[1] + rr[2] * vv[2]) / rt2;
            const double beta = (vv[0] * vv[0] + vv[1] * vv[1] + vv[2] * vv[2] +
                                 rr[0] * aa[0] + rr[1] * aa[1] + rr[2] * aa[2]) / rt2 +
                                alpha * alpha;
            for (int d = 0; d < 3; ++d) {
                const double pa = gm * rr[d] / rt3;
                const double pj = gm * vv[d] / rt3 - 3.0 * alpha * pa;
                const double ps = gm * aa[d] / rt3 - 6.0 * alpha * pj - 3.0 * beta * pa;
                A[d] += pa;
                J[d] += pj;
                S[d] += ps;
            }
            ph -= gm / rt;
        }
        for (int d = 0; d < 3; ++d) {
            acc[3 * k + d] = A[d];
            jerk[3 * k + d] = J[d];
            snap[3 * k + d] = S[d];
        }
        pot[k] = ph;
    }
}

/* Reading H1: Taylor predictor of r, v, a to time t from a, j, s and the  */
/* crackle c at each particle's own time t0.                                */
void orc_predict6(int64_t n, const double *r0, const double *v0, const double *a0,
                  const double *j0, const double *s0, const double *c0,
                  const double *t0, double t, double *rp, double *vp, double *ap)
{
    for (int64_t i = 0; i < n; ++i) {
        const double h = t - t0[i];
        const double h2 = h * h, h3 = h2 * h, h4 = h3 * h, h5 = h4 * h;
        for (int d = 0; d < 3; ++d) {
            const int64_t q = 3 * i + d;
            rp[q] = r0[q] + v0[q] * h + a0[q] / 2.0 * h2 + j0[q] / 6.0 * h3 +
                    s0[q] / 24.0 * h4 + c0[q] / 120.0 * h5;
            vp[q] = v0[q] + a0[q] * h + j0[q] / 2.0 * h2 + s0[q] / 6.0 * h3 +
                    c0[q] / 24.0 * h4;
            ap[q] = a0[q] + j0[q] * h + s0[q] / 2.0 * h2 + c0[q] / 6.0 * h3;
        }
    }
}

/* Corrector of the sixth-order scheme for one particle over a step h.      */
/* a(tau) on [0, h] is the quintic through a0, j0, s0 at 0 and a1, j1, s1 at */
/* h.  Its Taylor coefficients at 0 beyond s0 solve                          */
/*   c3 h^3/6 + c4 h^4/24 + c5 h^5/120 = a1 - a0 - j0 h - s0 h^2/2           */
/*   c3 h^2/2 + c4 h^3/6  + c5 h^4/24  = j1 - j0 - s0 h                      */
/*   c3 h     + c4 h^2/2  + c5 h^3/6   = s1 - s0                             */
/* (solved in closed form below), and its integrals give                    */
/*   v1 = v0 + h/2 (a0 + a1) - h^2/10 (j1 - j0) + h^3/120 (s0 + s1)          */
/*   r1 = r0 + h/2 (v0 + v1) - h^2/10 (a1 - a0) + h^3/120 (j0 + j1)          */
/* The third, fourth and fifth derivatives at h (crackle, pop, x) follow    */
/* from the Taylor series: c3 + c4 h + c5 h^2/2, c4 + c5 h, c5.             */
void orc_hermite6_correct(const double *r0, const double *v0, const double *a0,
                          const double *j0, const double *s0, const double *a1,
                          const double *j1, const double *s1, double h, double *r1,
                          double *v1, double *c1, double *d1, double *x1)
{
    const double h2 = h * h, h3 = h2 * h, h4 = h3 * h, h5 = h4 * h;
    for (int d = 0; d < 3; ++d) {
        const double Da = a1[d] - a0[d] - j0[d] * h - s0[d] / 2.0 * h2;
        const double Dj = j1[d] - j0[d] - s0[d] * h;
        const double Ds = s1[d] - s0[d];
        const double c3 = 3.0 * (20.0 * Da - 8.0 * Dj * h + Ds * h2) / h3;
        const double c4 = -24.0 * (15.0 * Da - 7.0 * Dj * h + Ds * h2) / h4;
        const double c5 = 60.0 * (12.0 * Da - 6.0 * Dj * h + Ds * h2) / h5;
        v1[d] = v0[d] + h / 2.0 * (a0[d] + a1[d]) - h2 / 10.0 * (j1[d] - j0[d]) +
                h3 / 120.0 * (s0[d] + s1[d]);
        r1[d] = r0[d] + h / 2.0 * (v0[d] + v1[d]) - h2 / 10.0 * (a1[d] - a0[d]) +
                h3 / 120.0 * (j0[d] + j1[d]);
        c1[d] = c3 + c4 * h + c5 / 2.0 * h2;
        d1[d] = c4 + c5 * h;
        x1[d] = c5;
    }
}

/* Reading H2: the timestep criterion of the sixth-order scheme. */
double orc_aarseth6_dt(double eta, const double *a, const double *j, const double *s,
                       const double *c, const double *d, const double *x)
{
    const double A = norm3(a), J = norm3(j), S = norm3(s);
    const double C = norm3(c), D = norm3(d), X = norm3(x);
    const double den = C * X + D * D;
    if (den == 0.0) return INFINITY; /* reading R5: no constraint */
    return eta * pow((A * S + J * J) / den, 1.0 / 6.0);
}

/* Reading H3: a, j from a force pass, s from a second pass with those      */
/* accelerations, c = 0, first timesteps by R3.                             */
int orc_init6(int64_t n, const double *m, double *r, double *v, double *a,
              double *j, double *s, double *c, double *t, double *dt, double t0,
              double eps, double G, double eta_start, double dt_max, double dt_min,
              int nthreads)
{
    int st = orc_init(n, m, r, v, a, j, t, dt, t0, eps, G, eta_start, dt_max, dt_min,
                      nthreads);
    if (st != ORC_OK) return st;
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    const size_t n3 = 3 * (size_t)(n > 0 ? n : 1);
    double *a2 = (double *)malloc(sizeof(double) * n3);
    double *j2 = (double *)malloc(sizeof(double) * n3);
    double *ph = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) idx[i] = i;
    orc_force_snap(n, m, r, v, a, eps, G, n, idx, a2, j2, s, ph, nthreads);
    for (size_t q = 0; q < 3 * (size_t)n; ++q) c[q] = 0.0;
    free(idx);
    free(a2);
    free(j2);
    free(ph);
    return st;
}

/* The block-timestep procedure with the sixth-order scheme. */
int orc_run6(int64_t n, const double *m, double *r, double *v, double *a, double *j,
             double *s, double *c, double *t, double *dt, double t_end, double eps,
             double G, double eta, double dt_max, double dt_min, int nthreads,
             int64_t max_steps, int64_t *n_steps, double *n_inter)
{
    const size_t n3 = 3 * (size_t)(n > 0 ? n : 1);
    double *rp = (double *)malloc(sizeof(double) * n3);
    double *vp = (double *)malloc(sizeof(double) * n3);
    double *ap = (double *)malloc(sizeof(double) * n3);
    double *a1 = (double *)malloc(sizeof(double) * n3);
    double *j1 = (double *)malloc(sizeof(double) * n3);
    double *s1 = (double *)malloc(sizeof(double) * n3);
    double *ph = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t *idx = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int st = ORC_OK;
    int64_t steps = 0;
    double inter = 0.0;
    for (;;) {
        double t_next;
        const int64_t n_act = orc_select(n, t, dt, &t_next, idx);
        if (n_act == 0 || t_next > t_end) break;
        if (max_steps > 0 && steps >= max_steps) break;
        orc_predict6(n, r, v, a, j, s, c, t, t_next, rp, vp, ap);
        orc_force_snap(n, m, rp, vp, ap, eps, G, n_act, idx, a1, j1, s1, ph, nthreads);
        inter += (double)n_act * (double)n;
        for (int64_t k = 0; k < n_act && st == ORC_OK; ++k) {
            const int64_t i = idx[k];
            for (int d = 0; d < 3; ++d)
                if (!isfinite(a1[3 * k + d]) || !isfinite(j1[3 * k + d]) ||
                    !isfinite(s1[3 * k + d]))
                    st = ORC_ENONFINITE;
            if (st != ORC_OK) break;
            double r1[3], v1[3], c1[3], d1[3], x1[3];
            const double h = dt[i];
            orc_hermite6_correct(r + 3 * i, v + 3 * i, a + 3 * i, j + 3 * i, s + 3 * i,
                                 a1 + 3 * k, j1 + 3 * k, s1 + 3 * k, h, r1, v1, c1, d1, x1);
            for (int d = 0; d < 3; ++d) {
                r[3 * i + d] = r1[d];
                v[3 * i + d] = v1[d];
                a[3 * i + d] = a1[3 * k + d];
                j[3 * i + d] = j1[3 * k + d];
                s[3 * i + d] = s1[3 * k + d];
                c[3 * i + d] = c1[d];
            }
            t[i] = t_next;
            const double dt_a = orc_aarseth6_dt(eta, a + 3 * i, j + 3 * i, s + 3 * i, c1, d1, x1);
            st = orc_quantize_dt(h, dt_a, t_next, dt_max, dt_min, dt + i);
        }
        ++steps;
        if (st != ORC_OK) break;
    }
    free(rp);
    free(vp);
    free(ap);
    free(a1);
    free(j1);
    free(s1);
    free(ph);
    free(idx);
    *n_steps = steps;
    *n_inter = inter;
    return st;
}

int orc_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
