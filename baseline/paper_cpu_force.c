/* The paper's mixed-precision force loop (Sec. 3.2-3.3) on the host CPU, as
 * a second CPU baseline beside the plain FP64 oracle.
 *
 * What it computes: Eqs. acc, jrk and pot for a list of active i against all
 * j, with the precision split of Sec. 3.2:
 *   - the relative position r_ij = x_j - x_i subtracted in double precision
 *     and then rounded to single;
 *   - everything else of a pair (r^2 + eps^2, the reciprocal square root,
 *     the pair terms) in single precision, the relative velocity included;
 *   - acceleration and potential accumulated in double precision;
 *   - the jerk accumulated in single precision (the paper's production
 *     choice, Sec. 4).
 * Data parallelism follows Sec. 3.3: one 8-lane single-precision vector holds
 * two i-particles against four j-particles.  The reciprocal square root is
 * an approximate estimate refined by Newton-Raphson, as the paper does with
 * its hardware estimate; here the estimate is the published integer-shift
 * approximation (C. Lomont, "Fast inverse square root", 2003, constant
 * 0x5f375a86; ~3.4 % from the true value) followed by three Newton steps
 * y <- y (3 - x y^2) / 2 (each squares the relative error: 1.8e-3, 4.6e-6,
 * then single-precision rounding).
 *
 * Written with 128-bit GCC vector extensions only (two 4-lane vectors, one
 * per i, make the paper's 8 lanes): the compiler maps them onto the host's
 * SIMD unit (SSE on x86-64, Advanced SIMD on AArch64).  Acceleration and
 * potential of each i go to one two-lane double accumulator per component.  Threads:
 * OpenMP over pairs of active i, as the paper parallelises its i loop.
 *
 * Layout (filled by pcf_pack): j-records padded to a multiple of 4 with
 * zero-mass ghosts far away, structure of arrays
 *   x, y, z   double   [n4]
 *   vx,vy,vz  float    [n4]
 *   m         float    [n4]
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef float v2f __attribute__((vector_size(8)));
typedef float v4f __attribute__((vector_size(16)));
typedef double v2d __attribute__((vector_size(16)));
typedef int32_t v4i __attribute__((vector_size(16)));

#define GHOST_POS 1.0e10

static int64_t pad4(int64_t n) { return (n + 3) & ~(int64_t)3; }

/* Bytes of the packed j layout for n particles. */
int64_t pcf_layout_bytes(int64_t n)
{
    const int64_t n4 = pad4(n);
    return n4 * (3 * (int64_t)sizeof(double) + 4 * (int64_t)sizeof(float));
}

struct layout {
    double *x, *y, *z;
    float *vx, *vy, *vz, *m;
    int64_t n4;
};

static struct layout carve(void *work, int64_t n)
{
    struct layout L;
    L.n4 = pad4(n);
    double *d = (double *)work;
    L.x = d;
    L.y = d + L.n4;
    L.z = d + 2 * L.n4;
    float *f = (float *)(d + 3 * L.n4);
    L.vx = f;
    L.vy = f + L.n4;
    L.vz = f + 2 * L.n4;
    L.m = f + 3 * L.n4;
    return L;
}

/* Pack m[n], r[n][3], v[n][3] (double, AoS) into the j layout at work
 * (pcf_layout_bytes(n) bytes, 8-byte aligned). */
void pcf_pack(int64_t n, const double *m, const double *r, const double *v, void *work)
{
    struct layout L = carve(work, n);
    for (int64_t k = 0; k < L.n4; ++k) {
        const int real = k < n;
        L.x[k] = real ? r[3 * k + 0] : GHOST_POS;
        L.y[k] = real ? r[3 * k + 1] : GHOST_POS;
        L.z[k] = real ? r[3 * k + 2] : GHOST_POS;
        L.vx[k] = real ? (float)v[3 * k + 0] : 0.f;
        L.vy[k] = real ? (float)v[3 * k + 1] : 0.f;
        L.vz[k] = real ? (float)v[3 * k + 2] : 0.f;
        L.m[k] = real ? (float)m[k] : 0.f;
    }
}

static inline v4f splat4(float a) { return (v4f){a, a, a, a}; }
static inline v2d splat2d(double a) { return (v2d){a, a}; }

/* (x_j - x_i) for four j, subtracted in double, rounded to single. */
static inline v4f rel_pos(v2d xa, v2d xb, double xi)
{
    const v2f lo = __builtin_convertvector(xa - splat2d(xi), v2f);
    const v2f hi = __builtin_convertvector(xb - splat2d(xi), v2f);
    return __builtin_shufflevector(lo, hi, 0, 1, 2, 3);
}

/* 1/sqrt(x): integer-shift estimate and three Newton-Raphson steps. */
static inline v4f rsqrt_nr(v4f x)
{
    v4f y = (v4f)((v4i){0x5f375a86, 0x5f375a86, 0x5f375a86, 0x5f375a86} - ((v4i)x >> 1));
    const v4f h = splat4(0.5f) * x;
    y = y * (splat4(1.5f) - h * y * y);
    y = y * (splat4(1.5f) - h * y * y);
    y = y * (splat4(1.5f) - h * y * y);
    return y;
}

/* The four single-precision terms of one i added to its double accumulator
 * (two lanes of double). */
static inline v2d add_dp(v2d acc, v4f t)
{
    const v2f lo = __builtin_shufflevector(t, t, 0, 1);
    const v2f hi = __builtin_shufflevector(t, t, 2, 3);
    return acc + __builtin_convertvector(lo, v2d) + __builtin_convertvector(hi, v2d);
}

static inline v2d load2d(const double *p)
{
    v2d a;
    memcpy(&a, p, sizeof a);
    return a;
}

static inline v4f load4f(const float *p)
{
    v4f a;
    memcpy(&a, p, sizeof a);
    return a;
}

/* Forces on two i (slots i0, i1 of the layout) from every j.  Each vector
 * quantity of the pair is a pair of 4-lane vectors, one per i (the 8 lanes
 * of Sec. 3.3: two i against four j). */
static void force_two(const struct layout *L, const int64_t ii[2], float eps2, double out[2][7])
{
    double xi[2], yi[2], zi[2];
    v4f vix[2], viy[2], viz[2];
    v4i self[2];
    v2d ax[2], ay[2], az[2], ph[2];
    v4f jx[2], jy[2], jz[2];
    for (int s = 0; s < 2; ++s) {
        const int64_t i = ii[s];
        xi[s] = L->x[i], yi[s] = L->y[i], zi[s] = L->z[i];
        vix[s] = splat4(L->vx[i]), viy[s] = splat4(L->vy[i]), viz[s] = splat4(L->vz[i]);
        self[s] = (v4i){(int32_t)i, (int32_t)i, (int32_t)i, (int32_t)i};
        ax[s] = ay[s] = az[s] = ph[s] = (v2d){0.0, 0.0};
        jx[s] = jy[s] = jz[s] = splat4(0.f);
    }
    const v4i lane = (v4i){0, 1, 2, 3};
    const v4f e2 = splat4(eps2);
    const v4f m3 = splat4(-3.f);

    for (int64_t j = 0; j < L->n4; j += 4) {
        const v2d xa = load2d(L->x + j), xb = load2d(L->x + j + 2);
        const v2d ya = load2d(L->y + j), yb = load2d(L->y + j + 2);
        const v2d za = load2d(L->z + j), zb = load2d(L->z + j + 2);
        const v4f vxj = load4f(L->vx + j), vyj = load4f(L->vy + j), vzj = load4f(L->vz + j);
        const v4f mj = load4f(L->m + j);
        const v4i jl = lane + (int32_t)j;
#pragma GCC unroll 2
        for (int s = 0; s < 2; ++s) {
            const v4f dx = rel_pos(xa, xb, xi[s]);
            const v4f dy = rel_pos(ya, yb, yi[s]);
            const v4f dz = rel_pos(za, zb, zi[s]);
            const v4f dvx = vxj - vix[s], dvy = vyj - viy[s], dvz = vzj - viz[s];
            const v4f r2 = dx * dx + dy * dy + dz * dz + e2;
            /* the self pair adds nothing */
            const v4f ri = (v4f)((v4i)rsqrt_nr(r2) & ~(jl == self[s]));
            const v4f mr = mj * ri;      /* m / r             (pot term) */
            const v4f ri2 = ri * ri;
            const v4f g = mr * ri2;      /* m / r^3                      */
            const v4f rv = dx * dvx + dy * dvy + dz * dvz;
            const v4f t = m3 * rv * ri2; /* -3 (r.v) / r^2               */
            ax[s] = add_dp(ax[s], g * dx);
            ay[s] = add_dp(ay[s], g * dy);
            az[s] = add_dp(az[s], g * dz);
            ph[s] = add_dp(ph[s], mr);
            jx[s] += g * (dvx + t * dx);
            jy[s] += g * (dvy + t * dy);
            jz[s] += g * (dvz + t * dz);
        }
    }
    for (int s = 0; s < 2; ++s) {
        out[s][0] = ax[s][0] + ax[s][1];
        out[s][1] = ay[s][0] + ay[s][1];
        out[s][2] = az[s][0] + az[s][1];
        out[s][3] = ((double)jx[s][0] + (double)jx[s][1]) + ((double)jx[s][2] + (double)jx[s][3]);
        out[s][4] = ((double)jy[s][0] + (double)jy[s][1]) + ((double)jy[s][2] + (double)jy[s][3]);
        out[s][5] = ((double)jz[s][0] + (double)jz[s][1]) + ((double)jz[s][2] + (double)jz[s][3]);
        out[s][6] = -(ph[s][0] + ph[s][1]);
    }
}

/* acc[k][3], jerk[k][3], pot[k] of the particles idx[k] (0 <= idx[k] < n),
 * from the layout packed by pcf_pack, with softening eps and constant G.
 * Returns 0, or -1 if an index is out of range (outputs then unspecified). */
int pcf_force(int64_t n, const void *work, double eps, double G, int64_t n_act,
              const int32_t *idx, double *acc, double *jerk, double *pot, int nthreads)
{
    for (int64_t k = 0; k < n_act; ++k)
        if (idx[k] < 0 || idx[k] >= n) return -1;
    const struct layout L = carve((void *)work, n);
    const float eps2 = (float)(eps * eps);
    const int64_t pairs = (n_act + 1) / 2;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for num_threads(nthreads) schedule(dynamic, 8)
    for (int64_t p = 0; p < pairs; ++p) {
        const int64_t k0 = 2 * p;
        const int64_t k1 = k0 + 1 < n_act ? k0 + 1 : k0;
        double out[2][7];
        const int64_t ii[2] = {idx[k0], idx[k1]};
        force_two(&L, ii, eps2, out);
        for (int s = 0; s < (k1 == k0 ? 1 : 2); ++s) {
            const int64_t k = k0 + s;
            for (int c = 0; c < 3; ++c) {
                acc[3 * k + c] = G * out[s][c];
                jerk[3 * k + c] = G * out[s][3 + c];
            }
            pot[k] = G * out[s][6];
        }
    }
    return 0;
}

int pcf_has_openmp(void)
{
#ifdef _OPENMP
    return 1;
#else
    return 0;
#endif
}
