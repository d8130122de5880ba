// Step 4 of the Hermite integration procedure (Sec. 2): acceleration, jerk
// and potential of the active i particles from every predicted j particle,
// Eqs. acc, jrk and pot, with the self pair excluded by index (Sec. 3.3,
// force-loop step 3).
//
// Work decomposition (GB300-first, not the paper's 2 i x 4 j AVX pairing):
//   * an i-group is 32*IT/S consecutive entries of the active list; each lane
//     of a warp holds IT i particles in registers, and S lanes (the j split,
//     1, 2, 4 or 8) share each i;
//   * the j particles stream through shared memory in tiles of TJ, staged by
//     1-D bulk copies (cp.async.bulk) into a STAGES-deep ring owned by the
//     warp and completed on mbarriers; lane slice s reads tile slots s,
//     s + S, ... (a shared-memory broadcast within the slice), and the
//     slices' partial sums are added by warp shuffles at the end of a group;
//   * the flattened (i-group, j-tile) space is cut into equal contiguous
//     ranges, one per persistent warp ("stream-K"), so every warp does the
//     same number of tiles whatever n_act is.  A group split across several
//     warps is summed by the last warp to finish, in warp order, from
//     partials in global scratch: deterministic, and no warp ever waits on
//     another.
#pragma once

#include <type_traits>

#include "nb_device.cuh"
#include "nb_launch.h"

namespace nb {

struct ForceParams {
    const void* jl0;
    const void* jl1;
    const void* jl2;
    const void* jl3;
    int64_t n;
    int64_t n_pad;
    const int32_t* idx;
    const int32_t* n_act_dev;
    double* acc;
    double* jerk;
    double* pot;
    double* snap;  // sixth-order variant: [n_act][3]
    double* scratch;
    uint32_t* counters;      // RLEVELS arrays of counter_stride entries
    int64_t counter_stride;  // >= warps + groups
    uint32_t* status;
    double eps2;
    int32_t nact_lo, nact_hi;  // the launch works only for n_act in [lo, hi)
    long long wait_limit;      // cycles before a tile wait gives up
    int32_t unfed_first_tile;  // self-test: never stage each warp's first tile
    // Ensemble plan (all null for one system): i-groups built by
    // plan_launch, and per-cluster particle / j-layout offsets and eps^2.
    const int32_t* grp_cluster;
    const int32_t* grp_act_begin;
    const int32_t* grp_act_count;
    const int64_t* grp_tile0;     // n_groups + 1 entries
    const int64_t* plan_scalars;  // [0] groups, [1] tiles
    const int64_t* cl_off;
    const int64_t* cl_joff;
    const double* cl_eps2;
    // Hybrid precision: the state's a, j (SoA, [c*n + i]) and the velocity
    // bound of the layout split (float bits).
    const double* st_a;
    const double* st_j;
    const uint32_t* bound_v;
    // and its integration guard: the state's dt, eta, and the far-field
    // noise estimate of each particle's last evaluation (written here)
    const double* st_dt;
    double* st_hq;
    double eta;
    // One system: the j tiles [jt_lo, jt_hi) this launch sums over (its part
    // of a j-partitioned force); jt_hi = 0 means every tile.
    int64_t jt_lo, jt_hi;
    // One system: sum small blocks CTA by CTA (see force_kernel)
    int32_t cta_mode;
    // n_act given at launch (>= 0; else read from n_act_dev), and an
    // optional map of the listed indices (caller numbering -> layout slot)
    int32_t n_act_host;
    const int32_t* idx_map;
    float guard_eta;  // HYBRID: the guard's coefficient times eta
    // Ensemble plans: stream-K chunks per warp, >= 2 handed out by a queue
    // (see force_kernel); the queue word, zero between launches.
    int32_t dyn_chunks;
    uint32_t* queue;
};

// A double narrowed to FP32 with integer operations only: the top 23
// mantissa bits (truncated), zero below FP32's normal range, infinity above
// it (and for NaN).  Within an FP32 ulp of the value, which suffices for the
// thresholds it feeds.
__device__ __forceinline__ float f32_trunc(double x)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const uint32_t hi = static_cast<uint32_t>(b >> 32);
    const uint32_t sign = hi & 0x80000000u;
    const int e = static_cast<int>((hi >> 20) & 0x7ffu) - 1023 + 127;
    if (e <= 0) return __uint_as_float(sign);
    if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
    const uint32_t mant = ((hi & 0xfffffu) << 3) | (static_cast<uint32_t>(b) >> 29);
    return __uint_as_float(sign | (static_cast<uint32_t>(e) << 23) | mant);
}

// eps^2 of a group's system, as the FP64 value and its FP32 hi + lo split
// (made once per group, so the tile loops do no FP64 conversion).
struct Eps2 {
    double d;
    float h, l;
};
__device__ __forceinline__ Eps2 make_eps2(double e2)
{
    Eps2 r;
    r.d = e2;
    r.h = static_cast<float>(e2);
    r.l = static_cast<float>(e2 - static_cast<double>(r.h));
    return r;
}

// ---------------------------------------------------------------------------
// Precision policies.  Each provides: the j-layout arrays it stages, the
// i state it keeps in registers, the per-tile pair loop and the final values.
// ---------------------------------------------------------------------------

// Plain FP64: the baseline path.
template <int IT>
struct PolicyFP64 {
    static constexpr bool GUARDED = false;
    static constexpr int MIN_CTAS = 3;  // registers capped for three CTAs per SM
    static constexpr int CHUNKS = 1;
    static constexpr int NARR = 2;
    __host__ __device__ static constexpr int elem(int a) { return a < 2 ? 32 : 0; }
    static constexpr int TILE_BYTES = TJ * 64;
    static constexpr int STAGES = 3;

    struct I {
        double x, y, z, vx, vy, vz;
        int p;
    };
    struct Acc {
        double ax, ay, az, jx, jy, jz, ph;
        __device__ void zero() { ax = ay = az = jx = jy = jz = ph = 0.0; }
    };

    __device__ static void load_i(const ForceParams& f, int p, int, I& s)
    {
        s.p = p;
        if (p < 0) {
            s.x = s.y = s.z = s.vx = s.vy = s.vz = 0.0;
            return;
        }
        const double2* P = static_cast<const double2*>(f.jl0) + 2 * (int64_t)p;
        const double2* V = static_cast<const double2*>(f.jl1) + 2 * (int64_t)p;
        const double2 p0 = __ldg(P), p1 = __ldg(P + 1);
        const double2 v0 = __ldg(V), v1 = __ldg(V + 1);
        s.x = p0.x, s.y = p0.y, s.z = p1.x;
        s.vx = v0.x, s.vy = v0.y, s.vz = v1.x;
    }

    // S lanes share each i; lane slice sl takes records sl, sl + S, ...
    template <bool MASK, int S>
    __device__ static void tile(const unsigned char* buf, int64_t j0, const Eps2& e2s,
                                I (&is)[IT], Acc (&ac)[IT], int sl)
    {
        const double eps2 = e2s.d;
        const double2* sP = reinterpret_cast<const double2*>(buf);
        const double2* sV = reinterpret_cast<const double2*>(buf + TJ * 32);
#pragma unroll 2
        for (int u = 0; u < TJ / S; ++u) {
            const int k = sl + S * u;
            const double2 p0 = sP[2 * k], p1 = sP[2 * k + 1];
            const double2 v0 = sV[2 * k], v1 = sV[2 * k + 1];
#pragma unroll
            for (int q = 0; q < IT; ++q) {
                const double dx = p0.x - is[q].x, dy = p0.y - is[q].y, dz = p1.x - is[q].z;
                const double dvx = v0.x - is[q].vx, dvy = v0.y - is[q].vy,
                             dvz = v1.x - is[q].vz;
                const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
                double ri = rsqrt(r2);
                if (MASK) ri = (j0 + k == is[q].p) ? 0.0 : ri;
                const double mr = p1.y * ri;
                const double ri2 = ri * ri;
                const double g = mr * ri2;
                const double rv = fma(dx, dvx, fma(dy, dvy, dz * dvz));
                const double t = -3.0 * rv * ri2;
                ac[q].ax = fma(g, dx, ac[q].ax);
                ac[q].ay = fma(g, dy, ac[q].ay);
                ac[q].az = fma(g, dz, ac[q].az);
                ac[q].jx = fma(g, fma(t, dx, dvx), ac[q].jx);
                ac[q].jy = fma(g, fma(t, dy, dvy), ac[q].jy);
                ac[q].jz = fma(g, fma(t, dz, dvz), ac[q].jz);
                ac[q].ph += mr;
            }
        }
    }

    static constexpr int NV = 7;  // reduced values: acc (3), jerk (3), pot
    using TV = double;            // value type of the split-group tree
    __device__ static void values(const Acc& a, TV (&v)[NV])
    {
        v[0] = a.ax, v[1] = a.ay, v[2] = a.az;
        v[3] = a.jx, v[4] = a.jy, v[5] = a.jz;
        v[6] = -a.ph;
    }
};

// FP64 with snap, for the sixth-order Hermite variant (adjacent to the
// paper): the j layout also carries each particle's predicted acceleration,
// and each pair adds the second time derivative of its acceleration term
// along the predicted trajectories,
//   S = G m a / r^3 - 6 alpha J - 3 beta A,
// alpha = (r.v) / r^2, beta = (v.v + r.a) / r^2 + alpha^2, with A and J
// the pair's acceleration and jerk terms (r, v, a relative, r softened).
template <int IT>
struct PolicyFP64Snap {
    static constexpr bool GUARDED = false;
    static constexpr int MIN_CTAS = 1;
    static constexpr int CHUNKS = 1;
    static constexpr int NARR = 3;
    __host__ __device__ static constexpr int elem(int a) { return a < 3 ? 32 : 0; }
    static constexpr int TILE_BYTES = TJ * 96;
    static constexpr int STAGES = 2;

    struct I {
        double x, y, z, vx, vy, vz, ax, ay, az;
        int p;
    };
    struct Acc {
        double ax, ay, az, jx, jy, jz, sx, sy, sz, ph;
        __device__ void zero() { ax = ay = az = jx = jy = jz = sx = sy = sz = ph = 0.0; }
    };

    __device__ static void load_i(const ForceParams& f, int p, int, I& s)
    {
        s.p = p;
        if (p < 0) {
            s.x = s.y = s.z = s.vx = s.vy = s.vz = s.ax = s.ay = s.az = 0.0;
            return;
        }
        const double2* P = static_cast<const double2*>(f.jl0) + 2 * (int64_t)p;
        const double2* V = static_cast<const double2*>(f.jl1) + 2 * (int64_t)p;
        const double2* A = static_cast<const double2*>(f.jl2) + 2 * (int64_t)p;
        const double2 p0 = __ldg(P), p1 = __ldg(P + 1);
        const double2 v0 = __ldg(V), v1 = __ldg(V + 1);
        const double2 a0 = __ldg(A), a1 = __ldg(A + 1);
        s.x = p0.x, s.y = p0.y, s.z = p1.x;
        s.vx = v0.x, s.vy = v0.y, s.vz = v1.x;
        s.ax = a0.x, s.ay = a0.y, s.az = a1.x;
    }

    template <bool MASK, int S>
    __device__ static void tile(const unsigned char* buf, int64_t j0, const Eps2& e2s,
                                I (&is)[IT], Acc (&ac)[IT], int sl)
    {
        const double eps2 = e2s.d;
        const double2* sP = reinterpret_cast<const double2*>(buf);
        const double2* sV = reinterpret_cast<const double2*>(buf + TJ * 32);
        const double2* sA = reinterpret_cast<const double2*>(buf + TJ * 64);
#pragma unroll 1
        for (int u = 0; u < TJ / S; ++u) {
            const int k = sl + S * u;
            const double2 p0 = sP[2 * k], p1 = sP[2 * k + 1];
            const double2 v0 = sV[2 * k], v1 = sV[2 * k + 1];
            const double2 a0 = sA[2 * k], a1 = sA[2 * k + 1];
#pragma unroll
            for (int q = 0; q < IT; ++q) {
                const double dx = p0.x - is[q].x, dy = p0.y - is[q].y, dz = p1.x - is[q].z;
                const double vx = v0.x - is[q].vx, vy = v0.y - is[q].vy, vz = v1.x - is[q].vz;
                const double wx = a0.x - is[q].ax, wy = a0.y - is[q].ay, wz = a1.x - is[q].az;
                const double r2 = fma(dx, dx, fma(dy, dy, fma(dz, dz, eps2)));
                double ri = rsqrt(r2);
                if (MASK) ri = (j0 + k == is[q].p) ? 0.0 : ri;
                const double mr = p1.y * ri;
                const double ri2 = ri * ri;
                const double g = mr * ri2;  // G m / r^3
                const double alpha = fma(dx, vx, fma(dy, vy, dz * vz)) * ri2;
                const double beta =
                    fma(fma(vx, vx, fma(vy, vy, vz * vz)) + fma(dx, wx, fma(dy, wy, dz * wz)), ri2,
                        alpha * alpha);
                const double Ax = g * dx, Ay = g * dy, Az = g * dz;
                const double Jx = fma(g, vx, -3.0 * alpha * Ax);
                const double Jy = fma(g, vy, -3.0 * alpha * Ay);
                const double Jz = fma(g, vz, -3.0 * alpha * Az);
                ac[q].ax += Ax, ac[q].ay += Ay, ac[q].az += Az;
                ac[q].jx += Jx, ac[q].jy += Jy, ac[q].jz += Jz;
                ac[q].sx += fma(g, wx, fma(-6.0 * alpha, Jx, -3.0 * beta * Ax));
                ac[q].sy += fma(g, wy, fma(-6.0 * alpha, Jy, -3.0 * beta * Ay));
                ac[q].sz += fma(g, wz, fma(-6.0 * alpha, Jz, -3.0 * beta * Az));
                ac[q].ph += mr;
            }
        }
    }

    static constexpr int NV = 10;  // acc (3), jerk (3), pot, snap (3)
    using TV = double;
    __device__ static void values(const Acc& a, TV (&v)[NV])
    {
        v[0] = a.ax, v[1] = a.ay, v[2] = a.az;
        v[3] = a.jx, v[4] = a.jy, v[5] = a.jz;
        v[6] = -a.ph;
        v[7] = a.sx, v[8] = a.sy, v[9] = a.sz;
    }

    __device__ static void finish(const ForceParams& f, const I&, int64_t row,
                                  const double (&v)[NV])
    {
        f.snap[3 * row + 0] = v[7];
        f.snap[3 * row + 1] = v[8];
        f.snap[3 * row + 2] = v[9];
    }
};

// Mixed precision (Sec. 3.2): r_ij from double-single positions (the
// double-single difference stands in for the paper's DP subtraction), the
// remaining pair arithmetic in FP32 with a hardware rsqrt, FP32 partial
// sums over each tile folded into double-single accumulators.  With SPJ the
// jerk instead runs in one plain FP32 sum over the warp's whole range of j,
// the accumulation of the paper's own kernel (Sec. 4, Fig. err_snp_djerk);
// the acceleration and potential arithmetic is unchanged.
template <int IT, bool SPJ = false>
struct PolicyMixed {
    static constexpr bool GUARDED = false;
    static constexpr int MIN_CTAS = IT > 1 ? 2 : 3;  // registers capped: 2 or 3 CTAs per SM
    static constexpr int CHUNKS = 1;
    static constexpr int NARR = 3;
    __host__ __device__ static constexpr int elem(int a) { return a < 2 ? 16 : (a == 2 ? 8 : 0); }
    static constexpr int TILE_BYTES = TJ * 40;
    static constexpr int STAGES = 4;

    struct I {
        float xh, yh, zh, xl, yl, zl, vx, vy, vz;
        int p;
    };
    struct Acc {
        DSAcc ax, ay, az, jx, jy, jz, ph;
        __device__ void zero()
        {
            ax.zero(), ay.zero(), az.zero(), jx.zero(), jy.zero(), jz.zero(), ph.zero();
        }
    };

    __device__ static void load_i(const ForceParams& f, int p, int, I& s)
    {
        s.p = p;
        if (p < 0) {
            s.xh = s.yh = s.zh = s.xl = s.yl = s.zl = s.vx = s.vy = s.vz = 0.f;
            return;
        }
        const float4 A = __ldg(static_cast<const float4*>(f.jl0) + p);
        const float4 B = __ldg(static_cast<const float4*>(f.jl1) + p);
        const float2 C = __ldg(static_cast<const float2*>(f.jl2) + p);
        s.xh = A.x, s.yh = A.y, s.zh = A.z;
        s.xl = B.x, s.yl = B.y, s.zl = B.z;
        s.vx = B.w, s.vy = C.x, s.vz = C.y;
    }

    template <bool MASK, int S>
    __device__ static void tile(const unsigned char* buf, int64_t j0, const Eps2& e2s,
                                I (&is)[IT], Acc (&ac)[IT], int sl)
    {
        const float4* sA = reinterpret_cast<const float4*>(buf);
        const float4* sB = reinterpret_cast<const float4*>(buf + TJ * 16);
        const float2* sC = reinterpret_cast<const float2*>(buf + TJ * 32);
        const float eps2 = e2s.h;
        float ax[IT], ay[IT], az[IT], jx[IT], jy[IT], jz[IT], ph[IT];
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            ax[q] = ay[q] = az[q] = ph[q] = 0.f;
            if (SPJ) {
                jx[q] = ac[q].jx.hi, jy[q] = ac[q].jy.hi, jz[q] = ac[q].jz.hi;
            } else {
                jx[q] = jy[q] = jz[q] = 0.f;
            }
        }
#pragma unroll 4
        for (int u = 0; u < TJ / S; ++u) {
            const int k = sl + S * u;
            const float4 A = sA[k];
            const float4 B = sB[k];
            const float2 C = sC[k];
#pragma unroll
            for (int q = 0; q < IT; ++q) {
                const float dx = (A.x - is[q].xh) + (B.x - is[q].xl);
                const float dy = (A.y - is[q].yh) + (B.y - is[q].yl);
                const float dz = (A.z - is[q].zh) + (B.z - is[q].zl);
                const float dvx = B.w - is[q].vx;
                const float dvy = C.x - is[q].vy;
                const float dvz = C.y - is[q].vz;
                const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                float ri = rsqrtf(r2);
                if (MASK) ri = (j0 + k == is[q].p) ? 0.f : ri;
                const float mr = A.w * ri;
                const float ri2 = ri * ri;
                const float g = mr * ri2;
                const float rv = fmaf(dx, dvx, fmaf(dy, dvy, dz * dvz));
                const float t = rv * (-3.f * ri2);
                ax[q] = fmaf(g, dx, ax[q]);
                ay[q] = fmaf(g, dy, ay[q]);
                az[q] = fmaf(g, dz, az[q]);
                jx[q] = fmaf(g, fmaf(t, dx, dvx), jx[q]);
                jy[q] = fmaf(g, fmaf(t, dy, dvy), jy[q]);
                jz[q] = fmaf(g, fmaf(t, dz, dvz), jz[q]);
                ph[q] += mr;
            }
        }
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            ac[q].ax.fold(ax[q]), ac[q].ay.fold(ay[q]), ac[q].az.fold(az[q]);
            if (SPJ) {
                ac[q].jx.hi = jx[q], ac[q].jy.hi = jy[q], ac[q].jz.hi = jz[q];
            } else {
                ac[q].jx.fold(jx[q]), ac[q].jy.fold(jy[q]), ac[q].jz.fold(jz[q]);
            }
            ac[q].ph.fold(ph[q]);
        }
    }

    static constexpr int NV = 7;  // reduced values: acc (3), jerk (3), pot
    using TV = DSPair;
    __device__ static void values(const Acc& a, TV (&v)[NV])
    {
        v[0] = ds_pair_of(a.ax), v[1] = ds_pair_of(a.ay), v[2] = ds_pair_of(a.az);
        v[3] = ds_pair_of(a.jx), v[4] = ds_pair_of(a.jy), v[5] = ds_pair_of(a.jz);
        v[6] = ds_pair_of(a.ph);
        v[6].h = -v[6].h, v[6].l = -v[6].l;
    }
};

// Double-single ("float-float") precision: the pair formulas of Eqs. acc,
// jrk and pot carried as unevaluated sums hi + lo of two FP32 numbers.  Each
// product is formed exactly with an FMA (TwoProd) and each sum with TwoSum;
// the rsqrt estimate is refined through its exact residual 1 - r^2 y^2, and
// only second-order terms (lo * lo) are dropped.  The result carries about
// 44 bits, so cancellation among pair terms (near neighbours around a
// particle with a small net acceleration or jerk) costs no accuracy at the
// 1e-6 level.  Positions and velocities arrive as grid-aligned splits, so
// their differences take one exact subtraction and a Fast2Sum (grid_diff).
// (ah + al) * (bh + bl) to first order: (p, e) with p = fl(ah * bh).
__device__ __forceinline__ void ds_mul(float ah, float al, float bh, float bl, float& p,
                                       float& e)
{
    two_prod(ah, bh, p, e);
    e = __fmaf_rn(ah, bl, __fmaf_rn(al, bh, e));
}

// i state and accumulators of the double-single pair (DS and HYBRID).
struct DSI {
    float xh, yh, zh, xl, yl, zl;
    float vxh, vyh, vzh, vxl, vyl, vzl;
    int p;
};
struct DSAccs {
    DSAcc ax, ay, az, jx, jy, jz, ph;
    __device__ void zero()
    {
        ax.zero(), ay.zero(), az.zero(), jx.zero(), jy.zero(), jz.zero(), ph.zero();
    }
    __device__ void values(DSPair (&v)[7]) const
    {
        v[0] = ds_pair_of(ax), v[1] = ds_pair_of(ay), v[2] = ds_pair_of(az);
        v[3] = ds_pair_of(jx), v[4] = ds_pair_of(jy), v[5] = ds_pair_of(jz);
        v[6] = ds_pair_of(ph);
        v[6].h = -v[6].h, v[6].l = -v[6].l;
    }
};

__device__ __forceinline__ void ds_load_i(const ForceParams& f, int p, DSI& s)
{
    s.p = p;
    if (p < 0) {
        s.xh = s.yh = s.zh = s.xl = s.yl = s.zl = 0.f;
        s.vxh = s.vyh = s.vzh = s.vxl = s.vyl = s.vzl = 0.f;
        return;
    }
    const float4 A = __ldg(static_cast<const float4*>(f.jl0) + p);
    const float4 B = __ldg(static_cast<const float4*>(f.jl1) + p);
    const float4 C = __ldg(static_cast<const float4*>(f.jl2) + p);
    const float4 D = __ldg(static_cast<const float4*>(f.jl3) + p);
    s.xh = A.x, s.yh = A.y, s.zh = A.z;
    s.xl = B.x, s.yl = B.y, s.zl = B.z;
    s.vxh = C.x, s.vyh = C.y, s.vzh = C.z;
    s.vxl = D.x, s.vyl = D.y, s.vzl = D.z;
}

// (jh + jl) - (ih + il) for double-single values whose hi parts share no
// grid (the hybrid layout's velocities): TwoSum of the hi parts, the lo
// parts added to its error, renormalised by TwoSum.
__device__ __forceinline__ void ds_diff(float jh, float jl, float ih, float il, float& dh,
                                        float& dl)
{
    float s, e;
    two_sum(jh, -ih, s, e);
    e = __fadd_rn(e, __fsub_rn(jl, il));
    two_sum(s, e, dh, dl);
}

// One pair (i = s, j = layout record A..D at slot j) in double-single,
// added to the accumulators.  With MASK the self pair (j == s.p) adds zero.
// GRIDV: the velocity hi parts lie on the layout's grid (DS); otherwise
// (HYBRID) they are plain FP32 values.
template <bool MASK, bool GRIDV = true>
__device__ __forceinline__ void ds_pair(const float4& A, const float4& B, const float4& C,
                                        const float4& D, const DSI& s, float e2h, float e2l,
                                        int64_t j, DSAccs& ac)
{
    float dxh, dxl, dyh, dyl, dzh, dzl;
    grid_diff(A.x, B.x, s.xh, s.xl, dxh, dxl);
    grid_diff(A.y, B.y, s.yh, s.yl, dyh, dyl);
    grid_diff(A.z, B.z, s.zh, s.zl, dzh, dzl);
    float vxh, vxl, vyh, vyl, vzh, vzl;
    if (GRIDV) {
        grid_diff(C.x, D.x, s.vxh, s.vxl, vxh, vxl);
        grid_diff(C.y, D.y, s.vyh, s.vyl, vyh, vyl);
        grid_diff(C.z, D.z, s.vzh, s.vzl, vzh, vzl);
    } else {
        ds_diff(C.x, D.x, s.vxh, s.vxl, vxh, vxl);
        ds_diff(C.y, D.y, s.vyh, s.vyl, vyh, vyl);
        ds_diff(C.z, D.z, s.vzh, s.vzl, vzh, vzl);
    }
    // r^2 = dx^2 + dy^2 + dz^2 + eps^2 (all terms >= 0)
    float px, pxe, py, pye, pz, pze;
    ds_mul(dxh, dxl, dxh, dxl, px, pxe);
    ds_mul(dyh, dyl, dyh, dyl, py, pye);
    ds_mul(dzh, dzl, dzh, dzl, pz, pze);
    float s1, e1, s2, e2, r2h, e3;
    two_sum(px, py, s1, e1);
    two_sum(s1, pz, s2, e2);
    two_sum(s2, e2h, r2h, e3);
    const float r2l = __fadd_rn(__fadd_rn(__fadd_rn(pxe, pye), __fadd_rn(pze, e1)),
                                __fadd_rn(__fadd_rn(e2, e3), e2l));
    // 1/r: hardware estimate y, refined by the exact residual
    // h = 1 - r^2 y^2, 1/r = y (1 + h/2 + O(h^2)).
    float y = rsqrtf(r2h);
    if (MASK) y = (j == s.p) ? 0.f : y;
    float y2, ey2;
    two_prod(y, y, y2, ey2);
    float h = __fmaf_rn(-r2h, y2, 1.f);
    h = __fmaf_rn(-r2h, ey2, h);
    h = __fmaf_rn(-r2l, y2, h);
    if (MASK) h = (j == s.p) ? 0.f : h;
    const float ril = __fmul_rn(0.5f, __fmul_rn(y, h));
    // m / r and 1 / r^2, then g = m / r^3
    float mrh, mrl;
    ds_mul(A.w, B.w, y, ril, mrh, mrl);
    const float ri2h = y2;
    const float ri2l = __fmaf_rn(__fadd_rn(y, y), ril, ey2);
    float gh, gl;
    ds_mul(mrh, mrl, ri2h, ri2l, gh, gl);
    // acceleration terms g * dr
    float t0, t1;
    ds_mul(gh, gl, dxh, dxl, t0, t1);
    ac.ax.add(t0, t1);
    ds_mul(gh, gl, dyh, dyl, t0, t1);
    ac.ay.add(t0, t1);
    ds_mul(gh, gl, dzh, dzl, t0, t1);
    ac.az.add(t0, t1);
    ac.ph.add(mrh, mrl);
    // r.v, then tau = -3 (r.v) / r^2
    float qx, qxe, qy, qye, qz, qze;
    ds_mul(dxh, dxl, vxh, vxl, qx, qxe);
    ds_mul(dyh, dyl, vyh, vyl, qy, qye);
    ds_mul(dzh, dzl, vzh, vzl, qz, qze);
    float u1, f1, rvh, f2;
    two_sum(qx, qy, u1, f1);
    two_sum(u1, qz, rvh, f2);
    const float rvl = __fadd_rn(__fadd_rn(qxe, qye), __fadd_rn(__fadd_rn(qze, f1), f2));
    float ch, cl;
    two_prod(-3.f, ri2h, ch, cl);
    cl = __fmaf_rn(-3.f, ri2l, cl);
    float tauh, taul;
    ds_mul(rvh, rvl, ch, cl, tauh, taul);
    // jerk terms g * (dv + tau dr)
    float wh, wl, th_, tl_, we;
    ds_mul(tauh, taul, dxh, dxl, th_, tl_);
    two_sum(vxh, th_, wh, we);
    wl = __fadd_rn(we, __fadd_rn(vxl, tl_));
    ds_mul(gh, gl, wh, wl, t0, t1);
    ac.jx.add(t0, t1);
    ds_mul(tauh, taul, dyh, dyl, th_, tl_);
    two_sum(vyh, th_, wh, we);
    wl = __fadd_rn(we, __fadd_rn(vyl, tl_));
    ds_mul(gh, gl, wh, wl, t0, t1);
    ac.jy.add(t0, t1);
    ds_mul(tauh, taul, dzh, dzl, th_, tl_);
    two_sum(vzh, th_, wh, we);
    wl = __fadd_rn(we, __fadd_rn(vzl, tl_));
    ds_mul(gh, gl, wh, wl, t0, t1);
    ac.jz.add(t0, t1);
}

template <int IT>
struct PolicyDS {
    static constexpr bool GUARDED = false;
    static constexpr int MIN_CTAS = 1;
    static constexpr int CHUNKS = 1;
    static constexpr int NARR = 4;
    __host__ __device__ static constexpr int elem(int a) { return a < 4 ? 16 : 0; }
    static constexpr int TILE_BYTES = TJ * 64;
    static constexpr int STAGES = 2;

    using I = DSI;
    using Acc = DSAccs;

    __device__ static void load_i(const ForceParams& f, int p, int, I& s) { ds_load_i(f, p, s); }

    template <bool MASK, int S>
    __device__ static void tile(const unsigned char* buf, int64_t j0, const Eps2& e2s,
                                I (&is)[IT], Acc (&ac)[IT], int sl)
    {
        const float4* sA = reinterpret_cast<const float4*>(buf);
        const float4* sB = reinterpret_cast<const float4*>(buf + TJ * 16);
        const float4* sC = reinterpret_cast<const float4*>(buf + TJ * 32);
        const float4* sD = reinterpret_cast<const float4*>(buf + TJ * 48);
        const float e2h = e2s.h;
        const float e2l = e2s.l;
#pragma unroll 1
        for (int u = 0; u < TJ / S; ++u) {
            const int k = sl + S * u;
            const float4 A = sA[k];
            const float4 B = sB[k];
            const float4 C = sC[k];
            const float4 D = sD[k];
#pragma unroll
            for (int q = 0; q < IT; ++q) ds_pair<MASK>(A, B, C, D, is[q], e2h, e2l, j0 + k, ac[q]);
        }
    }

    static constexpr int NV = 7;
    using TV = DSPair;
    __device__ static void values(const Acc& a, TV (&v)[NV]) { a.values(v); }
};

// Hybrid precision (no counterpart in the paper, which evaluates every pair
// the same way): each pair in FP32 unless it is a near pair, which is
// evaluated in double-single instead.  A pair is near when its acceleration
// term could exceed THETA |a_i| or its jerk term THETA |j_i|:
//   G m_j / r^2 <= THETA |a_i|          unless  r^2 < G m_j / (THETA |a_i|)
//   4 G m_j |dv| / r^3 <= THETA |j_i|   unless  r^2 < (G m_j)^(2/3) (4 V_i / (THETA |j_i|))^(2/3)
// with r^2 the softened distance, V_i = |v_i| + sqrt(3) B_v >= |v_j - v_i|,
// and |a_i|, |j_i| the particle's values at its last correction (its state
// a, j); a particle with no such values yet (a = j = 0) treats every pair as
// near, so the first evaluation after a load is plain DS.
//
// Two tile paths.  The j layout is in spatial order (a space-filling curve
// per system) and the active list in the same order, so a tile's 64 j and a
// warp's i are each close together in space.  The predictor stores a box
// around each tile and its largest G m and (G m)^(2/3); when the box is far
// enough from every i of the warp that no pair of the tile can be near by
// the test above (the far-tile test, evaluated with the box's distance and
// largest masses), the warp takes the far path: every pair in FP32 with no
// per-pair test, terms summed in FP32 runs of HY_RUN_FAR j (the whole tile:
// each term is small there, so one run per tile keeps the rounding of the
// run sums at the level of the shorter runs of the near path).  Any other tile
// takes the near path: the per-pair test, far pairs in FP32 in runs of
// HY_RUN_NEAR j (short: these tiles hold the largest far terms, side by side
// in space, and long runs of them raise the rounding of the run sums enough
// to switch on the integration guard below for many more particles), near
// pairs marked in a per-lane mask
// during the FP32 pass and evaluated in double-single after it, each lane
// walking its own list, so the warp runs the DS pair about
// max-over-lanes(near pairs in the tile) times per tile.  Each run is folded
// into double-single accumulators, so far-field rounding stays at the FP32
// level of each term and never accumulates; the rsqrt estimate is refined
// once through its residual.  Velocity differences of far pairs are taken
// between FP32 velocities (the layout stores v as its FP32 value plus the
// rest), positions as double-single differences.  With SPJ the far pairs'
// jerk is instead one plain FP32 sum across the warp's whole range of j, the
// paper's accumulation (Sec. 4, Fig. err_snp_djerk), for the study of its
// effect on an integration.
constexpr float HY_THETA = 0.1f;
constexpr int HY_RUN_FAR = 64;
constexpr int HY_RUN_NEAR = 8;
// Integration guard.  The Hermite interpolation divides a0 - a1 by dt^3
// (crackle), so an absolute force noise da sets a floor 12 da / dt^3 under
// the crackle that Eq. timestep sees; once that floor rivals the true value
// the timestep shrinks and keeps shrinking.  Each evaluation estimates its
// far-field noise from the FP32 roundings it made, bounded through the run
// sums: with b = G m / r^2 the |a| bound of a far pair, each run contributes
// (sum of its b)^2 >= sum of its b^2, and the estimate is
// 2 u sqrt(sum over runs of (sum b)^2).  When the last estimate exceeds
// HY_GUARD * eta |j| dt / 12 (the crackle scale of the particle's current
// step), the particle is evaluated entirely in double-single.  Switching
// between the two precisions itself steps a0 - a1 by the full noise, so the
// guard has hysteresis: once on, it stays on until the ratio falls below
// HY_GUARD_OFF (the stored estimate carries the guard state in its sign).
constexpr double HY_GUARD = 0.03;
constexpr double HY_GUARD_OFF = 0.1;  // of the turn-on level
constexpr double HY_U = 5.9604644775390625e-8;  // 2^-24

struct HybridI : DSI {
    float ca, cj;   // natural near test: r^2 < max(Gm_j * ca, (Gm_j)^(2/3) * cj)
    bool all_near;  // integration guard: every pair in double-single
    int particle;
};
struct HybridAcc : DSAccs {
    float q;  // far-field noise estimate: squared pair bounds and run sums
    __device__ void zero()
    {
        DSAccs::zero();
        q = 0.f;
    }
};

template <int IT, bool SPJ = false>
struct PolicyHybrid {
    static constexpr bool GUARDED = true;
    // registers capped so that three CTAs (two i per lane) or four (one)
    // fit on an SM
    static constexpr int MIN_CTAS = IT > 1 ? 3 : 4;
    static constexpr int CHUNKS = 4;  // tiles of unequal cost
    static constexpr int NARR = 4;
    __host__ __device__ static constexpr int elem(int a) { return a < 4 ? 16 : 0; }
    static constexpr int TILE_BYTES = TJ * 64;
    static constexpr int STAGES = 3;
    static constexpr int NV = 8;  // acc, jerk, pot and the noise estimate

    using I = HybridI;
    using Acc = HybridAcc;

    __device__ static void load_i(const ForceParams& f, int p, int particle, I& s)
    {
        ds_load_i(f, p, s);
        s.ca = s.cj = 0.f;
        s.all_near = false;
        s.particle = particle;
        if (p < 0) return;
        // The near radius and the guard are thresholds, not results: FP32
        // is ample, and the state's doubles are narrowed with integer
        // operations (f32_trunc), so this per-group set-up stays off GB300's
        // narrow FP64 pipe, which every warp of a launch would queue on.
        const int64_t n = f.n;
        float a2 = 0.f, j2 = 0.f;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float a = f32_trunc(f.st_a[c * n + particle]);
            const float jj = f32_trunc(f.st_j[c * n + particle]);
            a2 = fmaf(a, a, a2);
            j2 = fmaf(jj, jj, j2);
        }
        const float A = sqrtf(a2), J = sqrtf(j2);
        const float vi = sqrtf(s.vxh * s.vxh + s.vyh * s.vyh + s.vzh * s.vzh);
        const float V = vi + 1.7320509f * __uint_as_float(*f.bound_v) * 1.0001f;
        // 1/0 = inf: no estimate yet, every pair is near
        s.ca = 1.f / (HY_THETA * A);
        const float x = 4.f * V / (HY_THETA * J);
        const float cb = cbrtf(x);
        s.cj = cb * cb;
        const float hq = f32_trunc(f.st_hq[particle]);
        const float noise = 2.f * static_cast<float>(HY_U) * sqrtf(fabsf(hq));
        const float scale = f.guard_eta * J * f32_trunc(f.st_dt[particle]);
        // ratio = 12 noise / scale, compared without a division
        s.all_near = hq < 0.f ? 12.f * noise > static_cast<float>(HY_GUARD_OFF) * scale
                              : 12.f * noise > scale;
    }

    using TV = DSPair;
    __device__ static void values(const Acc& a, TV (&v)[NV])
    {
        DSPair w[7];
        a.values(w);
#pragma unroll
        for (int c = 0; c < 7; ++c) v[c] = w[c];
        v[7].h = a.q, v[7].l = 0.f;
    }

    __device__ static void finish(const ForceParams& f, const I& s, int64_t,
                                  const double (&v)[NV])
    {
        // a guarded evaluation stores its estimate negated (the guard state)
        if (s.particle >= 0) f.st_hq[s.particle] = s.all_near ? -v[7] : v[7];
    }

    __device__ static bool guarded(const I& s) { return s.all_near; }

    // The far-tile test of one i particle against the tile's box: true when
    // no pair of the tile can be near.  The predictor leaves the box in the
    // fourth component of the tile's first eight D records (lo_x, lo_y,
    // lo_z, max G m, hi_x, hi_y, hi_z, max (G m)^(2/3)), so it comes with
    // the staged tile.  It holds the tile's grid-rounded positions; the
    // 0.999 keeps the test on the safe side of that rounding.
    __device__ static bool tile_far(const unsigned char* buf, const I& s, float e2h)
    {
        if (s.p < 0) return true;  // an empty lane
        const float4* sD = reinterpret_cast<const float4*>(buf + TJ * 48);
        const float4 lo = make_float4(sD[0].w, sD[1].w, sD[2].w, sD[3].w);
        const float4 hi = make_float4(sD[4].w, sD[5].w, sD[6].w, sD[7].w);
        const float dx = fmaxf(fmaxf(lo.x - s.xh, s.xh - hi.x), 0.f);
        const float dy = fmaxf(fmaxf(lo.y - s.yh, s.yh - hi.y), 0.f);
        const float dz = fmaxf(fmaxf(lo.z - s.zh, s.zh - hi.z), 0.f);
        const float d2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, e2h))) * 0.999f;
        return d2 >= fmaxf(lo.w * s.ca, hi.w * s.cj);
    }

    // Far path: no pair of the tile is near for any lane of the warp, and no
    // lane's own particle is in it.  Lane slice sl takes records sl + S u.
    template <int S>
    __device__ static void far_tile(const unsigned char* buf, const Eps2& e2s, I (&is)[IT],
                                    Acc (&ac)[IT], int sl)
    {
        constexpr int R = TJ / S;
        constexpr int RUN = R < HY_RUN_FAR ? R : HY_RUN_FAR;
        const float4* sA = reinterpret_cast<const float4*>(buf);
        const float4* sB = reinterpret_cast<const float4*>(buf + TJ * 16);
        const float4* sC = reinterpret_cast<const float4*>(buf + TJ * 32);
        const float e2h = e2s.h;
#pragma unroll 1
        for (int u0 = 0; u0 < R; u0 += RUN) {
            float ax[IT], ay[IT], az[IT], jx[IT], jy[IT], jz[IT], ph[IT], bs[IT];
#pragma unroll
            for (int q = 0; q < IT; ++q) {
                ax[q] = ay[q] = az[q] = ph[q] = bs[q] = 0.f;
                if (SPJ) {  // the jerk: one plain FP32 sum across the warp's j
                    jx[q] = ac[q].jx.hi, jy[q] = ac[q].jy.hi, jz[q] = ac[q].jz.hi;
                } else {
                    jx[q] = jy[q] = jz[q] = 0.f;
                }
            }
#pragma unroll 4
            for (int du = 0; du < RUN; ++du) {
                const int k = sl + S * (u0 + du);
                const float4 A = sA[k];
                const float4 B = sB[k];
                const float4 C = sC[k];
#pragma unroll
                for (int q = 0; q < IT; ++q) {
                    const DSI& s = is[q];
                    const float dx = (A.x - s.xh) + (B.x - s.xl);
                    const float dy = (A.y - s.yh) + (B.y - s.yl);
                    const float dz = (A.z - s.zh) + (B.z - s.zl);
                    const float dvx = C.x - s.vxh;
                    const float dvy = C.y - s.vyh;
                    const float dvz = C.z - s.vzh;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, e2h)));
                    float y = rsqrtf(r2);
                    const float h = fmaf(-r2, y * y, 1.f);
                    y = fmaf(0.5f * y, h, y);
                    const float mr = A.w * y;
                    bs[q] = fmaf(mr, y, bs[q]);
                    const float ri2 = y * y;
                    const float g = mr * ri2;
                    const float rv = fmaf(dx, dvx, fmaf(dy, dvy, dz * dvz));
                    const float t = rv * (-3.f * ri2);
                    ax[q] = fmaf(g, dx, ax[q]);
                    ay[q] = fmaf(g, dy, ay[q]);
                    az[q] = fmaf(g, dz, az[q]);
                    jx[q] = fmaf(g, fmaf(t, dx, dvx), jx[q]);
                    jy[q] = fmaf(g, fmaf(t, dy, dvy), jy[q]);
                    jz[q] = fmaf(g, fmaf(t, dz, dvz), jz[q]);
                    ph[q] += mr;
                }
            }
#pragma unroll
            for (int q = 0; q < IT; ++q) {
                ac[q].ax.fold(ax[q]), ac[q].ay.fold(ay[q]), ac[q].az.fold(az[q]);
                if (SPJ) {
                    ac[q].jx.hi = jx[q], ac[q].jy.hi = jy[q], ac[q].jz.hi = jz[q];
                } else {
                    ac[q].jx.fold(jx[q]), ac[q].jy.fold(jy[q]), ac[q].jz.fold(jz[q]);
                }
                ac[q].ph.fold(ph[q]);
                ac[q].q = fmaf(bs[q], bs[q], ac[q].q);
            }
        }
    }

    // Near path.  GUARD: some lane of the warp has the integration guard on
    // (rare); the other instantiation assumes none has, so near is the
    // natural test and the noise estimate reuses the far-pair factor m / r.
    template <bool MASK, bool GUARD, int S>
    __device__ static void tile(const unsigned char* buf, int64_t j0, const Eps2& e2s,
                                I (&is)[IT], Acc (&ac)[IT], int sl)
    {
        static_assert(TJ == 64, "one 64-bit near mask per lane and tile");
        // this lane's records: tile slots sl + S u, u < R, in runs of RUN
        constexpr int R = TJ / S;
        constexpr int RUN = R < HY_RUN_NEAR ? R : HY_RUN_NEAR;
        const float4* sA = reinterpret_cast<const float4*>(buf);
        const float4* sB = reinterpret_cast<const float4*>(buf + TJ * 16);
        const float4* sC = reinterpret_cast<const float4*>(buf + TJ * 32);
        const float4* sD = reinterpret_cast<const float4*>(buf + TJ * 48);
        const float e2h = e2s.h;
        const float e2l = e2s.l;
        // Pass 1: every pair in FP32; near pairs add nothing here and are
        // marked in a per-lane 64-bit mask (bit u = slot sl + S u).
        uint32_t nlo[IT], nhi[IT];
#pragma unroll
        for (int q = 0; q < IT; ++q) nlo[q] = nhi[q] = 0u;
#pragma unroll 1
        for (int u0 = 0; u0 < R; u0 += RUN) {
            float ax[IT], ay[IT], az[IT], jx[IT], jy[IT], jz[IT], ph[IT], bs[IT];
            uint32_t run[IT];
#pragma unroll
            for (int q = 0; q < IT; ++q) {
                ax[q] = ay[q] = az[q] = ph[q] = bs[q] = 0.f;
                if (SPJ) {
                    jx[q] = ac[q].jx.hi, jy[q] = ac[q].jy.hi, jz[q] = ac[q].jz.hi;
                } else {
                    jx[q] = jy[q] = jz[q] = 0.f;
                }
                run[q] = 0u;
            }
#pragma unroll 4
            for (int du = 0; du < RUN; ++du) {
                const int k = sl + S * (u0 + du);
                const float4 A = sA[k];
                const float4 B = sB[k];
                const float4 C = sC[k];
#pragma unroll
                for (int q = 0; q < IT; ++q) {
                    const DSI& s = is[q];
                    // hi parts share one grid, so each hi difference is exact
                    const float dx = (A.x - s.xh) + (B.x - s.xl);
                    const float dy = (A.y - s.yh) + (B.y - s.yl);
                    const float dz = (A.z - s.zh) + (B.z - s.zl);
                    const float dvx = C.x - s.vxh;
                    const float dvy = C.y - s.vyh;
                    const float dvz = C.z - s.vzh;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, e2h)));
                    const bool self = MASK && (j0 + k == s.p);
                    const bool nat = r2 < fmaxf(A.w * is[q].ca, C.w * is[q].cj);
                    const bool near = (nat || (GUARD && is[q].all_near)) && !self;
                    // rsqrt refined once: y (1 + h/2) with the residual
                    // h = 1 - r^2 y^2 taken from the rounded y^2 (an error of
                    // at most an ulp of h, unbiased)
                    float y = rsqrtf(r2);
                    const float h = fmaf(-r2, y * y, 1.f);
                    y = fmaf(0.5f * y, h, y);
                    if (self) y = 0.f;  // r = 0 when eps = 0: keep inf out of every term
                    const float mr0 = A.w * y;
                    // near pairs (and the self pair, whose y is 0) add nothing
                    // here: every FP32 term below carries the factor m / r.
                    // The noise estimate sums m / r^2 over the pairs the
                    // natural test calls far.
                    float mr;
                    if (GUARD) {
                        bs[q] += (nat || self) ? 0.f : mr0 * y;
                        mr = (self || near) ? 0.f : mr0;
                    } else {
                        mr = nat ? 0.f : mr0;
                        bs[q] = fmaf(mr, y, bs[q]);
                    }
                    const float ri2 = y * y;
                    const float g = mr * ri2;
                    const float rv = fmaf(dx, dvx, fmaf(dy, dvy, dz * dvz));
                    const float t = rv * (-3.f * ri2);
                    ax[q] = fmaf(g, dx, ax[q]);
                    ay[q] = fmaf(g, dy, ay[q]);
                    az[q] = fmaf(g, dz, az[q]);
                    jx[q] = fmaf(g, fmaf(t, dx, dvx), jx[q]);
                    jy[q] = fmaf(g, fmaf(t, dy, dvy), jy[q]);
                    jz[q] = fmaf(g, fmaf(t, dz, dvz), jz[q]);
                    ph[q] += mr;
                    run[q] |= static_cast<uint32_t>(near) << du;
                }
            }
#pragma unroll
            for (int q = 0; q < IT; ++q) {
                ac[q].ax.fold(ax[q]), ac[q].ay.fold(ay[q]), ac[q].az.fold(az[q]);
                if (SPJ) {
                    ac[q].jx.hi = jx[q], ac[q].jy.hi = jy[q], ac[q].jz.hi = jz[q];
                } else {
                    ac[q].jx.fold(jx[q]), ac[q].jy.fold(jy[q]), ac[q].jz.fold(jz[q]);
                }
                ac[q].ph.fold(ph[q]);
                ac[q].q = fmaf(bs[q], bs[q], ac[q].q);
                if (u0 < 32) nlo[q] |= run[q] << u0;
                else nhi[q] |= run[q] << (u0 - 32);
            }
        }
        // Pass 2: the near pairs in double-single, each lane walking its own
        // mask; the warp loops max_lane(popcount) times, not once per j.
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            uint32_t lo = nlo[q], hi = nhi[q];
            while (__any_sync(0xffffffffu, (lo | hi) != 0u)) {
                if ((lo | hi) != 0u) {
                    int u;
                    if (lo) {
                        u = __ffs(lo) - 1;
                        lo &= lo - 1u;
                    } else {
                        u = 32 + __ffs(hi) - 1;
                        hi &= hi - 1u;
                    }
                    const int k = sl + S * u;
                    ds_pair<false, false>(sA[k], sB[k], sC[k], sD[k], is[q], e2h, e2l, j0 + k,
                                          ac[q]);
                }
            }
        }
    }

};

template <class K>
struct WarpSmem {
    static constexpr int BAR_BYTES = 128;  // STAGES mbarriers, padded
    static constexpr int BYTES = BAR_BYTES + K::STAGES * K::TILE_BYTES;
};

template <class K>
__device__ __forceinline__ void issue_tile(const ForceParams& f, unsigned char* stage,
                                           uint64_t* bar, int64_t jtile)
{
    mbar_arrive_expect_tx(bar, K::TILE_BYTES);
    const void* src[4] = {f.jl0, f.jl1, f.jl2, f.jl3};
    unsigned char* dst = stage;
#pragma unroll
    for (int a = 0; a < K::NARR; ++a) {
        const uint32_t bytes = TJ * K::elem(a);
        bulk_g2s(dst, static_cast<const unsigned char*>(src[a]) + jtile * (int64_t)bytes,
                 bytes, bar);
        dst += bytes;
    }
}

// Radix of the deterministic reduction tree over the warps sharing a group.
constexpr int RB = 16;
constexpr int RLEVELS = 4;  // RB^RLEVELS >= any warp count
constexpr int MAX_NV = 10;  // values a policy reduces (scratch is sized for the most)

// Chunk that holds flattened tile x when T tiles are cut into Pu ranges.
__device__ __forceinline__ int64_t owner_warp(int64_t x, int64_t T, int64_t Pu)
{
    return ((x + 1) * Pu - 1) / T;
}

// CTA mode: the most tiles per warp it takes on, and the most entries a
// thread loads in one batch when CTAs' entries are added (see force_kernel).
constexpr int64_t CTA_MAX_TILES = 4;
constexpr int CTA_BATCH = 16;

// Stream-K chunks per warp (largest; policies choose theirs) and the
// fewest tiles a chunk is cut down to.
constexpr int MAX_CHUNKS = 4;
constexpr int64_t CHUNK_MIN_TILES = 32;
constexpr int64_t DYN_MIN_TILES = 4;  // chunks handed out by the queue

// One i-group of a launch: up to 32*IT consecutive active-list entries of
// one system and the j tiles of that system, placed at flattened tile0.
struct GroupInfo {
    int64_t act_begin, act_count;  // active-list entries
    int64_t tile0, ntiles;         // flattened tiles of the group
    int64_t jtile0;                // first j tile of its system in the j layout
    int64_t jstride;               // tile walk: rank k -> j tile k * jstride mod ntiles
    int64_t pj_shift;              // j-layout slot of particle p = p + pj_shift
    Eps2 e2;
};

// A group walks its system's j tiles in the order k -> k * stride mod
// ntiles (a bijection, the stride being a prime that does not divide
// ntiles).  In the spatial order the tiles next to a group in space, where
// its near pairs are, sit side by side; walked in index order they would
// all fall to the one or two warps whose stream-K range covers them, and
// those warps would finish last.  The stride spreads them over the group's
// whole range, so equal tile counts per warp are also equal work.
__device__ __forceinline__ int64_t tile_stride(int64_t nt)
{
    const uint32_t m = static_cast<uint32_t>(nt);
    if (m <= 8u) return 1;
    const uint32_t primes[8] = {37u, 41u, 43u, 47u, 53u, 59u, 61u, 67u};
#pragma unroll
    for (int k = 0; k < 8; ++k)
        if (m % primes[k] != 0u) return static_cast<int64_t>(primes[k] % m);
    return 1;
}

// The j tile of rank k (0 <= k < ntiles) of a group.
__device__ __forceinline__ int64_t tile_at(const GroupInfo& g, int64_t k)
{
    if (g.ntiles < 65536)  // the product fits 32 bits: a much shorter division
        return static_cast<int64_t>((static_cast<uint32_t>(k) * static_cast<uint32_t>(g.jstride)) %
                                    static_cast<uint32_t>(g.ntiles));
    return static_cast<int64_t>((static_cast<uint64_t>(k) * static_cast<uint64_t>(g.jstride)) %
                                static_cast<uint64_t>(g.ntiles));
}

// One system over the whole j layout: groups of GI consecutive entries.
struct UniformPlan {
    static constexpr bool CHUNKED = true;
    int64_t n_act, G, NT, T, jstride, J0;
    Eps2 e2;
    int GI;
    template <int GI_>
    __device__ void init(const ForceParams& f)
    {
        GI = GI_;
        n_act = f.n_act_host >= 0 ? f.n_act_host : *f.n_act_dev;
        G = (n_act + GI_ - 1) / GI_;
        J0 = f.jt_hi > 0 ? f.jt_lo : 0;
        NT = f.jt_hi > 0 ? f.jt_hi - f.jt_lo : f.n_pad / TJ;
        T = G * NT;
        jstride = tile_stride(NT);
        e2 = make_eps2(f.eps2);
    }
    __device__ int64_t find(int64_t t, int) const { return t / NT; }
    __device__ GroupInfo group(int64_t g) const
    {
        GroupInfo gi;
        gi.act_begin = g * GI;
        gi.act_count = n_act - gi.act_begin < GI ? n_act - gi.act_begin : GI;
        gi.tile0 = g * NT;
        gi.ntiles = NT;
        gi.jtile0 = J0;
        gi.jstride = jstride;
        gi.pj_shift = 0;
        gi.e2 = e2;
        return gi;
    }
};

// Independent systems (ensemble): group descriptors from plan_launch.  The
// cost of a tile varies several-fold between systems and groups (far tiles,
// near tiles of compact systems, groups under the hybrid integration
// guard), so a launch may cut the tiles into several chunks per warp and
// hand them out from a queue (ForceParams::dyn_chunks).
struct ClusterPlan {
    static constexpr bool CHUNKED = false;
    const ForceParams* f;
    int64_t G, T;
    template <int GI_>
    __device__ void init(const ForceParams& fp)
    {
        f = &fp;
        G = fp.plan_scalars[0];
        T = fp.plan_scalars[1];
    }
    // The last group g with tile0[g] <= t, found by the whole warp (called
    // converged): each round the lanes test 32 evenly spaced tile0 entries
    // of [lo, hi), so a plan of G groups takes ceil(log32 G) rounds of one
    // load each instead of log2 G dependent loads.  tile0[lo] <= t holds
    // throughout (tile0[0] = 0), so lane 0's test always passes.
    __device__ int64_t find(int64_t t, int lane) const
    {
        int64_t lo = 0, hi = G;
        for (;;) {
            const int64_t step = hi - lo > 32 ? (hi - lo + 31) / 32 : 1;
            const int64_t k = lo + lane * step;
            const bool le = k < hi && f->grp_tile0[k] <= t;
            const uint32_t m = __ballot_sync(0xffffffffu, le);
            lo += static_cast<int64_t>(31 - __clz(m)) * step;
            if (step == 1) return lo;
            hi = lo + step < hi ? lo + step : hi;
        }
    }
    __device__ GroupInfo group(int64_t g) const
    {
        GroupInfo gi;
        const int c = f->grp_cluster[g];
        gi.act_begin = f->grp_act_begin[g];
        gi.act_count = f->grp_act_count[g];
        gi.tile0 = f->grp_tile0[g];
        gi.ntiles = f->grp_tile0[g + 1] - gi.tile0;
        gi.jtile0 = f->cl_joff[c] / TJ;
        gi.jstride = tile_stride(gi.ntiles);
        gi.pj_shift = f->cl_joff[c] - f->cl_off[c];
        gi.e2 = make_eps2(f->cl_eps2[c]);
        return gi;
    }
};

// CTA mode, after the tiles: this warp's sums (zeros if it had no tile) into
// its own ring, which no copy uses any more; the four warps added in warp
// order as the CTA's entry; the CTAs' entries of group cg added in a tree
// whose last CTA writes the results.  Kept out of line: inlined, it changed
// the register allocation of the tile loops and cost ~3 % on large blocks.
template <class K, int IT, int S>
__device__ __noinline__ void cta_finish(const ForceParams& f, unsigned char* smem,
                                        const typename K::I (&is)[IT],
                                        const typename K::Acc (&ac)[IT], const GroupInfo& cgi,
                                        int64_t cg, int64_t cR, int64_t crank)
{
    constexpr int IW = 32 / S;
    constexpr int GI = IW * IT;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int ir = lane % IW, sl = lane / IW;
    constexpr int NV = K::NV;
    using TV = typename K::TV;
    constexpr int VALS = NV * GI;
    constexpr int NTH = FORCE_WARPS * 32;
    constexpr int PARTS = VALS >= NTH ? 1 : NTH / VALS;
    static_assert(VALS * sizeof(TV) <= (size_t)K::STAGES * K::TILE_BYTES &&
                      PARTS * VALS <= (VALS > NTH ? VALS : NTH),
                  "a warp's ring holds the CTA-mode sums");
    auto ring_of = [&](int ww) {
        return reinterpret_cast<TV*>(smem + (size_t)ww * WarpSmem<K>::BYTES +
                                     WarpSmem<K>::BAR_BYTES);
    };
    TV v[IT][NV];
#pragma unroll
    for (int q = 0; q < IT; ++q) K::values(ac[q], v[q]);
#pragma unroll
    for (int o = IW; o < 32; o <<= 1)
#pragma unroll
        for (int q = 0; q < IT; ++q)
#pragma unroll
            for (int c = 0; c < NV; ++c) tree_xor(v[q][c], o);
    TV* mine = ring_of(wib);
    if (sl == 0) {
#pragma unroll
        for (int q = 0; q < IT; ++q)
#pragma unroll
            for (int c = 0; c < NV; ++c) mine[c * GI + q * IW + ir] = v[q][c];
    }
    __syncthreads();
    uint32_t* last_flag = reinterpret_cast<uint32_t*>(smem + 64);  // warp 0's barrier block
    const int tid = threadIdx.x;
    const int64_t key = cg * cR;  // slot of the group's first entry
    // Level 0: this CTA's entry, its warps' sums added in warp order.
    if (wib == 0) {
        for (int vi = lane; vi < VALS; vi += 32) {
            TV x;
            tree_zero(x);
#pragma unroll
            for (int ww = 0; ww < FORCE_WARPS; ++ww) tree_add(x, ring_of(ww)[vi]);
            tree_store(f.scratch, (size_t)(key + crank) * VALS + vi, x);
        }
    }
    // The entries meet in a tree, as the warps' sums do in warp mode, but
    // each chunk is added by all the threads of its last CTA, each thread
    // loading at most CTA_BATCH entries of one value in one batch: the
    // radix is CTA_BATCH times the parts the CTA's threads split a value
    // into.  Level L entry r sits in slot key + r * RADIX^L, and a chunk's
    // sum takes its first entry's slot.
    constexpr int RADIX = CTA_BATCH * PARTS;
    TV* part = ring_of(1);
    TV* fin = ring_of(2);
    int64_t kk = cR, r = crank, stride = 1;
    for (int level = 0;; ++level) {
        // every store of this CTA's entry precedes thread 0's release
        __syncthreads();
        const int64_t chunk = r / RADIX, first = chunk * RADIX;
        const int cs = static_cast<int>(kk - first < RADIX ? kk - first : RADIX);
        if (tid == 0) {
            uint32_t* cnt = f.counters + (size_t)level * f.counter_stride + key + chunk;
            const uint32_t prev = atomic_add_acq_rel_gpu(cnt, 1u);
            const bool last = prev == static_cast<uint32_t>(cs - 1);
            if (last) *cnt = 0u;  // the whole chunk is in: ready for the next launch
            *last_flag = last ? 1u : 0u;
        }
        __syncthreads();
        if (*last_flag == 0u) return;  // the whole CTA: another one carries the chunk on
        // (thread 0's acquire, passed on by the barrier, orders the loads below)
        const size_t e0 = (size_t)(key + first * stride) * VALS;
        const size_t es = (size_t)stride * VALS;
        auto sum_entries = [&](int vi, int u0, int u1) {  // u1 - u0 <= CTA_BATCH
            TV y[CTA_BATCH];
#pragma unroll
            for (int k = 0; k < CTA_BATCH; ++k)
                if (u0 + k < u1) tree_load(f.scratch, e0 + (size_t)(u0 + k) * es + vi, y[k]);
            TV x;
            tree_zero(x);
#pragma unroll
            for (int k = 0; k < CTA_BATCH; ++k)
                if (u0 + k < u1) tree_add(x, y[k]);
            return x;
        };
        if (PARTS == 1) {
            for (int vi = tid; vi < VALS; vi += NTH) fin[vi] = sum_entries(vi, 0, cs);
        } else {
            if (tid < PARTS * VALS) {
                const int vi = tid % VALS, pp = tid / VALS;
                part[pp * VALS + vi] = sum_entries(vi, cs * pp / PARTS, cs * (pp + 1) / PARTS);
            }
            __syncthreads();
            for (int vi = tid; vi < VALS; vi += NTH) {
                TV x;
                tree_zero(x);
                for (int pp = 0; pp < PARTS; ++pp) tree_add(x, part[pp * VALS + vi]);
                fin[vi] = x;
            }
        }
        __syncthreads();
        r = chunk;
        kk = (kk + RADIX - 1) / RADIX;
        stride *= RADIX;
        if (kk == 1) break;  // fin holds the group's sums
        for (int vi = tid; vi < VALS; vi += NTH)
            tree_store(f.scratch, (size_t)(key + r * stride) * VALS + vi, fin[vi]);
    }
    if (wib == 0 && sl == 0) {
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            const int64_t a = cgi.act_begin + q * IW + ir;
            if (a < cgi.act_begin + cgi.act_count) {
                double o[NV];
#pragma unroll
                for (int c = 0; c < NV; ++c) o[c] = tree_value(fin[c * GI + q * IW + ir]);
                f.acc[3 * a + 0] = o[0];
                f.acc[3 * a + 1] = o[1];
                f.acc[3 * a + 2] = o[2];
                f.jerk[3 * a + 0] = o[3];
                f.jerk[3 * a + 1] = o[4];
                f.jerk[3 * a + 2] = o[5];
                f.pot[a] = o[6];
                if constexpr (K::NV > 7) K::finish(f, is[q], a, o);
            }
        }
    }
}


// S: lanes per i (the j split inside a warp).  Lane = ir + IW sl: i slot ir
// of the warp's IW = 32 / S, j slice sl; the S slices of an i are summed with
// shuffles before the split-group tree.
template <class K, int IT, int S, class Plan, bool CTA>
__global__ void __launch_bounds__(FORCE_WARPS * 32, K::MIN_CTAS)
    force_kernel(const ForceParams f)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int64_t w = (int64_t)blockIdx.x * FORCE_WARPS + wib;
    const int64_t P = (int64_t)gridDim.x * FORCE_WARPS;

    static_assert(S == 1 || S == 2 || S == 4 || S == 8, "j split of 1, 2, 4 or 8 lanes");
    constexpr int IW = 32 / S;
    constexpr int GI = IW * IT;
    const int ir = lane % IW, sl = lane / IW;
    {
        // Launch variants tuned for different block sizes share one stream:
        // each works only inside its n_act window (read on the device, so
        // the host need not know the block size).
        const int na = f.n_act_host >= 0 ? f.n_act_host : *f.n_act_dev;
        if (na < f.nact_lo || na >= f.nact_hi) return;
    }
    Plan plan;
    plan.template init<GI>(f);
    const int64_t T = plan.T;
    if (T <= 0) return;
    // CTA mode (one system, few groups: at least four CTAs per group).  Group
    // g gets R consecutive CTAs, each a contiguous stretch of its tile walk,
    // cut in four for the CTA's warps.  The warps' sums meet in shared
    // memory, in warp order, and each CTA stores one entry; the last CTA of
    // the group to arrive adds the R entries with all its threads and
    // writes the results.  For small blocks that replaces the levels of the
    // warp tree below, each a chain of global-memory round trips, with one.
    // It is used while it leaves each warp at most CTA_MAX_TILES tiles: past
    // that the latency it saves is small against the stream-K balance.
    // (Only the CTA = true build carries it, the small-block launch variant:
    // the code of its reduction, present in the large-block build, cost that
    // build ~2 % through the register allocation of its tile loops.)
    bool cta = false;
    int64_t cg = 0, cR = 1, crank = 0;
    if constexpr (Plan::CHUNKED && CTA) {
        if (f.cta_mode && 4 * plan.G <= (int64_t)gridDim.x) {
            const int64_t rmax = (plan.NT + FORCE_WARPS - 1) / FORCE_WARPS;
            cR = gridDim.x / static_cast<uint32_t>(plan.G);  // G < gridDim.x / 4
            if (cR > rmax) cR = rmax;
            cta = plan.NT <= cR * FORCE_WARPS * CTA_MAX_TILES;
        }
        if (cta) {
            cg = blockIdx.x / static_cast<uint32_t>(cR);
            crank = blockIdx.x - static_cast<uint32_t>(cg * cR);
            if (cg >= plan.G) return;  // the whole CTA: no group left for it
        }
    }
    // The flattened (group, tile) space is cut into NCH equal chunks (the
    // stream-K split) and warp w takes chunks w, w + P, ...: KC chunks from
    // KC stretches of the space, so that regions of dearer tiles (the near
    // tiles of the hybrid precision crowd where the particles do) are shared
    // by all warps.  Chunks keep at least CHUNK_MIN_TILES tiles.
    //
    // Ensemble plans with dyn_chunks >= 2 cut the space into up to that many
    // chunks per warp instead, of at least DYN_MIN_TILES tiles: warp w takes
    // chunk w, then chunks P, P + 1, ... from a queue, in the order warps
    // come free, so warps whose tiles were cheap take more of them.  Chunk
    // bounds, and with them the split-group sums below, do not depend on
    // which warp takes a chunk.  Every warp makes exactly one fetch that
    // finds the queue empty, so the launch makes n_queued + P fetches, and
    // the one that draws the last value puts the queue word back to zero.
    const bool dyn = !Plan::CHUNKED && f.dyn_chunks > 1;
    int64_t KC = Plan::CHUNKED ? K::CHUNKS : (dyn ? f.dyn_chunks : 1);
    const int64_t min_tiles = dyn ? DYN_MIN_TILES : CHUNK_MIN_TILES;
    while (KC > 1 && T < P * KC * min_tiles) --KC;
    const int64_t NCH = cta ? 1 : (P * KC < T ? P * KC : T);
    if (!cta && !dyn && w >= NCH) return;
    const int64_t n_queued = dyn && NCH > P ? NCH - P : 0;
    auto next_chunk = [&](int64_t ch) -> int64_t {
        if (cta) return ch + 1;
        if (!dyn) return ch + P;
        uint32_t v = 0;
        if (lane == 0) {
            v = atomicAdd(f.queue, 1u);
            if (v == static_cast<uint32_t>(n_queued + P - 1)) atomicExch(f.queue, 0u);
        }
        v = __shfl_sync(0xffffffffu, v, 0);
        return v < n_queued ? P + static_cast<int64_t>(v) : NCH;
    };

    unsigned char* wsm = smem + (size_t)wib * WarpSmem<K>::BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(wsm);
    unsigned char* ring = wsm + WarpSmem<K>::BAR_BYTES;

    if (lane == 0) {
#pragma unroll
        for (int s = 0; s < K::STAGES; ++s) mbar_init(&bars[s], 1);
        fence_mbar_init();
    }
    __syncwarp();

    typename K::I is[IT];
    typename K::Acc ac[IT];
    // (32-bit: a warp's tiles and a system's j tiles stay below 2^31)
    uint32_t used = 0;    // tiles this warp has consumed: ring slot used % STAGES
    uint32_t issued = 0;  // tiles this warp has staged
    bool loaded = false;   // is[] and ac[] set up for a group
    bool aborted = false;  // a tile wait ran out (CTA mode: the CTA still meets)

    // i state of group gi's lanes, accumulators zeroed
    auto load_group = [&](const GroupInfo& gi) {
#pragma unroll
        for (int q = 0; q < IT; ++q) {
            const int64_t a = gi.act_begin + q * IW + ir;
            int p = -1, particle = -1;
            if (a < gi.act_begin + gi.act_count) {
                particle = f.idx[a];
                if (particle < 0 || particle >= f.n) {
                    atomicOr(f.status, ST_BADINDEX);
                    particle = -1;
                } else {
                    if (f.idx_map) particle = f.idx_map[particle];
                    p = static_cast<int>(particle + gi.pj_shift);
                }
            }
            K::load_i(f, p, particle, is[q]);
            ac[q].zero();
        }
        loaded = true;
    };

    for (int64_t ch = cta ? 0 : (w < NCH ? w : next_chunk(w)); ch < NCH; ch = next_chunk(ch)) {
    int64_t t0, t1;
    if (!cta) {
        t0 = T * ch / NCH;
        t1 = T * (ch + 1) / NCH;
    }
    if constexpr (Plan::CHUNKED) {
        if (cta) {
            int64_t c0, c1;
            if (plan.NT * cR < 0x7fffffff) {  // 32-bit divisions: much shorter
                const uint32_t nt = static_cast<uint32_t>(plan.NT), r = static_cast<uint32_t>(cR);
                c0 = nt * static_cast<uint32_t>(crank) / r;
                c1 = nt * static_cast<uint32_t>(crank + 1) / r;
            } else {
                c0 = plan.NT * crank / cR;
                c1 = plan.NT * (crank + 1) / cR;
            }
            const int64_t len = c1 - c0;
            t0 = cg * plan.NT + c0 + len * wib / FORCE_WARPS;
            t1 = cg * plan.NT + c0 + len * (wib + 1) / FORCE_WARPS;
        }
    }
    // Compute cursor (g, gi) and load cursor (lg, lgi): both start at the
    // group of tile t0; the load cursor runs STAGES tiles ahead.
    int64_t g = cta ? cg : plan.find(t0, lane);
    GroupInfo gi = plan.group(g);
    int64_t lg = g;
    GroupInfo lgi = gi;
    int64_t tl = t0;
    int32_t lpos = static_cast<int32_t>(tile_at(lgi, tl - lgi.tile0));  // j tile of the next load
    auto issue_next = [&]() {
        if (tl >= lgi.tile0 + lgi.ntiles) {
            while (tl >= lgi.tile0 + lgi.ntiles) lgi = plan.group(++lg);
            lpos = static_cast<int32_t>(tile_at(lgi, tl - lgi.tile0));
        }
        const int s = static_cast<int>(issued % K::STAGES);
        // (self-test: with unfed_first_tile the warp's first tile is never
        // staged, so its barrier never completes and the bounded wait runs out)
        if (lane == 0 && !(f.unfed_first_tile && issued == 0))
            issue_tile<K>(f, ring + s * K::TILE_BYTES, &bars[s], lgi.jtile0 + lpos);
        lpos += lgi.jstride;
        if (lpos >= lgi.ntiles) lpos -= lgi.ntiles;
        ++tl;
        ++issued;
    };
    // the ring is empty at a chunk's start: every staged tile was consumed
    for (int s = 0; s < K::STAGES && t0 + s < t1; ++s) issue_next();

    bool fresh = true;
    bool guard_any = false;  // some lane of this group has the hybrid guard on
    int32_t cpos = 0;        // j tile of the tile being computed (rank in the walk)

    for (int64_t t = t0; t < t1; ++t) {
        const uint32_t k = used;
        const int s = static_cast<int>(k % K::STAGES);
        const uint32_t parity = static_cast<uint32_t>((k / K::STAGES) & 1);
        while (t >= gi.tile0 + gi.ntiles) {
            gi = plan.group(++g);
            fresh = true;
        }
        if (fresh) {
            fresh = false;
            cpos = static_cast<int32_t>(tile_at(gi, t - gi.tile0));
            load_group(gi);
            if constexpr (K::GUARDED) {
                bool gq = false;
#pragma unroll
                for (int q = 0; q < IT; ++q) gq |= K::guarded(is[q]);
                guard_any = __any_sync(0xffffffffu, gq);
            }
        }
        const bool ok = mbar_wait_bounded(&bars[s], parity, f.wait_limit);
        if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0) atomicOr(f.status, ST_TIMEOUT);
            // Give up on this launch, but first let every bulk copy this warp
            // still has in flight (ring positions k .. issued - 1) land, each
            // wait bounded again, so no copy outlives the CTA.
            for (uint32_t kk = k; kk < issued; ++kk) {
                if (f.unfed_first_tile && kk == 0) continue;  // never issued
                mbar_wait_bounded(&bars[kk % K::STAGES],
                                  static_cast<uint32_t>((kk / K::STAGES) & 1));
            }
            if (!cta) return;
            aborted = true;  // no tile left in flight; meet the CTA below
            break;
        }
        ++used;
        const int64_t jt = t - gi.tile0;  // rank of the tile in the group's walk
        const int64_t j0 = (gi.jtile0 + cpos) * TJ;
        cpos += gi.jstride;
        if (cpos >= gi.ntiles) cpos -= gi.ntiles;
        bool self_here = false;
#pragma unroll
        for (int q = 0; q < IT; ++q)
            self_here |= (is[q].p >= j0 && is[q].p < j0 + TJ);
        const unsigned char* buf = ring + s * K::TILE_BYTES;
        const bool mask_self = __any_sync(0xffffffffu, self_here);
        if constexpr (K::GUARDED) {
            // the far path when no lane's particle is in the tile, no lane
            // has the guard on and the tile is far from every lane's i
            bool far = !mask_self && !guard_any;
            if (far) {
                const float e2h = gi.e2.h;
#pragma unroll
                for (int q = 0; q < IT; ++q) far &= K::tile_far(buf, is[q], e2h);
                far = __all_sync(0xffffffffu, far);
            }
            if (far) K::template far_tile<S>(buf, gi.e2, is, ac, sl);
            else if (guard_any) {
                if (mask_self) K::template tile<true, true, S>(buf, j0, gi.e2, is, ac, sl);
                else K::template tile<false, true, S>(buf, j0, gi.e2, is, ac, sl);
            } else {
                if (mask_self) K::template tile<true, false, S>(buf, j0, gi.e2, is, ac, sl);
                else K::template tile<false, false, S>(buf, j0, gi.e2, is, ac, sl);
            }
        } else {
            if (mask_self) K::template tile<true, S>(buf, j0, gi.e2, is, ac, sl);
            else K::template tile<false, S>(buf, j0, gi.e2, is, ac, sl);
        }
        __syncwarp();
        if (t + K::STAGES < t1) {
            if (lane == 0) fence_proxy_async_smem();
            issue_next();
        }

        if (!cta && (jt == gi.ntiles - 1 || t == t1 - 1)) {
            // This warp's share of group g is complete.  The warps that
            // share the group are summed by a radix-RB tree: within each
            // chunk of RB consecutive contributors the last to arrive adds
            // the chunk in order and carries the sum one level up.  Level-L
            // entry r lives in scratch slot key + r * RB^L (the first slot of
            // the chunk it replaces); each level has its own counters.
            const int64_t wf = owner_warp(gi.tile0, T, NCH);
            const int64_t wl = owner_warp(gi.tile0 + gi.ntiles - 1, T, NCH);
            constexpr int NV = K::NV;
            using TV = typename K::TV;
            TV v[IT][NV];
#pragma unroll
            for (int q = 0; q < IT; ++q) K::values(ac[q], v[q]);
            // the S slices of each i, summed in a fixed butterfly order
#pragma unroll
            for (int o = IW; o < 32; o <<= 1)
#pragma unroll
                for (int q = 0; q < IT; ++q)
#pragma unroll
                    for (int c = 0; c < NV; ++c) tree_xor(v[q][c], o);
            const int64_t key = wf + g;
            int64_t kk = wl - wf + 1;  // entries at this level
            int64_t r = ch - wf;       // my entry at this level
            int64_t stride = 1;
            bool final_here = true;
            for (int level = 0; kk > 1; ++level) {
                const size_t mine = (size_t)(key + r * stride) * NV * GI;
                if (sl == 0) {
#pragma unroll
                    for (int q = 0; q < IT; ++q)
#pragma unroll
                        for (int c = 0; c < NV; ++c)
                            tree_store(f.scratch, mine + c * GI + q * IW + ir, v[q][c]);
                }
                __threadfence();
                __syncwarp();
                const int64_t chunk = r / RB;
                const int64_t first = chunk * RB;
                const int64_t cs = kk - first < RB ? kk - first : RB;
                uint32_t* cnt = f.counters + (size_t)level * f.counter_stride + key + chunk;
                uint32_t prev = 0;
                if (lane == 0) prev = atomicAdd(cnt, 1u);
                prev = __shfl_sync(0xffffffffu, prev, 0);
                if (prev != static_cast<uint32_t>(cs - 1)) {
                    final_here = false;
                    break;
                }
                __threadfence();
                if (lane == 0) *cnt = 0u;
                // Entry by entry: each entry's NV values load together (and
                // two entries are in flight), then add into NV running sums;
                // every value still sums its entries in ascending order.
#pragma unroll
                for (int q = 0; q < IT; ++q) {
                    if (sl != 0) break;  // only slice 0 carries the sums on
#pragma unroll
                    for (int c = 0; c < NV; ++c) tree_zero(v[q][c]);
#pragma unroll 4
                    for (int64_t u = 0; u < cs; ++u) {
                        const size_t e = (size_t)(key + (first + u) * stride) * NV * GI + q * IW + ir;
                        TV x[NV];
#pragma unroll
                        for (int c = 0; c < NV; ++c) tree_load(f.scratch, e + c * GI, x[c]);
#pragma unroll
                        for (int c = 0; c < NV; ++c) tree_add(v[q][c], x[c]);
                    }
                }
                r = chunk;
                kk = (kk + RB - 1) / RB;
                stride *= RB;
            }
            if (final_here && sl == 0) {
#pragma unroll
                for (int q = 0; q < IT; ++q) {
                    const int64_t a = gi.act_begin + q * IW + ir;
                    if (a < gi.act_begin + gi.act_count) {
                        double o[NV];
#pragma unroll
                        for (int c = 0; c < NV; ++c) o[c] = tree_value(v[q][c]);
                        f.acc[3 * a + 0] = o[0];
                        f.acc[3 * a + 1] = o[1];
                        f.acc[3 * a + 2] = o[2];
                        f.jerk[3 * a + 0] = o[3];
                        f.jerk[3 * a + 1] = o[4];
                        f.jerk[3 * a + 2] = o[5];
                        f.pot[a] = o[6];
                        if constexpr (K::NV > 7) K::finish(f, is[q], a, o);
                    }
                }
            }
        }
    }
    }  // chunks

    if constexpr (CTA) {
        if (cta) {
            const GroupInfo cgi = plan.group(cg);
            if (!loaded) load_group(cgi);
            cta_finish<K, IT, S>(f, smem, is, ac, cgi, cg, cR, crank);
        }
    }
    (void)aborted;
    (void)loaded;
}

// The small-block (CTA-mode) builds of the single-system kernel, one i per
// lane and a j split of `split`; compiled in their own translation unit
// (force_cta.cu) so that the two halves of the kernel set build in parallel.
const void* cta_kernel_ptr(Prec p, int split);

}  // namespace nb
