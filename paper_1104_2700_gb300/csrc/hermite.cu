// O(N) and O(n_act) kernels of the Hermite block-timestep scheme (Sec. 2):
// step 1 (next block time and the active list), steps 2-3 (predictor, which
// also writes the j layout the force kernels stream), steps 5-8 (Hermite
// interpolation, corrector, a0 <- a1, Aarseth timestep in powers of two),
// the first timesteps and the energy diagnostic.
#include <cfloat>
#include <math_constants.h>
#include <cstring>

#include "nb_device.cuh"
#include "nb_launch.h"

namespace nb {

// Order-preserving map of doubles to unsigned 64-bit keys (for atomicMin).
__device__ __forceinline__ unsigned long long dkey(double x)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_decode(unsigned long long k)
{
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double(static_cast<long long>(b));
}

// ---------------------------------------------------------------------------
// Steps 2-3: Taylor predictor (Eqs. xpred, vpred) for every j particle, in
// Horner form with FMA, written straight into the FP64 force kernel's j layout.
// ---------------------------------------------------------------------------
__global__ void predict_fp64_kernel(const StateDev st, const JLayout jl, const double G,
                                    const unsigned long long* t_bits, const double t_host,
                                    const int32_t* n_act_dev, const int32_t* jsrc,
                                    const int32_t* cluster_of)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // j-layout slot
    if (q >= st.n_pad) return;
    const int64_t n = st.n;
    // particle in this slot (-1: a ghost that pads its system to the tile)
    const int64_t i = jsrc ? jsrc[q] : (q < n ? q : -1);
    double xp[3], vp[3], gm;
    if (i >= 0) {
        const double t =
            t_bits ? dkey_decode(t_bits[cluster_of ? cluster_of[i] : 0]) : t_host;
        const double h = t - st.t[i];
        gm = G * st.m[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double x = st.x[c * n + i], v = st.v[c * n + i];
            const double a = st.a[c * n + i], j = st.j[c * n + i];
            xp[c] = fma(h, fma(h, fma(h, j * (1.0 / 6.0), a * 0.5), v), x);
            vp[c] = fma(h, fma(h, j * 0.5, a), v);
        }
    } else {
        xp[0] = xp[1] = xp[2] = GHOST_POS;
        vp[0] = vp[1] = vp[2] = 0.0;
        gm = 0.0;
    }
    // an empty block step writes nothing (checked after the state loads, so
    // they need not wait for this one)
    if (n_act_dev && *n_act_dev == 0) return;
    double2* P = static_cast<double2*>(jl.arr[0]) + 2 * q;
    double2* V = static_cast<double2*>(jl.arr[1]) + 2 * q;
    P[0] = make_double2(xp[0], xp[1]);
    P[1] = make_double2(xp[2], gm);
    V[0] = make_double2(vp[0], vp[1]);
    V[1] = make_double2(vp[2], 0.0);
}

// The sixth-order variant's predictor (reading H1 of its oracle): x, v and
// a carried to time t with a, j, s and the crackle c, in FP64 Horner form,
// into the layout of the snap force kernel.
__global__ void predict_h6_kernel(const StateDev st, const JLayout jl, const double G,
                                  const unsigned long long* t_bits, const double t_host,
                                  const int32_t* n_act_dev)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // j-layout slot
    if (q >= st.n_pad) return;
    const int64_t n = st.n;
    const int64_t i = q < n ? q : -1;
    double xp[3], vp[3], ap[3], gm;
    if (i >= 0) {
        const double t = t_bits ? dkey_decode(t_bits[0]) : t_host;
        const double h = t - st.t[i];
        gm = G * st.m[i];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const double x = st.x[c * n + i], v = st.v[c * n + i], a = st.a[c * n + i];
            const double jj = st.j[c * n + i], sn = st.s[c * n + i], cr = st.c[c * n + i];
            xp[c] = fma(h, fma(h, fma(h, fma(h, fma(h, cr * (1.0 / 120.0), sn * (1.0 / 24.0)),
                                             jj * (1.0 / 6.0)), a * 0.5), v), x);
            vp[c] = fma(h, fma(h, fma(h, fma(h, cr * (1.0 / 24.0), sn * (1.0 / 6.0)), jj * 0.5), a), v);
            ap[c] = fma(h, fma(h, fma(h, cr * (1.0 / 6.0), sn * 0.5), jj), a);
        }
    } else {
        xp[0] = xp[1] = xp[2] = GHOST_POS;
        vp[0] = vp[1] = vp[2] = ap[0] = ap[1] = ap[2] = 0.0;
        gm = 0.0;
    }
    if (n_act_dev && *n_act_dev == 0) return;
    double2* P = static_cast<double2*>(jl.arr[0]) + 2 * q;
    double2* V = static_cast<double2*>(jl.arr[1]) + 2 * q;
    double2* A = static_cast<double2*>(jl.arr[2]) + 2 * q;
    P[0] = make_double2(xp[0], xp[1]);
    P[1] = make_double2(xp[2], gm);
    V[0] = make_double2(vp[0], vp[1]);
    V[1] = make_double2(vp[2], 0.0);
    A[0] = make_double2(ap[0], ap[1]);
    A[1] = make_double2(ap[2], 0.0);
}

// ---------------------------------------------------------------------------
// Steps 2-3 for the precisions whose j layout holds double-single values
// (MIXED, DS, HYBRID): the prediction in double-single arithmetic on the
// FP32 pipes.  GB300 spends ~68 cycles on each FP64 warp instruction, and the
// FP64 Horner form plus the FP64 split into the layout took ~80 of them per
// particle, so over a large system (an ensemble predicts every particle at
// each block step) the predictor was FP64-bound.  Here each FP64 state value
// is cut into hi + lo floats with integer operations on its bits (hi: the
// leading 24 significand bits; lo: the remaining 29 rounded to a float, so
// hi + lo keeps ~48 bits), Eqs. xpred and vpred run as double-single Horner
// steps (FMA-based TwoProd and TwoSum), and the grid-aligned split is taken
// from the double-single result.  The layout agrees with an FP64 prediction
// to its own resolution (~2^-47 of the bound); values far outside the
// layout's range (|x| < 2^-60 or > 2^60, or not finite) take FP64
// conversions instead.
// ---------------------------------------------------------------------------
struct Dsf {
    float hi, lo;
};

__device__ __forceinline__ Dsf dsf_of(double x)
{
    // work on the two 32-bit words (tests on the whole 64-bit pattern would
    // become FP64 compares, which cost as much as the conversion they avoid)
    const unsigned hw = static_cast<unsigned>(__double2hiint(x));
    const unsigned lw = static_cast<unsigned>(__double2loint(x));
    const unsigned e = (hw >> 20) & 0x7ffu;
    if (e - (1023u - 60u) > 120u) {  // zero, |x| < 2^-60 or > 2^60, not finite
        if (((hw & 0x7fffffffu) | lw) == 0u) return {0.f, 0.f};
        const float hi = __double2float_rn(x);
        return {hi, __double2float_rn(x - static_cast<double>(hi))};
    }
    const unsigned sign = hw & 0x80000000u;
    // 52 significand bits: 20 in hw, 32 in lw; hi keeps the leading 23
    const float hi =
        __uint_as_float(sign | ((e - 1023u + 127u) << 23) | ((hw & 0xfffffu) << 3) | (lw >> 29));
    // the remaining 29 significand bits are worth rest * 2^(e - 1075)
    const unsigned rest = lw & 0x1fffffffu;
    const float lo = __uint2float_rn(rest) * __uint_as_float((e - 1075u + 127u) << 23);
    return {hi, sign ? -lo : lo};
}

__device__ __forceinline__ Dsf dsf_add(Dsf a, Dsf b)
{
    float s, e;
    two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    const float h = __fadd_rn(s, e);
    return {h, __fsub_rn(e, __fsub_rn(h, s))};
}

__device__ __forceinline__ Dsf dsf_fma(Dsf a, Dsf b, Dsf c)  // a b + c
{
    float p, e;
    two_prod(a.hi, b.hi, p, e);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    const float h = __fadd_rn(p, e);
    return dsf_add({h, __fsub_rn(e, __fsub_rn(h, p))}, c);
}

__device__ __forceinline__ Dsf dsf_scale(Dsf a, float pow2) { return {a.hi * pow2, a.lo * pow2}; }

// The grid quantum of grid_quantum() as floats, from the bound's bits.
__device__ __forceinline__ void grid_quantum_f(uint32_t bound_bits, float& q, float& inv_q)
{
    const int eb = static_cast<int>((bound_bits >> 23) & 0xff);
    int e;
    if (eb == 0 || eb == 255)
        frexp(2.0 * static_cast<double>(__uint_as_float(bound_bits)), &e);
    else
        e = eb - 125;  // 2B = (1.f / 2) 2^(eb - 125), 1.f / 2 in [0.5, 1)
    q = ldexpf(1.f, e - 23);
    inv_q = ldexpf(1.f, 23 - e);
}

// x rounded to a multiple of q (hi) and the rest (lo); x.hi - hi is exact.
__device__ __forceinline__ void grid_split_ds(Dsf x, float q, float inv_q, float& hi, float& lo)
{
    hi = rintf(x.hi * inv_q) * q;
    lo = __fadd_rn(__fsub_rn(x.hi, hi), x.lo);
}

// Largest and smallest of a value over the 64 threads of a tile (two
// warps): butterfly within each warp, then the two warps through shared
// memory.  Every thread of the block must call it.
struct TileExtent {
    float lo[3], hi[3], gm, g23;
};

__device__ __forceinline__ void tile_extent_reduce(TileExtent& e)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e.lo[c] = fminf(e.lo[c], __shfl_xor_sync(0xffffffffu, e.lo[c], o));
            e.hi[c] = fmaxf(e.hi[c], __shfl_xor_sync(0xffffffffu, e.hi[c], o));
        }
        e.gm = fmaxf(e.gm, __shfl_xor_sync(0xffffffffu, e.gm, o));
        e.g23 = fmaxf(e.g23, __shfl_xor_sync(0xffffffffu, e.g23, o));
    }
    __shared__ TileExtent other;
    if (threadIdx.x == 32) other = e;
    __syncthreads();
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        e.lo[c] = fminf(e.lo[c], other.lo[c]);
        e.hi[c] = fmaxf(e.hi[c], other.hi[c]);
    }
    e.gm = fmaxf(e.gm, other.gm);
    e.g23 = fmaxf(e.g23, other.g23);
}

template <int PREC>
__global__ void predict_ds_kernel(const StateDev st, const JLayout jl, const double G,
                                  const unsigned long long* t_bits, const double t_host,
                                  const int32_t* n_act_dev, const int32_t* jsrc,
                                  const int32_t* cluster_of)
{
    constexpr bool HYB = PREC == static_cast<int>(Prec::HYBRID);
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // j-layout slot
    // (the hybrid layout's tile boxes need every thread of the tile: one
    // block is one tile, and n_pad is a whole number of tiles)
    if (q >= st.n_pad) return;
    const int64_t n = st.n;
    const int64_t i = jsrc ? jsrc[q] : (q < n ? q : -1);
    // an empty block step writes nothing; the ghosts' check is cheap, the
    // particles' comes after their state loads so that they need not wait
    if (i < 0 && !HYB) {  // a ghost: far away, zero mass
        if (n_act_dev && *n_act_dev == 0) return;
        const float g = static_cast<float>(GHOST_POS);
        if (PREC == static_cast<int>(Prec::MIXED)) {
            static_cast<float4*>(jl.arr[0])[q] = make_float4(g, g, g, 0.f);
            static_cast<float4*>(jl.arr[1])[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            static_cast<float2*>(jl.arr[2])[q] = make_float2(0.f, 0.f);
        } else {
            static_cast<float4*>(jl.arr[0])[q] = make_float4(g, g, g, 0.f);
            static_cast<float4*>(jl.arr[1])[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            static_cast<float4*>(jl.arr[2])[q] = make_float4(0.f, 0.f, 0.f, 0.f);
            static_cast<float4*>(jl.arr[3])[q] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        return;
    }
    float hi[3], lo[3];
    Dsf vp[3];
    Dsf gm = {0.f, 0.f};
    if (i >= 0) {
        const double t = t_bits ? dkey_decode(t_bits[cluster_of ? cluster_of[i] : 0]) : t_host;
        const Dsf h = dsf_of(t - st.t[i]);  // exact: both times are dyadic
        gm = dsf_fma(dsf_of(G), dsf_of(st.m[i]), Dsf{0.f, 0.f});
        const Dsf sixth = {0x1.555556p-3f, -0x1.555556p-28f};  // 1/6 to ~2^-50
        float qx, iqx;
        grid_quantum_f(st.bound[0], qx, iqx);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const Dsf x = dsf_of(st.x[c * n + i]), v = dsf_of(st.v[c * n + i]);
            const Dsf a = dsf_of(st.a[c * n + i]), j = dsf_of(st.j[c * n + i]);
            // Eq. xpred: x + h (v + h (a / 2 + h j / 6)); Eq. vpred: v + h (a + h j / 2)
            Dsf u = dsf_fma(j, sixth, Dsf{0.f, 0.f});
            u = dsf_fma(h, u, dsf_scale(a, 0.5f));
            u = dsf_fma(h, u, v);
            grid_split_ds(dsf_fma(h, u, x), qx, iqx, hi[c], lo[c]);
            vp[c] = dsf_fma(h, dsf_fma(h, dsf_scale(j, 0.5f), a), v);
        }
    } else {  // a ghost of the hybrid layout
        hi[0] = hi[1] = hi[2] = static_cast<float>(GHOST_POS);
        lo[0] = lo[1] = lo[2] = 0.f;
        vp[0] = vp[1] = vp[2] = Dsf{0.f, 0.f};
    }
    if (n_act_dev && *n_act_dev == 0) return;  // the same for every thread
    if (PREC == static_cast<int>(Prec::MIXED)) {
        static_cast<float4*>(jl.arr[0])[q] = make_float4(hi[0], hi[1], hi[2], __fadd_rn(gm.hi, gm.lo));
        static_cast<float4*>(jl.arr[1])[q] =
            make_float4(lo[0], lo[1], lo[2], __fadd_rn(vp[0].hi, vp[0].lo));
        static_cast<float2*>(jl.arr[2])[q] =
            make_float2(__fadd_rn(vp[1].hi, vp[1].lo), __fadd_rn(vp[2].hi, vp[2].lo));
    } else {
        float vh[3], vl[3];
        if (HYB) {
            // the FP32 value of v and the rest: far pairs difference FP32
            // velocities, near pairs the whole double-single value
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                vh[c] = __fadd_rn(vp[c].hi, vp[c].lo);
                vl[c] = __fadd_rn(__fsub_rn(vp[c].hi, vh[c]), vp[c].lo);
            }
        } else {
            float qv, iqv;
            grid_quantum_f(st.bound[1], qv, iqv);
#pragma unroll
            for (int c = 0; c < 3; ++c) grid_split_ds(vp[c], qv, iqv, vh[c], vl[c]);
        }
        static_cast<float4*>(jl.arr[0])[q] = make_float4(hi[0], hi[1], hi[2], gm.hi);
        static_cast<float4*>(jl.arr[1])[q] = make_float4(lo[0], lo[1], lo[2], gm.lo);
        // (G m)^(2/3): the hybrid precision's near-pair test
        const float g23 = cbrtf(gm.hi);
        static_cast<float4*>(jl.arr[2])[q] = make_float4(vh[0], vh[1], vh[2], g23 * g23);
        float box = 0.f;
        if (HYB) {
            // the tile's box (hi parts; a ghost adds nothing) and its
            // largest G m and (G m)^(2/3), for the force kernel's test of
            // whether a whole tile is far from an i particle.  It rides in
            // the spare fourth component of the tile's first eight D
            // records (lo_x, lo_y, lo_z, max G m, hi_x, hi_y, hi_z,
            // max (G m)^(2/3)), so it arrives with the tile at no extra copy.
            TileExtent e;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                e.lo[c] = i >= 0 ? hi[c] : CUDART_INF_F;
                e.hi[c] = i >= 0 ? hi[c] : -CUDART_INF_F;
            }
            e.gm = gm.hi;
            e.g23 = g23 * g23;
            tile_extent_reduce(e);
            switch (threadIdx.x) {
            case 0: box = e.lo[0]; break;
            case 1: box = e.lo[1]; break;
            case 2: box = e.lo[2]; break;
            case 3: box = e.gm; break;
            case 4: box = e.hi[0]; break;
            case 5: box = e.hi[1]; break;
            case 6: box = e.hi[2]; break;
            case 7: box = e.g23; break;
            default: break;
            }
        }
        static_cast<float4*>(jl.arr[3])[q] = make_float4(vl[0], vl[1], vl[2], box);
    }
}

// Bounds of the grid-aligned split: max |a_k| and max |b_k| (float bits,
// rounded up so the bound is never below the value).
__global__ void bounds_kernel(const double* __restrict__ a, const double* __restrict__ b,
                              int64_t count, uint32_t* bound)
{
    uint32_t ma = 0, mb = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t ea = __float_as_uint(__double2float_ru(fabs(a[k])));
        const uint32_t eb = __float_as_uint(__double2float_ru(fabs(b[k])));
        ma = ea > ma ? ea : ma;
        mb = eb > mb ? eb : mb;
    }
    ma = __reduce_max_sync(0xffffffffu, ma);
    mb = __reduce_max_sync(0xffffffffu, mb);
    if ((threadIdx.x & 31) == 0) {
        if (ma) atomicMax(&bound[0], ma);
        if (mb) atomicMax(&bound[1], mb);
    }
}

cudaError_t bounds_launch(const double* a, const double* b, int64_t count, uint32_t* bound,
                          cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t want = (count + threads - 1) / threads;
    const unsigned blocks = static_cast<unsigned>(want < 1024 ? want : 1024);
    bounds_kernel<<<blocks, threads, 0, s>>>(a, b, count, bound);
    return cudaGetLastError();
}

__global__ void next_key_kernel(const double* __restrict__ t, const double* __restrict__ dt,
                                int64_t n, unsigned long long* __restrict__ nkey)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        nkey[i] = dkey(t[i] + dt[i]);
}

cudaError_t next_key_launch(const StateDev& st, cudaStream_t s)
{
    if (st.n <= 0) return cudaSuccess;
    const int threads = 64;  // the FP64 adds spread over every SM
    const int64_t want = (st.n + threads - 1) / threads;
    const unsigned blocks = static_cast<unsigned>(want < 4096 ? want : 4096);
    next_key_kernel<<<blocks, threads, 0, s>>>(st.t, st.dt, st.n, st.nkey);
    return cudaGetLastError();
}

cudaError_t predict_launch(const StateDev& st, Prec p, const JLayout& jl, double G,
                           const unsigned long long* t_bits, double t_host,
                           const int32_t* n_act_dev, cudaStream_t s, const ClusterDev* cl)
{
    if (st.n_pad <= 0) return cudaSuccess;
    // Small blocks: the predictor is FP64-pipe bound per SM (GB300's FP64
    // rate is a small fraction of FP32), so it should reach every SM.  One
    // block is one tile of the j layout.
    constexpr int threads = 64;
    static_assert(threads == TJ, "the hybrid predictor reduces each tile in one block");
    const unsigned blocks = static_cast<unsigned>((st.n_pad + threads - 1) / threads);
    const int32_t* jsrc = cl ? cl->jsrc : nullptr;
    const int32_t* cof = cl ? cl->cluster_of : nullptr;
    switch (p) {
    case Prec::FP64:
        predict_fp64_kernel<<<blocks, threads, 0, s>>>(st, jl, G, t_bits, t_host, n_act_dev, jsrc, cof);
        break;
    case Prec::MIXED:
    case Prec::MIXED_SPJ:  // same j layout
        predict_ds_kernel<static_cast<int>(Prec::MIXED)>
            <<<blocks, threads, 0, s>>>(st, jl, G, t_bits, t_host, n_act_dev, jsrc, cof);
        break;
    case Prec::DS:
        predict_ds_kernel<static_cast<int>(Prec::DS)>
            <<<blocks, threads, 0, s>>>(st, jl, G, t_bits, t_host, n_act_dev, jsrc, cof);
        break;
    case Prec::FP64_H6:
        if (cl || !st.s || !st.c) return cudaErrorInvalidValue;
        predict_h6_kernel<<<blocks, threads, 0, s>>>(st, jl, G, t_bits, t_host, n_act_dev);
        break;
    case Prec::HYBRID:
    case Prec::HYBRID_SPJ:  // same j layout
        predict_ds_kernel<static_cast<int>(Prec::HYBRID)>
            <<<blocks, threads, 0, s>>>(st, jl, G, t_bits, t_host, n_act_dev, jsrc, cof);
        break;
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Step 1: next block time t_next = min_i (t_i + dt_i) and the stable
// (ascending-index) compaction of the block {i : t_i + dt_i == t_next}.
// Times are dyadic rationals, so the equality test is exact.
// ---------------------------------------------------------------------------
__global__ void tmin_kernel(const unsigned long long* __restrict__ nkey, int64_t n,
                            unsigned long long* tmin_bits)
{
    unsigned long long best = ~0ull;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = nkey[i];
        best = k < best ? k : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
        best = other < best ? other : best;
    }
    __shared__ unsigned long long wbest[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wbest[wid] = best;
    __syncthreads();
    if (wid == 0) {
        best = lane < (int)(blockDim.x >> 5) ? wbest[lane] : ~0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, best, o);
            best = other < best ? other : best;
        }
        if (lane == 0 && best != ~0ull) atomicMin(tmin_bits, best);
    }
}

// Particle i is in the block when its system's next time t_next (key in
// tkeys, per cluster when cluster_of is given) is within t_end and t_i + dt_i
// equals it.
__device__ __forceinline__ bool is_active(const unsigned long long* nkey, int64_t i,
                                          const unsigned long long* tkeys,
                                          const int32_t* cluster_of, double t_end)
{
    const unsigned long long k = tkeys[cluster_of ? cluster_of[i] : 0];
    return nkey[i] == k && dkey_decode(k) <= t_end;
}

// Block-wide exclusive scan of one int per thread (SCHED_THREADS threads).
__device__ int block_exclusive_scan(int v, int* total)
{
    __shared__ int wsum[SCHED_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = lane < SCHED_THREADS / 32 ? wsum[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < SCHED_THREADS / 32) wsum[lane] = s;
    }
    __syncthreads();
    const int before = wid > 0 ? wsum[wid - 1] : 0;
    *total = wsum[SCHED_THREADS / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(SCHED_THREADS)
    count_kernel(const unsigned long long* __restrict__ nkey, int64_t n,
                 const unsigned long long* tkeys, const int32_t* cluster_of, double t_end,
                 SchedDev sd)
{
    int c = 0;
    const int64_t base = (int64_t)blockIdx.x * SCHED_CHUNK + (int64_t)threadIdx.x * SCHED_PER_THREAD;
#pragma unroll
    for (int e = 0; e < SCHED_PER_THREAD; ++e) {
        const int64_t i = base + e;
        if (i < n && is_active(nkey, i, tkeys, cluster_of, t_end)) ++c;
    }
    int total;
    block_exclusive_scan(c, &total);
    __shared__ bool last;
    if (threadIdx.x == 0) {
        sd.block_counts[blockIdx.x] = total;
        __threadfence();
        last = atomicAdd(sd.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    // The last block scans the per-block counts in block order.
    const int nb = gridDim.x;
    int running = 0;
    for (int b0 = 0; b0 < nb; b0 += SCHED_THREADS) {
        const int b = b0 + threadIdx.x;
        const int v = b < nb ? __ldcg(sd.block_counts + b) : 0;
        int tot;
        const int ex = block_exclusive_scan(v, &tot);
        if (b < nb) sd.block_offsets[b] = running + ex;
        running += tot;
    }
    if (threadIdx.x == 0) {
        *sd.n_act = running;
        *sd.ticket = 0u;
    }
}

__global__ void __launch_bounds__(SCHED_THREADS)
    scatter_kernel(const unsigned long long* __restrict__ nkey, int64_t n,
                   const unsigned long long* tkeys, const int32_t* cluster_of, double t_end,
                   SchedDev sd)
{
    const int64_t base = (int64_t)blockIdx.x * SCHED_CHUNK + (int64_t)threadIdx.x * SCHED_PER_THREAD;
    unsigned flags = 0;
    int c = 0;
#pragma unroll
    for (int e = 0; e < SCHED_PER_THREAD; ++e) {
        const int64_t i = base + e;
        if (i < n && is_active(nkey, i, tkeys, cluster_of, t_end)) {
            flags |= 1u << e;
            ++c;
        }
    }
    int total;
    int pos = block_exclusive_scan(c, &total) + sd.block_offsets[blockIdx.x];
#pragma unroll
    for (int e = 0; e < SCHED_PER_THREAD; ++e)
        if (flags & (1u << e)) sd.idx[pos++] = static_cast<int32_t>(base + e);
}

// Step 1 in one CTA, for systems small enough that a single SM beats three
// launches.  Thread k owns particles k + SEL1_THREADS u (u < 32, coalesced).
// One pass over the next-time keys gives each thread its smallest key and a
// bitmask of the u that reach it; after the block minimum, a thread's block
// members are that mask if its minimum is the block's.  The ordered
// compaction then takes one warp ballot per u and a single block-wide scan
// of the per-(u, warp) counts, which keeps the list in ascending index order.
constexpr int SEL1_THREADS = 1024;
constexpr int64_t SEL1_MAX_N = 32 * SEL1_THREADS;

__global__ void __launch_bounds__(SEL1_THREADS)
    select_one_cta_kernel(const unsigned long long* __restrict__ nkey, int64_t n, double t_end,
                          SchedDev sd)
{
    __shared__ unsigned long long wmin[SEL1_THREADS / 32];
    __shared__ unsigned long long tkey;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    unsigned long long best = ~0ull;
    uint32_t mask = 0u;
    const int tiles = static_cast<int>((n + SEL1_THREADS - 1) / SEL1_THREADS);  // <= 32
    // keys in batches of 16 independent loads (one memory round trip each);
    // slots past n read as the largest key and never join the mask
    for (int u0 = 0; u0 < tiles; u0 += 16) {
        unsigned long long kk[16];
#pragma unroll
        for (int v = 0; v < 16; ++v) {
            const int64_t i = tid + static_cast<int64_t>(SEL1_THREADS) * (u0 + v);
            kk[v] = (u0 + v < tiles && i < n) ? __ldcg(nkey + i) : ~0ull;
        }
#pragma unroll
        for (int v = 0; v < 16; ++v) {
            const unsigned long long k = kk[v];
            if (k < best) {
                best = k;
                mask = 1u << (u0 + v);
            } else if (k == best && k != ~0ull) {
                mask |= 1u << (u0 + v);
            }
        }
    }
    unsigned long long bmin = best;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long other = __shfl_xor_sync(0xffffffffu, bmin, o);
        bmin = other < bmin ? other : bmin;
    }
    if (lane == 0) wmin[wid] = bmin;
    __syncthreads();
    if (wid == 0) {
        bmin = wmin[lane];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long other = __shfl_xor_sync(0xffffffffu, bmin, o);
            bmin = other < bmin ? other : bmin;
        }
        if (lane == 0) {
            tkey = bmin;
            *sd.tmin_bits = bmin;
        }
    }
    __syncthreads();
    if (best != tkey || !(dkey_decode(tkey) <= t_end)) mask = 0u;
    // Ordered compaction: slot of (tile u, warp w, lane) = members before
    // tile u + members of tile u in warps before w + lanes before it.  One
    // ballot per tile (lane u of each warp keeps its warp's ballot of tile
    // u), the warp counts in [u][w] order, one block-wide exclusive scan.
    __shared__ int cnt[32 * (SEL1_THREADS / 32)];
    __shared__ int wtot[SEL1_THREADS / 32];
    uint32_t bal = 0u;
    for (int u = 0; u < tiles; ++u) {
        const uint32_t b = __ballot_sync(0xffffffffu, (mask >> u) & 1u);
        if (lane == u) bal = b;
        if (lane == 0) cnt[u * 32 + wid] = __popc(b);
    }
    __syncthreads();
    const int mine = tid < tiles * 32 ? cnt[tid] : 0;  // entry tid = (u = wid, w = lane)
    int x = mine;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wtot[wid] = x;
    __syncthreads();
    if (wid == 0) {
        const int c = wtot[lane];
        int y = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        wtot[lane] = y - c;  // exclusive
        if (lane == 31) *sd.n_act = y;
    }
    __syncthreads();
    if (tid < tiles * 32) cnt[tid] = wtot[wid] + x - mine;
    __syncthreads();
    for (int u = 0; u < tiles; ++u) {
        const uint32_t b = __shfl_sync(0xffffffffu, bal, u);
        if ((mask >> u) & 1u)
            sd.idx[cnt[u * 32 + wid] + __popc(b & ((1u << lane) - 1u))] =
                static_cast<int32_t>(tid + SEL1_THREADS * u);
    }
}

cudaError_t select_launch(const StateDev& st, const SchedDev& sd, double t_end, cudaStream_t s)
{
    if (st.n > 0 && st.n <= SEL1_MAX_N) {
        select_one_cta_kernel<<<1, SEL1_THREADS, 0, s>>>(st.nkey, st.n, t_end, sd);
        return cudaGetLastError();
    }
    cudaError_t e = cudaMemsetAsync(sd.tmin_bits, 0xff, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (st.n <= 0) return cudaMemsetAsync(sd.n_act, 0, sizeof(int32_t), s);
    const int64_t nb64 = (st.n + SCHED_CHUNK - 1) / SCHED_CHUNK;
    if (nb64 > sd.max_blocks) return cudaErrorInvalidValue;
    const int nb = static_cast<int>(nb64);
    int tb = nb < 1024 ? nb : 1024;
    tmin_kernel<<<tb, 256, 0, s>>>(st.nkey, st.n, sd.tmin_bits);
    count_kernel<<<nb, SCHED_THREADS, 0, s>>>(st.nkey, st.n, sd.tmin_bits, nullptr, t_end, sd);
    scatter_kernel<<<nb, SCHED_THREADS, 0, s>>>(st.nkey, st.n, sd.tmin_bits, nullptr, t_end, sd);
    return cudaGetLastError();
}

// Ensemble step 1: block c finds the next time of cluster c and how many of
// its particles reach it (0 when that time lies past t_end): a reduction of
// (smallest key, count of that key) pairs.
__device__ __forceinline__ void min_count_merge(unsigned long long& best, int& n,
                                                unsigned long long ob, int on)
{
    if (ob < best) {
        best = ob;
        n = on;
    } else if (ob == best) {
        n += on;
    }
}

__global__ void cluster_tmin_kernel(const unsigned long long* __restrict__ nkey,
                                    const int64_t* off, unsigned long long* tkey, int32_t* cnt,
                                    double t_end)
{
    const int c = blockIdx.x;
    unsigned long long best = ~0ull;
    int n = 0;
    for (int64_t i = off[c] + threadIdx.x; i < off[c + 1]; i += blockDim.x)
        min_count_merge(best, n, nkey[i], 1);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int on = __shfl_xor_sync(0xffffffffu, n, o);
        min_count_merge(best, n, ob, on);
    }
    __shared__ unsigned long long wbest[32];
    __shared__ int wn[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) wbest[wid] = best, wn[wid] = n;
    __syncthreads();
    if (wid == 0) {
        const bool have = lane < (int)(blockDim.x >> 5);
        best = have ? wbest[lane] : ~0ull;
        n = have ? wn[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int on = __shfl_xor_sync(0xffffffffu, n, o);
            min_count_merge(best, n, ob, on);
        }
        if (lane == 0) {
            tkey[c] = best;
            cnt[c] = (best != ~0ull && dkey_decode(best) <= t_end) ? n : 0;
        }
    }
}

cudaError_t cluster_select_launch(const StateDev& st, const ClusterDev& cl, const SchedDev& sd,
                                  double t_end, cudaStream_t s)
{
    if (st.n <= 0 || cl.k <= 0) return cudaMemsetAsync(sd.n_act, 0, sizeof(int32_t), s);
    const int64_t nb64 = (st.n + SCHED_CHUNK - 1) / SCHED_CHUNK;
    if (nb64 > sd.max_blocks) return cudaErrorInvalidValue;
    const int nb = static_cast<int>(nb64);
    cluster_tmin_kernel<<<cl.k, 256, 0, s>>>(st.nkey, cl.off, cl.tkey, cl.cnt, t_end);
    count_kernel<<<nb, SCHED_THREADS, 0, s>>>(st.nkey, st.n, cl.tkey, cl.cluster_of, t_end, sd);
    scatter_kernel<<<nb, SCHED_THREADS, 0, s>>>(st.nkey, st.n, cl.tkey, cl.cluster_of, t_end, sd);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Ensemble force plan: the active list (ascending, so each cluster's block
// is contiguous) cut into i-groups of at most gi entries that never mix
// clusters, each with its cluster's j tiles, laid end to end.  One CTA.
// ---------------------------------------------------------------------------
constexpr int PLAN_THREADS = 1024;

__device__ int64_t lower_bound_i32(const int32_t* a, int64_t n, int64_t x)
{
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < x) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Block-wide exclusive scan of one int64 per thread (PLAN_THREADS threads).
__device__ int64_t plan_scan(int64_t v, int64_t* total)
{
    __shared__ int64_t ws[PLAN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) ws[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int64_t z = lane < PLAN_THREADS / 32 ? ws[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < PLAN_THREADS / 32) ws[lane] = z;
    }
    __syncthreads();
    const int64_t before = wid > 0 ? ws[wid - 1] : 0;
    *total = ws[PLAN_THREADS / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(PLAN_THREADS)
    plan_kernel(const ClusterDev cl, const int32_t* idx, const int32_t* n_act_dev, int gi,
                const int32_t* cnt)
{
    const int64_t n_act = *n_act_dev;
    const int K = cl.k;
    const int per = (K + PLAN_THREADS - 1) / PLAN_THREADS;
    const int c0 = threadIdx.x * per;
    const int c1 = c0 + per < K ? c0 + per : K;
    // cluster c's share [b, e) of the ascending active list: from the
    // select's counts (a scan), or by binary search in idx
    int64_t csum = 0;
    if (cnt)
        for (int c = c0; c < c1; ++c) csum += cnt[c];
    int64_t ctot;
    const int64_t cbase = plan_scan(csum, &ctot);
    auto share = [&](int c, int64_t& run, int64_t& b, int64_t& e) {
        if (cnt) {
            b = run;
            e = run + cnt[c];
            run = e;
        } else {
            b = lower_bound_i32(idx, n_act, cl.off[c]);
            e = lower_bound_i32(idx, n_act, cl.off[c + 1]);
        }
    };
    int64_t gsum = 0, tsum = 0, run = cbase;
    for (int c = c0; c < c1; ++c) {
        int64_t b, e;
        share(c, run, b, e);
        const int64_t gc = (e - b + gi - 1) / gi;
        gsum += gc;
        tsum += gc * ((cl.joff[c + 1] - cl.joff[c]) / TJ);
    }
    int64_t G, T;
    int64_t gbase = plan_scan(gsum, &G);
    int64_t tbase = plan_scan(tsum, &T);
    if (G > cl.max_groups) {  // cannot happen for a sorted active list
        if (threadIdx.x == 0) cl.plan_scalars[0] = cl.plan_scalars[1] = 0;
        return;
    }
    run = cbase;
    for (int c = c0; c < c1; ++c) {
        int64_t b, e;
        share(c, run, b, e);
        const int64_t nt = (cl.joff[c + 1] - cl.joff[c]) / TJ;
        for (int64_t a = b; a < e; a += gi) {
            cl.grp_cluster[gbase] = c;
            cl.grp_act_begin[gbase] = static_cast<int32_t>(a);
            cl.grp_act_count[gbase] = static_cast<int32_t>(e - a < gi ? e - a : gi);
            cl.grp_tile0[gbase] = tbase;
            ++gbase;
            tbase += nt;
        }
    }
    if (threadIdx.x == 0) {
        cl.grp_tile0[G] = T;
        cl.plan_scalars[0] = G;
        cl.plan_scalars[1] = T;
    }
}

cudaError_t plan_launch(const ClusterDev& cl, const int32_t* idx, const int32_t* n_act_dev,
                        int gi, cudaStream_t s, bool from_counts)
{
    plan_kernel<<<1, PLAN_THREADS, 0, s>>>(cl, idx, n_act_dev, gi, from_counts ? cl.cnt : nullptr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Steps 5-8 for each active particle.  The arithmetic is written operation
// by operation with non-contracted intrinsics in the order of the
// equations, so that identical inputs give the oracle's bits.
// ---------------------------------------------------------------------------
#define DADD __dadd_rn
#define DSUB __dsub_rn
#define DMUL __dmul_rn
#define DDIV __ddiv_rn

// Correctly rounded a / b for a constant b with y = RN(1/b): q0 = RN(a y)
// is within an ulp, the FMA residual r = a - b q0 is exact, and one
// correction RN(q0 + r y) gives RN(a / b) (Markstein's FMA division; an
// exhaustive random test of b = 6, 24, 120 finds no mismatch).  Three FP64
// operations instead of a general division, the same bits.
__device__ __forceinline__ double div_const(double a, double b, double y)
{
    const double q0 = __dmul_rn(a, y);
    const double r = __fma_rn(-q0, b, a);
    return __fma_rn(r, y, q0);
}

// 1 / p for p a normal power of two: exact, by its exponent alone.
__device__ __forceinline__ double recip_pow2(double p)
{
    const long long e = __double_as_longlong(p) >> 52;  // biased exponent (p > 0)
    return __longlong_as_double((2046LL - e) << 52);
}

__device__ __forceinline__ double norm3_rn(double x, double y, double z)
{
    return __dsqrt_rn(DADD(DADD(DMUL(x, x), DMUL(y, y)), DMUL(z, z)));
}

// Eq. timestep for the power-of-two rule only.  The rule compares the
// candidate with powers of two alone, so all it needs is the k with
// 2^k <= eta sqrt((|a||s| + |j|^2) / (|j||c| + |s|^2)) < 2^(k+1).  That is
// taken in FP32: each norm after scaling its vector by a power of two
// (|v| = nrm 2^E, the vector's largest component then in [0.5, 1)), the two
// sums after aligning their terms' exponents.  The truncated inputs and about
// fifteen FP32 roundings leave it within ~2e-6 of the FP64 value, so k is certain unless the value
// lies within 1e-5 of a power of two; then, or when a vector is zero, tiny or
// not finite, the function declines and the caller evaluates the formula in
// FP64 as written.  Either way the timestep chosen is the oracle's.
// A double truncated to a float from its two 32-bit words (within an ulp; a
// hardware conversion costs as much as an FP64 operation on GB300); values
// outside [2^-100, 2^100] become 0 or NaN, which the caller's range test
// rejects.
__device__ __forceinline__ float trunc_to_float(double x)
{
    const unsigned hw = static_cast<unsigned>(__double2hiint(x));
    const unsigned lw = static_cast<unsigned>(__double2loint(x));
    const unsigned e = (hw >> 20) & 0x7ffu;
    if (((hw & 0x7fffffffu) | lw) == 0u) return 0.f;
    if (e - (1023u - 100u) > 200u) return __int_as_float(0x7fc00000);  // NaN
    return __uint_as_float((hw & 0x80000000u) | ((e - 1023u + 127u) << 23) |
                           ((hw & 0xfffffu) << 3) | (lw >> 29));
}

__device__ __forceinline__ bool norm3_scaled(const double (&v)[3], float& nrm, int& E)
{
    const float f0 = trunc_to_float(v[0]);
    const float f1 = trunc_to_float(v[1]);
    const float f2 = trunc_to_float(v[2]);
    const float mx = fmaxf(fabsf(f0), fmaxf(fabsf(f1), fabsf(f2)));
    if (!(mx >= 1e-30f && mx <= 1e30f)) return false;  // NaN fails too
    frexpf(mx, &E);
    const float x0 = ldexpf(f0, -E), x1 = ldexpf(f1, -E), x2 = ldexpf(f2, -E);
    nrm = sqrtf(fmaf(x0, x0, fmaf(x1, x1, x2 * x2)));
    return true;
}

__device__ __forceinline__ bool aarseth_interval(const double (&a)[3], const double (&j)[3],
                                                 const double (&s)[3], const double (&c)[3],
                                                 double eta, int& k)
{
    float nA, nJ, nS, nC;
    int eA, eJ, eS, eC;
    if (!norm3_scaled(a, nA, eA) || !norm3_scaled(j, nJ, eJ) || !norm3_scaled(s, nS, eS) ||
        !norm3_scaled(c, nC, eC))
        return false;
    // numerator 2^en (..) and denominator 2^ed (..), each a sum of two
    // positive terms
    const int n1 = eA + eS, n2 = 2 * eJ, d1 = eJ + eC, d2 = 2 * eS;
    const int en = n1 > n2 ? n1 : n2, ed = d1 > d2 ? d1 : d2;
    const float num = ldexpf(nA * nS, n1 - en) + ldexpf(nJ * nJ, n2 - en);
    const float den = ldexpf(nJ * nC, d1 - ed) + ldexpf(nS * nS, d2 - ed);
    int ex = en - ed;
    float r = num / den;
    if (ex & 1) r *= 2.f, ex -= 1;  // an even exponent halves exactly
    int e;
    const float m = frexpf(static_cast<float>(eta) * sqrtf(r), &e);  // m in [0.5, 1)
    if (!(m > 0.500005f && m < 0.99999f)) return false;
    k = e - 1 + ex / 2;
    return k > -1000 && k < 1000;
}

// Step 8 for one particle: Eq. timestep at the new time (a1, j1, the snap
// carried to t_next, the crackle), then the power-of-two rule of the
// hierarchical scheme.  Returns false (and flags the status) when the
// formula is not a number.
__device__ __forceinline__ bool next_timestep(const double (&a1)[3], const double (&j1)[3],
                                              const double (&sn)[3], const double (&c0)[3],
                                              double h, double tn, const CorrectArgs& c,
                                              double& dt_new)
{
    // cand: min(dt_Aarseth, dt_max), or a power of two in the same
    // power-of-two interval, which is all the rule below looks at
    double cand;
    int kq;
    const int kmax = static_cast<int>((__double_as_longlong(c.dt_max) >> 52) & 0x7ff) - 1023;
    if (aarseth_interval(a1, j1, sn, c0, c.eta, kq)) {
        cand = kq >= kmax ? c.dt_max : __longlong_as_double(static_cast<long long>(kq + 1023) << 52);
    } else {
        const double A = norm3_rn(a1[0], a1[1], a1[2]);
        const double J = norm3_rn(j1[0], j1[1], j1[2]);
        const double S = norm3_rn(sn[0], sn[1], sn[2]);
        const double C = norm3_rn(c0[0], c0[1], c0[2]);
        // a zero denominator (a particle that feels nothing) sets no constraint
        const double den = DADD(DMUL(J, C), DMUL(S, S));
        const double dta =
            den == 0.0 ? CUDART_INF : DMUL(c.eta, __dsqrt_rn(DDIV(DADD(DMUL(A, S), DMUL(J, J)), den)));
        if (isnan(dta)) {
            atomicOr(c.status, ST_NONFINITE);
            return false;
        }
        cand = dta < c.dt_max ? dta : c.dt_max;
    }
    dt_new = h;
    // t_next a multiple of 2h (h a power of two, so t_next / 2h is exact)
    const double k2h = DMUL(tn, recip_pow2(DMUL(2.0, h)));
    if (cand >= DMUL(2.0, h) && k2h == rint(k2h)) {
        dt_new = DMUL(2.0, h);
    } else if (cand >= h) {
        dt_new = h;
    } else {
        while (dt_new > cand && dt_new >= c.dt_min) dt_new = DMUL(dt_new, 0.5);
    }
    return true;
}

__device__ __forceinline__ double pow2_floor(double x)
{
    int e;
    frexp(x, &e);
    return ldexp(1.0, e - 1);
}

// GB300's FP64 unit spends ~68 cycles on each warp instruction whatever
// its number of active lanes, and a warp has one in flight, so a block's
// latency is the FP64 instruction count of its busiest warp.  A block of
// three warps therefore takes 32 active particles: warp d does component d
// of the prediction, snap, crackle and corrector (the bulk of the FP64
// work), and warp 0 then takes each particle's timestep from the three
// components left in shared memory.
constexpr int CORR_P = 32;  // particles per block, one per lane

__global__ void __launch_bounds__(3 * CORR_P) correct_kernel(const StateDev st, const CorrectArgs c)
{
    __shared__ double sv[4][3][CORR_P];  // a1, j1, snap at t_next, crackle
    __shared__ int fin[3][CORR_P];
    const int d = threadIdx.x / CORR_P, lane = threadIdx.x % CORR_P;
    const int n_act = *c.n_act_dev;
    const int64_t n = st.n;
    if (blockIdx.x == 0 && threadIdx.x == 0 && n_act > 0) {
        if (c.step_counter) atomicAdd(c.step_counter, 1ull);
        // interactions: n_act * n for one system (an ensemble adds, per
        // active particle, its own system's size below)
        if (c.inter_counter && !c.cluster_of)
            atomicAdd(c.inter_counter, static_cast<unsigned long long>(n_act) *
                                           static_cast<unsigned long long>(n));
    }
    for (int64_t g = (int64_t)blockIdx.x * CORR_P; g < n_act; g += (int64_t)gridDim.x * CORR_P) {
        const int64_t k = g + lane;
        const bool act = k < n_act;
        const int64_t i = act ? c.idx[k] : -1;
        const bool inr = act && i >= 0 && i < n;
        if (d == 0) {
            if (act && !inr) atomicOr(c.status, ST_BADINDEX);
            if (c.inter_counter && c.cluster_of) {
                unsigned long long mine = 0;
                if (inr) {
                    const int cc = c.cluster_of[i];
                    mine = static_cast<unsigned long long>(c.cl_off[cc + 1] - c.cl_off[cc]);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) mine += __shfl_xor_sync(0xffffffffu, mine, o);
                if (lane == 0 && mine) atomicAdd(c.inter_counter, mine);
            }
        }
        double tn = 0.0, h = 0.0, t0 = 0.0, a1 = 0.0, j1 = 0.0;
        if (inr) {
            tn = dkey_decode(c.t_bits[c.cluster_of ? c.cluster_of[i] : 0]);
            h = st.dt[i];
            t0 = st.t[i];
            a1 = c.acc1[3 * k + d];
            j1 = c.jerk1[3 * k + d];
        }
        fin[d][lane] = isfinite(a1) && isfinite(j1);
        __syncthreads();
        const bool finite = fin[0][lane] && fin[1][lane] && fin[2][lane];
        const bool due = inr && DADD(t0, h) == tn;
        if (d == 0 && inr) {
            if (!due) atomicOr(c.status, ST_NOTDUE);
            else if (!finite) atomicOr(c.status, ST_NONFINITE);
        }
        const bool work = due && finite;
        if (work) {
            const double dtp = DSUB(tn, t0);
            const double p2 = DMUL(dtp, dtp), p3 = DMUL(p2, dtp);
            const double h2 = DMUL(h, h), h3 = DMUL(h2, h), h4 = DMUL(h3, h), h5 = DMUL(h4, h);
            // h is a power of two, so dividing by h^2 or h^3 (and by 2) is an
            // exact scaling: multiplying by the exact reciprocal gives the
            // quotient's bits.
            const double ih2 = recip_pow2(h2), ih3 = recip_pow2(h3);  // exact
            const int64_t q = d * n + i;
            const double x0 = st.x[q], v0 = st.v[q], a0 = st.a[q], j0 = st.j[q];
            // Eqs. xpred, vpred for the i particle (step 2).
            const double rp = DADD(DADD(DADD(x0, DMUL(v0, dtp)), DMUL(DMUL(a0, 0.5), p2)),
                                   DMUL(div_const(j0, 6.0, 1.0 / 6.0), p3));
            const double vp = DADD(DADD(v0, DMUL(a0, dtp)), DMUL(DMUL(j0, 0.5), p2));
            // Step 5: snap and crackle from the Hermite interpolation.
            const double da = DSUB(a0, a1);
            const double s0 = DMUL(DMUL(2.0, DSUB(DMUL(-3.0, da), DMUL(DADD(DMUL(2.0, j0), j1), h))), ih2);
            const double c0 = DMUL(DMUL(6.0, DADD(DMUL(2.0, da), DMUL(DADD(j0, j1), h))), ih3);
            // Step 6: corrector.
            const double r1 = DADD(DADD(rp, div_const(DMUL(s0, h4), 24.0, 1.0 / 24.0)),
                                   div_const(DMUL(c0, h5), 120.0, 1.0 / 120.0));
            const double v1 = DADD(DADD(vp, div_const(DMUL(s0, h3), 6.0, 1.0 / 6.0)),
                                   div_const(DMUL(c0, h4), 24.0, 1.0 / 24.0));
            // Step 7: a0 <- a1, j0 <- j1.
            st.x[q] = r1;
            st.v[q] = v1;
            st.a[q] = a1;
            st.j[q] = j1;
            // raise the layout bounds if this particle moved past them (rare)
            const uint32_t xb = __float_as_uint(__double2float_ru(fabs(r1)));
            const uint32_t vb = __float_as_uint(__double2float_ru(fabs(v1)));
            if (xb > st.bound[0]) atomicMax(&st.bound[0], xb);
            if (vb > st.bound[1]) atomicMax(&st.bound[1], vb);
            sv[0][d][lane] = a1;
            sv[1][d][lane] = j1;
            sv[2][d][lane] = DADD(s0, DMUL(c0, h));  // snap carried to t_next
            sv[3][d][lane] = c0;
        }
        __syncthreads();
        if (d == 0 && work) {
            st.t[i] = tn;
            double a3[3], j3[3], s3[3], c3[3];
#pragma unroll
            for (int e = 0; e < 3; ++e)
                a3[e] = sv[0][e][lane], j3[e] = sv[1][e][lane], s3[e] = sv[2][e][lane],
                c3[e] = sv[3][e][lane];
            double dt_new;
            if (next_timestep(a3, j3, s3, c3, h, tn, c, dt_new)) {
                st.dt[i] = dt_new;
                st.nkey[i] = dkey(DADD(tn, dt_new));
                if (dt_new < c.dt_min) atomicOr(c.status, ST_DTMIN);
            }
        }
        // fin and sv are written again only after the next iteration's
        // first barrier has seen warp 0 through its reads
    }
}

cudaError_t correct_launch(const StateDev& st, const CorrectArgs& c, cudaStream_t s)
{
    if (st.n <= 0) return cudaSuccess;
    // enough blocks for every particle to be active; each loops over groups
    const int64_t want = (st.n + CORR_P - 1) / CORR_P;
    const unsigned blocks = static_cast<unsigned>(want < 2432 ? want : 2432);
    correct_kernel<<<blocks, 3 * CORR_P, 0, s>>>(st, c);
    return cudaGetLastError();
}

// The sixth-order variant's steps 5-8 for one active particle per thread,
// written operation by operation in the order of its oracle (the quintic
// Hermite interpolant of a(t); readings H1-H2), so that identical inputs
// give the oracle's r, v, a, j, s and crackle.  The timestep uses the FP64
// pow of the criterion, whose last bit may differ from the host's: the
// power-of-two rule only looks at the candidate's interval.
__global__ void correct6_kernel(const StateDev st, const CorrectArgs c, const double* snap1)
{
    const int n_act = *c.n_act_dev;
    const int64_t n = st.n;
    if (blockIdx.x == 0 && threadIdx.x == 0 && n_act > 0) {
        if (c.step_counter) atomicAdd(c.step_counter, 1ull);
        if (c.inter_counter)
            atomicAdd(c.inter_counter, static_cast<unsigned long long>(n_act) *
                                           static_cast<unsigned long long>(n));
    }
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n_act;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = c.idx[k];
        if (i < 0 || i >= n) {
            atomicOr(c.status, ST_BADINDEX);
            continue;
        }
        const double tn = dkey_decode(c.t_bits[0]);
        const double h = st.dt[i];
        if (DADD(st.t[i], h) != tn) {
            atomicOr(c.status, ST_NOTDUE);
            continue;
        }
        double a1[3], j1[3], s1[3];
        bool finite = true;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            a1[d] = c.acc1[3 * k + d];
            j1[d] = c.jerk1[3 * k + d];
            s1[d] = snap1[3 * k + d];
            finite = finite && isfinite(a1[d]) && isfinite(j1[d]) && isfinite(s1[d]);
        }
        if (!finite) {
            atomicOr(c.status, ST_NONFINITE);
            continue;
        }
        const double h2 = DMUL(h, h), h3 = DMUL(h2, h), h4 = DMUL(h3, h), h5 = DMUL(h4, h);
        double c1[3], d1[3], x1[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const int64_t q = d * n + i;
            const double r0 = st.x[q], v0 = st.v[q], a0 = st.a[q], j0 = st.j[q], s0 = st.s[q];
            const double Da = DSUB(DSUB(DSUB(a1[d], a0), DMUL(j0, h)), DMUL(DDIV(s0, 2.0), h2));
            const double Dj = DSUB(DSUB(j1[d], j0), DMUL(s0, h));
            const double Ds = DSUB(s1[d], s0);
            const double c3 = DDIV(DMUL(3.0, DADD(DSUB(DMUL(20.0, Da), DMUL(DMUL(8.0, Dj), h)),
                                                  DMUL(Ds, h2))), h3);
            const double c4 = DDIV(DMUL(-24.0, DADD(DSUB(DMUL(15.0, Da), DMUL(DMUL(7.0, Dj), h)),
                                                    DMUL(Ds, h2))), h4);
            const double c5 = DDIV(DMUL(60.0, DADD(DSUB(DMUL(12.0, Da), DMUL(DMUL(6.0, Dj), h)),
                                                   DMUL(Ds, h2))), h5);
            const double v1 = DADD(DSUB(DADD(v0, DMUL(DDIV(h, 2.0), DADD(a0, a1[d]))),
                                        DMUL(DDIV(h2, 10.0), DSUB(j1[d], j0))),
                                   DMUL(DDIV(h3, 120.0), DADD(s0, s1[d])));
            const double r1 = DADD(DSUB(DADD(r0, DMUL(DDIV(h, 2.0), DADD(v0, v1))),
                                        DMUL(DDIV(h2, 10.0), DSUB(a1[d], a0))),
                                   DMUL(DDIV(h3, 120.0), DADD(j0, j1[d])));
            c1[d] = DADD(DADD(c3, DMUL(c4, h)), DMUL(DDIV(c5, 2.0), h2));
            d1[d] = DADD(c4, DMUL(c5, h));
            x1[d] = c5;
            st.x[q] = r1;
            st.v[q] = v1;
            st.a[q] = a1[d];
            st.j[q] = j1[d];
            st.s[q] = s1[d];
            st.c[q] = c1[d];
            const uint32_t xb = __float_as_uint(__double2float_ru(fabs(r1)));
            const uint32_t vb = __float_as_uint(__double2float_ru(fabs(v1)));
            if (xb > st.bound[0]) atomicMax(&st.bound[0], xb);
            if (vb > st.bound[1]) atomicMax(&st.bound[1], vb);
        }
        st.t[i] = tn;
        // reading H2: the sixth-order criterion at the new time, then R2
        const double A = norm3_rn(a1[0], a1[1], a1[2]), J = norm3_rn(j1[0], j1[1], j1[2]);
        const double S = norm3_rn(s1[0], s1[1], s1[2]), C = norm3_rn(c1[0], c1[1], c1[2]);
        const double D = norm3_rn(d1[0], d1[1], d1[2]), X = norm3_rn(x1[0], x1[1], x1[2]);
        const double den = DADD(DMUL(C, X), DMUL(D, D));
        const double dta = den == 0.0
                               ? CUDART_INF
                               : DMUL(c.eta, pow(DDIV(DADD(DMUL(A, S), DMUL(J, J)), den), 1.0 / 6.0));
        if (isnan(dta)) {
            atomicOr(c.status, ST_NONFINITE);
            continue;
        }
        const double cand = dta < c.dt_max ? dta : c.dt_max;
        double dt_new = h;
        const double k2h = DMUL(tn, recip_pow2(DMUL(2.0, h)));
        if (cand >= DMUL(2.0, h) && k2h == rint(k2h)) {
            dt_new = DMUL(2.0, h);
        } else if (cand >= h) {
            dt_new = h;
        } else {
            while (dt_new > cand && dt_new >= c.dt_min) dt_new = DMUL(dt_new, 0.5);
        }
        st.dt[i] = dt_new;
        st.nkey[i] = dkey(DADD(tn, dt_new));
        if (dt_new < c.dt_min) atomicOr(c.status, ST_DTMIN);
    }
}

cudaError_t correct6_launch(const StateDev& st, const CorrectArgs& c, const double* snap1,
                            cudaStream_t s)
{
    if (st.n <= 0) return cudaSuccess;
    if (!st.s || !st.c || !snap1 || c.cluster_of) return cudaErrorInvalidValue;
    const int threads = 64;  // FP64 bound: spread the particles over many SMs
    const int64_t want = (st.n + threads - 1) / threads;
    correct6_kernel<<<static_cast<unsigned>(want < 4096 ? want : 4096), threads, 0, s>>>(st, c,
                                                                                          snap1);
    return cudaGetLastError();
}

__global__ void init_snap_kernel(const StateDev st, const double* snap_rows)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 3 * st.n) return;
    const int64_t d = e / st.n, i = e - d * st.n;
    st.s[e] = snap_rows[3 * i + d];
    st.c[e] = 0.0;  // reading H1: no crackle yet
}

cudaError_t init_snap_launch(const StateDev& st, const double* snap_rows, cudaStream_t s)
{
    if (st.n <= 0) return cudaSuccess;
    init_snap_kernel<<<static_cast<unsigned>((3 * st.n + 255) / 256), 256, 0, s>>>(st, snap_rows);
    return cudaGetLastError();
}

// Reading R3 of the oracle: dt = pow2_floor(min(eta_start |a| / |j|, dt_max)).
__global__ void init_dt_kernel(const StateDev st, const double* acc, const double* jerk,
                               double eta_start, double dt_max, double dt_min, double t0,
                               uint32_t* status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= st.n) return;
    const double A = norm3_rn(acc[3 * i], acc[3 * i + 1], acc[3 * i + 2]);
    const double J = norm3_rn(jerk[3 * i], jerk[3 * i + 1], jerk[3 * i + 2]);
    double raw = J == 0.0 ? CUDART_INF : DDIV(DMUL(eta_start, A), J);
    st.t[i] = t0;
    if (isnan(raw)) {
        atomicOr(status, ST_NONFINITE);
        st.dt[i] = dt_max;
        st.nkey[i] = dkey(t0 + dt_max);
        return;
    }
    if (raw > dt_max) raw = dt_max;
    if (raw <= 0.0) {
        atomicOr(status, ST_DTMIN);
        st.dt[i] = dt_max;
        st.nkey[i] = dkey(t0 + dt_max);
        return;
    }
    const double dt = pow2_floor(raw);
    st.dt[i] = dt;
    st.nkey[i] = dkey(t0 + dt);
    if (dt < dt_min) atomicOr(status, ST_DTMIN);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        st.a[d * st.n + i] = acc[3 * i + d];
        st.j[d * st.n + i] = jerk[3 * i + d];
    }
}

cudaError_t init_dt_launch(const StateDev& st, const double* acc, const double* jerk,
                           double eta_start, double dt_max, double dt_min, double t0,
                           uint32_t* status, cudaStream_t s)
{
    if (st.n <= 0) return cudaSuccess;
    const int threads = 256;
    const unsigned blocks = static_cast<unsigned>((st.n + threads - 1) / threads);
    init_dt_kernel<<<blocks, threads, 0, s>>>(st, acc, jerk, eta_start, dt_max, dt_min, t0, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Energy diagnostic: per-block partial sums, then the last block adds the
// partials in block order (deterministic).
// ---------------------------------------------------------------------------
__global__ void energy_kernel(const StateDev st, const double* pot_all, double* partials,
                              double* out, uint32_t* ticket)
{
    __shared__ double sk[256], sw[256];
    double k = 0.0, w = 0.0;
    const int64_t n = st.n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double vx = st.v[i], vy = st.v[n + i], vz = st.v[2 * n + i];
        k += 0.5 * st.m[i] * (vx * vx + vy * vy + vz * vz);
        w += 0.5 * st.m[i] * pot_all[i];
    }
    sk[threadIdx.x] = k;
    sw[threadIdx.x] = w;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sk[threadIdx.x] += sk[threadIdx.x + o];
            sw[threadIdx.x] += sw[threadIdx.x + o];
        }
        __syncthreads();
    }
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = sk[0];
        partials[2 * blockIdx.x + 1] = sw[0];
        __threadfence();
        last = atomicAdd(ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        double K = 0.0, W = 0.0;
        for (unsigned b = 0; b < gridDim.x; ++b) {
            K += __ldcg(partials + 2 * b);
            W += __ldcg(partials + 2 * b + 1);
        }
        out[0] = K;
        out[1] = W;
        *ticket = 0u;
    }
}

cudaError_t energy_launch(const StateDev& st, const double* pot_all, double* partials,
                          int max_blocks, double* out, uint32_t* ticket, cudaStream_t s)
{
    int blocks = static_cast<int>((st.n + 255) / 256);
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    energy_kernel<<<blocks, 256, 0, s>>>(st, pot_all, partials, out, ticket);
    return cudaGetLastError();
}

__global__ void set_scalars_kernel(int32_t* i32, int32_t v, unsigned long long* t_bits,
                                   double t)
{
    if (i32) *i32 = v;
    if (t_bits) *t_bits = dkey(t);
}

cudaError_t set_scalars_launch(int32_t* i32, int32_t v, unsigned long long* t_bits, double t,
                               cudaStream_t s)
{
    set_scalars_kernel<<<1, 1, 0, s>>>(i32, v, t_bits, t);
    return cudaGetLastError();
}

double time_from_key(unsigned long long k)
{
    const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    double x;
    static_assert(sizeof(x) == sizeof(b), "double is 64-bit");
    memcpy(&x, &b, sizeof(x));
    return x;
}

// Per-cluster energies (block c sums cluster c in a fixed order).
__global__ void cluster_energy_kernel(const StateDev st, const int64_t* off, const double* pot_all,
                                      double* out)
{
    __shared__ double sk[256], sw[256];
    const int c = blockIdx.x;
    const int64_t n = st.n;
    double k = 0.0, w = 0.0;
    for (int64_t i = off[c] + threadIdx.x; i < off[c + 1]; i += blockDim.x) {
        const double vx = st.v[i], vy = st.v[n + i], vz = st.v[2 * n + i];
        k += 0.5 * st.m[i] * (vx * vx + vy * vy + vz * vz);
        w += 0.5 * st.m[i] * pot_all[i];
    }
    sk[threadIdx.x] = k;
    sw[threadIdx.x] = w;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sk[threadIdx.x] += sk[threadIdx.x + o];
            sw[threadIdx.x] += sw[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[2 * c] = sk[0];
        out[2 * c + 1] = sw[0];
    }
}

cudaError_t cluster_energy_launch(const StateDev& st, const ClusterDev& cl, const double* pot_all,
                                  double* out, cudaStream_t s)
{
    if (cl.k <= 0) return cudaSuccess;
    cluster_energy_kernel<<<cl.k, 256, 0, s>>>(st, cl.off, pot_all, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Layout helpers.
// ---------------------------------------------------------------------------
__global__ void aos_to_soa_kernel(const double* aos, double* soa, int64_t n)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 3 * n) return;
    const int64_t i = q / 3, c = q - 3 * i;
    soa[c * n + i] = aos[q];
}

__global__ void soa_to_aos_kernel(const double* soa, double* aos, int64_t n)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 3 * n) return;
    const int64_t i = q / 3, c = q - 3 * i;
    aos[q] = soa[c * n + i];
}

__global__ void iota_kernel(int32_t* idx, int64_t n, int32_t* n_act_dev)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) idx[i] = static_cast<int32_t>(i);
    if (i == 0 && n_act_dev) *n_act_dev = static_cast<int32_t>(n);
}

cudaError_t aos_to_soa_launch(const double* aos, double* soa, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    aos_to_soa_kernel<<<static_cast<unsigned>((3 * n + 255) / 256), 256, 0, s>>>(aos, soa, n);
    return cudaGetLastError();
}

cudaError_t soa_to_aos_launch(const double* soa, double* aos, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    soa_to_aos_kernel<<<static_cast<unsigned>((3 * n + 255) / 256), 256, 0, s>>>(soa, aos, n);
    return cudaGetLastError();
}

// Whole-state snapshot: buf = [m | x | v | a | j | t | dt | hq | nkey |
// bounds], the 17 n 64-bit words of the state (copied as bits) and one
// 8-byte slot for the two bounds.
__global__ void snapshot_kernel(StateDev st, double* __restrict__ buf, int to_buf)
{
    // row blockIdx.y copies one array; the rows' offsets in buf follow the
    // order m, x, v, a, j, t, dt, hq, nkey
    const int64_t n = st.n;
    unsigned long long* arr;
    int64_t len = n, off;
    switch (blockIdx.y) {
    case 0: arr = reinterpret_cast<unsigned long long*>(st.m), off = 0; break;
    case 1: arr = reinterpret_cast<unsigned long long*>(st.x), len = 3 * n, off = n; break;
    case 2: arr = reinterpret_cast<unsigned long long*>(st.v), len = 3 * n, off = 4 * n; break;
    case 3: arr = reinterpret_cast<unsigned long long*>(st.a), len = 3 * n, off = 7 * n; break;
    case 4: arr = reinterpret_cast<unsigned long long*>(st.j), len = 3 * n, off = 10 * n; break;
    case 5: arr = reinterpret_cast<unsigned long long*>(st.t), off = 13 * n; break;
    case 6: arr = reinterpret_cast<unsigned long long*>(st.dt), off = 14 * n; break;
    case 7: arr = reinterpret_cast<unsigned long long*>(st.hq), off = 15 * n; break;
    default: arr = st.nkey, off = 16 * n; break;
    }
    unsigned long long* w = reinterpret_cast<unsigned long long*>(buf) + off;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < len;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (to_buf) w[e] = arr[e];
        else arr[e] = w[e];
    }
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        uint32_t* b = reinterpret_cast<uint32_t*>(reinterpret_cast<unsigned long long*>(buf) + 17 * n);
        if (to_buf) b[0] = st.bound[0], b[1] = st.bound[1];
        else st.bound[0] = b[0], st.bound[1] = b[1];
    }
}

cudaError_t snapshot_launch(const StateDev& st, double* buf, bool to_buf, cudaStream_t s)
{
    if (st.n <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t want = (3 * st.n + threads - 1) / threads;  // the longest row
    const unsigned bx = static_cast<unsigned>(want < 512 ? want : 512);
    snapshot_kernel<<<dim3(bx, 9), threads, 0, s>>>(st, buf, to_buf ? 1 : 0);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// The context's particles are stored in its spatial order: internal index k
// holds the caller's particle perm[k].  These kernels move arrays across
// that boundary and re-order the stored state.
// ---------------------------------------------------------------------------
__global__ void permute_in_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                  int64_t n, int w, const int32_t* __restrict__ perm)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < w * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, k = e - c * n;
        dst[e] = src[w * static_cast<int64_t>(perm[k]) + c];
    }
}

__global__ void permute_out_kernel(const double* __restrict__ src, double* __restrict__ dst,
                                   int64_t n, int w, const int32_t* __restrict__ perm)
{
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < w * n;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = e / n, k = e - c * n;
        dst[w * static_cast<int64_t>(perm[k]) + c] = src[e];
    }
}

cudaError_t permute_in_launch(const double* src_aos, double* dst_soa, int64_t n, int w,
                              const int32_t* perm, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t want = (w * n + 255) / 256;
    permute_in_kernel<<<static_cast<unsigned>(want < 2048 ? want : 2048), 256, 0, s>>>(
        src_aos, dst_soa, n, w, perm);
    return cudaGetLastError();
}

cudaError_t permute_out_launch(const double* src_soa, double* dst_aos, int64_t n, int w,
                               const int32_t* perm, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t want = (w * n + 255) / 256;
    permute_out_kernel<<<static_cast<unsigned>(want < 2048 ? want : 2048), 256, 0, s>>>(
        src_soa, dst_aos, n, w, perm);
    return cudaGetLastError();
}

__global__ void map_index_kernel(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                 int32_t count, int64_t n, const int32_t* __restrict__ inv)
{
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= count) return;
    const int32_t u = in[a];
    out[a] = (u >= 0 && u < n) ? inv[u] : -1;  // -1: flagged by the kernel that reads it
}

cudaError_t map_index_launch(const int32_t* in, int32_t* out, int32_t count, int64_t n,
                             const int32_t* inv, cudaStream_t s)
{
    if (count <= 0) return cudaSuccess;
    map_index_kernel<<<static_cast<unsigned>((count + 255) / 256), 256, 0, s>>>(in, out, count,
                                                                                n, inv);
    return cudaGetLastError();
}

// Row r of the snapshot layout (m, x, v, a, j as 3 rows each, t, dt, hq,
// nkey: 17 rows of n words) gathered through map into the state.
__global__ void reorder_state_kernel(StateDev st, const double* __restrict__ buf,
                                     const int32_t* __restrict__ map)
{
    const int64_t n = st.n;
    const int r = blockIdx.y;
    unsigned long long* dst;
    if (r == 0) dst = reinterpret_cast<unsigned long long*>(st.m);
    else if (r < 4) dst = reinterpret_cast<unsigned long long*>(st.x) + (r - 1) * n;
    else if (r < 7) dst = reinterpret_cast<unsigned long long*>(st.v) + (r - 4) * n;
    else if (r < 10) dst = reinterpret_cast<unsigned long long*>(st.a) + (r - 7) * n;
    else if (r < 13) dst = reinterpret_cast<unsigned long long*>(st.j) + (r - 10) * n;
    else if (r == 13) dst = reinterpret_cast<unsigned long long*>(st.t);
    else if (r == 14) dst = reinterpret_cast<unsigned long long*>(st.dt);
    else if (r == 15) dst = reinterpret_cast<unsigned long long*>(st.hq);
    else dst = st.nkey;
    const unsigned long long* src = reinterpret_cast<const unsigned long long*>(buf) + r * n;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x)
        dst[k] = src[map[k]];
}

cudaError_t reorder_state_launch(const StateDev& st, const double* buf, const int32_t* map,
                                 cudaStream_t s)
{
    if (st.n <= 0) return cudaSuccess;
    const int64_t want = (st.n + 255) / 256;
    reorder_state_kernel<<<dim3(static_cast<unsigned>(want < 512 ? want : 512), 17), 256, 0, s>>>(
        st, buf, map);
    return cudaGetLastError();
}

__global__ void strided_list_kernel(int32_t* idx, int64_t k, int64_t n, int32_t* n_act_dev)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < k) idx[i] = static_cast<int32_t>(i * n / k);
    if (i == 0 && n_act_dev) *n_act_dev = static_cast<int32_t>(k);
}

cudaError_t strided_list_launch(int32_t* idx, int64_t k, int64_t n, int32_t* n_act_dev,
                                cudaStream_t s)
{
    const int64_t m = k > 0 ? k : 1;
    strided_list_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(idx, k, n,
                                                                               n_act_dev);
    return cudaGetLastError();
}

cudaError_t iota_launch(int32_t* idx, int64_t n, int32_t* n_act_dev, cudaStream_t s)
{
    const int64_t m = n > 0 ? n : 1;
    iota_kernel<<<static_cast<unsigned>((m + 255) / 256), 256, 0, s>>>(idx, n, n_act_dev);
    return cudaGetLastError();
}

}  // namespace nb
