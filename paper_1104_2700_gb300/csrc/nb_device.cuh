// Device-side building blocks shared by the kernels of libnbody: status bits,
// mbarrier / bulk-copy wrappers (inline PTX, sm_100+), error-free FP32
// transforms and the per-context launch arguments.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nb {

// ---------------------------------------------------------------------------
// Device status word (OR-ed by kernels, read back by the host).
// ---------------------------------------------------------------------------
enum : uint32_t {
    ST_TIMEOUT = 1u,    // a bounded wait on an mbarrier gave up
    ST_NONFINITE = 2u,  // a force/jerk value or a timestep was not finite
    ST_DTMIN = 4u,      // a timestep fell below dt_min
    ST_BADINDEX = 8u,   // an active index was outside [0, n)
    ST_NOTDUE = 16u,    // a corrected particle was not due at the block time
};

// j particles per staged tile (the depth of each warp's tile ring is a
// property of each precision policy).
constexpr int TJ = 64;
constexpr int FORCE_WARPS = 4;  // warps per CTA of the force kernels

// About one second at the GB300 SM clock: the bound on any spin wait.
constexpr long long WAIT_LIMIT_CYCLES = 2000000000LL;

// Ghost j particles pad every system to a multiple of TJ; they carry zero
// mass and sit this far away, so each of their terms is an exact zero.
constexpr double GHOST_POS = 1.0e10;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// One-dimensional bulk copy global -> shared, completing on `bar`.
// Both addresses must be 16-byte aligned and `bytes` a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes "
        "[%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// atomicAdd with acquire-release semantics at GPU scope: the caller's
// earlier writes are visible to whoever observes the add, and the writes
// released by earlier adds to the same word are visible to the caller.
__device__ __forceinline__ uint32_t atomic_add_acq_rel_gpu(uint32_t* p, uint32_t v)
{
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;"
                 : "=r"(old)
                 : "l"(p), "r"(v)
                 : "memory");
    return old;
}

// Bounded wait for phase `parity` of `bar`; false after `limit` cycles.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  long long limit = WAIT_LIMIT_CYCLES)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// Error-free FP32 transforms (Knuth TwoSum; FMA-based TwoProd).  The _rn
// intrinsics keep the compiler from contracting or reordering them.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// p + e == a * b exactly (FMA-based TwoProd).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e)
{
    p = __fmul_rn(a, b);
    e = __fmaf_rn(a, b, -p);
}

// Grid-aligned double-single split.  Given a bound B on every |x| of one
// layout, q = P 2^-23 with P the least power of two above 2B.  hi is x
// rounded to a multiple of q (|hi| <= 2^23 q, so it fits a float exactly) and
// lo = x - hi (|lo| <= q/2, kept to 24 bits: hi + lo is x to ~B 2^-47).  Since
// every hi part lies on the same grid and |hi_j - hi_i| <= 2^24 q, the FP32
// difference of two hi parts is exact.  The factor 2 leaves room for values
// that grow past B before the bound is raised; a value beyond 2B still splits
// into hi + lo = x, only its hi part leaves the grid.
struct GridQuantum {
    double q, inv_q;  // both powers of two, so x * inv_q and k * q are exact
};

__device__ __forceinline__ GridQuantum grid_quantum(uint32_t bound_bits)
{
    int e;
    frexp(2.0 * static_cast<double>(__uint_as_float(bound_bits)), &e);
    return {ldexp(1.0, e - 23), ldexp(1.0, 23 - e)};
}

__device__ __forceinline__ void grid_split(double x, const GridQuantum& g, float& hi, float& lo)
{
    hi = __double2float_rn(rint(x * g.inv_q) * g.q);
    lo = __double2float_rn(x - static_cast<double>(hi));
}

// (jh + jl) - (ih + il) for grid-aligned splits, as a normalised (dh, dl):
// jh - ih is exact, and its magnitude is 0 or at least q >= |jl - il|, so
// Fast2Sum renormalises exactly.
__device__ __forceinline__ void grid_diff(float jh, float jl, float ih, float il, float& dh,
                                          float& dl)
{
    const float s = __fsub_rn(jh, ih);
    const float t = __fsub_rn(jl, il);
    dh = __fadd_rn(s, t);
    dl = __fsub_rn(t, __fsub_rn(dh, s));
}

// Running double-single accumulator: hi carries the sum, lo the collected
// rounding errors of every fold.
struct DSAcc {
    float hi, lo;
    __device__ __forceinline__ void zero() { hi = 0.f, lo = 0.f; }
    __device__ __forceinline__ void fold(float x)
    {
        float s, e;
        two_sum(hi, x, s, e);
        hi = s;
        lo = __fadd_rn(lo, e);
    }
    // Add a double-single term (th + tl).
    __device__ __forceinline__ void add(float th, float tl)
    {
        float s, e;
        two_sum(hi, th, s, e);
        hi = s;
        lo = __fadd_rn(lo, __fadd_rn(e, tl));
    }
    __device__ __forceinline__ double value() const
    {
        return static_cast<double>(hi) + static_cast<double>(lo);
    }
};

// A value of the split-group reduction tree.  Policies that accumulate in
// double-single hand their partial sums on as normalised float pairs, which
// the tree adds with TwoSum on the FP32 pipe (GB300's FP64 rate is a small
// fraction of FP32); a pair occupies the 8 bytes of a double in scratch.
struct DSPair {
    float h, l;
};
__device__ __forceinline__ DSPair ds_pair_of(const DSAcc& a)
{
    DSPair p;
    two_sum(a.hi, a.lo, p.h, p.l);
    return p;
}
__device__ __forceinline__ void tree_zero(double& a) { a = 0.0; }
__device__ __forceinline__ void tree_zero(DSPair& a) { a.h = a.l = 0.f; }
__device__ __forceinline__ void tree_add(double& a, double b) { a += b; }
__device__ __forceinline__ void tree_add(DSPair& a, DSPair b)
{
    float s, e;
    two_sum(a.h, b.h, s, e);
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    a.h = __fadd_rn(s, e);
    a.l = __fsub_rn(e, __fsub_rn(a.h, s));
}
__device__ __forceinline__ void tree_store(double* base, size_t k, double x) { base[k] = x; }
__device__ __forceinline__ void tree_store(double* base, size_t k, DSPair x)
{
    reinterpret_cast<float2*>(base)[k] = make_float2(x.h, x.l);
}
__device__ __forceinline__ void tree_load(const double* base, size_t k, double& x)
{
    x = __ldcg(base + k);
}
__device__ __forceinline__ void tree_load(const double* base, size_t k, DSPair& x)
{
    const float2 v = __ldcg(reinterpret_cast<const float2*>(base) + k);
    x.h = v.x, x.l = v.y;
}
// a += the same value of the lane lane ^ o (butterfly step; the sum is the
// same in both lanes, since the addition of two values is symmetric)
__device__ __forceinline__ void tree_xor(double& a, int o)
{
    tree_add(a, __shfl_xor_sync(0xffffffffu, a, o));
}
__device__ __forceinline__ void tree_xor(DSPair& a, int o)
{
    DSPair b;
    b.h = __shfl_xor_sync(0xffffffffu, a.h, o);
    b.l = __shfl_xor_sync(0xffffffffu, a.l, o);
    tree_add(a, b);
}
__device__ __forceinline__ double tree_value(double x) { return x; }
__device__ __forceinline__ double tree_value(DSPair x)
{
    return static_cast<double>(x.h) + static_cast<double>(x.l);
}

}  // namespace nb
