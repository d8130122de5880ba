// Host side of the force kernel (its templates are in force_kernel.cuh):
// kernel selection by precision, i-tile, j split and build, attributes,
// occupancy, scratch sizing and the launch itself.
#include "force_kernel.cuh"

namespace nb {

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
namespace {

// The plain builds: ensembles use the cluster plan, one system the uniform
// plan.
template <class K, int IT, int S>
const void* kfn(bool ens)
{
    return ens ? reinterpret_cast<const void*>(&force_kernel<K, IT, S, ClusterPlan, false>)
               : reinterpret_cast<const void*>(&force_kernel<K, IT, S, UniformPlan, false>);
}

// One i per lane with any j split; two i per lane without one.
template <class K1, class K2>
const void* kfn_split(int it, int split, bool ens)
{
    if (it == 1) {
        switch (split) {
        case 1: return kfn<K1, 1, 1>(ens);
        case 2: return kfn<K1, 1, 2>(ens);
        case 4: return kfn<K1, 1, 4>(ens);
        case 8: return kfn<K1, 1, 8>(ens);
        }
        return nullptr;
    }
    if constexpr (!std::is_same<K2, void>::value)
        if (it == 2 && split == 1) return kfn<K2, 2, 1>(ens);
    return nullptr;
}

// The kernel of one launch: a single system's small-block build (CTA mode,
// one i per lane) when asked for, else the plain build.
const void* kernel_ptr(Prec p, int it, int split, bool ens = false, bool cta = false)
{
    if (cta && it == 1 && !ens) return cta_kernel_ptr(p, split);
    switch (p) {
    case Prec::FP64: return kfn_split<PolicyFP64<1>, void>(it, split, ens);
    case Prec::MIXED: return kfn_split<PolicyMixed<1>, PolicyMixed<2>>(it, split, ens);
    case Prec::MIXED_SPJ:
        return kfn_split<PolicyMixed<1, true>, PolicyMixed<2, true>>(it, split, ens);
    case Prec::DS: return kfn_split<PolicyDS<1>, void>(it, split, ens);
    case Prec::HYBRID: return kfn_split<PolicyHybrid<1>, PolicyHybrid<2>>(it, split, ens);
    case Prec::HYBRID_SPJ:
        return kfn_split<PolicyHybrid<1, true>, PolicyHybrid<2, true>>(it, split, ens);
    case Prec::FP64_H6: return kfn_split<PolicyFP64Snap<1>, void>(it, split, ens);
    }
    return nullptr;
}

}  // namespace

int jlayout_narr(Prec p)
{
    switch (p) {
    case Prec::FP64: return 2;
    case Prec::MIXED:
    case Prec::MIXED_SPJ: return 3;
    case Prec::DS: return 4;
    case Prec::HYBRID:
    case Prec::HYBRID_SPJ: return 4;
    case Prec::FP64_H6: return 3;
    }
    return 0;
}

int jlayout_elem_bytes(Prec p, int k)
{
    switch (p) {
    case Prec::FP64: return k < 2 ? 32 : 0;
    case Prec::MIXED:
    case Prec::MIXED_SPJ: return k < 2 ? 16 : (k == 2 ? 8 : 0);
    case Prec::DS: return k < 4 ? 16 : 0;
    case Prec::HYBRID:
    case Prec::HYBRID_SPJ: return k < 4 ? 16 : 0;
    case Prec::FP64_H6: return k < 3 ? 32 : 0;
    }
    return 0;
}

size_t force_smem_bytes(Prec p)
{
    switch (p) {
    case Prec::FP64: return (size_t)FORCE_WARPS * WarpSmem<PolicyFP64<1>>::BYTES;
    case Prec::MIXED:
    case Prec::MIXED_SPJ: return (size_t)FORCE_WARPS * WarpSmem<PolicyMixed<1>>::BYTES;
    case Prec::DS: return (size_t)FORCE_WARPS * WarpSmem<PolicyDS<1>>::BYTES;
    case Prec::HYBRID:
    case Prec::HYBRID_SPJ: return (size_t)FORCE_WARPS * WarpSmem<PolicyHybrid<1>>::BYTES;
    case Prec::FP64_H6: return (size_t)FORCE_WARPS * WarpSmem<PolicyFP64Snap<1>>::BYTES;
    }
    return 0;
}

bool force_variant_exists(Prec p, int it, int split) { return kernel_ptr(p, it, split) != nullptr; }

cudaError_t force_setup(Prec p, int it, int split)
{
    for (int e = 0; e < 3; ++e) {  // plain, ensemble, small-block builds
        const void* fn = kernel_ptr(p, it, split, e == 1, e == 2);
        if (!fn) return cudaErrorInvalidValue;
        const cudaError_t r = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   static_cast<int>(force_smem_bytes(p)));
        if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
}

int force_ctas_per_sm(Prec p, int it, int split)
{
    const void* fn = kernel_ptr(p, it, split);
    if (!fn) return 0;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, FORCE_WARPS * 32,
                                                      force_smem_bytes(p)) != cudaSuccess)
        return 0;
    return nb;
}

size_t force_scratch_doubles(int it, int64_t n_act_max, int warps)
{
    const int64_t GI = 32 * it;
    const int64_t G = (n_act_max + GI - 1) / GI;
    return (size_t)((int64_t)warps * MAX_CHUNKS + G) * MAX_NV * GI;
}

int64_t force_counter_stride(int64_t n_act_max, int warps)
{
    // chunks + groups (groups are at least 32 / 8 wide)
    return (int64_t)warps * MAX_CHUNKS + (n_act_max + 3) / 4;
}

int64_t force_counter_entries(int64_t n_act_max, int warps)
{
    // the reduction levels, then the chunk queue word
    return RLEVELS * force_counter_stride(n_act_max, warps) + 1;
}

cudaError_t force_launch(const ForceArgs& a, cudaStream_t s)
{
    const bool ens = a.plan.grp_tile0 != nullptr;
    const void* fn = kernel_ptr(a.prec, a.it, a.split, ens, a.cta_mode && !ens);
    if (!fn || a.grid <= 0) return cudaErrorInvalidValue;
    ForceParams f;
    f.jl0 = a.jl.arr[0];
    f.jl1 = a.jl.arr[1];
    f.jl2 = a.jl.arr[2];
    f.jl3 = a.jl.arr[3];
    f.n = a.n;
    f.n_pad = a.n_pad;
    f.idx = a.idx;
    f.n_act_dev = a.n_act_dev;
    f.acc = a.acc;
    f.jerk = a.jerk;
    f.pot = a.pot;
    f.snap = a.snap;
    f.scratch = a.scratch;
    f.counters = a.counters;
    f.counter_stride = a.counter_stride;
    f.status = a.status;
    f.eps2 = a.eps2;
    f.nact_lo = a.nact_lo;
    f.nact_hi = a.nact_hi;
    f.wait_limit = a.wait_limit > 0 ? a.wait_limit : WAIT_LIMIT_CYCLES;
    f.unfed_first_tile = a.unfed_first_tile;
    f.grp_cluster = a.plan.grp_cluster;
    f.grp_act_begin = a.plan.grp_act_begin;
    f.grp_act_count = a.plan.grp_act_count;
    f.grp_tile0 = a.plan.grp_tile0;
    f.plan_scalars = a.plan.scalars;
    f.cl_off = a.plan.cl_off;
    f.cl_joff = a.plan.cl_joff;
    f.cl_eps2 = a.plan.cl_eps2;
    f.st_a = a.st_a;
    f.st_j = a.st_j;
    f.bound_v = a.bound_v;
    f.st_dt = a.st_dt;
    f.st_hq = a.st_hq;
    f.eta = a.eta;
    f.jt_lo = a.jt_lo;
    f.jt_hi = a.jt_hi;
    f.cta_mode = a.cta_mode && !a.plan.grp_tile0;
    f.n_act_host = a.n_act_host;
    f.idx_map = a.idx_map;
    f.guard_eta = static_cast<float>(HY_GUARD * a.eta);
    f.dyn_chunks = ens ? (a.dyn_chunks < MAX_CHUNKS ? a.dyn_chunks : MAX_CHUNKS) : 0;
    f.queue = a.counters + RLEVELS * a.counter_stride;
    if (f.jt_hi > 0 && (a.plan.grp_tile0 || f.jt_lo < 0 || f.jt_hi <= f.jt_lo ||
                        f.jt_hi > f.n_pad / TJ))
        return cudaErrorInvalidValue;
    if (a.prec == Prec::FP64_H6 && !f.snap) return cudaErrorInvalidValue;
    if (is_hybrid(a.prec) &&
        (!f.st_a || !f.st_j || !f.bound_v || !f.st_dt || !f.st_hq))
        return cudaErrorInvalidValue;
    void* args[] = {&f};
    return cudaLaunchKernel(fn, dim3(a.grid), dim3(FORCE_WARPS * 32), args,
                            force_smem_bytes(a.prec), s);
}

}  // namespace nb
