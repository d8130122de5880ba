// The small-block builds of the force kernel (force_kernel.cuh with CTA =
// true: a block's CTAs sum their warps in shared memory and meet in a tree),
// one i per lane, every policy and j split.  Their own translation unit, so
// that they compile beside the plain builds in force.cu.
#include "force_kernel.cuh"

namespace nb {
namespace {

template <class K, int S>
const void* cta_k()
{
    return reinterpret_cast<const void*>(&force_kernel<K, 1, S, UniformPlan, true>);
}

template <class K>
const void* cta_split(int split)
{
    switch (split) {
    case 1: return cta_k<K, 1>();
    case 2: return cta_k<K, 2>();
    case 4: return cta_k<K, 4>();
    case 8: return cta_k<K, 8>();
    }
    return nullptr;
}

}  // namespace

const void* cta_kernel_ptr(Prec p, int split)
{
    switch (p) {
    case Prec::FP64: return cta_split<PolicyFP64<1>>(split);
    case Prec::MIXED: return cta_split<PolicyMixed<1>>(split);
    case Prec::MIXED_SPJ: return cta_split<PolicyMixed<1, true>>(split);
    case Prec::DS: return cta_split<PolicyDS<1>>(split);
    case Prec::HYBRID: return cta_split<PolicyHybrid<1>>(split);
    case Prec::HYBRID_SPJ: return cta_split<PolicyHybrid<1, true>>(split);
    case Prec::FP64_H6: return cta_split<PolicyFP64Snap<1>>(split);
    }
    return nullptr;
}

}  // namespace nb
