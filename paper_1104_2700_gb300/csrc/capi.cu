// C ABI of libnbody (declared in include/nbody.h): context lifetime, device
// buffers and the host-side sequencing of the Hermite block-timestep steps
// of Sec. 2.  All arithmetic of the method runs in the kernels of force.cu
// and hermite.cu; this file only moves data and launches them.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "nb_device.cuh"
#include "nb_launch.h"
#include "nbody.h"

using nb::Prec;

// Ensembles: stream-K chunks per warp by default.  Only the hybrid
// precisions have tiles of unequal cost (the far loop, the near pass, groups
// under the integration guard); there four chunks, those past a warp's
// first taken from a queue, took the 256-system ensemble's block step from
// 371 to 309 us (to t = 1/4).  Elsewhere every tile costs the same, and the
// queue's per-chunk set-up cost DS 3 %.
int32_t ens_chunks_default(Prec p) { return nb::is_hybrid(p) ? 4 : 1; }

struct nb_ctx {
    nb_config cfg{};
    Prec prec = Prec::MIXED;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    // A second stream for the launch variant that sits idle: both variants of
    // a device-sized block go out as parallel branches (fork on ev_fork, join
    // on ev_join), so the idle one's launch and exit cost no time in series.
    cudaStream_t aux = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int num_sms = 0;
    // Force launch variants of the context precision: [0] for blocks with
    // n_act < nact_split, [1] for larger ones, [2] for blocks of fewer than
    // tiny_split particles whose size the host knows (none while tiny_split
    // is 0).  A device-sized block never takes [2]: a third parallel branch
    // costs each block step more than the shape saves.
    struct Variant {
        int it = 1;
        int grid = 0;
        int split = 1;  // lanes per i (j split inside a warp)
    } var[3];
    int32_t nact_split = 1024;
    int32_t tiny_split = 0;
    int32_t ens_chunks = 1;  // ensembles: stream-K chunks per warp
    int grid64 = 0;      // persistent CTAs of the FP64 energy pass (1 i per thread)
    size_t scratch_cap = 0;    // doubles allocated for split-group partials
    int64_t counter_cap = 0;   // counter words allocated
    int64_t n = 0, n_pad = 0, cap = 0;
    double eps = 0.0, eta = 0.02;
    nb::StateDev st;
    nb::JLayout jl;      // context precision
    nb::JLayout jl64;    // FP64 layout for the FP64 potential (non-FP64 contexts)
    nb::SchedDev sd;
    int32_t* idx_user = nullptr;
    int32_t* n_act_user = nullptr;
    double* acc1 = nullptr;
    double* jerk1 = nullptr;
    double* pot1 = nullptr;
    double* snap1 = nullptr;  // sixth-order variant: the block's new snap
    double* scratch = nullptr;
    uint32_t* counters = nullptr;
    int64_t counter_stride = 0;
    int64_t counter_words = 0;
    uint32_t* status_dev = nullptr;
    unsigned long long* ctr64 = nullptr;  // [0] block steps, [1] interactions
    double* energy_partials = nullptr;
    double* energy_out = nullptr;
    uint32_t* energy_ticket = nullptr;
    double* staging = nullptr;  // 3n doubles
    // Ensemble mode (nb_set_ensemble): k independent systems in one context.
    bool ens = false;
    nb::ClusterDev cl;
    std::vector<int64_t> h_off;  // host copy of the particle offsets
    double* cl_energy = nullptr; // 2k
    int64_t cap_pad = 0, cap_k = 0;
    unsigned char* pinned = nullptr;
    int energy_blocks = 0;
    int32_t last_force_n_act = -1;
    bool loaded = false;
    nb_status sticky = NB_OK;
    std::string err;
    // CUDA graph of GRAPH_STEPS device-resident block steps for one t_end.
    cudaGraphExec_t step_graph = nullptr;
    double graph_t_end = 0.0;
    // The particles are stored in a spatial order: internal index k holds the
    // caller's particle perm[k] (inv is the inverse).  For one system the
    // order follows a Morton curve through its bounding box, so the j tiles
    // and the i-groups cut from the (ascending) active lists are each close
    // together in space, which the hybrid precision's far-tile test needs;
    // an ensemble keeps the order it was given (see order_of).  The order is a pure function of the caller-order positions it
    // was computed from (kept in order_pos, with the systems' offsets in
    // order_off): it is recomputed at every load and at the start of every
    // nb_step_until, so a run resumed from a checkpoint gets the order the
    // original had.  Device copies perm_dev / inv_dev are the reference;
    // the host copies are refreshed from them when host_order_stale (after
    // nb_restore, which restores the order stored with a snapshot).
    std::vector<int32_t> h_perm, h_inv;
    int32_t* perm_dev = nullptr;
    int32_t* inv_dev = nullptr;
    double* order_buf = nullptr;  // 17 n + 1 doubles: the state while it is re-ordered
    std::vector<double> order_pos;
    std::vector<int64_t> order_off;
    bool order_fresh = false;       // no step has moved the particles since
    bool host_order_stale = false;
    // j partition (nb_set_j_part): force evaluations of the context
    // precision sum over part j_part of j_parts contiguous ranges of tiles.
    int32_t j_part = 0, j_parts = 1;
};

namespace {

constexpr size_t PINNED_BYTES = 256;
constexpr int GRAPH_STEPS = 32;  // block steps per replay of the step graph

void drop_graph(nb_ctx* c)
{
    if (c->step_graph) cudaGraphExecDestroy(c->step_graph);
    c->step_graph = nullptr;
}

nb_status fail(nb_ctx* c, nb_status s, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
nb_status fail(nb_ctx* c, nb_status s, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    if (c) {
        c->err = buf;
        if (s != NB_EINVAL) c->sticky = s;
    }
    return s;
}

#define NB_CK(ctx, call)                                                                 \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail((ctx), e_ == cudaErrorMemoryAllocation ? NB_ENOMEM : NB_ECUDA,   \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                        __LINE__);                                                       \
    } while (0)

bool is_pow2(double x)
{
    if (!(x > 0.0) || !std::isfinite(x)) return false;
    int e;
    return std::frexp(x, &e) == 0.5;
}

template <class T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

void free_buffers(nb_ctx* c)
{
    dfree(c->st.m), dfree(c->st.x), dfree(c->st.v), dfree(c->st.a), dfree(c->st.j);
    dfree(c->st.t), dfree(c->st.dt), dfree(c->st.hq), dfree(c->st.nkey);
    dfree(c->perm_dev), dfree(c->inv_dev), dfree(c->order_buf);
    c->order_pos.clear();
    c->order_fresh = false;
    c->host_order_stale = false;
    for (int k = 0; k < 4; ++k) {
        if (c->jl.arr[k]) cudaFree(c->jl.arr[k]);
        if (c->jl64.arr[k]) cudaFree(c->jl64.arr[k]);
        c->jl.arr[k] = c->jl64.arr[k] = nullptr;
    }
    dfree(c->sd.tmin_bits), dfree(c->sd.idx), dfree(c->sd.n_act);
    dfree(c->sd.block_counts), dfree(c->sd.block_offsets), dfree(c->sd.ticket);
    dfree(c->idx_user), dfree(c->n_act_user), dfree(c->acc1), dfree(c->jerk1), dfree(c->pot1);
    dfree(c->snap1), dfree(c->st.s), dfree(c->st.c);
    dfree(c->scratch), dfree(c->counters), dfree(c->staging);
    dfree(c->energy_partials), dfree(c->energy_out), dfree(c->energy_ticket);
    dfree(c->cl.off), dfree(c->cl.joff), dfree(c->cl.eps2), dfree(c->cl.cluster_of);
    dfree(c->cl.jsrc), dfree(c->cl.tkey), dfree(c->cl.cnt), dfree(c->cl.grp_cluster);
    dfree(c->cl.grp_act_begin);
    dfree(c->cl.grp_act_count), dfree(c->cl.grp_tile0), dfree(c->cl.plan_scalars);
    dfree(c->cl_energy);
    c->cap = c->cap_pad = c->cap_k = 0;
}

nb_status alloc_layout(nb_ctx* c, Prec p, nb::JLayout& jl, int64_t n_pad)
{
    for (int k = 0; k < nb::jlayout_narr(p); ++k)
        NB_CK(c, cudaMalloc(&jl.arr[k], (size_t)n_pad * nb::jlayout_elem_bytes(p, k)));
    return NB_OK;
}

// Scratch for the split-group partials and reduction counters, enough for
// the three launch variants (and the FP64 energy pass) on up
// to cap particles in cap_k systems.  Grows only; drops the step graph when
// the buffers move.
nb_status ensure_force_scratch(nb_ctx* c)
{
    const int64_t n = c->cap, k = c->cap_k;
    const int64_t groups_bound = n + 32 * k;  // i-groups never mix systems
    size_t need = nb::force_scratch_doubles(1, groups_bound, c->grid64 * nb::FORCE_WARPS);
    int max_grid = c->grid64;
    for (const auto& var : c->var) {
        need = std::max(need, nb::force_scratch_doubles(var.it, groups_bound + 32 * var.it * k,
                                                        var.grid * nb::FORCE_WARPS));
        max_grid = std::max(max_grid, var.grid);
    }
    const int64_t stride = nb::force_counter_stride(groups_bound, max_grid * nb::FORCE_WARPS);
    const int64_t words = nb::force_counter_entries(groups_bound, max_grid * nb::FORCE_WARPS);
    if (need > c->scratch_cap) {
        dfree(c->scratch);
        NB_CK(c, cudaMalloc(&c->scratch, need * sizeof(double)));
        c->scratch_cap = need;
        drop_graph(c);
    }
    if (words > c->counter_cap) {
        dfree(c->counters);
        NB_CK(c, cudaMalloc(&c->counters, words * sizeof(uint32_t)));
        NB_CK(c, cudaMemset(c->counters, 0, words * sizeof(uint32_t)));
        c->counter_cap = words;
        drop_graph(c);
    }
    c->counter_stride = stride;
    c->counter_words = words;
    return NB_OK;
}

// Size every n-dependent buffer for n particles in k systems (k = 0: one
// system without cluster arrays) whose j layout has n_pad slots.
nb_status ensure_capacity(nb_ctx* c, int64_t n, int64_t n_pad, int64_t k)
{
    if (n <= c->cap && n_pad <= c->cap_pad && k <= c->cap_k) {
        c->n = n;
        c->n_pad = n_pad;
        c->st.n = n;
        c->st.n_pad = n_pad;
        c->cl.k = static_cast<int>(k);
        return NB_OK;
    }
    free_buffers(c);
    const size_t d = sizeof(double);
    NB_CK(c, cudaMalloc(&c->st.m, n * d));
    NB_CK(c, cudaMalloc(&c->st.x, 3 * n * d));
    NB_CK(c, cudaMalloc(&c->st.v, 3 * n * d));
    NB_CK(c, cudaMalloc(&c->st.a, 3 * n * d));
    NB_CK(c, cudaMalloc(&c->st.j, 3 * n * d));
    NB_CK(c, cudaMalloc(&c->st.t, n * d));
    NB_CK(c, cudaMalloc(&c->st.dt, n * d));
    NB_CK(c, cudaMalloc(&c->st.hq, n * d));
    NB_CK(c, cudaMalloc(&c->st.nkey, n * sizeof(unsigned long long)));
    NB_CK(c, cudaMalloc(&c->perm_dev, n * sizeof(int32_t)));
    NB_CK(c, cudaMalloc(&c->inv_dev, n * sizeof(int32_t)));
    // i-groups never mix systems: at most n / 32 + k of them
    const int64_t groups_bound = n + 32 * k;
    nb_status s = alloc_layout(c, c->prec, c->jl, n_pad);
    if (s != NB_OK) return s;
    if (c->prec != Prec::FP64) {
        s = alloc_layout(c, Prec::FP64, c->jl64, n_pad);
        if (s != NB_OK) return s;
    }
    c->sd.max_blocks = static_cast<int>((n + nb::SCHED_CHUNK - 1) / nb::SCHED_CHUNK);
    NB_CK(c, cudaMalloc(&c->sd.tmin_bits, sizeof(unsigned long long)));
    NB_CK(c, cudaMalloc(&c->sd.idx, n * sizeof(int32_t)));
    NB_CK(c, cudaMalloc(&c->sd.n_act, sizeof(int32_t)));
    NB_CK(c, cudaMalloc(&c->sd.block_counts, c->sd.max_blocks * sizeof(int32_t)));
    NB_CK(c, cudaMalloc(&c->sd.block_offsets, c->sd.max_blocks * sizeof(int32_t)));
    NB_CK(c, cudaMalloc(&c->sd.ticket, sizeof(uint32_t)));
    NB_CK(c, cudaMemset(c->sd.ticket, 0, sizeof(uint32_t)));
    NB_CK(c, cudaMemset(c->sd.n_act, 0, sizeof(int32_t)));
    NB_CK(c, cudaMalloc(&c->idx_user, n * sizeof(int32_t)));
    NB_CK(c, cudaMalloc(&c->n_act_user, sizeof(int32_t)));
    NB_CK(c, cudaMalloc(&c->acc1, 3 * n * d));
    NB_CK(c, cudaMalloc(&c->jerk1, 3 * n * d));
    NB_CK(c, cudaMalloc(&c->pot1, n * d));
    if (c->prec == Prec::FP64_H6) {
        NB_CK(c, cudaMalloc(&c->snap1, 3 * n * d));
        NB_CK(c, cudaMalloc(&c->st.s, 3 * n * d));
        NB_CK(c, cudaMalloc(&c->st.c, 3 * n * d));
    }
    NB_CK(c, cudaMalloc(&c->staging, 3 * n * d));
    c->scratch_cap = 0;
    c->counter_cap = 0;
    (void)groups_bound;
    c->energy_blocks = static_cast<int>(std::min<int64_t>((n + 255) / 256, 1024));
    NB_CK(c, cudaMalloc(&c->energy_partials, 2 * c->energy_blocks * d));
    NB_CK(c, cudaMalloc(&c->energy_out, 2 * d));
    NB_CK(c, cudaMalloc(&c->energy_ticket, sizeof(uint32_t)));
    NB_CK(c, cudaMemset(c->energy_ticket, 0, sizeof(uint32_t)));
    if (k > 0) {
        nb::ClusterDev& cl = c->cl;
        cl.max_groups = n / 4 + k + 1;  // groups are at least 32 / 8 wide
        NB_CK(c, cudaMalloc(&cl.off, (k + 1) * sizeof(int64_t)));
        NB_CK(c, cudaMalloc(&cl.joff, (k + 1) * sizeof(int64_t)));
        NB_CK(c, cudaMalloc(&cl.eps2, k * sizeof(double)));
        NB_CK(c, cudaMalloc(&cl.cluster_of, n * sizeof(int32_t)));
        NB_CK(c, cudaMalloc(&cl.jsrc, n_pad * sizeof(int32_t)));
        NB_CK(c, cudaMalloc(&cl.tkey, k * sizeof(unsigned long long)));
        NB_CK(c, cudaMalloc(&cl.cnt, k * sizeof(int32_t)));
        NB_CK(c, cudaMalloc(&cl.grp_cluster, cl.max_groups * sizeof(int32_t)));
        NB_CK(c, cudaMalloc(&cl.grp_act_begin, cl.max_groups * sizeof(int32_t)));
        NB_CK(c, cudaMalloc(&cl.grp_act_count, cl.max_groups * sizeof(int32_t)));
        NB_CK(c, cudaMalloc(&cl.grp_tile0, (cl.max_groups + 1) * sizeof(int64_t)));
        NB_CK(c, cudaMalloc(&cl.plan_scalars, 2 * sizeof(int64_t)));
        NB_CK(c, cudaMalloc(&c->cl_energy, 2 * k * sizeof(double)));
    }
    c->cl.k = static_cast<int>(k);
    c->cap_pad = n_pad;
    c->cap_k = k;
    c->cap = n;
    s = ensure_force_scratch(c);
    if (s != NB_OK) return s;
    c->n = n;
    c->n_pad = n_pad;
    c->st.n = n;
    c->st.n_pad = n_pad;
    return NB_OK;
}

nb_status enter(nb_ctx* c, bool need_particles)
{
    if (!c) return NB_EINVAL;
    c->err.clear();
    if (c->sticky != NB_OK) return fail(c, c->sticky, "context is in error state %d", c->sticky);
    if (need_particles && !c->loaded) return fail(c, NB_ESTATE, "no particles loaded");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, NB_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return NB_OK;
}

// Read the device status word (blocking) and turn it into an nb_status.
nb_status check_status(nb_ctx* c)
{
    uint32_t* h = reinterpret_cast<uint32_t*>(c->pinned);
    NB_CK(c, cudaMemcpyAsync(h, c->status_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                             c->stream));
    NB_CK(c, cudaStreamSynchronize(c->stream));
    const uint32_t st = *h;
    if (st == 0) return NB_OK;
    // Leave the split-group counters clean for the next launch.
    cudaMemsetAsync(c->counters, 0, c->counter_words * sizeof(uint32_t), c->stream);
    cudaMemsetAsync(c->status_dev, 0, sizeof(uint32_t), c->stream);
    cudaStreamSynchronize(c->stream);
    if (st & nb::ST_TIMEOUT) return fail(c, NB_ETIMEOUT, "device wait timed out");
    if (st & nb::ST_NONFINITE) return fail(c, NB_ENONFINITE, "non-finite force, jerk or timestep");
    if (st & nb::ST_DTMIN) return fail(c, NB_EDTMIN, "timestep below dt_min");
    if (st & nb::ST_BADINDEX) return fail(c, NB_EINVAL, "particle index out of range");
    if (st & nb::ST_NOTDUE) return fail(c, NB_ESTATE, "particle not due at the block time");
    return fail(c, NB_ECUDA, "unknown device status 0x%x", st);
}

// Force on the active list idx[0..*n_act_dev).  In the context precision the
// two launch variants go out back to back, each working only inside its
// n_act window (the block size is read on the device); when the caller
// knows n_act (n_act_host >= 0) only the matching variant is launched.
nb::ForceArgs force_args(nb_ctx* c, Prec p, const nb::JLayout& jl, const int32_t* idx,
                         const int32_t* n_act_dev);

nb_status run_force(nb_ctx* c, Prec p, const nb::JLayout& jl, const int32_t* idx,
                    const int32_t* n_act_dev, int32_t n_act_host = -1,
                    const int32_t* idx_map = nullptr)
{
    nb::ForceArgs f = force_args(c, p, jl, idx, n_act_dev);
    f.n_act_host = n_act_host;  // known here: the kernel need not read it
    f.idx_map = idx_map;
    if (p == c->prec && c->j_parts > 1) {
        const int64_t nt = c->n_pad / nb::TJ;
        f.jt_lo = nt * c->j_part / c->j_parts;
        f.jt_hi = nt * (c->j_part + 1) / c->j_parts;
    }
    if (p != c->prec) {  // the FP64 energy pass of a lower-precision context
        f.it = 1;
        f.split = 1;
        f.grid = c->grid64;
        NB_CK(c, nb::force_launch(f, c->stream));
        return NB_OK;
    }
    // With the block size known here, one launch of the variant whose
    // window holds it.
    if (n_act_host >= 0) {
        const int v = n_act_host < c->tiny_split ? 2 : n_act_host < c->nact_split ? 0 : 1;
        f.it = c->var[v].it;
        f.split = c->var[v].split;
        f.grid = c->var[v].grid;
        f.cta_mode = !c->ens && v != 1;  // small blocks: CTA-level sums
        f.nact_lo = 0;
        f.nact_hi = 0x7fffffff;
        NB_CK(c, nb::force_launch(f, c->stream));
        return NB_OK;
    }
    // With the block size on the device both the small and the large variant
    // are launched, the small one on the aux stream; exactly one of them does
    // any work, and neither touches memory the other uses before it has read
    // n_act.
    NB_CK(c, cudaEventRecord(c->ev_fork, c->stream));
    NB_CK(c, cudaStreamWaitEvent(c->aux, c->ev_fork, 0));
    for (int v = 0; v < 2; ++v) {
        f.it = c->var[v].it;
        f.split = c->var[v].split;
        f.grid = c->var[v].grid;
        f.cta_mode = !c->ens && v == 0;  // small blocks: CTA-level sums
        f.nact_lo = v == 0 ? 0 : c->nact_split;
        f.nact_hi = v == 0 ? c->nact_split : 0x7fffffff;
        NB_CK(c, nb::force_launch(f, v == 0 ? c->aux : c->stream));
    }
    NB_CK(c, cudaEventRecord(c->ev_join, c->aux));
    NB_CK(c, cudaStreamWaitEvent(c->stream, c->ev_join, 0));
    return NB_OK;
}

// Launch arguments shared by every force launch of the context.
nb::ForceArgs force_args(nb_ctx* c, Prec p, const nb::JLayout& jl, const int32_t* idx,
                         const int32_t* n_act_dev)
{
    nb::ForceArgs f;
    f.prec = p;
    f.jl = jl;
    f.n = c->n;
    f.n_pad = c->n_pad;
    f.idx = idx;
    f.n_act_dev = n_act_dev;
    f.acc = c->acc1;
    f.jerk = c->jerk1;
    f.pot = c->pot1;
    f.snap = c->snap1;
    f.scratch = c->scratch;
    f.st_a = c->st.a;
    f.st_j = c->st.j;
    f.bound_v = c->st.bound + 1;
    f.st_dt = c->st.dt;
    f.st_hq = c->st.hq;
    f.eta = c->eta;
    f.dyn_chunks = c->ens ? c->ens_chunks : 0;
    f.counters = c->counters;
    f.counter_stride = c->counter_stride;
    f.status = c->status_dev;
    f.eps2 = c->eps * c->eps;
    f.wait_limit = c->cfg.wait_limit_cycles;
    f.cta_mode = 0;  // the small-block build: run_force and the autotuner choose it
    if (c->ens) {
        // the plan for this active list must have been written by plan_launch
        f.plan.grp_cluster = c->cl.grp_cluster;
        f.plan.grp_act_begin = c->cl.grp_act_begin;
        f.plan.grp_act_count = c->cl.grp_act_count;
        f.plan.grp_tile0 = c->cl.grp_tile0;
        f.plan.scalars = c->cl.plan_scalars;
        f.plan.cl_off = c->cl.off;
        f.plan.cl_joff = c->cl.joff;
        f.plan.cl_eps2 = c->cl.eps2;
    }
    return f;
}

// Force on a sorted active list: in ensemble mode the plan comes first.
// plan_from_counts: idx is the select's list of this block step, so the plan
// may take each cluster's share from the select's per-cluster counts.
nb_status run_force_list(nb_ctx* c, Prec p, const nb::JLayout& jl, const int32_t* idx,
                         const int32_t* n_act_dev, int32_t n_act_host = -1,
                         bool plan_from_counts = false)
{
    if (c->ens) {
        // both variants of an ensemble context share one i-group width
        const int gi = p == c->prec ? 32 * c->var[0].it / c->var[0].split : 32;
        NB_CK(c, nb::plan_launch(c->cl, idx, n_act_dev, gi, c->stream, plan_from_counts));
    }
    return run_force(c, p, jl, idx, n_act_dev, n_act_host);
}

// Caller arrays in, through the spatial order: w doubles per particle (3: an
// n x 3 row-major array into SoA; 1: a scalar per particle).
nb_status upload_perm(nb_ctx* c, const double* src, double* dst, int w, int on_device)
{
    NB_CK(c, cudaMemcpyAsync(c->staging, src, w * c->n * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                             c->stream));
    NB_CK(c, nb::permute_in_launch(c->staging, dst, c->n, w, c->perm_dev, c->stream));
    return NB_OK;
}

nb_status upload_vec3(nb_ctx* c, const double* src, double* dst_soa, int on_device)
{
    return upload_perm(c, src, dst_soa, 3, on_device);
}

// State arrays out to the caller's order (w doubles per particle).
nb_status download_perm(nb_ctx* c, const double* src, double* dst, int w, int on_device)
{
    NB_CK(c, nb::permute_out_launch(src, c->staging, c->n, w, c->perm_dev, c->stream));
    NB_CK(c, cudaMemcpyAsync(dst, c->staging, w * c->n * sizeof(double),
                             on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream));
    return NB_OK;
}

// The host copies of the order, from the device copy when they are stale.
nb_status sync_host_order(nb_ctx* c)
{
    if (!c->host_order_stale) return NB_OK;
    c->h_perm.resize(c->n);
    NB_CK(c, cudaMemcpyAsync(c->h_perm.data(), c->perm_dev, c->n * sizeof(int32_t),
                             cudaMemcpyDeviceToHost, c->stream));
    NB_CK(c, cudaStreamSynchronize(c->stream));
    c->h_inv.resize(c->n);
    for (int64_t k = 0; k < c->n; ++k) c->h_inv[c->h_perm[k]] = static_cast<int32_t>(k);
    c->host_order_stale = false;
    return NB_OK;
}

// Morton key of a point of the box [lo, lo + ext): 16 bits per axis,
// interleaved (bit b of axis d at bit 3 b + d).
uint64_t morton48(const double* x, const double* lo, const double* ext)
{
    uint64_t key = 0;
    for (int d = 0; d < 3; ++d) {
        double u = ext[d] > 0.0 ? (x[d] - lo[d]) / ext[d] : 0.0;
        if (!(u >= 0.0)) u = 0.0;  // also NaN
        if (u > 1.0) u = 1.0;
        const uint32_t q = static_cast<uint32_t>(u * 65535.0);
        for (int b = 0; b < 16; ++b) key |= static_cast<uint64_t>((q >> b) & 1u) << (3 * b + d);
    }
    return key;
}

// The spatial order of caller-order positions r[n][3]: within each system
// (particles [off[q], off[q+1])), the particles sorted by the Morton key of
// their position in the system's bounding box, ties by index.  perm[k] is
// the caller's particle at internal index k.  An ensemble keeps the order it
// was given: its systems are small and its blocks few particles each, so its
// i-groups would not be compact anyway, and the far-tile path pays only for
// large blocks of large systems.
std::vector<int32_t> order_of(const double* r, const std::vector<int64_t>& off)
{
    std::vector<int32_t> perm(off.back());
    if (off.size() > 2) {
        for (int64_t k = 0; k < off.back(); ++k) perm[k] = static_cast<int32_t>(k);
        return perm;
    }
    std::vector<std::pair<uint64_t, int32_t>> keys;
    for (size_t q = 0; q + 1 < off.size(); ++q) {
        double lo[3], hi[3], ext[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = HUGE_VAL;
            hi[d] = -HUGE_VAL;
        }
        for (int64_t i = off[q]; i < off[q + 1]; ++i)
            for (int d = 0; d < 3; ++d) {
                const double x = r[3 * i + d];
                if (!std::isfinite(x)) continue;
                lo[d] = std::min(lo[d], x);
                hi[d] = std::max(hi[d], x);
            }
        for (int d = 0; d < 3; ++d) {
            if (!(lo[d] <= hi[d])) lo[d] = hi[d] = 0.0;  // no finite coordinate
            ext[d] = hi[d] - lo[d];
        }
        keys.clear();
        for (int64_t i = off[q]; i < off[q + 1]; ++i)
            keys.emplace_back(morton48(r + 3 * i, lo, ext), static_cast<int32_t>(i));
        std::sort(keys.begin(), keys.end());
        for (size_t k = 0; k < keys.size(); ++k) perm[off[q] + k] = keys[k].second;
    }
    return perm;
}

// Order of a load (caller-order host positions r): kept when the positions
// and systems are those the current order was computed from.  Returns in
// *same whether the order is unchanged.
nb_status load_order(nb_ctx* c, const double* r, bool* same = nullptr)
{
    const int64_t n = c->n;
    const std::vector<int64_t> off = c->ens ? c->h_off : std::vector<int64_t>{0, n};
    if (same) *same = false;
    if (c->order_pos.size() == static_cast<size_t>(3 * n) && c->order_off == off &&
        std::memcmp(c->order_pos.data(), r, 3 * n * sizeof(double)) == 0) {
        c->order_fresh = true;
        if (same) *same = true;
        return NB_OK;
    }
    c->h_perm = order_of(r, off);
    c->h_inv.assign(n, 0);
    for (int64_t k = 0; k < n; ++k) c->h_inv[c->h_perm[k]] = static_cast<int32_t>(k);
    c->host_order_stale = false;
    NB_CK(c, cudaMemcpyAsync(c->perm_dev, c->h_perm.data(), n * sizeof(int32_t),
                             cudaMemcpyHostToDevice, c->stream));
    NB_CK(c, cudaMemcpyAsync(c->inv_dev, c->h_inv.data(), n * sizeof(int32_t),
                             cudaMemcpyHostToDevice, c->stream));
    NB_CK(c, cudaStreamSynchronize(c->stream));  // the host vectors are copy sources
    c->order_pos.assign(r, r + 3 * n);
    c->order_off = off;
    c->order_fresh = true;
    return NB_OK;
}

// Re-order the stored particles to the spatial order of their current
// positions, when steps have moved them since the order was computed.
nb_status refresh_order(nb_ctx* c)
{
    if (c->order_fresh) return NB_OK;
    nb_status s = sync_host_order(c);
    if (s != NB_OK) return s;
    const int64_t n = c->n;
    std::vector<double> soa(3 * n), aos(3 * n);
    NB_CK(c, cudaMemcpyAsync(soa.data(), c->st.x, soa.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
    NB_CK(c, cudaStreamSynchronize(c->stream));
    for (int64_t k = 0; k < n; ++k)
        for (int d = 0; d < 3; ++d) aos[3 * static_cast<int64_t>(c->h_perm[k]) + d] = soa[d * n + k];
    const std::vector<int32_t> old_inv = c->h_inv;
    bool same = false;
    if ((s = load_order(c, aos.data(), &same)) != NB_OK) return s;
    if (same) return NB_OK;
    // new internal index k holds the particle that sat at old_inv[perm[k]]
    std::vector<int32_t> map(n);
    for (int64_t k = 0; k < n; ++k) map[k] = old_inv[c->h_perm[k]];
    if (!c->order_buf) NB_CK(c, cudaMalloc(&c->order_buf, (17 * n + 1) * sizeof(double)));
    NB_CK(c, cudaMemcpyAsync(c->idx_user, map.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice,
                             c->stream));
    NB_CK(c, nb::snapshot_launch(c->st, c->order_buf, true, c->stream));
    NB_CK(c, nb::reorder_state_launch(c->st, c->order_buf, c->idx_user, c->stream));
    NB_CK(c, cudaStreamSynchronize(c->stream));  // map is a copy source
    c->last_force_n_act = -1;
    return NB_OK;
}

// A caller's host list in internal indices, ascending (the order the select
// gives its own lists): sorted[k] = inv[idx[perm[k]]].
std::vector<int32_t> internal_sorted(const nb_ctx* c, int32_t n_act, const int32_t* idx,
                                     std::vector<int32_t>& perm)
{
    perm.resize(n_act);
    for (int32_t k = 0; k < n_act; ++k) perm[k] = k;
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) {
        return c->h_inv[idx[a]] < c->h_inv[idx[b]];
    });
    std::vector<int32_t> sorted(n_act);
    for (int32_t k = 0; k < n_act; ++k) sorted[k] = c->h_inv[idx[perm[k]]];
    return sorted;
}

nb_status validate_idx(nb_ctx* c, int32_t n_act, const int32_t* idx)
{
    for (int32_t k = 0; k < n_act; ++k)
        if (idx[k] < 0 || idx[k] >= c->n)
            return fail(c, NB_EINVAL, "idx[%d] = %d outside [0, %lld)", k, idx[k],
                        static_cast<long long>(c->n));
    return NB_OK;
}

nb_status block_step(nb_ctx* c, double t_end)
{
    const nb::ClusterDev* cl = c->ens ? &c->cl : nullptr;
    const unsigned long long* tkeys = c->ens ? c->cl.tkey : c->sd.tmin_bits;
    if (c->ens)
        NB_CK(c, nb::cluster_select_launch(c->st, c->cl, c->sd, t_end, c->stream));
    else
        NB_CK(c, nb::select_launch(c->st, c->sd, t_end, c->stream));
    NB_CK(c, nb::predict_launch(c->st, c->prec, c->jl, c->cfg.G, tkeys, 0.0, c->sd.n_act,
                                c->stream, cl));
    nb_status s = run_force_list(c, c->prec, c->jl, c->sd.idx, c->sd.n_act, -1, true);
    if (s != NB_OK) return s;
    nb::CorrectArgs ca;
    ca.idx = c->sd.idx;
    ca.n_act_dev = c->sd.n_act;
    ca.t_bits = tkeys;
    if (c->ens) {
        ca.cluster_of = c->cl.cluster_of;
        ca.cl_off = c->cl.off;
    }
    ca.acc1 = c->acc1;
    ca.jerk1 = c->jerk1;
    ca.eta = c->eta;
    ca.dt_max = c->cfg.dt_max;
    ca.dt_min = c->cfg.dt_min;
    ca.status = c->status_dev;
    ca.step_counter = c->ctr64;
    ca.inter_counter = c->ctr64 + 1;
    if (c->prec == Prec::FP64_H6)
        NB_CK(c, nb::correct6_launch(c->st, ca, c->snap1, c->stream));
    else
        NB_CK(c, nb::correct_launch(c->st, ca, c->stream));
    c->last_force_n_act = -1;
    c->order_fresh = false;  // the positions move
    return NB_OK;
}

// Capture GRAPH_STEPS block steps for t_end into c->step_graph.  Every node
// reads its block (t_next, n_act, idx) from device memory, so one graph
// serves every replay until t_end changes or the buffers are reallocated.
nb_status build_step_graph(nb_ctx* c, double t_end)
{
    drop_graph(c);
    NB_CK(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    nb_status s = NB_OK;
    for (int k = 0; k < GRAPH_STEPS && s == NB_OK; ++k) s = block_step(c, t_end);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
    if (s != NB_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (e != cudaSuccess) return fail(c, NB_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    const cudaError_t ei = cudaGraphInstantiate(&c->step_graph, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) {
        c->step_graph = nullptr;
        return fail(c, NB_ECUDA, "graph instantiate: %s", cudaGetErrorString(ei));
    }
    c->graph_t_end = t_end;
    return NB_OK;
}

// Bounds of the grid-aligned j-layout split, from the loaded positions and
// velocities (the corrector raises them from then on), a cleared far-field
// noise estimate, and the next-time keys of the loaded t, dt.
nb_status refresh_bounds(nb_ctx* c)
{
    // a fresh load has no far-field noise estimate yet
    NB_CK(c, cudaMemsetAsync(c->st.hq, 0, c->n * sizeof(double), c->stream));
    NB_CK(c, cudaMemsetAsync(c->st.bound, 0, 2 * sizeof(uint32_t), c->stream));
    NB_CK(c, nb::bounds_launch(c->st.x, c->st.v, 3 * c->n, c->st.bound, c->stream));
    NB_CK(c, nb::next_key_launch(c->st, c->stream));
    return NB_OK;
}

// Hybrid precision only, at a load with a fresh force evaluation: that
// evaluation ran every pair in double-single (the state had a = j = 0), so
// it left no far-field noise estimate, and the first block step would run
// unguarded (a DS a0 against an FP32-noisy a1).  One more evaluation with
// the new a, j and dt stores the estimate; its forces are discarded.
nb_status hybrid_noise_pass(nb_ctx* c, bool ensemble)
{
    if (!nb::is_hybrid(c->prec)) return NB_OK;
    NB_CK(c, nb::iota_launch(c->idx_user, c->n, c->n_act_user, c->stream));
    if (ensemble)
        return run_force_list(c, c->prec, c->jl, c->idx_user, c->n_act_user,
                              static_cast<int32_t>(c->n));
    return run_force(c, c->prec, c->jl, c->idx_user, c->n_act_user, static_cast<int32_t>(c->n));
}

// Sixth-order variant, at a load: every particle at time t with a, j in
// the state; its snap from a force pass with those accelerations (reading
// H3 of its oracle), crackle zero.
nb_status h6_start(nb_ctx* c, double t)
{
    NB_CK(c, cudaMemsetAsync(c->st.s, 0, 3 * c->n * sizeof(double), c->stream));
    NB_CK(c, cudaMemsetAsync(c->st.c, 0, 3 * c->n * sizeof(double), c->stream));
    NB_CK(c, nb::predict_launch(c->st, c->prec, c->jl, c->cfg.G, nullptr, t, nullptr, c->stream));
    NB_CK(c, nb::iota_launch(c->idx_user, c->n, c->n_act_user, c->stream));
    nb_status s = run_force(c, c->prec, c->jl, c->idx_user, c->n_act_user,
                            static_cast<int32_t>(c->n));
    if (s != NB_OK) return s;
    NB_CK(c, nb::init_snap_launch(c->st, c->snap1, c->stream));
    return NB_OK;
}

// Set-up shared by nb_set_particles / nb_set_state.
nb_status begin_load(nb_ctx* c, int64_t n, double eps, double eta)
{
    if (n < 1 || n > 0x7fffffffLL) return fail(c, NB_EINVAL, "n = %lld out of range", (long long)n);
    if (!(eps >= 0.0) || !std::isfinite(eps)) return fail(c, NB_EINVAL, "eps must be >= 0");
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(c, NB_EINVAL, "eta must be > 0");
    c->sticky = NB_OK;
    c->loaded = false;
    c->err.clear();
    drop_graph(c);
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return fail(c, NB_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    c->ens = false;
    c->j_part = 0;
    c->j_parts = 1;
    nb_status s = ensure_capacity(c, n, (n + nb::TJ - 1) / nb::TJ * nb::TJ, 0);
    if (s != NB_OK) return s;
    c->eps = eps;
    c->eta = eta;
    NB_CK(c, cudaMemsetAsync(c->status_dev, 0, sizeof(uint32_t), c->stream));
    NB_CK(c, cudaMemsetAsync(c->counters, 0, c->counter_words * sizeof(uint32_t), c->stream));
    c->last_force_n_act = -1;
    return NB_OK;
}

}  // namespace

extern "C" {

void nb_config_init(nb_config* cfg)
{
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->precision = NB_HYBRID;
    cfg->device = 0;
    cfg->G = 1.0;
    cfg->eta_start = 0.01;
    cfg->dt_max = 1.0 / 16.0;
    cfg->dt_min = std::ldexp(1.0, -40);
    cfg->stream = nullptr;
    cfg->i_per_thread = 0;
    cfg->ctas_per_sm = 0;
    cfg->autotune = 0;
    cfg->j_split = 0;
    cfg->wait_limit_cycles = 0;
}

nb_status nb_create(const nb_config* cfg, nb_ctx** out)
{
    if (!cfg || !out) return NB_EINVAL;
    *out = nullptr;
    if (cfg->precision < NB_FP64 || cfg->precision > NB_FP64_HERMITE6) return NB_EINVAL;
    if (cfg->j_split != 0 && cfg->j_split != 1 && cfg->j_split != 2 && cfg->j_split != 4 &&
        cfg->j_split != 8)
        return NB_EINVAL;
    if (!is_pow2(cfg->dt_max) || !(cfg->dt_min > 0.0) || cfg->dt_min > cfg->dt_max) return NB_EINVAL;
    if (!(cfg->eta_start > 0.0) || !std::isfinite(cfg->G)) return NB_EINVAL;
    nb_ctx* c = new (std::nothrow) nb_ctx;
    if (!c) return NB_ENOMEM;
    c->cfg = *cfg;
    c->prec = static_cast<Prec>(cfg->precision);
    c->ens_chunks = ens_chunks_default(c->prec);
    c->device = cfg->device;
    auto bail = [&](nb_status s) {
        nb_destroy(c);
        return s;
    };
    if (cudaSetDevice(c->device) != cudaSuccess) return bail(NB_ECUDA);
    if (cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess)
        return bail(NB_ECUDA);
    if (cfg->stream) {
        c->stream = static_cast<cudaStream_t>(cfg->stream);
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess)
            return bail(NB_ECUDA);
        c->own_stream = true;
    }
    if (cudaStreamCreateWithFlags(&c->aux, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return bail(NB_ECUDA);
    // Default launch shapes (measured on GB300 for N = 16384): one i per
    // thread for small blocks, two for large MIXED blocks; at most 4
    // persistent CTAs per SM.  nb_autotune replaces them by measurement.
    for (int v = 0; v < 2; ++v) {
        const int split = cfg->j_split > 0 ? cfg->j_split : 1;
        int it = cfg->i_per_thread;
        if (it == 0) it = (v == 1 && nb::is_mixed(c->prec) && split == 1) ? 2 : 1;
        if (!nb::force_variant_exists(c->prec, it, split)) return bail(NB_EINVAL);
        if (nb::force_setup(c->prec, it, split) != cudaSuccess) return bail(NB_ECUDA);
        const int occ = nb::force_ctas_per_sm(c->prec, it, split);
        if (occ < 1) return bail(NB_ECUDA);
        const int per_sm = cfg->ctas_per_sm > 0 ? cfg->ctas_per_sm : std::min(occ, 4);
        c->var[v].it = it;
        c->var[v].split = split;
        c->var[v].grid = per_sm * c->num_sms;
    }
    c->var[2] = c->var[0];  // no tiny variant until nb_autotune or nb_set_tuning sets one
    if (nb::force_setup(Prec::FP64, 1, 1) != cudaSuccess) return bail(NB_ECUDA);
    const int per_sm64 = nb::force_ctas_per_sm(Prec::FP64, 1, 1);
    if (per_sm64 < 1) return bail(NB_ECUDA);
    c->grid64 = per_sm64 * c->num_sms;
    if (cudaMalloc(&c->status_dev, sizeof(uint32_t)) != cudaSuccess) return bail(NB_ENOMEM);
    if (cudaMemset(c->status_dev, 0, sizeof(uint32_t)) != cudaSuccess) return bail(NB_ECUDA);
    if (cudaMalloc(&c->st.bound, 2 * sizeof(uint32_t)) != cudaSuccess) return bail(NB_ENOMEM);
    if (cudaMemset(c->st.bound, 0, 2 * sizeof(uint32_t)) != cudaSuccess) return bail(NB_ECUDA);
    if (cudaMalloc(&c->ctr64, 2 * sizeof(unsigned long long)) != cudaSuccess) return bail(NB_ENOMEM);
    if (cudaMemset(c->ctr64, 0, 2 * sizeof(unsigned long long)) != cudaSuccess) return bail(NB_ECUDA);
    if (cudaMallocHost(&c->pinned, PINNED_BYTES) != cudaSuccess) return bail(NB_ENOMEM);
    *out = c;
    return NB_OK;
}

nb_status nb_destroy(nb_ctx* c)
{
    if (!c) return NB_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graph(c);
    free_buffers(c);
    if (c->status_dev) cudaFree(c->status_dev);
    if (c->st.bound) cudaFree(c->st.bound);
    if (c->ctr64) cudaFree(c->ctr64);
    if (c->pinned) cudaFreeHost(c->pinned);
    if (c->aux) cudaStreamSynchronize(c->aux), cudaStreamDestroy(c->aux);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return NB_OK;
}

nb_status nb_set_particles(nb_ctx* c, int64_t n, const double* m, const double* r,
                           const double* v, double eps, double eta)
{
    if (!c) return NB_EINVAL;
    if (!m || !r || !v) return fail(c, NB_EINVAL, "NULL array");
    nb_status s = begin_load(c, n, eps, eta);
    if (s != NB_OK) return s;
    if ((s = load_order(c, r)) != NB_OK) return s;
    if ((s = upload_perm(c, m, c->st.m, 1, 0)) != NB_OK) return s;
    if ((s = upload_vec3(c, r, c->st.x, 0)) != NB_OK) return s;
    if ((s = upload_vec3(c, v, c->st.v, 0)) != NB_OK) return s;
    NB_CK(c, cudaMemsetAsync(c->st.a, 0, 3 * n * sizeof(double), c->stream));
    NB_CK(c, cudaMemsetAsync(c->st.j, 0, 3 * n * sizeof(double), c->stream));
    NB_CK(c, cudaMemsetAsync(c->st.t, 0, n * sizeof(double), c->stream));
    if (c->prec == Prec::FP64_H6) {
        NB_CK(c, cudaMemsetAsync(c->st.s, 0, 3 * n * sizeof(double), c->stream));
        NB_CK(c, cudaMemsetAsync(c->st.c, 0, 3 * n * sizeof(double), c->stream));
    }
    if ((s = refresh_bounds(c)) != NB_OK) return s;
    // Forces on every particle at t = 0, then the first timesteps.
    NB_CK(c, nb::predict_launch(c->st, c->prec, c->jl, c->cfg.G, nullptr, 0.0, nullptr, c->stream));
    NB_CK(c, nb::iota_launch(c->idx_user, n, c->n_act_user, c->stream));
    if ((s = run_force(c, c->prec, c->jl, c->idx_user, c->n_act_user, static_cast<int32_t>(n))) !=
        NB_OK)
        return s;
    NB_CK(c, nb::init_dt_launch(c->st, c->acc1, c->jerk1, c->cfg.eta_start, c->cfg.dt_max,
                                c->cfg.dt_min, 0.0, c->status_dev, c->stream));
    if (c->prec == Prec::FP64_H6 && (s = h6_start(c, 0.0)) != NB_OK) return s;
    if ((s = hybrid_noise_pass(c, false)) != NB_OK) return s;
    if ((s = check_status(c)) != NB_OK) return s;
    c->loaded = true;
    if (c->cfg.autotune) return nb_autotune(c, nullptr);
    return NB_OK;
}

nb_status nb_set_state(nb_ctx* c, int64_t n, const double* m, const double* r, const double* v,
                       const double* a, const double* j, const double* t, const double* dt,
                       double eps, double eta, int32_t on_device)
{
    if (!c) return NB_EINVAL;
    if (!m || !r || !v || !a || !j || !t || !dt) return fail(c, NB_EINVAL, "NULL array");
    nb_status s = begin_load(c, n, eps, eta);
    if (s != NB_OK) return s;
    if (on_device) {
        // the order is computed on the host from the positions
        std::vector<double> hr(3 * n);
        NB_CK(c, cudaMemcpyAsync(hr.data(), r, hr.size() * sizeof(double),
                                 cudaMemcpyDeviceToHost, c->stream));
        NB_CK(c, cudaStreamSynchronize(c->stream));
        if ((s = load_order(c, hr.data())) != NB_OK) return s;
    } else if ((s = load_order(c, r)) != NB_OK) {
        return s;
    }
    if ((s = upload_perm(c, m, c->st.m, 1, on_device)) != NB_OK) return s;
    if ((s = upload_vec3(c, r, c->st.x, on_device)) != NB_OK) return s;
    if ((s = upload_vec3(c, v, c->st.v, on_device)) != NB_OK) return s;
    if ((s = upload_vec3(c, a, c->st.a, on_device)) != NB_OK) return s;
    if ((s = upload_vec3(c, j, c->st.j, on_device)) != NB_OK) return s;
    if ((s = upload_perm(c, t, c->st.t, 1, on_device)) != NB_OK) return s;
    if ((s = upload_perm(c, dt, c->st.dt, 1, on_device)) != NB_OK) return s;
    if ((s = refresh_bounds(c)) != NB_OK) return s;
    if (c->prec == Prec::FP64_H6) {
        // the snap needs every particle at one time
        std::vector<double> ht(n);
        NB_CK(c, cudaMemcpyAsync(ht.data(), c->st.t, n * sizeof(double), cudaMemcpyDeviceToHost,
                                 c->stream));
        NB_CK(c, cudaStreamSynchronize(c->stream));
        for (int64_t q = 1; q < n; ++q)
            if (ht[q] != ht[0])
                return fail(c, NB_EINVAL, "the sixth-order variant loads synchronised states only");
        if ((s = h6_start(c, ht[0])) != NB_OK) return s;
        if ((s = check_status(c)) != NB_OK) return s;
    }
    if (!on_device) NB_CK(c, cudaStreamSynchronize(c->stream));
    c->loaded = true;
    return NB_OK;
}

int64_t nb_snapshot_bytes(const nb_ctx* c)
{
    if (!c || !c->loaded) return 0;
    // the state (17 n words and the bounds), then the order (perm, inv)
    return (18 * c->n + 1) * static_cast<int64_t>(sizeof(double));
}

nb_status nb_snapshot(nb_ctx* c, void* buf)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    if (c->prec == Prec::FP64_H6)
        return fail(c, NB_ESTATE, "no snapshots of the sixth-order variant (its snap and "
                                  "crackle are not in the snapshot layout)");
    if (!buf || (reinterpret_cast<uintptr_t>(buf) & 15u)) return fail(c, NB_EINVAL, "buf NULL or not 16-byte aligned");
    double* b = static_cast<double*>(buf);
    NB_CK(c, nb::snapshot_launch(c->st, b, true, c->stream));
    int32_t* ord = reinterpret_cast<int32_t*>(b + 17 * c->n + 1);
    NB_CK(c, cudaMemcpyAsync(ord, c->perm_dev, c->n * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                             c->stream));
    NB_CK(c, cudaMemcpyAsync(ord + c->n, c->inv_dev, c->n * sizeof(int32_t),
                             cudaMemcpyDeviceToDevice, c->stream));
    return NB_OK;
}

nb_status nb_restore(nb_ctx* c, const void* buf)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    if (c->prec == Prec::FP64_H6)
        return fail(c, NB_ESTATE, "no snapshots of the sixth-order variant (its snap and "
                                  "crackle are not in the snapshot layout)");
    if (!buf || (reinterpret_cast<uintptr_t>(buf) & 15u)) return fail(c, NB_EINVAL, "buf NULL or not 16-byte aligned");
    double* b = static_cast<double*>(const_cast<void*>(buf));
    NB_CK(c, nb::snapshot_launch(c->st, b, false, c->stream));
    const int32_t* ord = reinterpret_cast<const int32_t*>(b + 17 * c->n + 1);
    NB_CK(c, cudaMemcpyAsync(c->perm_dev, ord, c->n * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                             c->stream));
    NB_CK(c, cudaMemcpyAsync(c->inv_dev, ord + c->n, c->n * sizeof(int32_t),
                             cudaMemcpyDeviceToDevice, c->stream));
    // the host copies of the order follow the device ones when next needed
    c->host_order_stale = true;
    c->order_pos.clear();
    c->order_fresh = false;
    return NB_OK;
}

nb_status nb_get_snap(nb_ctx* c, double* sn, double* cr, int32_t on_device)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    if (c->prec != Prec::FP64_H6) return fail(c, NB_ESTATE, "no snap in this precision");
    double* src[2] = {c->st.s, c->st.c};
    double* dst[2] = {sn, cr};
    for (int q = 0; q < 2; ++q) {
        if (!dst[q]) continue;
        if ((s = download_perm(c, src[q], dst[q], 3, on_device)) != NB_OK) return s;
        if (!on_device) NB_CK(c, cudaStreamSynchronize(c->stream));
    }
    return NB_OK;
}

nb_status nb_get_state(nb_ctx* c, double* r, double* v, double* a, double* j, double* t,
                       double* dt, int32_t on_device)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    double* src[6] = {c->st.x, c->st.v, c->st.a, c->st.j, c->st.t, c->st.dt};
    double* dst[6] = {r, v, a, j, t, dt};
    for (int q = 0; q < 6; ++q) {
        if (!dst[q]) continue;
        if ((s = download_perm(c, src[q], dst[q], q < 4 ? 3 : 1, on_device)) != NB_OK) return s;
        // (one staging buffer: each host copy completes before the next)
        if (!on_device) NB_CK(c, cudaStreamSynchronize(c->stream));
    }
    return NB_OK;
}

nb_status nb_predict(nb_ctx* c, double t)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    if (!std::isfinite(t)) return fail(c, NB_EINVAL, "t not finite");
    NB_CK(c, nb::predict_launch(c->st, c->prec, c->jl, c->cfg.G, nullptr, t, nullptr, c->stream,
                                c->ens ? &c->cl : nullptr));
    return NB_OK;
}

nb_status nb_select(nb_ctx* c, double t_end, double* t_next, int32_t* n_act, int32_t* idx)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    unsigned long long* hk = reinterpret_cast<unsigned long long*>(c->pinned + 16);
    int32_t* hn = reinterpret_cast<int32_t*>(c->pinned + 24);
    if (c->ens) {
        NB_CK(c, nb::cluster_select_launch(c->st, c->cl, c->sd, t_end, c->stream));
        std::vector<unsigned long long> keys(c->cl.k);
        NB_CK(c, cudaMemcpyAsync(keys.data(), c->cl.tkey, keys.size() * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, c->stream));
        NB_CK(c, cudaMemcpyAsync(hn, c->sd.n_act, sizeof(*hn), cudaMemcpyDeviceToHost, c->stream));
        NB_CK(c, cudaStreamSynchronize(c->stream));
        *hk = *std::min_element(keys.begin(), keys.end());  // keys order like times
    } else {
        NB_CK(c, nb::select_launch(c->st, c->sd, t_end, c->stream));
        NB_CK(c, cudaMemcpyAsync(hk, c->sd.tmin_bits, sizeof(*hk), cudaMemcpyDeviceToHost, c->stream));
        NB_CK(c, cudaMemcpyAsync(hn, c->sd.n_act, sizeof(*hn), cudaMemcpyDeviceToHost, c->stream));
        NB_CK(c, cudaStreamSynchronize(c->stream));
    }
    if (t_next) *t_next = nb::time_from_key(*hk);
    if (n_act) *n_act = *hn;
    if (idx && *hn > 0) {
        if ((s = sync_host_order(c)) != NB_OK) return s;
        NB_CK(c, cudaMemcpyAsync(idx, c->sd.idx, (size_t)*hn * sizeof(int32_t),
                                 cudaMemcpyDeviceToHost, c->stream));
        NB_CK(c, cudaStreamSynchronize(c->stream));
        // internal indices to the caller's, reported ascending
        for (int32_t k = 0; k < *hn; ++k) idx[k] = c->h_perm[idx[k]];
        std::sort(idx, idx + *hn);
    }
    return NB_OK;
}

nb_status nb_force(nb_ctx* c, int32_t n_act, const int32_t* idx, double* acc, double* jerk,
                   double* pot, int32_t on_device)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    if (n_act < 0 || n_act > c->n) return fail(c, NB_EINVAL, "n_act = %d out of range", n_act);
    if (n_act > 0 && !idx) return fail(c, NB_EINVAL, "NULL idx");
    if (!on_device && n_act > 0 && (s = validate_idx(c, n_act, idx)) != NB_OK) return s;
    if (c->ens && !on_device)
        for (int32_t k = 1; k < n_act; ++k)
            if (idx[k] <= idx[k - 1])
                return fail(c, NB_EINVAL, "ensemble force needs idx strictly ascending");
    std::vector<int32_t> perm;  // host list: entry k of the internal list is idx[perm[k]]
    if (n_act > 0 && !on_device) {
        if ((s = sync_host_order(c)) != NB_OK) return s;
        const std::vector<int32_t> sorted = internal_sorted(c, n_act, idx, perm);
        NB_CK(c, cudaMemcpyAsync(c->idx_user, sorted.data(), (size_t)n_act * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, c->stream));
        NB_CK(c, cudaStreamSynchronize(c->stream));  // sorted is a copy source
    } else if (n_act > 0 && c->ens) {
        NB_CK(c, nb::map_index_launch(idx, c->idx_user, n_act, c->n, c->inv_dev, c->stream));
    }
    if (c->ens) {
        // the ensemble plan reads the block size on the device
        NB_CK(c, nb::set_scalars_launch(c->n_act_user, n_act, nullptr, 0.0, c->stream));
        if (n_act > 0 &&
            (s = run_force_list(c, c->prec, c->jl, c->idx_user, c->n_act_user, n_act)) != NB_OK)
            return s;
    } else if (n_act > 0) {
        // one launch: n_act as a parameter, and a device list in the caller's
        // numbering mapped to layout slots by the kernel itself
        if ((s = run_force(c, c->prec, c->jl, on_device ? idx : c->idx_user, c->n_act_user,
                           n_act, on_device ? c->inv_dev : nullptr)) != NB_OK)
            return s;
    }
    c->last_force_n_act = n_act;
    if (n_act > 0 && on_device) {
        const cudaMemcpyKind k = cudaMemcpyDeviceToDevice;
        if (acc) NB_CK(c, cudaMemcpyAsync(acc, c->acc1, 3 * (size_t)n_act * sizeof(double), k, c->stream));
        if (jerk) NB_CK(c, cudaMemcpyAsync(jerk, c->jerk1, 3 * (size_t)n_act * sizeof(double), k, c->stream));
        if (pot) NB_CK(c, cudaMemcpyAsync(pot, c->pot1, (size_t)n_act * sizeof(double), k, c->stream));
    }
    if (on_device || n_act == 0) return on_device ? NB_OK : check_status(c);
    // rows of the internal (ascending) list back to the caller's order
    std::vector<double> h(7 * (size_t)n_act);
    const auto d2h = cudaMemcpyDeviceToHost;
    NB_CK(c, cudaMemcpyAsync(h.data(), c->acc1, 3 * (size_t)n_act * sizeof(double), d2h, c->stream));
    NB_CK(c, cudaMemcpyAsync(h.data() + 3 * (size_t)n_act, c->jerk1,
                             3 * (size_t)n_act * sizeof(double), d2h, c->stream));
    NB_CK(c, cudaMemcpyAsync(h.data() + 6 * (size_t)n_act, c->pot1, (size_t)n_act * sizeof(double),
                             d2h, c->stream));
    if ((s = check_status(c)) != NB_OK) return s;
    for (int32_t k = 0; k < n_act; ++k) {
        const size_t u = static_cast<size_t>(perm[k]);
        for (int d = 0; d < 3; ++d) {
            if (acc) acc[3 * u + d] = h[3 * (size_t)k + d];
            if (jerk) jerk[3 * u + d] = h[3 * ((size_t)n_act + k) + d];
        }
        if (pot) pot[u] = h[6 * (size_t)n_act + k];
    }
    return NB_OK;
}

nb_status nb_correct(nb_ctx* c, double t, int32_t n_act, const int32_t* idx, const double* acc,
                     const double* jerk, int32_t on_device)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    if (c->ens)
        return fail(c, NB_ESTATE, "nb_correct works on one system; an ensemble advances with "
                                  "nb_block_step or nb_step_until");
    if (n_act < 0 || n_act > c->n) return fail(c, NB_EINVAL, "n_act = %d out of range", n_act);
    if (!std::isfinite(t)) return fail(c, NB_EINVAL, "t not finite");
    if (n_act > 0 && !idx) return fail(c, NB_EINVAL, "NULL idx");
    if ((acc == nullptr) != (jerk == nullptr)) return fail(c, NB_EINVAL, "give both acc and jerk or neither");
    if (acc && c->prec == Prec::FP64_H6)
        return fail(c, NB_EINVAL, "the sixth-order variant corrects with the last nb_force "
                                  "results (acc = jerk = NULL), which hold the snap");
    if (!acc && n_act != c->last_force_n_act)
        return fail(c, NB_ESTATE, "no nb_force result for a block of %d particles", n_act);
    if (n_act == 0) return NB_OK;
    if (!on_device && (s = validate_idx(c, n_act, idx)) != NB_OK) return s;
    const int32_t* idx_dev = c->idx_user;
    const double* a1 = acc ? acc : c->acc1;
    const double* j1 = jerk ? jerk : c->jerk1;
    std::vector<int32_t> list, perm;
    if (on_device) {
        NB_CK(c, nb::map_index_launch(idx, c->idx_user, n_act, c->n, c->inv_dev, c->stream));
    } else {
        // internal indices; without acc / jerk the last nb_force rows are used,
        // which follow the ascending internal order nb_force gave a host list
        if ((s = sync_host_order(c)) != NB_OK) return s;
        if (acc) {
            list.resize(n_act);
            for (int32_t k = 0; k < n_act; ++k) list[k] = c->h_inv[idx[k]];
        } else {
            list = internal_sorted(c, n_act, idx, perm);
        }
        NB_CK(c, cudaMemcpyAsync(c->idx_user, list.data(), (size_t)n_act * sizeof(int32_t),
                                 cudaMemcpyHostToDevice, c->stream));
        if (acc) {
            NB_CK(c, cudaMemcpyAsync(c->acc1, acc, 3 * (size_t)n_act * sizeof(double),
                                     cudaMemcpyHostToDevice, c->stream));
            NB_CK(c, cudaMemcpyAsync(c->jerk1, jerk, 3 * (size_t)n_act * sizeof(double),
                                     cudaMemcpyHostToDevice, c->stream));
            a1 = c->acc1;
            j1 = c->jerk1;
        }
    }
    NB_CK(c, nb::set_scalars_launch(c->n_act_user, n_act, c->sd.tmin_bits, t, c->stream));
    nb::CorrectArgs ca;
    ca.idx = idx_dev;
    ca.n_act_dev = c->n_act_user;
    ca.t_bits = c->sd.tmin_bits;
    ca.acc1 = a1;
    ca.jerk1 = j1;
    ca.eta = c->eta;
    ca.dt_max = c->cfg.dt_max;
    ca.dt_min = c->cfg.dt_min;
    ca.status = c->status_dev;
    if (c->prec == Prec::FP64_H6)
        NB_CK(c, nb::correct6_launch(c->st, ca, c->snap1, c->stream));
    else
        NB_CK(c, nb::correct_launch(c->st, ca, c->stream));
    c->last_force_n_act = -1;
    c->order_fresh = false;  // the positions move
    if (!on_device) return check_status(c);  // (also keeps list alive until the copy ran)
    return NB_OK;
}

nb_status nb_block_step(nb_ctx* c, double t_end)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    return block_step(c, t_end);
}

nb_status nb_step_until(nb_ctx* c, double t_end, uint64_t* n_steps, uint64_t* n_interactions)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    if (!std::isfinite(t_end)) return fail(c, NB_EINVAL, "t_end not finite");
    // the stored order from the current positions (a function of them, so a
    // run resumed from a checkpoint gets the order the original had)
    if ((s = refresh_order(c)) != NB_OK) return s;
    NB_CK(c, cudaMemsetAsync(c->ctr64, 0, 2 * sizeof(unsigned long long), c->stream));
    if (!c->step_graph || c->graph_t_end != t_end) {
        if ((s = build_step_graph(c, t_end)) != NB_OK) return s;
    }
    int32_t* hn = reinterpret_cast<int32_t*>(c->pinned + 24);
    uint32_t* hs = reinterpret_cast<uint32_t*>(c->pinned + 28);
    // Replay GRAPH_STEPS block steps at a time; once t_next passes t_end the
    // remaining steps of a replay are empty.  One host round trip per replay.
    for (;;) {
        NB_CK(c, cudaGraphLaunch(c->step_graph, c->stream));
        NB_CK(c, cudaMemcpyAsync(hn, c->sd.n_act, sizeof(int32_t), cudaMemcpyDeviceToHost, c->stream));
        NB_CK(c, cudaMemcpyAsync(hs, c->status_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
        NB_CK(c, cudaStreamSynchronize(c->stream));
        if (*hs != 0) return check_status(c);
        if (*hn == 0) break;
    }
    unsigned long long* hc = reinterpret_cast<unsigned long long*>(c->pinned + 32);
    NB_CK(c, cudaMemcpyAsync(hc, c->ctr64, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    NB_CK(c, cudaStreamSynchronize(c->stream));
    if (n_steps) *n_steps = hc[0];
    if (n_interactions) *n_interactions = hc[1];
    return NB_OK;
}

nb_status nb_energy(nb_ctx* c, int32_t fp64_potential, double* kin, double* pot)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    const bool use64 = fp64_potential || c->prec == Prec::FP64;
    const Prec p = use64 ? Prec::FP64 : c->prec;
    nb::JLayout& jl = (p == c->prec) ? c->jl : c->jl64;
    // Predict every particle to its own time (all t_i are equal at a
    // synchronised time, so this is the identity there).
    double* ht = reinterpret_cast<double*>(c->pinned + 48);
    NB_CK(c, cudaMemcpyAsync(ht, c->st.t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    NB_CK(c, cudaStreamSynchronize(c->stream));
    NB_CK(c, nb::predict_launch(c->st, p, jl, c->cfg.G, nullptr, *ht, nullptr, c->stream,
                                c->ens ? &c->cl : nullptr));
    NB_CK(c, nb::iota_launch(c->idx_user, c->n, c->n_act_user, c->stream));
    // the energy needs the whole potential: no j partition here
    const int32_t parts = c->j_parts;
    c->j_parts = 1;
    s = run_force_list(c, p, jl, c->idx_user, c->n_act_user, static_cast<int32_t>(c->n));
    c->j_parts = parts;
    if (s != NB_OK) return s;
    NB_CK(c, nb::energy_launch(c->st, c->pot1, c->energy_partials, c->energy_blocks,
                               c->energy_out, c->energy_ticket, c->stream));
    if (c->ens)
        NB_CK(c, nb::cluster_energy_launch(c->st, c->cl, c->pot1, c->cl_energy, c->stream));
    double* he = reinterpret_cast<double*>(c->pinned + 64);
    NB_CK(c, cudaMemcpyAsync(he, c->energy_out, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    if ((s = check_status(c)) != NB_OK) return s;
    if (kin) *kin = he[0];
    if (pot) *pot = he[1];
    c->last_force_n_act = -1;
    return NB_OK;
}

nb_status nb_synchronize(nb_ctx* c)
{
    nb_status s = enter(c, false);
    if (s != NB_OK) return s;
    NB_CK(c, cudaStreamSynchronize(c->stream));
    if (c->loaded) return check_status(c);
    return NB_OK;
}

nb_status nb_set_ensemble(nb_ctx* c, int32_t k, const int64_t* offsets, const double* m,
                          const double* r, const double* v, const double* eps, double eta)
{
    if (!c) return NB_EINVAL;
    if (k < 1 || !offsets || !m || !r || !v || !eps)
        return fail(c, NB_EINVAL, "need k >= 1 and non-NULL arrays");
    if (c->prec == Prec::FP64_H6)
        return fail(c, NB_EINVAL, "the sixth-order variant integrates one system");
    if (offsets[0] != 0) return fail(c, NB_EINVAL, "offsets[0] must be 0");
    for (int32_t q = 0; q < k; ++q) {
        if (offsets[q + 1] <= offsets[q])
            return fail(c, NB_EINVAL, "system %d is empty or offsets not increasing", q);
        if (!(eps[q] >= 0.0) || !std::isfinite(eps[q]))
            return fail(c, NB_EINVAL, "eps[%d] must be finite and >= 0", q);
    }
    const int64_t n = offsets[k];
    if (n > 0x7fffffffLL) return fail(c, NB_EINVAL, "too many particles");
    if (!(eta > 0.0) || !std::isfinite(eta)) return fail(c, NB_EINVAL, "eta must be > 0");
    c->sticky = NB_OK;
    c->loaded = false;
    c->err.clear();
    drop_graph(c);
    if (cudaSetDevice(c->device) != cudaSuccess) return fail(c, NB_ECUDA, "cudaSetDevice");
    // j layout: each system's particles, then ghosts up to a whole tile
    std::vector<int64_t> joff(k + 1, 0);
    for (int32_t q = 0; q < k; ++q)
        joff[q + 1] = joff[q] + (offsets[q + 1] - offsets[q] + nb::TJ - 1) / nb::TJ * nb::TJ;
    const int64_t n_pad = joff[k];
    std::vector<int32_t> cluster_of(n), jsrc(n_pad, -1);
    std::vector<double> eps2(k);
    for (int32_t q = 0; q < k; ++q) {
        eps2[q] = eps[q] * eps[q];
        for (int64_t i = offsets[q]; i < offsets[q + 1]; ++i) {
            cluster_of[i] = q;
            jsrc[joff[q] + (i - offsets[q])] = static_cast<int32_t>(i);
        }
    }
    c->ens = true;
    c->j_part = 0;
    c->j_parts = 1;
    nb_status s = ensure_capacity(c, n, n_pad, k);
    if (s != NB_OK) return s;
    // the ensemble plan cuts i-groups of one width for both variants, and
    // there is no tiny one
    c->tiny_split = 0;
    c->var[2] = c->var[0];
    if (c->var[1].it != c->var[0].it || c->var[1].split != c->var[0].split) {
        c->var[1].it = c->var[0].it;
        c->var[1].split = c->var[0].split;
        if ((s = ensure_force_scratch(c)) != NB_OK) return s;
    }
    c->eps = 0.0;  // per system: cl.eps2
    c->eta = eta;
    c->h_off.assign(offsets, offsets + k + 1);
    const auto h2d = cudaMemcpyHostToDevice;
    NB_CK(c, cudaMemcpyAsync(c->cl.off, offsets, (k + 1) * sizeof(int64_t), h2d, c->stream));
    NB_CK(c, cudaMemcpyAsync(c->cl.joff, joff.data(), (k + 1) * sizeof(int64_t), h2d, c->stream));
    NB_CK(c, cudaMemcpyAsync(c->cl.eps2, eps2.data(), k * sizeof(double), h2d, c->stream));
    NB_CK(c, cudaMemcpyAsync(c->cl.cluster_of, cluster_of.data(), n * sizeof(int32_t), h2d, c->stream));
    NB_CK(c, cudaMemcpyAsync(c->cl.jsrc, jsrc.data(), n_pad * sizeof(int32_t), h2d, c->stream));
    NB_CK(c, cudaMemsetAsync(c->status_dev, 0, sizeof(uint32_t), c->stream));
    NB_CK(c, cudaMemsetAsync(c->counters, 0, c->counter_words * sizeof(uint32_t), c->stream));
    if ((s = load_order(c, r)) != NB_OK) return s;
    if ((s = upload_perm(c, m, c->st.m, 1, 0)) != NB_OK) return s;
    if ((s = upload_vec3(c, r, c->st.x, 0)) != NB_OK) return s;
    if ((s = upload_vec3(c, v, c->st.v, 0)) != NB_OK) return s;
    NB_CK(c, cudaMemsetAsync(c->st.a, 0, 3 * n * sizeof(double), c->stream));
    NB_CK(c, cudaMemsetAsync(c->st.j, 0, 3 * n * sizeof(double), c->stream));
    NB_CK(c, cudaMemsetAsync(c->st.t, 0, n * sizeof(double), c->stream));
    if ((s = refresh_bounds(c)) != NB_OK) return s;
    // forces on every particle of every system at t = 0, first timesteps
    NB_CK(c, nb::predict_launch(c->st, c->prec, c->jl, c->cfg.G, nullptr, 0.0, nullptr, c->stream,
                                &c->cl));
    NB_CK(c, nb::iota_launch(c->idx_user, n, c->n_act_user, c->stream));
    if ((s = run_force_list(c, c->prec, c->jl, c->idx_user, c->n_act_user,
                            static_cast<int32_t>(n))) != NB_OK)
        return s;
    NB_CK(c, nb::init_dt_launch(c->st, c->acc1, c->jerk1, c->cfg.eta_start, c->cfg.dt_max,
                                c->cfg.dt_min, 0.0, c->status_dev, c->stream));
    if ((s = hybrid_noise_pass(c, true)) != NB_OK) return s;
    if ((s = check_status(c)) != NB_OK) return s;
    c->last_force_n_act = -1;
    c->loaded = true;
    if (c->cfg.autotune) return nb_autotune(c, nullptr);
    return NB_OK;
}

nb_status nb_energy_systems(nb_ctx* c, int32_t fp64_potential, double* kin, double* pot)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    if (!c->ens) {
        double K = 0.0, W = 0.0;
        if ((s = nb_energy(c, fp64_potential, &K, &W)) != NB_OK) return s;
        if (kin) kin[0] = K;
        if (pot) pot[0] = W;
        return NB_OK;
    }
    if ((s = nb_energy(c, fp64_potential, nullptr, nullptr)) != NB_OK) return s;
    std::vector<double> h(2 * c->cl.k);
    NB_CK(c, cudaMemcpyAsync(h.data(), c->cl_energy, h.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, c->stream));
    NB_CK(c, cudaStreamSynchronize(c->stream));
    for (int q = 0; q < c->cl.k; ++q) {
        if (kin) kin[q] = h[2 * q];
        if (pot) pot[q] = h[2 * q + 1];
    }
    return NB_OK;
}

int32_t nb_num_systems(const nb_ctx* c) { return c && c->loaded ? (c->ens ? c->cl.k : 1) : 0; }

nb_status nb_selftest_timeout(nb_ctx* c)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    uint32_t* h = reinterpret_cast<uint32_t*>(c->pinned);
    NB_CK(c, cudaMemsetAsync(c->status_dev, 0, sizeof(uint32_t), c->stream));
    NB_CK(c, nb::iota_launch(c->idx_user, c->n, c->n_act_user, c->stream));
    if (c->ens)
        NB_CK(c, nb::plan_launch(c->cl, c->idx_user, c->n_act_user,
                                 32 * c->var[0].it / c->var[0].split, c->stream));
    nb::ForceArgs f = force_args(c, c->prec, c->jl, c->idx_user, c->n_act_user);
    f.it = c->var[0].it;
    f.split = c->var[0].split;
    f.grid = c->var[0].grid;
    f.wait_limit = 200000;  // ~0.1 ms per warp
    f.unfed_first_tile = 1;
    NB_CK(c, nb::force_launch(f, c->stream));
    NB_CK(c, cudaMemcpyAsync(h, c->status_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
    NB_CK(c, cudaStreamSynchronize(c->stream));
    const uint32_t st = *h;
    // leave the context as it was: clean status and reduction counters
    NB_CK(c, cudaMemsetAsync(c->status_dev, 0, sizeof(uint32_t), c->stream));
    NB_CK(c, cudaMemsetAsync(c->counters, 0, c->counter_words * sizeof(uint32_t), c->stream));
    NB_CK(c, cudaStreamSynchronize(c->stream));
    c->last_force_n_act = -1;
    return (st & nb::ST_TIMEOUT) ? NB_ETIMEOUT : NB_OK;
}

nb_status nb_autotune(nb_ctx* c, nb_tuning* out)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    const int64_t n = c->n;
    // probes 0-3 are timed with the small-block build, 3-4 with the large one
    constexpr int NQ = 5;
    const int32_t probes[NQ] = {static_cast<int32_t>(std::min<int64_t>(32, n)),
                                static_cast<int32_t>(std::min<int64_t>(96, n)),
                                static_cast<int32_t>(std::min<int64_t>(256, n)),
                                static_cast<int32_t>(std::min<int64_t>(2048, n)),
                                static_cast<int32_t>(std::min<int64_t>(65536, n))};
    // candidates: (i per thread, j split) x CTAs per SM; two i per thread
    // only for MIXED and HYBRID single systems, and only without a j split
    std::vector<std::pair<int, int>> shapes = {{1, 1}, {1, 2}, {1, 4}, {1, 8}};
    if ((nb::is_mixed(c->prec) || nb::is_hybrid(c->prec)) && !c->ens) shapes.push_back({2, 1});
    struct Cand {
        int it, split, cps;
        double us[NQ];   // with the small-block build (probes 0-3)
        double usl[NQ];  // with the large-block build (probes 3-4)
    };
    std::vector<Cand> cands;
    int max_grid = 0;
    for (const auto& sh : shapes) {
        if (nb::force_setup(c->prec, sh.first, sh.second) != cudaSuccess)
            return fail(c, NB_ECUDA, "autotune: kernel attributes");
        const int occ = nb::force_ctas_per_sm(c->prec, sh.first, sh.second);
        for (int cps : {1, 2, 3, 4, 5, 6, 8})
            if (cps <= occ) {
                cands.push_back({sh.first, sh.second, cps, {}, {}});
                max_grid = std::max(max_grid, cps * c->num_sms);
            }
    }
    if (cands.empty()) return fail(c, NB_ECUDA, "no force launch shape fits on this device");
    // scratch for the largest candidate grid with either i per thread
    const nb_ctx::Variant keep0 = c->var[0], keep1 = c->var[1], keep2 = c->var[2];
    c->var[0] = c->var[2] = {1, max_grid};
    c->var[1] = {shapes.back().first, max_grid};
    s = ensure_force_scratch(c);
    c->var[0] = keep0;
    c->var[1] = keep1;
    c->var[2] = keep2;
    if (s != NB_OK) return s;
    double* ht = reinterpret_cast<double*>(c->pinned + 48);
    NB_CK(c, cudaMemcpyAsync(ht, c->st.t, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    NB_CK(c, cudaStreamSynchronize(c->stream));
    NB_CK(c, nb::predict_launch(c->st, c->prec, c->jl, c->cfg.G, nullptr, *ht, nullptr, c->stream,
                                c->ens ? &c->cl : nullptr));
    NB_CK(c, nb::iota_launch(c->idx_user, n, c->n_act_user, c->stream));
    // Hybrid: the shapes are timed with the integration guard idle (no noise
    // history), the steady state of an integration; the probe evaluations
    // write noise estimates of their own, so the particles' estimates are
    // kept aside and put back afterwards.
    double* hq_keep = nullptr;
    if (nb::is_hybrid(c->prec)) {
        if (!c->order_buf) NB_CK(c, cudaMalloc(&c->order_buf, (17 * n + 1) * sizeof(double)));
        hq_keep = c->order_buf;
        NB_CK(c, cudaMemcpyAsync(hq_keep, c->st.hq, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream));
        NB_CK(c, cudaMemsetAsync(c->st.hq, 0, n * sizeof(double), c->stream));
    }
    cudaEvent_t e0, e1;
    NB_CK(c, cudaEventCreate(&e0));
    NB_CK(c, cudaEventCreate(&e1));
    nb_status st = NB_OK;
    for (int q = 0; q < NQ && st == NB_OK; ++q) {
        // a probe block: particles spread evenly over the stored order, like
        // the scattered members of a real block step
        if (cudaSuccess != nb::strided_list_launch(c->idx_user, probes[q], n, c->n_act_user,
                                                   c->stream))
            st = fail(c, NB_ECUDA, "autotune: probe list");
        for (auto& cd : cands) {
            if (st != NB_OK) break;
            if (c->ens && cudaSuccess != nb::plan_launch(c->cl, c->idx_user, c->n_act_user,
                                                         32 * cd.it / cd.split, c->stream))
                st = fail(c, NB_ECUDA, "autotune: plan");
            nb::ForceArgs f = force_args(c, c->prec, c->jl, c->idx_user, c->n_act_user);
            f.it = cd.it;
            f.split = cd.split;
            f.grid = cd.cps * c->num_sms;
            // the small buckets' probes (0-3) with the build their variants
            // run (CTA-level sums), the large bucket's (3-4) with the plain one
            for (int build = 0; build < 2 && st == NB_OK; ++build) {
                const bool small = build == 0;
                if ((small && q > 3) || (!small && q < 3)) continue;
                f.cta_mode = small && !c->ens;
                const int reps = 3;
                cudaError_t e = nb::force_launch(f, c->stream);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
                for (int k = 0; k < reps && e == cudaSuccess; ++k) e = nb::force_launch(f, c->stream);
                if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) st = fail(c, NB_ECUDA, "autotune: %s", cudaGetErrorString(e));
                (small ? cd.us : cd.usl)[q] = 1e3 * ms / reps;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (hq_keep)
        NB_CK(c, cudaMemcpyAsync(c->st.hq, hq_keep, n * sizeof(double), cudaMemcpyDeviceToDevice,
                                 c->stream));
    if (st != NB_OK) return st;
    if ((s = check_status(c)) != NB_OK) return s;
    // Best shape per bucket; ties go to the smaller grid (listed first).  The
    // small bucket holds the probes below the split (three or four of them:
    // nact_split 1024 or 4096), the large one the rest.  An ensemble's plan
    // is cut once per block for both variants, so there the two share the
    // (i per thread, j split) with the least total time.  A single system
    // then may take a tiny shape for its first one or two probes, used only
    // by force calls whose block size the host knows (a device-sized block
    // step keeps two launch branches); it must beat the small shape there by
    // more than TINY_MARGIN_US, well above the timing noise.
    constexpr double TINY_MARGIN_US = 0.5;
    // lo == 0 or hi < NQ: a small or tiny bucket, timed with the small build
    auto bucket_us = [](const Cand& cd, int lo, int hi) {
        const bool small = lo == 0 || hi < NQ;
        double t = 0.0;
        for (int q = lo; q < hi; ++q) t += small ? cd.us[q] : cd.usl[q];
        return t;
    };
    auto best_of = [&](int lo, int hi, int it, int split) {
        const Cand* bc = nullptr;
        for (const auto& cd : cands) {
            if (it > 0 && (cd.it != it || cd.split != split)) continue;
            if (!bc || bucket_us(cd, lo, hi) < bucket_us(*bc, lo, hi)) bc = &cd;
        }
        return bc;
    };
    const Cand* best[3] = {nullptr, nullptr, nullptr};
    int split_probe = 3, tiny_probe = 0;
    double tbest = -1.0;
    for (int sp : {3, 4}) {  // probes [0, sp) are small
        const Cand* b[2] = {best_of(0, sp, 0, 0), best_of(sp, NQ, 0, 0)};
        if (c->ens) {
            b[0] = b[1] = nullptr;
            double tsh = -1.0;
            for (const auto& sh : shapes) {
                const Cand* b0 = best_of(0, sp, sh.first, sh.second);
                const Cand* b1 = best_of(sp, NQ, sh.first, sh.second);
                if (!b0 || !b1) continue;
                const double tot = bucket_us(*b0, 0, sp) + bucket_us(*b1, sp, NQ);
                if (tsh < 0.0 || tot < tsh) b[0] = b0, b[1] = b1, tsh = tot;
            }
        }
        const double tot = bucket_us(*b[0], 0, sp) + bucket_us(*b[1], sp, NQ);
        if (tbest < 0.0 || tot < tbest) best[0] = b[0], best[1] = b[1], split_probe = sp, tbest = tot;
    }
    if (!c->ens) {
        double gain = TINY_MARGIN_US;
        for (int tp : {1, 2}) {  // probes [0, tp) are tiny
            const Cand* bt = best_of(0, tp, 0, 0);
            const double g = bucket_us(*best[0], 0, tp) - bucket_us(*bt, 0, tp);
            if (g > gain) best[2] = bt, tiny_probe = tp, gain = g;
        }
    }
    c->var[0] = {best[0]->it, best[0]->cps * c->num_sms, best[0]->split};
    c->var[1] = {best[1]->it, best[1]->cps * c->num_sms, best[1]->split};
    c->var[2] = best[2] ? nb_ctx::Variant{best[2]->it, best[2]->cps * c->num_sms, best[2]->split}
                        : c->var[0];
    c->nact_split = split_probe == 3 ? 1024 : 4096;
    c->tiny_split = tiny_probe == 0 ? 0 : tiny_probe == 1 ? 64 : 160;
    drop_graph(c);
    c->last_force_n_act = -1;
    if (out) {
        *out = nb_tuning{};
        out->small_i_per_thread = best[0]->it;
        out->small_ctas_per_sm = best[0]->cps;
        out->large_i_per_thread = best[1]->it;
        out->large_ctas_per_sm = best[1]->cps;
        out->nact_split = c->nact_split;
        out->small_j_split = best[0]->split;
        out->large_j_split = best[1]->split;
        out->small_us = bucket_us(*best[0], 0, split_probe);
        out->large_us = bucket_us(*best[1], split_probe, NQ);
        if (best[2]) {
            out->tiny_split = c->tiny_split;
            out->tiny_i_per_thread = best[2]->it;
            out->tiny_ctas_per_sm = best[2]->cps;
            out->tiny_j_split = best[2]->split;
            out->tiny_us = bucket_us(*best[2], 0, tiny_probe);
        }
        out->ens_chunks = c->ens_chunks;
    }
    return NB_OK;
}

nb_status nb_set_tuning(nb_ctx* c, const nb_tuning* t)
{
    nb_status s = enter(c, false);
    if (s != NB_OK) return s;
    if (!t) return fail(c, NB_EINVAL, "no tuning given");
    struct Shape {
        const char* name;
        int it, split, cps;
    };
    const Shape sh[3] = {{"small", t->small_i_per_thread, t->small_j_split, t->small_ctas_per_sm},
                         {"large", t->large_i_per_thread, t->large_j_split, t->large_ctas_per_sm},
                         {"tiny", t->tiny_i_per_thread, t->tiny_j_split, t->tiny_ctas_per_sm}};
    if (t->nact_split < 1 || t->tiny_split < 0 || t->tiny_split >= t->nact_split)
        return fail(c, NB_EINVAL, "block-size boundaries tiny %d, small %d", t->tiny_split,
                    t->nact_split);
    if (c->ens && (t->tiny_split != 0 || sh[0].it != sh[1].it || sh[0].split != sh[1].split))
        return fail(c, NB_EINVAL, "an ensemble takes one i-tile and j split and no tiny shape");
    if (t->ens_chunks < 0 || t->ens_chunks > 4)
        return fail(c, NB_EINVAL, "%d stream-K chunks per warp (0 to 4)", t->ens_chunks);
    for (int v = 0; v < 3; ++v) {
        if (v == 2 && t->tiny_split == 0) continue;
        const Shape& q = sh[v];
        if (!nb::force_variant_exists(c->prec, q.it, q.split))
            return fail(c, NB_EINVAL, "%s shape: no kernel with %d i per thread, j split %d",
                        q.name, q.it, q.split);
        if (nb::force_setup(c->prec, q.it, q.split) != cudaSuccess)
            return fail(c, NB_ECUDA, "kernel attributes");
        const int occ = nb::force_ctas_per_sm(c->prec, q.it, q.split);
        if (q.cps < 1 || q.cps > occ)
            return fail(c, NB_EINVAL, "%s shape: %d CTAs per SM (1 to %d fit)", q.name, q.cps, occ);
    }
    for (int v = 0; v < 3; ++v) {
        const Shape& q = sh[v == 2 && t->tiny_split == 0 ? 0 : v];
        c->var[v] = {q.it, q.cps * c->num_sms, q.split};
    }
    c->nact_split = t->nact_split;
    c->tiny_split = t->tiny_split;
    c->ens_chunks = t->ens_chunks > 0 ? t->ens_chunks : ens_chunks_default(c->prec);
    if ((s = ensure_force_scratch(c)) != NB_OK) return s;
    drop_graph(c);
    c->last_force_n_act = -1;
    return NB_OK;
}

nb_status nb_set_j_part(nb_ctx* c, int32_t part, int32_t parts)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    if (parts < 1 || part < 0 || part >= parts)
        return fail(c, NB_EINVAL, "part %d of %d", part, parts);
    if (parts > 1 && c->ens)
        return fail(c, NB_EINVAL, "a j partition works on one system");
    if (parts > c->n_pad / nb::TJ)
        return fail(c, NB_EINVAL, "%d parts of %lld j tiles", parts,
                    static_cast<long long>(c->n_pad / nb::TJ));
    c->j_part = part;
    c->j_parts = parts;
    drop_graph(c);
    return NB_OK;
}

nb_status nb_spatial_order(nb_ctx* c, int32_t* order)
{
    nb_status s = enter(c, true);
    if (s != NB_OK) return s;
    if (!order) return fail(c, NB_EINVAL, "NULL order");
    if ((s = sync_host_order(c)) != NB_OK) return s;
    std::memcpy(order, c->h_perm.data(), c->n * sizeof(int32_t));
    return NB_OK;
}

int64_t nb_num_particles(const nb_ctx* c) { return c && c->loaded ? c->n : 0; }

const char* nb_last_error(const nb_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

const char* nb_status_string(nb_status s)
{
    switch (s) {
    case NB_OK: return "NB_OK";
    case NB_EINVAL: return "NB_EINVAL";
    case NB_ECUDA: return "NB_ECUDA";
    case NB_ENOMEM: return "NB_ENOMEM";
    case NB_ENONFINITE: return "NB_ENONFINITE";
    case NB_EDTMIN: return "NB_EDTMIN";
    case NB_ETIMEOUT: return "NB_ETIMEOUT";
    case NB_ESTATE: return "NB_ESTATE";
    }
    return "unknown";
}

}  // extern "C"
