// Host-side interface between the C ABI (capi.cu) and the kernel translation
// units (force.cu, hermite.cu).  Internal to libnbody; not installed.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace nb {

// Precision of the force path.
//   FP64  - every operation in double (the plain baseline).
//   MIXED - Sec. 3.2 "mixed" precision: r_ij from double-single positions,
//           the pair arithmetic in FP32, per-tile FP32 partial sums folded
//           into compensated (double-single) accumulators.
//   DS    - the same pair formulas evaluated in double-single ("float-float")
//           arithmetic on the FP32 pipes with error-free transforms.
//   HYBRID - FP32 far pairs, double-single near pairs.
//   MIXED_SPJ - MIXED with the jerk summed in plain FP32, the accumulation
//           the paper's own kernel uses (Sec. 4, Fig. err_snp_djerk).
//   HYBRID_SPJ - HYBRID with the far-field jerk summed in plain FP32 (the
//           same study on the precision that integrates).
//   FP64_H6 - FP64 with snap: the sixth-order Hermite variant (adjacent to
//           the paper, which integrates with the fourth-order scheme).
enum class Prec : int {
    FP64 = 0, MIXED = 1, DS = 2, HYBRID = 3, MIXED_SPJ = 4, HYBRID_SPJ = 5, FP64_H6 = 6
};

inline bool is_mixed(Prec p) { return p == Prec::MIXED || p == Prec::MIXED_SPJ; }
inline bool is_hybrid(Prec p) { return p == Prec::HYBRID || p == Prec::HYBRID_SPJ; }

// Device Hermite state of one context, structure of arrays.  x, v, a, j
// hold 3*n doubles: component c of particle i at [c*n + i].
struct StateDev {
    int64_t n = 0;      // real particles
    int64_t n_pad = 0;  // j-layout length (multiple of the tile size)
    double* m = nullptr;
    double* x = nullptr;
    double* v = nullptr;
    double* a = nullptr;
    double* j = nullptr;
    double* t = nullptr;
    double* dt = nullptr;
    // [0] bound on every |position component|, [1] on every |velocity
    // component| (float bits, never decreasing): set from the whole state at
    // load, raised by the corrector.  They fix the grid of the j layout's
    // double-single split (grid_split).
    uint32_t* bound = nullptr;
    // Hybrid precision: per particle, the far-field noise estimate of its
    // last force evaluation, negative when that evaluation was guarded
    // (all double-single); 0 = none yet.
    double* hq = nullptr;
    // Sixth-order variant only: snap s and crackle c at each particle's
    // time (3 n each, SoA like a and j).
    double* s = nullptr;
    double* c = nullptr;
    // Per particle, the order-preserving key of its next time t_i + dt_i,
    // kept by every writer of t and dt so that step 1 compares integers.
    unsigned long long* nkey = nullptr;
};

// bound[0] = max |a_k|, bound[1] = max |b_k| over k < count (float bits,
// rounded up), atomically raised; the caller zeroes bound first.
cudaError_t bounds_launch(const double* a, const double* b, int64_t count, uint32_t* bound,
                          cudaStream_t s);
// nkey[i] = key of t[i] + dt[i] for every particle.
cudaError_t next_key_launch(const StateDev& st, cudaStream_t s);

// Predicted j particles in the layout a force kernel streams.
//   FP64 : arr[0] = double4 (x, y, z, G m), arr[1] = double4 (vx, vy, vz, 0)
//   FP64_H6: as FP64 plus arr[2] = double4 (ax, ay, az, 0), the predicted
//          accelerations
//   MIXED: arr[0] = float4 (x_hi, y_hi, z_hi, G m), arr[1] = float4 (x_lo,
//          y_lo, z_lo, vx), arr[2] = float2 (vy, vz)
//   Position (and DS velocity) hi/lo pairs are grid-aligned splits
//   (grid_split): every hi part of the layout lies on one power-of-two grid.
//   DS:    arr[0] = float4 (x_hi, y_hi, z_hi, Gm_hi), arr[1] = float4
//          (x_lo, y_lo, z_lo, Gm_lo), arr[2] = float4 (vx_hi, vy_hi, vz_hi,
//          (Gm)^(2/3)), arr[3] = float4 (vx_lo, vy_lo, vz_lo, 0)
//   HYBRID: as DS, except that the velocity is split as hi = fl32(v) (its
//          FP32 value, the far pairs' operand) and lo = fl32(v - hi), off
//          the grid.
struct JLayout {
    void* arr[4] = {nullptr, nullptr, nullptr, nullptr};
};
int jlayout_narr(Prec p);
int jlayout_elem_bytes(Prec p, int k);

// Scheduler buffers (step 1 of the integration procedure).
struct SchedDev {
    unsigned long long* tmin_bits = nullptr;  // next block time, as bits
    int32_t* idx = nullptr;                   // active list, capacity n
    int32_t* n_act = nullptr;                 // device scalar
    int32_t* block_counts = nullptr;
    int32_t* block_offsets = nullptr;
    uint32_t* ticket = nullptr;
    int max_blocks = 0;
};
constexpr int SCHED_THREADS = 256;
constexpr int SCHED_PER_THREAD = 8;
constexpr int SCHED_CHUNK = SCHED_THREADS * SCHED_PER_THREAD;

// Ensemble of independent systems ("clusters") in one context.  Cluster c
// owns particles [off[c], off[c+1]) and j-layout slots [joff[c], joff[c+1])
// (its particles, then zero-mass ghosts up to a multiple of the tile).
struct ClusterDev {
    int k = 0;
    int64_t* off = nullptr;          // k + 1
    int64_t* joff = nullptr;         // k + 1
    double* eps2 = nullptr;          // k
    int32_t* cluster_of = nullptr;   // n: cluster of each particle
    int32_t* jsrc = nullptr;         // n_pad: particle of each j slot, -1 = ghost
    unsigned long long* tkey = nullptr;  // k: next block time of each cluster (key)
    int32_t* cnt = nullptr;              // k: members of each cluster's next block
                                         // (0 past t_end), from cluster_select_launch
    // force plan written by plan_launch
    int32_t* grp_cluster = nullptr;
    int32_t* grp_act_begin = nullptr;
    int32_t* grp_act_count = nullptr;
    int64_t* grp_tile0 = nullptr;    // max_groups + 1
    int64_t* plan_scalars = nullptr; // [0] groups, [1] tiles
    int64_t max_groups = 0;
};

// Force plan arrays handed to the kernel (all null for one system).
struct ForcePlan {
    const int32_t* grp_cluster = nullptr;
    const int32_t* grp_act_begin = nullptr;
    const int32_t* grp_act_count = nullptr;
    const int64_t* grp_tile0 = nullptr;
    const int64_t* scalars = nullptr;
    const int64_t* cl_off = nullptr;
    const int64_t* cl_joff = nullptr;
    const double* cl_eps2 = nullptr;
};

// Force launch (step 4): active list -> acc, jerk, pot.
struct ForceArgs {
    Prec prec = Prec::MIXED;
    int it = 1;          // i particles per thread (register blocking)
    int split = 1;       // lanes per i: the j split inside a warp (1, 2, 4, 8)
    JLayout jl;
    int64_t n = 0;       // real particles (index validation)
    int64_t n_pad = 0;   // j count incl. ghosts, multiple of TJ
    const int32_t* idx = nullptr;
    const int32_t* n_act_dev = nullptr;
    double* acc = nullptr;   // [n_act][3]
    double* jerk = nullptr;  // [n_act][3]
    double* pot = nullptr;   // [n_act]
    double* snap = nullptr;  // [n_act][3], FP64_H6 only
    double* scratch = nullptr;
    uint32_t* counters = nullptr;   // force_counter_entries() zeroed words
    int64_t counter_stride = 0;     // entries per reduction level
    uint32_t* status = nullptr;
    double eps2 = 0.0;
    int grid = 0;        // CTAs (persistent)
    int32_t nact_lo = 0;           // the launch does nothing unless
    int32_t nact_hi = 0x7fffffff;  // nact_lo <= n_act < nact_hi
    long long wait_limit = 0;      // cycles per tile wait; 0 = about one second
    int32_t unfed_first_tile = 0;  // self-test of the timeout path only
    ForcePlan plan;      // ensemble plan (empty: one system)
    // HYBRID only: the state's a, j (near-pair test) and the velocity bound.
    const double* st_a = nullptr;
    const double* st_j = nullptr;
    const uint32_t* bound_v = nullptr;
    const double* st_dt = nullptr;  // integration guard (see PolicyHybrid)
    double* st_hq = nullptr;
    double eta = 0.0;
    // One system only: sum over the j tiles [jt_lo, jt_hi) of the layout
    // (a part of a j-partitioned force); jt_hi = 0: every tile.
    int64_t jt_lo = 0, jt_hi = 0;
    // One system: blocks of at most a quarter as many i-groups as CTAs are summed
    // CTA by CTA (shared memory, then one global level) instead of by the
    // warp tree.
    int32_t cta_mode = 0;
    // n_act known at launch (>= 0): the kernel does not read n_act_dev.
    int32_t n_act_host = -1;
    // Optional: idx holds caller indices, idx_map[i] is the layout slot of i.
    const int32_t* idx_map = nullptr;
    // Ensemble plans: up to this many stream-K chunks per warp (at most
    // MAX_CHUNKS), the chunks after each warp's first taken from a queue in
    // the order warps come free; 0 or 1: one chunk per warp.
    int32_t dyn_chunks = 0;
};

cudaError_t force_setup(Prec p, int it, int split);  // one-time attribute setup
int force_ctas_per_sm(Prec p, int it, int split);
size_t force_smem_bytes(Prec p);
bool force_variant_exists(Prec p, int it, int split);
// Scratch needed for n_act_max active particles with `warps` persistent warps.
size_t force_scratch_doubles(int it, int64_t n_act_max, int warps);
// Arrival counters of the split-group reduction tree: stride per level and
// the total number of 32-bit words (all must start at zero; the kernel
// leaves them at zero).
int64_t force_counter_stride(int64_t n_act_max, int warps);
int64_t force_counter_entries(int64_t n_act_max, int warps);
cudaError_t force_launch(const ForceArgs& f, cudaStream_t s);

// Predictor (steps 2-3) to the time in t_bits (per cluster when cl is
// given, else t_bits[0]) or, with t_bits null, to t_host.  With n_act_dev
// non-null nothing is done when *n_act_dev == 0.
cudaError_t predict_launch(const StateDev& st, Prec p, const JLayout& jl, double G,
                           const unsigned long long* t_bits, double t_host,
                           const int32_t* n_act_dev, cudaStream_t s,
                           const ClusterDev* cl = nullptr);

// Ensemble step 1 (per-cluster next times, then one global compaction) and
// the force plan of the active list (idx ascending, clusters contiguous).
cudaError_t cluster_select_launch(const StateDev& st, const ClusterDev& cl, const SchedDev& sd,
                                  double t_end, cudaStream_t s);
// With from_counts the plan takes each cluster's share of the (sorted) active
// list from cl.cnt, written by the select of the same block step; otherwise
// it finds the shares in idx by binary search (any sorted list).
cudaError_t plan_launch(const ClusterDev& cl, const int32_t* idx, const int32_t* n_act_dev,
                        int gi, cudaStream_t s, bool from_counts = false);
// Per-cluster energies: out[2c] = sum 1/2 m v^2, out[2c+1] = sum 1/2 m phi.
cudaError_t cluster_energy_launch(const StateDev& st, const ClusterDev& cl, const double* pot_all,
                                  double* out, cudaStream_t s);

// Stream-ordered scalar stores: *i32 = v (if i32), *t_bits = key(t) (if t_bits).
cudaError_t set_scalars_launch(int32_t* i32, int32_t v, unsigned long long* t_bits,
                               double t, cudaStream_t s);
// Host mirror of the device time key.
double time_from_key(unsigned long long k);

// Step 1: t_next = min(t + dt), stable compaction of the active block.
// When t_next > t_end the block is empty (n_act = 0).
cudaError_t select_launch(const StateDev& st, const SchedDev& sd, double t_end,
                          cudaStream_t s);

// Steps 5-8 on the active list at the time in *t_bits.
struct CorrectArgs {
    const int32_t* idx = nullptr;
    const int32_t* n_act_dev = nullptr;
    const unsigned long long* t_bits = nullptr;
    const double* acc1 = nullptr;   // [n_act][3]
    const double* jerk1 = nullptr;  // [n_act][3]
    double eta = 0.02, dt_max = 1.0 / 16, dt_min = 0x1p-40;
    uint32_t* status = nullptr;
    unsigned long long* step_counter = nullptr;   // +1 per non-empty block
    unsigned long long* inter_counter = nullptr;  // += n_act * n (per cluster)
    const int32_t* cluster_of = nullptr;          // ensemble: t_bits per cluster
    const int64_t* cl_off = nullptr;
};
cudaError_t correct_launch(const StateDev& st, const CorrectArgs& c, cudaStream_t s);
// The sixth-order variant's steps 5-8 (snap1: the block's new snap rows).
cudaError_t correct6_launch(const StateDev& st, const CorrectArgs& c, const double* snap1,
                            cudaStream_t s);
// Its start: the snap rows of a full evaluation (in particle order) into
// the state, crackle zero.
cudaError_t init_snap_launch(const StateDev& st, const double* snap_rows, cudaStream_t s);

// Initial timesteps from a, j (reading R3), t = t0.
cudaError_t init_dt_launch(const StateDev& st, const double* acc, const double* jerk,
                           double eta_start, double dt_max, double dt_min, double t0,
                           uint32_t* status, cudaStream_t s);

// Deterministic sums: out[0] = sum 1/2 m v^2, out[1] = sum 1/2 m phi.
cudaError_t energy_launch(const StateDev& st, const double* pot_all, double* partials,
                          int max_blocks, double* out, uint32_t* ticket,
                          cudaStream_t s);

// Layout conversions between host AoS [n][3] and device SoA.
cudaError_t aos_to_soa_launch(const double* aos, double* soa, int64_t n, cudaStream_t s);
cudaError_t soa_to_aos_launch(const double* soa, double* aos, int64_t n, cudaStream_t s);
cudaError_t iota_launch(int32_t* idx, int64_t n, int32_t* n_act_dev, cudaStream_t s);
// idx[i] = floor(i n / k), i < k: k particles spread evenly over the stored
// order (ascending); *n_act_dev = k.
cudaError_t strided_list_launch(int32_t* idx, int64_t k, int64_t n, int32_t* n_act_dev,
                                cudaStream_t s);
// Copy the whole state (17 n words: m, x, v, a, j, t, dt, hq, nkey, then
// the two bounds) to (to_buf) or from a device buffer of 17 n + 1 doubles.
cudaError_t snapshot_launch(const StateDev& st, double* buf, bool to_buf, cudaStream_t s);

// The context stores its particles in its spatial order (internal index k
// holds the caller's particle perm[k]).  Boundary permutations of arrays of
// w doubles per particle:
//   permute_in:  dst_soa[c n + k] = src_aos[w perm[k] + c]   (caller -> state)
//   permute_out: dst_aos[w perm[k] + c] = src_soa[c n + k]   (state -> caller)
cudaError_t permute_in_launch(const double* src_aos, double* dst_soa, int64_t n, int w,
                              const int32_t* perm, cudaStream_t s);
cudaError_t permute_out_launch(const double* src_soa, double* dst_aos, int64_t n, int w,
                               const int32_t* perm, cudaStream_t s);
// Caller indices to internal ones: out[a] = inv[in[a]] (-1 outside [0, n)).
cudaError_t map_index_launch(const int32_t* in, int32_t* out, int32_t count, int64_t n,
                             const int32_t* inv, cudaStream_t s);
// Re-order the state from a snapshot buf (snapshot_launch layout): every
// per-particle word of internal index k takes the value of index map[k].
cudaError_t reorder_state_launch(const StateDev& st, const double* buf, const int32_t* map,
                                 cudaStream_t s);

}  // namespace nb
