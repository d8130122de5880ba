// nb_force_static: the force evaluation (Eqs. acc, jrk, pot, double-single
// pair arithmetic) for callers that cannot allocate device memory.
//
// The regular entry points keep their buffers in a context that
// nb_set_particles sizes with cudaMalloc.  Some callers cannot do that:
// code that runs where the allocator is not available or not allowed,
// such as a host framework that owns all device memory and forbids other
// allocations, or a process that has reserved the whole GPU for itself.
// This entry point takes the caller's device arrays and uses, as its only
// working memory, one file-scope device array of fixed size
// (NB_STATIC_SCRATCH_BYTES): the j layout the force kernel streams, the
// partial sums of i-groups split across warps, their arrival counters and a
// status word.  It calls no cudaMalloc, cudaFree or allocating library
// routine.
#include <cstdio>
#include <mutex>

#include "nb_device.cuh"
#include "nb_launch.h"
#include "nbody.h"

namespace {

// The working memory.  Every GPU that loads this library holds it until the
// process exits.  In host code the name is only a stand-in for the symbol:
// its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char nb_static_scratch[NB_STATIC_SCRATCH_BYTES];

constexpr int STATIC_CTAS_PER_SM = 4;  // fixes the number of warps, hence the scratch size
constexpr int MAX_DEVICES = 64;
constexpr size_t CONTROL_BYTES = 256;  // status word, n_act, layout bounds

struct DeviceSetup {
    bool ready = false;
    unsigned char* base = nullptr;  // device address of nb_static_scratch
    int grid = 0;                   // force CTAs
};
DeviceSetup g_setup[MAX_DEVICES];
std::mutex g_mutex;

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct Plan {
    size_t counters, layout, scratch, total;
    int64_t n_pad, counter_stride, counter_words;
};

Plan plan_for(int64_t n, int grid)
{
    Plan p;
    const int warps = grid * nb::FORCE_WARPS;
    p.n_pad = (n + nb::TJ - 1) / nb::TJ * nb::TJ;
    p.counter_stride = nb::force_counter_stride(n, warps);
    p.counter_words = nb::force_counter_entries(n, warps);
    p.counters = CONTROL_BYTES;
    p.layout = align256(p.counters + p.counter_words * sizeof(uint32_t));
    p.scratch = align256(p.layout + 4 * p.n_pad * 16);
    p.total = p.scratch + nb::force_scratch_doubles(1, n, warps) * sizeof(double);
    return p;
}

// Predicted particles (device, n x 3 doubles) -> the double-single j layout
// (grid-aligned splits on the grids of `bound`), with zero-mass ghosts far
// away up to n_pad.
__global__ void static_layout_kernel(int64_t n, int64_t n_pad, const double* m, const double* r,
                                     const double* v, double G, const uint32_t* bound, float4* A,
                                     float4* B, float4* C, float4* D)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    double x[3], u[3], gm;
    if (i < n) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            x[c] = r[3 * i + c];
            u[c] = v[3 * i + c];
        }
        gm = G * m[i];
    } else {
        x[0] = x[1] = x[2] = nb::GHOST_POS;
        u[0] = u[1] = u[2] = 0.0;
        gm = 0.0;
    }
    const nb::GridQuantum gx = nb::grid_quantum(bound[0]), gv = nb::grid_quantum(bound[1]);
    float xh[3], xl[3], vh[3], vl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (i < n) {
            nb::grid_split(x[c], gx, xh[c], xl[c]);
        } else {
            xh[c] = static_cast<float>(x[c]);
            xl[c] = 0.f;
        }
        nb::grid_split(u[c], gv, vh[c], vl[c]);
    }
    const float gh = __double2float_rn(gm);
    const float gl = __double2float_rn(gm - static_cast<double>(gh));
    A[i] = make_float4(xh[0], xh[1], xh[2], gh);
    B[i] = make_float4(xl[0], xl[1], xl[2], gl);
    C[i] = make_float4(vh[0], vh[1], vh[2], 0.f);
    D[i] = make_float4(vl[0], vl[1], vl[2], 0.f);
}

// One-time set-up for the current device: the symbol's device address and
// the force kernel's launch shape.
nb_status setup_device(int dev, DeviceSetup*& out)
{
    if (dev < 0 || dev >= MAX_DEVICES) return NB_EINVAL;
    std::lock_guard<std::mutex> lock(g_mutex);
    DeviceSetup& s = g_setup[dev];
    if (!s.ready) {
        void* addr = nullptr;
        if (cudaGetSymbolAddress(&addr, nb_static_scratch) != cudaSuccess) return NB_ECUDA;
        if (nb::force_setup(nb::Prec::DS, 1, 1) != cudaSuccess) return NB_ECUDA;
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            return NB_ECUDA;
        int per_sm = nb::force_ctas_per_sm(nb::Prec::DS, 1, 1);
        if (per_sm < 1) return NB_ECUDA;
        if (per_sm > STATIC_CTAS_PER_SM) per_sm = STATIC_CTAS_PER_SM;
        // The scratch of the split-group sums grows with the number of
        // persistent warps; shrink the grid until the largest system allowed
        // fits the array, so the limit on n holds whatever the SM count.
        int grid = per_sm * sms;
        while (grid > 1 && plan_for(NB_STATIC_MAX_N, grid).total > NB_STATIC_SCRATCH_BYTES)
            grid -= grid / 8 > 0 ? grid / 8 : 1;
        s.base = static_cast<unsigned char*>(addr);
        s.grid = grid;
        s.ready = true;
    }
    out = &s;
    return NB_OK;
}

}  // namespace

extern "C" nb_status nb_force_static(int64_t n, const double* m, const double* r,
                                     const double* v, double eps, double G, int32_t n_act,
                                     const int32_t* idx, double* acc, double* jerk,
                                     double* pot, void* stream)
{
    if (n < 1 || n > NB_STATIC_MAX_N) {
        std::fprintf(stderr, "nb_force_static: n = %lld outside [1, %d]\n",
                     static_cast<long long>(n), NB_STATIC_MAX_N);
        return NB_EINVAL;
    }
    if (n_act < 0 || n_act > n) {
        std::fprintf(stderr, "nb_force_static: n_act = %d outside [0, n]\n", n_act);
        return NB_EINVAL;
    }
    if (!m || !r || !v || (n_act > 0 && (!idx || !acc || !jerk || !pot))) return NB_EINVAL;
    if (!(eps >= 0.0)) return NB_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return NB_ECUDA;
    DeviceSetup* s = nullptr;
    nb_status st = setup_device(dev, s);
    if (st != NB_OK) return st;
    const Plan p = plan_for(n, s->grid);
    if (p.total > NB_STATIC_SCRATCH_BYTES) {
        std::fprintf(stderr, "nb_force_static: needs %zu bytes of scratch, has %d\n", p.total,
                     NB_STATIC_SCRATCH_BYTES);
        return NB_EINVAL;
    }
    if (n_act == 0) return NB_OK;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    uint32_t* status = reinterpret_cast<uint32_t*>(s->base);
    int32_t* n_act_dev = reinterpret_cast<int32_t*>(s->base + 4);
    uint32_t* bound = reinterpret_cast<uint32_t*>(s->base + 8);
    uint32_t* counters = reinterpret_cast<uint32_t*>(s->base + p.counters);
    float4* L = reinterpret_cast<float4*>(s->base + p.layout);
    double* scratch = reinterpret_cast<double*>(s->base + p.scratch);
    // The array keeps whatever the previous call left: the status word, the
    // layout bounds and the arrival counters must start from zero.
    if (cudaMemsetAsync(status, 0, 4 * sizeof(uint32_t), cs) != cudaSuccess) return NB_ECUDA;
    if (cudaMemsetAsync(counters, 0, p.counter_words * sizeof(uint32_t), cs) != cudaSuccess)
        return NB_ECUDA;
    if (nb::set_scalars_launch(n_act_dev, n_act, nullptr, 0.0, cs) != cudaSuccess) return NB_ECUDA;
    if (nb::bounds_launch(r, v, 3 * n, bound, cs) != cudaSuccess) return NB_ECUDA;
    static_layout_kernel<<<static_cast<unsigned>((p.n_pad + 255) / 256), 256, 0, cs>>>(
        n, p.n_pad, m, r, v, G, bound, L, L + p.n_pad, L + 2 * p.n_pad, L + 3 * p.n_pad);
    if (cudaGetLastError() != cudaSuccess) return NB_ECUDA;
    nb::ForceArgs f;
    f.prec = nb::Prec::DS;
    f.it = 1;
    for (int k = 0; k < 4; ++k) f.jl.arr[k] = L + k * p.n_pad;
    f.n = n;
    f.n_pad = p.n_pad;
    f.idx = idx;
    f.n_act_dev = n_act_dev;
    f.acc = acc;
    f.jerk = jerk;
    f.pot = pot;
    f.scratch = scratch;
    f.counters = counters;
    f.counter_stride = p.counter_stride;
    f.status = status;
    f.eps2 = eps * eps;
    f.grid = s->grid;
    if (nb::force_launch(f, cs) != cudaSuccess) return NB_ECUDA;
    uint32_t host_status = 0;
    if (cudaMemcpyAsync(&host_status, status, sizeof(host_status), cudaMemcpyDeviceToHost, cs) !=
            cudaSuccess ||
        cudaStreamSynchronize(cs) != cudaSuccess)
        return NB_ECUDA;
    if (host_status & nb::ST_BADINDEX) return NB_EINVAL;
    if (host_status & nb::ST_TIMEOUT) return NB_ETIMEOUT;
    return NB_OK;
}
