// k_noalloc.cu -- cosmica_propagate_noalloc: propagation that allocates nothing.
//
// Some callers cannot allocate device memory: code that runs under a memory
// pool it does not own (a framework's caching allocator may hold every free
// byte, so a raw cudaMalloc fails or fragments the pool), code that must not
// trigger the device-wide synchronisation cudaFree implies while other work
// is in flight, and hosts whose policy routes every device allocation
// through an approved allocator.  For them this entry point runs the same
// propagation kernels as cosmica_propagate, but keeps its scratch (parameter
// block, species, work items, prefix sums, queue cursor and step counter) in
// the fixed static device array below instead of in memory it allocates.
//
// Limits and rules:
//   * at most COSMICA_NOALLOC_MAX_ENERGIES energies per call (larger calls are
//     rejected with COSMICA_ERR_INVALID); the array is ~45 KB and every GPU
//     that loads the library holds it until the process exits;
//   * the exit states must be device memory (no host staging is possible
//     without allocating);
//   * the first call on a device looks the array's device address up
//     (cudaGetSymbolAddress with that device current); make that first call
//     before any stream capture;
//   * every call reuses the same array: the queue cursor and step counter are
//     cleared at the start of each call, the tables are overwritten, and two
//     calls whose work overlaps on the GPU (other streams, other threads)
//     race on the array -- serialise them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "cosmica.h"
#include "host_util.h"
#include "internal.h"

using namespace cosmica;
using namespace cosmica::host;

namespace {

constexpr uint32_t kMaxE = COSMICA_NOALLOC_MAX_ENERGIES;

// layout of the scratch array (every region 256-byte aligned)
constexpr size_t kOffParams = 0;
constexpr size_t kOffSpecies = (sizeof(DevParams) + 255) / 256 * 256;
constexpr size_t kOffItems = kOffSpecies + 256;
constexpr size_t kOffPrefix = kOffItems + (kMaxE * sizeof(DevItem) + 255) / 256 * 256;
constexpr size_t kOffCounters = kOffPrefix + ((kMaxE + 1) * sizeof(uint64_t) + 255) / 256 * 256;
constexpr size_t kOffF32 = kOffCounters + 256;          // one page of the FP32 parameter table
constexpr size_t kScratchBytes = kOffF32 + (f32_table_floats(1) * sizeof(float) + 255) / 256 * 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once per device).
cosmica_status scratch_address(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(COSMICA_ERR_INVALID, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_addr[dev] = p;
    }
    *out = (unsigned char *)g_addr[dev];
    return COSMICA_OK;
}

}  // namespace

extern "C" cosmica_status cosmica_propagate_noalloc(const cosmica_params *params, const cosmica_species *species,
                                                    const double *T_in, uint32_t n_energies,
                                                    const uint32_t *n_per_energy, uint64_t seed,
                                                    cosmica_exit_states *out, void *stream)
{
    cosmica_status st = check_params(params);
    if (st != COSMICA_OK) return st;
    st = check_species(species);
    if (st != COSMICA_OK) return st;
    if (n_energies > kMaxE)
        return fail(COSMICA_ERR_INVALID, "cosmica_propagate_noalloc: %u energies exceed the fixed scratch limit of %u",
                    n_energies, kMaxE);
    if (n_energies > 0 && (!T_in || !n_per_energy)) return fail(COSMICA_ERR_INVALID, "T_in / n_per_energy NULL");
    if (!out) return fail(COSMICA_ERR_INVALID, "out is NULL");
    // tables on the stack: no heap or device allocation anywhere in this call
    DevItem items[kMaxE];
    uint64_t prefix[kMaxE + 1];
    prefix[0] = 0;
    for (uint32_t e = 0; e < n_energies; ++e) {
        if (!(std::isfinite(T_in[e]) && T_in[e] > 0.0)) return fail(COSMICA_ERR_INVALID, "T_in[%u] must be > 0", e);
        items[e] = make_item(T_in[e], prefix[e], seed, 0u, 0u, params->r0_AU, params->th0_rad, params->ph0_rad, e);
        prefix[e + 1] = prefix[e] + n_per_energy[e];
    }
    const uint64_t total = prefix[n_energies];
    if (out->n != total)
        return fail(COSMICA_ERR_INVALID, "out->n = %llu, sum(n_per_energy) = %llu", (unsigned long long)out->n,
                    (unsigned long long)total);
    if (total == 0) return COSMICA_OK;
    if (!out->r || !out->th || !out->ph || !out->lnP || !out->s || !out->steps || !out->status || !out->item)
        return fail(COSMICA_ERR_INVALID, "exit-state arrays must be non-NULL");
    if (!is_device_ptr(out->r)) return fail(COSMICA_ERR_INVALID, "cosmica_propagate_noalloc needs device exit states");
    if (params->formulation == 1 && !out->lw) return fail(COSMICA_ERR_INVALID, "the energy form needs out->lw");

    unsigned char *base = nullptr;
    st = scratch_address(&base);
    if (st != COSMICA_OK) return st;
    DevParams *d_prm = (DevParams *)(base + kOffParams);
    DevSpecies *d_spc = (DevSpecies *)(base + kOffSpecies);
    DevItem *d_items = (DevItem *)(base + kOffItems);
    uint64_t *d_prefix = (uint64_t *)(base + kOffPrefix);
    unsigned long long *d_counters = (unsigned long long *)(base + kOffCounters);
    float *d_f32 = (float *)(base + kOffF32);

    cudaStream_t s = (cudaStream_t)stream;
    const DevParams hp = to_dev(*params);
    const DevSpecies hs = to_dev(*species);
    // pageable sources: each copy has consumed its source when the call returns
    cudaError_t e = cudaMemcpyAsync(d_prm, &hp, sizeof(hp), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_spc, &hs, sizeof(hs), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_items, items, n_energies * sizeof(DevItem), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_prefix, prefix, (n_energies + 1) * sizeof(uint64_t),
                                              cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_counters, 0, 2 * sizeof(unsigned long long), s);
    if (e == cudaSuccess) e = launch_derive(d_prm, 1, s);
    if (e == cudaSuccess) e = launch_f32_table(d_prm, 1, d_f32, s);
    if (e != cudaSuccess) return cuda_fail(e, "cosmica_propagate_noalloc set-up");

    LaunchArgs a{d_prm, d_spc, d_items, d_prefix, n_energies, total,
                 ExitPtrs{out->r, out->th, out->ph, out->lnP, out->s, out->steps, out->status, out->item, out->lw},
                 d_counters + 1, d_counters, nullptr, d_prefix, d_f32};
    if (params->precision == COSMICA_PREC_FP64) {
        e = launch_propagate_fp64(a, s);
    } else {
        const unsigned block = 128;
        const MixedVariant v{params->precision, params->formulation == 1,
                             params->n_shells > 0 || params->squashed != 0, full_model(*params)};
        const int bps = std::max(1, mixed_max_blocks_per_sm(v, block, true));
        uint64_t grid = (uint64_t)num_sms() * (uint64_t)bps;
        grid = std::max<uint64_t>(1, std::min<uint64_t>(grid, (total + block - 1) / block));
        e = launch_propagate_mixed(a, v, PersistentShape{block, (unsigned)grid, 64u}, s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "cosmica_propagate_noalloc launch");
    return COSMICA_OK;
}
