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
//     rejected with COSMICA_ERR_INVALID); the array is about 95 KB (kScratchBytes,
//     checked at compile time) and every GPU that loads the library holds it
//     until the process exits;
//   * the exit states must be device memory (no host staging is possible
//     without allocating);
//   * the tables reach the array as kernel parameters (small fixed-size chunks,
//     built in a few KB of the caller's stack), never as copies from host
//     memory, so nothing the call leaves on the stream refers to host memory
//     that the call has given back;
//   * the array's device address is looked up (cudaGetSymbolAddress, with the
//     device current) whenever the stream is not capturing, so a re-created
//     context is followed; under capture the address found by an earlier call
//     on that device is used, so make a first call on each device before any
//     stream capture.  That first call may also make the CUDA driver load the
//     library's device code (lazy module loading), which allocates on the
//     driver's side: make it during set-up;
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
static_assert(kScratchBytes <= 96 * 1024, "the documented size of the static scratch is about 95 KB");
static_assert(sizeof(DevSpecies) <= 256, "species region");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Tables travel as kernel parameters, in chunks well below the 4 KB parameter space.
constexpr uint32_t kChunkItems = 40;
struct HeadChunk {
    DevParams prm;
    DevSpecies spc;
};
struct ItemChunk {
    uint32_t first, n;                      // items first .. first + n - 1
    DevItem items[kChunkItems];
    uint64_t prefix_end[kChunkItems];       // prefix[first + i + 1]
};
static_assert(sizeof(HeadChunk) + 16 <= 4000 && sizeof(ItemChunk) + 16 <= 4000, "kernel parameter space");

// the parameter block and species; clears the queue cursor and step counter, sets prefix[0] = 0
__global__ void k_noalloc_head(const HeadChunk h)
{
    const uint32_t i = threadIdx.x;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(&h.prm);
    uint32_t *dst = reinterpret_cast<uint32_t *>(g_noalloc_scratch + kOffParams);
    for (uint32_t w = i; w < sizeof(DevParams) / 4; w += blockDim.x) dst[w] = src[w];
    const uint32_t *ss = reinterpret_cast<const uint32_t *>(&h.spc);
    uint32_t *sd = reinterpret_cast<uint32_t *>(g_noalloc_scratch + kOffSpecies);
    for (uint32_t w = i; w < sizeof(DevSpecies) / 4; w += blockDim.x) sd[w] = ss[w];
    if (i == 0) {
        unsigned long long *c = reinterpret_cast<unsigned long long *>(g_noalloc_scratch + kOffCounters);
        c[0] = 0ull;
        c[1] = 0ull;
        reinterpret_cast<uint64_t *>(g_noalloc_scratch + kOffPrefix)[0] = 0ull;
    }
}

// one chunk of work items and their prefix sums
__global__ void k_noalloc_items(const ItemChunk c)
{
    const uint32_t i = threadIdx.x;
    if (i >= c.n) return;
    reinterpret_cast<DevItem *>(g_noalloc_scratch + kOffItems)[c.first + i] = c.items[i];
    reinterpret_cast<uint64_t *>(g_noalloc_scratch + kOffPrefix)[c.first + i + 1] = c.prefix_end[i];
}

static_assert(sizeof(DevParams) % 4 == 0 && sizeof(DevSpecies) % 4 == 0, "word copies");

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device: looked up again on every call
// whose stream is not capturing (it changes if the context is re-created), taken from the
// last lookup on this device while the stream captures.
cosmica_status scratch_address(cudaStream_t s, unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(COSMICA_ERR_INVALID, "device ordinal %d out of range", dev);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(s, &cap);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamIsCapturing");
    std::lock_guard<std::mutex> lk(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-alloc scratch)");
        g_addr[dev] = p;
    } else if (!g_addr[dev]) {
        return fail(COSMICA_ERR_INVALID,
                    "cosmica_propagate_noalloc: make a first call on this device before any stream capture");
    }
    *out = (unsigned char *)g_addr[dev];
    return COSMICA_OK;
}

cudaError_t launch_head(const HeadChunk &h, cudaStream_t s)
{
    cudaGetLastError();
    k_noalloc_head<<<1, 128, 0, s>>>(h);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_items(const ItemChunk &c, cudaStream_t s)
{
    cudaGetLastError();
    k_noalloc_items<<<1, kChunkItems, 0, s>>>(c);
    note_launch();
    return cudaGetLastError();
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
    uint64_t total = 0;
    for (uint32_t e = 0; e < n_energies; ++e) {
        if (!(std::isfinite(T_in[e]) && T_in[e] > 0.0)) return fail(COSMICA_ERR_INVALID, "T_in[%u] must be > 0", e);
        total += n_per_energy[e];
    }
    if (out->n != total)
        return fail(COSMICA_ERR_INVALID, "out->n = %llu, sum(n_per_energy) = %llu", (unsigned long long)out->n,
                    (unsigned long long)total);
    if (total == 0) return COSMICA_OK;
    if (!out->r || !out->th || !out->ph || !out->lnP || !out->s || !out->steps || !out->status || !out->item)
        return fail(COSMICA_ERR_INVALID, "exit-state arrays must be non-NULL");
    if (!is_device_ptr(out->r)) return fail(COSMICA_ERR_INVALID, "cosmica_propagate_noalloc needs device exit states");
    if (params->formulation == 1 && !out->lw) return fail(COSMICA_ERR_INVALID, "the energy form needs out->lw");

    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    st = scratch_address(s, &base);
    if (st != COSMICA_OK) return st;
    DevParams *d_prm = (DevParams *)(base + kOffParams);
    DevSpecies *d_spc = (DevSpecies *)(base + kOffSpecies);
    DevItem *d_items = (DevItem *)(base + kOffItems);
    uint64_t *d_prefix = (uint64_t *)(base + kOffPrefix);
    unsigned long long *d_counters = (unsigned long long *)(base + kOffCounters);
    float *d_f32 = (float *)(base + kOffF32);

    // tables as kernel parameters: the head, then the items in chunks (a few KB of stack)
    HeadChunk head;
    head.prm = to_dev(*params);
    head.spc = to_dev(*species);
    cudaError_t e = launch_head(head, s);
    ItemChunk chunk;
    uint64_t run = 0;
    for (uint32_t first = 0; e == cudaSuccess && first < n_energies; first += kChunkItems) {
        chunk.first = first;
        chunk.n = std::min(kChunkItems, n_energies - first);
        for (uint32_t i = 0; i < chunk.n; ++i) {
            const uint32_t k = first + i;
            chunk.items[i] = make_item(T_in[k], run, seed, 0u, 0u, params->r0_AU, params->th0_rad, params->ph0_rad, k);
            run += n_per_energy[k];
            chunk.prefix_end[i] = run;
        }
        e = launch_items(chunk, s);
    }
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
