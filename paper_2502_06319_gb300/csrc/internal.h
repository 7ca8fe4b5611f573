// internal.h -- declarations shared by the translation units of libcosmica
// (launchers implemented in the kernel files, called by the C-ABI layer).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

#include "common.cuh"

namespace cosmica {

constexpr int kDebugEvalN = 21;   // quantities written per state by the debug evaluators

struct LaunchArgs {
    const DevParams *prm;
    const DevSpecies *spc;
    const DevItem *items;
    const uint64_t *prefix;
    uint32_t n_items;
    uint64_t n_total;
    ExitPtrs out;
    unsigned long long *steps_total;   // may be null
    unsigned long long *cursor;        // work-queue cursor (persistent kernels)
    const uint32_t *qitem;             // item of each queue slot (null: item order)
    const uint64_t *qprefix;           // prefix sums of particle counts in queue order
    const float *f32;                  // FP32 blocks of the parameter sets, paged field-major (P32)
};

struct PersistentShape {
    unsigned block;
    unsigned grid;
    unsigned compact_period;   // 0: no block compaction
};

// ---- continuous-batching server -------------------------------------------
// fresh particles of one (request, energy) slice, offered to one quantum
struct ServeItem {
    double T;                  // GeV/n
    uint64_t first_pid;        // pid of the slice's first particle
    uint64_t seed;
    uint64_t exit_idx;         // exit-arena index of the slice's first particle
    uint32_t slot;             // request slot: parameter set and species index
    uint32_t energy;           // energy index within the request
};

// an in-flight particle between two quanta (exact state)
struct Suspended {
    union {
        float f[10];           // compensated pairs (r, th, ph, lnP, s)
        double d[5];           // FP64 accumulation
    };
    uint32_t k, slot, energy, pad;
    uint64_t pid, seed, exit_idx;
};

struct ServeArgs {
    const DevParams *prm;      // per slot
    const DevSpecies *spc;     // per slot
    const ServeItem *items;
    const uint64_t *prefix;
    uint32_t n_items;
    uint64_t n_fresh;
    const Suspended *resume;
    uint64_t n_resume;
    Suspended *suspend;
    unsigned int *n_suspend;
    unsigned long long *cursors;   // [0] fresh, [1] resume
    ExitPtrs arena;
    unsigned int *req_done;        // per slot
    unsigned long long *req_steps; // per slot
    uint32_t budget;               // steps per lane per quantum
};

// full: every resident request is the full model (the variant without uniform branches)
cudaError_t launch_serve(const ServeArgs &a, int acc, bool ext, bool full, PersistentShape shape, cudaStream_t s);
int serve_max_blocks_per_sm(int acc, bool ext, bool full, unsigned block);

void note_launch();

cudaError_t launch_derive(DevParams *prm, uint32_t n, cudaStream_t s);
cudaError_t launch_f32_table(const DevParams *prm, uint32_t n, float *table, cudaStream_t s);
cudaError_t launch_propagate_fp64(const LaunchArgs &a, cudaStream_t s);

// mixed precision persistent kernel; acc = COSMICA_PREC_MIXED or COSMICA_PREC_MIXED_F64ACC
// compile-time variant of the mixed kernel a launch needs
struct MixedVariant {
    int acc;        // COSMICA_PREC_MIXED or COSMICA_PREC_MIXED_F64ACC
    bool energy;    // energy formulation (Eq. 1) instead of the momentum form
    bool extended;  // some parameter set of the launch has radial shells or a squashed heliosphere
    bool full;      // every set is the full model: drift and current sheet on, adaptive step
};
// a set is the full model of the mixed kernels' FULL variant
inline bool full_model(const cosmica_params &p)
{
    return !p.isotropic && p.drift_on && p.hcs_on && !(p.dt_fixed_day > 0.0);
}
cudaError_t launch_propagate_mixed(const LaunchArgs &a, MixedVariant v, PersistentShape shape, cudaStream_t s);
int mixed_max_blocks_per_sm(MixedVariant v, unsigned block, bool compact);

cudaError_t launch_histogram(const ExitPtrs &ex, uint64_t n, uint32_t n_items, uint32_t nbins, double x_lo,
                             double dx, unsigned long long *hist, cudaStream_t s);
struct SpecItem {
    double T;                  // GeV/n
    double A, Z, m0;           // species
};
cudaError_t launch_spectrum(const unsigned long long *hist, uint32_t n_items, uint32_t nbins,
                            double x_lo, double dx, const SpecItem *items, int lis_kind,
                            const double *lis_lnT, const double *lis_lnJ, uint32_t lis_n,
                            double *J, double *sigma, cudaStream_t s);

cudaError_t launch_spectrum_unbinned(const ExitPtrs &ex, const uint64_t *prefix, uint32_t n_items,
                                     const SpecItem *items, int form, int lis_kind, const double *lis_lnT,
                                     const double *lis_lnJ, uint32_t lis_n, double *J, double *sigma, cudaStream_t s);

cudaError_t launch_debug_eval64(const DevParams *prm, const DevSpecies *spc, uint32_t n, const double *st,
                                double *out, cudaStream_t s);
cudaError_t launch_debug_eval32(const DevParams *prm, const DevSpecies *spc, uint32_t n, const double *st,
                                double *out, cudaStream_t s);
cudaError_t launch_debug_fn64(int which, uint32_t n, const double *x, double *y, cudaStream_t s);
cudaError_t launch_debug_normals64(uint64_t seed, uint64_t pid0, uint32_t n, uint32_t step, double *z,
                                   cudaStream_t s);
cudaError_t launch_debug_normals32(uint64_t seed, uint64_t pid0, uint32_t n, uint32_t step, float *z,
                                   uint32_t *words, cudaStream_t s);
cudaError_t launch_debug_philox(uint32_t n, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                                cudaStream_t s);
cudaError_t launch_debug_curand_philox(uint32_t n, uint64_t seed, const unsigned long long *subseq,
                                       const unsigned long long *offset, uint32_t *out, cudaStream_t s);

}  // namespace cosmica
