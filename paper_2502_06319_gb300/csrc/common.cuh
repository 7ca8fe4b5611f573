// common.cuh -- device-side records shared by the kernels of libcosmica.
//
// DevParams holds one heliosphere (one cosmica_params) twice: the raw FP64
// values, from which the FP64 step derives every quantity in the same order
// as its definition, and a block of FP32 constants pre-derived for the mixed
// step.  The derived block is filled on the device by k_derive (FP64 unit,
// deterministic elementary functions) so that host and device never disagree
// on a constant.
#pragma once
#include <cstddef>
#include <cstdint>

#include "cosmica.h"

namespace cosmica {

constexpr double kPi = 3.141592653589793;
constexpr double kTwoPi = 6.283185307179586;
constexpr double kAU_m = 1.495978707e11;   // metres per AU
constexpr double kAU_km = 1.495978707e8;   // kilometres per AU
constexpr double kDay_s = 86400.0;         // seconds per day
constexpr double kC_ms = 299792458.0;      // speed of light
constexpr double kDeg = 0.017453292519943295;
constexpr double kLn10 = 2.302585092994046;

// FP32 constants of one heliosphere for the mixed-precision step.  The
// isotropic model is expressed through the same fields (Omega = 0,
// kperp fractions 1, one wind speed, no drift), so the step has no branch on it.
struct alignas(16) F32Params {
    float Vs, dV;              // slow wind and (fast - slow) [AU/day]
    float lat_f, inv_dlat;     // transition latitude [rad], 1/width [1/rad]
    float Omega;               // rotation rate [rad/day] (0 for isotropic)
    float K0;                  // AU^2/day
    float er, et;              // perpendicular fractions
    float ts_drop, R_ts, inv_dts;   // termination shock (ts_drop = 0: none)
    float r_in;
    float dt_max, dt_fixed, dt_min;
    float eps_adv2, eps_diff;  // 2 eps_adv, eps_diff
    float CA0;                 // kappa_A prefactor: C_A = CA0 * beta * P  [AU^2/day]
    float D2;                  // 2 r_L / r = D2 * P * r / sqrt(1 + Gamma^2)
    float dcs_min;             // sheet half-width floor [rad]
    float ta, ta2;             // tan(tilt), tan^2(tilt)
    float polarity;            // +1 / -1
    float drift, hcs;          // 0 / 1
    float sqrt2er;             // sqrt(2 er)
    float pad0, pad1;
    // radial shells (n_sh = 0: none); edge e at e * sh_dr, blend half-width sh_w
    float n_sh, sh_dr, sh_inv_dr, sh_w, sh_inv_2w;
    float pad2, pad3, pad4;
    float sh_K0[COSMICA_MAX_SHELLS];      // AU^2/day
    float sh_alpha[COSMICA_MAX_SHELLS];   // sheet tilt [rad]
    // nose-squashed spheroids (sq = 0: spheres): nose direction, and per surface the
    // centre offset c behind the Sun and 1/a^2, 1/b^2 of its semi-axes
    // (the shock's spheroid in units of its nose distance ts_R, C = c^2/a^2 - 1)
    float sq, nose_ph, sin_nth, cos_nth;
    float ts_R, ts_c, ts_ia2, ts_ib2, ts_C, hp_c, hp_ia2, hp_ib2;
};

struct DevParams {
    // raw values (FP64 step)
    double K0, er, et, B1AU, Vs_kms, Vf_kms, lat_fast_deg, tilt_deg, polarity;
    double drift_on, hcs_on, isotropic;
    double R_out, R_ts, ts_f, r_in, dt_max, dt_fixed, dt_min, eps_adv, eps_diff;
    double V_const_kms, dlat_deg, dts, dcs_min_deg, rot_period, r0, th0, ph0, max_steps;
    double formulation;        // 0 momentum form, 1 energy form
    double n_shells, shell_w;  // radial shells (0: one region), blend half-width [AU]
    double squashed, nose_th, nose_ph, ts_tail, ts_flank, hp_tail, hp_flank;   // nose-squashed surfaces
    double shell_K0[COSMICA_MAX_SHELLS], shell_tilt_deg[COSMICA_MAX_SHELLS];
    int32_t precision, pad;
    // derived on the device
    double B0;                 // nT, |B|(1 AU, equator) = B1AU
    F32Params f;
};

// Read-only view of one parameter set's FP32 block in a table where the block's
// fields come in quads (four consecutive fields, 16 bytes) and consecutive quads
// lie 4 S floats apart (a compile-time stride, so every field is an immediate
// offset from one 16-byte-aligned per-lane pointer, and the fields of a quad read
// together can be fetched by one 16-byte load).  S = 1 reads one F32Params in
// place.  The mixed kernels read the paged table (S = kSetsPerPage): page k holds
// sets 64k .. 64k+63, quad g of set i at k * kF32Fields * 64 + g * 64 * 4 +
// (i mod 64) * 4, so the lanes of a warp reading one field of different sets
// touch a few adjacent lines instead of one line per set (and different L1 banks).
template <uint32_t S>
struct P32 {
    const float *__restrict__ p;   // field 0 of the set, 16-byte aligned
    __device__ __forceinline__ float at(uint32_t field) const
    {
        const float *__restrict__ a = static_cast<const float *>(__builtin_assume_aligned(p, 16));
        return a[(field >> 2) * (4u * S) + (field & 3u)];
    }
};
constexpr uint32_t kSetsPerPage = 64;
#define P32F(q, m) ((q).at((uint32_t)(offsetof(F32Params, m) / sizeof(float))))
#define P32A(q, m, k) ((q).at((uint32_t)(offsetof(F32Params, m) / sizeof(float)) + (uint32_t)(k)))
constexpr uint32_t kF32Fields = sizeof(F32Params) / sizeof(float);
// floats of the paged field-major table for n sets, and the offset of set i's field 0
__host__ __device__ constexpr size_t f32_table_floats(uint32_t n)
{
    return (size_t)((n + kSetsPerPage - 1) / kSetsPerPage) * kF32Fields * kSetsPerPage;
}
__host__ __device__ constexpr size_t f32_table_offset(uint32_t i)
{
    return (size_t)(i / kSetsPerPage) * kF32Fields * kSetsPerPage + (size_t)(i % kSetsPerPage) * 4;
}
static_assert(kF32Fields % 4 == 0, "F32Params holds whole quads");
static_assert(sizeof(F32Params) % sizeof(float) == 0, "F32Params holds floats only");

struct DevSpecies {
    double A, Z, m0;           // as doubles, the FP64 step's arithmetic type
    float aoz_m0_sq;           // (A/|Z| m0)^2 [GV^2] for beta = P / sqrt(P^2 + M^2)
    float sgnq;                // sign of the charge
    float aoz;                 // A/|Z|
    float pad;
};

struct DevItem {
    double T;                  // GeV/n
    uint64_t first_pid;
    uint64_t seed;
    uint32_t param_idx, species_idx;
    double r0, th0, ph0;       // start position (detection point) of the item's particles
    uint32_t out_item;         // value written to the exit record's item field
    uint32_t pad;
};

struct ExitPtrs {
    double *r, *th, *ph, *lnP, *s;
    uint32_t *steps;
    uint8_t *status;
    uint32_t *item;
    double *lw;                // log loss weight (energy form), may be null
};

// Index of the work item owning global particle g: prefix[i] <= g < prefix[i+1].
__device__ __forceinline__ uint32_t find_item(const uint64_t *__restrict__ prefix, uint32_t n_items,
                                              uint64_t g)
{
    uint32_t lo = 0, hi = n_items;        // invariant: prefix[lo] <= g < prefix[hi]
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (__ldg(prefix + mid) <= g) lo = mid; else hi = mid;
    }
    return lo;
}

}  // namespace cosmica
