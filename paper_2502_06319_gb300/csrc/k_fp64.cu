// k_fp64.cu -- FP64 kernels.  Built with -fmad=false: every FP64 expression
// is evaluated exactly as written (no fused multiply-add contraction).
//
//   k_derive          per-parameter-set constants (FP64 and the FP32 block)
//   k_propagate_fp64  the plain FP64 path: one thread per quasi-particle
//                     (Sec. IV.A), Euler-Maruyama until the path exits
//   k_debug_*         coefficient / RNG / elementary-function probes used by
//                     the tests through cosmica_debug.h
#include <cstdint>

#include "common.cuh"
#include "internal.h"
#include "model64.cuh"

namespace cosmica {

__global__ void k_derive(DevParams *prm, uint32_t n)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    DevParams &p = prm[i];
    const bool iso = p.isotropic != 0.0;
    p.B0 = iso ? 0.0 : m64::field_B0(p);
    F32Params &f = p.f;
    const double Vs = iso ? p.V_const_kms * kDay_s / kAU_km : p.Vs_kms * kDay_s / kAU_km;
    const double Vf = iso ? Vs : p.Vf_kms * kDay_s / kAU_km;
    f.Vs = (float)Vs;
    f.dV = (float)(Vf - Vs);
    f.lat_f = (float)(p.lat_fast_deg * kDeg);
    f.inv_dlat = (float)(1.0 / (p.dlat_deg * kDeg));
    f.Omega = iso ? 0.0f : (float)(kTwoPi / p.rot_period);
    f.K0 = (float)p.K0;
    f.er = iso ? 1.0f : (float)p.er;
    f.et = iso ? 1.0f : (float)p.et;
    f.ts_drop = (p.R_ts > 0.0) ? (float)(1.0 - p.ts_f) : 0.0f;
    f.R_ts = (float)p.R_ts;
    f.inv_dts = (float)(1.0 / p.dts);
    f.r_in = (float)p.r_in;
    f.dt_max = (float)p.dt_max;
    f.dt_fixed = (float)p.dt_fixed;
    f.dt_min = (float)p.dt_min;
    f.eps_adv2 = (float)(2.0 * p.eps_adv);
    f.eps_diff = (float)p.eps_diff;
    const bool drift = !iso && p.drift_on != 0.0;
    const bool hcs = drift && p.hcs_on != 0.0;
    f.CA0 = drift ? (float)(1e9 * kDay_s / (3.0 * p.B0 * 1e-9 * kAU_m * kAU_m)) : 0.0f;
    f.D2 = iso ? 0.0f : (float)(2.0 * 1e9 / (kC_ms * p.B0 * 1e-9 * kAU_m));
    f.dcs_min = (float)(p.dcs_min_deg * kDeg);
    double sa, ca;
    dm::sincos(p.tilt_deg * kDeg, &sa, &ca);
    const double ta = sa / ca;
    f.ta = (float)ta;
    f.ta2 = (float)(ta * ta);
    f.polarity = (float)p.polarity;
    f.drift = drift ? 1.0f : 0.0f;
    f.hcs = hcs ? 1.0f : 0.0f;
    f.sqrt2er = (float)sqrt(2.0 * (double)f.er);
    f.pad0 = f.pad1 = 0.0f;
    const int ns = (int)p.n_shells;
    const double dR = ns > 0 ? ((p.R_ts > 0.0) ? p.R_ts : p.R_out) / ns : 1.0;
    f.n_sh = (float)ns;
    f.sh_dr = (float)dR;
    f.sh_inv_dr = (float)(1.0 / dR);
    f.sh_w = (float)p.shell_w;
    f.sh_inv_2w = ns > 1 ? (float)(1.0 / (2.0 * p.shell_w)) : 0.0f;
    f.pad2 = f.pad3 = f.pad4 = 0.0f;
    for (int k = 0; k < COSMICA_MAX_SHELLS; ++k) {
        f.sh_K0[k] = (float)p.shell_K0[k];
        f.sh_alpha[k] = (float)(p.shell_tilt_deg[k] * kDeg);
    }
    const bool sq = p.squashed != 0.0;
    f.sq = sq ? 1.0f : 0.0f;
    f.nose_ph = (float)(p.nose_ph - kTwoPi * floor(p.nose_ph / kTwoPi));
    f.sin_nth = (float)sin(p.nose_th);
    f.cos_nth = (float)cos(p.nose_th);
    {
        // shock spheroid with unit nose distance (scaled by ts_R), outer spheroid in AU
        const double a = (1.0 + p.ts_tail) / 2.0, b = p.ts_flank, c = (p.ts_tail - 1.0) / 2.0;
        f.ts_R = (float)p.R_ts;
        f.ts_c = (float)c;
        f.ts_ia2 = (float)(1.0 / (a * a));
        f.ts_ib2 = (float)(1.0 / (b * b));
        f.ts_C = (float)(c * c / (a * a) - 1.0);
        const double A = p.R_out * (1.0 + p.hp_tail) / 2.0, B = p.R_out * p.hp_flank;
        f.hp_c = (float)(p.R_out * (p.hp_tail - 1.0) / 2.0);
        f.hp_ia2 = (float)(1.0 / (A * A));
        f.hp_ib2 = (float)(1.0 / (B * B));
    }
}

__global__ void __launch_bounds__(128) k_propagate_fp64(const DevParams *__restrict__ prm,
                                                        const DevSpecies *__restrict__ spc,
                                                        const DevItem *__restrict__ items,
                                                        const uint64_t *__restrict__ prefix,
                                                        uint32_t n_items, uint64_t n_total,
                                                        ExitPtrs out,
                                                        unsigned long long *__restrict__ steps_total)
{
    const uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long my_steps = 0;
    if (g < n_total) {
        const uint32_t it = find_item(prefix, n_items, g);
        const DevItem item = items[it];
        const DevParams &p = prm[item.param_idx];
        const DevSpecies sp = spc[item.species_idx];
        const uint64_t pid = item.first_pid + (g - prefix[it]);
        m64::State x;
        m64::init_state(sp, item.T, item.r0, item.th0, item.ph0, x);
        while (x.status == COSMICA_PATH_RUNNING) m64::em_step(p, sp, item.seed, pid, x);
        out.r[g] = x.r;
        out.th[g] = x.th;
        out.ph[g] = x.ph;
        out.lnP[g] = x.lnP;
        out.s[g] = x.s;
        out.steps[g] = x.k;
        out.status[g] = (uint8_t)x.status;
        out.item[g] = item.out_item;
        if (out.lw) out.lw[g] = -x.Lam;
        my_steps = x.k;
    }
    if (steps_total) {
        for (int o = 16; o > 0; o >>= 1) my_steps += __shfl_down_sync(0xffffffffu, my_steps, o);
        if ((threadIdx.x & 31) == 0 && my_steps) atomicAdd(steps_total, my_steps);
    }
}

// ---------------------------------------------------------------- debug --
__global__ void k_debug_eval64(const DevParams *__restrict__ prm, const DevSpecies *__restrict__ spc,
                               uint32_t n, const double *__restrict__ st, double *__restrict__ out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    m64::Coef c;
    m64::eval(prm[0], spc[0], st[4 * i + 0], st[4 * i + 1], st[4 * i + 2], st[4 * i + 3], c);
    double *o = out + (size_t)i * kDebugEvalN;
    o[0] = c.V;   o[1] = c.Gam;  o[2] = c.Kpar; o[3] = c.K00;  o[4] = c.K11;  o[5] = c.K22;
    o[6] = c.K02; o[7] = c.Ar;   o[8] = c.Ath;  o[9] = c.Aph;  o[10] = c.l00; o[11] = c.l11;
    o[12] = c.l20; o[13] = c.l22; o[14] = c.h;  o[15] = c.delta_cs;
    o[16] = c.vd0; o[17] = c.vd1; o[18] = c.vd2; o[19] = c.dlnP; o[20] = c.dt;
}

__global__ void k_debug_fn64(int which, uint32_t n, const double *__restrict__ x, double *__restrict__ y)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s, c;
    switch (which) {
    case 0: y[i] = dm::exp(x[i]); break;
    case 1: y[i] = dm::log(x[i]); break;
    case 2: dm::sincos(x[i], &s, &c); y[i] = s; break;
    case 3: dm::sincos(x[i], &s, &c); y[i] = c; break;
    case 4: y[i] = dm::tanh(x[i]); break;
    default: y[i] = dm::atan(x[i]); break;
    }
}

__global__ void k_debug_normals64(uint64_t seed, uint64_t pid0, uint32_t n, uint32_t step, double *z)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    m64::normals(seed, pid0 + i, step, z + 3 * (size_t)i);
}

__global__ void k_debug_philox(uint32_t n, const uint32_t *__restrict__ ctr, uint32_t k0, uint32_t k1,
                               uint32_t *__restrict__ out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
    const uint4 w = philox4x32_10(c, k0, k1);
    out[4 * i] = w.x; out[4 * i + 1] = w.y; out[4 * i + 2] = w.z; out[4 * i + 3] = w.w;
}

// ---------------------------------------------------------------- launchers --
static inline unsigned grid_for(uint64_t n, unsigned block) { return (unsigned)((n + block - 1) / block); }

// Paged copy of the FP32 blocks of n parameter sets in quads (see P32): one
// thread per (set, field); the unused slots of the last page stay as they are.
__global__ void k_f32_table(const DevParams *__restrict__ prm, uint32_t n, float *__restrict__ table)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n * kF32Fields) return;
    const uint32_t i = j / kF32Fields, f = j - i * kF32Fields;
    table[f32_table_offset(i) + (size_t)(f >> 2) * kSetsPerPage * 4 + (f & 3)] =
        reinterpret_cast<const float *>(&prm[i].f)[f];
}

cudaError_t launch_f32_table(const DevParams *prm, uint32_t n, float *table, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaGetLastError();
    k_f32_table<<<grid_for(n * kF32Fields, 128), 128, 0, s>>>(prm, n, table);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_derive(DevParams *prm, uint32_t n, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaGetLastError();
    k_derive<<<grid_for(n, 64), 64, 0, s>>>(prm, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_propagate_fp64(const LaunchArgs &a, cudaStream_t s)
{
    if (a.n_total == 0) return cudaSuccess;
    cudaGetLastError();
    k_propagate_fp64<<<grid_for(a.n_total, 128), 128, 0, s>>>(a.prm, a.spc, a.items, a.prefix, a.n_items,
                                                             a.n_total, a.out, a.steps_total);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_debug_eval64(const DevParams *prm, const DevSpecies *spc, uint32_t n, const double *st,
                                double *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaGetLastError();
    k_debug_eval64<<<grid_for(n, 128), 128, 0, s>>>(prm, spc, n, st, out);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_debug_fn64(int which, uint32_t n, const double *x, double *y, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaGetLastError();
    k_debug_fn64<<<grid_for(n, 256), 256, 0, s>>>(which, n, x, y);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_debug_normals64(uint64_t seed, uint64_t pid0, uint32_t n, uint32_t step, double *z,
                                   cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaGetLastError();
    k_debug_normals64<<<grid_for(n, 256), 256, 0, s>>>(seed, pid0, n, step, z);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_debug_philox(uint32_t n, const uint32_t *ctr, uint32_t k0, uint32_t k1, uint32_t *out,
                                cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaGetLastError();
    k_debug_philox<<<grid_for(n, 256), 256, 0, s>>>(n, ctr, k0, k1, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace cosmica
