// cosmica_api.cu -- the C ABI of libcosmica (cosmica.h, cosmica_debug.h).
//
// Host-side responsibilities only: argument validation, packing of the small
// per-call tables (species, work items, prefix sums) into pinned staging
// memory, their asynchronous upload into device scratch owned by the handle,
// kernel launches on the caller's stream, staging of host-resident exit
// buffers, CUDA-graph capture of repeated batched launches, and the launch
// shape autotuner.  Every numeric step of the path runs in the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <vector>

#include "common.cuh"
#include "cosmica.h"
#include "cosmica_debug.h"
#include "host_util.h"
#include "internal.h"

using namespace cosmica;

// ------------------------------------------------------------------ errors --
namespace cosmica {
namespace host {
thread_local char g_err[512] = "";
std::atomic<unsigned long long> g_launches{0};

cosmica_status fail(cosmica_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

cosmica_status cuda_fail(cudaError_t e, const char *what)
{
    cudaGetLastError();   // a reported failure must not resurface at a later launch check
    if (e == cudaErrorMemoryAllocation)
        return fail(COSMICA_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(COSMICA_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}


size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

bool is_device_ptr(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Outside the outer boundary: r >= R_out, or outside the squashed outer spheroid.
static bool outside_host(const cosmica_params &p, double r, double th, double ph)
{
    if (!p.squashed) return r >= p.R_out_AU;
    const double mu = std::sin(th) * std::sin(p.nose_th_rad) * std::cos(ph - p.nose_ph_rad) +
                      std::cos(th) * std::cos(p.nose_th_rad);
    const double a = p.R_out_AU * (1.0 + p.hp_tail_ratio) / 2.0, b = p.R_out_AU * p.hp_flank_ratio;
    const double c = p.R_out_AU * (p.hp_tail_ratio - 1.0) / 2.0;
    const double xa = r * mu + c;
    return xa * xa / (a * a) + r * r * (1.0 - mu * mu) / (b * b) >= 1.0;
}

cosmica_status check_params(const cosmica_params *p)
{
    if (!p) return fail(COSMICA_ERR_INVALID, "params is NULL");
    if (p->struct_size != sizeof(cosmica_params))
        return fail(COSMICA_ERR_INVALID, "params.struct_size %u != %zu", p->struct_size, sizeof(cosmica_params));
    if (p->version != COSMICA_ABI_VERSION)
        return fail(COSMICA_ERR_INVALID, "params.version %u != %u", p->version, COSMICA_ABI_VERSION);
    auto pos = [](double x) { return std::isfinite(x) && x > 0.0; };
    if (!pos(p->K0)) return fail(COSMICA_ERR_INVALID, "K0 must be > 0");
    if (p->squashed != 0 && p->squashed != 1) return fail(COSMICA_ERR_INVALID, "squashed must be 0 or 1");
    if (p->squashed && !(pos(p->ts_tail_ratio) && pos(p->ts_flank_ratio) && pos(p->hp_tail_ratio) &&
                         pos(p->hp_flank_ratio) && std::isfinite(p->nose_th_rad) && std::isfinite(p->nose_ph_rad)))
        return fail(COSMICA_ERR_INVALID, "squashed heliosphere needs positive tail/flank ratios and a nose direction");
    if (!(p->r_in_AU > 0.0 && p->r0_AU >= p->r_in_AU && pos(p->R_out_AU)))
        return fail(COSMICA_ERR_INVALID, "need 0 < r_in <= r0 and R_out > 0");
    if (outside_host(*p, p->r0_AU, p->th0_rad, p->ph0_rad))
        return fail(COSMICA_ERR_INVALID, "the start point lies outside the outer boundary");
    if (!(p->th0_rad > 0.0 && p->th0_rad < kPi)) return fail(COSMICA_ERR_INVALID, "th0 must lie in (0, pi)");
    if (!std::isfinite(p->ph0_rad)) return fail(COSMICA_ERR_INVALID, "ph0 must be finite");
    if (!(p->dt_fixed_day > 0.0) && !(pos(p->dt_max_day) && pos(p->dt_min_day) && p->dt_min_day <= p->dt_max_day))
        return fail(COSMICA_ERR_INVALID, "need dt_fixed > 0 or 0 < dt_min <= dt_max");
    if (std::isinf(p->dt_fixed_day)) return fail(COSMICA_ERR_INVALID, "dt_fixed must be finite");
    if (!(p->dt_fixed_day > 0.0) && !(std::isfinite(p->eps_adv) && p->eps_adv >= 0.0 &&
                                      std::isfinite(p->eps_diff) && p->eps_diff >= 0.0))
        return fail(COSMICA_ERR_INVALID, "eps_adv and eps_diff must be finite and >= 0");
    if (p->max_steps < 1) return fail(COSMICA_ERR_INVALID, "max_steps must be >= 1");
    if (p->precision < COSMICA_PREC_FP64 || p->precision > COSMICA_PREC_MIXED_F64ACC)
        return fail(COSMICA_ERR_INVALID, "unknown precision %d", p->precision);
    if (p->formulation != 0 && p->formulation != 1)
        return fail(COSMICA_ERR_INVALID, "formulation %d: 0 (momentum) or 1 (energy)", p->formulation);
    if (p->n_shells > COSMICA_MAX_SHELLS)
        return fail(COSMICA_ERR_INVALID, "n_shells %u exceeds %u", p->n_shells, COSMICA_MAX_SHELLS);
    if (p->n_shells > 0) {
        const double edge = p->R_ts_AU > 0.0 ? p->R_ts_AU : p->R_out_AU;
        const double width = edge / (double)p->n_shells;
        if (p->n_shells > 1 && !(pos(p->shell_blend_AU) && 2.0 * p->shell_blend_AU < width))
            return fail(COSMICA_ERR_INVALID, "need 0 < 2 shell_blend_AU < shell width %g AU", width);
        for (uint32_t k = 0; k < p->n_shells; ++k) {
            if (!pos(p->shell_K0[k])) return fail(COSMICA_ERR_INVALID, "shell_K0[%u] must be > 0", k);
            if (!(std::fabs(p->shell_tilt_deg[k]) < 89.0))
                return fail(COSMICA_ERR_INVALID, "shell_tilt_deg[%u]: need |tilt| < 89 deg", k);
        }
    }
    if (!p->isotropic) {
        if (!(pos(p->V_slow_kms) && pos(p->V_fast_kms) && pos(p->B1AU_nT) && pos(p->rot_period_day) &&
              pos(p->dlat_deg)))
            return fail(COSMICA_ERR_INVALID, "wind, field, rotation and transition widths must be > 0");
        if (!(p->kperp_r_frac > 0.0 && p->kperp_th_frac > 0.0))
            return fail(COSMICA_ERR_INVALID, "perpendicular diffusion fractions must be > 0");
        if (p->polarity != 1 && p->polarity != -1) return fail(COSMICA_ERR_INVALID, "polarity must be +-1");
        if (!(std::isfinite(p->lat_fast_deg) && std::isfinite(p->tilt_deg)))
            return fail(COSMICA_ERR_INVALID, "lat_fast and tilt must be finite");
        if (p->hcs_on && !(std::fabs(p->tilt_deg) < 89.0 && pos(p->dcs_min_deg)))
            return fail(COSMICA_ERR_INVALID, "need |tilt| < 89 deg and dcs_min > 0");
        if (p->R_ts_AU > 0.0 && !(pos(p->dts_AU) && p->ts_K_factor > 0.0))
            return fail(COSMICA_ERR_INVALID, "termination shock needs dts > 0 and ts_K_factor > 0");
    } else if (!(p->V_const_kms >= 0.0)) {
        return fail(COSMICA_ERR_INVALID, "V_const must be >= 0");
    }
    return COSMICA_OK;
}

bool valid_start(const cosmica_params &p, double r0, double th0, double ph0)
{
    return std::isfinite(r0) && r0 >= p.r_in_AU && th0 > 0.0 && th0 < kPi && std::isfinite(ph0) &&
           !outside_host(p, r0, th0, ph0);
}

cosmica_status check_species(const cosmica_species *s)
{
    if (!s) return fail(COSMICA_ERR_INVALID, "species is NULL");
    if (s->A < 1 || s->Z == 0 || !(s->m0_GeV > 0.0))
        return fail(COSMICA_ERR_INVALID, "species needs A >= 1, Z != 0, m0 > 0");
    return COSMICA_OK;
}

DevParams to_dev(const cosmica_params &p)
{
    DevParams d;
    std::memset(&d, 0, sizeof(d));
    d.K0 = p.K0; d.er = p.kperp_r_frac; d.et = p.kperp_th_frac; d.B1AU = p.B1AU_nT;
    d.Vs_kms = p.V_slow_kms; d.Vf_kms = p.V_fast_kms; d.lat_fast_deg = p.lat_fast_deg;
    d.tilt_deg = p.tilt_deg; d.polarity = (double)p.polarity;
    d.drift_on = p.drift_on ? 1.0 : 0.0; d.hcs_on = p.hcs_on ? 1.0 : 0.0; d.isotropic = p.isotropic ? 1.0 : 0.0;
    d.R_out = p.R_out_AU; d.R_ts = p.R_ts_AU; d.ts_f = p.ts_K_factor; d.r_in = p.r_in_AU;
    d.dt_max = p.dt_max_day; d.dt_fixed = p.dt_fixed_day; d.dt_min = p.dt_min_day;
    d.eps_adv = p.eps_adv; d.eps_diff = p.eps_diff; d.V_const_kms = p.V_const_kms;
    d.dlat_deg = p.dlat_deg; d.dts = p.dts_AU; d.dcs_min_deg = p.dcs_min_deg; d.rot_period = p.rot_period_day;
    d.r0 = p.r0_AU; d.th0 = p.th0_rad; d.ph0 = p.ph0_rad; d.max_steps = (double)p.max_steps;
    d.formulation = (double)p.formulation;
    d.squashed = p.squashed ? 1.0 : 0.0;
    d.nose_th = p.nose_th_rad; d.nose_ph = p.nose_ph_rad;
    d.ts_tail = p.ts_tail_ratio; d.ts_flank = p.ts_flank_ratio;
    d.hp_tail = p.hp_tail_ratio; d.hp_flank = p.hp_flank_ratio;
    d.n_shells = (double)p.n_shells;
    d.shell_w = p.shell_blend_AU;
    for (uint32_t k = 0; k < COSMICA_MAX_SHELLS; ++k) {
        d.shell_K0[k] = p.shell_K0[k];
        d.shell_tilt_deg[k] = p.shell_tilt_deg[k];
    }
    d.precision = p.precision;
    return d;
}

DevSpecies to_dev(const cosmica_species &s)
{
    DevSpecies d;
    d.A = (double)s.A;
    d.Z = (double)s.Z;
    d.m0 = s.m0_GeV;
    const double aoz = (double)s.A / std::fabs((double)s.Z);
    d.aoz = (float)aoz;
    d.aoz_m0_sq = (float)(aoz * s.m0_GeV * aoz * s.m0_GeV);
    d.sgnq = s.Z > 0 ? 1.0f : -1.0f;
    d.pad = 0.0f;
    return d;
}

bool valid_exit(const cosmica_exit_states *o)
{
    return o && o->r && o->th && o->ph && o->lnP && o->s && o->steps && o->status && o->item;
}

ExitPtrs exit_ptrs(const cosmica_exit_states *o)
{
    return ExitPtrs{o->r, o->th, o->ph, o->lnP, o->s, o->steps, o->status, o->item, o->lw};
}

// Device exit buffers standing in for host-resident outputs.
struct ExitStage {
    DevBuf buf;
    cosmica_status make(uint64_t n, ExitPtrs &d, bool with_lw = false)
    {
        // up to nine arrays, each starting on a 256-byte boundary
        const size_t a8 = align_up(n * 8, 256), a4 = align_up(n * 4, 256), a1 = align_up(n, 256);
        cosmica_status st = buf.reserve((with_lw ? 6 : 5) * a8 + 2 * a4 + a1);
        if (st != COSMICA_OK) return st;
        char *p = (char *)buf.d;
        d.lw = nullptr;
        if (with_lw) {
            d.lw = (double *)p;
            p += a8;
        }
        d.r = (double *)p;   p += a8;
        d.th = (double *)p;  p += a8;
        d.ph = (double *)p;  p += a8;
        d.lnP = (double *)p; p += a8;
        d.s = (double *)p;   p += a8;
        d.steps = (uint32_t *)p; p += a4;
        d.item = (uint32_t *)p;  p += a4;
        d.status = (uint8_t *)p;
        return COSMICA_OK;
    }
    static cosmica_status copy_back(const ExitPtrs &d, const cosmica_exit_states *o, cudaStream_t s)
    {
        const uint64_t n = o->n;
        CK(cudaMemcpyAsync(o->r, d.r, n * 8, cudaMemcpyDeviceToHost, s), "D2H r");
        CK(cudaMemcpyAsync(o->th, d.th, n * 8, cudaMemcpyDeviceToHost, s), "D2H th");
        CK(cudaMemcpyAsync(o->ph, d.ph, n * 8, cudaMemcpyDeviceToHost, s), "D2H ph");
        CK(cudaMemcpyAsync(o->lnP, d.lnP, n * 8, cudaMemcpyDeviceToHost, s), "D2H lnP");
        CK(cudaMemcpyAsync(o->s, d.s, n * 8, cudaMemcpyDeviceToHost, s), "D2H s");
        CK(cudaMemcpyAsync(o->steps, d.steps, n * 4, cudaMemcpyDeviceToHost, s), "D2H steps");
        CK(cudaMemcpyAsync(o->item, d.item, n * 4, cudaMemcpyDeviceToHost, s), "D2H item");
        CK(cudaMemcpyAsync(o->status, d.status, n, cudaMemcpyDeviceToHost, s), "D2H status");
        if (o->lw && d.lw) CK(cudaMemcpyAsync(o->lw, d.lw, n * 8, cudaMemcpyDeviceToHost, s), "D2H lw");
        CK(cudaStreamSynchronize(s), "cudaStreamSynchronize(host exit states)");
        return COSMICA_OK;
    }
};

// Per-call tables: species/params are device-resident in the handle; items
// and prefix sums are uploaded each call into `tables`.
struct Tables {
    DevBuf dev;
    Staging stage;
    DevItem *items = nullptr;
    uint64_t *prefix = nullptr;
    uint32_t *qitem = nullptr;               // item of each queue slot
    uint64_t *qprefix = nullptr;             // prefix sums in queue order
    unsigned long long *counters = nullptr;   // [0] cursor, [1] steps
    uint64_t n_total = 0;
    uint32_t n_items = 0;

    // order: queue order of the items (a permutation of 0..n-1), or empty for item order
    cosmica_status build(const std::vector<DevItem> &its, const std::vector<uint64_t> &pre,
                         const std::vector<uint32_t> &order, cudaStream_t s)
    {
        const size_t nI = its.size();
        const size_t b_items = align_up(std::max<size_t>(1, nI) * sizeof(DevItem), 256);
        const size_t b_pre = align_up((nI + 1) * sizeof(uint64_t), 256);
        const size_t b_q = align_up(std::max<size_t>(1, nI) * sizeof(uint32_t), 256);
        const size_t up = b_items + 2 * b_pre + b_q;
        cosmica_status st = dev.reserve(up + 256);
        if (st != COSMICA_OK) return st;
        st = stage.reserve(up);
        if (st != COSMICA_OK) return st;
        char *h = (char *)stage.h;
        std::memcpy(h, its.data(), nI * sizeof(DevItem));
        std::memcpy(h + b_items, pre.data(), (nI + 1) * sizeof(uint64_t));
        uint32_t *hq = (uint32_t *)(h + 2 * b_pre + b_items);
        uint64_t *hqp = (uint64_t *)(h + b_items + b_pre);
        hqp[0] = 0;
        for (size_t k = 0; k < nI; ++k) {
            const uint32_t i = order.empty() ? (uint32_t)k : order[k];
            hq[k] = i;
            hqp[k + 1] = hqp[k] + (pre[i + 1] - pre[i]);
        }
        char *d = (char *)dev.d;
        items = (DevItem *)d;
        prefix = (uint64_t *)(d + b_items);
        qprefix = (uint64_t *)(d + b_items + b_pre);
        qitem = (uint32_t *)(d + b_items + 2 * b_pre);
        counters = (unsigned long long *)(d + up);
        n_items = (uint32_t)nI;
        n_total = pre[nI];
        return stage.upload(dev.d, up, s);
    }
    void release()
    {
        stage.release();
        dev.release();
    }
};

// K0 of the region holding radius r (the shell's, when the model has shells).
static double start_K0(const cosmica_params &p, double r)
{
    if (p.n_shells == 0) return p.K0;
    const double edge = p.R_ts_AU > 0.0 ? p.R_ts_AU : p.R_out_AU;
    const double k = std::floor(r / (edge / (double)p.n_shells));
    const uint32_t i = (uint32_t)std::min(std::max(k, 0.0), (double)(p.n_shells - 1));
    return p.shell_K0[i];
}

// Queue order with the longest expected paths first: items sorted by K0 beta0 P0
// ascending (a smaller diffusion coefficient at the start means more steps).
std::vector<uint32_t> cost_order(const std::vector<DevItem> &its, const cosmica_params *prm,
                                 const cosmica_species *spc)
{
    std::vector<std::pair<double, uint32_t>> key(its.size());
    for (size_t i = 0; i < its.size(); ++i) {
        const cosmica_species &sp = spc[its[i].species_idx];
        const double aoz = (double)sp.A / std::fabs((double)sp.Z);
        const double T = its[i].T;
        const double pn = std::sqrt(T * (T + 2.0 * sp.m0_GeV));
        const double P = aoz * pn;
        const double beta = pn / (T + sp.m0_GeV);
        key[i] = {start_K0(prm[its[i].param_idx], its[i].r0) * beta * P, (uint32_t)i};
    }
    std::stable_sort(key.begin(), key.end(),
                     [](const std::pair<double, uint32_t> &a, const std::pair<double, uint32_t> &b) {
                         return a.first < b.first;
                     });
    std::vector<uint32_t> order(its.size());
    for (size_t k = 0; k < its.size(); ++k) order[k] = key[k].second;
    return order;
}

// SM count of each device ordinal, looked up on first use (a process may drive
// GPUs with different SM counts; concurrent first calls store the same value)
constexpr int kMaxSmDevices = 64;
std::atomic<int> g_num_sms[kMaxSmDevices];
int num_sms()
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::atomic<int> *slot = (dev >= 0 && dev < kMaxSmDevices) ? &g_num_sms[dev] : nullptr;
    int n = slot ? slot->load(std::memory_order_relaxed) : 0;
    if (n == 0) {
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
        if (slot) slot->store(n, std::memory_order_relaxed);
    }
    return n;
}

PersistentShape shape_for(MixedVariant v, const cosmica_tuning *t, uint64_t n_total)
{
    unsigned block = (t && t->block) ? t->block : 128u;
    const unsigned period = t ? t->compact_period : 64u;
    block = std::min(256u, std::max(32u, block / 32u * 32u));
    int max_b = mixed_max_blocks_per_sm(v, block, period != 0);
    if (max_b < 1) max_b = 1;
    int bps = (t && t->blocks_per_sm) ? (int)t->blocks_per_sm : max_b;
    if (!t) {
        // no tuning given: a launch with few particles per resident lane is bound by its slowest
        // paths, which step faster when fewer warps share an SM (the autotuner picks 16 warps per
        // SM for 6e5 particles, about 5 per lane, and every resident block from 1.5e6 up)
        const uint64_t lanes = (uint64_t)num_sms() * (uint64_t)max_b * block;
        if (n_total < 8ull * lanes) bps = std::max(1, (int)(512u / block));
    }
    bps = std::min(bps, max_b);
    uint64_t grid = (uint64_t)num_sms() * (uint64_t)bps;
    const uint64_t need = (n_total + block - 1) / block;   // never more blocks than particles
    grid = std::max<uint64_t>(1, std::min(grid, need));
    return PersistentShape{block, (unsigned)grid, period};
}

}  // namespace host

void note_launch() { host::g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace cosmica

using namespace cosmica::host;

// =============================================================== model API ==
struct cosmica_model {
    cosmica_params p;
    DevParams *d_prm = nullptr;
    const float *d_f32 = nullptr;   // paged field-major FP32 block (inside the d_prm allocation)
    DevBuf spc;                 // DevSpecies[1] + spectrum items
    Staging spc_stage;
    Tables tab;
    ExitStage exit_stage;
    DevBuf spec_items;
    Staging spec_stage;
    DevBuf lis_buf;
    Staging lis_stage;
    DevBuf dbg;
};

extern "C" void cosmica_params_default(cosmica_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->struct_size = sizeof(cosmica_params);
    p->version = COSMICA_ABI_VERSION;
    p->K0 = 11.5;
    p->kperp_r_frac = 0.02;
    p->kperp_th_frac = 0.02;
    p->B1AU_nT = 5.0;
    p->V_slow_kms = 400.0;
    p->V_fast_kms = 760.0;
    p->lat_fast_deg = 30.0;
    p->tilt_deg = 20.0;
    p->polarity = 1;
    p->drift_on = 1;
    p->hcs_on = 1;
    p->isotropic = 0;
    p->R_out_AU = 100.0;
    p->R_ts_AU = 0.0;
    p->ts_K_factor = 0.5;
    p->r_in_AU = 0.1;
    p->dt_max_day = 0.1;
    p->dt_fixed_day = 0.0;
    p->dt_min_day = 1e-4;
    p->eps_adv = 0.01;
    p->eps_diff = 0.01;
    p->V_const_kms = 400.0;
    p->dlat_deg = 2.0;
    p->dts_AU = 1.0;
    p->dcs_min_deg = 1.0;
    p->rot_period_day = 25.38;
    p->r0_AU = 1.0;
    p->th0_rad = kPi / 2.0;
    p->ph0_rad = 0.0;
    p->max_steps = 100000000u;
    p->precision = COSMICA_PREC_FP64;
    p->n_shells = 0;
    p->shell_blend_AU = 0.5;
    p->squashed = 0;
    p->nose_th_rad = kPi / 2.0;
    p->nose_ph_rad = 0.0;
    p->ts_tail_ratio = p->ts_flank_ratio = p->hp_tail_ratio = p->hp_flank_ratio = 1.0;
}

// Upload n parameter sets, derive their constants on the device, and lay out
// their FP32 blocks paged field-major right after them in the same allocation
// (*f32, see P32), the layout the mixed kernels read.
static cosmica_status upload_params(const cosmica_params *ps, uint32_t n, DevParams **out, const float **f32)
{
    std::vector<DevParams> h(n);
    for (uint32_t i = 0; i < n; ++i) h[i] = to_dev(ps[i]);
    const size_t b_prm = align_up(n * sizeof(DevParams), 256);
    char *d = nullptr;
    CK(cudaMalloc(&d, b_prm + f32_table_floats(n) * sizeof(float)), "cudaMalloc(params)");
    DevParams *dp = reinterpret_cast<DevParams *>(d);
    float *table = reinterpret_cast<float *>(d + b_prm);
    cudaError_t e = cudaMemcpy(dp, h.data(), n * sizeof(DevParams), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_derive(dp, n, 0);
    if (e == cudaSuccess) e = launch_f32_table(dp, n, table, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e, "deriving parameter constants");
    }
    *out = dp;
    *f32 = table;
    return COSMICA_OK;
}

extern "C" cosmica_status cosmica_model_create(const cosmica_params *params, cosmica_model **out)
{
    if (!out) return fail(COSMICA_ERR_INVALID, "out is NULL");
    *out = nullptr;
    cosmica_status st = check_params(params);
    if (st != COSMICA_OK) return st;
    cosmica_model *m = new (std::nothrow) cosmica_model();
    if (!m) return fail(COSMICA_ERR_OOM, "host allocation of the model");
    m->p = *params;
    st = upload_params(params, 1, &m->d_prm, &m->d_f32);
    if (st != COSMICA_OK) {
        delete m;
        return st;
    }
    *out = m;
    return COSMICA_OK;
}

extern "C" void cosmica_model_destroy(cosmica_model *m)
{
    if (!m) return;
    cudaDeviceSynchronize();
    if (m->d_prm) cudaFree(m->d_prm);
    m->spc.release();
    m->spc_stage.release();
    m->tab.release();
    m->exit_stage.buf.release();
    m->spec_items.release();
    m->spec_stage.release();
    m->lis_buf.release();
    m->lis_stage.release();
    m->dbg.release();
    delete m;
}

static cosmica_status upload_species(DevBuf &buf, Staging &stage, const cosmica_species *sp, uint32_t n,
                                     cudaStream_t s, DevSpecies **out)
{
    cosmica_status st = buf.reserve(n * sizeof(DevSpecies));
    if (st != COSMICA_OK) return st;
    st = stage.reserve(n * sizeof(DevSpecies));
    if (st != COSMICA_OK) return st;
    for (uint32_t i = 0; i < n; ++i) ((DevSpecies *)stage.h)[i] = to_dev(sp[i]);
    st = stage.upload(buf.d, n * sizeof(DevSpecies), s);
    if (st != COSMICA_OK) return st;
    *out = (DevSpecies *)buf.d;
    return COSMICA_OK;
}

// Shared tail of cosmica_propagate and cosmica_propagate_orbit: upload the
// species and the item table, launch the path's kernel, copy host exits back.
static cosmica_status propagate_items(cosmica_model *m, const cosmica_species *species,
                                      const std::vector<DevItem> &its, const std::vector<uint64_t> &pre,
                                      cosmica_exit_states *out, cudaStream_t s)
{
    const uint64_t total = pre.back();
    if (out->n != total) return fail(COSMICA_ERR_INVALID, "out->n = %llu, sum(n_per_energy) = %llu",
                                     (unsigned long long)out->n, (unsigned long long)total);
    if (total == 0) return COSMICA_OK;
    if (!valid_exit(out)) return fail(COSMICA_ERR_INVALID, "exit-state arrays must be non-NULL");
    if (m->p.formulation == 1 && !out->lw) return fail(COSMICA_ERR_INVALID, "the energy form needs out->lw");

    DevSpecies *d_sp = nullptr;
    cosmica_status st = upload_species(m->spc, m->spc_stage, species, 1, s, &d_sp);
    if (st != COSMICA_OK) return st;
    st = m->tab.build(its, pre, cost_order(its, &m->p, species), s);
    if (st != COSMICA_OK) return st;

    const bool host_out = !is_device_ptr(out->r);
    ExitPtrs ex = exit_ptrs(out);
    if (host_out) {
        st = m->exit_stage.make(total, ex, out->lw != nullptr);
        if (st != COSMICA_OK) return st;
    }
    CK(cudaMemsetAsync(m->tab.counters, 0, 2 * sizeof(unsigned long long), s), "cudaMemsetAsync(counters)");
    LaunchArgs a{m->d_prm, d_sp, m->tab.items, m->tab.prefix, m->tab.n_items, total, ex,
                 m->tab.counters + 1, m->tab.counters, m->tab.qitem, m->tab.qprefix, m->d_f32};
    cudaError_t e;
    if (m->p.precision == COSMICA_PREC_FP64) {
        e = launch_propagate_fp64(a, s);
    } else {
        const MixedVariant v{m->p.precision, m->p.formulation == 1, m->p.n_shells > 0 || m->p.squashed != 0,
                             full_model(m->p)};
        e = launch_propagate_mixed(a, v, shape_for(v, nullptr, total), s);
    }
    if (e != cudaSuccess) return cuda_fail(e, "propagation kernel launch");
    if (host_out) return ExitStage::copy_back(ex, out, s);
    return COSMICA_OK;
}

static cosmica_status check_energies(const double *T_in, uint32_t n_energies, const uint32_t *n_per_energy)
{
    if (n_energies > 0 && (!T_in || !n_per_energy)) return fail(COSMICA_ERR_INVALID, "T_in / n_per_energy NULL");
    for (uint32_t e = 0; e < n_energies; ++e)
        if (!(std::isfinite(T_in[e]) && T_in[e] > 0.0)) return fail(COSMICA_ERR_INVALID, "T_in[%u] must be > 0", e);
    return COSMICA_OK;
}

extern "C" cosmica_status cosmica_propagate(cosmica_model *m, const cosmica_species *species,
                                            const double *T_in, uint32_t n_energies, const uint32_t *n_per_energy,
                                            uint64_t seed, cosmica_exit_states *out, void *stream)
{
    if (!m) return fail(COSMICA_ERR_INVALID, "model is NULL");
    cosmica_status st = check_species(species);
    if (st != COSMICA_OK) return st;
    st = check_energies(T_in, n_energies, n_per_energy);
    if (st != COSMICA_OK) return st;
    if (!out) return fail(COSMICA_ERR_INVALID, "out is NULL");
    std::vector<DevItem> its(n_energies);
    std::vector<uint64_t> pre(n_energies + 1, 0);
    for (uint32_t e = 0; e < n_energies; ++e) {
        its[e] = make_item(T_in[e], pre[e], seed, 0u, 0u, m->p.r0_AU, m->p.th0_rad, m->p.ph0_rad, e);
        pre[e + 1] = pre[e] + n_per_energy[e];
    }
    return propagate_items(m, species, its, pre, out, (cudaStream_t)stream);
}

// Split of n particles among positions by weight (Sec. IV.A, moving detection
// point): position m takes [c_m, c_(m+1)), c_m = floor(n W_m / W), W_m the
// weights summed in order.
static void orbit_split(uint64_t n, const cosmica_position *pos, uint32_t n_pos, std::vector<uint64_t> &cut)
{
    double W = 0.0;
    for (uint32_t j = 0; j < n_pos; ++j) W += pos[j].weight;
    cut.assign(n_pos + 1, 0);
    double Wm = 0.0;
    for (uint32_t j = 0; j < n_pos; ++j) {
        cut[j] = (uint64_t)std::floor((double)n * Wm / W);
        Wm += pos[j].weight;
    }
    cut[n_pos] = n;
}

extern "C" cosmica_status cosmica_propagate_orbit(cosmica_model *m, const cosmica_species *species,
                                                  const double *T_in, uint32_t n_energies,
                                                  const uint32_t *n_per_energy, const cosmica_position *positions,
                                                  uint32_t n_positions, uint64_t seed, cosmica_exit_states *out,
                                                  void *stream)
{
    if (!m) return fail(COSMICA_ERR_INVALID, "model is NULL");
    cosmica_status st = check_species(species);
    if (st != COSMICA_OK) return st;
    st = check_energies(T_in, n_energies, n_per_energy);
    if (st != COSMICA_OK) return st;
    if (!out) return fail(COSMICA_ERR_INVALID, "out is NULL");
    if (n_positions == 0 || !positions) return fail(COSMICA_ERR_INVALID, "need at least one position");
    for (uint32_t j = 0; j < n_positions; ++j) {
        const cosmica_position &q = positions[j];
        if (!valid_start(m->p, q.r_AU, q.th_rad, q.ph_rad))
            return fail(COSMICA_ERR_INVALID, "position %u: need r_in <= r < R_out, th in (0, pi), finite ph", j);
        if (!(std::isfinite(q.weight) && q.weight > 0.0))
            return fail(COSMICA_ERR_INVALID, "position %u: weight must be > 0", j);
    }
    std::vector<DevItem> its;
    std::vector<uint64_t> pre(1, 0), cut;
    uint64_t first = 0;
    for (uint32_t e = 0; e < n_energies; ++e) {
        orbit_split(n_per_energy[e], positions, n_positions, cut);
        for (uint32_t j = 0; j < n_positions; ++j) {
            const uint64_t n = cut[j + 1] - cut[j];
            if (n == 0) continue;
            const cosmica_position &q = positions[j];
            its.push_back(make_item(T_in[e], first + cut[j], seed, 0u, 0u, q.r_AU, q.th_rad, q.ph_rad, e));
            pre.push_back(pre.back() + n);
        }
        first += n_per_energy[e];
    }
    if (its.size() > UINT32_MAX) return fail(COSMICA_ERR_INVALID, "too many (energy, position) items");
    return propagate_items(m, species, its, pre, out, (cudaStream_t)stream);
}

// ============================================================ spectrum API ==
static cosmica_status check_bins(const cosmica_bins *b, double *x_lo, double *dx)
{
    if (!b) return fail(COSMICA_ERR_INVALID, "bins is NULL");
    if (!(b->P_min_GV > 0.0 && b->P_max_GV > b->P_min_GV && b->nbins >= 1))
        return fail(COSMICA_ERR_INVALID, "need 0 < P_min < P_max and nbins >= 1");
    *x_lo = std::log10(b->P_min_GV);
    *dx = (std::log10(b->P_max_GV) - *x_lo) / (double)b->nbins;
    return COSMICA_OK;
}

static cosmica_status upload_lis(const cosmica_lis *lis, DevBuf &buf, Staging &stage, cudaStream_t s,
                                 int *kind, const double **lnT, const double **lnJ, uint32_t *n)
{
    *kind = 0; *lnT = nullptr; *lnJ = nullptr; *n = 0;
    if (!lis || lis->kind == 0) return COSMICA_OK;
    if (lis->kind != 1 || lis->n < 2 || !lis->lnT || !lis->lnJ)
        return fail(COSMICA_ERR_INVALID, "LIS table needs kind 1, n >= 2 and both arrays");
    for (uint32_t i = 1; i < lis->n; ++i)
        if (!(lis->lnT[i] > lis->lnT[i - 1])) return fail(COSMICA_ERR_INVALID, "LIS lnT must ascend");
    const size_t bytes = 2 * lis->n * sizeof(double);
    cosmica_status st = buf.reserve(bytes);
    if (st != COSMICA_OK) return st;
    st = stage.reserve(bytes);
    if (st != COSMICA_OK) return st;
    std::memcpy(stage.h, lis->lnT, lis->n * sizeof(double));
    std::memcpy((double *)stage.h + lis->n, lis->lnJ, lis->n * sizeof(double));
    st = stage.upload(buf.d, bytes, s);
    if (st != COSMICA_OK) return st;
    *kind = 1;
    *lnT = (const double *)buf.d;
    *lnJ = (const double *)buf.d + lis->n;
    *n = lis->n;
    return COSMICA_OK;
}

static cosmica_status spectrum_of_hist(const std::vector<SpecItem> &its, const cosmica_lis *lis, uint32_t nbins,
                                       double x_lo, double dx, const uint64_t *hist, double *J, double *sigma,
                                       DevBuf &ibuf, Staging &istage, DevBuf &lbuf, Staging &lstage, cudaStream_t s);

static cosmica_status run_spectrum(const cosmica_exit_states *ex, const std::vector<SpecItem> &its,
                                   const cosmica_lis *lis, const cosmica_bins *bins, double *J, double *sigma,
                                   uint64_t *hist, DevBuf &ibuf, Staging &istage, DevBuf &lbuf, Staging &lstage,
                                   cudaStream_t s)
{
    double x_lo, dx;
    cosmica_status st = check_bins(bins, &x_lo, &dx);
    if (st != COSMICA_OK) return st;
    const uint32_t n_items = (uint32_t)its.size();
    if (n_items == 0) return COSMICA_OK;
    if (!J || !sigma || !hist) return fail(COSMICA_ERR_INVALID, "J / sigma / hist must be non-NULL");
    if (!ex) return fail(COSMICA_ERR_INVALID, "exit states NULL");
    if (ex->n > 0 && !valid_exit(ex)) return fail(COSMICA_ERR_INVALID, "exit-state arrays must be non-NULL");
    if (ex->n > 0 && !is_device_ptr(ex->lnP)) return fail(COSMICA_ERR_INVALID, "exit states must be device memory");
    if (!is_device_ptr(J) || !is_device_ptr(sigma) || !is_device_ptr(hist))
        return fail(COSMICA_ERR_INVALID, "J / sigma / hist must be device memory");
    const size_t hbytes = (size_t)n_items * COSMICA_HIST_STRIDE(bins->nbins) * sizeof(uint64_t);
    CK(cudaMemsetAsync(hist, 0, hbytes, s), "cudaMemsetAsync(hist)");
    cudaError_t e = launch_histogram(exit_ptrs(ex), ex->n, n_items, bins->nbins, x_lo, dx,
                                     (unsigned long long *)hist, s);
    if (e != cudaSuccess) return cuda_fail(e, "histogram kernel launch");
    return spectrum_of_hist(its, lis, bins->nbins, x_lo, dx, hist, J, sigma, ibuf, istage, lbuf, lstage, s);
}

// Eq. 4 per item from a histogram already in device memory (the second half of run_spectrum).
static cosmica_status spectrum_of_hist(const std::vector<SpecItem> &its, const cosmica_lis *lis, uint32_t nbins,
                                       double x_lo, double dx, const uint64_t *hist, double *J, double *sigma,
                                       DevBuf &ibuf, Staging &istage, DevBuf &lbuf, Staging &lstage, cudaStream_t s)
{
    const uint32_t n_items = (uint32_t)its.size();
    cosmica_status st = ibuf.reserve(n_items * sizeof(SpecItem));
    if (st != COSMICA_OK) return st;
    st = istage.reserve(n_items * sizeof(SpecItem));
    if (st != COSMICA_OK) return st;
    std::memcpy(istage.h, its.data(), n_items * sizeof(SpecItem));
    st = istage.upload(ibuf.d, n_items * sizeof(SpecItem), s);
    if (st != COSMICA_OK) return st;
    int kind; const double *lnT, *lnJ; uint32_t ln;
    st = upload_lis(lis, lbuf, lstage, s, &kind, &lnT, &lnJ, &ln);
    if (st != COSMICA_OK) return st;
    cudaError_t e = launch_spectrum((const unsigned long long *)hist, n_items, nbins, x_lo, dx,
                                    (const SpecItem *)ibuf.d, kind, lnT, lnJ, ln, J, sigma, s);
    if (e != cudaSuccess) return cuda_fail(e, "spectrum kernel launch");
    return COSMICA_OK;
}

extern "C" cosmica_status cosmica_spectrum(const cosmica_exit_states *exit, const cosmica_species *species,
                                           const double *T_in, uint32_t n_energies, const cosmica_lis *lis,
                                           const cosmica_bins *bins, double *J_out, double *sigma_out,
                                           uint64_t *hist_out, void *stream)
{
    cosmica_status st = check_species(species);
    if (st != COSMICA_OK) return st;
    if (n_energies > 0 && !T_in) return fail(COSMICA_ERR_INVALID, "T_in is NULL");
    std::vector<SpecItem> its(n_energies);
    for (uint32_t e = 0; e < n_energies; ++e)
        its[e] = SpecItem{T_in[e], (double)species->A, (double)species->Z, species->m0_GeV};
    // scratch of the calling thread: the spectrum call carries no handle
    thread_local DevBuf ibuf, lbuf;
    thread_local Staging istage, lstage;
    return run_spectrum(exit, its, lis, bins, J_out, sigma_out, hist_out, ibuf, istage, lbuf, lstage,
                        (cudaStream_t)stream);
}

extern "C" cosmica_status cosmica_spectrum_unbinned(const cosmica_exit_states *exit, const cosmica_species *species,
                                                    const double *T_in, uint32_t n_energies,
                                                    const uint32_t *n_per_energy, int32_t formulation,
                                                    const cosmica_lis *lis, double *J_out, double *sigma_out,
                                                    void *stream)
{
    cosmica_status st = check_species(species);
    if (st != COSMICA_OK) return st;
    if (formulation != 0 && formulation != 1) return fail(COSMICA_ERR_INVALID, "formulation %d", formulation);
    if (n_energies == 0) return COSMICA_OK;
    if (!T_in || !n_per_energy || !exit || !J_out || !sigma_out) return fail(COSMICA_ERR_INVALID, "NULL argument");
    uint64_t total = 0;
    for (uint32_t e = 0; e < n_energies; ++e) total += n_per_energy[e];
    if (exit->n != total) return fail(COSMICA_ERR_INVALID, "exit->n != sum(n_per_energy)");
    if (formulation == 1 && !exit->lw) return fail(COSMICA_ERR_INVALID, "the energy form needs exit->lw");
    if (total > 0 && (!valid_exit(exit) || !is_device_ptr(exit->lnP)))
        return fail(COSMICA_ERR_INVALID, "exit states must be device memory");
    if (!is_device_ptr(J_out) || !is_device_ptr(sigma_out)) return fail(COSMICA_ERR_INVALID, "J / sigma must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    thread_local DevBuf buf, lbuf;
    thread_local Staging stage, lstage;
    const size_t b_items = align_up(n_energies * sizeof(SpecItem), 256);
    const size_t bytes = b_items + (n_energies + 1) * sizeof(uint64_t);
    st = buf.reserve(bytes);
    if (st != COSMICA_OK) return st;
    st = stage.reserve(bytes);
    if (st != COSMICA_OK) return st;
    SpecItem *hi = (SpecItem *)stage.h;
    uint64_t *hp = (uint64_t *)((char *)stage.h + b_items);
    hp[0] = 0;
    for (uint32_t e = 0; e < n_energies; ++e) {
        hi[e] = SpecItem{T_in[e], (double)species->A, (double)species->Z, species->m0_GeV};
        hp[e + 1] = hp[e] + n_per_energy[e];
    }
    st = stage.upload(buf.d, bytes, s);
    if (st != COSMICA_OK) return st;
    int kind; const double *lnT, *lnJ; uint32_t ln;
    st = upload_lis(lis, lbuf, lstage, s, &kind, &lnT, &lnJ, &ln);
    if (st != COSMICA_OK) return st;
    cudaError_t e = launch_spectrum_unbinned(exit_ptrs(exit), (const uint64_t *)((char *)buf.d + b_items), n_energies,
                                             (const SpecItem *)buf.d, formulation, kind, lnT, lnJ, ln, J_out,
                                             sigma_out, s);
    return e == cudaSuccess ? COSMICA_OK : cuda_fail(e, "unbinned spectrum launch");
}

// =============================================================== batch API ==
struct cosmica_batch {
    std::vector<cosmica_params> params;
    std::vector<cosmica_species> species;
    int precision = 0;
    bool extended = false;     // some parameter set has radial shells or a squashed heliosphere
    bool full = true;          // every parameter set is the full model (see full_model)
    DevParams *d_prm = nullptr;
    const float *d_f32 = nullptr;   // paged field-major FP32 blocks (inside the d_prm allocation)
    DevSpecies *d_spc = nullptr;
    Tables tab;
    MixedVariant variant() const { return MixedVariant{precision, params[0].formulation == 1, extended, full}; }
    ExitStage exit_stage;
    DevBuf spec_items, lis_buf;
    Staging spec_stage, lis_stage;
    // CUDA graph of [memset counters, persistent kernel] for repeated runs
    cudaGraphExec_t gexec = nullptr;
    // every value the captured launch bakes in: a replay is valid only when all are unchanged
    struct GraphKey {
        uint64_t total = 0;
        uint32_t n_items = 0;
        const void *tables = nullptr;
        ExitPtrs ex{};
        PersistentShape shape{};
        cudaStream_t stream = nullptr;
        int precision = -1;
        bool operator==(const GraphKey &o) const
        {
            return total == o.total && n_items == o.n_items && tables == o.tables && ex.r == o.ex.r &&
                   ex.th == o.ex.th && ex.ph == o.ex.ph && ex.lnP == o.ex.lnP && ex.s == o.ex.s &&
                   ex.steps == o.ex.steps && ex.status == o.ex.status && ex.item == o.ex.item &&
                   ex.lw == o.ex.lw && shape.block == o.shape.block && shape.grid == o.shape.grid &&
                   shape.compact_period == o.shape.compact_period && stream == o.stream &&
                   precision == o.precision;
        }
    } gkey;
};

extern "C" cosmica_status cosmica_batch_create(const cosmica_params *params, uint32_t n_params,
                                               const cosmica_species *species, uint32_t n_species,
                                               cosmica_batch **out)
{
    if (!out) return fail(COSMICA_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (n_params == 0 || n_species == 0 || !params || !species)
        return fail(COSMICA_ERR_INVALID, "need at least one parameter set and one species");
    for (uint32_t i = 0; i < n_params; ++i) {
        cosmica_status st = check_params(params + i);
        if (st != COSMICA_OK) return st;
        if (params[i].precision != params[0].precision)
            return fail(COSMICA_ERR_INVALID, "all parameter sets of a batch must share one precision");
        if (params[i].formulation != params[0].formulation)
            return fail(COSMICA_ERR_INVALID, "all parameter sets of a batch must share one formulation");
    }
    for (uint32_t i = 0; i < n_species; ++i) {
        cosmica_status st = check_species(species + i);
        if (st != COSMICA_OK) return st;
    }
    cosmica_batch *b = new (std::nothrow) cosmica_batch();
    if (!b) return fail(COSMICA_ERR_OOM, "host allocation of the batch");
    b->params.assign(params, params + n_params);
    b->species.assign(species, species + n_species);
    b->precision = params[0].precision;
    for (uint32_t i = 0; i < n_params; ++i) {
        b->extended = b->extended || params[i].n_shells > 0 || params[i].squashed != 0;
        b->full = b->full && full_model(params[i]);
    }
    cosmica_status st = upload_params(params, n_params, &b->d_prm, &b->d_f32);
    if (st == COSMICA_OK) {
        std::vector<DevSpecies> hs(n_species);
        for (uint32_t i = 0; i < n_species; ++i) hs[i] = to_dev(species[i]);
        cudaError_t e = cudaMalloc(&b->d_spc, n_species * sizeof(DevSpecies));
        if (e == cudaSuccess) e = cudaMemcpy(b->d_spc, hs.data(), n_species * sizeof(DevSpecies), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) st = cuda_fail(e, "species upload");
    }
    if (st != COSMICA_OK) {
        cosmica_batch_destroy(b);
        return st;
    }
    *out = b;
    return COSMICA_OK;
}

extern "C" void cosmica_batch_destroy(cosmica_batch *b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->d_prm) cudaFree(b->d_prm);
    if (b->d_spc) cudaFree(b->d_spc);
    b->tab.release();
    b->exit_stage.buf.release();
    b->spec_items.release();
    b->lis_buf.release();
    b->spec_stage.release();
    b->lis_stage.release();
    delete b;
}

static cosmica_status batch_items(const cosmica_batch *b, const cosmica_work_item *items, uint32_t n_items,
                                  std::vector<DevItem> &its, std::vector<uint64_t> &pre)
{
    if (n_items > 0 && !items) return fail(COSMICA_ERR_INVALID, "items is NULL");
    its.resize(n_items);
    pre.assign(n_items + 1, 0);
    for (uint32_t i = 0; i < n_items; ++i) {
        const cosmica_work_item &w = items[i];
        if (w.param_idx >= b->params.size() || w.species_idx >= b->species.size())
            return fail(COSMICA_ERR_INVALID, "item %u: parameter or species index out of range", i);
        if (!(std::isfinite(w.T_GeVn) && w.T_GeVn > 0.0)) return fail(COSMICA_ERR_INVALID, "item %u: T must be > 0", i);
        const cosmica_params &p = b->params[w.param_idx];
        const bool own = w.r0_AU != 0.0;
        if (own && !valid_start(p, w.r0_AU, w.th0_rad, w.ph0_rad))
            return fail(COSMICA_ERR_INVALID, "item %u: start position outside the heliosphere", i);
        its[i] = make_item(w.T_GeVn, w.first_pid, w.seed, w.param_idx, w.species_idx, own ? w.r0_AU : p.r0_AU,
                           own ? w.th0_rad : p.th0_rad, own ? w.ph0_rad : p.ph0_rad,
                           w.exit_item_plus1 ? w.exit_item_plus1 - 1u : i);
        pre[i + 1] = pre[i] + w.n;
    }
    return COSMICA_OK;
}

static cosmica_status batch_launch(cosmica_batch *b, uint64_t total, const ExitPtrs &ex,
                                   const cosmica_tuning *tuning, cudaStream_t s)
{
    LaunchArgs a{b->d_prm, b->d_spc, b->tab.items, b->tab.prefix, b->tab.n_items, total, ex,
                 b->tab.counters + 1, b->tab.counters, b->tab.qitem, b->tab.qprefix, b->d_f32};
    auto direct = [&]() -> cosmica_status {
        CK(cudaMemsetAsync(b->tab.counters, 0, 2 * sizeof(unsigned long long), s), "cudaMemsetAsync(counters)");
        cudaError_t e = (b->precision == COSMICA_PREC_FP64)
                            ? launch_propagate_fp64(a, s)
                            : launch_propagate_mixed(a, b->variant(), shape_for(b->variant(), tuning, total), s);
        if (e != cudaSuccess) return cuda_fail(e, "propagation kernel launch");
        return COSMICA_OK;
    };
    const bool graph = tuning && tuning->use_graph && s != nullptr;
    if (!graph) return direct();
    const PersistentShape sh = shape_for(b->variant(), tuning, total);
    cosmica_batch::GraphKey key;
    key.total = total;
    key.n_items = b->tab.n_items;
    key.tables = b->tab.dev.d;
    key.ex = ex;
    key.shape = sh;
    key.stream = s;
    key.precision = b->precision;
    if (!b->gexec || !(b->gkey == key)) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
        cosmica_status st = direct();
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s, &g);
        if (st != COSMICA_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            b->gexec = nullptr;
            return cuda_fail(e, "cudaGraphInstantiate");
        }
        b->gkey = key;
    }
    CK(cudaGraphLaunch(b->gexec, s), "cudaGraphLaunch");
    note_launch();
    return COSMICA_OK;
}

extern "C" cosmica_status cosmica_batch_run(cosmica_batch *b, const cosmica_work_item *items, uint32_t n_items,
                                            const cosmica_tuning *tuning, cosmica_exit_states *out,
                                            uint64_t *steps_out, void *stream)
{
    if (!b) return fail(COSMICA_ERR_INVALID, "batch is NULL");
    if (!out) return fail(COSMICA_ERR_INVALID, "out is NULL");
    std::vector<DevItem> its;
    std::vector<uint64_t> pre;
    cosmica_status st = batch_items(b, items, n_items, its, pre);
    if (st != COSMICA_OK) return st;
    const uint64_t total = pre[n_items];
    if (out->n != total) return fail(COSMICA_ERR_INVALID, "out->n = %llu, particles = %llu",
                                     (unsigned long long)out->n, (unsigned long long)total);
    cudaStream_t s = (cudaStream_t)stream;
    if (total == 0) {
        if (steps_out) CK(cudaMemsetAsync(steps_out, 0, sizeof(uint64_t), s), "cudaMemsetAsync(steps)");
        return COSMICA_OK;
    }
    if (!valid_exit(out)) return fail(COSMICA_ERR_INVALID, "exit-state arrays must be non-NULL");
    const bool by_cost = tuning ? tuning->queue_order != 0 : true;
    st = b->tab.build(its, pre, by_cost ? cost_order(its, b->params.data(), b->species.data())
                                        : std::vector<uint32_t>(), s);
    if (st != COSMICA_OK) return st;
    if (b->params[0].formulation == 1 && !out->lw)
        return fail(COSMICA_ERR_INVALID, "the energy form needs out->lw");
    const bool host_out = !is_device_ptr(out->r);
    ExitPtrs ex = exit_ptrs(out);
    if (host_out) {
        st = b->exit_stage.make(total, ex, out->lw != nullptr);
        if (st != COSMICA_OK) return st;
    }
    st = batch_launch(b, total, ex, tuning, s);
    if (st != COSMICA_OK) return st;
    if (steps_out)
        CK(cudaMemcpyAsync(steps_out, b->tab.counters + 1, sizeof(uint64_t), cudaMemcpyDeviceToDevice, s),
           "copy steps");
    if (host_out) return ExitStage::copy_back(ex, out, s);
    return COSMICA_OK;
}

extern "C" cosmica_status cosmica_batch_spectrum(cosmica_batch *b, const cosmica_work_item *items,
                                                 uint32_t n_items, const cosmica_exit_states *exit,
                                                 const cosmica_lis *lis, const cosmica_bins *bins, double *J_out,
                                                 double *sigma_out, uint64_t *hist_out, void *stream)
{
    if (!b) return fail(COSMICA_ERR_INVALID, "batch is NULL");
    if (n_items > 0 && !items) return fail(COSMICA_ERR_INVALID, "items is NULL");
    std::vector<SpecItem> its(n_items);
    for (uint32_t i = 0; i < n_items; ++i) {
        if (items[i].species_idx >= b->species.size()) return fail(COSMICA_ERR_INVALID, "species index out of range");
        const cosmica_species &sp = b->species[items[i].species_idx];
        its[i] = SpecItem{items[i].T_GeVn, (double)sp.A, (double)sp.Z, sp.m0_GeV};
    }
    return run_spectrum(exit, its, lis, bins, J_out, sigma_out, hist_out, b->spec_items, b->spec_stage,
                        b->lis_buf, b->lis_stage, (cudaStream_t)stream);
}

extern "C" cosmica_status cosmica_batch_spectrum_hist(cosmica_batch *b, const cosmica_work_item *items,
                                                      uint32_t n_items, const cosmica_lis *lis,
                                                      const cosmica_bins *bins, const uint64_t *hist, double *J_out,
                                                      double *sigma_out, void *stream)
{
    if (!b) return fail(COSMICA_ERR_INVALID, "batch is NULL");
    if (n_items > 0 && !items) return fail(COSMICA_ERR_INVALID, "items is NULL");
    double x_lo, dx;
    cosmica_status st = check_bins(bins, &x_lo, &dx);
    if (st != COSMICA_OK) return st;
    if (n_items == 0) return COSMICA_OK;
    if (!J_out || !sigma_out || !hist) return fail(COSMICA_ERR_INVALID, "J / sigma / hist must be non-NULL");
    if (!is_device_ptr(J_out) || !is_device_ptr(sigma_out) || !is_device_ptr(hist))
        return fail(COSMICA_ERR_INVALID, "J / sigma / hist must be device memory");
    std::vector<SpecItem> its(n_items);
    for (uint32_t i = 0; i < n_items; ++i) {
        if (items[i].species_idx >= b->species.size()) return fail(COSMICA_ERR_INVALID, "species index out of range");
        const cosmica_species &sp = b->species[items[i].species_idx];
        its[i] = SpecItem{items[i].T_GeVn, (double)sp.A, (double)sp.Z, sp.m0_GeV};
    }
    return spectrum_of_hist(its, lis, bins->nbins, x_lo, dx, hist, J_out, sigma_out, b->spec_items, b->spec_stage,
                            b->lis_buf, b->lis_stage, (cudaStream_t)stream);
}

// =============================================================== autotune ==
// Tuned shapes are cached per (device, configuration class): the precision,
// whether the sets have a drift / a termination shock, the particle count to
// within a factor of two (it sets the particles per lane, hence the tail), and
// the kernel variant (energy form, radial shells or squashed heliosphere).
namespace {
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int, int, int>, std::pair<cosmica_tuning, double>> g_tune_cache;
}  // namespace

extern "C" cosmica_status cosmica_autotune(cosmica_batch *b, const cosmica_work_item *items, uint32_t n_items,
                                           cosmica_tuning *best, double *best_rate)
{
    if (!b || !best) return fail(COSMICA_ERR_INVALID, "batch / best is NULL");
    int dev = 0;
    cudaGetDevice(&dev);
    int drift = 0, ts = 0;
    for (const cosmica_params &p : b->params) {
        drift |= p.drift_on != 0;
        ts |= p.R_ts_AU > 0.0;
    }
    uint64_t n_all = 0;
    for (uint32_t i = 0; i < n_items && items; ++i) n_all += items[i].n;
    int size_class = 0;
    while ((n_all >> size_class) > 1) ++size_class;
    // the kernel variant (energy form, shells) has its own registers, hence its own best shape
    const int variant = (b->params[0].formulation == 1 ? 1 : 0) | (b->extended ? 2 : 0) | (b->full ? 4 : 0);
    const auto key = std::make_tuple(dev, b->precision, drift, ts, size_class, variant);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            *best = it->second.first;
            if (best_rate) *best_rate = it->second.second;
            return COSMICA_OK;
        }
    }
    if (b->precision == COSMICA_PREC_FP64) {
        *best = cosmica_tuning{128, 0, 0, 0, 0};
        if (best_rate) *best_rate = 0.0;
        return COSMICA_OK;
    }
    std::vector<DevItem> its;
    std::vector<uint64_t> pre;
    cosmica_status st = batch_items(b, items, n_items, its, pre);
    if (st != COSMICA_OK) return st;
    if (pre[n_items] == 0) return fail(COSMICA_ERR_INVALID, "autotune needs particles");
    // A launch's time is about t(P) = a + b P in its particle count P: b is the cost of a
    // particle at full occupancy, a the tail that no launch avoids (its slowest paths run
    // alone at the end).  Small batches (up to ~30 particles per SM thread slot) are timed
    // whole; larger ones on two scaled samples (~10 and ~30 per slot), from which each
    // candidate's time for the whole batch is extrapolated.  Small samples over-weight the
    // tail and favour shapes with fewer resident warps: with samples of ~2 and ~6 per slot
    // the tuner chose 3 blocks of 256 on config 3, which runs 2.6 % slower than 4.
    const uint64_t lanes = (uint64_t)num_sms() * 2048u;
    const uint64_t n_full = pre[n_items];
    const double s_hi = std::min(1.0, 30.0 * (double)lanes / (double)n_full);
    const double s_lo = std::min(1.0, 10.0 * (double)lanes / (double)n_full);
    const bool whole = s_hi >= 1.0;
    auto make_sample = [&](double scale, uint64_t *total) {
        std::vector<cosmica_work_item> v(items, items + n_items);
        *total = 0;
        for (auto &w : v) {
            w.n = (uint32_t)std::ceil(w.n * scale);
            *total += w.n;
        }
        return v;
    };
    uint64_t n_hi = 0, n_lo = 0;
    std::vector<cosmica_work_item> sample_hi = make_sample(s_hi, &n_hi);
    std::vector<cosmica_work_item> sample_lo = make_sample(s_lo, &n_lo);
    DevBuf out_buf;
    ExitPtrs ex;
    {
        ExitStage tmp;
        st = tmp.make(n_hi, ex, b->params[0].formulation == 1);
        if (st != COSMICA_OK) return st;
        out_buf = tmp.buf;
    }
    unsigned long long *d_steps = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t ce = cudaMalloc(&d_steps, sizeof(unsigned long long));
    if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    // time one run of a sample with shape t: milliseconds and steps
    auto run = [&](const std::vector<cosmica_work_item> &smp, uint64_t n, const cosmica_tuning &t, double *ms_out,
                   double *steps_out) -> bool {
        cosmica_exit_states eo{ex.r, ex.th, ex.ph, ex.lnP, ex.s, ex.steps, ex.status, ex.item, n, ex.lw};
        ce = cudaEventRecord(e0, s);
        if (ce != cudaSuccess) return false;
        st = cosmica_batch_run(b, smp.data(), n_items, &t, &eo, (uint64_t *)d_steps, s);
        if (st != COSMICA_OK) return false;
        ce = cudaEventRecord(e1, s);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        if (ce != cudaSuccess) return false;
        float ms = 0.0f;
        unsigned long long steps = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        ce = cudaMemcpy(&steps, d_steps, sizeof(steps), cudaMemcpyDeviceToHost);
        if (ce != cudaSuccess) return false;
        *ms_out = ms;
        *steps_out = (double)steps;
        return true;
    };
    double best_r = -1.0;
    cosmica_tuning bt{128, 0, 64, 0, 1};
    if (ce == cudaSuccess) {
        const unsigned blocks[] = {128, 256};
        const unsigned periods[] = {0, 64};
        std::vector<cosmica_tuning> cands;
        for (unsigned blk : blocks) {
            for (unsigned per : periods) {
                const unsigned maxb = (unsigned)std::max(1, mixed_max_blocks_per_sm(b->variant(), blk, per != 0));
                // all resident blocks, one fewer, and half: fewer resident warps can win when the
                // register file or the L1 is the contended resource, or when the tail dominates
                cands.push_back(cosmica_tuning{blk, maxb, per, 0, 1});
                if (maxb >= 3) cands.push_back(cosmica_tuning{blk, maxb - 1, per, 0, 1});
                if (maxb / 2 >= 1 && maxb / 2 != maxb && maxb / 2 != maxb - 1)
                    cands.push_back(cosmica_tuning{blk, maxb / 2, per, 0, 1});
            }
        }
        for (const cosmica_tuning &t : cands) {
            double ms_hi = 0.0, st_hi = 0.0, ms_lo = 0.0, st_lo = 0.0;
            if (!run(sample_hi, n_hi, t, &ms_hi, &st_hi)) break;
            double ms_pred = ms_hi, steps_pred = st_hi;
            if (!whole) {
                if (!run(sample_lo, n_lo, t, &ms_lo, &st_lo)) break;
                const double ratio = (double)n_full / (double)n_hi;
                const double slope = n_hi > n_lo ? (ms_hi - ms_lo) / (double)(n_hi - n_lo) : 0.0;   // ms per particle
                ms_pred = slope > 0.0 ? ms_hi + slope * (double)(n_full - n_hi) : ms_hi * ratio;
                steps_pred = st_hi * ratio;
            }
            const double rate = ms_pred > 0.0 ? steps_pred / (ms_pred * 1e-3) : 0.0;
            if (rate > best_r) {
                best_r = rate;
                bt = t;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    if (d_steps) cudaFree(d_steps);
    out_buf.release();
    if (st != COSMICA_OK) return st;
    if (ce != cudaSuccess) return cuda_fail(ce, "autotune");
    *best = bt;
    if (best_rate) *best_rate = best_r;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = {bt, best_r};
    return COSMICA_OK;
}

// ================================================================== misc ==
extern "C" const char *cosmica_last_error(void) { return g_err; }

extern "C" uint64_t cosmica_launch_count(void) { return g_launches.load(); }

// ================================================================= debug ==
extern "C" cosmica_status cosmica_debug_philox(uint32_t n, const uint32_t *ctr, uint32_t k0, uint32_t k1,
                                               uint32_t *out, void *stream)
{
    if (n && (!ctr || !out)) return fail(COSMICA_ERR_INVALID, "NULL array");
    cudaError_t e = launch_debug_philox(n, ctr, k0, k1, out, (cudaStream_t)stream);
    return e == cudaSuccess ? COSMICA_OK : cuda_fail(e, "philox probe");
}

extern "C" cosmica_status cosmica_debug_curand_philox(uint32_t n, uint64_t seed, const uint64_t *subseq,
                                                      const uint64_t *offset, uint32_t *out, void *stream)
{
    if (n && (!subseq || !offset || !out)) return fail(COSMICA_ERR_INVALID, "NULL array");
    cudaError_t e = launch_debug_curand_philox(n, seed, (const unsigned long long *)subseq,
                                               (const unsigned long long *)offset, out, (cudaStream_t)stream);
    return e == cudaSuccess ? COSMICA_OK : cuda_fail(e, "curand probe");
}

extern "C" cosmica_status cosmica_debug_normals64(uint64_t seed, uint64_t pid0, uint32_t n, uint32_t step,
                                                  double *z, void *stream)
{
    if (n && !z) return fail(COSMICA_ERR_INVALID, "NULL array");
    cudaError_t e = launch_debug_normals64(seed, pid0, n, step, z, (cudaStream_t)stream);
    return e == cudaSuccess ? COSMICA_OK : cuda_fail(e, "normals probe");
}

extern "C" cosmica_status cosmica_debug_normals32(uint64_t seed, uint64_t pid0, uint32_t n, uint32_t step,
                                                  float *z, uint32_t *words, void *stream)
{
    if (n && !z) return fail(COSMICA_ERR_INVALID, "NULL array");
    if (n > (1u << 28)) return fail(COSMICA_ERR_INVALID, "n = %u too large for one probe", n);
    cudaError_t e = launch_debug_normals32(seed, pid0, n, step, z, words, (cudaStream_t)stream);
    return e == cudaSuccess ? COSMICA_OK : cuda_fail(e, "FP32 normals probe");
}

extern "C" cosmica_status cosmica_debug_fn64(int32_t which, uint32_t n, const double *x, double *y, void *stream)
{
    if (which < 0 || which > 5) return fail(COSMICA_ERR_INVALID, "function code %d", which);
    if (n && (!x || !y)) return fail(COSMICA_ERR_INVALID, "NULL array");
    cudaError_t e = launch_debug_fn64(which, n, x, y, (cudaStream_t)stream);
    return e == cudaSuccess ? COSMICA_OK : cuda_fail(e, "elementary-function probe");
}

extern "C" cosmica_status cosmica_debug_eval(cosmica_model *m, const cosmica_species *species, int32_t precision,
                                             uint32_t n, const double *states, double *out, void *stream)
{
    if (!m) return fail(COSMICA_ERR_INVALID, "model is NULL");
    cosmica_status st = check_species(species);
    if (st != COSMICA_OK) return st;
    if (n && (!states || !out)) return fail(COSMICA_ERR_INVALID, "NULL array");
    cudaStream_t s = (cudaStream_t)stream;
    DevSpecies *d_sp = nullptr;
    st = upload_species(m->spc, m->spc_stage, species, 1, s, &d_sp);
    if (st != COSMICA_OK) return st;
    cudaError_t e = precision == 0 ? launch_debug_eval64(m->d_prm, d_sp, n, states, out, s)
                                   : launch_debug_eval32(m->d_prm, d_sp, n, states, out, s);
    return e == cudaSuccess ? COSMICA_OK : cuda_fail(e, "evaluator probe");
}
