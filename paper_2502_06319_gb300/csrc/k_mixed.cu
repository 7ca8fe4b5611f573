// k_mixed.cu -- the batched persistent kernel of the mixed-precision path.
//
// One launch of (SMs x resident blocks) threads drains a device work queue:
// an atomic cursor over the prefix-summed particle counts of all work items
// (parameter set x species x energy).  Each lane owns one quasi-particle at a
// time and steps it until it leaves the heliosphere; a lane whose particle
// exits writes the exit state and immediately takes the next particle from
// the queue (refill), so that warps stay full while the queue lasts despite
// the long tail of exit times.  Lanes needing work in the same step take
// consecutive particles with one atomic per warp.  The paper's thread-per-
// quasi-particle mapping (Sec. IV.A) is kept; its one-launch-per-energy-bin
// loop (Sec. IV.A, last paragraph) becomes this single launch.
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "mixed_state.cuh"
#include "model32.cuh"

namespace cosmica {

namespace {

template <int ACC, bool EN>
__device__ __forceinline__ void start_particle(const LaunchArgs &a, uint64_t q, Lane &L, Acc<ACC> &x,
                                               EnergyAcc<ACC, EN> &en)
{
    // queue slot q -> (item, index within the item); the exit record keeps item order
    const uint32_t iq = find_item(a.qprefix, a.n_items, q);
    const uint32_t it = a.qitem ? a.qitem[iq] : iq;
    const uint64_t local = q - a.qprefix[iq];
    const DevItem item = a.items[it];
    const DevParams &p = a.prm[item.param_idx];
    const DevSpecies &sp = a.spc[item.species_idx];
    L.q = a.f32 + f32_table_offset(item.param_idx);
    L.M2 = sp.aoz_m0_sq;
    L.sq = sp.sgnq;
    L.pid = item.first_pid + local;
    L.seed = item.seed;
    L.g = a.prefix[it] + local;
    L.item = item.out_item;
    L.k = 0;
    L.max_steps = (uint32_t)p.max_steps;
    const double T = item.T;
    const double P0 = sp.A / fabs(sp.Z) * sqrt(T * (T + 2.0 * sp.m0));
    x.init(item.r0, item.th0, item.ph0, log(P0), p.R_out, p.f.r_in);
    en.init(T, (float)sp.m0, sp.aoz);
}

// One Euler-Maruyama step (Eq. 3, Eq. 6) of an active lane, with the normals z0, z1, z2
// of step L.k (drawn before); true when the path ended (exit record written), else the
// normals of the next step are left in z0, z1, z2.
template <int ACC, bool EN, bool EXT, bool FULL>
__device__ __forceinline__ bool step(const LaunchArgs &a, Lane &L, Acc<ACC> &x, EnergyAcc<ACC, EN> &en,
                                     unsigned long long &my_steps, float &z0, float &z1, float &z2)
{
    m32::Drift c;
    const P32<kSetsPerPage> q{L.q};
    float lnP;
    if constexpr (EN) {
        // rigidity from the integrated kinetic energy: P = (A/|Z|) sqrt(T (T + 2 m0))
        const float T = en.fT();
        lnP = __logf(en.aoz * sqrtf(T * (T + 2.0f * en.m0)));
    } else {
        lnP = x.flnP();
    }
    m32::eval<EXT, FULL, kSetsPerPage>(q, L.M2, L.sq, x.fr(), x.fth(), x.sin_th(), x.fph(), lnP, c);
    const float sdt = sqrtf(c.dt);
    const float dr = fmaf(c.Ar_tot, c.dt, c.l00 * z0 * sdt);
    const float dth = fmaf(c.dth_drift, c.dt, c.l11 * z1 * sdt * c.inv_r);
    const float dph = fmaf(c.dph_drift, c.dt, fmaf(c.l20, z0, c.l22 * z2) * sdt * c.inv_rs);
    if constexpr (EN) {
        // Eq. 1 backward: A_T = (2/3)(V/r) alpha T, loss L = (2V/(3r)) (1 + beta^2)
        const float T = en.fT();
        const float alpha = __fdividef(T + 2.0f * en.m0, T + en.m0);
        en.add(c.dlnP * alpha * T * c.dt, c.dlnP * fmaf(c.beta, c.beta, 1.0f) * c.dt);
        x.add(dr, dth, dph, 0.0f, c.dt);
    } else {
        x.add(dr, dth, dph, c.dlnP * c.dt, c.dt);
    }
    x.boundaries(P32F(q, r_in));
    L.k += 1u;

    const bool fin = x.finite();
    const bool out = (EXT && P32F(q, sq) != 0.0f) ? m32::outside_squashed(q, x.fr(), x.fth(), x.fph()) : x.exited();
    const bool lim = L.k >= L.max_steps;
    if (fin & !out & !lim) {     // one rarely taken branch for the three ends of a path
        // the next step's normals, drawn after this step's arithmetic: the Philox block and
        // the eval of the coefficients are then never live at the same time (64 instead of
        // 74 registers in the variant without compaction: 32 resident warps per SM instead
        // of 24, +2.6 % steps/s on config 3; a lone path's step takes 12 % longer, as the
        // block no longer hides under the eval's latency)
        m32::normals(L.seed, L.pid, L.k, z0, z1, z2);
        return false;
    }
    const int status = !fin ? COSMICA_PATH_NONFINITE : (out ? COSMICA_PATH_EXIT : COSMICA_PATH_STEP_LIMIT);
    x.write(a.out, L.g);
    if constexpr (EN) {
        const double T = en.T64();
        a.out.lnP[L.g] = log((double)en.aoz * sqrt(T * (T + 2.0 * (double)en.m0)));
        if (a.out.lw) a.out.lw[L.g] = en.lw();
    } else {
        if (a.out.lw) a.out.lw[L.g] = 0.0;
    }
    a.out.steps[L.g] = L.k;
    a.out.status[L.g] = (uint8_t)status;
    a.out.item[L.g] = L.item;
    my_steps += L.k;
    return true;
}

// Persistent propagation.
// Phase 1: lanes take particles from the device queue (one atomic per warp for all
// lanes needing work), step them, write the exit record and refill, until the queue
// is drained.  Phase 2 (COMPACT): every `period` steps the block meets at a
// checkpoint; the active particles are counted and, if they occupy more warps than
// they need, repacked through shared memory into the block's lowest lanes, so that
// issued warp instructions keep carrying full lanes while the long tail of exit
// times plays out.  Both phases share one step site (one copy of the step code).
template <int ACC, bool COMPACT, bool EN, bool EXT, bool FULL>
__global__ void __launch_bounds__(256) k_propagate_mixed(LaunchArgs a, uint32_t period)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ unsigned s_count;
    __shared__ unsigned s_warp[8];
    const unsigned lane = threadIdx.x & 31u;
    const unsigned warp = threadIdx.x >> 5;
    Lane L;
    Acc<ACC> x;
    EnergyAcc<ACC, EN> en;
    bool active = false, drained = false, phase2 = false;
    float z0 = 0.0f, z1 = 0.0f, z2 = 0.0f;   // normals of the lane's next step
    unsigned long long my_steps = 0;
    uint32_t tick = 0;   // phase 1: steps since the last drained check; phase 2: steps since the checkpoint

    while (true) {
        if (!COMPACT && drained) {
            // the queue is exhausted (warp-uniform): finish the particles in hand
            if (!__any_sync(0xffffffffu, active)) break;
        } else if (!phase2) {
            const unsigned need = __ballot_sync(0xffffffffu, !active && !drained);
            if (need) {
                unsigned long long base = 0;
                const unsigned leader = __ffs(need) - 1;
                if (lane == leader) base = atomicAdd(a.cursor, (unsigned long long)__popc(need));
                base = __shfl_sync(0xffffffffu, base, leader);
                if (need & (1u << lane)) {
                    const uint64_t q = base + __popc(need & ((1u << lane) - 1u));
                    if (q < a.n_total) {
                        start_particle<ACC, EN>(a, q, L, x, en);
                        m32::normals(L.seed, L.pid, L.k, z0, z1, z2);
                        active = true;
                    } else {
                        drained = true;
                    }
                }
                // without compaction a lane that was refused never asks again, so once any lane
                // of the warp is refused the whole warp can stop asking
                if (!COMPACT && base + __popc(need) > a.n_total) drained = true;
            }
            if (COMPACT) {
                // learn of the drained queue even when no lane of the warp needed work
                if (++tick >= period) {
                    tick = 0;
                    unsigned dq = 0;
                    if (lane == 0) dq = *(volatile unsigned long long *)a.cursor >= a.n_total;
                    if (__shfl_sync(0xffffffffu, dq, 0)) drained = true;
                }
                if (__all_sync(0xffffffffu, drained || active) && __any_sync(0xffffffffu, drained)) {
                    drained = true;
                    phase2 = true;
                    tick = 0;
                }
            }
        }
        if (COMPACT && phase2) {
            if (tick == 0) {
                // checkpoint: every warp of the block arrives here once per epoch
                if (threadIdx.x == 0) s_count = 0;
                __syncthreads();
                const unsigned bal = __ballot_sync(0xffffffffu, active);
                if (lane == 0) {
                    s_warp[warp] = __popc(bal);
                    atomicAdd(&s_count, (unsigned)__popc(bal));
                }
                __syncthreads();
                const unsigned n = s_count;
                if (n == 0) break;
                unsigned occupied = 0, before = 0;
                for (unsigned w = 0; w < (blockDim.x >> 5); ++w) {
                    occupied += s_warp[w] > 0;
                    if (w < warp) before += s_warp[w];
                }
                if (occupied > (n + 31) / 32) {
                    Packed<ACC, EN> *pack = reinterpret_cast<Packed<ACC, EN> *>(smem_raw);
                    if (active) {
                        const unsigned rank = before + __popc(bal & ((1u << lane) - 1u));
                        pack[rank].L = L;
                        pack[rank].x = x;
                        pack[rank].en = en;
                    }
                    __syncthreads();
                    active = threadIdx.x < n;
                    if (active) {
                        L = pack[threadIdx.x].L;
                        x = pack[threadIdx.x].x;
                        en = pack[threadIdx.x].en;
                        m32::normals(L.seed, L.pid, L.k, z0, z1, z2);
                    }
                }
                __syncthreads();
            }
            // an idle warp goes straight to the next checkpoint
            tick = __any_sync(0xffffffffu, active) ? (tick + 1 == period ? 0 : tick + 1) : 0;
        }
        if (active && step<ACC, EN, EXT, FULL>(a, L, x, en, my_steps, z0, z1, z2)) active = false;
    }
    if (a.steps_total) {
        for (int o = 16; o > 0; o >>= 1) my_steps += __shfl_down_sync(0xffffffffu, my_steps, o);
        if (lane == 0 && my_steps) atomicAdd(a.steps_total, my_steps);
    }
}

// debug: mixed coefficients at given states (FP64 in, FP64 out)
__global__ void k_debug_eval32(const DevParams *__restrict__ prm, const DevSpecies *__restrict__ spc,
                               uint32_t n, const double *__restrict__ st, double *__restrict__ out)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float dbg[kDebugEvalN];
    m32::Drift c;
    m32::eval<true, false, 1>(P32<1>{reinterpret_cast<const float *>(&prm[0].f)}, spc[0].aoz_m0_sq, spc[0].sgnq,
                              (float)st[4 * i], (float)st[4 * i + 1], m32::sin_theta_f64(st[4 * i + 1]),
                              (float)st[4 * i + 2], (float)st[4 * i + 3], c, dbg);
    for (int j = 0; j < kDebugEvalN; ++j) out[(size_t)i * kDebugEvalN + j] = dbg[j];
}

}  // namespace

template <int ACC, bool EN>
static size_t pack_bytes(unsigned block) { return (size_t)block * sizeof(Packed<ACC, EN>); }

// Call fn(acc, compact, energy, extended, full) with each flag as a compile-time constant.
template <class Fn>
static void visit_variant(MixedVariant v, bool compact, Fn &&fn)
{
    auto on_acc = [&](auto A) {
        auto on_compact = [&](auto C) {
            auto on_energy = [&](auto E) {
                auto on_ext = [&](auto X) {
                    if (v.full) fn(A, C, E, X, std::true_type{});
                    else fn(A, C, E, X, std::false_type{});
                };
                if (v.extended) on_ext(std::true_type{});
                else on_ext(std::false_type{});
            };
            if (v.energy) on_energy(std::true_type{});
            else on_energy(std::false_type{});
        };
        if (compact) on_compact(std::true_type{});
        else on_compact(std::false_type{});
    };
    if (v.acc == COSMICA_PREC_MIXED_F64ACC) on_acc(std::integral_constant<int, COSMICA_PREC_MIXED_F64ACC>{});
    else on_acc(std::integral_constant<int, COSMICA_PREC_MIXED>{});
}

int mixed_max_blocks_per_sm(MixedVariant v, unsigned block, bool compact)
{
    int nb = 0;
    visit_variant(v, compact, [&](auto A, auto C, auto E, auto S, auto F) {
        constexpr int acc = decltype(A)::value;
        constexpr bool c = decltype(C)::value, en = decltype(E)::value, sh = decltype(S)::value;
        constexpr bool fu = decltype(F)::value;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_propagate_mixed<acc, c, en, sh, fu>, (int)block,
                                                      c ? pack_bytes<acc, en>(block) : 0);
    });
    return nb;
}

cudaError_t launch_propagate_mixed(const LaunchArgs &a, MixedVariant v, PersistentShape shape, cudaStream_t s)
{
    if (a.n_total == 0) return cudaSuccess;
    cudaGetLastError();
    const uint32_t per = shape.compact_period;
    visit_variant(v, per != 0, [&](auto A, auto C, auto E, auto S, auto F) {
        constexpr int acc = decltype(A)::value;
        constexpr bool c = decltype(C)::value, en = decltype(E)::value, sh = decltype(S)::value;
        constexpr bool fu = decltype(F)::value;
        k_propagate_mixed<acc, c, en, sh, fu><<<shape.grid, shape.block, c ? pack_bytes<acc, en>(shape.block) : 0, s>>>(
            a, c ? per : 1u);
    });
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_debug_eval32(const DevParams *prm, const DevSpecies *spc, uint32_t n, const double *st,
                                double *out, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    cudaGetLastError();
    k_debug_eval32<<<(n + 127) / 128, 128, 0, s>>>(prm, spc, n, st, out);
    note_launch();
    return cudaGetLastError();
}

}  // namespace cosmica
