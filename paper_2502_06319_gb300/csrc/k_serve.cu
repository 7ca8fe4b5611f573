// k_serve.cu -- one quantum of the continuous-batching server.
//
// The server keeps the state of every in-flight quasi-particle resident on
// the device between launches.  Each quantum is one persistent launch in
// which every lane
//   1. takes work: first a particle suspended by the previous quantum (the
//      resume list), then a fresh particle of any admitted request (a work
//      queue over (request, energy) slices, oldest request first);
//   2. steps it exactly as the batched kernel does;
//   3. on exit writes the exit record into the request's slice of the exit
//      arena and counts the particle done for its request;
//   4. after `budget` steps in this launch suspends its particle (exact
//      state: compensated pairs or FP64, step counter, identity) to the
//      suspend list and stops.
// Between quanta the host admits newly arrived requests into the queue and
// retires finished ones, so requests that arrive while others run share the
// device with them.  A particle's path depends only on (seed, pid, request
// parameters), and suspension stores its state exactly, so every result is
// the same alone and in any mix.
#include <cstdint>
#include <type_traits>

#include "common.cuh"
#include "internal.h"
#include "mixed_state.cuh"
#include "model32.cuh"

namespace cosmica {

namespace {

template <int ACC>
__device__ __forceinline__ void save(const Acc<ACC> &x, Suspended &s);
template <int ACC>
__device__ __forceinline__ void load(Acc<ACC> &x, const Suspended &s, const DevParams &p);

template <>
__device__ __forceinline__ void save(const Acc<COSMICA_PREC_MIXED> &x, Suspended &s)
{
    s.f[0] = x.r.hi; s.f[1] = x.r.lo; s.f[2] = x.th.hi; s.f[3] = x.th.lo; s.f[4] = x.ph.hi;
    s.f[5] = x.ph.lo; s.f[6] = x.lnP.hi; s.f[7] = x.lnP.lo; s.f[8] = x.s.hi; s.f[9] = x.s.lo;
}
template <>
__device__ __forceinline__ void load(Acc<COSMICA_PREC_MIXED> &x, const Suspended &s, const DevParams &p)
{
    x.init(p.r0, p.th0, p.ph0, 0.0, p.R_out, p.f.r_in);
    x.r.hi = s.f[0]; x.r.lo = s.f[1]; x.th.hi = s.f[2]; x.th.lo = s.f[3]; x.ph.hi = s.f[4];
    x.ph.lo = s.f[5]; x.lnP.hi = s.f[6]; x.lnP.lo = s.f[7]; x.s.hi = s.f[8]; x.s.lo = s.f[9];
}
template <>
__device__ __forceinline__ void save(const Acc<COSMICA_PREC_MIXED_F64ACC> &x, Suspended &s)
{
    s.d[0] = x.r; s.d[1] = x.th; s.d[2] = x.ph; s.d[3] = x.lnP; s.d[4] = x.s;
}
template <>
__device__ __forceinline__ void load(Acc<COSMICA_PREC_MIXED_F64ACC> &x, const Suspended &s, const DevParams &p)
{
    x.init(s.d[0], s.d[1], s.d[2], s.d[3], p.R_out, p.f.r_in);
    x.s = s.d[4];
}

struct ServeLane {
    Lane L;
    uint32_t slot, energy;
    uint64_t exit_idx;
};

// EXT: some resident request has radial shells or a squashed heliosphere (the
// extended model; compile-time, as in the batched kernel).  FULL: every resident
// request is the full model (drift and current sheet on, adaptive step), so the step
// carries no uniform branch on those switches (the same DAG as the batched kernel's
// full-model variant).
template <int ACC, bool EXT, bool FULL>
__global__ void __launch_bounds__(256) k_serve(ServeArgs a)
{
    const unsigned lane = threadIdx.x & 31u;
    ServeLane S;
    Acc<ACC> x;
    bool active = false, done = false;
    uint32_t used = 0;
    float z0 = 0.0f, z1 = 0.0f, z2 = 0.0f;   // normals of the lane's next step (drawn one step ahead)

    while (true) {
        unsigned need = __ballot_sync(0xffffffffu, !active && !done);
        if (need) {
            // 1. resumed particles
            unsigned long long base = 0;
            const unsigned leader = __ffs(need) - 1;
            if (lane == leader) base = atomicAdd(a.cursors + 1, (unsigned long long)__popc(need));
            base = __shfl_sync(0xffffffffu, base, leader);
            bool got = false;
            if (need & (1u << lane)) {
                const uint64_t i = base + __popc(need & ((1u << lane) - 1u));
                if (i < a.n_resume) {
                    const Suspended rec = a.resume[i];
                    const DevParams &p = a.prm[rec.slot];
                    const DevSpecies &sp = a.spc[rec.slot];
                    load<ACC>(x, rec, p);
                    S.L.q = reinterpret_cast<const float *>(&p.f);
                    S.L.M2 = sp.aoz_m0_sq;
                    S.L.sq = sp.sgnq;
                    S.L.pid = rec.pid;
                    S.L.seed = rec.seed;
                    S.L.k = rec.k;
                    S.L.max_steps = (uint32_t)p.max_steps;
                    S.slot = rec.slot;
                    S.energy = rec.energy;
                    S.exit_idx = rec.exit_idx;
                    m32::normals(S.L.seed, S.L.pid, S.L.k, z0, z1, z2);
                    active = got = true;
                }
            }
            // 2. fresh particles for the lanes the resume list could not serve
            need = __ballot_sync(0xffffffffu, (need & (1u << lane)) && !got);
            if (need) {
                const unsigned ld = __ffs(need) - 1;
                if (lane == ld) base = atomicAdd(a.cursors, (unsigned long long)__popc(need));
                base = __shfl_sync(0xffffffffu, base, ld);
                if (need & (1u << lane)) {
                    const uint64_t g = base + __popc(need & ((1u << lane) - 1u));
                    if (g < a.n_fresh) {
                        const uint32_t it = find_item(a.prefix, a.n_items, g);
                        const ServeItem item = a.items[it];
                        const DevParams &p = a.prm[item.slot];
                        const DevSpecies &sp = a.spc[item.slot];
                        const uint64_t off = g - a.prefix[it];
                        S.L.q = reinterpret_cast<const float *>(&p.f);
                        S.L.M2 = sp.aoz_m0_sq;
                        S.L.sq = sp.sgnq;
                        S.L.pid = item.first_pid + off;
                        S.L.seed = item.seed;
                        S.L.k = 0;
                        S.L.max_steps = (uint32_t)p.max_steps;
                        S.slot = item.slot;
                        S.energy = item.energy;
                        S.exit_idx = item.exit_idx + off;
                        const double T = item.T;
                        const double P0 = sp.A / fabs(sp.Z) * sqrt(T * (T + 2.0 * sp.m0));
                        x.init(p.r0, p.th0, p.ph0, log(P0), p.R_out, p.f.r_in);
                        m32::normals(S.L.seed, S.L.pid, S.L.k, z0, z1, z2);
                        active = true;
                    } else {
                        done = true;
                    }
                }
            }
        }
        if (!__any_sync(0xffffffffu, active)) break;
        if (!active) continue;

        m32::Drift c;
        const P32<1> q{S.L.q};
        m32::eval<EXT, FULL, 1>(q, S.L.M2, S.L.sq, x.fr(), x.fth(), x.sin_th(), x.fph(), x.flnP(), c);
        const float sdt = sqrtf(c.dt);
        const float dr = fmaf(c.Ar_tot, c.dt, c.l00 * z0 * sdt);
        const float dth = fmaf(c.dth_drift, c.dt, c.l11 * z1 * sdt * c.inv_r);
        const float dph = fmaf(c.dph_drift, c.dt, fmaf(c.l20, z0, c.l22 * z2) * sdt * c.inv_rs);
        x.add(dr, dth, dph, c.dlnP * c.dt, c.dt);
        x.boundaries(P32F(q, r_in));
        S.L.k += 1u;
        used += 1u;

        const bool fin = x.finite();
        const bool out = (EXT && P32F(q, sq) != 0.0f) ? m32::outside_squashed(q, x.fr(), x.fth(), x.fph())
                                                       : x.exited();
        const bool lim = S.L.k >= S.L.max_steps;
        if (!(fin & !out & !lim)) {      // one rarely taken branch for the three ends of a path
            const int status = !fin ? COSMICA_PATH_NONFINITE : (out ? COSMICA_PATH_EXIT : COSMICA_PATH_STEP_LIMIT);
            const uint64_t g = S.exit_idx;
            x.write(a.arena, g);
            a.arena.steps[g] = S.L.k;
            a.arena.status[g] = (uint8_t)status;
            a.arena.item[g] = S.energy;
            atomicAdd(a.req_done + S.slot, 1u);
            atomicAdd(a.req_steps + S.slot, (unsigned long long)S.L.k);
            active = false;
        } else if (used >= a.budget) {
            const unsigned j = atomicAdd(a.n_suspend, 1u);
            Suspended rec;
            save<ACC>(x, rec);
            rec.k = S.L.k;
            rec.slot = S.slot;
            rec.energy = S.energy;
            rec.pad = 0u;
            rec.pid = S.L.pid;
            rec.seed = S.L.seed;
            rec.exit_idx = S.exit_idx;
            a.suspend[j] = rec;     // j < grid x block: each lane suspends at most once
            active = false;
            done = true;
        } else {
            // the next step's normals, drawn after this step's arithmetic (as in the batched
            // kernel: the Philox block and the coefficient evaluation are never live together)
            m32::normals(S.L.seed, S.L.pid, S.L.k, z0, z1, z2);
        }
        if (used >= a.budget) done = true;
    }
}

}  // namespace

// Call fn(acc, extended, full) with each flag as a compile-time constant.
template <class Fn>
static void visit_serve(int acc, bool ext, bool full, Fn &&fn)
{
    auto on_acc = [&](auto A) {
        auto on_ext = [&](auto X) {
            if (full) fn(A, X, std::true_type{});
            else fn(A, X, std::false_type{});
        };
        if (ext) on_ext(std::true_type{});
        else on_ext(std::false_type{});
    };
    if (acc == COSMICA_PREC_MIXED_F64ACC) on_acc(std::integral_constant<int, COSMICA_PREC_MIXED_F64ACC>{});
    else on_acc(std::integral_constant<int, COSMICA_PREC_MIXED>{});
}

int serve_max_blocks_per_sm(int acc, bool ext, bool full, unsigned block)
{
    int nb = 0;
    visit_serve(acc, ext, full, [&](auto A, auto X, auto F) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_serve<decltype(A)::value, decltype(X)::value,
                                                                    decltype(F)::value>,
                                                      (int)block, 0);
    });
    return nb;
}

cudaError_t launch_serve(const ServeArgs &a, int acc, bool ext, bool full, PersistentShape shape, cudaStream_t s)
{
    cudaGetLastError();
    visit_serve(acc, ext, full, [&](auto A, auto X, auto F) {
        k_serve<decltype(A)::value, decltype(X)::value, decltype(F)::value><<<shape.grid, shape.block, 0, s>>>(a);
    });
    note_launch();
    return cudaGetLastError();
}

}  // namespace cosmica
