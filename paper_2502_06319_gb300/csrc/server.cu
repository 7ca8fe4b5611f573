// server.cu -- continuous-batching spectrum server (cosmica_server_*).
//
// A scheduler thread owns one CUDA stream and loops over quanta.  Before each
// quantum it admits waiting requests first come, first served, as long as a
// parameter slot and a contiguous range of the exit arena are free (the
// arena is the memory budget: 49 B per admitted particle); after it, it
// retires finished requests (histogram + spectrum on their arena range,
// copied to host memory) and frees their memory.  Particles still in flight
// at the end of a quantum are suspended exactly on the device and resumed by
// the next quantum together with the fresh particles of newly admitted
// requests, so new arrivals overlap with running work.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "cosmica.h"
#include "host_util.h"
#include "internal.h"

using namespace cosmica;
using namespace cosmica::host;

namespace {

struct Req {
    cosmica_params p;
    cosmica_species sp;
    std::vector<double> T;
    std::vector<uint32_t> n;
    std::vector<uint64_t> e_off;     // offset of each energy within the request
    std::vector<uint64_t> started;   // fresh particles handed to a quantum, per energy
    uint64_t seed = 0, total = 0, steps = 0;
    cosmica_bins bins{};
    int state = 0;                   // 0 waiting, 1 admitted, 2 done, 3 failed
    int slot = -1;
    uint64_t base = 0;               // first exit-arena index
    std::vector<double> J, S;
    std::vector<uint64_t> H;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

// first-fit allocator of contiguous particle ranges in the exit arena
struct RangeAlloc {
    std::map<uint64_t, uint64_t> free_;   // offset -> length
    uint64_t used = 0;
    void init(uint64_t cap) { free_.clear(); if (cap) free_[0] = cap; used = 0; }
    bool alloc(uint64_t n, uint64_t *off)
    {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= n) {
                *off = it->first;
                const uint64_t rest = it->second - n, at = it->first + n;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used += n;
                return true;
            }
        }
        return false;
    }
    void release(uint64_t off, uint64_t n)
    {
        used -= n;
        auto it = free_.emplace(off, n).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
};

constexpr uint32_t kMaxSlots = 256;
constexpr uint32_t kMaxEnergies = 256;
constexpr uint32_t kMaxBins = 8192;

double now_s(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct cosmica_server {
    int device = 0, precision = COSMICA_PREC_MIXED;
    uint32_t budget = 4096;
    cudaStream_t stream = nullptr;
    std::chrono::steady_clock::time_point t0;
    PersistentShape shape{128, 1};
    // device memory, allocated at create
    void *arena_mem = nullptr;
    ExitPtrs arena{};
    uint64_t arena_cap = 0;
    DevParams *d_prm = nullptr;
    DevSpecies *d_spc = nullptr;
    unsigned int *d_done = nullptr;
    unsigned long long *d_steps = nullptr;
    Suspended *d_susp[2] = {nullptr, nullptr};
    uint64_t lane_cap = 0;
    unsigned int *d_nsusp = nullptr;
    unsigned long long *d_cursors = nullptr;
    unsigned long long *d_hist = nullptr;
    double *d_J = nullptr, *d_S = nullptr;
    SpecItem *d_spec_items = nullptr;
    DevBuf tables;
    Staging stage;
    // pinned read-back of the per-quantum counters
    unsigned long long *h_cursor = nullptr;
    unsigned int *h_nsusp = nullptr;
    unsigned int *h_done = nullptr;
    unsigned long long *h_steps = nullptr;
    // host bookkeeping (guarded by mu)
    std::mutex mu;
    std::condition_variable cv_submit, cv_done;
    std::deque<uint64_t> waiting;
    std::map<uint64_t, Req> reqs;
    std::vector<int> free_slots;
    RangeAlloc ranges;
    uint64_t next_ticket = 1;
    bool stop = false, failed = false;
    std::string fail_msg;
    cosmica_server_stats st{};
    std::thread th;
    // scheduler-thread state
    uint64_t n_resume = 0;
    int cur = 0;

    void run();
    bool quantum(std::vector<uint64_t> &admitted_now);
    bool retire(uint64_t ticket, Req &r);
    bool upload_slot(Req &r);
    void set_failed(const std::string &m)
    {
        std::lock_guard<std::mutex> lk(mu);
        failed = true;
        fail_msg = m;
        for (auto &kv : reqs)
            if (kv.second.state < 2) kv.second.state = 3;
        cv_done.notify_all();
    }
};

bool cosmica_server::upload_slot(Req &r)
{
    DevParams dp = to_dev(r.p);
    DevSpecies ds = to_dev(r.sp);
    cudaError_t e = cudaMemcpyAsync(d_prm + r.slot, &dp, sizeof(dp), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_spc + r.slot, &ds, sizeof(ds), cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = launch_derive(d_prm + r.slot, 1, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_done + r.slot, 0, sizeof(unsigned int), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_steps + r.slot, 0, sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);   // dp, ds live on this stack frame
    if (e != cudaSuccess) {
        set_failed(std::string("server slot upload: ") + cudaGetErrorString(e));
        return false;
    }
    return true;
}

bool cosmica_server::retire(uint64_t ticket, Req &r)
{
    const uint32_t nE = (uint32_t)r.T.size(), nb = r.bins.nbins, stride = nb + 3u;
    const double x_lo = std::log10(r.bins.P_min_GV);
    const double dx = (std::log10(r.bins.P_max_GV) - x_lo) / (double)nb;
    ExitPtrs ex{arena.r + r.base, arena.th + r.base, arena.ph + r.base, arena.lnP + r.base, arena.s + r.base,
                arena.steps + r.base, arena.status + r.base, arena.item + r.base};
    std::vector<SpecItem> its(nE);
    for (uint32_t e = 0; e < nE; ++e) its[e] = SpecItem{r.T[e], (double)r.sp.A, (double)r.sp.Z, r.sp.m0_GeV};
    r.H.assign((size_t)nE * stride, 0);
    r.J.assign(nE, 0.0);
    r.S.assign(nE, 0.0);
    cudaError_t e = cudaMemsetAsync(d_hist, 0, (size_t)nE * stride * 8, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_spec_items, its.data(), nE * sizeof(SpecItem),
                                              cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = launch_histogram(ex, r.total, nE, nb, x_lo, dx, d_hist, stream);
    if (e == cudaSuccess)
        e = launch_spectrum(d_hist, nE, nb, x_lo, dx, d_spec_items, 0, nullptr, nullptr, 0, d_J, d_S, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.H.data(), d_hist, (size_t)nE * stride * 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.J.data(), d_J, nE * 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(r.S.data(), d_S, nE * 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        set_failed(std::string("server retire: ") + cudaGetErrorString(e));
        return false;
    }
    std::lock_guard<std::mutex> lk(mu);
    r.state = 2;
    r.t_done = now_s(t0);
    ranges.release(r.base, r.total);
    free_slots.push_back(r.slot);
    st.completed += 1;
    st.steps += r.steps;
    cv_done.notify_all();
    (void)ticket;
    return true;
}

bool cosmica_server::quantum(std::vector<uint64_t> &admitted_now)
{
    for (uint64_t t : admitted_now) {
        Req *r;
        {
            std::lock_guard<std::mutex> lk(mu);
            r = &reqs[t];
        }
        if (!upload_slot(*r)) return false;
    }
    // fresh slices of every admitted request, oldest first
    std::vector<ServeItem> its;
    std::vector<uint64_t> pre(1, 0);
    std::vector<std::pair<uint64_t, uint32_t>> owner;   // (ticket, energy) per item
    bool ext = false;   // a resident request has radial shells or a squashed heliosphere
    bool full = true;   // every resident request is the full model
    {
        std::lock_guard<std::mutex> lk(mu);
        for (auto &kv : reqs) {
            Req &r = kv.second;
            if (r.state != 1) continue;
            ext = ext || r.p.n_shells > 0 || r.p.squashed != 0;
            full = full && full_model(r.p);
            for (uint32_t e = 0; e < r.T.size(); ++e) {
                const uint64_t left = r.n[e] - r.started[e];
                if (!left) continue;
                its.push_back(ServeItem{r.T[e], r.e_off[e] + r.started[e], r.seed, r.base + r.e_off[e] + r.started[e],
                                        (uint32_t)r.slot, e});
                pre.push_back(pre.back() + left);
                owner.emplace_back(kv.first, e);
            }
        }
    }
    const uint64_t n_fresh = pre.back();
    if (n_fresh == 0 && n_resume == 0) return true;
    const size_t nI = its.size();
    const size_t b_items = align_up(std::max<size_t>(1, nI) * sizeof(ServeItem), 256);
    const size_t b_pre = align_up((nI + 1) * sizeof(uint64_t), 256);
    if (tables.reserve(b_items + b_pre) != COSMICA_OK || stage.reserve(b_items + b_pre) != COSMICA_OK) {
        set_failed(std::string("server tables: ") + cosmica_last_error());
        return false;
    }
    std::memcpy(stage.h, its.data(), nI * sizeof(ServeItem));
    std::memcpy((char *)stage.h + b_items, pre.data(), (nI + 1) * sizeof(uint64_t));
    if (stage.upload(tables.d, b_items + b_pre, stream) != COSMICA_OK) {
        set_failed(std::string("server tables: ") + cosmica_last_error());
        return false;
    }
    const auto q0 = std::chrono::steady_clock::now();
    ServeArgs a;
    a.prm = d_prm;
    a.spc = d_spc;
    a.items = (const ServeItem *)tables.d;
    a.prefix = (const uint64_t *)((char *)tables.d + b_items);
    a.n_items = (uint32_t)nI;
    a.n_fresh = n_fresh;
    a.resume = d_susp[cur];
    a.n_resume = n_resume;
    a.suspend = d_susp[cur ^ 1];
    a.n_suspend = d_nsusp;
    a.cursors = d_cursors;
    a.arena = arena;
    a.req_done = d_done;
    a.req_steps = d_steps;
    a.budget = budget;
    cudaError_t e = cudaMemsetAsync(d_cursors, 0, 2 * sizeof(unsigned long long), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_nsusp, 0, sizeof(unsigned int), stream);
    if (e == cudaSuccess) e = launch_serve(a, precision, ext, full, shape, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_cursor, d_cursors, sizeof(unsigned long long), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_nsusp, d_nsusp, sizeof(unsigned int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_done, d_done, kMaxSlots * sizeof(unsigned int), cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h_steps, d_steps, kMaxSlots * 8, cudaMemcpyDeviceToHost, stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) {
        set_failed(std::string("server quantum: ") + cudaGetErrorString(e));
        return false;
    }
    // account the fresh particles this quantum started, in table order
    uint64_t taken = std::min<uint64_t>(*h_cursor, n_fresh);
    std::vector<uint64_t> done_tickets;
    {
        std::lock_guard<std::mutex> lk(mu);
        for (size_t i = 0; i < nI && taken; ++i) {
            const uint64_t cnt = std::min<uint64_t>(taken, pre[i + 1] - pre[i]);
            reqs[owner[i].first].started[owner[i].second] += cnt;
            taken -= cnt;
        }
        st.quanta += 1;
        st.busy_seconds += std::chrono::duration<double>(std::chrono::steady_clock::now() - q0).count();
        uint64_t inflight = 0;
        for (auto &kv : reqs) {
            Req &r = kv.second;
            if (r.state != 1) continue;
            const uint64_t d = h_done[r.slot];
            inflight += r.total - d;
            if (d == r.total) {
                r.steps = h_steps[r.slot];
                done_tickets.push_back(kv.first);
            }
        }
        st.in_flight_particles = inflight;
    }
    n_resume = *h_nsusp;
    cur ^= 1;
    for (uint64_t t : done_tickets) {
        Req *r;
        {
            std::lock_guard<std::mutex> lk(mu);
            r = &reqs[t];
        }
        if (!retire(t, *r)) return false;
    }
    return true;
}

void cosmica_server::run()
{
    cudaSetDevice(device);
    while (true) {
        std::vector<uint64_t> admitted_now;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) break;   // in-flight particles are abandoned with the server
            while (!waiting.empty() && !free_slots.empty()) {
                Req &r = reqs[waiting.front()];
                uint64_t off;
                if (!ranges.alloc(r.total, &off)) break;   // first come, first served: wait for memory
                r.base = off;
                r.slot = free_slots.back();
                free_slots.pop_back();
                r.state = 1;
                r.t_admit = now_s(t0);
                admitted_now.push_back(waiting.front());
                waiting.pop_front();
                st.admitted += 1;
            }
            st.arena_used = ranges.used;
            bool any_admitted = false;
            for (auto &kv : reqs)
                if (kv.second.state == 1) { any_admitted = true; break; }
            if (!any_admitted && n_resume == 0 && admitted_now.empty()) {
                cv_submit.wait_for(lk, std::chrono::milliseconds(2));
                continue;
            }
        }
        if (!quantum(admitted_now)) break;
    }
}

extern "C" cosmica_status cosmica_server_create(size_t mem_budget, int32_t precision, uint32_t budget_steps,
                                                cosmica_server **out)
{
    if (!out) return fail(COSMICA_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (precision != COSMICA_PREC_MIXED && precision != COSMICA_PREC_MIXED_F64ACC)
        return fail(COSMICA_ERR_INVALID, "server precision must be MIXED or MIXED_F64ACC");
    cosmica_server *s = new (std::nothrow) cosmica_server();
    if (!s) return fail(COSMICA_ERR_OOM, "host allocation of the server");
    s->precision = precision;
    s->budget = budget_steps ? budget_steps : 4096u;
    s->t0 = std::chrono::steady_clock::now();
    cudaGetDevice(&s->device);
    const unsigned block = 128;
    // sized for the full model's kernel (the common case); a variant with fewer resident
    // blocks (extended heliosphere, or a model without drift or sheet) starts its extra
    // blocks as others finish, and they take whatever work is left
    const int bps = std::max(1, serve_max_blocks_per_sm(precision, false, true, block));
    s->shape = PersistentShape{block, (unsigned)(num_sms() * bps), 0u};
    s->lane_cap = (uint64_t)s->shape.grid * block;
    const size_t fixed = 2 * s->lane_cap * sizeof(Suspended) + kMaxSlots * (sizeof(DevParams) + sizeof(DevSpecies) + 12) +
                         (size_t)kMaxEnergies * (kMaxBins + 3) * 8 + kMaxEnergies * (16 + sizeof(SpecItem)) + 4096;
    const size_t per = 5 * 8 + 4 + 4 + 1;
    if (mem_budget <= fixed + 256 * per) {
        delete s;
        return fail(COSMICA_ERR_INVALID, "mem_budget %zu below the server's fixed %zu bytes", mem_budget, fixed);
    }
    s->arena_cap = (mem_budget - fixed) / per - 64;
    const uint64_t C = s->arena_cap;
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    auto A = [&](void **p, size_t n) { if (e == cudaSuccess) e = cudaMalloc(p, n); };
    A(&s->arena_mem, C * per + 8 * 256);
    A((void **)&s->d_prm, kMaxSlots * sizeof(DevParams));
    A((void **)&s->d_spc, kMaxSlots * sizeof(DevSpecies));
    A((void **)&s->d_done, kMaxSlots * sizeof(unsigned int));
    A((void **)&s->d_steps, kMaxSlots * 8);
    A((void **)&s->d_susp[0], s->lane_cap * sizeof(Suspended));
    A((void **)&s->d_susp[1], s->lane_cap * sizeof(Suspended));
    A((void **)&s->d_nsusp, sizeof(unsigned int));
    A((void **)&s->d_cursors, 2 * sizeof(unsigned long long));
    A((void **)&s->d_hist, (size_t)kMaxEnergies * (kMaxBins + 3) * 8);
    A((void **)&s->d_J, kMaxEnergies * 8);
    A((void **)&s->d_S, kMaxEnergies * 8);
    A((void **)&s->d_spec_items, kMaxEnergies * sizeof(SpecItem));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s->h_cursor, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s->h_nsusp, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s->h_done, kMaxSlots * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s->h_steps, kMaxSlots * 8);
    if (e == cudaSuccess) e = cudaMemset(s->d_done, 0, kMaxSlots * sizeof(unsigned int));
    if (e != cudaSuccess) {
        cosmica_status rs = cuda_fail(e, "server allocation");
        cosmica_server_destroy(s);
        return rs;
    }
    char *p = (char *)s->arena_mem;
    auto take = [&](size_t n) { char *q = p; p += align_up(n, 256); return q; };
    s->arena.r = (double *)take(C * 8); s->arena.th = (double *)take(C * 8); s->arena.ph = (double *)take(C * 8);
    s->arena.lnP = (double *)take(C * 8); s->arena.s = (double *)take(C * 8);
    s->arena.steps = (uint32_t *)take(C * 4); s->arena.item = (uint32_t *)take(C * 4);
    s->arena.status = (uint8_t *)take(C);
    s->ranges.init(C);
    for (int i = (int)kMaxSlots - 1; i >= 0; --i) s->free_slots.push_back(i);
    s->st.arena_capacity = C;
    s->th = std::thread([s] { s->run(); });
    *out = s;
    return COSMICA_OK;
}

extern "C" cosmica_status cosmica_server_submit(cosmica_server *s, const cosmica_request *q, uint64_t *ticket)
{
    if (!s || !q || !ticket) return fail(COSMICA_ERR_INVALID, "server / request / ticket is NULL");
    cosmica_status stt = check_params(&q->params);
    if (stt != COSMICA_OK) return stt;
    stt = check_species(&q->species);
    if (stt != COSMICA_OK) return stt;
    if (q->params.precision != s->precision) return fail(COSMICA_ERR_INVALID, "request precision differs from the server's");
    if (q->params.formulation != 0) return fail(COSMICA_ERR_INVALID, "the server runs the momentum form only");
    if (q->n_energies == 0 || q->n_energies > kMaxEnergies || !q->T_GeVn || !q->n_per_energy)
        return fail(COSMICA_ERR_INVALID, "need 1..%u energies with T and counts", kMaxEnergies);
    if (!(q->bins.P_min_GV > 0.0 && q->bins.P_max_GV > q->bins.P_min_GV && q->bins.nbins >= 1 &&
          q->bins.nbins <= kMaxBins))
        return fail(COSMICA_ERR_INVALID, "bins: need 0 < P_min < P_max and 1..%u bins", kMaxBins);
    Req r;
    r.p = q->params;
    r.sp = q->species;
    r.T.assign(q->T_GeVn, q->T_GeVn + q->n_energies);
    r.n.assign(q->n_per_energy, q->n_per_energy + q->n_energies);
    r.seed = q->seed;
    r.bins = q->bins;
    r.e_off.resize(q->n_energies);
    r.started.assign(q->n_energies, 0);
    for (uint32_t e = 0; e < q->n_energies; ++e) {
        if (!(std::isfinite(r.T[e]) && r.T[e] > 0.0)) return fail(COSMICA_ERR_INVALID, "T[%u] must be > 0", e);
        r.e_off[e] = r.total;
        r.total += r.n[e];
    }
    if (r.total == 0) return fail(COSMICA_ERR_INVALID, "request has no particles");
    if (r.total > s->arena_cap) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->st.rejected += 1;
        return fail(COSMICA_ERR_INVALID, "request of %llu particles exceeds the server's memory (%llu)",
                    (unsigned long long)r.total, (unsigned long long)s->arena_cap);
    }
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->failed) return fail(COSMICA_ERR_CUDA, "server failed: %s", s->fail_msg.c_str());
    r.t_submit = now_s(s->t0);
    const uint64_t t = s->next_ticket++;
    s->reqs.emplace(t, std::move(r));
    s->waiting.push_back(t);
    s->st.submitted += 1;
    *ticket = t;
    s->cv_submit.notify_all();
    return COSMICA_OK;
}

static cosmica_status take_result(cosmica_server *s, std::map<uint64_t, Req>::iterator it, cosmica_result *res)
{
    Req &r = it->second;
    if (res) {
        if (res->J) std::memcpy(res->J, r.J.data(), r.J.size() * 8);
        if (res->sigma) std::memcpy(res->sigma, r.S.data(), r.S.size() * 8);
        if (res->hist) std::memcpy(res->hist, r.H.data(), r.H.size() * 8);
        res->steps = r.steps;
        res->t_submit = r.t_submit;
        res->t_admit = r.t_admit;
        res->t_done = r.t_done;
    }
    s->reqs.erase(it);
    return COSMICA_OK;
}

extern "C" cosmica_status cosmica_server_poll(cosmica_server *s, uint64_t ticket, cosmica_result *res)
{
    if (!s) return fail(COSMICA_ERR_INVALID, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(COSMICA_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second.state == 3) return fail(COSMICA_ERR_CUDA, "server failed: %s", s->fail_msg.c_str());
    if (it->second.state != 2) return COSMICA_ERR_BUSY;
    return take_result(s, it, res);
}

extern "C" cosmica_status cosmica_server_wait(cosmica_server *s, uint64_t ticket, uint32_t timeout_ms,
                                              cosmica_result *res)
{
    if (!s) return fail(COSMICA_ERR_INVALID, "server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(COSMICA_ERR_INVALID, "unknown ticket %llu", (unsigned long long)ticket);
    const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        auto jt = s->reqs.find(ticket);
        return jt == s->reqs.end() || jt->second.state >= 2;
    });
    it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(COSMICA_ERR_INVALID, "ticket %llu was taken", (unsigned long long)ticket);
    if (it->second.state == 3) return fail(COSMICA_ERR_CUDA, "server failed: %s", s->fail_msg.c_str());
    if (!ok) return fail(COSMICA_ERR_TIMEOUT, "request %llu not finished after %u ms", (unsigned long long)ticket,
                         timeout_ms);
    return take_result(s, it, res);
}

extern "C" cosmica_status cosmica_server_stats_get(cosmica_server *s, cosmica_server_stats *st)
{
    if (!s || !st) return fail(COSMICA_ERR_INVALID, "server / stats is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    *st = s->st;
    st->arena_used = s->ranges.used;
    return COSMICA_OK;
}

extern "C" void cosmica_server_destroy(cosmica_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        s->waiting.clear();
        for (auto &kv : s->reqs)
            if (kv.second.state < 2) kv.second.state = 3;
        s->fail_msg = "server destroyed";
        s->cv_submit.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    if (s->stream) cudaStreamSynchronize(s->stream);
    s->tables.release();
    s->stage.release();
    void *dev[] = {s->arena_mem, s->d_prm, s->d_spc, s->d_done, s->d_steps, s->d_susp[0], s->d_susp[1],
                   s->d_nsusp, s->d_cursors, s->d_hist, s->d_J, s->d_S, s->d_spec_items};
    for (void *p : dev)
        if (p) cudaFree(p);
    void *hst[] = {s->h_cursor, s->h_nsusp, s->h_done, s->h_steps};
    for (void *p : hst)
        if (p) cudaFreeHost(p);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}
