// sfhk_server.cu -- continuous-batching spectrum server (include/sfhk.h,
// "serving").  One host thread per server owns a private context and runs
//   admit -> slice -> harvest
// in a loop: admitted requests are sampled on the device and their work items
// appended to a device ring (one for diatomic targets, one for polyatomic
// ones, whose integrator is a separate kernel); a slice is one launch of the
// integrator over each ring's unprocessed items that stops taking items after
// slice_ms; finished requests are copied out and their device memory released.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sfhk_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

// per-ring counters and slice start times share one small buffer each, one
// entry every kCtrStride bytes
constexpr size_t kCtrStride = 64;

enum ReqState { kPending = 0, kActive = 1, kEnded = 2 };

struct Req {
    uint64_t id = 0;
    sfhk_request r;
    int state = kPending;
    int status = SFHK_OK;
    bool cancel = false;
    sfhk_target* tgt = nullptr;
    sfhk_pulse* pul = nullptr;
    sfhk_ensemble* ens = nullptr;
    int slot = -1;
    int n_items = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int nt = 0;
    double t_origin = 0, dt = 0;
    std::vector<double> vz, yield, phase;
    uint64_t traj_steps = 0, n_filtered = 0, n_unstable = 0, n_nonfinite = 0, recomb_evals = 0;
    int ring = 0;                    // 0: diatomic target, 1: polyatomic
    int poly_slots = 0;              // centre-table rows of a polyatomic target
    bool fixed = false;              // has the fixed parameters (sfhk::fixed_params)
    bool generic = false;            // counted in its ring's n_generic
};

size_t bytes_estimate(uint64_t n, int nt)
{
    // ensemble: SoA 96 B + n0 + perm 8 B per trajectory, items, tables, pulse tables
    return (size_t)n * 104 + ((size_t)n / 32 + 1) * sizeof(sfhk::WorkItem) + (size_t)nt * 80 +
           (1 << 16);
}

int pulse_nt(const sfhk_pulse_desc& d)
{
    if (!(d.lambda_nm > 0.0) || !(d.dt > 0.0) || !(d.n_cycles >= 1.5)) return -1;
    const double omega = 45.5633525 / d.lambda_nm;
    const double Tp = d.n_cycles * 2.0 * 3.14159265358979323846 / omega;
    const double steps = std::floor(Tp / d.dt * (1.0 + 1e-12));
    if (!(steps >= 1.0) || steps > double(1 << 26)) return -1;
    return (int)steps + 1;
}

}  // namespace

struct sfhk_server {
    sfhk_ctx* ctx = nullptr;
    sfhk_server_opts o;
    sfhk_run_opts ro;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<uint64_t> pending;
    std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
    uint64_t next_id = 1;
    Clock::time_point t_start;
    // device side
    cudaStream_t s = nullptr;
    sfhk::DeviceBuf insts, done, cancelf, ctr, t0, spec;   // ctr, t0: one slot per ring
    unsigned int ring_cap = 0, mask = 0;
    // work rings: [0] diatomic, [1] polyatomic targets.  Positions are
    // monotonic except that head steps back when a short request is put in
    // front; they start far from zero so that this is possible even before
    // the first slice has taken anything
    struct Ring {
        sfhk::DeviceBuf items;
        uint64_t head = uint64_t(1) << 40, tail = uint64_t(1) << 40;
        double queued_work = 0;      // items x Nt not yet taken (estimate)
        double rate = 0;             // work taken per second of slice time (smoothed; 0 = none yet)
        int n_generic = 0;           // active requests without the fixed parameters: while
                                     // there are any, the slice runs the generic integrator
        // items the last slice parked (resumed by the next one), in park[cur],
        // and their remaining work (in the units of queued_work)
        sfhk::DeviceBuf park_hdr[2], park_state[2];
        int cur = 0, n_parked = 0;
        double parked_work = 0;
    } rings[2];
    int park_cap = 0;                 // entries of each park buffer
    sfhk::DeviceBuf pctr;             // per ring: resume and park counters (kCtrStride apart)
    unsigned int* h_pctr = nullptr;   // pinned copy of the park counters
    std::vector<int> free_slots;
    std::vector<uint64_t> slot_req;
    unsigned int* h_done = nullptr;   // pinned
    unsigned int* h_ctr = nullptr;    // pinned, one counter per ring (kCtrStride apart)
    int max_nt = 0;
    size_t base_bytes = 0;            // the server's own device buffers
    // stats
    sfhk_server_stats st;

    double now() const
    {
        return std::chrono::duration<double>(Clock::now() - t_start).count();
    }
};

namespace {

void release(sfhk_server* S, Req& q)
{
    if (q.ens) sfhk_destroy_ensemble(q.ens);
    if (q.pul) sfhk_destroy_pulse(q.pul);
    if (q.tgt) sfhk_destroy_target(q.tgt);
    q.ens = nullptr;
    q.pul = nullptr;
    q.tgt = nullptr;
    (void)S;
}

void end_request(sfhk_server* S, Req& q, int status)
{
    // caller holds no lock; takes it for the state change
    std::lock_guard<std::mutex> lk(S->mu);
    q.status = status;
    q.state = kEnded;
    q.t_done = S->now();
    // a request ends once all its items have been taken, so none is left in the ring
    if (q.generic) {
        --S->rings[q.ring].n_generic;
        q.generic = false;
    }
    if (q.slot >= 0) {
        S->slot_req[q.slot] = 0;
        S->free_slots.push_back(q.slot);
        q.slot = -1;
    }
    if (status == SFHK_OK) ++S->st.completed;
    else if (status == SFHK_E_CANCELLED) ++S->st.cancelled;
    else ++S->st.failed;
    S->cv_done.notify_all();
}

// whether an admitted request on ring k has waited longer than the age limit
// of short-first (caller holds the lock)
// the park buffers of both rings, sized for the largest slice launch of the
// server's launch shape (every warp can park one item)
int alloc_park(sfhk_server* S)
{
    const int prec = S->ro.precision;
    sfhk::Ctx* c = S->ctx;
    const int* t = c->tuned[prec][sfhk::kPotAny];    // the server's slices use this shape
    S->park_cap = sfhk::slice_max_warps(prec, t[1], t[0], c->sm_count);
    if (S->park_cap <= 0) return SFHK_E_CUDA;
    const size_t elem = prec == SFHK_MIXED ? sizeof(float) : sizeof(double);
    for (auto& G : S->rings)
        for (int b = 0; b < 2; ++b) {
            int rc = c->alloc(G.park_hdr[b], sizeof(sfhk::ParkHdr) * (size_t)S->park_cap);
            if (!rc)
                rc = c->alloc(G.park_state[b],
                              elem * sfhk::kParkWords * sfhk::kWarp * (size_t)S->park_cap);
            if (rc) return rc;
        }
    return SFHK_OK;
}

bool aged(sfhk_server* S, int k)
{
    if (!(S->o.max_reorder_s > 0.0)) return false;
    const double now = S->now();
    for (uint64_t id : S->slot_req) {
        if (!id) continue;
        const Req* r = S->reqs[id].get();
        if (r->state == kActive && r->ring == k && now - r->t_admit > S->o.max_reorder_s)
            return true;
    }
    return false;
}

// admit queued requests while slots, ring space and memory allow
void admit(sfhk_server* S)
{
    for (;;) {
        Req* q = nullptr;
        int slot = -1;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->pending.empty() || S->free_slots.empty()) return;
            // cancelled requests leave the queue wherever they are
            for (auto it = S->pending.begin(); it != S->pending.end();) {
                Req* c = S->reqs[*it].get();
                if (!c->cancel) {
                    ++it;
                    continue;
                }
                c->status = SFHK_E_CANCELLED;
                c->state = kEnded;
                c->t_done = S->now();
                ++S->st.cancelled;
                S->cv_done.notify_all();
                it = S->pending.erase(it);
            }
            if (S->pending.empty()) return;
            // admission in arrival order (short-first acts on the ring)
            q = S->reqs[S->pending.front()].get();
            const uint64_t items = (q->r.n_traj + 31) / 32;
            const auto& G = S->rings[q->r.target.kind == SFHK_POT_POLYATOMIC ? 1 : 0];
            if (G.tail - G.head + items > S->ring_cap) return;
            // admission horizon: enough work is already queued on this ring
            if (S->o.max_queued_s > 0.0 && (G.tail > G.head || G.n_parked > 0) && G.rate > 0.0 &&
                G.queued_work + G.parked_work >= S->o.max_queued_s * G.rate)
                return;
            const size_t est = bytes_estimate(q->r.n_traj, pulse_nt(q->r.pulse));
            size_t used = 0;
            sfhk_mem_used(S->ctx, &used);
            if (S->o.device_mem_budget && used + est > S->o.device_mem_budget) return;
            S->pending.pop_front();
            slot = S->free_slots.back();
            S->free_slots.pop_back();
            q->slot = slot;
            S->slot_req[slot] = q->id;
        }
        int rc = sfhk_create_target(S->ctx, &q->r.target, &q->tgt);
        if (!rc) rc = sfhk_set_pulse(S->ctx, &q->r.pulse, &q->pul);
        if (!rc)
            rc = sfhk_sample_initial(S->ctx, q->tgt, q->pul, &q->r.align, q->r.n_traj, q->r.seed,
                                     q->r.instance, &q->ens, S->s);
        if (!rc) rc = sfhk::prepare_outputs(q->ens, S->ro, S->s);
        if (!rc) {
            sfhk::DevInstance I = sfhk::make_instance(q->ens, S->ro);
            q->fixed = sfhk::fixed_params(I);
            I.done_items = (unsigned int*)S->done.p + slot;
            I.cancel = (const int*)S->cancelf.p + slot;
            if (cudaMemcpyAsync((sfhk::DevInstance*)S->insts.p + slot, &I, sizeof I,
                                cudaMemcpyHostToDevice, S->s) != cudaSuccess ||
                cudaMemsetAsync((unsigned int*)S->done.p + slot, 0, sizeof(unsigned int), S->s) !=
                    cudaSuccess ||
                cudaMemsetAsync((int*)S->cancelf.p + slot, 0, sizeof(int), S->s) != cudaSuccess)
                rc = SFHK_E_CUDA;
        }
        if (!rc) {
            // work items of this request (instance = its slot), appended to its ring
            sfhk_ensemble* e = q->ens;
            q->ring = q->tgt->dev.kind == SFHK_POT_POLYATOMIC ? 1 : 0;
            q->poly_slots = q->ring ? std::max(1, q->tgt->dev.n_slots) : 0;
            auto& G = S->rings[q->ring];
            rc = sfhk::launch_build_items((const int*)e->perm.p, (const int*)e->n0.p, e->n, slot,
                                          (sfhk::WorkItem*)e->items.p, S->s);
            const unsigned int n = (unsigned int)e->n_items;
            const double work = double(n) * q->pul->nt;
            // short-first: in front of the queued items when smaller than them,
            // unless a request of this ring has waited past the age limit
            bool front;
            uint64_t pos;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                front = !S->o.fifo && G.tail > G.head && work < G.queued_work + G.parked_work &&
                        G.head >= n && !aged(S, q->ring);
                pos = front ? G.head - n : G.tail;
            }
            const unsigned int at = (unsigned int)(pos & S->mask);
            const unsigned int first = std::min(n, S->ring_cap - at);
            sfhk::WorkItem* ring = (sfhk::WorkItem*)G.items.p;
            const sfhk::WorkItem* src = (const sfhk::WorkItem*)e->items.p;
            if (!rc && cudaMemcpyAsync(ring + at, src, sizeof(sfhk::WorkItem) * first,
                                       cudaMemcpyDeviceToDevice, S->s) != cudaSuccess)
                rc = SFHK_E_CUDA;
            if (!rc && n > first &&
                cudaMemcpyAsync(ring, src + first, sizeof(sfhk::WorkItem) * (n - first),
                                cudaMemcpyDeviceToDevice, S->s) != cudaSuccess)
                rc = SFHK_E_CUDA;
            if (!rc) {
                q->n_items = (int)n;
                q->nt = q->pul->nt;
                q->t_origin = q->pul->t_origin;
                q->dt = q->pul->dt;
                std::lock_guard<std::mutex> lk(S->mu);
                if (front) G.head -= n;
                else G.tail += n;
                G.queued_work += work;
                if (!q->fixed) {
                    q->generic = true;
                    ++G.n_generic;
                }
                q->state = kActive;
                q->t_admit = S->now();
            }
        }
        if (rc) {
            cudaStreamSynchronize(S->s);
            release(S, *q);
            end_request(S, *q, rc);
        }
    }
}

// copy out and release every request whose items have all run
void harvest(sfhk_server* S)
{
    std::vector<std::pair<Req*, bool>> ready;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (size_t slot = 0; slot < S->slot_req.size(); ++slot) {
            const uint64_t id = S->slot_req[slot];
            if (!id) continue;
            Req* q = S->reqs[id].get();
            if (q->state == kActive && (int)S->h_done[slot] >= q->n_items)
                ready.emplace_back(q, q->cancel);
        }
    }
    for (auto& rq : ready) {
        Req* q = rq.first;
        int status = rq.second ? SFHK_E_CANCELLED : SFHK_OK;
        if (status == SFHK_OK) {
            sfhk_ensemble* e = q->ens;
            q->vz.resize(q->nt);
            unsigned long long c[6] = {0, 0, 0, 0, 0, 0};
            if (cudaMemcpyAsync(q->vz.data(), e->vz.p, sizeof(double) * q->nt,
                                cudaMemcpyDeviceToHost, S->s) != cudaSuccess ||
                cudaMemcpyAsync(c, e->counters.p, sizeof c, cudaMemcpyDeviceToHost, S->s) !=
                    cudaSuccess)
                status = SFHK_E_CUDA;
            if (status == SFHK_OK && S->o.spectrum) {
                const int n_out = q->nt / 2;
                double* sp = (double*)S->spec.p;           // [twiddle 24 nt | yield | phase]
                double* y = sp + 3 * (size_t)S->max_nt;
                double* ph = y + S->max_nt;
                int rc = sfhk::launch_spectrum((const double*)e->vz.p, q->nt, q->dt, q->t_origin,
                                               0.5 * q->pul->Tp, nullptr, y, ph, n_out,
                                               (double2*)sp, S->s);
                q->yield.resize(n_out);
                q->phase.resize(n_out);
                if (rc || cudaMemcpyAsync(q->yield.data(), y, sizeof(double) * n_out,
                                          cudaMemcpyDeviceToHost, S->s) != cudaSuccess ||
                    cudaMemcpyAsync(q->phase.data(), ph, sizeof(double) * n_out,
                                    cudaMemcpyDeviceToHost, S->s) != cudaSuccess)
                    status = SFHK_E_CUDA;
            }
            if (cudaStreamSynchronize(S->s) != cudaSuccess) status = SFHK_E_CUDA;
            q->n_filtered = c[0];
            q->n_nonfinite = c[1];
            q->traj_steps = c[2];
            q->n_unstable = c[4];
            q->recomb_evals = c[5];
            if (status == SFHK_OK && S->o.check_nonfinite && c[1] > S->o.max_nonfinite) {
                status = SFHK_E_NUMERIC;       // over the limit: no dipole or spectrum
                q->vz.clear();
                q->yield.clear();
                q->phase.clear();
            }
            std::lock_guard<std::mutex> lk(S->mu);
            S->st.traj_steps += c[2];
        }
        release(S, *q);
        end_request(S, *q, status);
    }
}

void run_slice(sfhk_server* S)
{
    uint64_t n64[2];
    int parked[2];                   // items the last slice parked, resumed first
    int slots = 0;                   // centre-table rows the polyatomic slice needs
    bool fixed = false;              // every diatomic request has the fixed parameters
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (int k = 0; k < 2; ++k) {
            n64[k] = S->rings[k].tail - S->rings[k].head;
            parked[k] = S->rings[k].n_parked;
        }
        fixed = S->rings[0].n_generic == 0;
        // cancellations of running requests reach the device before the slice
        for (size_t slot = 0; slot < S->slot_req.size(); ++slot) {
            const uint64_t id = S->slot_req[slot];
            if (!id) continue;
            Req* q = S->reqs[id].get();
            if (q->state == kActive) slots = std::max(slots, q->poly_slots);
            if (q->cancel) {
                static const int one = 1;
                cudaMemcpyAsync((int*)S->cancelf.p + slot, &one, sizeof(int),
                                cudaMemcpyHostToDevice, S->s);
            }
        }
    }
    if (n64[0] == 0 && n64[1] == 0 && parked[0] == 0 && parked[1] == 0) return;
    if ((n64[1] > 0 || parked[1] > 0) && slots < 1) slots = 1;
    int bt = S->ctx->tuned[S->ro.precision][sfhk::kPotAny][0];
    int var = S->ctx->tuned[S->ro.precision][sfhk::kPotAny][1];
    const auto t_a = Clock::now();
    int rc = SFHK_OK;
    int n[2] = {0, 0};
    // one slice of each ring that has work, one after the other on the
    // server's stream (each kernel fills the GPU while it runs)
    bool ran[2] = {false, false};
    for (int k = 0; k < 2 && !rc; ++k) {
        if (n64[k] == 0 && parked[k] == 0) continue;
        auto& G = S->rings[k];
        n[k] = (int)std::min<uint64_t>(n64[k], 0x7fffffffu);
        unsigned int* ctr = (unsigned int*)((char*)S->ctr.p + k * kCtrStride);
        unsigned int* pc = (unsigned int*)((char*)S->pctr.p + k * kCtrStride);
        sfhk::ParkBufs pk;
        pk.in_hdr = (const sfhk::ParkHdr*)G.park_hdr[G.cur].p;
        pk.in_state = G.park_state[G.cur].p;
        pk.n_in = parked[k];
        pk.in_ctr = pc;
        pk.out_hdr = (sfhk::ParkHdr*)G.park_hdr[1 - G.cur].p;
        pk.out_state = G.park_state[1 - G.cur].p;
        pk.out_ctr = pc + 1;
        pk.out_work = (unsigned long long*)(pc + 2);
        pk.cap = S->park_cap;
        rc = sfhk::launch_propagate_slice(
            S->ro.precision, var, (const sfhk::DevInstance*)S->insts.p,
            (const sfhk::WorkItem*)G.items.p, S->mask, (unsigned int)(G.head & S->mask), n[k],
            ctr, (unsigned long long)(S->o.slice_ms * 1e6),
            (unsigned long long*)((char*)S->t0.p + k * kCtrStride), bt, S->ctx->sm_count, S->s,
            pk, k == 1 ? slots : 0, k == 0 && fixed);
        if (!rc && (cudaMemcpyAsync((char*)S->h_ctr + k * kCtrStride, ctr, sizeof(unsigned int),
                                    cudaMemcpyDeviceToHost, S->s) != cudaSuccess ||
                    cudaMemcpyAsync((char*)S->h_pctr + k * kCtrStride, pc,
                                    2 * sizeof(unsigned int) + sizeof(unsigned long long),
                                    cudaMemcpyDeviceToHost, S->s) != cudaSuccess))
            rc = SFHK_E_CUDA;
        ran[k] = !rc;
    }
    if (!rc && cudaMemcpyAsync(S->h_done, S->done.p, sizeof(unsigned int) * S->slot_req.size(),
                               cudaMemcpyDeviceToHost, S->s) != cudaSuccess)
        rc = SFHK_E_CUDA;
    if (!rc && cudaStreamSynchronize(S->s) != cudaSuccess) rc = SFHK_E_CUDA;
    const double busy = std::chrono::duration<double>(Clock::now() - t_a).count();
    std::lock_guard<std::mutex> lk(S->mu);
    ++S->st.slices;
    S->st.gpu_busy_s += busy;
    if (!rc) {
        for (int k = 0; k < 2; ++k) {
            if (!ran[k]) continue;
            auto& G = S->rings[k];
            const double before = G.queued_work + G.parked_work;
            // this slice's parked items are the next slice's to resume; their
            // remaining work stays queued
            const unsigned int* hp =
                (const unsigned int*)((const char*)S->h_pctr + k * kCtrStride);
            G.n_parked = (int)std::min<unsigned int>(hp[1], (unsigned int)S->park_cap);
            G.parked_work = (double)*(const unsigned long long*)(hp + 2);
            G.cur = 1 - G.cur;
            S->st.parked += (uint64_t)G.n_parked;
            uint64_t taken = 0;
            if (n64[k] > 0) {
                const unsigned int got =
                    *(const unsigned int*)((const char*)S->h_ctr + k * kCtrStride);
                taken = std::min<uint64_t>(got, (uint64_t)n[k]);
                G.queued_work = taken >= n64[k]
                                    ? 0.0
                                    : G.queued_work * double(n64[k] - taken) / double(n64[k]);
                G.head += taken;
            }
            // the ring's rate over a slice that did not run out of work (a
            // drained ring says nothing about how fast it goes)
            if ((taken < n64[k] || G.n_parked > 0) && busy > 0.0) {
                const double r = (before - G.queued_work - G.parked_work) / busy;
                G.rate = G.rate > 0.0 ? 0.7 * G.rate + 0.3 * r : r;
            }
        }
    }
}

void loop(sfhk_server* S)
{
    cudaSetDevice(S->ctx->device);
    uint64_t seen = 0;
    for (;;) {
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->stop) break;
        }
        admit(S);
        bool work;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            work = S->rings[0].tail > S->rings[0].head || S->rings[1].tail > S->rings[1].head ||
                   S->rings[0].n_parked > 0 || S->rings[1].n_parked > 0;
        }
        if (work) {
            run_slice(S);
            harvest(S);
        } else {
            // nothing on the device: sleep until a submission, a cancellation
            // check or shutdown (a queued request that does not fit yet waits here)
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv_work.wait_for(lk, std::chrono::milliseconds(2),
                                [&] { return S->stop || S->st.submitted != seen; });
            seen = S->st.submitted;
        }
    }
    cudaStreamSynchronize(S->s);
    for (auto& kv : S->reqs) release(S, *kv.second);
}

int copy_result(Req& q, sfhk_result* r)
{
    if (!r) return SFHK_OK;
    r->status = q.status;
    r->nt = q.nt;
    r->t_origin = q.t_origin;
    r->dt = q.dt;
    r->n_out = q.nt / 2;
    if (r->vz && !q.vz.empty())
        std::memcpy(r->vz, q.vz.data(), sizeof(double) * std::min(r->vz_capacity, q.vz.size()));
    if (r->yield && !q.yield.empty())
        std::memcpy(r->yield, q.yield.data(),
                    sizeof(double) * std::min(r->spec_capacity, q.yield.size()));
    if (r->phase && !q.phase.empty())
        std::memcpy(r->phase, q.phase.data(),
                    sizeof(double) * std::min(r->spec_capacity, q.phase.size()));
    r->t_submit = q.t_submit;
    r->t_admit = q.t_admit;
    r->t_done = q.t_done;
    r->traj_steps = q.traj_steps;
    r->n_filtered = q.n_filtered;
    r->n_unstable = q.n_unstable;
    r->n_nonfinite = q.n_nonfinite;
    r->recomb_evals = q.recomb_evals;
    return SFHK_OK;
}

}  // namespace

extern "C" {

int sfhk_server_create(int device, const sfhk_server_opts* opts, sfhk_server** out)
{
    if (!opts || !out) return SFHK_E_INVAL;
    if (opts->precision != SFHK_FP64 && opts->precision != SFHK_MIXED) return SFHK_E_INVAL;
    if (!(opts->stability_taper == 0.0 || opts->stability_taper > 1.0) ||
        !std::isfinite(opts->stability_taper))
        return SFHK_E_INVAL;
    if (!(opts->gamma > 0.0) || opts->prefactor_cutoff < 0.0 || opts->stability_cutoff < 0.0 ||
        opts->slice_ms < 0.0 || opts->max_pending < 0 || opts->max_active < 0 ||
        (opts->check_nonfinite != 0 && opts->check_nonfinite != 1) ||
        !(opts->max_reorder_s >= 0.0) || !(opts->max_queued_s >= 0.0))
        return SFHK_E_INVAL;
    sfhk_server* S = new (std::nothrow) sfhk_server;
    if (!S) return SFHK_E_NOMEM;
    S->o = *opts;
    if (S->o.max_pending == 0) S->o.max_pending = 4096;
    if (S->o.max_active == 0) S->o.max_active = 512;
    if (S->o.slice_ms == 0.0) S->o.slice_ms = 50.0;
    std::memset(&S->st, 0, sizeof S->st);
    std::memset(&S->ro, 0, sizeof S->ro);
    S->ro.precision = opts->precision;
    S->ro.gamma = opts->gamma;
    S->ro.prefactor_cutoff = opts->prefactor_cutoff;
    S->ro.stability_cutoff = opts->stability_cutoff;
    S->ro.stability_taper = opts->stability_taper;
    int rc = sfhk_create(&S->ctx, device, 0);
    if (rc) {
        delete S;
        return rc;
    }
    S->max_nt = (1 << 16);
    S->ring_cap = 1u << 22;                  // work items per ring (64 MiB)
    S->mask = S->ring_cap - 1;
    sfhk::Ctx* c = S->ctx;
    if ((rc = c->alloc(S->insts, sizeof(sfhk::DevInstance) * S->o.max_active)) ||
        (rc = c->alloc(S->rings[0].items, sizeof(sfhk::WorkItem) * (size_t)S->ring_cap)) ||
        (rc = c->alloc(S->rings[1].items, sizeof(sfhk::WorkItem) * (size_t)S->ring_cap)) ||
        (rc = c->alloc(S->done, sizeof(unsigned int) * S->o.max_active)) ||
        (rc = c->alloc(S->cancelf, sizeof(int) * S->o.max_active)) ||
        (rc = c->alloc(S->ctr, 2 * kCtrStride)) || (rc = c->alloc(S->t0, 2 * kCtrStride)) ||
        (rc = c->alloc(S->pctr, 2 * kCtrStride)) ||
        (rc = c->alloc(S->spec, sizeof(double) * 5 * (size_t)S->max_nt)) ||
        (rc = alloc_park(S))) {
        sfhk_destroy(S->ctx);
        delete S;
        return rc;
    }
    if (cudaStreamCreateWithFlags(&S->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaHostAlloc((void**)&S->h_done, sizeof(unsigned int) * S->o.max_active,
                      cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&S->h_ctr, 2 * kCtrStride, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void**)&S->h_pctr, 2 * kCtrStride, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        sfhk_destroy(S->ctx);
        delete S;
        return SFHK_E_CUDA;
    }
    std::memset(S->h_done, 0, sizeof(unsigned int) * S->o.max_active);
    sfhk_mem_used(S->ctx, &S->base_bytes);
    S->slot_req.assign(S->o.max_active, 0);
    for (int i = S->o.max_active - 1; i >= 0; --i) S->free_slots.push_back(i);
    S->t_start = Clock::now();
    S->th = std::thread(loop, S);
    *out = S;
    return SFHK_OK;
}

int sfhk_server_destroy(sfhk_server* S)
{
    if (!S) return SFHK_E_INVAL;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    sfhk::Ctx* c = S->ctx;
    for (sfhk::DeviceBuf* b : {&S->insts, &S->rings[0].items, &S->rings[1].items, &S->done,
                               &S->cancelf, &S->ctr, &S->t0, &S->pctr, &S->spec})
        c->release(*b);
    for (auto& G : S->rings)
        for (int b = 0; b < 2; ++b) {
            c->release(G.park_hdr[b]);
            c->release(G.park_state[b]);
        }
    if (S->s) cudaStreamDestroy(S->s);
    if (S->h_done) cudaFreeHost(S->h_done);
    if (S->h_ctr) cudaFreeHost(S->h_ctr);
    if (S->h_pctr) cudaFreeHost(S->h_pctr);
    sfhk_destroy(S->ctx);
    delete S;
    return SFHK_OK;
}

int sfhk_submit(sfhk_server* S, const sfhk_request* r, uint64_t* id)
{
    if (!S || !r || !id) return SFHK_E_INVAL;
    const int nt = pulse_nt(r->pulse);
    if (nt < 2 || nt > S->max_nt || r->n_traj == 0 || r->n_traj > 2147483647ull ||
        !(r->target.Ip > 0.0) || r->target.n_prim < 1 || r->target.n_prim > SFHK_MAX_PRIM ||
        !sfhk::align_valid(r->align) ||
        (r->target.kind == SFHK_POT_POLYATOMIC &&
         (r->align.kind == SFHK_ALIGN_QUADRATURE || r->target.ionization != SFHK_IONIZE_SFA)))
        return SFHK_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    const size_t est = bytes_estimate(r->n_traj, nt);
    if ((int)S->pending.size() >= S->o.max_pending ||
        (S->o.device_mem_budget && est + S->base_bytes > S->o.device_mem_budget) ||
        (r->n_traj + 31) / 32 > S->ring_cap) {
        ++S->st.rejected;
        return SFHK_E_NOMEM;
    }
    auto q = std::make_unique<Req>();
    q->id = S->next_id++;
    q->r = *r;
    q->t_submit = S->now();
    *id = q->id;
    S->pending.push_back(q->id);
    S->reqs.emplace(q->id, std::move(q));
    ++S->st.submitted;
    S->cv_work.notify_all();
    return SFHK_OK;
}

int sfhk_poll(sfhk_server* S, uint64_t id, sfhk_result* r)
{
    if (!S) return SFHK_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return SFHK_E_NOTFOUND;
    if (it->second->state != kEnded) return SFHK_E_BUSY;
    copy_result(*it->second, r);
    S->reqs.erase(it);
    return SFHK_OK;
}

int sfhk_wait(sfhk_server* S, uint64_t id, double timeout_s, sfhk_result* r)
{
    if (!S) return SFHK_E_INVAL;
    std::unique_lock<std::mutex> lk(S->mu);
    auto ended = [&] {
        auto it = S->reqs.find(id);
        return it == S->reqs.end() || it->second->state == kEnded;
    };
    if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), ended))
        return SFHK_E_TIMEOUT;
    auto it = S->reqs.find(id);
    if (it == S->reqs.end()) return SFHK_E_NOTFOUND;
    copy_result(*it->second, r);
    S->reqs.erase(it);
    return SFHK_OK;
}

int sfhk_cancel(sfhk_server* S, uint64_t id)
{
    if (!S) return SFHK_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end() || it->second->state == kEnded) return SFHK_E_NOTFOUND;
    it->second->cancel = true;
    return SFHK_OK;
}

int sfhk_server_stats_get(sfhk_server* S, sfhk_server_stats* out)
{
    if (!S || !out) return SFHK_E_INVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->pending = (int)S->pending.size();
    int active = 0;
    for (uint64_t id : S->slot_req) active += id != 0;
    out->active = active;
    out->uptime_s = S->now();
    size_t used = 0;
    sfhk_mem_used(S->ctx, &used);
    out->device_bytes = used;
    return SFHK_OK;
}

}  // extern "C"
