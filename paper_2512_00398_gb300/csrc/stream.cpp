// stream.cpp -- the streaming runtime behind hp_stream_* (include/hp.h):
// gulps of many beams searched as they arrive, each beam's tail of earlier
// gulps resident on the device, beams admitted by device budget, and the
// gulps that are ready batched into steps by a native scheduler thread
// (continuous batching, up to two steps in flight).
//
// The gulp rule (Sections III-B, V-C: chunks whose time segments overlap so a
// dispersed pulse stays whole; Section IV-C: transfers overlapped with
// computation): gulp g of a beam searches input [B0, E), E = (g+1) G,
// B0 = max(0, g G - H), H = max_delay + Wmax - 1, reports runs whose first
// boxcar start lies in the window [0, nwin), nwin = E - H - B0, and passes a
// per-(trial, width) "run still open" flag to the next gulp.
//
// Device memory (one allocation): per step slot j < max_batch a search
// workspace for G + H samples and a candidate buffer; per beam slot a ring of
// R = ceil(H / G) + 1 gulps ([G][nchans] each; the buffer of gulp g is gulps
// g - R + 1 .. g) and two [ndm][nw] carry arrays used alternately.  Host
// uploads, kernels and result copies of a step are ordered on one stream, so a
// ring slot is rewritten only after every step that read it has finished.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "plan_internal.h"

using namespace hp;

namespace {

constexpr int kMaxRing = 64;
constexpr int kSets = 2;   // steps in flight (pinned result sets)

size_t al256(size_t v) { return (v + 255) / 256 * 256; }

int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch())
        .count();
}

struct Pending {
    int64_t index;
    const uint8_t* host;
    int64_t t_push;
};

struct BeamSlot {
    uint8_t* ring = nullptr;
    uint8_t* carry[2] = {nullptr, nullptr};
    int beam = -1;
};

struct Beam {
    int slot = -1;
    bool waiting = false;
    bool ended = false;
    int64_t pushed = 0;
    int64_t done = 0;
    int parity = 0;            // carry array that holds the latest flags
    bool have_carry = false;   // a searched gulp has written them
    std::deque<Pending> q;
};

struct Item {
    int beam, slot;
    const uint8_t* host;
    int64_t index, B0, E, nwin, t_push;
    bool carry_valid;
    int cin;                   // carry array read (the other one is written)
};

struct Step {
    std::vector<Item> items;
    int set = 0;
    bool complete = false;
    int error = HP_OK;
    int64_t t_done = 0;
    hp_stream* owner = nullptr;   // (declared in hp.h)
};

struct Result {
    hp_gulp_result r;
    std::vector<hp_cand> cands;
};

}  // namespace

struct hp_stream {
    hp_plan* plan = nullptr;               // the stream's own copy
    hp_stream_config cfg{};
    int device = 0;
    int64_t G = 0, H = 0;
    int R = 0, nch = 0, ndm = 0, nw = 0, max_batch = 0, beam_slots = 0;
    size_t ws_bytes = 0, cand_dev_bytes = 0, beam_bytes = 0, set_bytes = 0, per_item_host = 0;
    uint8_t* arena = nullptr;
    size_t arena_bytes = 0;
    uint8_t* pinned = nullptr;
    std::vector<uint8_t*> ws;
    std::vector<hp_cand*> dcand;
    std::vector<int64_t*> dcount;
    std::vector<BeamSlot> slots;
    std::deque<int> free_slots;
    std::vector<Beam> beams;
    std::deque<int> wait_q;
    cudaStream_t main = nullptr;
    std::vector<cudaStream_t> side;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    std::thread th;
    std::mutex mu;
    std::condition_variable cv, cv_res;
    bool stop = false;
    int error = HP_OK;
    std::deque<Step*> inflight;
    bool set_busy[kSets] = {false, false};
    std::deque<Result> results;
    int64_t steps_done = 0, gulps_done = 0, max_batch_seen = 0;
};

namespace {

void CUDART_CB step_done(void* arg) {
    Step* st = static_cast<Step*>(arg);
    hp_stream* s = st->owner;
    std::lock_guard<std::mutex> lk(s->mu);
    st->complete = true;
    st->t_done = now_ns();
    s->cv.notify_all();
}

uint8_t* set_base(hp_stream* s, int set) { return s->pinned + (size_t)set * s->set_bytes; }
int* set_status(hp_stream* s, int set) { return reinterpret_cast<int*>(set_base(s, set)); }
int64_t* item_count(hp_stream* s, int set, int j) {
    return reinterpret_cast<int64_t*>(set_base(s, set) + 256 + (size_t)j * s->per_item_host);
}
hp_cand* item_cands(hp_stream* s, int set, int j) {
    return reinterpret_cast<hp_cand*>(set_base(s, set) + 256 + (size_t)j * s->per_item_host + 64);
}

// Buffer geometry of gulp g.
void geometry(const hp_stream* s, int64_t g, int64_t* B0, int64_t* E, int64_t* nwin) {
    *E = (g + 1) * s->G;
    *B0 = std::max<int64_t>(0, g * s->G - s->H);
    *nwin = *E - s->H - *B0;
}

// (under the lock) release the slot of a beam that ended and finished
void maybe_release(hp_stream* s, int b) {
    Beam& B = s->beams[b];
    if (B.slot < 0 || !B.ended || B.done != B.pushed || !B.q.empty()) return;
    s->slots[B.slot].beam = -1;
    s->free_slots.push_back(B.slot);
    B.slot = -1;
}

// (under the lock) give free slots to waiting beams, first come first served
void admit(hp_stream* s) {
    while (!s->free_slots.empty() && !s->wait_q.empty()) {
        const int b = s->wait_q.front();
        s->wait_q.pop_front();
        Beam& B = s->beams[b];
        B.waiting = false;
        if (B.ended && B.q.empty()) continue;
        const int sl = s->free_slots.front();
        s->free_slots.pop_front();
        s->slots[sl].beam = b;
        B.slot = sl;
        B.parity = 0;
        B.have_carry = false;
    }
}

// (under the lock) finished steps, oldest first: results to the queue
void retire(hp_stream* s) {
    while (!s->inflight.empty() && s->inflight.front()->complete) {
        Step* st = s->inflight.front();
        s->inflight.pop_front();
        const int status = st->error ? st->error : *set_status(s, st->set);
        int j = 0;
        for (const Item& it : st->items) {
            Result res;
            std::memset(&res.r, 0, sizeof(res.r));
            res.r.beam = it.beam;
            res.r.status = status;
            res.r.gulp_index = it.index;
            res.r.window_start = it.B0;
            res.r.window_len = std::max<int64_t>(it.nwin, 0);
            res.r.latency_s = (double)(st->t_done - it.t_push) * 1e-9;
            res.r.batch_size = (int32_t)st->items.size();
            if (it.nwin > 0 && !st->error) {
                const int64_t n = *item_count(s, st->set, j);
                res.r.ncand = n;
                const int64_t keep = std::min<int64_t>(n, s->cfg.cand_capacity);
                const hp_cand* c = item_cands(s, st->set, j);
                res.cands.assign(c, c + std::max<int64_t>(keep, 0));
            }
            if (it.nwin > 0) ++j;
            s->results.push_back(std::move(res));
            Beam& B = s->beams[it.beam];
            ++B.done;
            maybe_release(s, it.beam);
            ++s->gulps_done;
        }
        s->set_busy[st->set] = false;
        ++s->steps_done;
        delete st;
        s->cv_res.notify_all();
    }
}

// (under the lock) the gulps that are ready: at most one per admitted beam,
// oldest push first, up to max_batch
Step* form_step(hp_stream* s) {
    int set = -1;
    for (int k = 0; k < kSets; ++k)
        if (!s->set_busy[k]) { set = k; break; }
    if (set < 0) return nullptr;
    std::vector<std::pair<int64_t, int>> ready;
    for (size_t sl = 0; sl < s->slots.size(); ++sl) {
        const int b = s->slots[sl].beam;
        if (b >= 0 && !s->beams[b].q.empty()) ready.push_back({s->beams[b].q.front().t_push, b});
    }
    if (ready.empty()) return nullptr;
    std::sort(ready.begin(), ready.end());
    if ((int)ready.size() > s->max_batch) ready.resize(s->max_batch);
    Step* st = new (std::nothrow) Step;
    if (!st) return nullptr;
    st->set = set;
    st->owner = s;
    for (const auto& r : ready) {
        Beam& B = s->beams[r.second];
        const Pending p = B.q.front();
        B.q.pop_front();
        Item it;
        it.beam = r.second;
        it.slot = B.slot;
        it.host = p.host;
        it.index = p.index;
        it.t_push = p.t_push;
        geometry(s, p.index, &it.B0, &it.E, &it.nwin);
        it.carry_valid = B.have_carry;
        it.cin = B.parity;
        if (it.nwin > 0) {
            B.parity ^= 1;
            B.have_carry = true;
        }
        st->items.push_back(it);
    }
    s->set_busy[set] = true;
    s->max_batch_seen = std::max<int64_t>(s->max_batch_seen, (int64_t)st->items.size());
    return st;
}

// Enqueue one step (no lock held: only this thread touches the device state).
int enqueue_step(hp_stream* s, Step* st) {
    hp_plan* p = s->plan;
    cudaStream_t m = s->main;
    const size_t gbytes = (size_t)s->G * s->nch;
    int rc = HP_OK;
    // this step's gulps into their ring slots (after every earlier step on m)
    for (const Item& it : st->items) {
        uint8_t* dst = s->slots[it.slot].ring + (size_t)(it.index % s->R) * gbytes;
        rc = check_cuda(cudaMemcpyAsync(dst, it.host, gbytes, cudaMemcpyHostToDevice, m));
        if (rc) return rc;
    }
    TransposeBatch tb;
    std::memset(&tb, 0, sizeof(tb));
    DedispBatch db;
    std::memset(&db, 0, sizeof(db));
    std::vector<Layout> Ls;
    std::vector<const Item*> work;
    for (const Item& it : st->items) {
        if (it.nwin <= 0) continue;
        const int j = (int)work.size();
        const int64_t nsamps = it.E - it.B0;
        Ls.push_back(make_layout(p, nsamps, true));
        const Layout& L = Ls.back();
        // the plan's parameters set the layout; one changed since the stream
        // opened may need more than the step slot holds
        if (L.total > s->ws_bytes) return HP_ERR_INVALID_ARG;
        uint8_t* ws = s->ws[j];
        TransposeJob J = make_transpose_job(s->slots[it.slot].ring, nsamps, s->nch, ws + L.xt,
                                            L.xt_pitch);
        J.ring_len = s->G;
        J.a0 = it.B0;
        J.ring_slots = s->R;
        tb.jobs[j] = J;
        tb.prefix[j + 1] = tb.prefix[j] + J.ttiles * J.ctiles;
        if (p->sb_chans <= 0) {   // the sub-band variant runs its own two stages per gulp
            if (!reach_ok(p, L.nout, L.xt_pitch)) return HP_ERR_INVALID_ARG;
            db.jobs[j] = make_job(p, ws + L.xt, L.xt_pitch, (int32_t*)(ws + L.D), L.dpitch, L.nout);
            fuse_levels(db.jobs[j], L, ws);
            db.prefix[j + 1] = db.prefix[j] + (int64_t)db.jobs[j].ntt * db.jobs[j].ndt;
        }
        work.push_back(&it);
    }
    const int n = (int)work.size();
    if (n > 0) {
        tb.njobs = n;
        db.njobs = p->sb_chans > 0 ? 0 : n;
        rc = check_cuda(launch_transpose_batch(tb, m));
        int64_t rfi_kernels = 0;
        for (int j = 0; j < n && !rc && p->rfi; ++j) {   // RFI mitigation per searched buffer
            const RfiArgs r = make_rfi_args(p, Ls[j], s->ws[j], nullptr, s->ws[j] + Ls[j].xt,
                                            Ls[j].xt_pitch, work[j]->E - work[j]->B0, nullptr);
            rc = check_cuda(launch_rfi(r, m, &rfi_kernels));
        }
        if (!rc && db.njobs > 0)
            rc = check_cuda(launch_dedisp(p->dedisp_cfg, db, p->status, p->timeout_ns, m));
        for (int j = 0; j < n && !rc && p->sb_chans > 0; ++j)
            rc = run_subband(p, Ls[j], s->ws[j], (int32_t*)(s->ws[j] + Ls[j].D), Ls[j].dpitch, m);
        if (!rc) rc = check_cuda(cudaEventRecord(s->fork, m));
        if (rc) return rc;
        int64_t kernels = 0;
        for (int j = 0; j < n; ++j) {
            const Item& it = *work[j];
            const Layout& L = Ls[j];
            uint8_t* ws = s->ws[j];
            cudaStream_t sj = s->side[j];
            BeamSlot& B = s->slots[it.slot];
            rc = check_cuda(cudaStreamWaitEvent(sj, s->fork, 0));
            if (rc) return rc;
            hp_raw_cand* raw = (hp_raw_cand*)(ws + L.raw);
            int64_t* raw_count = (int64_t*)(ws + L.raw_count);
            SearchArgs a = make_search_args(p, L, ws, (int32_t*)(ws + L.D), L.dpitch, L.nout, raw,
                                            p->raw_capacity, raw_count);
            if (p->sb_chans <= 0) fuse_levels(a, L, ws, p->dedisp_cfg);
            a.nwin = it.nwin;
            a.carry_in = it.carry_valid ? B.carry[it.cin] : nullptr;
            a.carry_out = B.carry[it.cin ^ 1];
            a.t_offset = it.B0;
            rc = check_cuda(launch_search(a, sj, &kernels));
            if (rc) return rc;
            hp_cand_buf out;
            out.data = s->dcand[j];
            out.capacity = s->cfg.cand_capacity;
            out.count = s->dcount[j];
            MergeArgs mg = make_merge_args(p, L, ws, raw, raw_count, p->raw_capacity, a.sigma, &out);
            mg.sigw = a.width_sigma ? a.sigw : nullptr;
            rc = check_cuda(launch_merge(mg, sj, &kernels));
            if (rc) return rc;
            rc = check_cuda(cudaMemcpyAsync(item_count(s, st->set, j), s->dcount[j], sizeof(int64_t),
                                            cudaMemcpyDeviceToHost, sj));
            if (!rc)
                rc = check_cuda(cudaMemcpyAsync(item_cands(s, st->set, j), s->dcand[j],
                                                (size_t)s->cfg.cand_capacity * sizeof(hp_cand),
                                                cudaMemcpyDeviceToHost, sj));
            if (!rc) rc = check_cuda(cudaEventRecord(s->joins[j], sj));
            if (!rc) rc = check_cuda(cudaStreamWaitEvent(m, s->joins[j], 0));
            if (rc) return rc;
        }
    }
    // the step's device status (timeouts, overflows), then clear it
    rc = check_cuda(cudaMemcpyAsync(set_status(s, st->set), p->status, sizeof(int),
                                    cudaMemcpyDeviceToHost, m));
    if (!rc) rc = check_cuda(cudaMemsetAsync(p->status, 0, sizeof(int), m));
    if (!rc) rc = check_cuda(cudaLaunchHostFunc(m, step_done, st));
    return rc;
}

void scheduler(hp_stream* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        retire(s);
        admit(s);
        if (s->stop && s->inflight.empty()) break;
        Step* st = nullptr;
        if (!s->stop && s->error == HP_OK && (int)s->inflight.size() < kSets) st = form_step(s);
        if (st) {
            lk.unlock();
            const int rc = enqueue_step(s, st);
            lk.lock();
            if (rc) {
                // nothing more is enqueued after a failed call: wait for the
                // device, then report the step's gulps with the error
                lk.unlock();
                cudaStreamSynchronize(s->main);
                for (cudaStream_t x : s->side) cudaStreamSynchronize(x);
                lk.lock();
                s->error = rc;
                st->error = rc;
                st->complete = true;
                st->t_done = now_ns();
            }
            s->inflight.push_back(st);
            continue;
        }
        s->cv.wait(lk);
    }
}

int copy_plan(const hp_plan* t, int64_t raw_capacity, hp_plan** out) {
    std::vector<int> w(t->widths.begin(), t->widths.end());
    int rc = hp_plan_create(out, t->nchans, t->f_top, t->chan_bw, t->tsamp, t->dm_list.data(),
                            t->ndm(), w.data(), t->nw(), t->thr);
    if (rc) return rc;
    hp_plan* p = *out;
    p->baseline_mode = t->baseline_mode;
    p->baseline_s = t->baseline_s;
    p->dm_tol = t->dm_tol;
    p->t_gap = t->t_gap;
    p->w_tol = t->w_tol;
    p->dedisp_cfg = t->dedisp_cfg;
    p->dedisp_cfg_set = t->dedisp_cfg_set;
    p->timeout_ns = t->timeout_ns;
    p->raw_capacity = raw_capacity;
    p->rfi = t->rfi;
    p->rfi_nb_k = t->rfi_nb_k;
    p->rfi_bb_k = t->rfi_bb_k;
    p->width_sigma = t->width_sigma;
    if (t->sb_chans > 0) {
        rc = hp_plan_set_param(p, HP_PARAM_SUBBAND_GROUP, t->sb_group);
        if (!rc) rc = hp_plan_set_param(p, HP_PARAM_SUBBAND_CHANS, t->sb_chans);
        if (rc) {
            hp_plan_destroy(p);
            *out = nullptr;
            return rc;
        }
    }
    return HP_OK;
}

void release(hp_stream* s) {
    if (s->main) cudaStreamSynchronize(s->main);
    for (cudaStream_t x : s->side) {
        cudaStreamSynchronize(x);
        cudaStreamDestroy(x);
    }
    for (cudaEvent_t e : s->joins) cudaEventDestroy(e);
    if (s->fork) cudaEventDestroy(s->fork);
    if (s->main) cudaStreamDestroy(s->main);
    if (s->arena) cudaFree(s->arena);
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->plan) hp_plan_destroy(s->plan);
    delete s;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

int hp_stream_open(hp_stream** out, const hp_plan* tmpl, const hp_stream_config* cfg) {
    if (!out) return HP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!tmpl || !cfg) return HP_ERR_INVALID_ARG;
    if (tmpl->decimate > 0) return HP_ERR_INVALID_ARG;   // every start in a stream's window
    if (cfg->nbeams < 1 || cfg->nbeams > HP_STREAM_MAX_BEAMS) return HP_ERR_INVALID_ARG;
    if (cfg->max_batch < 0 || cfg->max_batch > HP_BATCH_MAX_FILES) return HP_ERR_INVALID_ARG;
    if (cfg->gulp < 64 || cfg->gulp >= kMaxSamples / 4) return HP_ERR_INVALID_ARG;
    if (cfg->hbm_budget < 0 || cfg->cand_capacity < 1 || cfg->cand_capacity > ((int64_t)1 << 24))
        return HP_ERR_INVALID_ARG;
    if (cfg->raw_capacity < 1024 || cfg->raw_capacity > ((int64_t)1 << 30)) return HP_ERR_INVALID_ARG;
    hp_stream* s = new (std::nothrow) hp_stream;
    if (!s) return HP_ERR_OOM;
    s->cfg = *cfg;
    int rc = copy_plan(tmpl, cfg->raw_capacity, &s->plan);
    if (rc) { delete s; return rc; }
    hp_plan* p = s->plan;
    s->G = cfg->gulp;
    s->H = (int64_t)p->maxd + p->wmax - 1;
    s->R = (int)((s->H + s->G - 1) / s->G) + 1;
    s->nch = p->nchans;
    s->ndm = p->ndm();
    s->nw = p->nw();
    if (s->R > kMaxRing) { release(s); return HP_ERR_INVALID_ARG; }
    if (cudaGetDevice(&s->device) != cudaSuccess) { release(s); return HP_ERR_CUDA; }
    rc = ensure_device_tables(p);
    if (rc) { release(s); return rc; }

    // sizes: step slots (search workspace + candidates), beam slots (ring + carries)
    const Layout L = make_layout(p, s->G + s->H, true);
    s->ws_bytes = al256(L.total);
    s->cand_dev_bytes = 256 + al256((size_t)cfg->cand_capacity * sizeof(hp_cand));
    s->beam_bytes = al256((size_t)s->R * s->G * s->nch) + 2 * al256((size_t)s->ndm * s->nw);
    int mb = cfg->max_batch ? cfg->max_batch : std::min(cfg->nbeams, HP_BATCH_MAX_FILES);
    mb = std::min(mb, cfg->nbeams);
    int slots = cfg->nbeams;
    if (cfg->hbm_budget > 0) {
        const int64_t avail = cfg->hbm_budget - (int64_t)p->tables_bytes;
        const int64_t step1 = (int64_t)(s->ws_bytes + s->cand_dev_bytes);
        while (mb >= 1 && mb * step1 + (int64_t)s->beam_bytes > avail) --mb;
        if (mb < 1) { release(s); return HP_ERR_OOM; }
        slots = (int)std::min<int64_t>(cfg->nbeams, (avail - mb * step1) / (int64_t)s->beam_bytes);
        mb = std::min(mb, slots);
    }
    s->max_batch = mb;
    s->beam_slots = slots;
    s->arena_bytes = (size_t)mb * (s->ws_bytes + s->cand_dev_bytes) + (size_t)slots * s->beam_bytes;
    rc = check_cuda(cudaMalloc(&s->arena, s->arena_bytes));
    if (rc) { s->arena = nullptr; release(s); return rc; }
    uint8_t* a = s->arena;
    for (int j = 0; j < mb; ++j) {
        s->ws.push_back(a);
        a += s->ws_bytes;
        s->dcount.push_back((int64_t*)a);
        s->dcand.push_back((hp_cand*)(a + 256));
        a += s->cand_dev_bytes;
    }
    s->slots.resize(slots);
    for (int k = 0; k < slots; ++k) {
        s->slots[k].ring = a;
        a += al256((size_t)s->R * s->G * s->nch);
        s->slots[k].carry[0] = a;
        a += al256((size_t)s->ndm * s->nw);
        s->slots[k].carry[1] = a;
        a += al256((size_t)s->ndm * s->nw);
        s->free_slots.push_back(k);
    }
    // pinned host results: per set a status word, then per step slot the count
    // and the candidates
    s->per_item_host = 64 + al256((size_t)cfg->cand_capacity * sizeof(hp_cand));
    s->set_bytes = 256 + (size_t)mb * s->per_item_host;
    void* hbuf = nullptr;
    rc = check_cuda(cudaHostAlloc(&hbuf, kSets * s->set_bytes, cudaHostAllocDefault));
    if (rc) { release(s); return rc; }
    s->pinned = (uint8_t*)hbuf;
    std::memset(s->pinned, 0, kSets * s->set_bytes);
    rc = check_cuda(cudaStreamCreateWithFlags(&s->main, cudaStreamNonBlocking));
    if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&s->fork, cudaEventDisableTiming));
    for (int j = 0; j < mb && !rc; ++j) {
        cudaStream_t x;
        cudaEvent_t e;
        rc = check_cuda(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
        if (rc) break;
        s->side.push_back(x);
        rc = check_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        if (rc) break;
        s->joins.push_back(e);
    }
    if (rc) { release(s); return rc; }
    s->beams.resize(cfg->nbeams);
    try {
        s->th = std::thread(scheduler, s);
    } catch (...) {
        release(s);
        return HP_ERR_OOM;
    }
    *out = s;
    return HP_OK;
}

int hp_stream_push(hp_stream* s, int beam, const uint8_t* gulp_host, int64_t nsamps) {
    if (!s || !gulp_host) return HP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->error) return s->error;
    if (beam < 0 || beam >= (int)s->beams.size() || nsamps != s->G || s->stop)
        return HP_ERR_INVALID_ARG;
    Beam& B = s->beams[beam];
    if (B.ended || (B.pushed + 2) * s->G >= kMaxSamples) return HP_ERR_INVALID_ARG;
    B.q.push_back({B.pushed++, gulp_host, now_ns()});
    if (B.slot < 0 && !B.waiting) {
        B.waiting = true;
        s->wait_q.push_back(beam);
    }
    s->cv.notify_all();
    return HP_OK;
}

int hp_stream_end_beam(hp_stream* s, int beam) {
    if (!s) return HP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (beam < 0 || beam >= (int)s->beams.size()) return HP_ERR_INVALID_ARG;
    s->beams[beam].ended = true;
    maybe_release(s, beam);
    s->cv.notify_all();
    return HP_OK;
}

int hp_stream_poll(hp_stream* s, hp_gulp_result* result, hp_cand* cands, int64_t cand_cap,
                   int timeout_ms) {
    if (!s || !result || cand_cap < 0 || (cand_cap > 0 && !cands)) return HP_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    auto ready = [&] { return !s->results.empty(); };
    if (timeout_ms < 0)
        s->cv_res.wait(lk, ready);
    else if (!s->cv_res.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return HP_STREAM_EMPTY;
    Result r = std::move(s->results.front());
    s->results.pop_front();
    lk.unlock();
    *result = r.r;
    const int64_t n = std::min<int64_t>((int64_t)r.cands.size(), cand_cap);
    if (n > 0) std::memcpy(cands, r.cands.data(), (size_t)n * sizeof(hp_cand));
    return HP_OK;
}

int hp_stream_get_stats(hp_stream* s, hp_stream_stats* out) {
    if (!s || !out) return HP_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->steps = s->steps_done;
    out->gulps = s->gulps_done;
    out->beam_slots = s->beam_slots;
    out->max_batch = s->max_batch;
    for (const BeamSlot& b : s->slots) out->admitted += b.beam >= 0;
    out->waiting = (int32_t)s->wait_q.size();
    out->device_bytes = (int64_t)(s->arena_bytes + s->plan->tables_bytes);
    out->tail_samples = s->H;
    out->max_batch_seen = s->max_batch_seen;
    out->device_allocs = (s->arena ? 1 : 0) + s->plan->device_allocs;
    return HP_OK;
}

int hp_stream_close(hp_stream* s) {
    if (!s) return HP_OK;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
        for (Beam& B : s->beams) B.q.clear();
        s->cv.notify_all();
    }
    if (s->th.joinable()) s->th.join();
    release(s);
    return HP_OK;
}

}  // extern "C"
