// K8: serving with continuous batching.
//
// A worker thread runs the loop:
//   admit   pending requests while a slot (max_active) and arena space are
//           free; upload their parameters and sample all their
//           perturbations on their scene's lane (stream);
//   batch   per lane, one render launch (the persistent / per-item render
//           kernels of that scene) over chunks of every active request on the
//           scene, through a by-value table of (request buffers, perturbation
//           range); a request whose last chunk is in the launch gets its sums
//           and result copy queued right after it;
//   retire  requests whose completion event fired: copy the result, free the
//           slot and the arena block, wake the waiter.
// Lanes keep at most two batched launches in flight, so new requests join
// within a chunk's time.  Newton-CG step requests replay the state's step on
// the state's own stream; a step request waits in the queue while its state
// has a step in flight, so steps on one state run in submission order.
// Waits on the device are event queries; the worker sleeps briefly when
// nothing progressed.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hr.h"
#include "hr_api_internal.h"
#include "hr_device.cuh"
#include "hr_internal.h"

using namespace hr;

namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxResultBytes = HR_MAX_PARAMS * HR_MAX_PARAMS * 8;

size_t up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct SrvReq {
    uint64_t ticket = 0;
    hr_request req{};
    std::vector<double> theta, v;
    int n = 0, E = 0, G = 0, P = 0;
    int64_t M = 0, Mt = 0;
    // arena block and the request's device buffers inside it
    size_t off = 0, bytes = 0;
    float* theta32 = nullptr;
    double* vdev = nullptr;
    SampleGroup* groups = nullptr;
    float* tau = nullptr;
    float* w = nullptr;
    uint2* meta = nullptr;
    float* loss = nullptr;
    double* flat = nullptr;
    double* full = nullptr;
    int64_t launched = 0;
    bool finishing = false;
    cudaEvent_t done = nullptr;
    int slot = -1;
    int state = 0;   // 0 queued, 1 active, 2 done
    hr_status status = HR_OK;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int batches = 0;
    std::vector<unsigned char> result;
};

struct Lane {
    cudaStream_t stream = nullptr;
    std::deque<cudaEvent_t> inflight;
};

// first-fit allocator over the arena, adjacent free blocks merged
struct Arena {
    unsigned char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_blocks;   // offset -> bytes
    bool alloc(size_t bytes, size_t& off) {
        for (auto it = free_blocks.begin(); it != free_blocks.end(); ++it) {
            if (it->second >= bytes) {
                off = it->first;
                const size_t rest = it->second - bytes;
                free_blocks.erase(it);
                if (rest) free_blocks[off + bytes] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        auto it = free_blocks.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_blocks.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_blocks.erase(nx);
        }
        if (it != free_blocks.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_blocks.erase(it);
            }
        }
    }
};

int n_elem(int quantity, int n) { return quantity == HR_HESSIAN ? n * (n + 1) / 2 : n; }

size_t request_bytes(int n, int E, int G, int64_t Mt) {
    return up(sizeof(float) * n) + up(sizeof(double) * n) + up(sizeof(SampleGroup) * (size_t)G) +
           up(sizeof(float) * (size_t)Mt * n) + up(sizeof(float) * (size_t)Mt * E) + up(sizeof(uint2) * (size_t)Mt) +
           up(sizeof(float) * (size_t)Mt) + up(sizeof(double) * E) + up(sizeof(double) * n * n);
}

}  // namespace

struct hr_server_s {
    hr_server_opts opts{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::deque<SrvReq*> pending;
    std::unordered_map<uint64_t, SrvReq*> tickets;
    uint64_t next_ticket = 1;
    std::thread worker;
    // worker-owned
    std::vector<SrvReq*> active;
    Arena arena;
    unsigned char* pinned = nullptr;
    std::vector<int> free_slots;
    // optimizer states with a step in flight (worker thread only, like
    // free_slots): a second step request on the same state waits in the
    // queue, since both would copy their step records into the state's one
    // pinned buffer
    std::vector<hr_optstate> busy_states;
    std::unordered_map<hr_scene, Lane> lanes;
    cudaStream_t upload = nullptr;
    std::vector<cudaEvent_t> event_pool;
    std::chrono::steady_clock::time_point t0;

    double now_ms() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    cudaEvent_t get_event() {
        if (!event_pool.empty()) {
            cudaEvent_t e = event_pool.back();
            event_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        return e;
    }
    void put_event(cudaEvent_t e) { if (e) event_pool.push_back(e); }
    Lane& lane(hr_scene sc) {
        Lane& l = lanes[sc];
        if (!l.stream) cudaStreamCreateWithFlags(&l.stream, cudaStreamNonBlocking);
        return l;
    }

    bool admit(SrvReq* r);
    void setup(SrvReq* r);
    bool launch_batches();
    bool retire();
    void run();
};

bool hr_server_s::admit(SrvReq* r) {
    if (free_slots.empty()) return false;
    if (r->req.quantity == HR_NEWTON_STEP) {
        if (std::find(busy_states.begin(), busy_states.end(), r->req.optstate) != busy_states.end()) return false;
        busy_states.push_back(r->req.optstate);
        r->slot = free_slots.back();
        free_slots.pop_back();
        return true;
    }
    size_t off = 0;
    if (!arena.alloc(r->bytes, off)) return false;
    r->off = off;
    r->slot = free_slots.back();
    free_slots.pop_back();
    return true;
}

// Upload parameters and group table, then sample every perturbation.
void hr_server_s::setup(SrvReq* r) {
    r->t_admit = now_ms();
    if (r->req.quantity == HR_NEWTON_STEP) {
        const hr_status s = optstate_launch_step(r->req.optstate, true);
        if (s != HR_OK) { r->status = s; return; }
        r->done = get_event();
        cudaEventRecord(r->done, optstate_stream(r->req.optstate));
        r->finishing = true;
        return;
    }
    const int n = r->n;
    unsigned char* b = arena.base + r->off;
    size_t o = 0;
    r->theta32 = reinterpret_cast<float*>(b + o); o += up(sizeof(float) * n);
    r->vdev = reinterpret_cast<double*>(b + o); o += up(sizeof(double) * n);
    r->groups = reinterpret_cast<SampleGroup*>(b + o); o += up(sizeof(SampleGroup) * (size_t)r->G);
    r->tau = reinterpret_cast<float*>(b + o); o += up(sizeof(float) * (size_t)r->Mt * n);
    r->w = reinterpret_cast<float*>(b + o); o += up(sizeof(float) * (size_t)r->Mt * r->E);
    r->meta = reinterpret_cast<uint2*>(b + o); o += up(sizeof(uint2) * (size_t)r->Mt);
    r->loss = reinterpret_cast<float*>(b + o); o += up(sizeof(float) * (size_t)r->Mt);
    r->flat = reinterpret_cast<double*>(b + o); o += up(sizeof(double) * r->E);
    r->full = reinterpret_cast<double*>(b + o);
    // staging: theta32 | v | groups, laid out as in the arena
    const size_t head = up(sizeof(float) * n) + up(sizeof(double) * n) + up(sizeof(SampleGroup) * (size_t)r->G);
    std::vector<unsigned char> stage(head, 0);
    float* t32 = reinterpret_cast<float*>(stage.data());
    for (int i = 0; i < n; ++i) t32[i] = (float)r->theta[i];
    if (!r->v.empty()) memcpy(stage.data() + up(sizeof(float) * n), r->v.data(), sizeof(double) * n);
    SampleGroup* gs = reinterpret_cast<SampleGroup*>(stage.data() + up(sizeof(float) * n) + up(sizeof(double) * n));
    const hr_opts& o2 = r->req.opts;
    for (int g = 0; g < r->G; ++g) {
        SampleGroup& gr = gs[g];
        gr.m0 = (int32_t)(g * r->M);
        gr.P = r->P;
        gr.lobe = r->req.quantity == HR_GRAD ? 0 : 1;
        gr.quantity = r->req.quantity;
        gr.sub = o2.sub + (uint32_t)g;
        gr.request = o2.request_id;
        gr.theta_row = 0;
        gr.pad = 0;
        if (o2.strategy == HR_AGGREGATE) { gr.comp_i = -1; gr.comp_j = -1; }
        else if (o2.strategy == HR_PLAIN) { gr.comp_i = -3; gr.comp_j = -3; }
        else if (r->req.quantity == HR_GRAD) { gr.comp_i = g; gr.comp_j = g; }
        else if (r->req.quantity == HR_HVP) { gr.comp_i = g; gr.comp_j = -2; gr.quantity = 4; }
        else {
            int row = 0, rem = g;
            while (rem >= n - row) { rem -= n - row; ++row; }
            gr.comp_i = row; gr.comp_j = row + rem;
        }
    }
    Lane& L = lane(r->req.scene);
    cudaError_t e = cudaMemcpyAsync(b, stage.data(), head, cudaMemcpyHostToDevice, upload);
    cudaEvent_t up_ev = get_event();
    if (e == cudaSuccess) e = cudaEventRecord(up_ev, upload);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(L.stream, up_ev, 0);
    if (e != cudaSuccess) { r->status = HR_ERR_CUDA; put_event(up_ev); return; }
    SampleArgs sa{};
    sa.groups = r->groups;
    sa.n = n;
    sa.E = r->E;
    sa.sigma = o2.sigma;
    const double s2 = o2.sigma * o2.sigma;
    sa.Zg = std::sqrt(2.0 / M_PI) / o2.sigma;
    sa.Zd = 4.0 * std::exp(-0.5) / (std::sqrt(2.0 * M_PI) * s2);
    sa.Zo = sa.Zg * sa.Zg;
    sa.seed = o2.seed;
    sa.v = r->req.quantity == HR_HVP ? r->vdev : nullptr;   // also the row-mixture weights
    sa.tau = r->tau;
    sa.w = r->w;
    sa.invS = nullptr;
    sa.meta = r->meta;
    sa.step = nullptr;
    sa.threads = r->req.scene->sc.sample_threads;
    launch_sample(sa, r->G, r->P, L.stream);
    // the upload event may be reused once the lane has consumed it
    cudaEventRecord(up_ev, L.stream);
    L.inflight.push_back(up_ev);
}

bool hr_server_s::launch_batches() {
    bool progress = false;
    for (auto& kv : lanes) {
        hr_scene sc = kv.first;
        Lane& L = kv.second;
        while (!L.inflight.empty() && cudaEventQuery(L.inflight.front()) == cudaSuccess) {
            put_event(L.inflight.front());
            L.inflight.pop_front();
        }
        if (L.inflight.size() >= 3) continue;
        RenderBatch rb{};
        std::vector<SrvReq*> rows, closing;
        int items = 0;
        for (SrvReq* r : active) {
            if (r->req.scene != sc || r->req.quantity == HR_NEWTON_STEP || r->finishing || r->status != HR_OK) continue;
            if (r->launched >= r->Mt || (int)rows.size() >= kMaxBatchRows) continue;
            const int64_t c = std::min<int64_t>(opts.chunk, r->Mt - r->launched);
            BatchRow& br = rb.rows[rows.size()];
            br.theta32 = r->theta32;
            br.tau = r->tau;
            br.meta = r->meta;
            br.loss = r->loss;
            br.seed = r->req.opts.seed;
            br.request = r->req.opts.request_id;
            br.m_begin = (int32_t)r->launched;
            br.start = items;
            br.pad = 0;
            items += (int)c;
            r->launched += c;
            r->batches += 1;
            rows.push_back(r);
            if (r->launched == r->Mt) closing.push_back(r);
        }
        if (rows.empty()) continue;
        rb.table_rows = (int32_t)rows.size();
        rb.M = items;
        rb.n = sc->sc.n;
        rb.per_row = 1;
        launch_render_loss(sc->sc, rb, L.stream);
        for (SrvReq* r : closing) {
            FinalizeArgs fa{};
            fa.w = r->w;
            fa.loss = r->loss;
            fa.E = r->E;
            fa.n = r->n;
            fa.pairs2 = (int32_t)r->M;
            fa.elementwise = r->req.opts.strategy == HR_ELEMENTWISE;
            fa.hessian = r->req.quantity == HR_HESSIAN;
            fa.inv2P = 1.0 / (double)r->M;
            fa.out_flat = r->flat;
            fa.out_scale = nullptr;
            fa.out_full = r->req.quantity == HR_HESSIAN ? r->full : nullptr;
            launch_finalize(fa, L.stream);
            const size_t rb_bytes = sizeof(double) * (r->req.quantity == HR_HESSIAN ? r->n * r->n : r->n);
            cudaMemcpyAsync(pinned + (size_t)r->slot * kMaxResultBytes,
                            r->req.quantity == HR_HESSIAN ? (void*)r->full : (void*)r->flat, rb_bytes,
                            cudaMemcpyDeviceToHost, L.stream);
            r->done = get_event();
            cudaEventRecord(r->done, L.stream);
            r->finishing = true;
        }
        cudaEvent_t ev = get_event();
        cudaEventRecord(ev, L.stream);
        L.inflight.push_back(ev);
        if (cudaGetLastError() != cudaSuccess) {
            for (SrvReq* r : rows) r->status = HR_ERR_CUDA;
        }
        progress = true;
    }
    return progress;
}

bool hr_server_s::retire() {
    bool progress = false;
    std::vector<SrvReq*> still;
    std::vector<SrvReq*> done;
    for (SrvReq* r : active) {
        bool fin = false;
        if (r->status != HR_OK && !r->done) {
            fin = true;
        } else if (r->done) {
            const cudaError_t q = cudaEventQuery(r->done);
            if (q == cudaSuccess) fin = true;
            else if (q != cudaErrorNotReady) { r->status = HR_ERR_CUDA; fin = true; }
        }
        if (!fin) { still.push_back(r); continue; }
        if (r->status == HR_OK) {
            if (r->req.quantity == HR_NEWTON_STEP) {
                const int B = optstate_instances(r->req.optstate);
                r->result.resize(sizeof(hr_step_info) * B);
                optstate_copy_info(r->req.optstate, reinterpret_cast<hr_step_info*>(r->result.data()));
            } else {
                const size_t nb = sizeof(double) * (r->req.quantity == HR_HESSIAN ? r->n * r->n : r->n);
                r->result.assign(pinned + (size_t)r->slot * kMaxResultBytes, pinned + (size_t)r->slot * kMaxResultBytes + nb);
            }
        }
        if (r->done) { put_event(r->done); r->done = nullptr; }
        if (r->status != HR_OK && r->req.quantity != HR_NEWTON_STEP) {
            // a failed request may still have launches in flight on its lane:
            // drain them before its arena block can be handed out again
            cudaStreamSynchronize(lane(r->req.scene).stream);
        }
        if (r->req.quantity != HR_NEWTON_STEP) {
            arena.release(r->off, r->bytes);
        } else {
            busy_states.erase(std::find(busy_states.begin(), busy_states.end(), r->req.optstate));
        }
        free_slots.push_back(r->slot);
        r->slot = -1;
        r->t_done = now_ms();
        done.push_back(r);
        progress = true;
    }
    active.swap(still);
    if (!done.empty()) {
        std::lock_guard<std::mutex> lk(mu);
        for (SrvReq* r : done) r->state = 2;
        cv_done.notify_all();
    }
    return progress;
}

void hr_server_s::run() {
    cudaSetDevice(device);
    for (;;) {
        std::vector<SrvReq*> admitted;
        {
            std::unique_lock<std::mutex> lk(mu);
            if (stop) {
                for (SrvReq* r : pending) { r->status = HR_ERR_BUSY; r->state = 2; r->t_done = now_ms(); }
                pending.clear();
                cv_done.notify_all();
                if (active.empty()) break;
            }
            while (!pending.empty()) {
                SrvReq* r = pending.front();
                if (!admit(r)) break;
                pending.pop_front();
                r->state = 1;
                admitted.push_back(r);
            }
            if (admitted.empty() && active.empty() && pending.empty() && !stop) {
                cv_work.wait(lk);
                continue;
            }
        }
        bool progress = !admitted.empty();
        for (SrvReq* r : admitted) {
            setup(r);
            active.push_back(r);
        }
        progress |= launch_batches();
        progress |= retire();
        if (!progress) std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
}

extern "C" {

hr_status hr_server_create(const hr_server_opts* o, hr_server* out) {
    clear_error();
    if (!o || !out) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (o->max_active < 1 || o->max_active > kMaxBatchRows) return fail(HR_ERR_INVALID_ARG, "max_active must be 1..48");
    if (o->hbm_budget < (int64_t)(1 << 20)) return fail(HR_ERR_INVALID_ARG, "hbm_budget below 1 MiB");
    if (o->chunk < 0) return fail(HR_ERR_INVALID_ARG, "chunk must be >= 0");
    hr_server_s* S = new hr_server_s();
    S->opts = *o;
    if (S->opts.chunk == 0) S->opts.chunk = 2048;
    S->opts.chunk += S->opts.chunk & 1;
    cudaGetDevice(&S->device);
    cudaError_t e = cudaMalloc((void**)&S->arena.base, (size_t)o->hbm_budget);
    if (e != cudaSuccess) { delete S; return fail(HR_ERR_OOM, "arena: %s", cudaGetErrorString(e)); }
    S->arena.size = (size_t)o->hbm_budget;
    S->arena.free_blocks[0] = S->arena.size;
    e = cudaMallocHost((void**)&S->pinned, (size_t)kMaxResultBytes * o->max_active);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->upload, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        cudaFree(S->arena.base);
        if (S->pinned) cudaFreeHost(S->pinned);
        delete S;
        return fail(HR_ERR_CUDA, "server setup: %s", cudaGetErrorString(e));
    }
    for (int i = o->max_active - 1; i >= 0; --i) S->free_slots.push_back(i);
    S->t0 = std::chrono::steady_clock::now();
    S->worker = std::thread([S] { S->run(); });
    *out = S;
    return HR_OK;
}

hr_status hr_server_destroy(hr_server S) {
    if (!S) return HR_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->lanes) {
        cudaStreamSynchronize(kv.second.stream);
        for (cudaEvent_t e : kv.second.inflight) cudaEventDestroy(e);
        cudaStreamDestroy(kv.second.stream);
    }
    for (cudaEvent_t e : S->event_pool) cudaEventDestroy(e);
    for (auto& kv : S->tickets) delete kv.second;
    if (S->upload) cudaStreamDestroy(S->upload);
    cudaFree(S->arena.base);
    cudaFreeHost(S->pinned);
    delete S;
    return HR_OK;
}

hr_status hr_server_submit(hr_server S, const hr_request* q, uint64_t* ticket) {
    clear_error();
    if (!S || !q || !ticket) return fail(HR_ERR_INVALID_ARG, "NULL argument");
    if (!q->scene) return fail(HR_ERR_INVALID_ARG, "request has no scene");
    SrvReq* r = new SrvReq();
    r->req = *q;
    if (q->quantity == HR_NEWTON_STEP) {
        if (!q->optstate || optstate_scene(q->optstate) != q->scene) {
            delete r;
            return fail(HR_ERR_INVALID_ARG, "Newton-CG step request needs its scene's optimizer state");
        }
    } else {
        const hr_opts* o = &q->opts;
        if (q->quantity < HR_GRAD || q->quantity > HR_HVP) { delete r; return fail(HR_ERR_INVALID_ARG, "unknown quantity"); }
        if (!q->h_theta || (q->quantity == HR_HVP && !q->h_v)) { delete r; return fail(HR_ERR_INVALID_ARG, "theta/v missing"); }
        if (!(o->sigma > 0.0) || o->n_perturb < 2 || (o->n_perturb & 1) ||
            (o->strategy != HR_ELEMENTWISE && o->strategy != HR_AGGREGATE && o->strategy != HR_PLAIN) ||
            o->n_perturb / 2 >= (1 << 24)) {
            delete r;
            return fail(HR_ERR_INVALID_ARG, "invalid estimate options");
        }
        r->n = q->scene->sc.n;
        r->E = n_elem(q->quantity, r->n);
        r->G = o->strategy == HR_ELEMENTWISE ? r->E : 1;
        r->M = o->n_perturb;
        r->P = (int)(r->M / 2);
        r->Mt = (int64_t)r->G * r->M;
        if ((uint64_t)o->sub + (uint64_t)r->G > (1u << 24) || r->Mt > ((int64_t)1 << 28)) {
            delete r;
            return fail(HR_ERR_INVALID_ARG, "request too large");
        }
        r->bytes = request_bytes(r->n, r->E, r->G, r->Mt);
        if (r->bytes > S->arena.size) {
            const size_t b = r->bytes;
            delete r;
            return fail(HR_ERR_OOM, "request needs %zu bytes, more than the server's budget", b);
        }
        r->theta.assign(q->h_theta, q->h_theta + r->n);
        if (q->quantity == HR_HVP) r->v.assign(q->h_v, q->h_v + r->n);
    }
    r->req.h_theta = nullptr;
    r->req.h_v = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) { delete r; return fail(HR_ERR_BUSY, "server is shutting down"); }
        r->ticket = S->next_ticket++;
        r->t_submit = S->now_ms();
        S->tickets[r->ticket] = r;
        S->pending.push_back(r);
        *ticket = r->ticket;
    }
    S->cv_work.notify_all();
    return HR_OK;
}

hr_status hr_server_wait(hr_server S, uint64_t ticket, void* h_out, hr_request_info* info, int32_t timeout_ms) {
    clear_error();
    if (!S) return fail(HR_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return fail(HR_ERR_INVALID_ARG, "unknown ticket %llu", (unsigned long long)ticket);
    SrvReq* r = it->second;
    auto ready = [r] { return r->state == 2; };
    if (timeout_ms < 0) S->cv_done.wait(lk, ready);
    else if (!S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
        return fail(HR_ERR_TIMEOUT, "request %llu not finished", (unsigned long long)ticket);
    S->tickets.erase(it);
    lk.unlock();
    if (info) {
        info->submit_ms = r->t_submit;
        info->admit_ms = r->t_admit;
        info->done_ms = r->t_done;
        info->status = r->status;
        info->batches = r->batches;
    }
    const hr_status st = r->status;
    if (st == HR_OK && h_out && !r->result.empty()) memcpy(h_out, r->result.data(), r->result.size());
    delete r;
    if (st != HR_OK) return fail(st, "request failed");
    return HR_OK;
}

}  // extern "C"
