// Serving: a request loop over frame-denoise requests of mixed sizes.
//
// Clients submit frames (device buffers) tagged with a stream id.  A
// scheduler thread admits queued requests while the admitted footprint
// (bytes of device memory their batch touches) fits the budget, groups
// requests of equal size into batches, and runs each batch on a free
// worker: one CUDA stream and one context (weights and workspaces
// resident) per worker, inputs copied into the worker's fixed staging
// slots and the denoise replayed from a CUDA graph captured once per
// (worker, h, w, batch).  Batches on different workers overlap on the
// device; requests arriving meanwhile are admitted as workers and budget
// free up (continuous batching).  Completions are polled with events and
// delivered in submission order per stream; latency is submit -> delivery.
// Temporal requests (Sec. 4.3) carry world position and motion; the server
// keeps each stream's accumulation history on the device, runs one frame of
// a temporal stream at a time in submission order, and writes the
// accumulated radiance straight into the batch's radiance slot before the
// denoise.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "ctx.h"

namespace wskpn {

using Clock = std::chrono::steady_clock;

struct Request {
    uint64_t ticket = 0;
    int stream_id = 0;
    wskpn_frame frame{};
    int h = 0, w = 0;
    float* out = nullptr;
    const float* position = nullptr;  // temporal requests: world position [3][h][w]
    const float* motion = nullptr;    // and motion [2][h][w]
    int temporal = 0, reset = 0;
    size_t footprint = 0;
    Clock::time_point t_submit, t_dispatch, t_done;
    int worker = -1, batch = 0;  // worker that ran it and frames in its batch
    int state = 0;  // 0 queued, 1 running, 2 complete, 3 delivered
    wskpn_status status = WSKPN_OK;
};

struct Worker {
    wskpn_ctx* ctx = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    float* slot_in = nullptr;   // [max_batch][10][max_px]
    float* slot_out = nullptr;  // [max_batch][3][max_px]
    std::map<std::tuple<int, int, int>, cudaGraphExec_t> graphs;
    std::vector<Request*> batch;
    bool busy = false;
};

// Temporal history of one client stream; `running` while one of its frames
// is on the GPU (the next frame reads the state that frame writes).
struct TStream {
    wskpn_temporal* t = nullptr;
    bool running = false;
};

}  // namespace wskpn

struct wskpn_server {
    wskpn_config cfg{};
    wskpn_serve_config scfg{};
    int device = 0;
    size_t max_px = 0;
    size_t bytes_per_px = 0;
    std::vector<wskpn::Worker> workers;
    std::mutex mu;
    std::condition_variable cv_sched, cv_done;
    std::deque<wskpn::Request*> queue;
    std::unordered_map<uint64_t, wskpn::Request*> reqs;
    std::unordered_map<int, std::deque<wskpn::Request*>> pending;  // per stream, submission order
    std::unordered_map<int, wskpn::TStream> tstreams;              // temporal histories per stream
    uint64_t next_ticket = 1;
    size_t mem_in_use = 0, mem_peak = 0;
    bool paused = false, stopping = false;
    std::thread sched;
    // statistics
    uint64_t submitted = 0, completed = 0, rejected = 0, failed = 0, batches = 0, graph_launches = 0,
             graph_captures = 0, batched_frames = 0, temporal_frames = 0;
    std::vector<double> lat_ms;
    bool any_submit = false;
    wskpn::Clock::time_point t_start, t_first, t_last;
    std::string err;
};

namespace wskpn {

size_t tc_act_bytes_per_pixel(const wskpn_config& c, int which);

static size_t footprint_per_px(const wskpn_config& c) {
    size_t ws;
    if (c.prec == WSKPN_FP32) {
        int wa = 0, wb = 0;
        for (int l = 0; l < c.n_layers; ++l) (l % 2 == 0 ? wa : wb) = std::max(l % 2 == 0 ? wa : wb, c.widths[l]);
        ws = (size_t)(wa + wb) * 4;
    } else {
        ws = tc_act_bytes_per_pixel(c, 0) + tc_act_bytes_per_pixel(c, 1);
    }
    return ws + (size_t)c.widths[c.n_layers] * 4 + 13 * 4;  // + network output + staging in/out
}

// Copies the batch in, runs the denoise (graph or direct), copies results out.
static wskpn_status dispatch(wskpn_server* s, Worker& wk) {
    const int B = (int)wk.batch.size();
    const int h = wk.batch[0]->h, w = wk.batch[0]->w;
    const size_t px = (size_t)h * w;
    std::vector<wskpn_frame> slots(B);
    for (int j = 0; j < B; ++j) {
        const Request* r = wk.batch[j];
        float* base = wk.slot_in + (size_t)j * 10 * px;
        const float* src[4] = {r->frame.radiance, r->frame.albedo, r->frame.normal, r->frame.depth};
        const int ch[4] = {3, 3, 3, 1};
        size_t off = 0;
        for (int k = 0; k < 4; ++k) {
            if (k > 0 || !r->temporal)  // a temporal frame's radiance slot is written by the accumulation
                WSKPN_CUDA_TRY(cudaMemcpyAsync(base + off, src[k], ch[k] * px * sizeof(float),
                                               cudaMemcpyDeviceToDevice, wk.stream),
                               s->err);
            off += ch[k] * px;
        }
        slots[j] = {base, base + 3 * px, base + 6 * px, base + 9 * px};
    }
    // temporal accumulation of the batch's temporal frames, written straight
    // into their radiance slots (the stream's previous frame has completed)
    {
        std::vector<const float*> tc, tP, tn, tm, tprev;
        std::vector<float*> tnext, tout;
        for (int j = 0; j < B; ++j) {
            Request* r = wk.batch[j];
            if (!r->temporal) continue;
            TStream& ts = s->tstreams[r->stream_id];
            if (ts.t && (ts.t->h != h || ts.t->w != w)) {
                wskpn_temporal_destroy(ts.t);
                ts.t = nullptr;
            }
            if (!ts.t) {
                if (wskpn_temporal_create(&s->scfg.temporal, h, w, &ts.t) != WSKPN_OK) {
                    s->err = "temporal history allocation failed";
                    return WSKPN_ENOMEM;
                }
            } else if (r->reset) {
                WSKPN_CUDA_TRY(cudaMemsetAsync(ts.t->state[ts.t->cur], 0, TEMPORAL_PLANES * px * sizeof(float),
                                               wk.stream),
                               s->err);
            }
            tc.push_back(r->frame.radiance);
            tP.push_back(r->position);
            tn.push_back(r->frame.normal);
            tm.push_back(r->motion);
            tprev.push_back(ts.t->state[ts.t->cur]);
            tnext.push_back(ts.t->state[ts.t->cur ^ 1]);
            tout.push_back(const_cast<float*>(slots[j].radiance));
            ts.t->cur ^= 1;
        }
        if (!tc.empty()) {
            const wskpn_status ts = launch_temporal(s->scfg.temporal, tc.data(), tP.data(), tn.data(), tm.data(),
                                                    tprev.data(), tnext.data(), tout.data(), (int)tc.size(), h, w,
                                                    wk.stream, s->err);
            if (ts) return ts;
            s->temporal_frames += tc.size();
        }
    }
    wskpn_status st = WSKPN_OK;
    if (s->scfg.use_graphs) {
        const auto key = std::make_tuple(h, w, B);
        auto it = wk.graphs.find(key);
        if (it == wk.graphs.end()) {
            // one direct call first (sets kernel attributes outside capture)
            st = wskpn_denoise(wk.ctx, slots.data(), B, h, w, wk.slot_out, wk.stream);
            if (st) return st;
            cudaGraph_t g = nullptr;
            cudaGraphExec_t ge = nullptr;
            WSKPN_CUDA_TRY(cudaStreamBeginCapture(wk.stream, cudaStreamCaptureModeThreadLocal), s->err);
            st = wskpn_denoise(wk.ctx, slots.data(), B, h, w, wk.slot_out, wk.stream);
            cudaError_t ce = cudaStreamEndCapture(wk.stream, &g);
            if (st || ce != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                s->err = "graph capture failed";
                return st ? st : WSKPN_ECUDA;
            }
            ce = cudaGraphInstantiate(&ge, g, 0);
            cudaGraphDestroy(g);
            if (ce != cudaSuccess) {
                s->err = std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ce);
                return WSKPN_ECUDA;
            }
            it = wk.graphs.emplace(key, ge).first;
            ++s->graph_captures;
        }
        WSKPN_CUDA_TRY(cudaGraphLaunch(it->second, wk.stream), s->err);
        ++s->graph_launches;
    } else {
        st = wskpn_denoise(wk.ctx, slots.data(), B, h, w, wk.slot_out, wk.stream);
        if (st) return st;
    }
    for (int j = 0; j < B; ++j)
        WSKPN_CUDA_TRY(cudaMemcpyAsync(wk.batch[j]->out, wk.slot_out + (size_t)j * 3 * px, 3 * px * sizeof(float),
                                       cudaMemcpyDeviceToDevice, wk.stream),
                       s->err);
    WSKPN_CUDA_TRY(cudaEventRecord(wk.done, wk.stream), s->err);
    return WSKPN_OK;
}

// Delivers completed requests at the head of each stream's order.
static void deliver(wskpn_server* s) {
    bool any = false;
    for (auto& kv : s->pending) {
        auto& dq = kv.second;
        while (!dq.empty() && dq.front()->state == 2) {
            Request* r = dq.front();
            dq.pop_front();
            r->state = 3;
            const double ms = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
            if (r->status == WSKPN_OK) {
                s->lat_ms.push_back(ms);
                ++s->completed;
            } else {
                ++s->failed;
            }
            s->t_last = std::max(s->t_last, r->t_done);
            any = true;
        }
    }
    if (any) s->cv_done.notify_all();
}

static void scheduler(wskpn_server* s) {
    cudaSetDevice(s->device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (true) {
        // 1. completions
        for (auto& wk : s->workers) {
            if (!wk.busy) continue;
            const cudaError_t q = cudaEventQuery(wk.done);
            if (q == cudaErrorNotReady) continue;
            const auto now = Clock::now();
            for (Request* r : wk.batch) {
                r->state = 2;
                r->t_done = now;
                if (q != cudaSuccess) r->status = WSKPN_ECUDA;
                s->mem_in_use -= r->footprint;
                if (r->temporal) s->tstreams[r->stream_id].running = false;
            }
            wk.batch.clear();
            wk.busy = false;
        }
        deliver(s);
        // 2. admission and dispatch
        bool dispatched = false;
        if (!s->paused) {
            for (size_t wi = 0; wi < s->workers.size(); ++wi) {
                Worker& wk = s->workers[wi];
                if (wk.busy || s->queue.empty()) continue;
                // the oldest request that may run now: a temporal stream runs one
                // frame at a time, in submission order
                Request* head = nullptr;
                {
                    std::unordered_set<int> blocked;
                    for (Request* r : s->queue) {
                        if (r->temporal && (blocked.count(r->stream_id) || s->tstreams[r->stream_id].running)) {
                            blocked.insert(r->stream_id);
                            continue;
                        }
                        head = r;
                        break;
                    }
                }
                if (!head) break;
                if (s->mem_in_use + head->footprint > s->scfg.mem_budget) break;  // wait for memory
                const double age_us =
                    std::chrono::duration<double, std::micro>(Clock::now() - head->t_submit).count();
                int same = 0;
                for (Request* r : s->queue)
                    if (r->h == head->h && r->w == head->w) ++same;
                if (same < s->scfg.max_batch && age_us < s->scfg.batch_window_us && !s->stopping) break;
                size_t mem = s->mem_in_use;
                std::unordered_set<int> tblocked;  // temporal streams that may not join this batch
                for (auto it = s->queue.begin(); it != s->queue.end() && (int)wk.batch.size() < s->scfg.max_batch;) {
                    Request* r = *it;
                    bool ok = r->h == head->h && r->w == head->w && mem + r->footprint <= s->scfg.mem_budget;
                    if (r->temporal) {
                        if (tblocked.count(r->stream_id) || s->tstreams[r->stream_id].running) ok = false;
                        tblocked.insert(r->stream_id);  // one frame per stream per batch, and none after a skip
                    }
                    if (ok) {
                        mem += r->footprint;
                        r->state = 1;
                        wk.batch.push_back(r);
                        it = s->queue.erase(it);
                    } else {
                        ++it;
                    }
                }
                s->mem_in_use = mem;
                s->mem_peak = std::max(s->mem_peak, mem);
                const auto t_disp = Clock::now();
                for (Request* r : wk.batch) {
                    if (r->temporal) s->tstreams[r->stream_id].running = true;
                    r->worker = (int)wi;
                    r->batch = (int)wk.batch.size();
                    r->t_dispatch = t_disp;
                }
                const wskpn_status st = dispatch(s, wk);
                ++s->batches;
                s->batched_frames += wk.batch.size();
                if (st) {
                    const auto now = Clock::now();
                    for (Request* r : wk.batch) {
                        r->state = 2;
                        r->status = st;
                        r->t_done = now;
                        s->mem_in_use -= r->footprint;
                        if (r->temporal) s->tstreams[r->stream_id].running = false;
                    }
                    wk.batch.clear();
                } else {
                    wk.busy = true;
                }
                dispatched = true;
            }
        }
        bool busy = false;
        for (auto& wk : s->workers) busy |= wk.busy;
        if (s->stopping && s->queue.empty() && !busy) break;
        if (dispatched) continue;
        if (busy || !s->queue.empty())
            s->cv_sched.wait_for(lk, std::chrono::microseconds(20));
        else
            s->cv_sched.wait(lk);
    }
    deliver(s);
}

}  // namespace wskpn

using namespace wskpn;

extern "C" {

wskpn_status wskpn_serve_config_default(wskpn_serve_config* c) {
    if (!c) return WSKPN_EINVAL;
    c->n_workers = 4;
    c->max_batch = 4;
    c->max_queue = 8192;
    c->mem_budget = (size_t)8 << 30;
    c->use_graphs = 1;
    c->batch_window_us = 200;
    wskpn_temporal_config_default(&c->temporal);
    return WSKPN_OK;
}

wskpn_status wskpn_serve_start(const wskpn_config* cfg, const float* host_weights, size_t n,
                               const wskpn_serve_config* scfg_in, wskpn_server** out) {
    if (!out || !cfg || !host_weights) {
        set_thread_error("wskpn_serve_start: NULL argument");
        return WSKPN_EINVAL;
    }
    *out = nullptr;
    wskpn_serve_config scfg;
    wskpn_serve_config_default(&scfg);
    if (scfg_in) scfg = *scfg_in;
    if (scfg.mem_budget == 0) scfg.mem_budget = (size_t)8 << 30;
    if (scfg.n_workers < 1 || scfg.n_workers > 32 || scfg.max_batch < 1 || scfg.max_batch > WSKPN_MAX_BATCH ||
        scfg.max_queue < 1 || scfg.batch_window_us < 0 || !temporal_config_valid(scfg.temporal)) {
        set_thread_error("wskpn_serve_start: serve config out of range");
        return WSKPN_EINVAL;
    }
    wskpn_server* s = new wskpn_server();
    s->cfg = *cfg;
    s->cfg.max_batch = scfg.max_batch;
    s->scfg = scfg;
    cudaGetDevice(&s->device);
    s->max_px = (size_t)s->cfg.max_h * s->cfg.max_w;
    s->bytes_per_px = footprint_per_px(s->cfg);
    s->workers.resize(scfg.n_workers);
    for (auto& wk : s->workers) {
        wskpn_status st = wskpn_create(&s->cfg, host_weights, n, &wk.ctx);
        if (st == WSKPN_OK) {
            const size_t n_in = (size_t)scfg.max_batch * 10 * s->max_px, n_out = (size_t)scfg.max_batch * 3 * s->max_px;
            if (cudaStreamCreateWithFlags(&wk.stream, cudaStreamNonBlocking) != cudaSuccess ||
                cudaEventCreateWithFlags(&wk.done, cudaEventDisableTiming) != cudaSuccess ||
                cudaMalloc(&wk.slot_in, n_in * sizeof(float)) != cudaSuccess ||
                cudaMalloc(&wk.slot_out, n_out * sizeof(float)) != cudaSuccess) {
                set_thread_error("wskpn_serve_start: worker allocation failed");
                st = WSKPN_ENOMEM;
            }
        }
        if (st) {
            wskpn_serve_stop(s);
            return st;
        }
    }
    s->t_start = Clock::now();
    s->sched = std::thread(scheduler, s);
    *out = s;
    return WSKPN_OK;
}

static wskpn_status submit(wskpn_server* s, int stream_id, const wskpn_frame* frame, const float* position,
                           const float* motion, int temporal, int reset, int h, int w, float* out,
                           uint64_t* ticket) {
    if (!s) return WSKPN_EINVAL;
    if (!frame || !out || !frame->radiance || !frame->albedo || !frame->normal || !frame->depth || h < 1 || w < 1 ||
        h > s->cfg.max_h || w > s->cfg.max_w || (temporal && (!position || !motion))) {
        std::lock_guard<std::mutex> lk(s->mu);
        s->err = "wskpn_serve_submit: invalid frame, output or size";
        return WSKPN_EINVAL;
    }
    Request* r = new Request();
    r->position = position;
    r->motion = motion;
    r->temporal = temporal;
    r->reset = reset;
    r->stream_id = stream_id;
    r->frame = *frame;
    r->h = h;
    r->w = w;
    r->out = out;
    r->footprint = (size_t)h * w * s->bytes_per_px;
    r->t_submit = Clock::now();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if ((int)s->queue.size() >= s->scfg.max_queue || r->footprint > s->scfg.mem_budget || s->stopping) {
            ++s->rejected;
            s->err = s->stopping ? "server stopping"
                                 : (r->footprint > s->scfg.mem_budget ? "request footprint exceeds the memory budget"
                                                                      : "queue full");
            delete r;
            return WSKPN_EBUSY;
        }
        r->ticket = s->next_ticket++;
        s->reqs[r->ticket] = r;
        s->pending[stream_id].push_back(r);
        s->queue.push_back(r);
        ++s->submitted;
        if (!s->any_submit) {
            s->any_submit = true;
            s->t_first = r->t_submit;
            s->t_last = r->t_submit;
        }
        if (ticket) *ticket = r->ticket;
    }
    s->cv_sched.notify_one();
    return WSKPN_OK;
}

wskpn_status wskpn_serve_submit(wskpn_server* s, int stream_id, const wskpn_frame* frame, int h, int w, float* out,
                                uint64_t* ticket) {
    return submit(s, stream_id, frame, nullptr, nullptr, 0, 0, h, w, out, ticket);
}

wskpn_status wskpn_serve_submit_temporal(wskpn_server* s, int stream_id, const wskpn_frame* frame,
                                         const float* position, const float* motion, int reset_history, int h,
                                         int w, float* out, uint64_t* ticket) {
    return submit(s, stream_id, frame, position, motion, 1, reset_history != 0, h, w, out, ticket);
}

wskpn_status wskpn_serve_wait(wskpn_server* s, uint64_t ticket, int timeout_ms) {
    return wskpn_serve_wait_info(s, ticket, timeout_ms, nullptr);
}

wskpn_status wskpn_serve_wait_info(wskpn_server* s, uint64_t ticket, int timeout_ms, wskpn_serve_ticket_info* info) {
    if (!s) return WSKPN_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) {
        s->err = "unknown ticket";
        return WSKPN_EINVAL;
    }
    Request* r = it->second;
    auto done = [&] { return r->state == 3; };
    if (timeout_ms < 0)
        s->cv_done.wait(lk, done);
    else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), done))
        return WSKPN_ETIMEOUT;
    const wskpn_status st = r->status;
    if (info) {
        auto ms = [&](Clock::time_point t) { return std::chrono::duration<double, std::milli>(t - s->t_start).count(); };
        info->h = r->h;
        info->w = r->w;
        info->worker = r->worker;
        info->batch = r->batch;
        info->submit_ms = ms(r->t_submit);
        info->dispatch_ms = r->worker >= 0 ? ms(r->t_dispatch) : -1.0;
        info->done_ms = ms(r->t_done);
    }
    s->reqs.erase(it);
    delete r;
    return st;
}

wskpn_status wskpn_serve_pause(wskpn_server* s, int paused) {
    if (!s) return WSKPN_EINVAL;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->paused = paused != 0;
    }
    s->cv_sched.notify_one();
    return WSKPN_OK;
}

wskpn_status wskpn_serve_stats_get(wskpn_server* s, wskpn_serve_stats* st) {
    if (!s || !st) return WSKPN_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    *st = wskpn_serve_stats{};
    st->submitted = s->submitted;
    st->completed = s->completed;
    st->rejected = s->rejected;
    st->failed = s->failed;
    st->batches = s->batches;
    st->graph_launches = s->graph_launches;
    st->graph_captures = s->graph_captures;
    st->mem_in_use = s->mem_in_use;
    st->mem_peak = s->mem_peak;
    st->mean_batch = s->batches ? (double)s->batched_frames / s->batches : 0.0;
    st->temporal_frames = s->temporal_frames;
    for (const auto& kv : s->tstreams)
        if (kv.second.t) {
            ++st->temporal_streams;
            st->temporal_bytes += 2 * TEMPORAL_PLANES * sizeof(float) * (size_t)kv.second.t->h * kv.second.t->w;
        }
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) { return v[std::min(v.size() - 1, (size_t)(p * (v.size() - 1) + 0.5))]; };
        st->p50_ms = pct(0.50);
        st->p99_ms = pct(0.99);
        st->max_ms = v.back();
        double sum = 0;
        for (double x : v) sum += x;
        st->mean_ms = sum / v.size();
        const double span = std::chrono::duration<double>(s->t_last - s->t_first).count();
        st->fps = span > 0 ? s->completed / span : 0.0;
    }
    return WSKPN_OK;
}

void wskpn_serve_stop(wskpn_server* s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stopping = true;
        s->paused = false;
    }
    s->cv_sched.notify_one();
    if (s->sched.joinable()) s->sched.join();
    for (auto& wk : s->workers) {
        if (wk.stream) cudaStreamSynchronize(wk.stream);
        for (auto& kv : wk.graphs) cudaGraphExecDestroy(kv.second);
        if (wk.done) cudaEventDestroy(wk.done);
        if (wk.stream) cudaStreamDestroy(wk.stream);
        cudaFree(wk.slot_in);
        cudaFree(wk.slot_out);
        wskpn_destroy(wk.ctx);
    }
    for (auto& kv : s->tstreams) wskpn_temporal_destroy(kv.second.t);
    for (auto& kv : s->reqs) delete kv.second;
    delete s;
}

}  // extern "C"
