// mg_server.cu -- request loop with continuous batching, the host runtime
// around the query (Sec. 3.6), propagation (Sec. 3.4) and lookup (Sec. 4)
// kernels.
//
// Resident volumes are admitted against a memory budget; each gets, per slot
// (one CUDA stream), a captured query plan and staging buffers, so nothing is
// allocated while serving.  Requests enter per-volume FIFOs (boxes and TF
// frames apart).  A worker thread polls the slots' completion events and,
// whenever a slot is free, takes the oldest request: a TF frame together with
// the next queued frames of the same volume (up to `frames` of them: one
// multi-TF propagation and one lookup launch for all), or a box together with
// the next queued boxes of the same volume while they fit the slot's batch --
// max_batch boxes whose footprint blocks and work chunks (counted on the host
// at submission, in closed form as the plan kernel does) fit the plan's
// capacities.  The batch
// is staged straight into the plan's input buffers and run as one graph
// launch; results come back through pinned memory and are copied into the
// callers' buffers when the slot's event fires, which also ends each
// request's latency.
#include "mg_internal.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <thread>
#include <unordered_map>
#include <vector>

namespace mg {
namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxRunsHost = 40;   // runs per axis, as in the plan kernels

// Footprint size of one box (Algorithm 1): per axis the aligned power-of-two
// runs of the clipped range; the blocks are their tensor product.  The cubes
// follow in closed form, as in the plan kernel: with F(m) the sum over an
// axis's runs of level >= m of 2^(level - m) and P(m) = Fx Fy Fz, the blocks
// hold P(0) - 7 * sum over m >= 1 of P(m) cubes; an axis's steps rise and then
// fall, so a level occurs at most twice and two bit masks give F(m).
void box_work(const int32_t* b, const int32_t* dims, uint32_t chunk, uint64_t* blocks, uint64_t* chunks) {
    uint64_t once[3], twice[3];
    uint64_t n[3];
    for (int a = 0; a < 3; a++) {
        int64_t i = b[a], di = std::min<int64_t>((int64_t)b[a] + b[3 + a], dims[a]) - b[a];
        once[a] = twice[a] = 0;
        n[a] = 0;
        while (di > 0 && n[a] < (uint64_t)kMaxRunsHost) {
            int hi = 63;
            while (!((di >> hi) & 1)) hi--;
            int lo = 63;
            if (i != 0) {
                lo = 0;
                while (!((i >> lo) & 1)) lo++;
            }
            const int l = std::min(hi, lo);
            const uint64_t bit = 1ull << l;
            if (once[a] & bit) twice[a] |= bit;
            else once[a] |= bit;
            n[a]++;
            di -= (int64_t)1 << l;
            i += (int64_t)1 << l;
        }
    }
    auto P = [&](int m) {
        uint64_t v = 1;
        for (int a = 0; a < 3; a++) v *= (once[a] >> m) + (twice[a] >> m);
        return v;
    };
    uint64_t rest = 0;
    for (int m = 1; m < 64 && (once[0] >> m) && (once[1] >> m) && (once[2] >> m); m++) rest += P(m);
    const uint64_t cubes = P(0) - 7 * rest;
    *blocks = n[0] * n[1] * n[2];
    *chunks = (cubes + chunk - 1) / chunk;
}

enum : int { kQueued = 0, kRunning = 1, kDone = 2 };

struct Req {
    mg_request r{};
    uint64_t ticket = 0;
    Clock::time_point arrival;
    uint64_t blocks = 0, chunks = 0;   // footprint of a box request
    int64_t frame_off = 0;             // TF frame: first sample in its work item's lookup
};

struct Rec {
    int state = kQueued;
    mg_status status = MG_OK;
    double latency = 0.0;
    std::string error;
};

struct VolSlot {              // one slot's resources for one volume
    mg_query_plan* plan = nullptr;   // batched mode
    PlanParts pp{};
    Buf boxes_dev, out_dev;          // plain mode
    Buf tf_dev, vals_dev, samples_dev, render_dev;
    unsigned char* pin = nullptr;    // pinned staging, carved below
    int64_t* pin_q = nullptr;
    unsigned* pin_status = nullptr;
    int32_t* pin_boxes = nullptr;
    void* pin_out = nullptr;
    float* pin_tf = nullptr;
    float* pin_samples = nullptr;
    void* pin_render = nullptr;
};

struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Req> work;
    std::vector<VolSlot> vols;
};

constexpr int kMaxVolumes = 1024;   // admitted over a server's life (slots reserved up front)

struct Volume {
    mg_graph* g = nullptr;
    int C = 0;
    bool removed = false;   // mg_server_remove_volume: no new requests, resources released
    int frames = 1;   // TF frames one work item propagates together (frames * C channels)
    int32_t dims[3] = {0, 0, 0};
    uint32_t chunk = 2048;
    uint64_t cap_blocks = 0, cap_chunks = 0;
    int64_t bytes = 0;   // admitted memory
};

// queued requests of one volume, boxes and TF frames apart, each in arrival
// (ticket) order: a work item takes from the front of one of them
struct VolQueue {
    std::deque<Req> box, tf;
};

size_t round_up(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace
}  // namespace mg

struct mg_server {
    mg_server_opts o{};
    int device = 0;
    size_t esize = 4;   // bytes of one stored TF value
    std::vector<mg::Volume> vols;
    std::vector<mg::Slot> slots;
    int64_t budget_used = 0;

    std::mutex mu;
    std::condition_variable work_cv;   // worker: new requests or stop
    std::condition_variable done_cv;   // waiters: completions
    std::vector<mg::VolQueue> vq;   // per volume (reserved like vols)
    int64_t queued = 0;             // requests in vq
    std::unordered_map<uint64_t, mg::Rec> recs;
    uint64_t next_ticket = 0;
    mg_server_stats stats{};
    std::thread worker;
    std::atomic<bool> stop{false};
    bool started = false;
};

namespace mg {
namespace {

size_t pinned_bytes(size_t Q, size_t S, int C, int F, size_t ms, size_t esize) {
    return round_up(8) + round_up(4) + round_up(Q * 24) + round_up(Q * S * 4) + round_up((size_t)F * S * C * 4) +
           round_up((size_t)F * ms * 16) + round_up((size_t)F * ms * C * esize);
}

// TF frames propagated together: the most, up to 8, whose k * C channels a
// multi-TF propagation supports
int frames_for(int C) {
    for (int k = 8; k > 1; k--) {
        const int t = k * C;
        if (t <= 8 || t == 12 || t == 16 || t == 20 || t == 24 || t == 28 || t == 32) return k;
    }
    return 1;
}

// copy a finished slot's results into the callers' buffers (worker thread,
// lock not held: the slot's work and the callers' buffers are the worker's
// until the requests are marked done, and a volume with work in flight is
// not removed)
void copy_results(const mg_server* sv, const Slot& sl) {
    for (size_t i = 0; i < sl.work.size(); i++) {
        const Req& q = sl.work[i];
        if (!q.r.result) continue;
        const Volume& v = sv->vols[q.r.volume];
        const VolSlot& vs = sl.vols[q.r.volume];
        if (q.r.kind == MG_REQ_BOX)
            std::memcpy(q.r.result, static_cast<const char*>(vs.pin_out) + i * (size_t)v.g->S * 4, (size_t)v.g->S * 4);
        else if (q.r.P > 0)
            std::memcpy(q.r.result, static_cast<const char*>(vs.pin_render) + q.frame_off * v.C * sv->esize,
                        (size_t)q.r.P * v.C * sv->esize);
    }
}

// complete the requests of a finished slot (lock held by the caller; results
// already copied when st is MG_OK)
void finish_locked(mg_server* sv, Slot& sl, Clock::time_point now, mg_status st, const std::string& err) {
    for (size_t i = 0; i < sl.work.size(); i++) {
        const Req& q = sl.work[i];
        Rec& rec = sv->recs[q.ticket];
        rec.state = kDone;
        rec.status = st;
        rec.error = err;
        rec.latency = std::chrono::duration<double>(now - q.arrival).count();
        if (st != MG_OK) sv->stats.failed++;
        else if (q.r.kind == MG_REQ_BOX) sv->stats.box_requests++;
        else sv->stats.tf_requests++;
    }
    sl.work.clear();
    sl.busy = false;
}

// the next work item, for the oldest queued request: a TF frame with the
// next queued frames of its volume (up to `frames`), or a box with the next
// queued boxes of its volume, in order, while they fit one batch (the plain
// mode takes one box).  Every take is from the front of a per-volume queue.
std::vector<Req> take_locked(mg_server* sv) {
    std::vector<Req> w;
    if (!sv->queued) return w;
    std::deque<Req>* best = nullptr;
    for (VolQueue& q : sv->vq) {
        if (!q.box.empty() && (!best || q.box.front().ticket < best->front().ticket)) best = &q.box;
        if (!q.tf.empty() && (!best || q.tf.front().ticket < best->front().ticket)) best = &q.tf;
    }
    std::deque<Req>& d = *best;
    const Volume& vol = sv->vols[d.front().r.volume];
    if (d.front().r.kind == MG_REQ_TF) {
        while (!d.empty() && (int)w.size() < vol.frames) {
            w.push_back(d.front());
            d.pop_front();
        }
    } else if (sv->o.plain) {
        w.push_back(d.front());
        d.pop_front();
    } else {
        uint64_t blocks = 0, chunks = 0;
        while (!d.empty() && (int64_t)w.size() < sv->o.max_batch && blocks + d.front().blocks <= vol.cap_blocks &&
               chunks + d.front().chunks <= vol.cap_chunks) {
            blocks += d.front().blocks;
            chunks += d.front().chunks;
            w.push_back(d.front());
            d.pop_front();
        }
    }
    sv->queued -= (int64_t)w.size();
    return w;
}

mg_status cuda_ok(cudaError_t e, const char* what) { return e == cudaSuccess ? MG_OK : cuda_fail(e, what); }

// stage and enqueue one work item on a free slot
mg_status launch(mg_server* sv, Slot& sl, std::vector<Req>& w) {
    const Req& head = w[0];
    MG_RANGE(head.r.kind == MG_REQ_TF ? "mg_server frame" : "mg_server box batch");
    const Volume& vol = sv->vols[head.r.volume];
    VolSlot& vs = sl.vols[head.r.volume];
    mg_graph* g = vol.g;
    const size_t S = g->S;
    cudaStream_t s = sl.s;
    if (head.r.kind == MG_REQ_TF) {
        // k frames: k TFs through one multi-TF propagation, every frame's
        // samples looked up against its slice in one launch
        const int k = (int)w.size();
        const size_t tf_bytes = S * vol.C * 4;
        int64_t off[33];
        off[0] = 0;
        for (int j = 0; j < k; j++) {
            std::memcpy(reinterpret_cast<char*>(vs.pin_tf) + j * tf_bytes, w[j].r.tf, tf_bytes);
            if (w[j].r.P > 0)
                std::memcpy(vs.pin_samples + 4 * off[j], w[j].r.samples, (size_t)w[j].r.P * 16);
            w[j].frame_off = off[j];
            off[j + 1] = off[j] + w[j].r.P;
        }
        MG_TRY(cuda_ok(cudaMemcpyAsync(vs.tf_dev.p, vs.pin_tf, k * tf_bytes, cudaMemcpyHostToDevice, s), "TF upload"));
        MG_TRY(propagate_multi(g, vs.tf_dev.as<float>(), k, vol.C, (mg_dtype)sv->o.storage, vs.vals_dev.p, s));
        const int64_t P = off[k];
        if (P > 0) {
            MG_TRY(cuda_ok(cudaMemcpyAsync(vs.samples_dev.p, vs.pin_samples, (size_t)P * 16, cudaMemcpyHostToDevice, s),
                           "sample upload"));
            MG_TRY(render_lookup_multi(g, vs.vals_dev.p, k, vol.C, (mg_dtype)sv->o.storage, vs.samples_dev.as<float>(),
                                       off, vs.render_dev.p, s));
            MG_TRY(cuda_ok(cudaMemcpyAsync(vs.pin_render, vs.render_dev.p, (size_t)P * vol.C * sv->esize,
                                           cudaMemcpyDeviceToHost, s),
                           "frame readback"));
        }
    } else {
        const int64_t Q = (int64_t)w.size();
        for (int64_t i = 0; i < Q; i++) std::memcpy(vs.pin_boxes + 6 * i, w[(size_t)i].r.box, 24);
        void* result = nullptr;
        if (sv->o.plain) {
            MG_TRY(cuda_ok(cudaMemcpyAsync(vs.boxes_dev.p, vs.pin_boxes, (size_t)Q * 24, cudaMemcpyHostToDevice, s),
                           "box upload"));
            mg_query_opts o{};
            o.hist_type = sv->o.hist_type;
            o.schedule = MG_SCHED_PLAIN;
            MG_TRY(query_boxes(g, vs.boxes_dev.as<int32_t>(), Q, o, vs.out_dev.p, (size_t)Q * S, nullptr, nullptr,
                               nullptr, s));
            result = vs.out_dev.p;
        } else {
            *vs.pin_q = Q;
            MG_TRY(cuda_ok(cudaMemcpyAsync(vs.pp.boxes, vs.pin_boxes, (size_t)Q * 24, cudaMemcpyHostToDevice, s),
                           "box upload"));
            MG_TRY(cuda_ok(cudaMemcpyAsync(vs.pp.Qd, vs.pin_q, 8, cudaMemcpyHostToDevice, s), "batch size upload"));
            MG_TRY(cuda_ok(cudaGraphLaunch(vs.pp.exec, s), "plan launch"));
            result = vs.pp.result;
        }
        MG_TRY(cuda_ok(cudaMemcpyAsync(vs.pin_out, result, (size_t)Q * S * 4, cudaMemcpyDeviceToHost, s),
                       "histogram readback"));
    }
    // a status bit raised by this work (or by anything else on the graph
    // meanwhile) fails the work item rather than passing a wrong result
    MG_TRY(cuda_ok(cudaMemcpyAsync(vs.pin_status, g->status.p, 4, cudaMemcpyDeviceToHost, s), "status readback"));
    MG_TRY(cuda_ok(cudaEventRecord(sl.done, s), "event record"));
    return MG_OK;
}

void worker_loop(mg_server* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    for (;;) {
        bool progressed = false;
        bool any_busy = false;
        for (Slot& sl : sv->slots) {
            if (!sl.busy) continue;
            const cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaErrorNotReady) {
                any_busy = true;
                continue;
            }
            mg_status st = MG_OK;
            std::string err;
            if (e != cudaSuccess) {
                st = cuda_fail(e, "request loop");
                err = mg_last_error();
            } else {
                const unsigned bits = *sl.vols[sl.work[0].r.volume].pin_status;
                if (bits) {
                    st = status_from_bits(bits);
                    err = mg_last_error();
                }
            }
            const Clock::time_point now = Clock::now();
            if (st == MG_OK) {
                lk.unlock();
                copy_results(sv, sl);
                lk.lock();
            }
            finish_locked(sv, sl, now, st, err);
            progressed = true;
        }
        if (progressed) sv->done_cv.notify_all();
        if (sv->stop.load() && !any_busy && !progressed) break;
        for (Slot& sl : sv->slots) {
            if (sl.busy || sv->stop.load()) continue;
            std::vector<Req> w = take_locked(sv);
            if (w.empty()) break;
            for (const Req& q : w) sv->recs[q.ticket].state = kRunning;
            if (w[0].r.kind == MG_REQ_BOX) {
                sv->stats.box_launches++;
                sv->stats.max_batch_seen = std::max<int64_t>(sv->stats.max_batch_seen, (int64_t)w.size());
            } else {
                sv->stats.tf_launches++;
            }
            sl.busy = true;
            // stage outside the lock: submissions continue meanwhile
            lk.unlock();
            const mg_status st = launch(sv, sl, w);
            const std::string err = st == MG_OK ? std::string() : std::string(mg_last_error());
            if (st != MG_OK) cudaStreamSynchronize(sl.s);
            lk.lock();
            sl.work = std::move(w);
            if (st != MG_OK) {
                finish_locked(sv, sl, Clock::now(), st, err);
                sv->done_cv.notify_all();
            } else {
                any_busy = true;
            }
            progressed = true;
        }
        if (progressed) continue;
        if (any_busy) {
            lk.unlock();
            std::this_thread::yield();   // poll the events again
            lk.lock();
        } else if (!sv->stop.load()) {
            sv->work_cv.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
    // stopping: what is still queued is cancelled
    for (VolQueue& vq : sv->vq)
        for (std::deque<Req>* d : {&vq.box, &vq.tf}) {
            for (const Req& q : *d) {
                Rec& rec = sv->recs[q.ticket];
                rec.state = kDone;
                rec.status = MG_ERR_CANCELLED;
                rec.error = "server stopped before the request was launched";
                sv->stats.cancelled++;
            }
            d->clear();
        }
    sv->queued = 0;
    sv->done_cv.notify_all();
}

mg_status check_request(const mg_server* sv, const mg_request& r, Req* q) {
    if (r.volume < 0 || r.volume >= (int)sv->vols.size()) return fail(MG_ERR_INVALID_ARG, "unknown volume");
    const Volume& v = sv->vols[r.volume];
    if (v.removed) return fail(MG_ERR_INVALID_ARG, "volume removed from the server");
    q->blocks = q->chunks = 0;
    if (r.kind == MG_REQ_BOX) {
        const int32_t* b = r.box;
        if (b[0] < 0 || b[0] >= v.dims[0] || b[1] < 0 || b[1] >= v.dims[1] || b[2] < 0 || b[2] >= v.dims[2] ||
            b[3] < 1 || b[4] < 1 || b[5] < 1)
            return fail(MG_ERR_INVALID_ARG, "box must start inside the volume and have sides >= 1");
        if (!sv->o.plain) {
            box_work(b, v.dims, v.chunk, &q->blocks, &q->chunks);
            if (q->blocks > v.cap_blocks || q->chunks > v.cap_chunks)
                return fail(MG_ERR_CAPACITY, "the box's footprint exceeds one batch's capacity");
        }
        return MG_OK;
    }
    if (r.kind == MG_REQ_TF) {
        if (!r.tf) return fail(MG_ERR_INVALID_ARG, "a TF frame needs its S x C transfer function");
        if (r.P < 0 || r.P > sv->o.max_samples) return fail(MG_ERR_INVALID_ARG, "P must be in 0..max_samples");
        if (r.P > 0 && !r.samples) return fail(MG_ERR_INVALID_ARG, "samples is NULL");
        return MG_OK;
    }
    return fail(MG_ERR_INVALID_ARG, "request kind must be MG_REQ_BOX or MG_REQ_TF");
}

mg_status submit(mg_server* sv, const mg_request& r, Clock::time_point arrival, uint64_t* ticket) {
    Req q;
    q.r = r;
    q.arrival = arrival;
    {
        // checked under the lock: volumes may be admitted or removed meanwhile
        std::lock_guard<std::mutex> lk(sv->mu);
        MG_TRY(check_request(sv, r, &q));
        if (sv->stop.load()) return fail(MG_ERR_INVALID_ARG, "server is stopping");
        q.ticket = sv->next_ticket++;
        sv->recs.emplace(q.ticket, Rec{});
        VolQueue& vq = sv->vq[r.volume];
        (r.kind == MG_REQ_BOX ? vq.box : vq.tf).push_back(q);
        sv->queued++;
    }
    sv->work_cv.notify_one();
    if (ticket) *ticket = q.ticket;
    return MG_OK;
}

void release_slot_volume(VolSlot& vs) {
    if (vs.plan) mg_query_plan_free(vs.plan);
    vs.plan = nullptr;
    if (vs.pin) cudaFreeHost(vs.pin);
    vs.pin = nullptr;
}

}  // namespace
}  // namespace mg

using namespace mg;

extern "C" {

MG_API mg_status mg_server_create(const mg_server_opts* opts, mg_server** out) {
    if (!out) return fail(MG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    mg_server_opts o{};
    if (opts) o = *opts;
    if (o.slots == 0) o.slots = 4;
    if (o.max_batch == 0) o.max_batch = 1024;
    if (o.max_samples == 0) o.max_samples = 65536;
    if (o.slots < 1 || o.slots > 64) return fail(MG_ERR_INVALID_ARG, "slots must be in 1..64");
    if (o.max_batch < 1 || o.max_batch > (1 << 20)) return fail(MG_ERR_INVALID_ARG, "max_batch must be in 1..2^20");
    if (o.max_samples < 1 || o.max_samples > (1ll << 31)) return fail(MG_ERR_INVALID_ARG, "max_samples out of range");
    if (o.hist_type != MG_HIST_U32 && o.hist_type != MG_HIST_F32) return fail(MG_ERR_INVALID_ARG, "bad hist_type");
    if (o.storage != MG_F32 && o.storage != MG_F16 && o.storage != MG_BF16)
        return fail(MG_ERR_INVALID_ARG, "bad storage dtype");
    if (o.memory_budget < 0) return fail(MG_ERR_INVALID_ARG, "negative memory_budget");
    if (o.plain != 0 && o.plain != 1) return fail(MG_ERR_INVALID_ARG, "plain must be 0 or 1");
    std::unique_ptr<mg_server> sv(new (std::nothrow) mg_server());
    if (!sv) return fail(MG_ERR_OOM, "host allocation failed");
    sv->o = o;
    sv->esize = o.storage == MG_F32 ? 4 : 2;
    MG_CUDA(cudaGetDevice(&sv->device));
    sv->slots.resize((size_t)o.slots);
    sv->vols.reserve(kMaxVolumes);
    sv->vq.reserve(kMaxVolumes);
    for (Slot& sl : sv->slots) sl.vols.reserve(kMaxVolumes);
    mg_status st = MG_OK;
    for (Slot& sl : sv->slots) {
        if (st == MG_OK) st = cuda_ok(cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking), "cudaStreamCreate");
        if (st == MG_OK) st = cuda_ok(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming), "cudaEventCreate");
    }
    if (st != MG_OK) {
        mg_server_free(sv.release());
        return st;
    }
    *out = sv.release();
    return MG_OK;
}

MG_API mg_status mg_server_add_volume(mg_server* sv, mg_graph* g, int C, int* volume) {
    if (!sv || !g || !volume) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if ((int)sv->vols.size() >= kMaxVolumes) return fail(MG_ERR_CAPACITY, "at most 1024 volumes per server");
    if (!((C >= 1 && C <= 8) || C == 12 || C == 16)) return fail(MG_ERR_INVALID_ARG, "C must be 1-8, 12 or 16");
    if (g->device != sv->device) return fail(MG_ERR_INVALID_ARG, "graph lives on another device");
    if (g->L < 1) return fail(MG_ERR_INVALID_ARG, "empty volume");
    MG_CUDA(cudaSetDevice(sv->device));
    Volume v;
    v.g = g;
    v.C = C;
    for (int a = 0; a < 3; a++) v.dims[a] = g->geom.dims[0][a];
    const size_t Q = (size_t)sv->o.max_batch, S = g->S, N = (size_t)g->N;
    const size_t ms = (size_t)sv->o.max_samples;
    const size_t cap_blocks = std::max<size_t>(Q * 1024, 1 << 20), cap_chunks = std::max<size_t>(Q * 256, 1 << 18);
    // per slot: the plan (or the plain form's buffers and scratch) and the TF frame buffers
    const int F = frames_for(C);
    v.frames = F;
    const size_t tf_bytes = round_up((size_t)F * S * C * 4) + round_up(N * F * C * sv->esize) +
                            round_up((size_t)F * ms * 16) + round_up((size_t)F * ms * C * sv->esize);
    const size_t query_bytes =
        sv->o.plain ? round_up(Q * 24) + round_up(Q * S * 4) + 2 * Q * S * 4
                    : Q * 24 + Q * S * 4 * (sv->o.hist_type == MG_HIST_F32 ? 2 : 1) + Q * 64 + cap_blocks * 12 +
                          cap_chunks * 8;
    const int64_t need = (int64_t)((tf_bytes + query_bytes) * sv->slots.size()) + g->device_bytes();
    if (sv->o.memory_budget > 0 && sv->budget_used + need > sv->o.memory_budget)
        return fail(MG_ERR_CAPACITY, "volume not admitted: it needs " + std::to_string(need >> 20) + " MiB and " +
                                         std::to_string((sv->o.memory_budget - sv->budget_used) >> 20) +
                                         " MiB of the budget remain");
    if (sv->o.storage != MG_F32) MG_TRY(ensure_alpha16(g, (mg_dtype)sv->o.storage, nullptr));
    const size_t pin_bytes = pinned_bytes(Q, S, C, F, ms, sv->esize);
    std::vector<VolSlot> made(sv->slots.size());
    mg_status st = MG_OK;
    for (size_t k = 0; k < made.size() && st == MG_OK; k++) {
        VolSlot& vs = made[k];
        if (sv->o.plain) {
            st = vs.boxes_dev.alloc(&g->al, Q * 24, nullptr);
            if (st == MG_OK) st = vs.out_dev.alloc(&g->al, Q * S * 4, nullptr);
        } else {
            mg_query_opts qo{};
            qo.hist_type = sv->o.hist_type;
            st = mg_query_plan_create(g, (int64_t)Q, &qo, (int64_t)cap_blocks, (int64_t)cap_chunks, &vs.plan);
            if (st == MG_OK) vs.pp = plan_parts(vs.plan);
        }
        if (st == MG_OK) st = vs.tf_dev.alloc(&g->al, (size_t)F * S * C * 4, nullptr);
        if (st == MG_OK) st = vs.vals_dev.alloc(&g->al, N * F * C * sv->esize, nullptr);
        if (st == MG_OK) st = vs.samples_dev.alloc(&g->al, (size_t)F * ms * 16, nullptr);
        if (st == MG_OK) st = vs.render_dev.alloc(&g->al, (size_t)F * ms * C * sv->esize, nullptr);
        for (Buf* b : {&vs.boxes_dev, &vs.out_dev, &vs.tf_dev, &vs.vals_dev, &vs.samples_dev, &vs.render_dev})
            b->s = nullptr;
        if (st == MG_OK) st = cuda_ok(cudaMallocHost(&vs.pin, pin_bytes), "cudaMallocHost");
        if (st == MG_OK) {
            unsigned char* p = vs.pin;
            vs.pin_q = reinterpret_cast<int64_t*>(p);
            p += round_up(8);
            vs.pin_status = reinterpret_cast<unsigned*>(p);
            p += round_up(4);
            vs.pin_boxes = reinterpret_cast<int32_t*>(p);
            p += round_up(Q * 24);
            vs.pin_out = p;
            p += round_up(Q * S * 4);
            vs.pin_tf = reinterpret_cast<float*>(p);
            p += round_up((size_t)F * S * C * 4);
            vs.pin_samples = reinterpret_cast<float*>(p);
            p += round_up((size_t)F * ms * 16);
            vs.pin_render = p;
        }
    }
    // settle the per-stream scratch arenas of the propagation (and of the
    // plain query) with two calls on every slot, so serving allocates nothing
    for (size_t k = 0; k < made.size() && st == MG_OK; k++) {
        VolSlot& vs = made[k];
        cudaStream_t s = sv->slots[k].s;
        st = cuda_ok(cudaMemsetAsync(vs.tf_dev.p, 0, (size_t)F * S * C * 4, s), "admission");
        for (int rep = 0; rep < 2 && st == MG_OK; rep++) {
            st = propagate_multi(g, vs.tf_dev.as<float>(), F, C, (mg_dtype)sv->o.storage, vs.vals_dev.p, s);
            if (st == MG_OK && sv->o.plain) {
                const int32_t unit[6] = {0, 0, 0, 1, 1, 1};
                st = cuda_ok(cudaMemcpyAsync(vs.boxes_dev.p, unit, 24, cudaMemcpyHostToDevice, s), "admission");
                mg_query_opts o{};
                o.hist_type = sv->o.hist_type;
                o.schedule = MG_SCHED_PLAIN;
                if (st == MG_OK)
                    st = query_boxes(g, vs.boxes_dev.as<int32_t>(), 1, o, vs.out_dev.p, S, nullptr, nullptr, nullptr, s);
            }
            if (st == MG_OK) st = cuda_ok(cudaStreamSynchronize(s), "admission");
        }
    }
    if (st == MG_OK) st = cuda_ok(cudaDeviceSynchronize(), "admission");
    if (st != MG_OK) {
        cudaDeviceSynchronize();
        for (VolSlot& vs : made) release_slot_volume(vs);
        return st;
    }
    if (made[0].plan) {
        v.chunk = made[0].pp.chunk;
        v.cap_blocks = made[0].pp.cap_blocks;
        v.cap_chunks = made[0].pp.cap_chunks;
    } else {
        v.cap_blocks = v.cap_chunks = ~0ull;
    }
    v.bytes = need;
    {
        // capacity is reserved: no element moves while the worker reads them
        std::lock_guard<std::mutex> lk(sv->mu);
        for (size_t k = 0; k < sv->slots.size(); k++) sv->slots[k].vols.push_back(std::move(made[k]));
        sv->vols.push_back(v);
        sv->vq.emplace_back();
        sv->budget_used += need;
        *volume = (int)sv->vols.size() - 1;
    }
    return MG_OK;
}

MG_API mg_status mg_server_remove_volume(mg_server* sv, int volume, double timeout_s) {
    if (!sv) return fail(MG_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    if (volume < 0 || volume >= (int)sv->vols.size() || sv->vols[volume].removed)
        return fail(MG_ERR_INVALID_ARG, "unknown or removed volume");
    Volume& v = sv->vols[volume];
    v.removed = true;   // submissions now fail
    if (!sv->started) {
        // nothing runs before the start: its queued requests are cancelled
        for (std::deque<Req>* d : {&sv->vq[volume].box, &sv->vq[volume].tf}) {
            for (const Req& q : *d) {
                Rec& rec = sv->recs[q.ticket];
                rec.state = kDone;
                rec.status = MG_ERR_CANCELLED;
                rec.error = "volume removed before the request was launched";
                sv->stats.cancelled++;
            }
            sv->queued -= (int64_t)d->size();
            d->clear();
        }
        sv->done_cv.notify_all();
    }
    // wait until no queued or running work refers to the volume
    auto busy = [&]() {
        if (!sv->vq[volume].box.empty() || !sv->vq[volume].tf.empty()) return true;
        for (const Slot& sl : sv->slots)
            if (sl.busy && !sl.work.empty() && sl.work[0].r.volume == volume) return true;
        return false;
    };
    const auto until = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 1e9);
    while (busy()) {
        if (sv->done_cv.wait_until(lk, until) == std::cv_status::timeout && busy()) {
            v.removed = false;
            return fail(MG_ERR_TIMEOUT, "the volume's requests did not finish in time");
        }
    }
    // its per-slot plans and buffers go back to the graph's allocator
    for (Slot& sl : sv->slots) {
        cudaStreamSynchronize(sl.s);
        arena_drop(v.g, sl.s);
        release_slot_volume(sl.vols[volume]);
        VolSlot empty;
        std::swap(sl.vols[volume], empty);
    }
    sv->budget_used -= v.bytes;
    v.bytes = 0;
    return MG_OK;
}

MG_API mg_status mg_server_start(mg_server* sv) {
    if (!sv) return fail(MG_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->started) return MG_OK;
    if (sv->vols.empty()) return fail(MG_ERR_INVALID_ARG, "no volume admitted");
    sv->worker = std::thread(worker_loop, sv);
    sv->started = true;
    return MG_OK;
}

MG_API mg_status mg_server_submit(mg_server* sv, const mg_request* r, uint64_t* ticket) {
    if (!sv || !r) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    return submit(sv, *r, Clock::now(), ticket);
}

MG_API mg_status mg_server_cancel(mg_server* sv, uint64_t ticket) {
    if (!sv) return fail(MG_ERR_INVALID_ARG, "server is NULL");
    std::lock_guard<std::mutex> lk(sv->mu);
    for (VolQueue& vq : sv->vq)
        for (std::deque<Req>* d : {&vq.box, &vq.tf})
            for (auto it = d->begin(); it != d->end(); ++it) {
                if (it->ticket != ticket) continue;
                Rec& rec = sv->recs[ticket];
                rec.state = kDone;
                rec.status = MG_ERR_CANCELLED;
                rec.error = "request cancelled";
                d->erase(it);
                sv->queued--;
                sv->stats.cancelled++;
                sv->done_cv.notify_all();
                return MG_OK;
            }
    return fail(MG_ERR_INVALID_ARG, "request is not queued (already launched, done or unknown)");
}

MG_API mg_status mg_server_wait(mg_server* sv, uint64_t ticket, double timeout_s, double* latency_s) {
    if (!sv) return fail(MG_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(sv->mu);
    if (sv->recs.find(ticket) == sv->recs.end()) return fail(MG_ERR_INVALID_ARG, "unknown ticket (or already waited for)");
    auto ready = [&] { return sv->recs[ticket].state == kDone; };
    if (timeout_s > 0) {
        if (!sv->done_cv.wait_for(lk, std::chrono::duration<double>(timeout_s), ready))
            return fail(MG_ERR_TIMEOUT, "request not completed within the timeout");
    } else {
        sv->done_cv.wait(lk, ready);
    }
    const Rec rec = sv->recs[ticket];
    sv->recs.erase(ticket);
    if (latency_s) *latency_s = rec.latency;
    if (rec.status != MG_OK) return fail(rec.status, rec.error);
    return MG_OK;
}

MG_API mg_status mg_server_replay(mg_server* sv, const mg_request* reqs, int64_t n, double* latency_s,
                                  double* wall_s) {
    if (!sv || (n > 0 && !reqs)) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (!sv->started) return fail(MG_ERR_INVALID_ARG, "server not started");
    if (n < 0) return fail(MG_ERR_INVALID_ARG, "negative request count");
    for (int64_t i = 0; i < n; i++) {
        if (!(reqs[i].arrival_s >= 0.0) || (i > 0 && reqs[i].arrival_s < reqs[i - 1].arrival_s))
            return fail(MG_ERR_INVALID_ARG, "arrival times must be non-negative and non-decreasing");
        Req q;
        MG_TRY(check_request(sv, reqs[i], &q));
    }
    std::vector<uint64_t> tickets((size_t)n);
    const Clock::time_point t0 = Clock::now();
    for (int64_t i = 0; i < n; i++) {
        const Clock::time_point at =
            t0 + std::chrono::duration_cast<Clock::duration>(std::chrono::duration<double>(reqs[i].arrival_s));
        for (Clock::time_point now = Clock::now(); now < at; now = Clock::now()) {
            if (at - now > std::chrono::microseconds(300))
                std::this_thread::sleep_for(at - now - std::chrono::microseconds(200));
        }
        MG_TRY(submit(sv, reqs[i], at, &tickets[(size_t)i]));
    }
    mg_status first = MG_OK;
    std::string first_err;
    for (int64_t i = 0; i < n; i++) {
        double lat = 0.0;
        const mg_status st = mg_server_wait(sv, tickets[(size_t)i], 0.0, &lat);
        if (st != MG_OK && first == MG_OK) {
            first = st;
            first_err = mg_last_error();
        }
        if (latency_s) latency_s[i] = lat;
    }
    if (wall_s) *wall_s = std::chrono::duration<double>(Clock::now() - t0).count();
    if (first != MG_OK) return fail(first, first_err);
    return MG_OK;
}

MG_API mg_status mg_server_stats_get(mg_server* sv, mg_server_stats* stats) {
    if (!sv || !stats) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    *stats = sv->stats;
    stats->memory_admitted = sv->budget_used;
    return MG_OK;
}

MG_API void mg_server_free(mg_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop.store(true);
    }
    sv->work_cv.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->device);
    cudaDeviceSynchronize();
    for (Slot& sl : sv->slots) {
        for (const Volume& v : sv->vols) arena_drop(v.g, sl.s);
        for (VolSlot& vs : sl.vols) release_slot_volume(vs);
        sl.vols.clear();   // device buffers go back to the graphs' allocators
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.s) cudaStreamDestroy(sl.s);
    }
    delete sv;
}

}  // extern "C"
