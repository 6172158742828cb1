// mg_abi.cu -- the extern "C" entry points of libmg: argument checks on the
// host, device selection, graph lifetime, error reporting.
#include "mg_internal.cuh"

#include <chrono>
#include <new>
#include <cstring>
#include <vector>

namespace mg {

namespace {
thread_local std::string t_err;

}  // namespace

mg_status status_from_bits(unsigned bits) {
    if (bits & kStatBadInput) return fail(MG_ERR_INVALID_ARG, "device saw invalid input (ID >= num_segments or malformed box)");
    if (bits & kStatCapacity) return fail(MG_ERR_CAPACITY, "node table capacity exceeded on the device");
    if (bits & kStatTimeout) return fail(MG_ERR_TIMEOUT, "a bounded device wait expired");
    if (bits & kStatInexact) return fail(MG_ERR_INEXACT, "integer push met a weight not divisible by a+b");
    return MG_OK;
}

void set_error(const std::string& msg) { t_err = msg; }

mg_status fail(mg_status st, const std::string& msg) {
    t_err = msg;
    return st;
}

mg_status cuda_fail(cudaError_t e, const char* what) {
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    return MG_ERR_CUDA;
}

void* Alloc::get(size_t bytes, cudaStream_t s) const {
    if (bytes == 0) bytes = 16;
    if (custom) return a.alloc(a.ctx, bytes, reinterpret_cast<mg_stream>(s));
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void Alloc::put(void* p, size_t bytes, cudaStream_t s) const {
    if (!p) return;
    if (bytes == 0) bytes = 16;
    if (custom) {
        a.free(a.ctx, p, bytes, reinterpret_cast<mg_stream>(s));
    } else {
        cudaFreeAsync(p, s);
    }
}

mg_status Buf::alloc(const Alloc* a, size_t n, cudaStream_t st) {
    release();
    al = a;
    s = st;
    bytes = n;
    p = a->get(n, st);
    if (!p) {
        bytes = 0;
        return fail(MG_ERR_OOM, "device allocation of " + std::to_string(n) + " bytes failed");
    }
    if (reinterpret_cast<uintptr_t>(p) % 256) {   // the kernels' vector loads rely on it
        release();
        return fail(MG_ERR_INVALID_ARG, "the allocator returned a pointer that is not 256-byte aligned");
    }
    return MG_OK;
}

void Buf::release() {
    if (p && al) al->put(p, bytes, s);
    p = nullptr;
    bytes = 0;
}

namespace {
void* arena_alloc(void* ctx, size_t bytes, mg_stream s) {
    Arena* a = static_cast<Arena*>(ctx);
    const size_t n = (bytes + 255) & ~(size_t)255;
    if (a->buf.p && a->used + n <= a->buf.bytes) {
        void* p = static_cast<char*>(a->buf.p) + a->used;
        a->used += n;
        if (a->used > a->need) a->need = a->used;
        return p;
    }
    if (a->used + n > a->need) a->need = a->used + n;
    return a->fallback->get(bytes, reinterpret_cast<cudaStream_t>(s));
}

void arena_free(void* ctx, void* p, size_t bytes, mg_stream s) {
    Arena* a = static_cast<Arena*>(ctx);
    char* lo = static_cast<char*>(a->buf.p);
    if (lo && static_cast<char*>(p) >= lo && static_cast<char*>(p) < lo + a->buf.bytes) return;
    a->fallback->put(p, bytes, reinterpret_cast<cudaStream_t>(s));
}
}  // namespace

mg_status arena_begin(mg_graph* g, cudaStream_t s, Arena** out) {
    std::lock_guard<std::mutex> lk(g->arena_mu);
    auto& slot = g->arenas[s];
    if (!slot) {
        slot.reset(new (std::nothrow) Arena());
        if (!slot) return fail(MG_ERR_OOM, "host allocation failed");
        slot->fallback = &g->al;
        slot->view.a.ctx = slot.get();
        slot->view.a.alloc = arena_alloc;
        slot->view.a.free = arena_free;
        slot->view.custom = true;
        if (cudaMallocHost(&slot->pinned, 8 * sizeof(uint64_t)) != cudaSuccess) {
            cudaGetLastError();
            slot->pinned = nullptr;
        }
    }
    Arena* a = slot.get();
    if (a->need > a->buf.bytes) {
        a->buf.release();   // stream-ordered after the previous call on s
        MG_TRY(a->buf.alloc(&g->al, a->need + a->need / 4, s));
    }
    a->used = 0;
    *out = a;
    return MG_OK;
}

void arena_drop(mg_graph* g, cudaStream_t s) {
    std::lock_guard<std::mutex> lk(g->arena_mu);
    auto it = g->arenas.find(s);
    if (it == g->arenas.end()) return;
    it->second->buf.s = nullptr;   // the caller has synchronised the device
    g->arenas.erase(it);
}

mg_status sync_status(mg_graph* g, cudaStream_t s) {
    MG_CUDA(cudaStreamSynchronize(s));
    unsigned bits = 0;
    MG_CUDA(cudaMemcpy(&bits, g->status.p, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (bits) MG_CUDA(cudaMemset(g->status.p, 0, sizeof(unsigned)));
    return status_from_bits(bits);
}

}  // namespace mg

int64_t mg_graph::device_bytes() const {
    return (int64_t)(mip0.bytes + mip.bytes + mip0x[0].bytes + mip0x[1].bytes + mip0x[2].bytes + mipx[0].bytes +
                     mipx[1].bytes + mipx[2].bytes + pq.bytes + ab.bytes + ab32.bytes + alpha.bytes + alpha16.bytes +
                     alphab16.bytes + status.bytes + lut_meta.bytes + lut.bytes + wq.bytes + dw.bytes +
                     err_off.bytes + err_src.bytes + err_mu.bytes + err_dmu.bytes);
}

using namespace mg;

extern "C" {

MG_API const char* mg_last_error(void) { return t_err.c_str(); }

MG_API const char* mg_version(void) { return "mixgraph-gb300 0.1 (sm_103a)"; }

MG_API mg_status mg_build(const void* ids, int64_t nx, int64_t ny, int64_t nz, uint32_t num_segments,
                          const mg_build_opts* opts, const mg_allocator* allocator, mg_stream stream,
                          mg_graph** out) {
    MG_RANGE("mg_build");
    t_err.clear();
    if (!out) return fail(MG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ids) return fail(MG_ERR_INVALID_ARG, "ids is NULL");
    if (nx < 1 || ny < 1 || nz < 1) return fail(MG_ERR_INVALID_ARG, "dims must be >= 1");
    if (nx > 65535 || ny > 65535 || nz > 65535)
        return fail(MG_ERR_UNSUPPORTED, "each axis must be at most 65535 voxels");
    if ((uint64_t)nx * (uint64_t)ny * (uint64_t)nz >= (1ull << 32))
        return fail(MG_ERR_UNSUPPORTED, "volumes must hold fewer than 2^32 voxels");
    if (num_segments < 1 || num_segments > (1u << 31))
        return fail(MG_ERR_INVALID_ARG, "num_segments must be in 1..2^31");
    int id_bytes = opts ? opts->id_bytes : 2;
    if (id_bytes != 2 && id_bytes != 4) return fail(MG_ERR_INVALID_ARG, "id_bytes must be 2 or 4");
    if (allocator && (!allocator->alloc || !allocator->free))
        return fail(MG_ERR_INVALID_ARG, "allocator needs alloc and free");
    mg_graph* g = new (std::nothrow) mg_graph();
    if (!g) return fail(MG_ERR_OOM, "host allocation failed");
    if (allocator) {
        g->al.a = *allocator;
        g->al.custom = true;
    }
    g->S = num_segments;
    cudaGetDevice(&g->device);
    auto t0 = std::chrono::steady_clock::now();
    mg_status st = build_graph(g, ids, id_bytes, nx, ny, nz, reinterpret_cast<cudaStream_t>(stream));
    if (st == MG_OK) {
        cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
        if (e != cudaSuccess) st = cuda_fail(e, "mg_build sync");
    }
    if (st != MG_OK) {
        std::string msg = t_err;
        cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
        delete g;
        t_err = msg;
        return st;
    }
    g->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();

    // graph buffers are released on the legacy stream after a device sync
    for (Buf* b : {&g->mip0, &g->mip, &g->mip0x[0], &g->mip0x[1], &g->mip0x[2], &g->mipx[0], &g->mipx[1],
                   &g->mipx[2], &g->pq, &g->ab, &g->ab32, &g->alpha, &g->status})
        b->s = nullptr;
    *out = g;
    return MG_OK;
}

MG_API mg_status mg_graph_info_get(const mg_graph* g, mg_graph_info* info) {
    if (!g || !info) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->num_segments = g->S;
    info->levels = g->L;
    info->depth = g->D;
    info->num_nodes = g->N;
    for (int l = 0; l < g->L; l++)
        for (int k = 0; k < 3; k++) info->dims[l][k] = g->geom.dims[l][k];
    for (int d = 0; d <= g->D + 1 && d < MG_MAX_DEPTH + 2; d++) info->bucket[d] = g->bucket[d];
    info->max_list = g->max_list;
    info->pairs = g->pairs;
    info->device_bytes = g->device_bytes();
    info->build_ms = g->build_ms;
    info->lut_entries = g->lut_entries;
    return MG_OK;
}

MG_API mg_status mg_graph_copy_nodes(const mg_graph* g, uint32_t* p, uint32_t* q, uint64_t* a, uint64_t* b,
                                     mg_stream stream) {
    if (!g) return fail(MG_ERR_INVALID_ARG, "graph is NULL");
    DeviceGuard dg(g->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t N = (size_t)g->N;
    std::vector<uint2> hpq(N);
    std::vector<ulonglong2> hab(N);
    MG_CUDA(cudaMemcpyAsync(hpq.data(), g->pq.p, N * sizeof(uint2), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaMemcpyAsync(hab.data(), g->ab.p, N * sizeof(ulonglong2), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    std::vector<uint32_t> t32(N);
    std::vector<uint64_t> t64(N);
    if (p) {
        for (size_t i = 0; i < N; i++) t32[i] = hpq[i].x;
        MG_CUDA(cudaMemcpyAsync(p, t32.data(), N * 4, cudaMemcpyDefault, s));
        MG_CUDA(cudaStreamSynchronize(s));
    }
    if (q) {
        for (size_t i = 0; i < N; i++) t32[i] = hpq[i].y;
        MG_CUDA(cudaMemcpyAsync(q, t32.data(), N * 4, cudaMemcpyDefault, s));
        MG_CUDA(cudaStreamSynchronize(s));
    }
    if (a) {
        for (size_t i = 0; i < N; i++) t64[i] = hab[i].x;
        MG_CUDA(cudaMemcpyAsync(a, t64.data(), N * 8, cudaMemcpyDefault, s));
        MG_CUDA(cudaStreamSynchronize(s));
    }
    if (b) {
        for (size_t i = 0; i < N; i++) t64[i] = hab[i].y;
        MG_CUDA(cudaMemcpyAsync(b, t64.data(), N * 8, cudaMemcpyDefault, s));
        MG_CUDA(cudaStreamSynchronize(s));
    }
    return MG_OK;
}

MG_API mg_status mg_graph_copy_mip(const mg_graph* g, int level, uint32_t* dst, mg_stream stream) {
    if (!g || !dst) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (level < 0 || level >= g->L) return fail(MG_ERR_INVALID_ARG, "level out of range");
    DeviceGuard dg(g->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t n = (int64_t)g->geom.dims[level][0] * g->geom.dims[level][1] * g->geom.dims[level][2];
    if (level == 0 && g->id0_bytes == 2) {
        std::vector<uint16_t> h16((size_t)n);
        std::vector<uint32_t> h32((size_t)n);
        MG_CUDA(cudaMemcpyAsync(h16.data(), g->mip0.p, (size_t)n * 2, cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < n; i++) h32[(size_t)i] = h16[(size_t)i];
        MG_CUDA(cudaMemcpyAsync(dst, h32.data(), (size_t)n * 4, cudaMemcpyDefault, s));
    } else if (level == 0) {
        MG_CUDA(cudaMemcpyAsync(dst, g->mip0.p, (size_t)n * 4, cudaMemcpyDefault, s));
    } else {
        const uint32_t* src = g->mip.as<uint32_t>() + g->geom.off[level];
        MG_CUDA(cudaMemcpyAsync(dst, src, (size_t)n * 4, cudaMemcpyDefault, s));
    }
    MG_CUDA(cudaStreamSynchronize(s));
    return MG_OK;
}

MG_API mg_status mg_propagate_tf(mg_graph* g, const float* tf, int C, mg_dtype storage, void* vals,
                                 mg_stream stream) {
    MG_RANGE("mg_propagate_tf");
    if (!g || !tf || !vals) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (C < 1 || C > 16) return fail(MG_ERR_INVALID_ARG, "C must be in 1..16");
    if (storage != MG_F32 && storage != MG_F16 && storage != MG_BF16)
        return fail(MG_ERR_INVALID_ARG, "storage must be MG_F32, MG_F16 or MG_BF16");
    DeviceGuard dg(g->device);
    return propagate(g, tf, C, storage, vals, reinterpret_cast<cudaStream_t>(stream));
}

MG_API mg_status mg_propagate_tf_multi(mg_graph* g, const float* tfs, int k, int C, mg_dtype storage, void* vals,
                                       mg_stream stream) {
    MG_RANGE("mg_propagate_tf_multi");
    if (!g || !tfs || !vals) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (k < 1 || k > 32) return fail(MG_ERR_INVALID_ARG, "k must be in 1..32");
    if (C < 1 || C > 16) return fail(MG_ERR_INVALID_ARG, "C must be in 1..16");
    if (storage != MG_F32 && storage != MG_F16 && storage != MG_BF16)
        return fail(MG_ERR_INVALID_ARG, "storage must be MG_F32, MG_F16 or MG_BF16");
    DeviceGuard dg(g->device);
    return propagate_multi(g, tfs, k, C, storage, vals, reinterpret_cast<cudaStream_t>(stream));
}

MG_API mg_status mg_query_boxes(const mg_graph* g, const int32_t* boxes, int64_t Q, const mg_query_opts* opts,
                                void* out, size_t out_capacity, uint32_t* seg, uint64_t* offsets,
                                size_t* out_required, mg_stream stream) {
    MG_RANGE("mg_query_boxes");
    if (!g) return fail(MG_ERR_INVALID_ARG, "graph is NULL");
    if (Q < 0) return fail(MG_ERR_INVALID_ARG, "Q must be >= 0");
    mg_query_opts o{};
    if (opts) o = *opts;
    if (o.hist_type != MG_HIST_U32 && o.hist_type != MG_HIST_F32)
        return fail(MG_ERR_INVALID_ARG, "hist_type must be MG_HIST_U32 or MG_HIST_F32");
    if (o.layout != MG_LAYOUT_DENSE && o.layout != MG_LAYOUT_CSR)
        return fail(MG_ERR_INVALID_ARG, "layout must be MG_LAYOUT_DENSE or MG_LAYOUT_CSR");
    if (o.alpha_dtype != MG_F32 && o.alpha_dtype != MG_F16 && o.alpha_dtype != MG_BF16)
        return fail(MG_ERR_INVALID_ARG, "alpha_dtype must be MG_F32, MG_F16 or MG_BF16");
    if (o.hist_type == MG_HIST_U32 && o.alpha_dtype != MG_F32)
        return fail(MG_ERR_INVALID_ARG, "16-bit weights apply to the fp32 push only");
    if (g->quantised && o.hist_type == MG_HIST_U32)
        return fail(MG_ERR_UNSUPPORTED, "a quantised graph has no exact weights: use MG_HIST_F32");
    if (o.schedule != MG_SCHED_BATCHED && o.schedule != MG_SCHED_PLAIN && o.schedule != MG_SCHED_NAIVE)
        return fail(MG_ERR_INVALID_ARG, "schedule must be MG_SCHED_BATCHED, MG_SCHED_PLAIN or MG_SCHED_NAIVE");
    if (o.chunk_cubes < 0 || o.block_threads < 0) return fail(MG_ERR_INVALID_ARG, "negative tuning option");
    if (o.block_threads && o.block_threads != 128 && o.block_threads != 256 && o.block_threads != 512)
        return fail(MG_ERR_INVALID_ARG, "block_threads must be 128, 256 or 512");
    if (Q > 0 && !boxes) return fail(MG_ERR_INVALID_ARG, "boxes is NULL");
    if (o.layout == MG_LAYOUT_CSR && !offsets) return fail(MG_ERR_INVALID_ARG, "offsets is NULL");
    if (o.layout == MG_LAYOUT_CSR && out_capacity > 0 && (!seg || !out))
        return fail(MG_ERR_INVALID_ARG, "seg/out is NULL");
    if (o.layout == MG_LAYOUT_DENSE && Q > 0) {
        if (!out) return fail(MG_ERR_INVALID_ARG, "out is NULL");
        if ((uint64_t)out_capacity < (uint64_t)Q * g->S)
            return fail(MG_ERR_INVALID_ARG, "dense out_capacity must be >= Q*S");
    }
    if (Q >= (1ll << 31)) return fail(MG_ERR_UNSUPPORTED, "Q must be < 2^31");
    DeviceGuard dg(g->device);
    return query_boxes(g, boxes, Q, o, out, out_capacity, seg, offsets, out_required,
                       reinterpret_cast<cudaStream_t>(stream));
}

MG_API mg_status mg_query_timing(const mg_graph* g, float* plan_ms, float* main_ms, float* output_ms) {
    if (!g) return fail(MG_ERR_INVALID_ARG, "graph is NULL");
    DeviceGuard dg(g->device);
    return query_timing(g, plan_ms, main_ms, output_ms);
}

MG_API mg_status mg_count_cubes(const mg_graph* g, const int32_t* boxes, int64_t Q, uint64_t* cubes,
                                mg_stream stream) {
    MG_RANGE("mg_count_cubes");
    if (!g) return fail(MG_ERR_INVALID_ARG, "graph is NULL");
    if (Q < 0) return fail(MG_ERR_INVALID_ARG, "Q must be >= 0");
    if (Q == 0) return MG_OK;
    if (!boxes || !cubes) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (Q >= (1ll << 31)) return fail(MG_ERR_UNSUPPORTED, "Q must be < 2^31");
    DeviceGuard dg(g->device);
    return count_cubes(g, boxes, Q, cubes, reinterpret_cast<cudaStream_t>(stream));
}

MG_API mg_status mg_render_lookup(const mg_graph* g, const void* vals, int C, mg_dtype dtype, const float* samples,
                                  int64_t P, void* out, mg_stream stream) {
    MG_RANGE("mg_render_lookup");
    if (!g) return fail(MG_ERR_INVALID_ARG, "graph is NULL");
    if (C < 1 || C > 16) return fail(MG_ERR_INVALID_ARG, "C must be in 1..16");
    if (dtype != MG_F32 && dtype != MG_F16 && dtype != MG_BF16)
        return fail(MG_ERR_INVALID_ARG, "dtype must be MG_F32, MG_F16 or MG_BF16");
    if (P < 0) return fail(MG_ERR_INVALID_ARG, "P must be >= 0");
    if (P == 0) return MG_OK;
    if (!vals || !samples || !out) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(g->device);
    return render_lookup(g, vals, C, dtype, samples, P, out, reinterpret_cast<cudaStream_t>(stream));
}

MG_API mg_status mg_render_lookup_multi(const mg_graph* g, const void* vals, int k, int C, mg_dtype dtype,
                                        const float* samples, const int64_t* offsets, void* out, mg_stream stream) {
    MG_RANGE("mg_render_lookup_multi");
    if (!g || !offsets) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (k < 1 || k > 32) return fail(MG_ERR_INVALID_ARG, "k must be in 1..32");
    if (C < 1 || C > 16) return fail(MG_ERR_INVALID_ARG, "C must be in 1..16");
    if (dtype != MG_F32 && dtype != MG_F16 && dtype != MG_BF16)
        return fail(MG_ERR_INVALID_ARG, "dtype must be MG_F32, MG_F16 or MG_BF16");
    if (offsets[0] != 0) return fail(MG_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int j = 0; j < k; j++)
        if (offsets[j + 1] < offsets[j]) return fail(MG_ERR_INVALID_ARG, "offsets must be non-decreasing");
    if (offsets[k] == 0) return MG_OK;
    if (!vals || !samples || !out) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(g->device);
    return render_lookup_multi(g, vals, k, C, dtype, samples, offsets, out, reinterpret_cast<cudaStream_t>(stream));
}

MG_API mg_status mg_raymarch(const mg_graph* g, const float* vals, const float* opacity, const mg_camera* cam,
                             float* image, int32_t* steps, mg_stream stream) {
    MG_RANGE("mg_raymarch");
    if (!g || !vals || !cam || !image) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (cam->width < 1 || cam->height < 1 || cam->width > 16384 || cam->height > 16384)
        return fail(MG_ERR_INVALID_ARG, "image size must be 1..16384 per side");
    if (!(cam->pix > 0.0f) || !(cam->base_step > 0.0f) || cam->max_steps < 1)
        return fail(MG_ERR_INVALID_ARG, "pix and base_step must be > 0 and max_steps >= 1");
    if (cam->lod_bias < -64 || cam->lod_bias > 64) return fail(MG_ERR_INVALID_ARG, "lod_bias must be in -64..64");
    DeviceGuard dg(g->device);
    return raymarch(g, vals, opacity, *cam, image, steps, reinterpret_cast<cudaStream_t>(stream));
}

MG_API mg_status mg_sync_status(mg_graph* g, mg_stream stream) {
    if (!g) return fail(MG_ERR_INVALID_ARG, "graph is NULL");
    DeviceGuard dg(g->device);
    return sync_status(g, reinterpret_cast<cudaStream_t>(stream));
}

MG_API mg_status mg_selftest_bounded_wait(int satisfied, unsigned spin_limit, mg_stream stream) {
    if (satisfied != 0 && satisfied != 1) return fail(MG_ERR_INVALID_ARG, "satisfied must be 0 or 1");
    if (spin_limit < 1 || spin_limit > (1u << 22)) return fail(MG_ERR_INVALID_ARG, "spin_limit must be in 1..2^22");
    return selftest_wait(satisfied == 1, spin_limit, reinterpret_cast<cudaStream_t>(stream));
}

MG_API void mg_free(mg_graph* g) {
    if (!g) return;
    DeviceGuard dg(g->device);
    cudaDeviceSynchronize();
    for (auto& kv : g->arenas) kv.second->buf.s = nullptr;   // the device is idle; the call streams may be gone
    delete g;
}

}  // extern "C"
