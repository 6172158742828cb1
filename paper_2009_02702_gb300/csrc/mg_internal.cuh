// mg_internal.cuh -- internal declarations shared by the libmg translation units.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>
#include <map>
#include <memory>
#include <mutex>
#include <string>

#include "mg.h"

#include <nvtx3/nvToolsExt.h>

namespace mg {

// ---------------------------------------------------------------------------
// status word bits set by kernels (read by mg_sync_status)
// ---------------------------------------------------------------------------
enum : unsigned {
    kStatBadInput = 1u << 0,   // ID >= S, malformed box
    kStatCapacity = 1u << 1,   // node table or hash full
    kStatTimeout = 1u << 2,    // bounded wait expired
    kStatInexact = 1u << 3,    // integer push met W % (a+b) != 0
};

constexpr uint32_t kNone = 0xFFFFFFFFu;   // no predecessor
constexpr uint32_t kDead = 0xFFFFFFFEu;   // node slot lost a publication race

// ---------------------------------------------------------------------------
// profiler ranges (NVTX; no cost unless a profiler is attached)
// ---------------------------------------------------------------------------
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};
#define MG_RANGE(name) ::mg::Range mg_range_scope_(name)

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
mg_status fail(mg_status st, const std::string& msg);
mg_status cuda_fail(cudaError_t e, const char* what);
// the error of the first bit set in a device status word (MG_OK for 0)
mg_status status_from_bits(unsigned bits);

#define MG_CUDA(call)                                            \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return ::mg::cuda_fail(e_, #call); \
    } while (0)

#define MG_TRY(call)                         \
    do {                                     \
        mg_status s_ = (call);               \
        if (s_ != MG_OK) return s_;          \
    } while (0)

// ---------------------------------------------------------------------------
// memory through the caller's allocator (or cudaMallocAsync)
// ---------------------------------------------------------------------------
struct Alloc {
    mg_allocator a{};
    bool custom = false;
    void* get(size_t bytes, cudaStream_t s) const;
    void put(void* p, size_t bytes, cudaStream_t s) const;
};

// RAII scratch buffer released in stream order
struct Buf {
    const Alloc* al = nullptr;
    cudaStream_t s = nullptr;
    void* p = nullptr;
    size_t bytes = 0;
    Buf() = default;
    Buf(const Buf&) = delete;
    Buf& operator=(const Buf&) = delete;
    Buf(Buf&& o) noexcept { *this = static_cast<Buf&&>(o); }
    Buf& operator=(Buf&& o) noexcept {
        release();
        al = o.al; s = o.s; p = o.p; bytes = o.bytes;
        o.p = nullptr; o.bytes = 0;
        return *this;
    }
    ~Buf() { release(); }
    mg_status alloc(const Alloc* a, size_t n, cudaStream_t st);
    void release();
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

// Scratch arena for the calls made on one stream: bump allocation from one
// buffer, reset at the start of every call.  What does not fit comes from the
// graph's allocator; the next call on the stream grows the buffer to the
// high-water mark.  Calls on one stream run in order, so reuse is safe.
struct Arena {
    Buf buf;
    size_t used = 0, need = 0;
    const Alloc* fallback = nullptr;
    Alloc view;                  // an Alloc whose alloc/free go through this arena
    uint64_t* pinned = nullptr;  // 8 pinned host words for readbacks on this stream
    ~Arena() {
        if (pinned) cudaFreeHost(pinned);
    }
};

// ---------------------------------------------------------------------------
// the graph
// ---------------------------------------------------------------------------
struct LevelGeom {
    int L;
    int32_t dims[MG_MAX_LEVELS][3];
    int64_t off[MG_MAX_LEVELS];   // offset of level l (l >= 1) in the concatenated mip array
};

}  // namespace mg

struct mg_graph {
    mg::Alloc al;
    int device = 0;
    uint32_t S = 0;
    int L = 0;
    int D = 0;
    int64_t N = 0;
    mg::LevelGeom geom{};
    int64_t bucket[MG_MAX_DEPTH + 2] = {};
    int64_t max_list = 0, pairs = 0;
    double build_ms = 0.0;

    // level 0: segment IDs (uint16 when S <= 65536, else uint32)
    int id0_bytes = 2;
    mg::Buf mip0;
    // levels 1..L-1 concatenated, uint32 node IDs
    mg::Buf mip;
    // axis-major copies of the same IDs for box queries: copy 0 is x-fastest
    // (order x, y, z), copy 1 y-fastest (order y, z, x), copy 2 z-fastest
    // (order z, x, y).  A footprint block reads the copy whose fastest axis is
    // its longest side.  Rows of copy c at level l are qpitch[l][c] IDs apart,
    // the row length rounded up to 32 bytes, so every row starts on a 32-byte
    // boundary; levels >= 1 are concatenated at qoff[l][c].  Copy 0 of level 0
    // is mip0 itself when its rows need no padding (mip0x[0] empty then).
    mg::Buf mip0x[3];
    mg::Buf mipx[3];
    int32_t qpitch[MG_MAX_LEVELS][3] = {};
    int64_t qoff[MG_MAX_LEVELS][3] = {};
    // node table, canonical order, N entries
    mg::Buf pq;       // uint2 (p, q); (kNone, kNone) for sources
    mg::Buf ab;       // ulonglong2 (a, b) exact coprime weights
    mg::Buf ab32;     // uint2 (a, b) when a+b < 2^32, else (0, 0)
    mg::Buf alpha;    // float b/(a+b)
    mg::Buf alpha16;  // lazily: signed __half alpha, swap flag in the sign
    mg::Buf alphab16; // lazily: signed __nv_bfloat16 alpha, swap flag in the sign
    mg::Buf status;   // unsigned int status word
    // mixture lookup table of the range queries (empty if too large):
    // lut_meta[n] = (first entry, entries << 8 | lmin), lut = (source, count)
    mg::Buf lut_meta;
    mg::Buf lut;
    int64_t lut_entries = 0;
    // quantised graph (from the greedy factorisation): a node's weight is its
    // bin's codeword, no exact weights (a = b = 0), so only fp32 pushes apply
    bool quantised = false;
    mg::Buf wq;        // double: weight of q of every node (quantised graphs)
    mg::Buf dw;        // double: its uncertainty (the bin's sigma)
    // mixture table with uncertainties (Sec. 3.5), built on request:
    // node n's row is [err_off[n], err_off[n+1]) of (source, mu, dmu)
    mg::Buf err_off, err_src, err_mu, err_dmu;
    int64_t err_entries = 0;
    // launch shape chosen by mg_query_autotune, per histogram type (0 = none yet)
    int tuned_chunk[2] = {0, 0};
    int tuned_threads[2] = {0, 0};
    // per-stream scratch arenas of query calls
    std::mutex arena_mu;
    std::map<cudaStream_t, std::unique_ptr<mg::Arena>> arenas;
    // events of the last timed query call: plan start, main start, main end, output end
    cudaEvent_t qev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool qev_valid = false;
    ~mg_graph() {
        for (auto& e : qev)
            if (e) cudaEventDestroy(e);
    }

    int64_t device_bytes() const;
};

namespace mg {

// ---------------------------------------------------------------------------
// device primitives (mg_prims.cu)
// ---------------------------------------------------------------------------
// exclusive scan of n elements; if total != nullptr, writes the sum there (device)
mg_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                             const Alloc& al, cudaStream_t s);
mg_status scan_exclusive_u64(const uint64_t* in, uint64_t* out, int64_t n, uint64_t* total,
                             const Alloc& al, cudaStream_t s);
// stable LSD radix sort of (key, value) by key bits [0, bits); result in keys/vals
mg_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, const Alloc& al,
                           cudaStream_t s);

// ---------------------------------------------------------------------------
// stages
// ---------------------------------------------------------------------------
mg_status build_graph(mg_graph* g, const void* ids, int id_bytes, int64_t nx, int64_t ny, int64_t nz,
                      cudaStream_t s);
mg_status propagate(mg_graph* g, const float* tf, int C, mg_dtype storage, void* vals, cudaStream_t s);
mg_status propagate_multi(mg_graph* g, const float* tf, int k, int C, mg_dtype storage, void* vals, cudaStream_t s);
// the per-node mixture lookup table of the range queries (after the build)
mg_status build_lut(mg_graph* g, cudaStream_t s);
// the padded axis-major copies of the box queries, from mip0 and mip
mg_status build_query_copies(mg_graph* g, cudaStream_t s);
// box histograms summed from the mixture table, with error bars (Sec. 3.5-3.6)
mg_status query_lut(const mg_graph* g, const int32_t* boxes, int64_t Q, double* hist, double* err, cudaStream_t s);
mg_status ensure_alpha16(mg_graph* g, mg_dtype dt, cudaStream_t s);
mg_status query_boxes(const mg_graph* g, const int32_t* boxes, int64_t Q, const mg_query_opts& o,
                      void* out, size_t cap, uint32_t* seg, uint64_t* offsets, size_t* required,
                      cudaStream_t s);
mg_status query_timing(const mg_graph* g, float* plan_ms, float* main_ms, float* out_ms);
// the arena of `s` on graph g, reset for a new call (grown if the last call overflowed)
mg_status arena_begin(mg_graph* g, cudaStream_t s, Arena** out);
// release the arena of a stream that is about to be destroyed (device idle)
void arena_drop(mg_graph* g, cudaStream_t s);
mg_status count_cubes(const mg_graph* g, const int32_t* boxes, int64_t Q, uint64_t* cubes,
                      cudaStream_t s);
// the bounded wait of the propagation on a flag that is set (or never set)
mg_status selftest_wait(bool satisfied, unsigned limit, cudaStream_t s);
mg_status render_lookup(const mg_graph* g, const void* vals, int C, mg_dtype dt, const float* samples,
                        int64_t P, void* out, cudaStream_t s);
mg_status render_lookup_multi(const mg_graph* g, const void* vals, int k, int C, mg_dtype dt, const float* samples,
                              const int64_t* offsets, void* out, cudaStream_t s);
mg_status raymarch(const mg_graph* g, const float* vals, const float* opacity, const mg_camera& cam, float* image,
                   int32_t* steps, cudaStream_t s);

// A query plan's own buffers, executable graph and footprint capacities, for
// the request loop, which stages boxes straight into them: a run is the boxes
// in `boxes`, Q in `Qd`, a launch of `exec`, and Q x S values in `result`.
struct PlanParts {
    int32_t* boxes;
    int64_t* Qd;
    void* result;
    cudaGraphExec_t exec;
    uint32_t chunk;
    uint64_t cap_blocks, cap_chunks;
};
PlanParts plan_parts(const mg_query_plan* p);

// ---------------------------------------------------------------------------
// small device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" : : "l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ uint8_t ld_relaxed_u8(const uint8_t* p) {
    uint16_t v;
    asm volatile("ld.relaxed.gpu.global.u8 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
    return (uint8_t)v;
}
// Programmatic dependent launch: a kernel launched with programmatic stream
// serialisation may start before the previous kernel on its stream has
// finished; grid_dependency_wait() blocks until that kernel has completed and
// its writes are visible (a no-op for an ordinary launch).  The previous kernel
// lets it start early with grid_dependents_launch().
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dependents_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }

__device__ __forceinline__ void set_status(unsigned* st, unsigned bit) {
    if (st) atomicOr(st, bit);
}

// Poll *p (acquire) until it reaches `need`, sleeping between polls.  After
// `limit` polls give up: record kStatTimeout in *status and return false, so
// the caller can leave its kernel instead of hanging the GPU.
__device__ __forceinline__ bool bounded_wait_geq(const unsigned* p, unsigned need, unsigned limit,
                                                 unsigned* status) {
    unsigned it = 0;
    while (ld_acquire_u32(p) < need) {
        if (++it > limit) {
            set_status(status, kStatTimeout);
            return false;
        }
        __nanosleep(100);
    }
    return true;
}

// makes `dev` current for the scope of a call and restores the caller's device
struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};

inline unsigned grid_for(int64_t n, int threads, int64_t cap = 1 << 30) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (unsigned)b;
}

}  // namespace mg
