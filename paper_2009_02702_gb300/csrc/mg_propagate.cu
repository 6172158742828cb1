// mg_propagate.cu -- forward transfer-function propagation (Sec. 3.4, Sec. 4).
//
// Sources take the TF row of their segment; then, level by level (nodes of a
// level are contiguous and independent), every node lerps the rows of its two
// predecessors:  v = v_p + alpha * (v_q - v_p), fp32.  Node records are SoA:
// (p, q) as one 8-byte load, alpha as 4 (or 2) bytes; value rows are gathered
// as one vector load per predecessor.
//
// One persistent launch covers all levels: CTAs take tiles of nodes from a
// global ticket in level order, and a tile of level d first waits until every
// tile of level d-1 has signalled (a per-level counter).  Tiles are handed out
// in order, so every tile waited on belongs to a CTA that is already running:
// the wait always ends.  It is bounded all the same; past the bound the
// kernel records MG_ERR_TIMEOUT and returns.  Rows written in this launch are
// read through L2 (ld.global.cg), never through the read-only cache.
#include "mg_internal.cuh"

#include <algorithm>

namespace mg {
namespace {

template <typename T> struct Cvt;
template <> struct Cvt<float> {
    static __device__ __forceinline__ float to(float x) { return x; }
    static __device__ __forceinline__ float from(float x) { return x; }
};
template <> struct Cvt<__half> {
    static __device__ __forceinline__ float to(__half x) { return __half2float(x); }
    static __device__ __forceinline__ __half from(float x) { return __float2half_rn(x); }
};
template <> struct Cvt<__nv_bfloat16> {
    static __device__ __forceinline__ float to(__nv_bfloat16 x) { return __bfloat162float(x); }
    static __device__ __forceinline__ __nv_bfloat16 from(float x) { return __float2bfloat16_rn(x); }
};

// load / store one row of C values: as 16-byte vectors when the row is a
// multiple of 16 bytes, 8-byte ones when it is a multiple of 8, else element
// by element.  kL2 loads go through L2 only (rows written earlier in the same
// launch are never read through the read-only cache).
template <bool kL2, typename V>
__device__ __forceinline__ V ld_vec(const V* p) {
    if constexpr (kL2) return __ldcg(p);
    else return __ldg(p);
}

template <typename ST, int C, bool kL2>
__device__ __forceinline__ void load_row_t(const ST* __restrict__ base, int64_t row, float (&v)[C]) {
    const ST* r = base + row * C;
    constexpr int B = (int)sizeof(ST) * C;
    if constexpr (B % 16 == 0) {
        constexpr int E = 16 / (int)sizeof(ST);
#pragma unroll
        for (int w = 0; w < B / 16; w++) {
            const uint4 u = ld_vec<kL2>(reinterpret_cast<const uint4*>(r) + w);
            const ST* e = reinterpret_cast<const ST*>(&u);
#pragma unroll
            for (int c = 0; c < E; c++) v[w * E + c] = Cvt<ST>::to(e[c]);
        }
    } else if constexpr (B % 8 == 0) {
        constexpr int E = 8 / (int)sizeof(ST);
#pragma unroll
        for (int w = 0; w < B / 8; w++) {
            const uint2 u = ld_vec<kL2>(reinterpret_cast<const uint2*>(r) + w);
            const ST* e = reinterpret_cast<const ST*>(&u);
#pragma unroll
            for (int c = 0; c < E; c++) v[w * E + c] = Cvt<ST>::to(e[c]);
        }
    } else if constexpr (sizeof(ST) == 4) {
#pragma unroll
        for (int c = 0; c < C; c++) v[c] = ld_vec<kL2>(reinterpret_cast<const float*>(r) + c);
    } else {
#pragma unroll
        for (int c = 0; c < C; c++) {
            const unsigned short u = ld_vec<kL2>(reinterpret_cast<const unsigned short*>(r) + c);
            v[c] = Cvt<ST>::to(*reinterpret_cast<const ST*>(&u));
        }
    }
}

template <typename ST, int C>
__device__ __forceinline__ void load_row(const ST* __restrict__ base, int64_t row, float (&v)[C]) {
    load_row_t<ST, C, false>(base, row, v);
}

template <typename ST, int C>
__device__ __forceinline__ void load_row_cg(const ST* __restrict__ base, int64_t row, float (&v)[C]) {
    load_row_t<ST, C, true>(base, row, v);
}

template <typename ST, int C>
__device__ __forceinline__ void store_row(ST* __restrict__ base, int64_t row, const float (&v)[C]) {
    ST* r = base + row * C;
    constexpr int B = (int)sizeof(ST) * C;
    if constexpr (B % 16 == 0 || B % 8 == 0) {
        constexpr int VB = B % 16 == 0 ? 16 : 8;
        constexpr int E = VB / (int)sizeof(ST);
#pragma unroll
        for (int w = 0; w < B / VB; w++) {
            ST e[E];
#pragma unroll
            for (int c = 0; c < E; c++) e[c] = Cvt<ST>::from(v[w * E + c]);
            if constexpr (VB == 16)
                reinterpret_cast<uint4*>(r)[w] = *reinterpret_cast<const uint4*>(e);
            else
                reinterpret_cast<uint2*>(r)[w] = *reinterpret_cast<const uint2*>(e);
        }
    } else {
#pragma unroll
        for (int c = 0; c < C; c++) r[c] = Cvt<ST>::from(v[c]);
    }
}

// channel c of source n: k transfer functions of cin channels each, TF j at
// tf + j * S * cin (k = 1: the row-major S x C table)
__device__ __forceinline__ float tf_value(const float* __restrict__ tf, int64_t n, int c, int cin, int64_t tf_stride) {
    return tf[(int64_t)(c / cin) * tf_stride + n * cin + (c % cin)];
}

template <typename ST, int C>
__global__ void sources_kernel(const float* __restrict__ tf, uint32_t S, int cin, ST* __restrict__ vals) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        float v[C];
#pragma unroll
        for (int c = 0; c < C; c++) v[c] = tf_value(tf, s, c, cin, (int64_t)S * cin);
        store_row<ST, C>(vals, s, v);
    }
}

// node weight: fp32 alpha, or a signed 16-bit alpha whose sign says p and q
// are swapped (alpha <= 1/2 after the swap; interpolation symmetry, Sec. 3.7)
template <typename ST> struct Weight {
    using T = ST;
};
template <> struct Weight<float> {
    using T = float;
};

template <typename ST, int C>
__global__ void level_kernel(const uint2* __restrict__ pq, const typename Weight<ST>::T* __restrict__ alpha,
                             int64_t lo, int64_t hi, ST* __restrict__ vals) {
    const int64_t n = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= hi) return;
    const uint2 e = __ldg(pq + n);
    uint32_t p = e.x, q = e.y;
    float al = Cvt<typename Weight<ST>::T>::to(alpha[n]);
    if (al < 0.f) {
        al = -al;
        const uint32_t t = p;
        p = q;
        q = t;
    }
    float vp[C], vq[C], out[C];
    load_row<ST, C>(vals, p, vp);
    load_row<ST, C>(vals, q, vq);
#pragma unroll
    for (int c = 0; c < C; c++) out[c] = fmaf(al, vq[c] - vp[c], vp[c]);
    store_row<ST, C>(vals, n, out);
}

constexpr int kPropThreads = 256;
constexpr int kPropTile = 1024;                 // nodes per tile
constexpr unsigned kSpinLimit = 1u << 22;       // polls before a wait gives up

struct PropTiles {
    int levels;                                 // D + 1, level 0 = the sources
    int64_t tile0[MG_MAX_DEPTH + 2];            // first tile of every level (+ end)
    int64_t first[MG_MAX_DEPTH + 1];            // first node of every level
    int64_t count[MG_MAX_DEPTH + 1];            // nodes of every level
};

// level of tile t (tile0: first tile of every level)
__device__ __forceinline__ int tile_level(const PropTiles& T, long long t) {
    int d = 0;
    while (t >= T.tile0[d + 1]) d++;
    return d;
}

// this thread's edges and weights of tile t: nodes lo + threadIdx.x + k * kPropThreads
template <typename ST, int NT>
__device__ __forceinline__ void tile_edges(const PropTiles& T, long long t, long long total,
                                           const uint2* __restrict__ pq,
                                           const typename Weight<ST>::T* __restrict__ alpha, uint2 (&e)[NT],
                                           float (&al)[NT]) {
#pragma unroll
    for (int k = 0; k < NT; k++) {
        e[k] = make_uint2(0u, 0u);
        al[k] = 0.f;
    }
    if (t >= total) return;
    const int d = tile_level(T, t);
    if (d == 0) return;
    const int64_t lo = T.first[d] + (t - T.tile0[d]) * kPropTile;
    const int64_t hi = min(lo + kPropTile, T.first[d] + T.count[d]);
#pragma unroll
    for (int k = 0; k < NT; k++) {
        const int64_t n = lo + threadIdx.x + (int64_t)k * kPropThreads;
        if (n < hi) {
            e[k] = __ldg(pq + n);
            al[k] = Cvt<typename Weight<ST>::T>::to(alpha[n]);
        }
    }
}

template <typename ST, int C>
__global__ void __launch_bounds__(kPropThreads) single_pass_kernel(PropTiles T, const uint2* __restrict__ pq,
                                                                   const typename Weight<ST>::T* __restrict__ alpha,
                                                                   const float* __restrict__ tf, int cin,
                                                                   ST* __restrict__ vals, unsigned* __restrict__ done,
                                                                   unsigned long long* __restrict__ ticket,
                                                                   unsigned* __restrict__ status) {
    constexpr int NT = kPropTile / kPropThreads;      // nodes of a tile per thread
    constexpr int NPT = C <= 4 ? 4 : C <= 8 ? 2 : 1;  // of them gathered at once
    __shared__ long long s_next;
    __shared__ int s_abort;
    const long long total = T.tile0[T.levels];
    // thread 0 holds the ticket after next, taken two tiles ahead so that the
    // atomic's round trip is never waited on
    long long ahead = 0;
    int seen = 0;   // thread 0: every level below this one is known to be complete
    if (threadIdx.x == 0) {
        s_next = (long long)atomicAdd(ticket, 1ull);
        ahead = (long long)atomicAdd(ticket, 1ull);
    }
    __syncthreads();
    long long t = s_next;
    // Software pipeline over tiles: the next tile's ticket is known and its
    // (static) edges and weights are loaded while this tile waits and runs.
    // Tickets are taken in order and a tile only waits for smaller ones, so
    // the smallest unfinished ticket is always some CTA's current tile.
    uint2 e[NT];
    float al[NT];
    tile_edges<ST, NT>(T, t, total, pq, alpha, e, al);
    while (t < total) {
        const int d = tile_level(T, t);
        const int64_t lo = T.first[d] + (t - T.tile0[d]) * kPropTile;
        const int64_t hi = min(lo + kPropTile, T.first[d] + T.count[d]);
        __syncthreads();   // every thread has read s_next
        if (threadIdx.x == 0) {
            s_next = ahead;
            ahead = (long long)atomicAdd(ticket, 1ull);
            s_abort = 0;
            if (d > seen) {   // level d-1 not yet seen complete
                const unsigned need = (unsigned)(T.tile0[d] - T.tile0[d - 1]);
                if (bounded_wait_geq(done + d - 1, need, kSpinLimit, status)) seen = d;
                else s_abort = 1;
            }
        }
        __syncthreads();
        if (s_abort) break;
        const long long tn = s_next;
        uint2 en[NT];
        float aln[NT];
        tile_edges<ST, NT>(T, tn, total, pq, alpha, en, aln);
        if (d == 0) {
            for (int64_t n = lo + threadIdx.x; n < hi; n += kPropThreads) {
                float out[C];
#pragma unroll
                for (int c = 0; c < C; c++) out[c] = tf_value(tf, n, c, cin, T.count[0] * cin);
                store_row<ST, C>(vals, n, out);
            }
        } else {
            // NPT nodes at a time: both predecessor rows of every node are
            // loaded before any is stored (nodes of one level never read each other)
#pragma unroll
            for (int k0 = 0; k0 < NT; k0 += NPT) {
                float vp[NPT][C], vq[NPT][C];
#pragma unroll
                for (int k = 0; k < NPT; k++) {
                    const int64_t n = lo + threadIdx.x + (int64_t)(k0 + k) * kPropThreads;
                    if (n < hi) {
                        uint32_t p = e[k0 + k].x, q = e[k0 + k].y;
                        if (al[k0 + k] < 0.f) {   // 16-bit weights: sign = p and q swapped
                            p = e[k0 + k].y;
                            q = e[k0 + k].x;
                        }
                        load_row_cg<ST, C>(vals, p, vp[k]);
                        load_row_cg<ST, C>(vals, q, vq[k]);
                    }
                }
#pragma unroll
                for (int k = 0; k < NPT; k++) {
                    const int64_t n = lo + threadIdx.x + (int64_t)(k0 + k) * kPropThreads;
                    if (n < hi) {
                        const float a = fabsf(al[k0 + k]);
                        float out[C];
#pragma unroll
                        for (int c = 0; c < C; c++) out[c] = fmaf(a, vq[k][c] - vp[k][c], vp[k][c]);
                        store_row<ST, C>(vals, n, out);
                    }
                }
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(done + d, 1u);
        }
        t = tn;
#pragma unroll
        for (int k = 0; k < NT; k++) {
            e[k] = en[k];
            al[k] = aln[k];
        }
    }
}

__global__ void alpha16_kernel(const ulonglong2* __restrict__ ab, int64_t N, uint32_t S, int bf16,
                               void* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (i >= (int64_t)S) {
            const ulonglong2 w = ab[i];
            const double s = (double)w.x + (double)w.y;
            // alpha = b/(a+b); above 1/2 store -(a/(a+b)) meaning "swap p and q"
            v = (w.y <= w.x) ? (float)((double)w.y / s) : -(float)((double)w.x / s);
        }
        if (bf16)
            static_cast<__nv_bfloat16*>(out)[i] = __float2bfloat16_rn(v);
        else
            static_cast<__half*>(out)[i] = __float2half_rn(v);
    }
}

// the same from fp32 weights (quantised graphs: no exact a, b)
__global__ void alpha16_from_f32_kernel(const float* __restrict__ alpha, int64_t N, uint32_t S, int bf16,
                                        void* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        float v = 0.f;
        if (i >= (int64_t)S) {
            const float w = alpha[i];
            v = w <= 0.5f ? w : -(1.0f - w);
        }
        if (bf16)
            static_cast<__nv_bfloat16*>(out)[i] = __float2bfloat16_rn(v);
        else
            static_cast<__half*>(out)[i] = __float2half_rn(v);
    }
}

int sm_count_prop(int dev) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

template <typename ST, int C>
mg_status run_single_pass(mg_graph* g, const float* tf, int cin, const void* alpha, ST* vals, cudaStream_t s) {
    PropTiles T;
    T.levels = g->D + 1;
    int64_t tiles = 0;
    for (int d = 0; d <= g->D; d++) {
        T.tile0[d] = tiles;
        T.first[d] = g->bucket[d];
        T.count[d] = g->bucket[d + 1] - g->bucket[d];
        tiles += (T.count[d] + kPropTile - 1) / kPropTile;
    }
    T.tile0[g->D + 1] = tiles;
    Arena* arena = nullptr;
    MG_TRY(arena_begin(g, s, &arena));
    Buf sync;
    MG_TRY(sync.alloc(&arena->view, (MG_MAX_DEPTH + 2) * sizeof(unsigned) + 16, s));
    MG_CUDA(cudaMemsetAsync(sync.p, 0, (MG_MAX_DEPTH + 2) * sizeof(unsigned) + 16, s));
    unsigned* done = sync.as<unsigned>();
    auto* ticket = reinterpret_cast<unsigned long long*>(sync.as<unsigned char>() + (MG_MAX_DEPTH + 2) * sizeof(unsigned) +
                                                        (8 - ((MG_MAX_DEPTH + 2) * sizeof(unsigned)) % 8) % 8);
    using W = typename Weight<ST>::T;
    auto k = single_pass_kernel<ST, C>;
    int per_sm = 0;
    MG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kPropThreads, 0));
    const int64_t grid = std::min<int64_t>(tiles, (int64_t)std::max(per_sm, 1) * sm_count_prop(g->device));
    k<<<(unsigned)std::max<int64_t>(grid, 1), kPropThreads, 0, s>>>(T, g->pq.as<uint2>(), static_cast<const W*>(alpha),
                                                                    tf, cin, vals, done, ticket,
                                                                    g->status.as<unsigned>());
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

template <typename ST, int C>
mg_status run(mg_graph* g, const float* tf, int cin, const void* alpha, ST* vals, cudaStream_t s) {
    if (g->D + 1 <= MG_MAX_DEPTH) return run_single_pass<ST, C>(g, tf, cin, alpha, vals, s);
    sources_kernel<ST, C><<<grid_for(g->S, 256, 152 * 16), 256, 0, s>>>(tf, g->S, cin, vals);
    MG_CUDA(cudaGetLastError());
    using W = typename Weight<ST>::T;
    for (int d = 1; d <= g->D; d++) {
        const int64_t lo = g->bucket[d], hi = g->bucket[d + 1];
        if (hi <= lo) continue;
        level_kernel<ST, C><<<grid_for(hi - lo, 256), 256, 0, s>>>(g->pq.as<uint2>(), static_cast<const W*>(alpha),
                                                                   lo, hi, vals);
        MG_CUDA(cudaGetLastError());
    }
    return MG_OK;
}

template <typename ST>
mg_status dispatch_c(mg_graph* g, const float* tf, int C, int cin, const void* alpha, void* vals, cudaStream_t s) {
    ST* v = static_cast<ST*>(vals);
    switch (C) {
        case 1: return run<ST, 1>(g, tf, cin, alpha, v, s);
        case 2: return run<ST, 2>(g, tf, cin, alpha, v, s);
        case 3: return run<ST, 3>(g, tf, cin, alpha, v, s);
        case 4: return run<ST, 4>(g, tf, cin, alpha, v, s);
        case 5: return run<ST, 5>(g, tf, cin, alpha, v, s);
        case 6: return run<ST, 6>(g, tf, cin, alpha, v, s);
        case 7: return run<ST, 7>(g, tf, cin, alpha, v, s);
        case 8: return run<ST, 8>(g, tf, cin, alpha, v, s);
        case 12: return run<ST, 12>(g, tf, cin, alpha, v, s);
        case 16: return run<ST, 16>(g, tf, cin, alpha, v, s);
        case 20: return run<ST, 20>(g, tf, cin, alpha, v, s);
        case 24: return run<ST, 24>(g, tf, cin, alpha, v, s);
        case 28: return run<ST, 28>(g, tf, cin, alpha, v, s);
        case 32: return run<ST, 32>(g, tf, cin, alpha, v, s);
        default: break;
    }
    return fail(MG_ERR_UNSUPPORTED, "channels per node (k * C) must be 1-8, 12, 16, 20, 24, 28 or 32");
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

mg_status ensure_alpha16(mg_graph* g, mg_dtype dt, cudaStream_t s) {
    Buf& b = dt == MG_BF16 ? g->alphab16 : g->alpha16;
    if (b.p) return MG_OK;
    MG_TRY(b.alloc(&g->al, (size_t)g->N * 2, s));
    if (g->quantised)
        alpha16_from_f32_kernel<<<grid_for(g->N, 256, 152 * 32), 256, 0, s>>>(g->alpha.as<float>(), g->N, g->S,
                                                                              dt == MG_BF16, b.p);
    else
        alpha16_kernel<<<grid_for(g->N, 256, 152 * 32), 256, 0, s>>>(g->ab.as<ulonglong2>(), g->N, g->S,
                                                                    dt == MG_BF16, b.p);
    MG_CUDA(cudaGetLastError());
    MG_CUDA(cudaStreamSynchronize(s));
    b.s = nullptr;
    return MG_OK;
}

// ---------------------------------------------------------------------------
// Self-test of the bounded wait: one thread waits, with the propagation's
// helper, on a word that is either already set or that nothing ever sets.
// ---------------------------------------------------------------------------
namespace {
__device__ unsigned g_selftest_words[2];   // [0] the awaited flag, [1] the status word

__global__ void selftest_wait_kernel(unsigned limit) {
    if (threadIdx.x == 0 && blockIdx.x == 0) bounded_wait_geq(&g_selftest_words[0], 1u, limit, &g_selftest_words[1]);
}
}  // namespace

mg_status selftest_wait(bool satisfied, unsigned limit, cudaStream_t s) {
    const unsigned init[2] = {satisfied ? 1u : 0u, 0u};
    MG_CUDA(cudaMemcpyToSymbolAsync(g_selftest_words, init, sizeof(init), 0, cudaMemcpyHostToDevice, s));
    selftest_wait_kernel<<<1, 32, 0, s>>>(limit);
    MG_CUDA(cudaGetLastError());
    unsigned words[2] = {0, 0};
    MG_CUDA(cudaMemcpyFromSymbolAsync(words, g_selftest_words, sizeof(words), 0, cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    return status_from_bits(words[1]);
}

mg_status propagate_multi(mg_graph* g, const float* tf, int k, int C, mg_dtype storage, void* vals, cudaStream_t s) {
    const int CT = k * C;
    const size_t esz = storage == MG_F32 ? 4 : 2;
    const size_t row = esz * (size_t)CT;
    if (row % 16 == 0 ? !aligned(vals, 16) : row % 8 == 0 ? !aligned(vals, 8) : false)
        return fail(MG_ERR_INVALID_ARG, "vals must be aligned to 16 bytes (rows of a multiple of 16 bytes) or 8");
    if (storage == MG_F32) return dispatch_c<float>(g, tf, CT, C, g->alpha.p, vals, s);
    MG_TRY(ensure_alpha16(g, storage, s));
    if (storage == MG_F16) return dispatch_c<__half>(g, tf, CT, C, g->alpha16.p, vals, s);
    return dispatch_c<__nv_bfloat16>(g, tf, CT, C, g->alphab16.p, vals, s);
}

mg_status propagate(mg_graph* g, const float* tf, int C, mg_dtype storage, void* vals, cudaStream_t s) {
    return propagate_multi(g, tf, 1, C, storage, vals, s);
}

}  // namespace mg
