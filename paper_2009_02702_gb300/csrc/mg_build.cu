// mg_build.cu -- Mixture Graph construction on the GPU.
//
//  A1  Sec. 3.1, Eq. 4: normalised histogram mipmap.  Each level is a CSR of
//      (segment id, integer weight) lists, weight = 8^l * H; a parent's list is
//      the merge of its <= 8 children's lists scaled by 8/N, N the children in
//      support (1, 2, 4 or 8).  Count pass, scan, write pass per level.
//  A2  Sec. 3.2-3.3, Eq. 5-7: every list longer than one entry is factorised
//      into binary lerps, pairing positions (0,1),(2,3),... per round with an
//      odd last entry carried.  A lerp is the key (p, q, a, b) with a:b the
//      reduced weight ratio; a global open-addressing hash returns the existing
//      node for a key or publishes a new one (lock-free: the node row is written
//      first, then its index is CAS-ed into the slot).
//  A3  Sec. 3.4, Fig. 5: topological level = max(level of p, level of q) + 1;
//      nodes are renumbered in ascending (level, p', q', a, b) with p', q' the
//      new IDs of the predecessors, by a stable radix sort per level; bucket
//      offsets delimit the levels; mip IDs are rewritten.
#include "mg_internal.cuh"

#include <algorithm>
#include <vector>

namespace mg {
namespace {

struct Dims3 {
    int32_t x, y, z;
};

__host__ __device__ __forceinline__ int64_t nvox(Dims3 d) { return (int64_t)d.x * d.y * d.z; }

// ---------------------------------------------------------------------------
// level 0 checks and copy
// ---------------------------------------------------------------------------
template <typename IdT, typename OutT>
__global__ void copy_ids_kernel(const IdT* __restrict__ in, OutT* __restrict__ out, int64_t n, uint32_t S,
                                unsigned* __restrict__ status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t v = (uint32_t)in[i];
        if (v >= S) {
            set_status(status, kStatBadInput);
            v = 0;
        }
        out[i] = (OutT)v;
    }
}

// ---------------------------------------------------------------------------
// A1: level 0 -> level 1 (sort <= 8 IDs per parent)
// ---------------------------------------------------------------------------
template <typename IdT>
__device__ __forceinline__ int gather_l0(const IdT* __restrict__ ids, Dims3 d0, int X, int Y, int Z, uint32_t v[8]) {
    int n = 0;
#pragma unroll
    for (int k = 0; k < 2; k++)
#pragma unroll
        for (int j = 0; j < 2; j++)
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int x = 2 * X + i, y = 2 * Y + j, z = 2 * Z + k;
                if (x < d0.x && y < d0.y && z < d0.z) v[n++] = (uint32_t)ids[((int64_t)z * d0.y + y) * d0.x + x];
            }
    // insertion sort, at most 8 elements
    for (int a = 1; a < n; a++) {
        uint32_t t = v[a];
        int b = a - 1;
        while (b >= 0 && v[b] > t) {
            v[b + 1] = v[b];
            b--;
        }
        v[b + 1] = t;
    }
    return n;
}

template <typename IdT>
__global__ void l1_count_kernel(const IdT* __restrict__ ids, Dims3 d0, Dims3 d1, uint32_t* __restrict__ nnz) {
    const int64_t V1 = nvox(d1);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V1; v += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(v % d1.x), Y = (int)((v / d1.x) % d1.y), Z = (int)(v / ((int64_t)d1.x * d1.y));
        uint32_t s[8];
        const int n = gather_l0(ids, d0, X, Y, Z, s);
        uint32_t c = 1;
        for (int a = 1; a < n; a++) c += s[a] != s[a - 1];
        nnz[v] = c;
    }
}

template <typename IdT>
__global__ void l1_write_kernel(const IdT* __restrict__ ids, Dims3 d0, Dims3 d1, const uint32_t* __restrict__ off,
                                uint32_t* __restrict__ out_ids, uint64_t* __restrict__ out_w) {
    const int64_t V1 = nvox(d1);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V1; v += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(v % d1.x), Y = (int)((v / d1.x) % d1.y), Z = (int)(v / ((int64_t)d1.x * d1.y));
        uint32_t s[8];
        const int n = gather_l0(ids, d0, X, Y, Z, s);
        const uint64_t scale = 8u / (unsigned)n;   // Eq. 4: divide by N, times 8^l
        uint32_t o = off[v];
        uint32_t run = 1;
        for (int a = 1; a <= n; a++) {
            if (a < n && s[a] == s[a - 1]) {
                run++;
                continue;
            }
            out_ids[o] = s[a - 1];
            out_w[o] = (uint64_t)run * scale;
            o++;
            run = 1;
        }
    }
}

// ---------------------------------------------------------------------------
// A1: level l -> level l+1 (merge <= 8 sorted child lists)
// ---------------------------------------------------------------------------
struct Heads {
    uint32_t pos[8], end[8], head[8];
    int n;
};

__device__ __forceinline__ void load_children(const uint32_t* __restrict__ off, const uint32_t* __restrict__ ids,
                                              Dims3 dl, int X, int Y, int Z, Heads& h) {
    h.n = 0;
#pragma unroll
    for (int k = 0; k < 2; k++)
#pragma unroll
        for (int j = 0; j < 2; j++)
#pragma unroll
            for (int i = 0; i < 2; i++) {
                const int x = 2 * X + i, y = 2 * Y + j, z = 2 * Z + k;
                const int c = 4 * k + 2 * j + i;
                if (x < dl.x && y < dl.y && z < dl.z) {
                    const int64_t cv = ((int64_t)z * dl.y + y) * dl.x + x;
                    h.pos[c] = off[cv];
                    h.end[c] = off[cv + 1];
                    h.n++;
                } else {
                    h.pos[c] = 0;
                    h.end[c] = 0;
                }
                h.head[c] = h.pos[c] < h.end[c] ? ids[h.pos[c]] : kNone;
            }
}

__device__ __forceinline__ uint32_t heads_min(const Heads& h) {
    uint32_t m = kNone;
#pragma unroll
    for (int c = 0; c < 8; c++) m = min(m, h.head[c]);
    return m;
}

__global__ void next_count_kernel(const uint32_t* __restrict__ off, const uint32_t* __restrict__ ids, Dims3 dl,
                                  Dims3 dn, uint32_t* __restrict__ nnz) {
    const int64_t Vn = nvox(dn);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < Vn; v += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(v % dn.x), Y = (int)((v / dn.x) % dn.y), Z = (int)(v / ((int64_t)dn.x * dn.y));
        Heads h;
        load_children(off, ids, dl, X, Y, Z, h);
        uint32_t cnt = 0;
        for (;;) {
            const uint32_t m = heads_min(h);
            if (m == kNone) break;
            cnt++;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                if (h.head[c] == m) {
                    h.pos[c]++;
                    h.head[c] = h.pos[c] < h.end[c] ? ids[h.pos[c]] : kNone;
                }
            }
        }
        nnz[v] = cnt;
    }
}

__global__ void next_write_kernel(const uint32_t* __restrict__ off, const uint32_t* __restrict__ ids,
                                  const uint64_t* __restrict__ w, Dims3 dl, Dims3 dn,
                                  const uint32_t* __restrict__ noff, uint32_t* __restrict__ nids,
                                  uint64_t* __restrict__ nw) {
    const int64_t Vn = nvox(dn);
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < Vn; v += (int64_t)gridDim.x * blockDim.x) {
        const int X = (int)(v % dn.x), Y = (int)((v / dn.x) % dn.y), Z = (int)(v / ((int64_t)dn.x * dn.y));
        Heads h;
        load_children(off, ids, dl, X, Y, Z, h);
        const uint64_t scale = 8u / (unsigned)h.n;   // Eq. 4
        uint32_t o = noff[v];
        for (;;) {
            const uint32_t m = heads_min(h);
            if (m == kNone) break;
            uint64_t sum = 0;
#pragma unroll
            for (int c = 0; c < 8; c++) {
                if (h.head[c] == m) {
                    sum += w[h.pos[c]];
                    h.pos[c]++;
                    h.head[c] = h.pos[c] < h.end[c] ? ids[h.pos[c]] : kNone;
                }
            }
            nids[o] = m;
            nw[o] = sum * scale;
            o++;
        }
    }
}

// ---------------------------------------------------------------------------
// A2: node table with lock-free hash pruning
// ---------------------------------------------------------------------------
struct NodeTab {
    uint32_t* p;
    uint32_t* q;
    uint64_t* a;
    uint64_t* b;
    uint8_t* depth;
    uint32_t* slots;       // node index or kNone
    uint64_t mask;         // slots - 1
    unsigned long long* count;
    uint64_t cap;
    unsigned* status;
};

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
    x ^= x >> 31;
    x *= 0x7fb5d329728ea185ull;
    x ^= x >> 27;
    x *= 0x81dadef4bc2dd44dull;
    x ^= x >> 33;
    return x;
}

__device__ __forceinline__ uint64_t key_hash(uint32_t p, uint32_t q, uint64_t a, uint64_t b) {
    return mix64(mix64(((uint64_t)p << 32 | q) ^ 0x9e3779b97f4a7c15ull) ^ a * 0xc2b2ae3d27d4eb4full ^
                 (b + 0x165667b19e3779f9ull) * 0x27d4eb2f165667c5ull);
}

__device__ __forceinline__ uint64_t gcd64(uint64_t u, uint64_t v) {
    if (u == 0) return v;
    if (v == 0) return u;
    const int shift = __ffsll((long long)(u | v)) - 1;
    u >>= __ffsll((long long)u) - 1;
    do {
        v >>= __ffsll((long long)v) - 1;
        if (u > v) {
            uint64_t t = u;
            u = v;
            v = t;
        }
        v -= u;
    } while (v);
    return u << shift;
}

// Eq. 5-6 with Sec. 3.3 re-use: node for the lerp of (p, wp) and (q, wq).
__device__ uint32_t node_get(const NodeTab& t, uint32_t p, uint32_t q, uint64_t wp, uint64_t wq) {
    if (p >= kDead || q >= kDead) return kNone;   // an earlier failure propagates
    const uint64_t g = gcd64(wp, wq);
    const uint64_t a = wp / g, b = wq / g;
    uint64_t h = key_hash(p, q, a, b) & t.mask;
    uint32_t mine = kNone;
    for (uint64_t probe = 0; probe <= t.mask; probe++) {
        uint32_t s = ld_acquire_u32(t.slots + h);
        if (s == kNone) {
            if (mine == kNone) {
                const unsigned long long k = atomicAdd(t.count, 1ull);
                if (k >= t.cap) {
                    set_status(t.status, kStatCapacity);
                    return kNone;
                }
                mine = (uint32_t)k;
                t.p[mine] = p;
                t.q[mine] = q;
                t.a[mine] = a;
                t.b[mine] = b;
                // Sec. 3.4: topological level, the predecessors are complete
                const uint8_t dp = ld_relaxed_u8(t.depth + p), dq = ld_relaxed_u8(t.depth + q);
                t.depth[mine] = (uint8_t)(max(dp, dq) + 1);
                __threadfence();
            }
            const uint32_t old = atomicCAS(t.slots + h, kNone, mine);
            if (old == kNone) return mine;
            s = old;
            __threadfence();
        }
        if (ld_relaxed_u32(t.p + s) == p && ld_relaxed_u32(t.q + s) == q && ld_relaxed_u64(t.a + s) == a &&
            ld_relaxed_u64(t.b + s) == b) {
            if (mine != kNone) t.p[mine] = kDead;   // our unpublished row is never referenced
            return s;
        }
        h = (h + 1) & t.mask;
    }
    set_status(t.status, kStatCapacity);
    return kNone;
}

constexpr int kShortList = 16;

__global__ void factor_short_kernel(NodeTab t, const uint32_t* __restrict__ off, const uint32_t* __restrict__ ids,
                                    const uint64_t* __restrict__ w, int64_t V, uint32_t* __restrict__ mip_out,
                                    uint32_t* __restrict__ long_list, unsigned* __restrict__ long_count) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t b = off[v];
        int n = (int)(off[v + 1] - b);
        if (n == 1) {
            mip_out[v] = ids[b];
            continue;
        }
        if (n > kShortList) {
            const unsigned i = atomicAdd(long_count, 1u);
            long_list[i] = (uint32_t)v;
            continue;
        }
        uint32_t nd[kShortList];
        uint64_t ww[kShortList];
        for (int i = 0; i < n; i++) {
            nd[i] = ids[b + i];
            ww[i] = w[b + i];
        }
        while (n > 1) {
            int m = 0;
            for (int k = 0; k + 1 < n; k += 2) {
                const uint32_t r = node_get(t, nd[k], nd[k + 1], ww[k], ww[k + 1]);
                const uint64_t s = ww[k] + ww[k + 1];
                nd[m] = r;
                ww[m] = s;
                m++;
            }
            if (n & 1) {
                nd[m] = nd[n - 1];
                ww[m] = ww[n - 1];
                m++;
            }
            n = m;
        }
        mip_out[v] = nd[0];
    }
}

// One CTA per long list; rounds in place in the level's CSR arrays (all reads
// of a round's slice happen before its writes, separated by a barrier).
__global__ void factor_long_kernel(NodeTab t, const uint32_t* __restrict__ off, uint32_t* ids, uint64_t* w,
                                   const uint32_t* __restrict__ long_list, const unsigned* __restrict__ long_count,
                                   uint32_t* __restrict__ mip_out) {
    const unsigned nlong = *long_count;
    for (unsigned i = blockIdx.x; i < nlong; i += gridDim.x) {
        const uint32_t v = long_list[i];
        const uint32_t b = off[v];
        int64_t n = (int64_t)(off[v + 1] - b);
        uint32_t* nd = ids + b;
        uint64_t* ww = w + b;
        while (n > 1) {
            const int64_t half = n / 2;
            for (int64_t base = 0; base < half; base += blockDim.x) {
                const int64_t k = base + threadIdx.x;
                uint32_t n0 = 0, n1 = 0;
                uint64_t w0 = 0, w1 = 0;
                if (k < half) {
                    n0 = nd[2 * k];
                    n1 = nd[2 * k + 1];
                    w0 = ww[2 * k];
                    w1 = ww[2 * k + 1];
                }
                __syncthreads();
                if (k < half) {
                    nd[k] = node_get(t, n0, n1, w0, w1);
                    ww[k] = w0 + w1;
                }
                __syncthreads();
            }
            if (n & 1) {
                if (threadIdx.x == 0) {
                    nd[half] = nd[n - 1];
                    ww[half] = ww[n - 1];
                }
                __syncthreads();
            }
            n = (n + 1) / 2;
        }
        if (threadIdx.x == 0) mip_out[v] = nd[0];
        __syncthreads();
    }
}

__global__ void list_max_kernel(const uint32_t* __restrict__ off, int64_t V, unsigned* __restrict__ out) {
    unsigned m = 0;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x)
        m = max(m, off[v + 1] - off[v]);
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0 && m) atomicMax(out, m);
}

__global__ void rehash_kernel(NodeTab t, uint64_t lo, uint64_t hi) {
    for (uint64_t k = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < hi;
         k += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t p = t.p[k];
        if (p >= kDead) continue;
        uint64_t h = key_hash(p, t.q[k], t.a[k], t.b[k]) & t.mask;
        for (uint64_t probe = 0; probe <= t.mask; probe++) {
            if (atomicCAS(t.slots + h, kNone, (uint32_t)k) == kNone) break;
            h = (h + 1) & t.mask;
        }
    }
}

// ---------------------------------------------------------------------------
// A3: canonical relabel
// ---------------------------------------------------------------------------
__global__ void depth_hist_kernel(const uint32_t* __restrict__ p, const uint8_t* __restrict__ depth, uint64_t lo,
                                  uint64_t hi, unsigned long long* __restrict__ hist) {
    __shared__ unsigned int sh[MG_MAX_DEPTH + 1];
    for (int i = threadIdx.x; i <= MG_MAX_DEPTH; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    for (uint64_t k = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < hi;
         k += (uint64_t)gridDim.x * blockDim.x) {
        if (p[k] < kDead) atomicAdd(&sh[min((int)depth[k], MG_MAX_DEPTH)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i <= MG_MAX_DEPTH; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

__global__ void scatter_depth_kernel(const uint32_t* __restrict__ p, const uint8_t* __restrict__ depth, uint64_t lo,
                                     uint64_t hi, unsigned long long* __restrict__ cursor,
                                     uint32_t* __restrict__ order) {
    for (uint64_t k = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; k < hi;
         k += (uint64_t)gridDim.x * blockDim.x) {
        if (p[k] < kDead) {
            const unsigned long long pos = atomicAdd(&cursor[depth[k]], 1ull);
            order[pos] = (uint32_t)k;
        }
    }
}

// key for the stable sort: field 0 = b, 1 = a, 2 = a<<sh | b, 3 = p'<<sh | q'
__global__ void sort_key_kernel(const uint32_t* __restrict__ perm, int64_t n, int field, int sh,
                                const uint32_t* __restrict__ p, const uint32_t* __restrict__ q,
                                const uint64_t* __restrict__ a, const uint64_t* __restrict__ b,
                                const uint32_t* __restrict__ canon, uint64_t* __restrict__ keys) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = perm[i];
        uint64_t key;
        if (field == 0) key = b[k];
        else if (field == 1) key = a[k];
        else if (field == 2) key = a[k] << sh | b[k];
        else key = (uint64_t)canon[p[k]] << sh | canon[q[k]];
        keys[i] = key;
    }
}

__global__ void assign_kernel(const uint32_t* __restrict__ perm, int64_t n, uint32_t first,
                              const uint32_t* __restrict__ p, const uint32_t* __restrict__ q,
                              const uint64_t* __restrict__ a, const uint64_t* __restrict__ b,
                              uint32_t* __restrict__ canon, uint2* __restrict__ pq, ulonglong2* __restrict__ ab) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = perm[i];
        const uint32_t c = first + (uint32_t)i;
        canon[k] = c;
        pq[c] = make_uint2(canon[p[k]], canon[q[k]]);
        ab[c] = make_ulonglong2(a[k], b[k]);
    }
}

__global__ void sources_kernel(uint32_t S, uint32_t* __restrict__ canon, uint2* __restrict__ pq,
                               ulonglong2* __restrict__ ab) {
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < S; s += gridDim.x * blockDim.x) {
        canon[s] = s;
        pq[s] = make_uint2(kNone, kNone);
        ab[s] = make_ulonglong2(0, 0);
    }
}

__global__ void remap_kernel(uint32_t* __restrict__ mip, int64_t n, const uint32_t* __restrict__ canon,
                             unsigned* __restrict__ status) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t t = mip[i];
        if (t >= kDead) {
            set_status(status, kStatCapacity);
            mip[i] = 0;
        } else {
            mip[i] = canon[t];
        }
    }
}

__global__ void weights_kernel(const ulonglong2* __restrict__ ab, int64_t N, uint32_t S, uint2* __restrict__ ab32,
                               float* __restrict__ alpha) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        if (i < (int64_t)S) {
            ab32[i] = make_uint2(0, 0);
            alpha[i] = 0.f;
            continue;
        }
        const ulonglong2 w = ab[i];
        const uint64_t s = w.x + w.y;
        ab32[i] = s < (1ull << 32) ? make_uint2((uint32_t)w.x, (uint32_t)w.y) : make_uint2(0, 0);
        alpha[i] = (float)((double)w.y / (double)s);   // weight of q, rounded to fp32
    }
}

// ---------------------------------------------------------------------------
// axis-major copies: copy 0 orders (x, y, z), copy 1 (y, z, x), copy 2
// (z, x, y); rows of `pitch` IDs, the ones past the row's end set to 0
// ---------------------------------------------------------------------------
template <typename T>
__global__ void transpose_copy_kernel(const T* __restrict__ src, T* __restrict__ dst, Dims3 d, int copy,
                                      int64_t pitch) {
    const int32_t d0 = copy == 0 ? d.x : copy == 1 ? d.y : d.z;
    const int32_t d1 = copy == 0 ? d.y : copy == 1 ? d.z : d.x;
    const int32_t d2 = copy == 0 ? d.z : copy == 1 ? d.x : d.y;
    const int64_t n = pitch * d1 * d2;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = i % pitch, r = i / pitch;
        if (f >= d0) {
            dst[i] = T(0);
            continue;
        }
        const int64_t sc = r % d1, t = r / d1;
        int64_t x, y, z;
        if (copy == 0) {
            x = f; y = sc; z = t;
        } else if (copy == 1) {
            y = f; z = sc; x = t;
        } else {
            z = f; x = sc; y = t;
        }
        dst[i] = src[(z * d.y + y) * d.x + x];
    }
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
struct HostTable {
    Buf p, q, a, b, depth, slots;
    uint64_t cap = 0, nslots = 0;
    Buf count;   // unsigned long long
};

unsigned grid_n(int64_t n, int threads = 256) { return grid_for(n, threads, 152 * 64); }

mg_status grow_table(HostTable& t, uint64_t need, uint64_t used, const Alloc& al, cudaStream_t s) {
    if (need <= t.cap) return MG_OK;
    uint64_t ncap = std::max<uint64_t>(need, t.cap * 2);
    if (ncap >= (uint64_t)kDead) return fail(MG_ERR_UNSUPPORTED, "more than 2^32-2 nodes");
    Buf np, nq, na, nb, nd;
    MG_TRY(np.alloc(&al, ncap * 4, s));
    MG_TRY(nq.alloc(&al, ncap * 4, s));
    MG_TRY(na.alloc(&al, ncap * 8, s));
    MG_TRY(nb.alloc(&al, ncap * 8, s));
    MG_TRY(nd.alloc(&al, ncap, s));
    if (used) {
        MG_CUDA(cudaMemcpyAsync(np.p, t.p.p, used * 4, cudaMemcpyDeviceToDevice, s));
        MG_CUDA(cudaMemcpyAsync(nq.p, t.q.p, used * 4, cudaMemcpyDeviceToDevice, s));
        MG_CUDA(cudaMemcpyAsync(na.p, t.a.p, used * 8, cudaMemcpyDeviceToDevice, s));
        MG_CUDA(cudaMemcpyAsync(nb.p, t.b.p, used * 8, cudaMemcpyDeviceToDevice, s));
        MG_CUDA(cudaMemcpyAsync(nd.p, t.depth.p, used, cudaMemcpyDeviceToDevice, s));
    }
    t.p = std::move(np);
    t.q = std::move(nq);
    t.a = std::move(na);
    t.b = std::move(nb);
    t.depth = std::move(nd);
    t.cap = ncap;
    uint64_t ns = 1024;
    while (ns < 2 * ncap) ns <<= 1;
    if (ns != t.nslots) {
        MG_TRY(t.slots.alloc(&al, ns * 4, s));
        MG_CUDA(cudaMemsetAsync(t.slots.p, 0xFF, ns * 4, s));
        t.nslots = ns;
    }
    return MG_OK;
}

NodeTab view(HostTable& t, unsigned* status) {
    NodeTab v;
    v.p = t.p.as<uint32_t>();
    v.q = t.q.as<uint32_t>();
    v.a = t.a.as<uint64_t>();
    v.b = t.b.as<uint64_t>();
    v.depth = t.depth.as<uint8_t>();
    v.slots = t.slots.as<uint32_t>();
    v.mask = t.nslots - 1;
    v.count = t.count.as<unsigned long long>();
    v.cap = t.cap;
    v.status = status;
    return v;
}

template <typename T>
mg_status read_scalar(T* host, const void* dev, cudaStream_t s) {
    MG_CUDA(cudaMemcpyAsync(host, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    return MG_OK;
}

int bits_for(uint64_t maxval) {
    int b = 0;
    while (b < 64 && (maxval >> b)) b++;
    return b;
}

}  // namespace

mg_status build_graph(mg_graph* g, const void* ids, int id_bytes, int64_t nx, int64_t ny, int64_t nz,
                      cudaStream_t s) {
    const Alloc& al = g->al;
    const uint32_t S = g->S;
    LevelGeom& G = g->geom;

    // ---- Eq. 4 level geometry: round up until 1^3 ----
    int64_t d[3] = {nx, ny, nz};
    int L = 0;
    for (;;) {
        if (L >= MG_MAX_LEVELS) return fail(MG_ERR_UNSUPPORTED, "too many mip levels");
        for (int k = 0; k < 3; k++) G.dims[L][k] = (int32_t)d[k];
        L++;
        if (d[0] == 1 && d[1] == 1 && d[2] == 1) break;
        for (int k = 0; k < 3; k++) d[k] = (d[k] + 1) / 2;
    }
    G.L = g->L = L;
    auto dims_of = [&](int l) { return Dims3{G.dims[l][0], G.dims[l][1], G.dims[l][2]}; };
    int64_t total_hi = 0;
    G.off[0] = 0;
    for (int l = 1; l < L; l++) {
        G.off[l] = total_hi;
        total_hi += nvox(dims_of(l));
    }

    MG_TRY(g->status.alloc(&al, sizeof(unsigned), s));
    MG_CUDA(cudaMemsetAsync(g->status.p, 0, sizeof(unsigned), s));
    unsigned* status = g->status.as<unsigned>();

    // ---- level 0: the IDs themselves (lossless, Sec. 3.4) ----
    const int64_t V0 = nx * ny * nz;
    g->id0_bytes = S <= 65536u ? 2 : 4;
    MG_TRY(g->mip0.alloc(&al, (size_t)V0 * g->id0_bytes, s));
    {
        const unsigned gb = grid_n(V0);
        if (id_bytes == 2 && g->id0_bytes == 2)
            copy_ids_kernel<uint16_t, uint16_t><<<gb, 256, 0, s>>>((const uint16_t*)ids, g->mip0.as<uint16_t>(), V0, S, status);
        else if (id_bytes == 2)
            copy_ids_kernel<uint16_t, uint32_t><<<gb, 256, 0, s>>>((const uint16_t*)ids, g->mip0.as<uint32_t>(), V0, S, status);
        else if (g->id0_bytes == 2)
            copy_ids_kernel<uint32_t, uint16_t><<<gb, 256, 0, s>>>((const uint32_t*)ids, g->mip0.as<uint16_t>(), V0, S, status);
        else
            copy_ids_kernel<uint32_t, uint32_t><<<gb, 256, 0, s>>>((const uint32_t*)ids, g->mip0.as<uint32_t>(), V0, S, status);
        MG_CUDA(cudaGetLastError());
        unsigned bits = 0;
        MG_TRY(read_scalar(&bits, status, s));
        if (bits & kStatBadInput) return fail(MG_ERR_INVALID_ARG, "a segment ID is >= num_segments");
    }

    // ---- node table: sources 0..S-1 ----
    HostTable t;
    MG_TRY(t.count.alloc(&al, sizeof(unsigned long long), s));
    {
        unsigned long long c0 = S;
        MG_CUDA(cudaMemcpyAsync(t.count.p, &c0, sizeof(c0), cudaMemcpyHostToDevice, s));
    }
    MG_TRY(grow_table(t, (uint64_t)S + 4096, 0, al, s));
    MG_CUDA(cudaMemsetAsync(t.p.p, 0xFF, (size_t)S * 4, s));
    MG_CUDA(cudaMemsetAsync(t.q.p, 0xFF, (size_t)S * 4, s));
    MG_CUDA(cudaMemsetAsync(t.a.p, 0, (size_t)S * 8, s));
    MG_CUDA(cudaMemsetAsync(t.b.p, 0, (size_t)S * 8, s));
    MG_CUDA(cudaMemsetAsync(t.depth.p, 0, (size_t)S, s));
    uint64_t used = S;

    if (total_hi > 0) MG_TRY(g->mip.alloc(&al, (size_t)total_hi * 4, s));
    Buf maxlen;
    MG_TRY(maxlen.alloc(&al, sizeof(unsigned), s));
    MG_CUDA(cudaMemsetAsync(maxlen.p, 0, sizeof(unsigned), s));
    Buf long_list, long_count;
    MG_TRY(long_count.alloc(&al, sizeof(unsigned), s));

    // ---- A1 + A2, level by level ----
    struct Lists {
        Buf off, ids, w;
        int64_t V = 0;
        uint32_t nnz = 0;
    };
    auto make_level1 = [&](Lists& out) -> mg_status {
        const Dims3 d0 = dims_of(0), d1 = dims_of(1);
        out.V = nvox(d1);
        MG_TRY(out.off.alloc(&al, (size_t)(out.V + 1) * 4, s));
        const unsigned gb = grid_n(out.V);
        if (g->id0_bytes == 2)
            l1_count_kernel<uint16_t><<<gb, 256, 0, s>>>(g->mip0.as<uint16_t>(), d0, d1, out.off.as<uint32_t>());
        else
            l1_count_kernel<uint32_t><<<gb, 256, 0, s>>>(g->mip0.as<uint32_t>(), d0, d1, out.off.as<uint32_t>());
        MG_CUDA(cudaGetLastError());
        MG_TRY(scan_exclusive_u32(out.off.as<uint32_t>(), out.off.as<uint32_t>(), out.V,
                                  out.off.as<uint32_t>() + out.V, al, s));
        MG_TRY(read_scalar(&out.nnz, out.off.as<uint32_t>() + out.V, s));
        MG_TRY(out.ids.alloc(&al, (size_t)out.nnz * 4, s));
        MG_TRY(out.w.alloc(&al, (size_t)out.nnz * 8, s));
        if (g->id0_bytes == 2)
            l1_write_kernel<uint16_t><<<gb, 256, 0, s>>>(g->mip0.as<uint16_t>(), d0, d1, out.off.as<uint32_t>(),
                                                         out.ids.as<uint32_t>(), out.w.as<uint64_t>());
        else
            l1_write_kernel<uint32_t><<<gb, 256, 0, s>>>(g->mip0.as<uint32_t>(), d0, d1, out.off.as<uint32_t>(),
                                                         out.ids.as<uint32_t>(), out.w.as<uint64_t>());
        MG_CUDA(cudaGetLastError());
        return MG_OK;
    };
    auto make_next = [&](const Lists& in, int l, Lists& out) -> mg_status {
        const Dims3 dl = dims_of(l), dn = dims_of(l + 1);
        out.V = nvox(dn);
        MG_TRY(out.off.alloc(&al, (size_t)(out.V + 1) * 4, s));
        const unsigned gb = grid_n(out.V);
        next_count_kernel<<<gb, 256, 0, s>>>(in.off.as<uint32_t>(), in.ids.as<uint32_t>(), dl, dn,
                                             out.off.as<uint32_t>());
        MG_CUDA(cudaGetLastError());
        MG_TRY(scan_exclusive_u32(out.off.as<uint32_t>(), out.off.as<uint32_t>(), out.V,
                                  out.off.as<uint32_t>() + out.V, al, s));
        MG_TRY(read_scalar(&out.nnz, out.off.as<uint32_t>() + out.V, s));
        MG_TRY(out.ids.alloc(&al, (size_t)out.nnz * 4, s));
        MG_TRY(out.w.alloc(&al, (size_t)out.nnz * 8, s));
        next_write_kernel<<<gb, 256, 0, s>>>(in.off.as<uint32_t>(), in.ids.as<uint32_t>(), in.w.as<uint64_t>(), dl,
                                             dn, out.off.as<uint32_t>(), out.ids.as<uint32_t>(),
                                             out.w.as<uint64_t>());
        MG_CUDA(cudaGetLastError());
        return MG_OK;
    };

    int64_t max_list = 1;
    Lists cur;
    if (L > 1) MG_TRY(make_level1(cur));
    for (int l = 1; l < L; l++) {
        Lists nxt;
        if (l + 1 < L) MG_TRY(make_next(cur, l, nxt));
        // factorise level l (in place on cur)
        const uint64_t pairs = (uint64_t)cur.nnz - (uint64_t)cur.V;
        g->pairs += (int64_t)pairs;
        if (pairs > 0) {
            unsigned long long cnt = 0;
            MG_TRY(read_scalar(&cnt, t.count.p, s));
            used = cnt;
            const uint64_t old_slots = t.nslots;
            MG_TRY(grow_table(t, used + pairs, used, al, s));
            if (t.nslots != old_slots && used > S) {
                rehash_kernel<<<grid_n((int64_t)(used - S)), 256, 0, s>>>(view(t, status), S, used);
                MG_CUDA(cudaGetLastError());
            }
        }
        MG_CUDA(cudaMemsetAsync(long_count.p, 0, sizeof(unsigned), s));
        if (long_list.bytes < (size_t)cur.V * 4) MG_TRY(long_list.alloc(&al, (size_t)cur.V * 4, s));
        uint32_t* mip_out = g->mip.as<uint32_t>() + G.off[l];
        factor_short_kernel<<<grid_n(cur.V), 256, 0, s>>>(view(t, status), cur.off.as<uint32_t>(),
                                                          cur.ids.as<uint32_t>(), cur.w.as<uint64_t>(), cur.V,
                                                          mip_out, long_list.as<uint32_t>(),
                                                          long_count.as<unsigned>());
        MG_CUDA(cudaGetLastError());
        factor_long_kernel<<<152 * 4, 256, 0, s>>>(view(t, status), cur.off.as<uint32_t>(), cur.ids.as<uint32_t>(),
                                                   cur.w.as<uint64_t>(), long_list.as<uint32_t>(),
                                                   long_count.as<unsigned>(), mip_out);
        MG_CUDA(cudaGetLastError());
        // longest list of this level (statistics)
        list_max_kernel<<<grid_n(cur.V), 256, 0, s>>>(cur.off.as<uint32_t>(), cur.V, maxlen.as<unsigned>());
        MG_CUDA(cudaGetLastError());
        cur = std::move(nxt);
    }
    {
        unsigned long long cnt = 0;
        MG_TRY(read_scalar(&cnt, t.count.p, s));
        used = std::min<uint64_t>(cnt, t.cap);
        unsigned bits = 0;
        MG_TRY(read_scalar(&bits, status, s));
        if (bits & kStatCapacity) return fail(MG_ERR_CAPACITY, "node table overflow during factorisation");
    }
    {
        unsigned ml = 1;
        MG_TRY(read_scalar(&ml, maxlen.p, s));
        max_list = std::max<int64_t>(1, ml);
    }
    g->max_list = max_list;

    // ---- A3: topological levels and canonical numbering ----
    Buf hist;
    MG_TRY(hist.alloc(&al, (MG_MAX_DEPTH + 1) * sizeof(unsigned long long), s));
    MG_CUDA(cudaMemsetAsync(hist.p, 0, (MG_MAX_DEPTH + 1) * sizeof(unsigned long long), s));
    if (used > S) {
        depth_hist_kernel<<<grid_n((int64_t)(used - S)), 256, 0, s>>>(t.p.as<uint32_t>(), t.depth.as<uint8_t>(), S,
                                                                       used, hist.as<unsigned long long>());
        MG_CUDA(cudaGetLastError());
    }
    unsigned long long hh[MG_MAX_DEPTH + 1];
    MG_CUDA(cudaMemcpyAsync(hh, hist.p, sizeof(hh), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    if (hh[MG_MAX_DEPTH]) return fail(MG_ERR_UNSUPPORTED, "topological depth above the supported maximum");
    int D = 0;
    for (int k = 1; k < MG_MAX_DEPTH; k++)
        if (hh[k]) D = k;
    g->D = D;
    g->bucket[0] = 0;
    g->bucket[1] = S;
    for (int k = 1; k <= D; k++) g->bucket[k + 1] = g->bucket[k] + (int64_t)hh[k];
    const int64_t N = g->N = g->bucket[D + 1];
    const int64_t NI = N - S;

    MG_TRY(g->pq.alloc(&al, (size_t)N * sizeof(uint2), s));
    MG_TRY(g->ab.alloc(&al, (size_t)N * sizeof(ulonglong2), s));
    Buf canon;
    MG_TRY(canon.alloc(&al, (size_t)std::max<uint64_t>(used, 1) * 4, s));
    sources_kernel<<<grid_n(S), 256, 0, s>>>(S, canon.as<uint32_t>(), g->pq.as<uint2>(), g->ab.as<ulonglong2>());
    MG_CUDA(cudaGetLastError());
    if (NI > 0) {
        Buf order, cursor, keys;
        MG_TRY(order.alloc(&al, (size_t)NI * 4, s));
        MG_TRY(cursor.alloc(&al, (MG_MAX_DEPTH + 1) * sizeof(unsigned long long), s));
        MG_TRY(keys.alloc(&al, (size_t)NI * 8, s));
        unsigned long long hc[MG_MAX_DEPTH + 1] = {};
        for (int k = 1; k <= D; k++) hc[k] = (unsigned long long)(g->bucket[k] - S);
        MG_CUDA(cudaMemcpyAsync(cursor.p, hc, sizeof(hc), cudaMemcpyHostToDevice, s));
        scatter_depth_kernel<<<grid_n((int64_t)(used - S)), 256, 0, s>>>(t.p.as<uint32_t>(), t.depth.as<uint8_t>(), S,
                                                                          used, cursor.as<unsigned long long>(),
                                                                          order.as<uint32_t>());
        MG_CUDA(cudaGetLastError());
        const int bits_ab = std::max(1, 3 * (L - 1));
        const int bits_n = bits_for((uint64_t)N);
        for (int k = 1; k <= D; k++) {
            const int64_t n = g->bucket[k + 1] - g->bucket[k];
            uint32_t* perm = order.as<uint32_t>() + (g->bucket[k] - S);
            uint64_t* kk = keys.as<uint64_t>();
            auto key_pass = [&](int field, int sh, int bits) -> mg_status {
                sort_key_kernel<<<grid_n(n), 256, 0, s>>>(perm, n, field, sh, t.p.as<uint32_t>(), t.q.as<uint32_t>(),
                                                          t.a.as<uint64_t>(), t.b.as<uint64_t>(),
                                                          canon.as<uint32_t>(), kk);
                MG_CUDA(cudaGetLastError());
                return radix_sort_pairs(kk, perm, n, bits, al, s);
            };
            if (2 * bits_ab <= 64) {
                MG_TRY(key_pass(2, bits_ab, 2 * bits_ab));
            } else {
                MG_TRY(key_pass(0, 0, bits_ab));
                MG_TRY(key_pass(1, 0, bits_ab));
            }
            MG_TRY(key_pass(3, bits_n, 2 * bits_n));
            assign_kernel<<<grid_n(n), 256, 0, s>>>(perm, n, (uint32_t)g->bucket[k], t.p.as<uint32_t>(),
                                                    t.q.as<uint32_t>(), t.a.as<uint64_t>(), t.b.as<uint64_t>(),
                                                    canon.as<uint32_t>(), g->pq.as<uint2>(), g->ab.as<ulonglong2>());
            MG_CUDA(cudaGetLastError());
        }
    }
    if (total_hi > 0) {
        remap_kernel<<<grid_n(total_hi), 256, 0, s>>>(g->mip.as<uint32_t>(), total_hi, canon.as<uint32_t>(), status);
        MG_CUDA(cudaGetLastError());
    }
    MG_TRY(build_query_copies(g, s));
    MG_TRY(g->ab32.alloc(&al, (size_t)N * sizeof(uint2), s));
    MG_TRY(g->alpha.alloc(&al, (size_t)N * sizeof(float), s));
    weights_kernel<<<grid_n(N), 256, 0, s>>>(g->ab.as<ulonglong2>(), N, S, g->ab32.as<uint2>(), g->alpha.as<float>());
    MG_CUDA(cudaGetLastError());
    MG_TRY(build_lut(g, s));
    unsigned bits = 0;
    MG_TRY(read_scalar(&bits, status, s));
    if (bits) return fail(MG_ERR_CAPACITY, "node table overflow during the build");
    MG_CUDA(cudaMemsetAsync(status, 0, sizeof(unsigned), s));
    return MG_OK;
}

// The padded axis-major copies of the box queries (copy c of level l: rows
// of the copy's fastest axis, qpitch[l][c] IDs apart, a multiple of 32 bytes
// unless that would take a copy past 2^32 IDs).
mg_status build_query_copies(mg_graph* g, cudaStream_t s) {
    const int L = g->L;
    auto dims_of = [&](int l) {
        Dims3 d;
        d.x = g->geom.dims[l][0];
        d.y = g->geom.dims[l][1];
        d.z = g->geom.dims[l][2];
        return d;
    };
    auto grid_n = [](int64_t n) { return (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 64); };
    int64_t hi_total[3] = {0, 0, 0};
    for (int c = 0; c < 3; c++) {
        for (int l = 0; l < L; l++) {
            const Dims3 d = dims_of(l);
            const int64_t d0 = c == 0 ? d.x : c == 1 ? d.y : d.z;
            const int64_t rows = nvox(d) / d0;
            const int64_t per32 = l == 0 ? 32 / g->id0_bytes : 8;
            int64_t pitch = (d0 + per32 - 1) / per32 * per32;
            if (pitch * rows >= (1ll << 32)) pitch = d0;
            g->qpitch[l][c] = (int32_t)pitch;
            if (l >= 1) {
                g->qoff[l][c] = hi_total[c];
                hi_total[c] += pitch * rows;
            }
        }
    }
    for (int c = 0; c < 3; c++) {
        const Dims3 d0 = dims_of(0);
        const int64_t pitch0 = g->qpitch[0][c];
        if (c > 0 || pitch0 != d0.x) {
            const int64_t n = pitch0 * (nvox(d0) / (c == 0 ? d0.x : c == 1 ? d0.y : d0.z));
            MG_TRY(g->mip0x[c].alloc(&g->al, (size_t)n * g->id0_bytes, s));
            if (g->id0_bytes == 2)
                transpose_copy_kernel<uint16_t><<<grid_n(n), 256, 0, s>>>(g->mip0.as<uint16_t>(),
                                                                          g->mip0x[c].as<uint16_t>(), d0, c, pitch0);
            else
                transpose_copy_kernel<uint32_t><<<grid_n(n), 256, 0, s>>>(g->mip0.as<uint32_t>(),
                                                                          g->mip0x[c].as<uint32_t>(), d0, c, pitch0);
            MG_CUDA(cudaGetLastError());
        }
        if (hi_total[c] > 0) {
            MG_TRY(g->mipx[c].alloc(&g->al, (size_t)hi_total[c] * 4, s));
            for (int l = 1; l < L; l++) {
                const Dims3 d = dims_of(l);
                const int64_t pitch = g->qpitch[l][c];
                const int64_t n = pitch * (nvox(d) / (c == 0 ? d.x : c == 1 ? d.y : d.z));
                transpose_copy_kernel<uint32_t><<<grid_n(n), 256, 0, s>>>(
                    g->mip.as<uint32_t>() + g->geom.off[l], g->mipx[c].as<uint32_t>() + g->qoff[l][c], d, c, pitch);
                MG_CUDA(cudaGetLastError());
            }
        }
    }
    return MG_OK;
}

}  // namespace mg
