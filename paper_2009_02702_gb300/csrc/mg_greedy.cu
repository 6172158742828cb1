// mg_greedy.cu -- greedy factorisation of the histogram mipmap (Sec. 3.3,
// Eq. 10-13; Sec. 3.7: the tau cutoff and the scalar quantiser).
//
// H is every mixture of levels 1..L-1 (Eq. 4 integer weights 8^l H), built
// here level by level from the volume.  Stage 1, round by round: every pair
// i < j of components occurring together in a mixture with more than tau
// components is scored into a hash histogram (phi_1: 1 per mixture, phi_2:
// |h| - 1 if |h| > 2, else 2); the highest score wins, ties to the smallest
// (i, j); every such mixture holding both is factored -- i and j replaced by
// their lerp with the summed exact weight.  Stage 2, in waves: every mixture
// left with two or more components lerps its two lowest-numbered ones.
// A lerp of p < q with weights c_p, c_q is the node (p, q, a, b) of the
// reduced ratio (exact), or (p, q, k, 0) with k = floor(c_q 2^b / (c_p +
// c_q)) (b-bit quantiser, bins of equal width, codeword the centre, sigma
// the rms of the weights' distance to it).  New nodes of a round or wave
// are numbered in the scan order of the first mixture that made them, so
// the parallel build numbers (and therefore breaks ties) exactly as a
// sequential scan would.  The result is renumbered canonically on the host
// (level, p', q', a, b).
#include "mg_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

namespace mg {
namespace {

constexpr uint32_t kEmpty = 0u, kWriting = 1u, kReady = 2u;
constexpr uint32_t kUnset = 0xFFFFFFFFu;
constexpr unsigned kSpin = 1u << 20;

__device__ __forceinline__ uint64_t gmix(uint64_t x) {
    x ^= x >> 31;
    x *= 0x7fb5d329728ea185ull;
    x ^= x >> 27;
    x *= 0x81dadef4bc2dd44dull;
    x ^= x >> 33;
    return x;
}

// ---------------------------------------------------------------------------
// mixture lists of every level >= 1: per mixture a capacity region
// [off, off + cap) of which the first len entries are used (ascending IDs)
// ---------------------------------------------------------------------------
struct Mix {
    uint64_t* off;
    uint32_t* len;
    uint32_t* comp;
    uint64_t* wt;
};

__global__ void l1_cap_kernel(int32_t dx, int32_t dy, int32_t dz, int32_t ex, int32_t ey, int32_t ez,
                              uint64_t* __restrict__ cap) {
    const int64_t n = (int64_t)ex * ey * ez;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t X = v % ex, Y = (v / ex) % ey, Z = v / ((int64_t)ex * ey);
        const int64_t cx = min((int64_t)2, dx - 2 * X), cy = min((int64_t)2, dy - 2 * Y), cz = min((int64_t)2, dz - 2 * Z);
        cap[v] = (uint64_t)(cx * cy * cz);
    }
}

// children of parent (X, Y, Z): up to 8 voxels of the level below
template <typename F>
__device__ __forceinline__ int for_children(int64_t X, int64_t Y, int64_t Z, int32_t dx, int32_t dy, int32_t dz, F f) {
    int N = 0;
    for (int k = 0; k < 2; k++)
        for (int j = 0; j < 2; j++)
            for (int i = 0; i < 2; i++) {
                const int64_t x = 2 * X + i, y = 2 * Y + j, z = 2 * Z + k;
                if (x >= dx || y >= dy || z >= dz) continue;
                N++;
                f((z * dy + y) * dx + x);
            }
    return N;
}

// level 1 from the level-0 IDs: sort the children's IDs, merge, weight 8/N each
template <typename T>
__global__ void l1_lists_kernel(const T* __restrict__ ids, int32_t dx, int32_t dy, int32_t dz, int32_t ex, int32_t ey,
                                int32_t ez, Mix X1, int64_t m0) {
    const int64_t n = (int64_t)ex * ey * ez;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t X = v % ex, Y = (v / ex) % ey, Z = v / ((int64_t)ex * ey);
        uint32_t c[8];
        int cnt = 0;
        const int N = for_children(X, Y, Z, dx, dy, dz, [&](int64_t i) { c[cnt++] = (uint32_t)ids[i]; });
        for (int a = 1; a < cnt; a++)
            for (int b = a; b > 0 && c[b - 1] > c[b]; b--) {
                const uint32_t t = c[b];
                c[b] = c[b - 1];
                c[b - 1] = t;
            }
        const uint64_t scale = (uint64_t)(8 / N);
        const int64_t m = m0 + v;
        const uint64_t o = X1.off[m];
        uint32_t L = 0;
        for (int a = 0; a < cnt;) {
            int b = a;
            while (b < cnt && c[b] == c[a]) b++;
            X1.comp[o + L] = c[a];
            X1.wt[o + L] = (uint64_t)(b - a) * scale;
            L++;
            a = b;
        }
        X1.len[m] = L;
    }
}

__global__ void next_cap_kernel(Mix Xs, int64_t mprev, int32_t dx, int32_t dy, int32_t dz, int32_t ex, int32_t ey,
                                int32_t ez, uint64_t* __restrict__ cap) {
    const int64_t n = (int64_t)ex * ey * ez;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t X = v % ex, Y = (v / ex) % ey, Z = v / ((int64_t)ex * ey);
        uint64_t s = 0;
        for_children(X, Y, Z, dx, dy, dz, [&](int64_t i) { s += Xs.len[mprev + i]; });
        cap[v] = s;
    }
}

// level l+1 from level l: merge the children's sorted lists, weight 8/N
__global__ void next_lists_kernel(Mix Xs, int64_t mprev, int32_t dx, int32_t dy, int32_t dz, int32_t ex, int32_t ey,
                                  int32_t ez, int64_t m0) {
    const int64_t n = (int64_t)ex * ey * ez;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const int64_t X = v % ex, Y = (v / ex) % ey, Z = v / ((int64_t)ex * ey);
        int64_t ch[8];
        uint32_t pos[8];
        int k = 0;
        const int N = for_children(X, Y, Z, dx, dy, dz, [&](int64_t i) { ch[k++] = mprev + i; });
        for (int a = 0; a < k; a++) pos[a] = 0;
        const uint64_t scale = (uint64_t)(8 / N);
        const int64_t m = m0 + v;
        const uint64_t o = Xs.off[m];
        uint32_t L = 0;
        for (;;) {
            uint32_t best = 0xFFFFFFFFu;
            for (int a = 0; a < k; a++)
                if (pos[a] < Xs.len[ch[a]]) best = min(best, Xs.comp[Xs.off[ch[a]] + pos[a]]);
            if (best == 0xFFFFFFFFu) break;
            uint64_t s = 0;
            for (int a = 0; a < k; a++)
                if (pos[a] < Xs.len[ch[a]] && Xs.comp[Xs.off[ch[a]] + pos[a]] == best) {
                    s += Xs.wt[Xs.off[ch[a]] + pos[a]];
                    pos[a]++;
                }
            Xs.comp[o + L] = best;
            Xs.wt[o + L] = s * scale;
            L++;
        }
        Xs.len[m] = L;
    }
}

// ---------------------------------------------------------------------------
// node table and its key hash
// ---------------------------------------------------------------------------
struct Nodes {
    uint32_t* p;
    uint32_t* q;
    uint64_t* a;
    uint64_t* b;
    uint32_t* depth;
    // key hash: slots of (state, key, value = node, first mixture)
    uint32_t* st;
    uint32_t* kp;
    uint32_t* kq;
    uint64_t* ka;
    uint64_t* kb;
    uint32_t* val;
    uint64_t* firstm;
    uint64_t mask;
    uint32_t* fresh;           // slots created in this pass
    unsigned long long* nfresh;
    unsigned* status;
};

// the slot of key (p, q, a, b), created if new (then `fresh`); records the
// smallest mixture index that asked for it
__device__ uint64_t node_slot(const Nodes& T, uint32_t p, uint32_t q, uint64_t a, uint64_t b, uint64_t m) {
    uint64_t h = gmix(((uint64_t)p << 32 | q) ^ gmix(a ^ (b * 0x9e3779b97f4a7c15ull))) & T.mask;
    for (uint64_t probe = 0; probe <= T.mask; probe++) {
        const uint32_t old = atomicCAS(T.st + h, kEmpty, kWriting);
        if (old == kEmpty) {
            T.kp[h] = p;
            T.kq[h] = q;
            T.ka[h] = a;
            T.kb[h] = b;
            T.val[h] = kUnset;
            T.firstm[h] = m;
            __threadfence();
            atomicExch(T.st + h, kReady);
            T.fresh[atomicAdd(T.nfresh, 1ull)] = (uint32_t)h;
            return h;
        }
        unsigned spins = 0;
        while (ld_acquire_u32(T.st + h) != kReady) {
            if (++spins > kSpin) {
                set_status(T.status, kStatTimeout);
                return ~0ull;
            }
        }
        if (T.kp[h] == p && T.kq[h] == q && T.ka[h] == a && T.kb[h] == b) {
            atomicMin(reinterpret_cast<unsigned long long*>(T.firstm + h), (unsigned long long)m);
            return h;
        }
        h = (h + 1) & T.mask;
    }
    set_status(T.status, kStatCapacity);
    return ~0ull;
}

__device__ __forceinline__ uint64_t gcd64(uint64_t x, uint64_t y) {
    while (y) {
        const uint64_t r = x % y;
        x = y;
        y = r;
    }
    return x;
}

// the key of the lerp of (p, cp), (q, cq), p < q
__device__ __forceinline__ void lerp_key(uint64_t cp, uint64_t cq, int bitrate, uint64_t& a, uint64_t& b) {
    if (bitrate == 0) {
        const uint64_t g = gcd64(cp, cq);
        a = cp / g;
        b = cq / g;
        return;
    }
    const uint64_t nb = 1ull << bitrate;
    uint64_t k = (cq << bitrate) / (cp + cq);
    if (k >= nb) k = nb - 1;
    a = k;
    b = 0;
}

__device__ __forceinline__ int find_comp(const Mix& X, int64_t m, uint32_t id) {
    const uint32_t* c = X.comp + X.off[m];
    int lo = 0, hi = (int)X.len[m];
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (c[mid] < id) lo = mid + 1;
        else hi = mid;
    }
    return lo < (int)X.len[m] && c[lo] == id ? lo : -1;
}

// ---------------------------------------------------------------------------
// stage 1: scores, argmax, factoring
// ---------------------------------------------------------------------------
struct Pairs {
    unsigned long long* key;   // i << 32 | j, ~0 = empty
    unsigned long long* score;
    uint64_t mask;
};

__global__ void score_kernel(Mix X, int64_t M, int tau, int strategy, Pairs PH, unsigned* status) {
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t m = warp; m < M; m += nw) {
        const int n = (int)X.len[m];
        if (n <= tau) continue;
        const unsigned long long add = strategy == 1 ? 1ull : (n > 2 ? (unsigned long long)(n - 1) : 2ull);
        const uint32_t* c = X.comp + X.off[m];
        const int64_t np = (int64_t)n * (n - 1) / 2;
        for (int64_t t = lane; t < np; t += 32) {
            // pair t of the upper triangle: row a, column b > a
            int64_t a = 0, rem = t;
            while (rem >= n - 1 - a) {
                rem -= n - 1 - a;
                a++;
            }
            const int64_t b = a + 1 + rem;
            const unsigned long long key = (unsigned long long)c[a] << 32 | c[b];
            uint64_t h = gmix(key) & PH.mask;
            for (uint64_t probe = 0;; probe++) {
                if (probe > PH.mask) {
                    set_status(status, kStatCapacity);
                    break;
                }
                const unsigned long long old = atomicCAS(PH.key + h, ~0ull, key);
                if (old == ~0ull || old == key) {
                    atomicAdd(PH.score + h, add);
                    break;
                }
                h = (h + 1) & PH.mask;
            }
        }
    }
}

__global__ void best_score_kernel(Pairs PH, unsigned long long* best) {
    unsigned long long m = 0;
    for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h <= PH.mask; h += (uint64_t)gridDim.x * blockDim.x)
        if (PH.key[h] != ~0ull) m = max(m, PH.score[h]);
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(best, m);
}

__global__ void best_key_kernel(Pairs PH, unsigned long long* best) {
    const unsigned long long top = best[0];
    unsigned long long k = ~0ull;
    for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h <= PH.mask; h += (uint64_t)gridDim.x * blockDim.x)
        if (PH.key[h] != ~0ull && PH.score[h] == top) k = min(k, PH.key[h]);
    for (int o = 16; o > 0; o >>= 1) k = min(k, __shfl_xor_sync(0xffffffffu, k, o));
    if ((threadIdx.x & 31) == 0 && k != ~0ull) atomicMin(best + 1, k);
}

// phase A: the slot of every mixture's lerp (stage 1: pair (i, j) in the
// mixtures with more than tau components; stage 2: the two lowest components
// of every mixture with two or more); mslot[m] = slot, or ~0
__global__ void factor_slots_kernel(Mix X, int64_t M, int stage, int tau, uint32_t i, uint32_t j, int bitrate,
                                    Nodes T, uint64_t* __restrict__ mslot, unsigned long long* __restrict__ active) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        mslot[m] = ~0ull;
        const int n = (int)X.len[m];
        int ii, jj;
        if (stage == 1) {
            if (n <= tau) continue;
            ii = find_comp(X, m, i);
            jj = ii < 0 ? -1 : find_comp(X, m, j);
            if (jj < 0) continue;
        } else {
            if (n < 2) continue;
            ii = 0;
            jj = 1;
        }
        const uint32_t p = X.comp[X.off[m] + ii], q = X.comp[X.off[m] + jj];
        uint64_t a, b;
        lerp_key(X.wt[X.off[m] + ii], X.wt[X.off[m] + jj], bitrate, a, b);
        mslot[m] = node_slot(T, p, q, a, b, (uint64_t)m);
        atomicAdd(active, 1ull);
    }
}

// phase B: the fresh slots' first mixtures as sort keys
__global__ void fresh_keys_kernel(Nodes T, int64_t n, uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t h = T.fresh[t];
        keys[t] = T.firstm[h];
        vals[t] = h;
    }
}

// phase B: node IDs base + rank for the sorted fresh slots
__global__ void assign_kernel(Nodes T, const uint32_t* __restrict__ sorted, int64_t n, uint32_t base) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t h = sorted[t];
        const uint32_t id = base + (uint32_t)t;
        T.val[h] = id;
        const uint32_t p = T.kp[h], q = T.kq[h];
        T.p[id] = p;
        T.q[id] = q;
        T.a[id] = T.ka[h];
        T.b[id] = T.kb[h];
        T.depth[id] = max(T.depth[p], T.depth[q]) + 1;
    }
}

// phase C: replace the lerped components by their node; quantiser records
__global__ void merge_kernel(Mix X, int64_t M, int stage, uint32_t i, uint32_t j, int bitrate, Nodes T,
                             const uint64_t* __restrict__ mslot, double* __restrict__ ssq,
                             unsigned long long* __restrict__ bincnt) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t h = mslot[m];
        if (h == ~0ull) continue;
        const int n = (int)X.len[m];
        const int ii = stage == 1 ? find_comp(X, m, i) : 0, jj = stage == 1 ? find_comp(X, m, j) : 1;
        uint32_t* c = X.comp + X.off[m];
        uint64_t* w = X.wt + X.off[m];
        const uint64_t cp = w[ii], cq = w[jj];
        if (bitrate) {
            const uint64_t nb = 1ull << bitrate;
            const uint64_t k = T.ka[h];
            const double x = (double)cq / (double)(cp + cq), cw = (double)(2 * k + 1) / (double)(2 * nb);
            atomicAdd(ssq + k, (x - cw) * (x - cw));
            atomicAdd(bincnt + k, 1ull);
        }
        const uint32_t node = T.val[h];
        int o = 0;
        for (int e = 0; e < n; e++) {
            if (e == ii || e == jj) continue;
            c[o] = c[e];
            w[o] = w[e];
            o++;
        }
        int pos = o;
        while (pos > 0 && c[pos - 1] > node) {
            c[pos] = c[pos - 1];
            w[pos] = w[pos - 1];
            pos--;
        }
        c[pos] = node;
        w[pos] = cp + cq;
        X.len[m] = (uint32_t)(o + 1);
    }
}

__global__ void final_ids_kernel(Mix X, int64_t M, uint32_t* __restrict__ out) {
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < M; m += (int64_t)gridDim.x * blockDim.x)
        out[m] = X.comp[X.off[m]];
}

__global__ void init_sources_kernel(Nodes T, uint32_t S) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        T.p[s] = MG_NO_NODE;
        T.q[s] = MG_NO_NODE;
        T.a[s] = 0;
        T.b[s] = 0;
        T.depth[s] = 0;
    }
}

template <typename T>
mg_status read_back(T* host, const void* dev, size_t n, cudaStream_t s) {
    MG_CUDA(cudaMemcpyAsync(host, dev, n * sizeof(T), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    return MG_OK;
}

}  // namespace
}  // namespace mg

struct mg_greedy {
    uint32_t S = 0;
    int L = 0, D = 0;
    int64_t N = 0;
    int64_t dims[MG_MAX_LEVELS][3] = {};
    std::vector<uint32_t> p, q;
    std::vector<uint64_t> a, b;
    std::vector<std::vector<uint32_t>> mip;
    std::vector<uint32_t> picks;
    std::vector<double> codebook, sigma;
    int64_t waves = 0;
    double ms = 0.0;
};

namespace mg {
namespace {

mg_status greedy_run(mg_greedy* R, const void* ids, int id_bytes, int64_t nx, int64_t ny, int64_t nz,
                     const mg_greedy_opts& o, cudaStream_t s) {
    const Alloc al{};
    const uint32_t S = R->S;
    int64_t d[3] = {nx, ny, nz};
    for (;;) {
        if (R->L >= MG_MAX_LEVELS) return fail(MG_ERR_UNSUPPORTED, "too many mip levels");
        for (int k = 0; k < 3; k++) R->dims[R->L][k] = d[k];
        R->L++;
        if (d[0] == 1 && d[1] == 1 && d[2] == 1) break;
        for (int k = 0; k < 3; k++) d[k] = (d[k] + 1) / 2;
    }
    const int L = R->L;
    R->mip.resize(L);
    const int64_t V0 = nx * ny * nz;
    R->mip[0].resize((size_t)V0);
    if (id_bytes == 2) {
        std::vector<uint16_t> h((size_t)V0);
        MG_CUDA(cudaMemcpyAsync(h.data(), ids, (size_t)V0 * 2, cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < V0; i++) R->mip[0][i] = h[i];
    } else {
        MG_CUDA(cudaMemcpyAsync(R->mip[0].data(), ids, (size_t)V0 * 4, cudaMemcpyDeviceToHost, s));
        MG_CUDA(cudaStreamSynchronize(s));
    }
    for (int64_t i = 0; i < V0; i++)
        if (R->mip[0][i] >= S) return fail(MG_ERR_INVALID_ARG, "segment ID >= num_segments");
    if (L == 1) {
        R->N = S;
        R->p.assign(S, MG_NO_NODE);
        R->q.assign(S, MG_NO_NODE);
        R->a.assign(S, 0);
        R->b.assign(S, 0);
        return MG_OK;
    }
    // mixtures: levels 1..L-1, capacities from the children
    std::vector<int64_t> m0(L, 0);
    int64_t M = 0;
    for (int l = 1; l < L; l++) {
        m0[l] = M;
        M += R->dims[l][0] * R->dims[l][1] * R->dims[l][2];
    }
    Buf off, len, cap;
    MG_TRY(off.alloc(&al, (size_t)(M + 1) * 8, s));
    MG_TRY(len.alloc(&al, (size_t)M * 4, s));
    MG_TRY(cap.alloc(&al, (size_t)M * 8, s));
    Mix X;
    X.off = off.as<uint64_t>();
    X.len = len.as<uint32_t>();
    Buf comp, wt;
    auto dims3 = [&](int l, int k) { return (int32_t)R->dims[l][k]; };
    // capacities level by level need the level below's lengths: build in
    // two sweeps (capacity of level 1 from the geometry, of level l+1 from
    // the lengths of level l)
    int64_t used = 0;
    std::vector<uint64_t> capacity_total(L, 0);
    l1_cap_kernel<<<grid_for(M, 256, 152 * 32), 256, 0, s>>>(dims3(0, 0), dims3(0, 1), dims3(0, 2), dims3(1, 0), dims3(1, 1),
                                                             dims3(1, 2), cap.as<uint64_t>());
    MG_CUDA(cudaGetLastError());
    // the whole upper bound: sum of the level-0 voxels feeding each level
    // (entries never grow from one level to the next)
    const int64_t E = V0 * (L - 1);
    MG_TRY(comp.alloc(&al, (size_t)std::max<int64_t>(E, 1) * 4, s));
    MG_TRY(wt.alloc(&al, (size_t)std::max<int64_t>(E, 1) * 8, s));
    X.comp = comp.as<uint32_t>();
    X.wt = wt.as<uint64_t>();
    // level 1
    {
        const int64_t n1 = R->dims[1][0] * R->dims[1][1] * R->dims[1][2];
        MG_TRY(scan_exclusive_u64(cap.as<uint64_t>(), X.off, n1, nullptr, al, s));
        uint64_t tot = 0;
        std::vector<uint64_t> last(2);
        MG_TRY(read_back(last.data(), X.off + n1 - 1, 1, s));
        MG_TRY(read_back(last.data() + 1, cap.as<uint64_t>() + n1 - 1, 1, s));
        tot = last[0] + last[1];
        if (id_bytes == 2)
            l1_lists_kernel<uint16_t><<<grid_for(n1, 256, 152 * 32), 256, 0, s>>>(
                static_cast<const uint16_t*>(ids), dims3(0, 0), dims3(0, 1), dims3(0, 2), dims3(1, 0), dims3(1, 1),
                dims3(1, 2), X, 0);
        else
            l1_lists_kernel<uint32_t><<<grid_for(n1, 256, 152 * 32), 256, 0, s>>>(
                static_cast<const uint32_t*>(ids), dims3(0, 0), dims3(0, 1), dims3(0, 2), dims3(1, 0), dims3(1, 1),
                dims3(1, 2), X, 0);
        MG_CUDA(cudaGetLastError());
        used = (int64_t)tot;
    }
    for (int l = 1; l + 1 < L; l++) {
        const int64_t n = R->dims[l + 1][0] * R->dims[l + 1][1] * R->dims[l + 1][2];
        next_cap_kernel<<<grid_for(n, 256, 152 * 32), 256, 0, s>>>(X, m0[l], dims3(l, 0), dims3(l, 1), dims3(l, 2),
                                                                   dims3(l + 1, 0), dims3(l + 1, 1), dims3(l + 1, 2),
                                                                   cap.as<uint64_t>());
        MG_CUDA(cudaGetLastError());
        MG_TRY(scan_exclusive_u64(cap.as<uint64_t>(), X.off + m0[l + 1], n, nullptr, al, s));
        // shift this level's offsets past the entries already placed
        std::vector<uint64_t> offs((size_t)n), caps((size_t)n);
        MG_TRY(read_back(offs.data(), X.off + m0[l + 1], (size_t)n, s));
        MG_TRY(read_back(caps.data(), cap.as<uint64_t>(), (size_t)n, s));
        for (int64_t v = 0; v < n; v++) offs[v] += (uint64_t)used;
        if (used + (int64_t)(offs[n - 1] - used + caps[n - 1]) > E) return fail(MG_ERR_CAPACITY, "mixture lists overflow");
        MG_CUDA(cudaMemcpyAsync(X.off + m0[l + 1], offs.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
        used = (int64_t)(offs[n - 1] + caps[n - 1]);
        next_lists_kernel<<<grid_for(n, 256, 152 * 32), 256, 0, s>>>(X, m0[l], dims3(l, 0), dims3(l, 1), dims3(l, 2),
                                                                     dims3(l + 1, 0), dims3(l + 1, 1), dims3(l + 1, 2),
                                                                     m0[l + 1]);
        MG_CUDA(cudaGetLastError());
        MG_CUDA(cudaStreamSynchronize(s));
    }
    // node table: at most one node per lerp, sum over mixtures of (len - 1)
    std::vector<uint32_t> lens((size_t)M);
    MG_TRY(read_back(lens.data(), X.len, (size_t)M, s));
    int64_t lerps = 0, pairs_ub = 0;
    for (int64_t m = 0; m < M; m++) {
        lerps += lens[m] - 1;
        if ((int)lens[m] > o.tau) pairs_ub += (int64_t)lens[m] * (lens[m] - 1) / 2;
    }
    const int64_t cap_nodes = S + lerps + 1;
    if (cap_nodes >= (1ll << 32)) return fail(MG_ERR_UNSUPPORTED, "more than 2^32 nodes");
    uint64_t hs = 1024;
    while (hs < 2 * (uint64_t)cap_nodes) hs <<= 1;
    Buf np_, nq_, na_, nb_, ndep, st, kp, kq, ka, kb, kval, kfirst, fresh, scal;
    MG_TRY(np_.alloc(&al, (size_t)cap_nodes * 4, s));
    MG_TRY(nq_.alloc(&al, (size_t)cap_nodes * 4, s));
    MG_TRY(na_.alloc(&al, (size_t)cap_nodes * 8, s));
    MG_TRY(nb_.alloc(&al, (size_t)cap_nodes * 8, s));
    MG_TRY(ndep.alloc(&al, (size_t)cap_nodes * 4, s));
    MG_TRY(st.alloc(&al, hs * 4, s));
    MG_TRY(kp.alloc(&al, hs * 4, s));
    MG_TRY(kq.alloc(&al, hs * 4, s));
    MG_TRY(ka.alloc(&al, hs * 8, s));
    MG_TRY(kb.alloc(&al, hs * 8, s));
    MG_TRY(kval.alloc(&al, hs * 4, s));
    MG_TRY(kfirst.alloc(&al, hs * 8, s));
    MG_TRY(fresh.alloc(&al, (size_t)std::max<int64_t>(M, 1) * 4, s));
    MG_TRY(scal.alloc(&al, 64, s));
    MG_CUDA(cudaMemsetAsync(st.p, 0, hs * 4, s));
    MG_CUDA(cudaMemsetAsync(scal.p, 0, 64, s));
    Nodes T;
    T.p = np_.as<uint32_t>();
    T.q = nq_.as<uint32_t>();
    T.a = na_.as<uint64_t>();
    T.b = nb_.as<uint64_t>();
    T.depth = ndep.as<uint32_t>();
    T.st = st.as<uint32_t>();
    T.kp = kp.as<uint32_t>();
    T.kq = kq.as<uint32_t>();
    T.ka = ka.as<uint64_t>();
    T.kb = kb.as<uint64_t>();
    T.val = kval.as<uint32_t>();
    T.firstm = kfirst.as<uint64_t>();
    T.mask = hs - 1;
    T.fresh = fresh.as<uint32_t>();
    T.nfresh = scal.as<unsigned long long>();
    unsigned* status = reinterpret_cast<unsigned*>(scal.as<unsigned long long>() + 7);
    T.status = status;
    init_sources_kernel<<<grid_for(S, 256), 256, 0, s>>>(T, S);
    MG_CUDA(cudaGetLastError());
    const int nbins = o.bitrate ? 1 << o.bitrate : 1;
    Buf ssq, bincnt, mslot, best, active, skeys, svals;
    MG_TRY(ssq.alloc(&al, (size_t)nbins * 8, s));
    MG_TRY(bincnt.alloc(&al, (size_t)nbins * 8, s));
    MG_TRY(mslot.alloc(&al, (size_t)M * 8, s));
    MG_TRY(best.alloc(&al, 16, s));
    MG_TRY(active.alloc(&al, 8, s));
    MG_TRY(skeys.alloc(&al, (size_t)std::max<int64_t>(M, 1) * 8, s));
    MG_TRY(svals.alloc(&al, (size_t)std::max<int64_t>(M, 1) * 4, s));
    MG_CUDA(cudaMemsetAsync(ssq.p, 0, (size_t)nbins * 8, s));
    MG_CUDA(cudaMemsetAsync(bincnt.p, 0, (size_t)nbins * 8, s));
    int mbits = 1;
    while (mbits < 63 && (1ll << mbits) < M) mbits++;
    uint32_t next_id = S;
    // one factoring pass (phase A slots, B numbering, C merge)
    auto pass = [&](int stage, uint32_t i, uint32_t j, unsigned long long* act) -> mg_status {
        MG_CUDA(cudaMemsetAsync(T.nfresh, 0, 8, s));
        MG_CUDA(cudaMemsetAsync(active.p, 0, 8, s));
        factor_slots_kernel<<<grid_for(M, 256, 152 * 32), 256, 0, s>>>(X, M, stage, o.tau, i, j, o.bitrate, T,
                                                                       mslot.as<uint64_t>(),
                                                                       active.as<unsigned long long>());
        MG_CUDA(cudaGetLastError());
        unsigned long long nf = 0;
        MG_TRY(read_back(&nf, T.nfresh, 1, s));
        MG_TRY(read_back(act, active.p, 1, s));
        if (nf) {
            fresh_keys_kernel<<<grid_for((int64_t)nf, 256), 256, 0, s>>>(T, (int64_t)nf, skeys.as<uint64_t>(),
                                                                          svals.as<uint32_t>());
            MG_CUDA(cudaGetLastError());
            MG_TRY(radix_sort_pairs(skeys.as<uint64_t>(), svals.as<uint32_t>(), (int64_t)nf, mbits, al, s));
            if ((int64_t)next_id + (int64_t)nf > cap_nodes) return fail(MG_ERR_CAPACITY, "node table overflow");
            assign_kernel<<<grid_for((int64_t)nf, 256), 256, 0, s>>>(T, svals.as<uint32_t>(), (int64_t)nf, next_id);
            MG_CUDA(cudaGetLastError());
            next_id += (uint32_t)nf;
        }
        merge_kernel<<<grid_for(M, 256, 152 * 32), 256, 0, s>>>(X, M, stage, i, j, o.bitrate, T, mslot.as<uint64_t>(),
                                                                ssq.as<double>(),
                                                                bincnt.as<unsigned long long>());
        MG_CUDA(cudaGetLastError());
        return MG_OK;
    };
    // stage 1
    if (pairs_ub > 0) {
        uint64_t ps = 1024;
        while (ps < 2 * (uint64_t)pairs_ub) ps <<= 1;
        if (ps > (1ull << 30)) return fail(MG_ERR_UNSUPPORTED, "too many component pairs for the score table");
        Buf pk, psc;
        MG_TRY(pk.alloc(&al, ps * 8, s));
        MG_TRY(psc.alloc(&al, ps * 8, s));
        Pairs PH{pk.as<unsigned long long>(), psc.as<unsigned long long>(), ps - 1};
        for (;;) {
            MG_CUDA(cudaMemsetAsync(pk.p, 0xFF, ps * 8, s));
            MG_CUDA(cudaMemsetAsync(psc.p, 0, ps * 8, s));
            const unsigned long long init[2] = {0ull, ~0ull};
            MG_CUDA(cudaMemcpyAsync(best.p, init, 16, cudaMemcpyHostToDevice, s));
            score_kernel<<<152 * 16, 256, 0, s>>>(X, M, o.tau, o.strategy, PH, status);
            best_score_kernel<<<grid_for((int64_t)ps, 256, 152 * 16), 256, 0, s>>>(PH, best.as<unsigned long long>());
            best_key_kernel<<<grid_for((int64_t)ps, 256, 152 * 16), 256, 0, s>>>(PH, best.as<unsigned long long>());
            MG_CUDA(cudaGetLastError());
            unsigned long long b2[2];
            MG_TRY(read_back(b2, best.p, 2, s));
            if (b2[0] == 0) break;
            const uint32_t bi = (uint32_t)(b2[1] >> 32), bj = (uint32_t)(b2[1] & 0xFFFFFFFFu);
            R->picks.push_back(bi);
            R->picks.push_back(bj);
            unsigned long long act = 0;
            MG_TRY(pass(1, bi, bj, &act));
        }
    }
    // stage 2: waves
    for (;;) {
        unsigned long long act = 0;
        MG_TRY(pass(2, 0, 0, &act));
        if (!act) break;
        R->waves++;
    }
    unsigned bits = 0;
    MG_TRY(read_back(&bits, status, 1, s));
    if (bits) return fail(status_from_bits(bits), "greedy factorisation: a device table overflowed or a wait expired");
    // results to the host, canonical numbering (level, p', q', a, b)
    const int64_t N = next_id;
    std::vector<uint32_t> tp((size_t)N), tq((size_t)N), tdep((size_t)N), roots((size_t)M);
    std::vector<uint64_t> ta((size_t)N), tb((size_t)N);
    MG_TRY(read_back(tp.data(), T.p, (size_t)N, s));
    MG_TRY(read_back(tq.data(), T.q, (size_t)N, s));
    MG_TRY(read_back(ta.data(), T.a, (size_t)N, s));
    MG_TRY(read_back(tb.data(), T.b, (size_t)N, s));
    MG_TRY(read_back(tdep.data(), T.depth, (size_t)N, s));
    Buf rt;
    MG_TRY(rt.alloc(&al, (size_t)M * 4, s));
    final_ids_kernel<<<grid_for(M, 256), 256, 0, s>>>(X, M, rt.as<uint32_t>());
    MG_CUDA(cudaGetLastError());
    MG_TRY(read_back(roots.data(), rt.p, (size_t)M, s));
    if (o.bitrate) {
        std::vector<double> sq((size_t)nbins);
        std::vector<unsigned long long> cn((size_t)nbins);
        MG_TRY(read_back(sq.data(), ssq.p, (size_t)nbins, s));
        MG_TRY(read_back(cn.data(), bincnt.p, (size_t)nbins, s));
        R->codebook.resize((size_t)nbins);
        R->sigma.resize((size_t)nbins);
        for (int k = 0; k < nbins; k++) {
            R->codebook[k] = (double)(2 * k + 1) / (double)(2 * nbins);
            R->sigma[k] = cn[k] ? std::sqrt(sq[k] / (double)cn[k]) : 0.0;
        }
    }
    int D = 0;
    for (int64_t n = S; n < N; n++) D = std::max(D, (int)tdep[n]);
    std::vector<int64_t> canon((size_t)N);
    for (uint32_t k = 0; k < S; k++) canon[k] = k;
    R->p.assign((size_t)N, MG_NO_NODE);
    R->q.assign((size_t)N, MG_NO_NODE);
    R->a.assign((size_t)N, 0);
    R->b.assign((size_t)N, 0);
    int64_t nextc = S;
    struct Key {
        uint32_t cp, cq;
        uint64_t a, b;
        int64_t t;
    };
    std::vector<Key> keys;
    for (int dd = 1; dd <= D; dd++) {
        keys.clear();
        for (int64_t n = S; n < N; n++)
            if ((int)tdep[n] == dd) keys.push_back({(uint32_t)canon[tp[n]], (uint32_t)canon[tq[n]], ta[n], tb[n], n});
        std::sort(keys.begin(), keys.end(), [](const Key& x, const Key& y) {
            if (x.cp != y.cp) return x.cp < y.cp;
            if (x.cq != y.cq) return x.cq < y.cq;
            if (x.a != y.a) return x.a < y.a;
            return x.b < y.b;
        });
        for (const Key& k : keys) {
            canon[k.t] = nextc;
            R->p[nextc] = k.cp;
            R->q[nextc] = k.cq;
            R->a[nextc] = k.a;
            R->b[nextc] = k.b;
            nextc++;
        }
    }
    R->N = N;
    R->D = D;
    for (int l = 1; l < L; l++) {
        const int64_t n = R->dims[l][0] * R->dims[l][1] * R->dims[l][2];
        R->mip[l].resize((size_t)n);
        for (int64_t v = 0; v < n; v++) R->mip[l][v] = (uint32_t)canon[roots[m0[l] + v]];
    }
    (void)capacity_total;
    return MG_OK;
}

}  // namespace
}  // namespace mg

using namespace mg;

extern "C" {

MG_API mg_status mg_factor_greedy(const void* ids, int64_t nx, int64_t ny, int64_t nz, uint32_t num_segments,
                                  const mg_build_opts* bopts, const mg_greedy_opts* opts, mg_stream stream,
                                  mg_greedy** out) {
    MG_RANGE("mg_factor_greedy");
    if (!out) return fail(MG_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!ids || !opts) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (nx < 1 || ny < 1 || nz < 1) return fail(MG_ERR_INVALID_ARG, "dims must be >= 1");
    if (nx > 65535 || ny > 65535 || nz > 65535 || (uint64_t)nx * ny * nz >= (1ull << 32))
        return fail(MG_ERR_UNSUPPORTED, "volume too large");
    if (num_segments < 1) return fail(MG_ERR_INVALID_ARG, "num_segments must be >= 1");
    const int id_bytes = bopts ? bopts->id_bytes : 2;
    if (id_bytes != 2 && id_bytes != 4) return fail(MG_ERR_INVALID_ARG, "id_bytes must be 2 or 4");
    if (opts->strategy != 1 && opts->strategy != 2) return fail(MG_ERR_INVALID_ARG, "strategy must be 1 or 2");
    if (opts->tau < 1) return fail(MG_ERR_INVALID_ARG, "tau must be >= 1");
    if (opts->bitrate < 0 || opts->bitrate > 16) return fail(MG_ERR_INVALID_ARG, "bitrate must be in 0..16");
    std::unique_ptr<mg_greedy> R(new (std::nothrow) mg_greedy());
    if (!R) return fail(MG_ERR_OOM, "host allocation failed");
    R->S = num_segments;
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const mg_status st = greedy_run(R.get(), ids, id_bytes, nx, ny, nz, *opts, s);
    cudaStreamSynchronize(s);
    if (st != MG_OK) return st;
    R->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = R.release();
    return MG_OK;
}

MG_API mg_status mg_greedy_info_get(const mg_greedy* r, mg_greedy_info* info) {
    if (!r || !info) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->num_segments = r->S;
    info->levels = r->L;
    info->depth = r->D;
    info->num_nodes = r->N;
    info->picks = (int64_t)r->picks.size() / 2;
    info->waves = r->waves;
    info->ms = r->ms;
    return MG_OK;
}

MG_API mg_status mg_greedy_copy_nodes(const mg_greedy* r, uint32_t* p, uint32_t* q, uint64_t* a, uint64_t* b) {
    if (!r) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    const size_t N = (size_t)r->N;
    if (p) std::memcpy(p, r->p.data(), N * 4);
    if (q) std::memcpy(q, r->q.data(), N * 4);
    if (a) std::memcpy(a, r->a.data(), N * 8);
    if (b) std::memcpy(b, r->b.data(), N * 8);
    return MG_OK;
}

MG_API mg_status mg_greedy_copy_mip(const mg_greedy* r, int level, uint32_t* dst) {
    if (!r || !dst) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (level < 0 || level >= r->L) return fail(MG_ERR_INVALID_ARG, "level out of range");
    std::memcpy(dst, r->mip[level].data(), r->mip[level].size() * 4);
    return MG_OK;
}

MG_API mg_status mg_greedy_copy_picks(const mg_greedy* r, uint32_t* picks) {
    if (!r || !picks) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    std::memcpy(picks, r->picks.data(), r->picks.size() * 4);
    return MG_OK;
}

MG_API mg_status mg_greedy_copy_codebook(const mg_greedy* r, double* codebook, double* sigma) {
    if (!r) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (codebook && !r->codebook.empty()) std::memcpy(codebook, r->codebook.data(), r->codebook.size() * 8);
    if (sigma && !r->sigma.empty()) std::memcpy(sigma, r->sigma.data(), r->sigma.size() * 8);
    return MG_OK;
}

MG_API void mg_greedy_free(mg_greedy* r) { delete r; }

}  // extern "C"

extern "C" MG_API mg_status mg_graph_from_greedy(const mg_greedy* r, const mg_allocator* allocator, mg_stream stream,
                                                mg_graph** out) {
    MG_RANGE("mg_graph_from_greedy");
    using namespace mg;
    if (!r || !out) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (r->codebook.empty()) return fail(MG_ERR_INVALID_ARG, "an exact greedy result: build with mg_build instead");
    if (r->D + 1 > MG_MAX_DEPTH) return fail(MG_ERR_UNSUPPORTED, "graph deeper than MG_MAX_DEPTH");
    std::unique_ptr<mg_graph> g(new (std::nothrow) mg_graph());
    if (!g) return fail(MG_ERR_OOM, "host allocation failed");
    if (allocator) {
        if (!allocator->alloc || !allocator->free) return fail(MG_ERR_INVALID_ARG, "allocator needs alloc and free");
        g->al.a = *allocator;
        g->al.custom = true;
    }
    MG_CUDA(cudaGetDevice(&g->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t N = r->N;
    const uint32_t S = r->S;
    g->S = S;
    g->N = N;
    g->L = r->L;
    g->D = r->D;
    g->quantised = true;
    g->geom.L = r->L;
    int64_t hi = 0;
    for (int l = 0; l < r->L; l++) {
        for (int k = 0; k < 3; k++) g->geom.dims[l][k] = (int32_t)r->dims[l][k];
        if (l >= 1) {
            g->geom.off[l] = hi;
            hi += (int64_t)r->mip[l].size();
        }
    }
    // depth buckets of the canonical numbering
    std::vector<int> depth((size_t)N, 0);
    for (int64_t n = S; n < N; n++) depth[n] = std::max(depth[r->p[n]], depth[r->q[n]]) + 1;
    g->bucket[0] = 0;
    for (int d = 0; d <= r->D; d++) {
        int64_t c = 0;
        for (int64_t n = 0; n < N; n++) c += depth[n] == d;
        g->bucket[d + 1] = g->bucket[d] + c;
    }
    g->id0_bytes = S <= 65536u ? 2 : 4;
    const size_t V0 = r->mip[0].size();
    MG_TRY(g->mip0.alloc(&g->al, V0 * g->id0_bytes, s));
    if (g->id0_bytes == 2) {
        std::vector<uint16_t> v16(V0);
        for (size_t i = 0; i < V0; i++) v16[i] = (uint16_t)r->mip[0][i];
        MG_CUDA(cudaMemcpyAsync(g->mip0.p, v16.data(), V0 * 2, cudaMemcpyHostToDevice, s));
        MG_CUDA(cudaStreamSynchronize(s));
    } else {
        MG_CUDA(cudaMemcpyAsync(g->mip0.p, r->mip[0].data(), V0 * 4, cudaMemcpyHostToDevice, s));
    }
    if (hi > 0) {
        MG_TRY(g->mip.alloc(&g->al, (size_t)hi * 4, s));
        for (int l = 1; l < r->L; l++)
            MG_CUDA(cudaMemcpyAsync(g->mip.as<uint32_t>() + g->geom.off[l], r->mip[l].data(), r->mip[l].size() * 4,
                                    cudaMemcpyHostToDevice, s));
    }
    std::vector<uint2> pq((size_t)N);
    std::vector<float> alpha((size_t)N, 0.f);
    std::vector<double> wq((size_t)N, 0.0), dw((size_t)N, 0.0);
    for (int64_t n = 0; n < N; n++) {
        pq[n] = make_uint2(r->p[n], r->q[n]);
        if (n >= (int64_t)S) {
            wq[n] = r->codebook[r->a[n]];
            dw[n] = r->sigma[r->a[n]];
            alpha[n] = (float)wq[n];
        }
    }
    MG_TRY(g->pq.alloc(&g->al, (size_t)N * 8, s));
    MG_TRY(g->ab.alloc(&g->al, (size_t)N * 16, s));
    MG_TRY(g->ab32.alloc(&g->al, (size_t)N * 8, s));
    MG_TRY(g->alpha.alloc(&g->al, (size_t)N * 4, s));
    MG_TRY(g->wq.alloc(&g->al, (size_t)N * 8, s));
    MG_TRY(g->dw.alloc(&g->al, (size_t)N * 8, s));
    MG_TRY(g->status.alloc(&g->al, 4, s));
    MG_CUDA(cudaMemcpyAsync(g->pq.p, pq.data(), (size_t)N * 8, cudaMemcpyHostToDevice, s));
    MG_CUDA(cudaMemsetAsync(g->ab.p, 0, (size_t)N * 16, s));
    MG_CUDA(cudaMemsetAsync(g->ab32.p, 0, (size_t)N * 8, s));
    MG_CUDA(cudaMemcpyAsync(g->alpha.p, alpha.data(), (size_t)N * 4, cudaMemcpyHostToDevice, s));
    MG_CUDA(cudaMemcpyAsync(g->wq.p, wq.data(), (size_t)N * 8, cudaMemcpyHostToDevice, s));
    MG_CUDA(cudaMemcpyAsync(g->dw.p, dw.data(), (size_t)N * 8, cudaMemcpyHostToDevice, s));
    MG_CUDA(cudaMemsetAsync(g->status.p, 0, 4, s));
    MG_TRY(build_query_copies(g.get(), s));
    MG_CUDA(cudaStreamSynchronize(s));   // the host staging above is freed on return
    for (Buf* b : {&g->mip0, &g->mip, &g->pq, &g->ab, &g->ab32, &g->alpha, &g->wq, &g->dw, &g->status}) b->s = nullptr;
    for (int c = 0; c < 3; c++) g->mip0x[c].s = g->mipx[c].s = nullptr;
    *out = g.release();
    return MG_OK;
}
