// mg_lut.cu -- the mixture lookup table of the range queries (Sec. 3.6: one
// mixture per node, summed over the footprint's samples; Sec. 5.2: built once
// per data set by propagating unit vectors through the DAG).
//
// Exact integer form.  A node that is the ID of some voxel at levels
// 1..kLutMaxLevel gets its mixture as integer counts over its sources, scaled
// to 8^lmin, lmin the lowest level at which the node is a voxel ID: the counts
// are what the exact push of weight 8^lmin through the node's lerp tree
// delivers to each source (Sec. 3.2's factor trees have distinct sources as
// leaves, so the tree has exactly one leaf per mixture entry).  A query cube
// at level l >= lmin with run count k carries W = k * 8^l and adds
// (W >> 3 lmin) * count to each source -- the same integers the push would
// produce, without walking the tree.
//
// Layout: meta[n] = (first entry, entries << 8 | lmin), zero for nodes without
// a table; entries are (source, count) pairs, uint2.
#include "mg_internal.cuh"

#include <algorithm>

namespace mg {
namespace {

constexpr int kLutMaxLevel = 10;   // 8^10 = 2^30: counts and weights stay in uint32

__global__ void lut_lmin_kernel(const uint32_t* __restrict__ ids, int64_t n, uint32_t S, uint32_t l,
                                uint32_t* __restrict__ lmin) {
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t id = __ldg(ids + v);
        if (id >= S && id != kNone) atomicMin(lmin + id, l);
    }
}

// leaves of a node = leaves of p + leaves of q; nodes of one topological level
__global__ void lut_leaves_kernel(const uint2* __restrict__ pq, int64_t lo, int64_t hi, uint32_t* __restrict__ leaves) {
    for (int64_t n = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < hi; n += (int64_t)gridDim.x * blockDim.x) {
        const uint2 e = pq[n];
        leaves[n] = leaves[e.x] + leaves[e.y];
    }
}

__global__ void lut_ones_kernel(uint32_t* __restrict__ a, uint32_t n) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = 1u;
}

__global__ void lut_size_kernel(int64_t N, uint32_t S, const uint32_t* __restrict__ lmin,
                                const uint32_t* __restrict__ leaves, uint64_t* __restrict__ size) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x)
        size[n] = (n >= S && lmin[n] <= (uint32_t)kLutMaxLevel && leaves[n] < (1u << 24)) ? leaves[n] : 0u;
}

// one thread per tabled node: exact push of 8^lmin through its lerp tree
// (p receives W*a/(a+b), q the rest), the leaves written in visiting order
__global__ void lut_fill_kernel(int64_t N, uint32_t S, const uint2* __restrict__ pq, const uint2* __restrict__ ab32,
                                const uint32_t* __restrict__ lmin, const uint64_t* __restrict__ off,
                                const uint64_t* __restrict__ size, uint2* __restrict__ lut, uint2* __restrict__ meta,
                                unsigned* __restrict__ status) {
    constexpr int kStack = 64;
    for (int64_t n0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n0 < N; n0 += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t len = size[n0];
        if (len == 0) {
            meta[n0] = make_uint2(0u, 0u);
            continue;
        }
        const uint32_t l = lmin[n0];
        uint2* out = lut + off[n0];
        uint32_t sn[kStack], sw[kStack];
        int sp = 0;
        uint32_t n = (uint32_t)n0, w = 1u << (3 * l);
        uint64_t k = 0;
        bool ok = true;
        for (;;) {
            if (n < S) {
                if (k < len) out[k] = make_uint2(n, w);
                k++;
                if (sp == 0) break;
                --sp;
                n = sn[sp];
                w = sw[sp];
                continue;
            }
            const uint2 e = pq[n];
            const uint2 ab = ab32[n];
            const uint32_t t = ab.x + ab.y;
            const uint32_t q = t ? w / t : 0u;
            if (t == 0 || q * t != w || sp >= kStack) {
                ok = false;
                break;
            }
            sn[sp] = e.y;
            sw[sp] = q * ab.y;
            sp++;
            n = e.x;
            w = q * ab.x;
        }
        if (!ok || k != len) {
            set_status(status, kStatInexact);
            meta[n0] = make_uint2(0u, 0u);
            continue;
        }
        meta[n0] = make_uint2((uint32_t)off[n0], (uint32_t)(len << 8) | l);
    }
}

unsigned grid_of(int64_t n) { return grid_for(n, 256, 152 * 32); }

}  // namespace

mg_status build_lut(mg_graph* g, cudaStream_t s) {
    const int64_t N = g->N;
    const uint32_t S = g->S;
    g->lut_entries = 0;
    if (N <= (int64_t)S || g->L < 2) return MG_OK;   // no internal nodes
    const Alloc& al = g->al;
    Buf lmin, leaves, size, off;
    MG_TRY(lmin.alloc(&al, (size_t)N * 4, s));
    MG_TRY(leaves.alloc(&al, (size_t)N * 4, s));
    MG_TRY(size.alloc(&al, (size_t)N * 8, s));
    MG_TRY(off.alloc(&al, (size_t)(N + 1) * 8, s));
    MG_CUDA(cudaMemsetAsync(lmin.p, 0xFF, (size_t)N * 4, s));
    for (int l = 1; l < g->L && l <= kLutMaxLevel; l++) {
        const int64_t nv = (int64_t)g->geom.dims[l][0] * g->geom.dims[l][1] * g->geom.dims[l][2];
        lut_lmin_kernel<<<grid_of(nv), 256, 0, s>>>(g->mip.as<uint32_t>() + g->geom.off[l], nv, S, (uint32_t)l,
                                                    lmin.as<uint32_t>());
        MG_CUDA(cudaGetLastError());
    }
    // sources have one leaf; nodes of level d only read levels < d
    lut_ones_kernel<<<grid_of(S), 256, 0, s>>>(leaves.as<uint32_t>(), S);
    MG_CUDA(cudaGetLastError());
    for (int d = 1; d <= g->D; d++) {
        const int64_t lo = g->bucket[d], hi = g->bucket[d + 1];
        if (hi <= lo) continue;
        lut_leaves_kernel<<<grid_of(hi - lo), 256, 0, s>>>(g->pq.as<uint2>(), lo, hi, leaves.as<uint32_t>());
        MG_CUDA(cudaGetLastError());
    }
    lut_size_kernel<<<grid_of(N), 256, 0, s>>>(N, S, lmin.as<uint32_t>(), leaves.as<uint32_t>(), size.as<uint64_t>());
    MG_CUDA(cudaGetLastError());
    MG_TRY(scan_exclusive_u64(size.as<uint64_t>(), off.as<uint64_t>(), N, off.as<uint64_t>() + N, al, s));
    uint64_t total = 0;
    MG_CUDA(cudaMemcpyAsync(&total, off.as<uint64_t>() + N, 8, cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    if (total >= (1ull << 32)) return MG_OK;   // too large to index with uint32: queries walk the trees
    MG_TRY(g->lut_meta.alloc(&al, (size_t)N * sizeof(uint2), s));
    MG_TRY(g->lut.alloc(&al, (size_t)std::max<uint64_t>(total, 1) * sizeof(uint2), s));
    lut_fill_kernel<<<grid_of(N), 256, 0, s>>>(N, S, g->pq.as<uint2>(), g->ab32.as<uint2>(), lmin.as<uint32_t>(),
                                               off.as<uint64_t>(), size.as<uint64_t>(), g->lut.as<uint2>(),
                                               g->lut_meta.as<uint2>(), g->status.as<unsigned>());
    MG_CUDA(cudaGetLastError());
    g->lut_entries = (int64_t)total;
    return MG_OK;
}

}  // namespace mg
