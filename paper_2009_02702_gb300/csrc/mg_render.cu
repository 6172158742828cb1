// mg_render.cu -- ray-sample node lookup (Sec. 4: rendering from the Mixture
// Graph is a paletted lookup).  One thread per sample: pick the level nearest
// to the sample's LOD, the voxel containing the sample at that level, read its
// node ID and copy the node's value row.  The level and voxel are decided in
// fp32, the precision of the samples.
#include "mg_internal.cuh"

namespace mg {
namespace {

struct Geom {
    int L;
    int id0_bytes;
    int32_t dims[MG_MAX_LEVELS][3];
    int64_t off[MG_MAX_LEVELS];
};

__device__ __forceinline__ int64_t floor_coord(float x, int32_t d0) {
    float xc = x;
    if (!(xc >= 0.f)) xc = 0.f;                  // negatives and NaN
    if (xc > (float)d0) xc = (float)d0;
    return (int64_t)xc;                         // truncation is the floor for xc >= 0
}

// 128-thread CTAs of at most 32 registers a thread: one fits beside a
// persistent query kernel that leaves 4,096 registers of an SM free, so a
// lookup issued on another stream runs concurrently with it
constexpr int kLookupThreads = 128;

template <typename RowT>
__global__ void __launch_bounds__(kLookupThreads, 16) lookup_kernel(Geom G, const void* __restrict__ mip0, const uint32_t* __restrict__ mip,
                              const float4* __restrict__ samples, int64_t P, const RowT* __restrict__ vals,
                              int words, RowT* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float4 smp = __ldg(samples + i);
    const float t = smp.w + 0.5f;                 // nearest level
    int l;
    if (!(t >= 0.f)) l = 0;
    else if (t >= (float)(G.L - 1)) l = G.L - 1;
    else l = (int)t;
    int64_t v[3];
    const float c[3] = {smp.x, smp.y, smp.z};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int64_t x = floor_coord(c[k], G.dims[0][k]) >> l;
        v[k] = min(x, (int64_t)G.dims[l][k] - 1);
    }
    const int64_t idx = (v[2] * G.dims[l][1] + v[1]) * G.dims[l][0] + v[0];
    uint32_t node;
    if (l == 0)
        node = G.id0_bytes == 2 ? (uint32_t)__ldg(static_cast<const uint16_t*>(mip0) + idx)
                                : __ldg(static_cast<const uint32_t*>(mip0) + idx);
    else
        node = __ldg(mip + G.off[l] + idx);
    const RowT* src = vals + (int64_t)node * words;
    RowT* dst = out + i * words;
    for (int w = 0; w < words; w++) dst[w] = __ldg(src + w);
}

// k frames in one launch: samples [off[j], off[j+1]) belong to frame j and
// read the j-th slice of `words` words of every value row (rows of k slices,
// the layout of a k-TF propagation)
constexpr int kMaxFrames = 32;
struct FrameOffsets {
    int64_t off[kMaxFrames + 1];
};

template <typename RowT>
__global__ void __launch_bounds__(kLookupThreads, 16) lookup_multi_kernel(Geom G, const void* __restrict__ mip0,
                                                                          const uint32_t* __restrict__ mip,
                                                                          const float4* __restrict__ samples,
                                                                          FrameOffsets F, int k,
                                                                          const RowT* __restrict__ vals, int words,
                                                                          RowT* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= F.off[k]) return;
    int j = 0;
    while (j + 1 < k && F.off[j + 1] <= i) j++;
    const float4 smp = __ldg(samples + i);
    const float t = smp.w + 0.5f;
    int l;
    if (!(t >= 0.f)) l = 0;
    else if (t >= (float)(G.L - 1)) l = G.L - 1;
    else l = (int)t;
    int64_t v[3];
    const float c[3] = {smp.x, smp.y, smp.z};
#pragma unroll
    for (int a = 0; a < 3; a++) {
        const int64_t x = floor_coord(c[a], G.dims[0][a]) >> l;
        v[a] = min(x, (int64_t)G.dims[l][a] - 1);
    }
    const int64_t idx = (v[2] * G.dims[l][1] + v[1]) * G.dims[l][0] + v[0];
    uint32_t node;
    if (l == 0)
        node = G.id0_bytes == 2 ? (uint32_t)__ldg(static_cast<const uint16_t*>(mip0) + idx)
                                : __ldg(static_cast<const uint32_t*>(mip0) + idx);
    else
        node = __ldg(mip + G.off[l] + idx);
    const RowT* src = vals + ((int64_t)node * k + j) * words;
    RowT* dst = out + i * words;
    for (int w = 0; w < words; w++) dst[w] = __ldg(src + w);
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

Geom render_geom(const mg_graph* g) {
    Geom G;
    G.L = g->L;
    G.id0_bytes = g->id0_bytes;
    for (int l = 0; l < MG_MAX_LEVELS; l++) {
        for (int a = 0; a < 3; a++) G.dims[l][a] = g->geom.dims[l][a];
        G.off[l] = g->geom.off[l];
    }
    return G;
}

}  // namespace

mg_status render_lookup_multi(const mg_graph* g, const void* vals, int k, int C, mg_dtype dt, const float* samples,
                              const int64_t* offsets, void* out, cudaStream_t s) {
    if (k < 1 || k > kMaxFrames) return fail(MG_ERR_INVALID_ARG, "k must be 1..32 frames");
    if (!aligned(samples, 16)) return fail(MG_ERR_INVALID_ARG, "samples must be 16-byte aligned");
    FrameOffsets F;
    for (int j = 0; j <= kMaxFrames; j++) F.off[j] = offsets[j <= k ? j : k];
    if (F.off[0] != 0) return fail(MG_ERR_INVALID_ARG, "offsets[0] must be 0");
    for (int j = 0; j < k; j++)
        if (F.off[j + 1] < F.off[j]) return fail(MG_ERR_INVALID_ARG, "offsets must be non-decreasing");
    const int64_t P = F.off[k];
    if (P == 0) return MG_OK;
    const Geom G = render_geom(g);
    const size_t row = (size_t)C * (dt == MG_F32 ? 4 : 2);
    const unsigned grid = grid_for(P, kLookupThreads);
    const float4* sm = reinterpret_cast<const float4*>(samples);
    const uint32_t* mip = g->mip.as<uint32_t>();
    if (row % 16 == 0 && aligned(vals, 16) && aligned(out, 16))
        lookup_multi_kernel<uint4><<<grid, kLookupThreads, 0, s>>>(G, g->mip0.p, mip, sm, F, k, (const uint4*)vals,
                                                                  (int)(row / 16), (uint4*)out);
    else if (row % 8 == 0 && aligned(vals, 8) && aligned(out, 8))
        lookup_multi_kernel<uint2><<<grid, kLookupThreads, 0, s>>>(G, g->mip0.p, mip, sm, F, k, (const uint2*)vals,
                                                                  (int)(row / 8), (uint2*)out);
    else if (row % 4 == 0 && aligned(vals, 4) && aligned(out, 4))
        lookup_multi_kernel<uint32_t><<<grid, kLookupThreads, 0, s>>>(G, g->mip0.p, mip, sm, F, k,
                                                                     (const uint32_t*)vals, (int)(row / 4),
                                                                     (uint32_t*)out);
    else
        lookup_multi_kernel<uint16_t><<<grid, kLookupThreads, 0, s>>>(G, g->mip0.p, mip, sm, F, k,
                                                                     (const uint16_t*)vals, (int)(row / 2),
                                                                     (uint16_t*)out);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

mg_status render_lookup(const mg_graph* g, const void* vals, int C, mg_dtype dt, const float* samples, int64_t P,
                        void* out, cudaStream_t s) {
    if (!aligned(samples, 16)) return fail(MG_ERR_INVALID_ARG, "samples must be 16-byte aligned");
    const Geom G = render_geom(g);
    const size_t row = (size_t)C * (dt == MG_F32 ? 4 : 2);
    const unsigned grid = grid_for(P, kLookupThreads);
    const float4* sm = reinterpret_cast<const float4*>(samples);
    const uint32_t* mip = g->mip.as<uint32_t>();
    if (row % 16 == 0 && aligned(vals, 16) && aligned(out, 16))
        lookup_kernel<uint4><<<grid, kLookupThreads, 0, s>>>(G, g->mip0.p, mip, sm, P, (const uint4*)vals, (int)(row / 16),
                                                  (uint4*)out);
    else if (row % 8 == 0 && aligned(vals, 8) && aligned(out, 8))
        lookup_kernel<uint2><<<grid, kLookupThreads, 0, s>>>(G, g->mip0.p, mip, sm, P, (const uint2*)vals, (int)(row / 8),
                                                  (uint2*)out);
    else if (row % 4 == 0 && aligned(vals, 4) && aligned(out, 4))
        lookup_kernel<uint32_t><<<grid, kLookupThreads, 0, s>>>(G, g->mip0.p, mip, sm, P, (const uint32_t*)vals,
                                                     (int)(row / 4), (uint32_t*)out);
    else
        lookup_kernel<uint16_t><<<grid, kLookupThreads, 0, s>>>(G, g->mip0.p, mip, sm, P, (const uint16_t*)vals,
                                                     (int)(row / 2), (uint16_t*)out);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

}  // namespace mg
