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

// ---------------------------------------------------------------------------
// Ray marching through the node values (Sec. 4): for every pixel a ray from
// the camera through the volume, samples on the lattice t_k = t_start +
// k * base; a sample's LOD, floor(log2(t * pixel angle)) + bias, picks level m
// (clamped to the pyramid) and the step 2^m * base (the step adjusted to the
// LOD, with opacity correction alpha' = 1 - (1 - alpha)^(2^m)); its value is
// trilinear within level m between the 8 voxel centres around it and linear
// between levels m and m+1 by the fractional LOD; front-to-back compositing
// stops at the early-termination opacity.  With node opacities (the TF's
// alpha propagated through the graph), empty space is skipped: climbing from
// level m+2 while the voxel around the sample has opacity exactly 0, the
// lattice samples inside the largest such voxel shrunk by the reach of the
// interpolation (3 * 2^m: levels m and m+1 read voxels within 1.5 of their
// widths of the sample), and before the next LOD change, are skipped; each
// would add exactly nothing, so the image is the same with and without it.
// Decisions (lattice, level, skip, termination) use one rounding per fp32
// operation (no contraction), so they are reproducible off the GPU.
// ---------------------------------------------------------------------------
namespace mg {
namespace {

struct MarchArgs {
    Geom G;
    const void* mip0;
    const uint32_t* mip;
    const float4* vals;
    const float* opac;
    const uint32_t* occ;              // occupancy bits of levels >= 2 (skipping on)
    int64_t occ_off[MG_MAX_LEVELS];   // first word of every level's bits
    mg_camera cam;
    float4* img;
    int32_t* steps;
};

__device__ __forceinline__ uint32_t march_node(const MarchArgs& A, int l, int64_t x, int64_t y, int64_t z) {
    const int64_t idx = (z * A.G.dims[l][1] + y) * A.G.dims[l][0] + x;
    if (l == 0)
        return A.G.id0_bytes == 2 ? (uint32_t)__ldg(static_cast<const uint16_t*>(A.mip0) + idx)
                                  : __ldg(static_cast<const uint32_t*>(A.mip0) + idx);
    return __ldg(A.mip + A.G.off[l] + idx);
}

// voxel of level l holding coordinate x of axis c (clamped to the level)
__device__ __forceinline__ int64_t march_voxel(const MarchArgs& A, int l, float x, int c) {
    int64_t v = (int64_t)floorf(x);
    v = v < 0 ? 0 : v;
    v >>= l;
    return v > A.G.dims[l][c] - 1 ? A.G.dims[l][c] - 1 : v;
}

__device__ __forceinline__ int64_t march_index(const MarchArgs& A, int l, const int64_t (&b)[3]) {
    return (b[2] * A.G.dims[l][1] + b[1]) * A.G.dims[l][0] + b[0];
}

__device__ __forceinline__ float rn_lerp(float a, float b, float f) { return __fadd_rn(a, __fmul_rn(f, __fsub_rn(b, a))); }

__device__ __forceinline__ float4 lerp4(float4 a, float4 b, float f) {
    return make_float4(rn_lerp(a.x, b.x, f), rn_lerp(a.y, b.y, f), rn_lerp(a.z, b.z, f), rn_lerp(a.w, b.w, f));
}

// trilinear value of level l at p (level-0 units), voxel centres clamped to the level
__device__ float4 march_tri(const MarchArgs& A, int l, const float (&p)[3]) {
    const float scale = ldexpf(1.0f, -l);
    int64_t i0[3], i1[3];
    float f[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float u = __fsub_rn(__fmul_rn(p[c], scale), 0.5f);
        const float fl = floorf(u);
        f[c] = __fsub_rn(u, fl);
        const int64_t k = (int64_t)fl, d = A.G.dims[l][c];
        i0[c] = k < 0 ? 0 : (k > d - 1 ? d - 1 : k);
        i1[c] = k + 1 < 0 ? 0 : (k + 1 > d - 1 ? d - 1 : k + 1);
    }
    uint32_t n[8];
#pragma unroll
    for (int corner = 0; corner < 8; corner++)
        n[corner] = march_node(A, l, corner & 1 ? i1[0] : i0[0], corner & 2 ? i1[1] : i0[1], corner & 4 ? i1[2] : i0[2]);
    float4 v[8];
#pragma unroll
    for (int corner = 0; corner < 8; corner++) v[corner] = __ldg(A.vals + n[corner]);
    const float4 x00 = lerp4(v[0], v[1], f[0]), x10 = lerp4(v[2], v[3], f[0]);
    const float4 x01 = lerp4(v[4], v[5], f[0]), x11 = lerp4(v[6], v[7], f[0]);
    return lerp4(lerp4(x00, x10, f[1]), lerp4(x01, x11, f[1]), f[2]);
}

constexpr int kPreload = 1;   // climb levels whose bits are loaded up front (1 measured best of 1, 2, 3, 5)

__global__ void __launch_bounds__(128) march_kernel(MarchArgs A) {
    const mg_camera& cam = A.cam;
    const int i = blockIdx.x * blockDim.x + threadIdx.x, j = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= cam.width || j >= cam.height) return;
    const int L = A.G.L;
    const float inf = 3.0e38f;
    const float sx = __fmul_rn(__fsub_rn(__fadd_rn((float)i, 0.5f), __fmul_rn(0.5f, (float)cam.width)), cam.pix);
    const float sy = __fmul_rn(__fsub_rn(__fsub_rn(__fmul_rn(0.5f, (float)cam.height), (float)j), 0.5f), cam.pix);
    float d[3];
#pragma unroll
    for (int c = 0; c < 3; c++)
        d[c] = __fadd_rn(__fadd_rn(cam.fwd[c], __fmul_rn(sx, cam.right[c])), __fmul_rn(sy, cam.up[c]));
    const float nrm = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(d[0], d[0]), __fmul_rn(d[1], d[1])), __fmul_rn(d[2], d[2])));
#pragma unroll
    for (int c = 0; c < 3; c++) d[c] = __fdiv_rn(d[c], nrm);
    float tmin = -inf, tmax = inf;
    bool miss = false;
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const float dim = (float)A.G.dims[0][c];
        if (d[c] == 0.0f) {
            if (cam.eye[c] < 0.0f || cam.eye[c] > dim) miss = true;
            continue;
        }
        const float t0 = __fdiv_rn(__fsub_rn(0.0f, cam.eye[c]), d[c]), t1 = __fdiv_rn(__fsub_rn(dim, cam.eye[c]), d[c]);
        const float lo = t0 < t1 ? t0 : t1, hi = t0 < t1 ? t1 : t0;
        if (lo > tmin) tmin = lo;
        if (hi < tmax) tmax = hi;
    }
    const float ts = tmin > 0.0f ? tmin : 0.0f;
    float C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, Aacc = 0.0f;
    int32_t taken = 0;
    if (!miss && tmax > ts) {
        int64_t k = 0;
        while (k < cam.max_steps) {
            const float t = __fadd_rn(ts, __fmul_rn((float)k, cam.base_step));
            if (!(t < tmax)) break;
            const float x = __fmul_rn(t, cam.pix);
            const int lam = x > 0.0f ? ilogbf(x) + cam.lod_bias : -1000000;
            const int m = lam < 0 ? 0 : (lam > L - 1 ? L - 1 : lam);
            float fr = 0.0f;
            if (lam >= 0 && m < L - 1) {
                fr = __fsub_rn(__fadd_rn(log2f(x), (float)cam.lod_bias), (float)lam);
                fr = fr < 0.0f ? 0.0f : (fr > 1.0f ? 1.0f : fr);
            }
            float p[3];
#pragma unroll
            for (int c = 0; c < 3; c++) p[c] = __fadd_rn(cam.eye[c], __fmul_rn(t, d[c]));
            // the occupancy bits of the climb's first kPreload levels are
            // loaded before the sample's own values, so that these loads and
            // the sample's two dependent ones overlap; most climbs stop
            // within them
            uint32_t pre = 0;   // bit j: level m + 2 + j occupied
            const bool climb = A.occ && m + 2 < L;
            if (climb) {
#pragma unroll
                for (int j = 0; j < kPreload; j++) {
                    const int jl = m + 2 + j;
                    if (jl >= L) break;
                    int64_t b[3];
#pragma unroll
                    for (int c = 0; c < 3; c++) b[c] = march_voxel(A, jl, p[c], c);
                    const int64_t vi = march_index(A, jl, b);
                    pre |= ((__ldg(A.occ + A.occ_off[jl] + (vi >> 5)) >> (vi & 31)) & 1u) << j;
                }
            }
            float4 s = march_tri(A, m, p);
            if (fr > 0.0f) s = lerp4(s, march_tri(A, m + 1, p), fr);
            if (climb) {
                int jz = -1;
                int64_t bz[3] = {0, 0, 0};
                for (int jl = m + 2; jl < L; jl++) {
                    int64_t b[3];
#pragma unroll
                    for (int c = 0; c < 3; c++) b[c] = march_voxel(A, jl, p[c], c);
                    const int64_t vi = march_index(A, jl, b);
                    const bool occ = jl < m + 2 + kPreload
                                         ? ((pre >> (jl - m - 2)) & 1u)
                                         : ((__ldg(A.occ + A.occ_off[jl] + (vi >> 5)) >> (vi & 31)) & 1u);
                    if (occ) break;
                    jz = jl;
#pragma unroll
                    for (int c = 0; c < 3; c++) bz[c] = b[c];
                }
                if (jz >= 0) {
                    const float size = ldexpf(1.0f, jz), gap = ldexpf(3.0f, m);
                    float lo[3], hi[3];
                    bool inside = true;
#pragma unroll
                    for (int c = 0; c < 3; c++) {
                        lo[c] = __fadd_rn(__fmul_rn((float)bz[c], size), gap);
                        hi[c] = __fsub_rn(__fmul_rn(__fadd_rn((float)bz[c], 1.0f), size), gap);
                        if (!(p[c] > lo[c] && p[c] < hi[c])) inside = false;
                    }
                    if (inside) {
                        float tout = inf;
#pragma unroll
                        for (int c = 0; c < 3; c++) {
                            const float te = d[c] > 0.0f ? __fdiv_rn(__fsub_rn(hi[c], cam.eye[c]), d[c])
                                             : d[c] < 0.0f ? __fdiv_rn(__fsub_rn(lo[c], cam.eye[c]), d[c]) : inf;
                            if (te < tout) tout = te;
                        }
                        const float tch = m < L - 1 ? __fdiv_rn(ldexpf(1.0f, lam + 1 - cam.lod_bias), cam.pix) : inf;
                        const float tl = tout < tch ? tout : tch;
                        const float len = __fmul_rn((float)((int64_t)1 << m), cam.base_step);
                        const int64_t n = (int64_t)floorf(__fdiv_rn(__fsub_rn(tl, t), len)) - 1;
                        if (n >= 1) {
                            k += n << m;
                            continue;
                        }
                    }
                }
            }
            float q = __fsub_rn(1.0f, s.w);
            for (int e = 0; e < m; e++) q = __fmul_rn(q, q);
            const float ap = __fsub_rn(1.0f, q);
            const float w = __fmul_rn(__fsub_rn(1.0f, Aacc), ap);
            C0 = __fadd_rn(C0, __fmul_rn(w, s.x));
            C1 = __fadd_rn(C1, __fmul_rn(w, s.y));
            C2 = __fadd_rn(C2, __fmul_rn(w, s.z));
            Aacc = __fadd_rn(Aacc, w);
            taken++;
            if (cam.ert <= 1.0f && Aacc >= cam.ert) break;
            k += (int64_t)1 << m;
        }
    }
    const int64_t o = (int64_t)j * cam.width + i;
    A.img[o] = make_float4(C0, C1, C2, Aacc);
    if (A.steps) A.steps[o] = taken;
}

// bit v of a level's words: the opacity of voxel v's node is non-zero (one
// lane per voxel, a warp's ballot is one word)
__global__ void occ_bits_kernel(const uint32_t* __restrict__ ids, int64_t n, const float* __restrict__ opac,
                                uint32_t* __restrict__ words) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x; i0 < n; i0 += stride) {
        const int64_t i = i0 + threadIdx.x;
        const bool occ = i < n && __ldg(opac + __ldg(ids + i)) != 0.0f;
        const unsigned w = __ballot_sync(0xffffffffu, occ);
        if ((threadIdx.x & 31) == 0 && i < n) words[i >> 5] = w;
    }
}

}  // namespace

mg_status raymarch(const mg_graph* g, const float* vals, const float* opacity, const mg_camera& cam, float* image,
                   int32_t* steps, cudaStream_t s) {
    if (!aligned(vals, 16) || !aligned(image, 16)) return fail(MG_ERR_INVALID_ARG, "vals and image must be 16-byte aligned");
    MarchArgs A;
    A.G = render_geom(g);
    A.mip0 = g->mip0.p;
    A.mip = g->mip.as<uint32_t>();
    A.vals = reinterpret_cast<const float4*>(vals);
    A.opac = opacity;
    A.occ = nullptr;
    for (int l = 0; l < MG_MAX_LEVELS; l++) A.occ_off[l] = 0;
    if (opacity) {
        // the climbs of empty-space skipping read one bit per voxel of levels
        // >= 2 (built here, in the graph's per-stream scratch) instead of a
        // node ID and its opacity
        int64_t words = 0;
        for (int l = 2; l < g->L; l++) {
            A.occ_off[l] = words;
            words += ((int64_t)A.G.dims[l][0] * A.G.dims[l][1] * A.G.dims[l][2] + 31) / 32;
        }
        if (words > 0) {
            Arena* arena = nullptr;
            MG_TRY(arena_begin(const_cast<mg_graph*>(g), s, &arena));
            Buf bits;
            MG_TRY(bits.alloc(&arena->view, (size_t)words * 4, s));
            for (int l = 2; l < g->L; l++) {
                const int64_t n = (int64_t)A.G.dims[l][0] * A.G.dims[l][1] * A.G.dims[l][2];
                occ_bits_kernel<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(g->mip.as<uint32_t>() + A.G.off[l], n, opacity,
                                                                           bits.as<uint32_t>() + A.occ_off[l]);
                MG_CUDA(cudaGetLastError());
            }
            A.occ = bits.as<uint32_t>();
        }
    }
    A.cam = cam;
    A.img = reinterpret_cast<float4*>(image);
    A.steps = steps;
    const dim3 block(16, 8);
    const dim3 grid((unsigned)((cam.width + 15) / 16), (unsigned)((cam.height + 7) / 8));
    march_kernel<<<grid, block, 0, s>>>(A);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

}  // namespace mg
