// mg_bitstream.cu -- the graph as the bitstream of Table 1 (Sec. 3.3,
// Eq. 14-15) and the ray-sample lookup decoding it in place (Sec. 4: the
// voxel data are read by bit address).
//
// Layout (bit i of the stream is bit i % 8 of byte i / 8; every field least
// significant bit first): (1) sources, 32 bits; (2) fractional input, 1 bit;
// (3) bits per node ID minus one, 6 bits (nb = ceil(log2 N)); (4) sigma_max,
// 32 bits (0: no quantiser); (5) resolution, 3 x 32 bits; (6) quantisation
// bitrate minus one, 4 bits; (7) internal nodes, nb bits; then the lossless
// extension -- one bit "exact weights" and six bits w - 1 -- since the exact
// graph keeps coprime integer weights a:b instead of codebook indices; per
// level (8) its voxel bits r(l) and (9) i_min(l), nb bits each; (A) every
// level's node IDs x fastest as ID - i_min(l) at r(l) bits, r(l) =
// ceil(log2(i_max(l) - i_min(l) + 1)); (B) every internal node's p and q at
// nb bits and a and b at w bits; zero padding to a multiple of 8 bytes.
#include "mg_internal.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

namespace mg {
namespace {

int bits_for(uint64_t range) {   // ceil(log2(range)), range >= 1
    int b = 0;
    while (b < 64 && (1ull << b) < range) b++;
    return b;
}

struct Layout {
    int nb = 1, wbits = 1, L = 0;
    uint32_t S = 0;
    int64_t N = 0;
    int64_t dims[MG_MAX_LEVELS][3];
    int32_t r[MG_MAX_LEVELS];
    uint32_t imin[MG_MAX_LEVELS];
    int64_t level_bit[MG_MAX_LEVELS];
    int64_t node_bit = 0, total_bits = 0, bytes = 0, header_bits = 0;
};

void finish_layout(Layout& Y) {
    int64_t bit = 32 + 1 + 6 + 32 + 96 + 4 + Y.nb + 1 + 6 + (int64_t)Y.L * 2 * Y.nb;
    Y.header_bits = bit;
    for (int l = 0; l < Y.L; l++) {
        Y.level_bit[l] = bit;
        bit += Y.dims[l][0] * Y.dims[l][1] * Y.dims[l][2] * Y.r[l];
    }
    Y.node_bit = bit;
    bit += (Y.N - Y.S) * 2 * (int64_t)(Y.nb + Y.wbits);
    Y.total_bits = bit;
    Y.bytes = (((bit + 7) >> 3) + 7) & ~(int64_t)7;
}

struct HostBits {
    std::vector<uint8_t> buf;
    int64_t bit = 0;
    void put(uint64_t v, int n) {
        for (int i = 0; i < n; i++, bit++) {
            if ((size_t)(bit >> 3) >= buf.size()) buf.resize((bit >> 3) + 1, 0);
            if ((v >> i) & 1u) buf[bit >> 3] |= (uint8_t)(1u << (bit & 7));
        }
    }
};

struct BitsReader {
    const uint8_t* p;
    size_t n;
    int64_t bit = 0;
    bool ok = true;
    uint64_t get(int k) {
        uint64_t v = 0;
        for (int i = 0; i < k; i++, bit++) {
            if ((size_t)(bit >> 3) >= n) {
                ok = false;
                return 0;
            }
            v |= (uint64_t)((p[bit >> 3] >> (bit & 7)) & 1u) << i;
        }
        return v;
    }
};

__global__ void level_range_kernel(const void* __restrict__ ids, int id_bytes, int64_t n, uint32_t* __restrict__ mm) {
    uint32_t lo = 0xFFFFFFFFu, hi = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t v = id_bytes == 2 ? (uint32_t)static_cast<const uint16_t*>(ids)[i] : static_cast<const uint32_t*>(ids)[i];
        lo = min(lo, v);
        hi = max(hi, v);
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(mm, lo);
        atomicMax(mm + 1, hi);
    }
}

// (A) of one level: thread per 32-bit word of the stream, gathering the fields
// that overlap it
__global__ void pack_level_kernel(const void* __restrict__ ids, int id_bytes, int64_t n, uint32_t imin, int r,
                                  int64_t s0, uint32_t* __restrict__ words) {
    const int64_t w0 = s0 >> 5, w1 = (s0 + n * r - 1) >> 5;
    for (int64_t w = w0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w <= w1; w += (int64_t)gridDim.x * blockDim.x) {
        const int64_t lo_bit = max(w * 32, s0), hi_bit = min(w * 32 + 31, s0 + n * r - 1);
        const int64_t i0 = (lo_bit - s0) / r, i1 = (hi_bit - s0) / r;
        uint32_t acc = 0;
        for (int64_t i = i0; i <= i1; i++) {
            const uint64_t v = (uint64_t)((id_bytes == 2 ? (uint32_t)static_cast<const uint16_t*>(ids)[i]
                                                         : static_cast<const uint32_t*>(ids)[i]) - imin);
            const int64_t rel = s0 + i * r - w * 32;
            acc |= (uint32_t)(rel >= 0 ? (v << rel) : (v >> -rel));
        }
        if (acc) atomicOr(words + w, acc);
    }
}

__device__ __forceinline__ void or_field(uint32_t* words, int64_t bit, uint64_t v, int n) {
    // a field of n <= 64 bits at `bit`: at most three words
    const int64_t w = bit >> 5;
    const int sh = (int)(bit & 31);
    const uint32_t a = (uint32_t)(v << sh);
    const uint32_t b = (uint32_t)((sh ? v >> (32 - sh) : v >> 32) & 0xFFFFFFFFull);
    const uint32_t c = sh ? (uint32_t)(v >> (64 - sh)) : 0u;
    if (a) atomicOr(words + w, a);
    if (sh + n > 32 && b) atomicOr(words + w + 1, b);
    if (sh + n > 64 && c) atomicOr(words + w + 2, c);
}

// (B): thread per internal node record
__global__ void pack_nodes_kernel(const uint2* __restrict__ pq, const ulonglong2* __restrict__ ab, uint32_t S, int64_t N,
                                  int nb, int wbits, int64_t s0, uint32_t* __restrict__ words) {
    const int64_t R = 2 * (int64_t)(nb + wbits);
    for (int64_t n = S + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const int64_t bit = s0 + (n - S) * R;
        const uint2 e = pq[n];
        const ulonglong2 w = ab[n];
        or_field(words, bit, e.x, nb);
        or_field(words, bit + nb, e.y, nb);
        or_field(words, bit + 2 * nb, w.x, wbits);
        or_field(words, bit + 2 * nb + wbits, w.y, wbits);
    }
}

__device__ __forceinline__ uint64_t read_field(const uint32_t* __restrict__ words, int64_t bit, int n) {
    if (n == 0) return 0;
    const int64_t w = bit >> 5;
    const int sh = (int)(bit & 31);
    uint64_t v = (uint64_t)__ldg(words + w) >> sh;
    if (sh + n > 32) v |= (uint64_t)__ldg(words + w + 1) << (32 - sh);
    if (sh + n > 64) v |= (uint64_t)__ldg(words + w + 2) << (64 - sh);
    return n == 64 ? v : v & ((1ull << n) - 1);
}

struct StreamGeom {
    int L;
    int32_t dims[MG_MAX_LEVELS][3];
    int32_t r[MG_MAX_LEVELS];
    uint32_t imin[MG_MAX_LEVELS];
    int64_t level_bit[MG_MAX_LEVELS];
};

__global__ void decode_level_kernel(const uint32_t* __restrict__ words, int64_t s0, int r, uint32_t imin, int64_t n,
                                    uint32_t* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = imin + (uint32_t)read_field(words, s0 + i * r, r);
}

__global__ void decode_nodes_kernel(const uint32_t* __restrict__ words, int64_t s0, int nb, int wbits, uint32_t S,
                                    int64_t N, uint32_t* __restrict__ p, uint32_t* __restrict__ q,
                                    uint64_t* __restrict__ a, uint64_t* __restrict__ b) {
    const int64_t R = 2 * (int64_t)(nb + wbits);
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        if (n < S) {
            if (p) p[n] = MG_NO_NODE;
            if (q) q[n] = MG_NO_NODE;
            if (a) a[n] = 0;
            if (b) b[n] = 0;
            continue;
        }
        const int64_t bit = s0 + (n - S) * R;
        if (p) p[n] = (uint32_t)read_field(words, bit, nb);
        if (q) q[n] = (uint32_t)read_field(words, bit + nb, nb);
        if (a) a[n] = read_field(words, bit + 2 * nb, wbits);
        if (b) b[n] = read_field(words, bit + 2 * nb + wbits, wbits);
    }
}

__device__ __forceinline__ int64_t floor_coord_bs(float x, int32_t d0) {
    float xc = x;
    if (!(xc >= 0.f)) xc = 0.f;
    if (xc > (float)d0) xc = (float)d0;
    return (int64_t)xc;
}

// the lookup of mg_render_lookup with the voxel's node ID read from the stream
template <typename RowT>
__global__ void __launch_bounds__(128) stream_lookup_kernel(StreamGeom G, const uint32_t* __restrict__ words,
                                                            const float4* __restrict__ samples, int64_t P,
                                                            const RowT* __restrict__ vals, int row_words,
                                                            RowT* __restrict__ out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P) return;
    const float4 smp = __ldg(samples + i);
    const float t = smp.w + 0.5f;
    int l;
    if (!(t >= 0.f)) l = 0;
    else if (t >= (float)(G.L - 1)) l = G.L - 1;
    else l = (int)t;
    int64_t v[3];
    const float c[3] = {smp.x, smp.y, smp.z};
#pragma unroll
    for (int k = 0; k < 3; k++) {
        const int64_t x = floor_coord_bs(c[k], G.dims[0][k]) >> l;
        v[k] = min(x, (int64_t)G.dims[l][k] - 1);
    }
    const int64_t idx = (v[2] * G.dims[l][1] + v[1]) * G.dims[l][0] + v[0];
    const uint32_t node = G.imin[l] + (uint32_t)read_field(words, G.level_bit[l] + idx * G.r[l], G.r[l]);
    const RowT* src = vals + (int64_t)node * row_words;
    RowT* dst = out + i * row_words;
    for (int w = 0; w < row_words; w++) dst[w] = __ldg(src + w);
}

mg_status layout_of(const mg_graph* g, Layout& Y, cudaStream_t s) {
    Y.S = g->S;
    Y.N = g->N;
    Y.L = g->L;
    Y.nb = std::max(1, bits_for((uint64_t)g->N));
    for (int l = 0; l < g->L; l++)
        for (int k = 0; k < 3; k++) Y.dims[l][k] = g->geom.dims[l][k];
    // per-level ID ranges (Eq. 14) and the widest weight
    Buf mm;
    MG_TRY(mm.alloc(&g->al, (size_t)g->L * 8, s));
    std::vector<uint32_t> init((size_t)g->L * 2);
    for (int l = 0; l < g->L; l++) {
        init[2 * l] = 0xFFFFFFFFu;
        init[2 * l + 1] = 0u;
    }
    MG_CUDA(cudaMemcpyAsync(mm.p, init.data(), init.size() * 4, cudaMemcpyHostToDevice, s));
    for (int l = 0; l < g->L; l++) {
        const int64_t n = Y.dims[l][0] * Y.dims[l][1] * Y.dims[l][2];
        const void* ids = l == 0 ? g->mip0.p : static_cast<const void*>(g->mip.as<uint32_t>() + g->geom.off[l]);
        level_range_kernel<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(ids, l == 0 ? g->id0_bytes : 4, n,
                                                                     mm.as<uint32_t>() + 2 * l);
        MG_CUDA(cudaGetLastError());
    }
    std::vector<uint32_t> r((size_t)g->L * 2);
    MG_CUDA(cudaMemcpyAsync(r.data(), mm.p, r.size() * 4, cudaMemcpyDeviceToHost, s));
    std::vector<uint64_t> ab((size_t)std::max<int64_t>(g->N, 1) * 2);
    MG_CUDA(cudaMemcpyAsync(ab.data(), g->ab.p, (size_t)g->N * 16, cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    for (int l = 0; l < g->L; l++) {
        Y.imin[l] = r[2 * l];
        Y.r[l] = bits_for((uint64_t)(r[2 * l + 1] - r[2 * l]) + 1);
    }
    uint64_t wmax = 1;
    for (int64_t n = g->S; n < g->N; n++) wmax = std::max(wmax, std::max(ab[2 * n], ab[2 * n + 1]));
    Y.wbits = std::max(1, bits_for(wmax + 1));
    finish_layout(Y);
    return MG_OK;
}

HostBits header_of(const Layout& Y) {
    HostBits hb;
    hb.put(Y.S, 32);
    hb.put(0, 1);
    hb.put((uint64_t)(Y.nb - 1), 6);
    hb.put(0, 32);
    for (int k = 0; k < 3; k++) hb.put((uint64_t)Y.dims[0][k], 32);
    hb.put(0, 4);
    hb.put((uint64_t)(Y.N - Y.S), Y.nb);
    hb.put(1, 1);
    hb.put((uint64_t)(Y.wbits - 1), 6);
    for (int l = 0; l < Y.L; l++) {
        hb.put((uint64_t)Y.r[l], Y.nb);
        hb.put(Y.imin[l], Y.nb);
    }
    return hb;
}

mg_status parse(const void* host, size_t bytes, Layout& Y) {
    BitsReader rd{static_cast<const uint8_t*>(host), bytes};
    Y.S = (uint32_t)rd.get(32);
    const uint64_t frac = rd.get(1);
    Y.nb = (int)rd.get(6) + 1;
    rd.get(32);
    int64_t d[3];
    for (int k = 0; k < 3; k++) d[k] = (int64_t)rd.get(32);
    rd.get(4);
    const int64_t internal = (int64_t)rd.get(Y.nb);
    const uint64_t exact = rd.get(1);
    Y.wbits = (int)rd.get(6) + 1;
    if (!rd.ok) return fail(MG_ERR_INVALID_ARG, "bitstream shorter than its header");
    if (frac || !exact) return fail(MG_ERR_UNSUPPORTED, "only exact-weight streams of label volumes are read");
    if (Y.S < 1 || d[0] < 1 || d[1] < 1 || d[2] < 1 || d[0] > 65535 || d[1] > 65535 || d[2] > 65535)
        return fail(MG_ERR_INVALID_ARG, "bitstream header out of range");
    Y.N = Y.S + internal;
    // the level geometry follows from the resolution (Eq. 4)
    int64_t c[3] = {d[0], d[1], d[2]};
    Y.L = 0;
    for (;;) {
        if (Y.L >= MG_MAX_LEVELS) return fail(MG_ERR_UNSUPPORTED, "too many levels");
        for (int k = 0; k < 3; k++) Y.dims[Y.L][k] = c[k];
        Y.L++;
        if (c[0] == 1 && c[1] == 1 && c[2] == 1) break;
        for (int k = 0; k < 3; k++) c[k] = (c[k] + 1) / 2;
    }
    for (int l = 0; l < Y.L; l++) {
        Y.r[l] = (int32_t)rd.get(Y.nb);
        Y.imin[l] = (uint32_t)rd.get(Y.nb);
        if (Y.r[l] > 32) return fail(MG_ERR_INVALID_ARG, "voxel bits above 32");
    }
    if (!rd.ok) return fail(MG_ERR_INVALID_ARG, "bitstream shorter than its header");
    finish_layout(Y);
    return MG_OK;
}

void to_info(const Layout& Y, mg_bitstream_info* info) {
    std::memset(info, 0, sizeof(*info));
    info->num_segments = Y.S;
    info->levels = Y.L;
    info->node_bits = Y.nb;
    info->weight_bits = Y.wbits;
    info->num_nodes = Y.N;
    for (int l = 0; l < Y.L; l++) {
        for (int k = 0; k < 3; k++) info->dims[l][k] = Y.dims[l][k];
        info->voxel_bits[l] = Y.r[l];
        info->imin[l] = Y.imin[l];
        info->level_bit[l] = Y.level_bit[l];
    }
    info->node_bit = Y.node_bit;
    info->header_bits = Y.header_bits;
    info->bytes = Y.bytes;
}

Layout from_info(const mg_bitstream_info* info) {
    Layout Y;
    Y.S = info->num_segments;
    Y.L = info->levels;
    Y.nb = info->node_bits;
    Y.wbits = info->weight_bits;
    Y.N = info->num_nodes;
    for (int l = 0; l < Y.L; l++) {
        for (int k = 0; k < 3; k++) Y.dims[l][k] = info->dims[l][k];
        Y.r[l] = info->voxel_bits[l];
        Y.imin[l] = (uint32_t)info->imin[l];
    }
    finish_layout(Y);
    return Y;
}

bool info_ok(const mg_bitstream_info* info) {
    if (info->levels < 1 || info->levels > MG_MAX_LEVELS || info->node_bits < 1 || info->node_bits > 64 ||
        info->weight_bits < 1 || info->weight_bits > 64 || info->num_nodes < info->num_segments)
        return false;
    for (int l = 0; l < info->levels; l++)
        if (info->voxel_bits[l] < 0 || info->voxel_bits[l] > 32) return false;
    return from_info(info).bytes == info->bytes;
}

}  // namespace
}  // namespace mg

using namespace mg;

extern "C" {

MG_API mg_status mg_bitstream_size(const mg_graph* g, size_t* bytes) {
    MG_RANGE("mg_bitstream_size");
    if (!g || !bytes) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (g->quantised) return fail(MG_ERR_UNSUPPORTED, "the stream holds exact weights; this graph is quantised");
    DeviceGuard dg(g->device);
    Layout Y;
    MG_TRY(layout_of(g, Y, nullptr));
    *bytes = (size_t)Y.bytes;
    return MG_OK;
}

MG_API mg_status mg_bitstream_write(const mg_graph* g, void* dst, size_t bytes, mg_stream stream) {
    MG_RANGE("mg_bitstream_write");
    if (!g || !dst) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (reinterpret_cast<uintptr_t>(dst) % 8) return fail(MG_ERR_INVALID_ARG, "dst must be 8-byte aligned");
    if (g->quantised) return fail(MG_ERR_UNSUPPORTED, "the stream holds exact weights; this graph is quantised");
    DeviceGuard dg(g->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    Layout Y;
    MG_TRY(layout_of(g, Y, s));
    if (bytes < (size_t)Y.bytes) return fail(MG_ERR_CAPACITY, "dst smaller than mg_bitstream_size");
    const HostBits hb = header_of(Y);
    MG_CUDA(cudaMemsetAsync(dst, 0, (size_t)Y.bytes, s));
    MG_CUDA(cudaMemcpyAsync(dst, hb.buf.data(), hb.buf.size(), cudaMemcpyHostToDevice, s));
    uint32_t* words = static_cast<uint32_t*>(dst);
    for (int l = 0; l < Y.L; l++) {
        if (Y.r[l] == 0) continue;
        const int64_t n = Y.dims[l][0] * Y.dims[l][1] * Y.dims[l][2];
        const void* ids = l == 0 ? g->mip0.p : static_cast<const void*>(g->mip.as<uint32_t>() + g->geom.off[l]);
        const int64_t nw = ((Y.level_bit[l] + n * Y.r[l] - 1) >> 5) - (Y.level_bit[l] >> 5) + 1;
        pack_level_kernel<<<grid_for(nw, 256, 152 * 32), 256, 0, s>>>(ids, l == 0 ? g->id0_bytes : 4, n, Y.imin[l],
                                                                       Y.r[l], Y.level_bit[l], words);
        MG_CUDA(cudaGetLastError());
    }
    if (Y.N > Y.S) {
        pack_nodes_kernel<<<grid_for(Y.N - Y.S, 256, 152 * 32), 256, 0, s>>>(
            g->pq.as<uint2>(), g->ab.as<ulonglong2>(), Y.S, Y.N, Y.nb, Y.wbits, Y.node_bit, words);
        MG_CUDA(cudaGetLastError());
    }
    // the host header buffer is freed on return: wait for its copy
    MG_CUDA(cudaStreamSynchronize(s));
    return MG_OK;
}

MG_API mg_status mg_bitstream_parse(const void* host, size_t bytes, mg_bitstream_info* info) {
    if (!host || !info) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    Layout Y;
    MG_TRY(parse(host, bytes, Y));
    to_info(Y, info);
    return MG_OK;
}

MG_API mg_status mg_bitstream_decode_mip(const void* stream_dev, const mg_bitstream_info* info, int level,
                                         uint32_t* out, mg_stream stream) {
    MG_RANGE("mg_bitstream_decode_mip");
    if (!stream_dev || !info || !out) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (!info_ok(info)) return fail(MG_ERR_INVALID_ARG, "inconsistent bitstream info");
    if (level < 0 || level >= info->levels) return fail(MG_ERR_INVALID_ARG, "level out of range");
    const Layout Y = from_info(info);
    const int64_t n = Y.dims[level][0] * Y.dims[level][1] * Y.dims[level][2];
    decode_level_kernel<<<grid_for(n, 256, 152 * 32), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint32_t*>(stream_dev), Y.level_bit[level], Y.r[level], Y.imin[level], n, out);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

MG_API mg_status mg_bitstream_decode_nodes(const void* stream_dev, const mg_bitstream_info* info, uint32_t* p,
                                           uint32_t* q, uint64_t* a, uint64_t* b, mg_stream stream) {
    MG_RANGE("mg_bitstream_decode_nodes");
    if (!stream_dev || !info) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (!info_ok(info)) return fail(MG_ERR_INVALID_ARG, "inconsistent bitstream info");
    const Layout Y = from_info(info);
    decode_nodes_kernel<<<grid_for(Y.N, 256, 152 * 32), 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint32_t*>(stream_dev), Y.node_bit, Y.nb, Y.wbits, Y.S, Y.N, p, q, a, b);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

MG_API mg_status mg_bitstream_lookup(const void* stream_dev, const mg_bitstream_info* info, const void* vals, int C,
                                     mg_dtype dtype, const float* samples, int64_t P, void* out, mg_stream stream) {
    MG_RANGE("mg_bitstream_lookup");
    if (!stream_dev || !info) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (!info_ok(info)) return fail(MG_ERR_INVALID_ARG, "inconsistent bitstream info");
    if (C < 1 || C > 16) return fail(MG_ERR_INVALID_ARG, "C must be in 1..16");
    if (dtype != MG_F32 && dtype != MG_F16 && dtype != MG_BF16)
        return fail(MG_ERR_INVALID_ARG, "dtype must be MG_F32, MG_F16 or MG_BF16");
    if (P < 0) return fail(MG_ERR_INVALID_ARG, "P must be >= 0");
    if (P == 0) return MG_OK;
    if (!vals || !samples || !out) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (reinterpret_cast<uintptr_t>(samples) % 16) return fail(MG_ERR_INVALID_ARG, "samples must be 16-byte aligned");
    const Layout Y = from_info(info);
    StreamGeom G;
    G.L = Y.L;
    for (int l = 0; l < MG_MAX_LEVELS; l++) {
        for (int k = 0; k < 3; k++) G.dims[l][k] = l < Y.L ? (int32_t)Y.dims[l][k] : 1;
        G.r[l] = l < Y.L ? Y.r[l] : 0;
        G.imin[l] = l < Y.L ? Y.imin[l] : 0;
        G.level_bit[l] = l < Y.L ? Y.level_bit[l] : 0;
    }
    const size_t row = (size_t)C * (dtype == MG_F32 ? 4 : 2);
    const uint32_t* words = static_cast<const uint32_t*>(stream_dev);
    const float4* sm = reinterpret_cast<const float4*>(samples);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const unsigned grid = grid_for(P, 128);
    auto al = [](const void* p, size_t a) { return reinterpret_cast<uintptr_t>(p) % a == 0; };
    if (row % 16 == 0 && al(vals, 16) && al(out, 16))
        stream_lookup_kernel<uint4><<<grid, 128, 0, s>>>(G, words, sm, P, (const uint4*)vals, (int)(row / 16), (uint4*)out);
    else if (row % 8 == 0 && al(vals, 8) && al(out, 8))
        stream_lookup_kernel<uint2><<<grid, 128, 0, s>>>(G, words, sm, P, (const uint2*)vals, (int)(row / 8), (uint2*)out);
    else if (row % 4 == 0 && al(vals, 4) && al(out, 4))
        stream_lookup_kernel<uint32_t><<<grid, 128, 0, s>>>(G, words, sm, P, (const uint32_t*)vals, (int)(row / 4),
                                                            (uint32_t*)out);
    else
        stream_lookup_kernel<uint16_t><<<grid, 128, 0, s>>>(G, words, sm, P, (const uint16_t*)vals, (int)(row / 2),
                                                            (uint16_t*)out);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

}  // extern "C"
