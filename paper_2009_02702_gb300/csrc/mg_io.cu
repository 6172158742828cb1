// mg_io.cu -- export and import of a built graph through host memory
// (checkpoint / resume: a graph built once can be stored and reloaded without
// rebuilding).  The paper's own persistence is its bit-packed stream
// (Table 1); this image holds the raw device arrays instead.
//
// Image: a fixed header (magic, version, sizes, geometry, depth buckets, the
// byte size of every array), then the arrays in header order, each starting
// on a 256-byte boundary.  Import validates the header and every size before
// allocating anything.  The padded axis-major copies of the box queries are
// not stored: import rebuilds them from the mip levels.
#include "mg_internal.cuh"

#include <cstring>

namespace mg {
namespace {

constexpr char kMagic[8] = {'M', 'G', 'R', 'A', 'P', 'H', '0', '1'};
constexpr uint32_t kVersion = 2;
constexpr int kArrays = 8;   // mip0, mip, pq, ab, ab32, alpha, lut_meta, lut

struct Header {
    char magic[8];
    uint32_t version, S;
    int32_t L, D, id0_bytes, reserved;
    int64_t N, max_list, pairs, lut_entries;
    int32_t dims[MG_MAX_LEVELS][3];
    int64_t off[MG_MAX_LEVELS];
    int64_t bucket[MG_MAX_DEPTH + 2];
    uint64_t bytes[kArrays];
};

size_t round_up(size_t n) { return (n + 255) & ~(size_t)255; }

Buf* arrays(mg_graph* g, int k) {
    Buf* a[kArrays] = {&g->mip0, &g->mip, &g->pq, &g->ab, &g->ab32, &g->alpha, &g->lut_meta, &g->lut};
    return a[k];
}

size_t image_bytes(const uint64_t (&bytes)[kArrays]) {
    size_t n = round_up(sizeof(Header));
    for (int k = 0; k < kArrays; k++) n += round_up(bytes[k]);
    return n;
}

}  // namespace
}  // namespace mg

using namespace mg;

extern "C" {

MG_API mg_status mg_graph_export_size(const mg_graph* g, size_t* bytes) {
    if (!g || !bytes) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (g->quantised) return fail(MG_ERR_UNSUPPORTED, "quantised graphs are not exported");
    uint64_t b[kArrays];
    for (int k = 0; k < kArrays; k++) b[k] = arrays(const_cast<mg_graph*>(g), k)->bytes;
    *bytes = image_bytes(b);
    return MG_OK;
}

MG_API mg_status mg_graph_export(const mg_graph* g, void* host, size_t bytes, mg_stream stream) {
    MG_RANGE("mg_graph_export");
    if (!g || !host) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    if (g->quantised) return fail(MG_ERR_UNSUPPORTED, "quantised graphs are not exported");
    mg_graph* gm = const_cast<mg_graph*>(g);
    Header h;
    std::memset(&h, 0, sizeof(h));
    std::memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.S = g->S;
    h.L = g->L;
    h.D = g->D;
    h.id0_bytes = g->id0_bytes;
    h.N = g->N;
    h.max_list = g->max_list;
    h.pairs = g->pairs;
    h.lut_entries = g->lut_entries;
    for (int l = 0; l < MG_MAX_LEVELS; l++) {
        for (int k = 0; k < 3; k++) h.dims[l][k] = g->geom.dims[l][k];
        h.off[l] = g->geom.off[l];
    }
    for (int d = 0; d < MG_MAX_DEPTH + 2; d++) h.bucket[d] = g->bucket[d];
    for (int k = 0; k < kArrays; k++) h.bytes[k] = arrays(gm, k)->bytes;
    if (bytes < image_bytes(h.bytes)) return fail(MG_ERR_CAPACITY, "buffer smaller than mg_graph_export_size");
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != g->device) MG_CUDA(cudaSetDevice(g->device));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    unsigned char* p = static_cast<unsigned char*>(host);
    std::memcpy(p, &h, sizeof(h));
    size_t at = round_up(sizeof(Header));
    mg_status st = MG_OK;
    for (int k = 0; k < kArrays && st == MG_OK; k++) {
        const Buf* a = arrays(gm, k);
        if (a->bytes) {
            const cudaError_t e = cudaMemcpyAsync(p + at, a->p, a->bytes, cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) st = cuda_fail(e, "mg_graph_export");
        }
        at += round_up(a->bytes);
    }
    if (st == MG_OK) {
        const cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_fail(e, "mg_graph_export");
    }
    if (prev >= 0 && prev != g->device) cudaSetDevice(prev);
    return st;
}

MG_API mg_status mg_graph_import(const void* host, size_t bytes, const mg_allocator* allocator, mg_stream stream,
                                 mg_graph** out) {
    MG_RANGE("mg_graph_import");
    if (!host || !out) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (bytes < sizeof(Header)) return fail(MG_ERR_INVALID_ARG, "image shorter than its header");
    if (allocator && (!allocator->alloc || !allocator->free))
        return fail(MG_ERR_INVALID_ARG, "allocator needs alloc and free");
    Header h;
    std::memcpy(&h, host, sizeof(h));
    if (std::memcmp(h.magic, kMagic, 8) != 0) return fail(MG_ERR_INVALID_ARG, "not a Mixture Graph image");
    if (h.version != kVersion) return fail(MG_ERR_UNSUPPORTED, "image version " + std::to_string(h.version));
    // the arrays' sizes follow from the header's counts; reject anything else
    int64_t V0 = 0, hi = 0;
    bool ok = h.L >= 1 && h.L <= MG_MAX_LEVELS && h.D >= 0 && h.D < MG_MAX_DEPTH && h.S >= 1 && h.N >= h.S &&
              (h.id0_bytes == 2 || h.id0_bytes == 4);
    if (ok) {
        for (int l = 0; l < h.L; l++) {
            const int64_t n = (int64_t)h.dims[l][0] * h.dims[l][1] * h.dims[l][2];
            if (h.dims[l][0] < 1 || h.dims[l][1] < 1 || h.dims[l][2] < 1) ok = false;
            if (l == 0) V0 = n;
            else if (h.off[l] != hi) ok = false;
            else hi += n;
        }
    }
    if (ok) {
        const uint64_t want[kArrays] = {(uint64_t)V0 * h.id0_bytes, (uint64_t)hi * 4,
                                        (uint64_t)h.N * 8, (uint64_t)h.N * 16, (uint64_t)h.N * 8, (uint64_t)h.N * 4,
                                        h.bytes[6] ? (uint64_t)h.N * 8 : 0ull, h.bytes[7]};
        for (int k = 0; k < kArrays; k++)
            if (h.bytes[k] != want[k]) ok = false;
        // the table: a row directory of N entries, or none; entries at least lut_entries
        if (h.bytes[7] < (uint64_t)h.lut_entries * 8) ok = false;
        if (!h.bytes[6] && (h.bytes[7] || h.lut_entries)) ok = false;
        if (h.bucket[0] != 0 || h.bucket[1] != (int64_t)h.S || h.bucket[h.D + 1] != h.N) ok = false;
        for (int d = 0; d <= h.D; d++)
            if (h.bucket[d + 1] < h.bucket[d]) ok = false;
    }
    if (!ok) return fail(MG_ERR_INVALID_ARG, "inconsistent Mixture Graph image header");
    if (bytes < image_bytes(h.bytes)) return fail(MG_ERR_INVALID_ARG, "image shorter than its arrays");
    std::unique_ptr<mg_graph> g(new (std::nothrow) mg_graph());
    if (!g) return fail(MG_ERR_OOM, "host allocation failed");
    MG_CUDA(cudaGetDevice(&g->device));
    if (allocator) {
        g->al.a = *allocator;
        g->al.custom = true;
    }
    g->S = h.S;
    g->L = h.L;
    g->D = h.D;
    g->N = h.N;
    g->id0_bytes = h.id0_bytes;
    g->max_list = h.max_list;
    g->pairs = h.pairs;
    g->lut_entries = h.lut_entries;
    g->geom.L = h.L;
    for (int l = 0; l < MG_MAX_LEVELS; l++) {
        for (int k = 0; k < 3; k++) g->geom.dims[l][k] = h.dims[l][k];
        g->geom.off[l] = h.off[l];
    }
    for (int d = 0; d < MG_MAX_DEPTH + 2; d++) g->bucket[d] = h.bucket[d];
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const unsigned char* p = static_cast<const unsigned char*>(host);
    size_t at = round_up(sizeof(Header));
    for (int k = 0; k < kArrays; k++) {
        Buf* a = arrays(g.get(), k);
        if (h.bytes[k]) {
            MG_TRY(a->alloc(&g->al, h.bytes[k], s));
            MG_CUDA(cudaMemcpyAsync(a->p, p + at, h.bytes[k], cudaMemcpyHostToDevice, s));
        }
        at += round_up(h.bytes[k]);
    }
    MG_TRY(g->status.alloc(&g->al, sizeof(unsigned), s));
    MG_CUDA(cudaMemsetAsync(g->status.p, 0, sizeof(unsigned), s));
    MG_TRY(build_query_copies(g.get(), s));
    MG_CUDA(cudaStreamSynchronize(s));   // the host image may be freed on return
    for (int k = 0; k < kArrays; k++) arrays(g.get(), k)->s = nullptr;
    for (int c = 0; c < 3; c++) g->mip0x[c].s = g->mipx[c].s = nullptr;
    g->status.s = nullptr;
    *out = g.release();
    return MG_OK;
}

}  // extern "C"
