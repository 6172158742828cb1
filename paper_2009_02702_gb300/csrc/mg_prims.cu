// mg_prims.cu -- device-wide exclusive scan and stable LSD radix sort.
//
// Scan: reduce-then-scan over tiles of 2048 elements (256 threads x 8), the
// per-tile partial sums scanned recursively.  Sort: 8-bit digits, one
// histogram pass and one scatter pass per digit; ranks inside a tile are made
// stable with warp match + per-warp digit counts in shared memory.
#include "mg_internal.cuh"

namespace mg {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// exclusive prefix of v over the block; *block_total receives the sum
template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* wsum, T* block_total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    T x = warp_incl_scan(v, lane);
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < nw ? wsum[lane] : T(0);
        w = warp_incl_scan(w, lane);
        wsum[lane] = w;
    }
    __syncthreads();
    T pre = warp > 0 ? wsum[warp - 1] : T(0);
    *block_total = wsum[nw - 1];
    return pre + x - v;
}

template <typename T>
__global__ void scan_reduce_kernel(const T* __restrict__ in, int64_t n, T* __restrict__ partial) {
    __shared__ T wsum[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    T s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) s += in[idx];
    }
    T tot;
    block_excl_scan(s, wsum, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

template <typename T>
__global__ void scan_tile_kernel(const T* in, T* out, int64_t n, const T* __restrict__ partial_ex,
                                 T* __restrict__ total) {
    __shared__ T tile[kScanTile];
    __shared__ T wsum[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        tile[i * kScanThreads + threadIdx.x] = idx < n ? in[idx] : T(0);
    }
    __syncthreads();
    T loc[kScanItems];
    T sum = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        loc[i] = tile[threadIdx.x * kScanItems + i];
        sum += loc[i];
    }
    T bt;
    T ex = block_excl_scan(sum, wsum, &bt);
    const T off = partial_ex ? partial_ex[blockIdx.x] : T(0);
    T run = ex + off;
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        tile[threadIdx.x * kScanItems + i] = run;
        run += loc[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanItems; i++) {
        int64_t idx = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (idx < n) out[idx] = tile[i * kScanThreads + threadIdx.x];
    }
    if (total && blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) *total = off + bt;
}

template <typename T>
mg_status scan_impl(const T* in, T* out, int64_t n, T* total, const Alloc& al, cudaStream_t s) {
    if (n <= 0) {
        if (total) MG_CUDA(cudaMemsetAsync(total, 0, sizeof(T), s));
        return MG_OK;
    }
    const int64_t nb = (n + kScanTile - 1) / kScanTile;
    if (nb == 1) {
        scan_tile_kernel<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr, total);
        MG_CUDA(cudaGetLastError());
        return MG_OK;
    }
    Buf part, part_ex;
    MG_TRY(part.alloc(&al, (size_t)nb * sizeof(T), s));
    MG_TRY(part_ex.alloc(&al, (size_t)nb * sizeof(T), s));
    scan_reduce_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, part.as<T>());
    MG_CUDA(cudaGetLastError());
    MG_TRY(scan_impl<T>(part.as<T>(), part_ex.as<T>(), nb, nullptr, al, s));
    scan_tile_kernel<T><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, part_ex.as<T>(), total);
    MG_CUDA(cudaGetLastError());
    return MG_OK;
}

// ---------------------------------------------------------------------------
// radix sort
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kSortWarps = kSortThreads / 32;

__global__ void rs_hist_kernel(const uint64_t* __restrict__ keys, int64_t n, int shift,
                               uint32_t* __restrict__ hist, int64_t nb) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
    for (int i = 0; i < kSortItems; i++) {
        int64_t idx = base + (int64_t)i * kSortThreads + threadIdx.x;
        if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

__global__ void rs_scatter_kernel(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                                  int64_t n, int shift, const uint32_t* __restrict__ offs, int64_t nb,
                                  uint64_t* __restrict__ kout, uint32_t* __restrict__ vout) {
    __shared__ uint32_t running[256];
    __shared__ uint32_t wcnt[kSortWarps][256];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    running[threadIdx.x] = offs[(int64_t)threadIdx.x * nb + blockIdx.x];
    const unsigned lt = (1u << lane) - 1u;
    const int64_t base = (int64_t)blockIdx.x * kSortTile;
    for (int i = 0; i < kSortItems; i++) {
#pragma unroll
        for (int w = 0; w < kSortWarps; w++) wcnt[w][threadIdx.x] = 0;
        __syncthreads();
        const int64_t idx = base + (int64_t)i * kSortThreads + threadIdx.x;
        const bool valid = idx < n;
        uint64_t k = valid ? kin[idx] : 0;
        uint32_t v = valid ? vin[idx] : 0;
        const uint32_t digit = valid ? (uint32_t)((k >> shift) & 255u) : 256u;
        const unsigned peers = __match_any_sync(0xffffffffu, digit);
        const uint32_t rank = __popc(peers & lt);
        if (valid && lane == __ffs(peers) - 1) wcnt[warp][digit] = __popc(peers);
        __syncthreads();
        {
            uint32_t s = running[threadIdx.x];
#pragma unroll
            for (int w = 0; w < kSortWarps; w++) {
                uint32_t c = wcnt[w][threadIdx.x];
                wcnt[w][threadIdx.x] = s;
                s += c;
            }
            running[threadIdx.x] = s;
        }
        __syncthreads();
        if (valid) {
            const uint32_t pos = wcnt[warp][digit] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
    }
}

}  // namespace

mg_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total,
                             const Alloc& al, cudaStream_t s) {
    return scan_impl<uint32_t>(in, out, n, total, al, s);
}

mg_status scan_exclusive_u64(const uint64_t* in, uint64_t* out, int64_t n, uint64_t* total,
                             const Alloc& al, cudaStream_t s) {
    return scan_impl<uint64_t>(in, out, n, total, al, s);
}

mg_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, int64_t n, int bits, const Alloc& al,
                           cudaStream_t s) {
    if (n <= 1 || bits <= 0) return MG_OK;
    if (n >= (int64_t)1 << 32) return fail(MG_ERR_UNSUPPORTED, "radix sort of more than 2^32 items");
    const int64_t nb = (n + kSortTile - 1) / kSortTile;
    Buf k2, v2, hist;
    MG_TRY(k2.alloc(&al, (size_t)n * sizeof(uint64_t), s));
    MG_TRY(v2.alloc(&al, (size_t)n * sizeof(uint32_t), s));
    MG_TRY(hist.alloc(&al, (size_t)nb * 256 * sizeof(uint32_t), s));
    uint64_t* ks = keys;
    uint32_t* vs = vals;
    uint64_t* kd = k2.as<uint64_t>();
    uint32_t* vd = v2.as<uint32_t>();
    for (int shift = 0; shift < bits; shift += 8) {
        rs_hist_kernel<<<(unsigned)nb, kSortThreads, 0, s>>>(ks, n, shift, hist.as<uint32_t>(), nb);
        MG_CUDA(cudaGetLastError());
        MG_TRY(scan_exclusive_u32(hist.as<uint32_t>(), hist.as<uint32_t>(), nb * 256, nullptr, al, s));
        rs_scatter_kernel<<<(unsigned)nb, kSortThreads, 0, s>>>(ks, vs, n, shift, hist.as<uint32_t>(), nb,
                                                                kd, vd);
        MG_CUDA(cudaGetLastError());
        uint64_t* tk = ks; ks = kd; kd = tk;
        uint32_t* tv = vs; vs = vd; vd = tv;
    }
    if (ks != keys) {
        MG_CUDA(cudaMemcpyAsync(keys, ks, (size_t)n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
        MG_CUDA(cudaMemcpyAsync(vals, vs, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    return MG_OK;
}

}  // namespace mg
