// synth_dev.cu -- seeded synthetic segmentation volumes on the GPU.
//
// Input generation only: no Mixture Graph arithmetic lives here.  Implements
// the integer Voronoi rule of synth_host.c (doubled voxel centres, axis metric,
// integer seed weights, ties to the lowest index), so volumes match the host
// generator bit for bit.  Used to make the large test and benchmark volumes.
#include <cstdint>
#include <cuda_runtime.h>

namespace {

constexpr int kTile = 512;

template <bool kWeighted, typename OutT>
__global__ void voronoi_kernel(int64_t nx, int64_t ny, int64_t nz, const int64_t* __restrict__ seeds2,
                               const int64_t* __restrict__ weight, int64_t K, int64_t mx, int64_t my,
                               int64_t mz, OutT* __restrict__ out)
{
    __shared__ int32_t s_x[kTile], s_y[kTile], s_z[kTile];
    __shared__ int64_t s_w[kTile];
    const int64_t V = nx * ny * nz;
    const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int64_t x = 0, y = 0, z = 0;
    if (v < V) {
        x = v % nx;
        y = (v / nx) % ny;
        z = v / (nx * ny);
    }
    const int64_t px = 2 * x + 1, py = 2 * y + 1, pz = 2 * z + 1;
    int64_t best = 0, bd = -1, bw = 1;
    for (int64_t t0 = 0; t0 < K; t0 += kTile) {
        const int n = (int)((K - t0) < kTile ? (K - t0) : kTile);
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            s_x[i] = (int32_t)seeds2[3 * (t0 + i)];
            s_y[i] = (int32_t)seeds2[3 * (t0 + i) + 1];
            s_z[i] = (int32_t)seeds2[3 * (t0 + i) + 2];
            s_w[i] = kWeighted ? weight[t0 + i] : 1;
        }
        __syncthreads();
        for (int i = 0; i < n; i++) {
            const int64_t ex = px - s_x[i], ey = py - s_y[i], ez = pz - s_z[i];
            const int64_t d = mx * ex * ex + my * ey * ey + mz * ez * ez;
            bool better;
            if (kWeighted) better = (bd < 0) || (d * bw < bd * s_w[i]);
            else better = (bd < 0) || (d < bd);
            if (better) {
                best = t0 + i;
                bd = d;
                if (kWeighted) bw = s_w[i];
            }
        }
    }
    if (v < V) out[v] = (OutT)best;
}

}  // namespace

extern "C" __attribute__((visibility("default"))) int mgs_voronoi_dev(int64_t nx, int64_t ny, int64_t nz, const int64_t* seeds2_dev,
                               const int64_t* weight_dev, int64_t K, const int64_t* metric_host,
                               int out_bytes, void* out_dev, cudaStream_t stream)
{
    const int64_t V = nx * ny * nz;
    if (V <= 0 || K <= 0) return 1;
    const int threads = 256;
    const int64_t blocks = (V + threads - 1) / threads;
    const bool weighted = weight_dev != nullptr;
    if (out_bytes == 2) {
        auto* o = static_cast<uint16_t*>(out_dev);
        if (weighted)
            voronoi_kernel<true><<<(unsigned)blocks, threads, 0, stream>>>(
                nx, ny, nz, seeds2_dev, weight_dev, K, metric_host[0], metric_host[1], metric_host[2], o);
        else
            voronoi_kernel<false><<<(unsigned)blocks, threads, 0, stream>>>(
                nx, ny, nz, seeds2_dev, weight_dev, K, metric_host[0], metric_host[1], metric_host[2], o);
    } else {
        auto* o = static_cast<uint32_t*>(out_dev);
        if (weighted)
            voronoi_kernel<true><<<(unsigned)blocks, threads, 0, stream>>>(
                nx, ny, nz, seeds2_dev, weight_dev, K, metric_host[0], metric_host[1], metric_host[2], o);
        else
            voronoi_kernel<false><<<(unsigned)blocks, threads, 0, stream>>>(
                nx, ny, nz, seeds2_dev, weight_dev, K, metric_host[0], metric_host[1], metric_host[2], o);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
