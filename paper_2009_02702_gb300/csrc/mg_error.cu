// mg_error.cu -- the mixture table with uncertainties (Sec. 3.5, Eq. 16-17)
// and box histograms summed from it (Sec. 3.6).
//
// Every node's row lists the sources under it with mu (its share of the
// node's mixture) and dmu (Eq. 17): a lerp n of p and q with weight w of q
// and uncertainty dw gives mu_i(n) = (1 - w) mu_i(p) + w mu_i(q) and
// dmu_i(n)^2 = mu_i(n)^2 ((dmu_i(p)/mu_i(p))^2 + (dmu_i(q)/mu_i(q))^2 +
// 2 (dw/w)^2), a ratio term being 0 where the component is absent.  Exact
// graphs have w = b/(a+b) and dw = 0; quantised ones their bin's codeword
// and sigma.  Rows are built level by level (predecessors first), fp64.
#include "mg_internal.cuh"

#include <vector>

namespace mg {
namespace {

__global__ void exact_weights_kernel(const ulonglong2* __restrict__ ab, int64_t N, uint32_t S, double* __restrict__ w,
                                     double* __restrict__ dw) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        double x = 0.0;
        if (n >= (int64_t)S) {
            const ulonglong2 v = ab[n];
            x = (double)v.y / ((double)v.x + (double)v.y);
        }
        w[n] = x;
        dw[n] = 0.0;
    }
}

__global__ void source_rows_kernel(const uint64_t* __restrict__ off, uint32_t S, uint32_t* __restrict__ src,
                                   double* __restrict__ mu, double* __restrict__ dmu) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S; s += (int64_t)gridDim.x * blockDim.x) {
        src[off[s]] = (uint32_t)s;
        mu[off[s]] = 1.0;
        dmu[off[s]] = 0.0;
    }
}

__global__ void level_rows_kernel(const uint2* __restrict__ pq, const double* __restrict__ w,
                                  const double* __restrict__ dw, int64_t lo, int64_t hi,
                                  const uint64_t* __restrict__ off, uint32_t* __restrict__ src, double* __restrict__ mu,
                                  double* __restrict__ dmu) {
    for (int64_t n = lo + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < hi; n += (int64_t)gridDim.x * blockDim.x) {
        const uint2 e = pq[n];
        uint64_t a = off[e.x], ae = off[e.x + 1], b = off[e.y], be = off[e.y + 1], k = off[n];
        const double wq = w[n], wp = 1.0 - wq;
        const double rw = wq > 0.0 ? dw[n] / wq : 0.0;
        while (a < ae || b < be) {
            const bool fa = b >= be || (a < ae && src[a] <= src[b]);
            const bool fb = a >= ae || (b < be && src[b] <= src[a]);
            const uint32_t s = fa ? src[a] : src[b];
            double m = 0.0, r2 = 2.0 * rw * rw;
            if (fa) {
                m += wp * mu[a];
                if (mu[a] > 0.0) r2 += (dmu[a] / mu[a]) * (dmu[a] / mu[a]);
                a++;
            }
            if (fb) {
                m += wq * mu[b];
                if (mu[b] > 0.0) r2 += (dmu[b] / mu[b]) * (dmu[b] / mu[b]);
                b++;
            }
            src[k] = s;
            mu[k] = m;
            dmu[k] = sqrt(m * m * r2);
            k++;
        }
        for (; k < off[n + 1]; k++) {
            src[k] = 0xFFFFFFFFu;
            mu[k] = 0.0;
            dmu[k] = 0.0;
        }
    }
}

mg_status error_table(mg_graph* g, cudaStream_t s) {
    const int64_t N = g->N;
    const uint32_t S = g->S;
    std::vector<uint2> pq((size_t)N);
    MG_CUDA(cudaMemcpyAsync(pq.data(), g->pq.p, (size_t)N * sizeof(uint2), cudaMemcpyDeviceToHost, s));
    MG_CUDA(cudaStreamSynchronize(s));
    std::vector<uint64_t> off((size_t)N + 1);
    off[0] = 0;
    for (int64_t n = 0; n < N; n++) {
        uint64_t len = 1;
        if (n >= (int64_t)S) {
            if (pq[n].x >= (uint64_t)n || pq[n].y >= (uint64_t)n) return fail(MG_ERR_INVALID_ARG, "malformed node table");
            len = (off[pq[n].x + 1] - off[pq[n].x]) + (off[pq[n].y + 1] - off[pq[n].y]);
        }
        off[n + 1] = off[n] + len;
    }
    const uint64_t E = off[N];
    if (E >= (1ull << 31)) return fail(MG_ERR_UNSUPPORTED, "mixture table above 2^31 entries");
    Buf w_own, dw_own;
    const double *w = nullptr, *dw = nullptr;
    if (g->quantised) {
        w = g->wq.as<double>();
        dw = g->dw.as<double>();
    } else {
        MG_TRY(w_own.alloc(&g->al, (size_t)N * 8, s));
        MG_TRY(dw_own.alloc(&g->al, (size_t)N * 8, s));
        exact_weights_kernel<<<grid_for(N, 256, 152 * 16), 256, 0, s>>>(g->ab.as<ulonglong2>(), N, S,
                                                                        w_own.as<double>(), dw_own.as<double>());
        MG_CUDA(cudaGetLastError());
        w = w_own.as<double>();
        dw = dw_own.as<double>();
    }
    MG_TRY(g->err_off.alloc(&g->al, ((size_t)N + 1) * 8, s));
    MG_TRY(g->err_src.alloc(&g->al, (size_t)std::max<uint64_t>(E, 1) * 4, s));
    MG_TRY(g->err_mu.alloc(&g->al, (size_t)std::max<uint64_t>(E, 1) * 8, s));
    MG_TRY(g->err_dmu.alloc(&g->al, (size_t)std::max<uint64_t>(E, 1) * 8, s));
    MG_CUDA(cudaMemcpyAsync(g->err_off.p, off.data(), ((size_t)N + 1) * 8, cudaMemcpyHostToDevice, s));
    source_rows_kernel<<<grid_for(S, 256), 256, 0, s>>>(g->err_off.as<uint64_t>(), S, g->err_src.as<uint32_t>(),
                                                       g->err_mu.as<double>(), g->err_dmu.as<double>());
    MG_CUDA(cudaGetLastError());
    for (int d = 1; d <= g->D; d++) {
        const int64_t lo = g->bucket[d], hi = g->bucket[d + 1];
        if (hi <= lo) continue;
        level_rows_kernel<<<grid_for(hi - lo, 256, 152 * 16), 256, 0, s>>>(
            g->pq.as<uint2>(), w, dw, lo, hi, g->err_off.as<uint64_t>(), g->err_src.as<uint32_t>(),
            g->err_mu.as<double>(), g->err_dmu.as<double>());
        MG_CUDA(cudaGetLastError());
    }
    MG_CUDA(cudaStreamSynchronize(s));
    for (Buf* b : {&g->err_off, &g->err_src, &g->err_mu, &g->err_dmu}) b->s = nullptr;
    g->err_entries = (int64_t)E;
    return MG_OK;
}

}  // namespace
}  // namespace mg

using namespace mg;

extern "C" {

MG_API mg_status mg_error_table_build(mg_graph* g, int64_t* entries, mg_stream stream) {
    MG_RANGE("mg_error_table_build");
    if (!g) return fail(MG_ERR_INVALID_ARG, "graph is NULL");
    DeviceGuard dg(g->device);
    if (!g->err_off.p) MG_TRY(error_table(g, reinterpret_cast<cudaStream_t>(stream)));
    if (entries) *entries = g->err_entries;
    return MG_OK;
}

MG_API mg_status mg_error_table_copy(const mg_graph* g, int64_t* off, uint32_t* src, double* mu, double* dmu) {
    if (!g) return fail(MG_ERR_INVALID_ARG, "graph is NULL");
    if (!g->err_off.p) return fail(MG_ERR_INVALID_ARG, "no mixture table built (mg_error_table_build)");
    DeviceGuard dg(g->device);
    const size_t E = (size_t)g->err_entries;
    if (off) MG_CUDA(cudaMemcpy(off, g->err_off.p, ((size_t)g->N + 1) * 8, cudaMemcpyDefault));
    if (src) MG_CUDA(cudaMemcpy(src, g->err_src.p, E * 4, cudaMemcpyDefault));
    if (mu) MG_CUDA(cudaMemcpy(mu, g->err_mu.p, E * 8, cudaMemcpyDefault));
    if (dmu) MG_CUDA(cudaMemcpy(dmu, g->err_dmu.p, E * 8, cudaMemcpyDefault));
    return MG_OK;
}

MG_API mg_status mg_query_lut(const mg_graph* g, const int32_t* boxes, int64_t Q, double* hist, double* err,
                              mg_stream stream) {
    MG_RANGE("mg_query_lut");
    if (!g) return fail(MG_ERR_INVALID_ARG, "graph is NULL");
    if (Q < 0 || Q >= (1ll << 31)) return fail(MG_ERR_INVALID_ARG, "Q must be in 0..2^31-1");
    if (Q > 0 && (!boxes || !hist)) return fail(MG_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard dg(g->device);
    return query_lut(g, boxes, Q, hist, err, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"
