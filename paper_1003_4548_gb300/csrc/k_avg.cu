// k_avg.cu -- time averaging, probe points and scalar CDFs (Section 3: once
// the flow is statistically stationary, velocity and scalar statistics are
// averaged in time; scalar concentrations are sampled at wall locations, and
// the cumulative distribution of the scalar is shown at selected points).
//
// While averaging is on, every step adds the element statistics (means,
// second moments, scalar variance) and the node means to FP64 running sums,
// counts the step on the device (so graph replays count too), and adds the
// scalar values of the particles in each CDF probe's element to a histogram.
// Probes locate their element by brute force over the elements (the largest
// smallest barycentric coordinate: the containing element, or the nearest
// one for a point on a wall) and interpolate node fields linearly.
#include <algorithm>
#include <vector>

#include "pdf_internal.cuh"

namespace {

__global__ void k_avg_accumulate(int nt, int nn, const double* __restrict__ emean, const double* __restrict__ eR,
                                 const double* __restrict__ epsivar, const double* __restrict__ nmean,
                                 double* sum, unsigned long long* count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *count += 1ull;
    if (i < nt) {
        double* s = sum + 12 * (size_t)i;
#pragma unroll
        for (int q = 0; q < 5; ++q) s[q] += emean[5 * (size_t)i + q];
#pragma unroll
        for (int q = 0; q < 6; ++q) s[5 + q] += eR[6 * (size_t)i + q];
        s[11] += epsivar[i];
    }
    if (i < nn) {
        double* s = sum + 12 * (size_t)nt + 4 * (size_t)i;
#pragma unroll
        for (int q = 0; q < 4; ++q) s[q] += nmean[4 * (size_t)i + q];
    }
}

// one block per CDF probe: histogram of psi in [0, 1] over its element
template <typename T>
__global__ void __launch_bounds__(256) k_cdf_accumulate(const int* __restrict__ off, const T* __restrict__ psi,
                                                        const int* __restrict__ pelem, int nbins,
                                                        unsigned long long* hist) {
    extern __shared__ unsigned sh[];
    for (int b = threadIdx.x; b < nbins; b += blockDim.x) sh[b] = 0u;
    __syncthreads();
    const int e = pelem[blockIdx.x];
    for (int q = off[e] + threadIdx.x; q < off[e + 1]; q += blockDim.x) {
        const double v = (double)psi[q];
        int b = (int)(v * nbins);
        b = b < 0 ? 0 : (b >= nbins ? nbins - 1 : b);
        atomicAdd(&sh[b], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < nbins; b += blockDim.x)
        hist[(size_t)blockIdx.x * nbins + b] += (unsigned long long)sh[b];
}

// element of each point: the largest smallest barycentric coordinate (x taken
// modulo the period)
__global__ void __launch_bounds__(256) k_locate_points(int nt, const double* __restrict__ egeo, double period,
                                                       const double* __restrict__ px, const double* __restrict__ py,
                                                       int* elem, double* bary) {
    __shared__ double best[256];
    __shared__ int who[256];
    double x = px[blockIdx.x];
    x -= period * floor(x / period);
    const double y = py[blockIdx.x];
    double bm = -1e300;
    int be = 0;
    for (int e = threadIdx.x; e < nt; e += blockDim.x) {
        const double* g = egeo + EGEO_W * (size_t)e;
        const double dx = x - g[0], dy = y - g[1];
        const double l0 = g[2] * dx + g[3] * dy + g[4], l1 = g[5] * dx + g[6] * dy + g[7];
        const double l2 = g[8] * dx + g[9] * dy + g[10];
        const double m = fmin(l0, fmin(l1, l2));
        if (m > bm || (m == bm && e < be)) { bm = m; be = e; }
    }
    best[threadIdx.x] = bm;
    who[threadIdx.x] = be;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            const double o = best[threadIdx.x + w];
            const int oe = who[threadIdx.x + w];
            if (o > best[threadIdx.x] || (o == best[threadIdx.x] && oe < who[threadIdx.x])) {
                best[threadIdx.x] = o;
                who[threadIdx.x] = oe;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int e = who[0];
        elem[blockIdx.x] = e;
        const double* g = egeo + EGEO_W * (size_t)e;
        const double dx = x - g[0], dy = y - g[1];
        bary[3 * blockIdx.x + 0] = g[2] * dx + g[3] * dy + g[4];
        bary[3 * blockIdx.x + 1] = g[5] * dx + g[6] * dy + g[7];
        bary[3 * blockIdx.x + 2] = g[8] * dx + g[9] * dy + g[10];
    }
}

int locate(pdf_ctx* c, const double* x, const double* y, int n, std::vector<int>& elem, std::vector<double>& bary) {
    double* d = nullptr;
    int* de = nullptr;
    PDF_CUDA(c, cudaMalloc((void**)&d, sizeof(double) * 5 * (size_t)n));
    cudaError_t err = cudaMalloc((void**)&de, sizeof(int) * (size_t)n);
    if (err != cudaSuccess) {
        cudaFree(d);
        return fail(c, PDF_ERR_CUDA, std::string("cudaMalloc: ") + cudaGetErrorString(err));
    }
    int st = PDF_OK;
    elem.resize(n);
    bary.resize(3 * (size_t)n);
    err = cudaMemcpyAsync(d, x, sizeof(double) * n, cudaMemcpyHostToDevice, c->s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(d + n, y, sizeof(double) * n, cudaMemcpyHostToDevice, c->s);
    if (err == cudaSuccess) {
        k_locate_points<<<n, 256, 0, c->s>>>(c->m.nt, c->m.egeo_d, c->p.period, d, d + n, de, d + 2 * n);
        ++c->launches;
        err = cudaGetLastError();
    }
    if (err == cudaSuccess) err = cudaMemcpyAsync(elem.data(), de, sizeof(int) * n, cudaMemcpyDeviceToHost, c->s);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(bary.data(), d + 2 * n, sizeof(double) * 3 * n, cudaMemcpyDeviceToHost, c->s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(c->s);
    if (err != cudaSuccess) st = fail(c, PDF_ERR_CUDA, std::string("probe location: ") + cudaGetErrorString(err));
    cudaFree(d);
    cudaFree(de);
    return st;
}

}  // namespace

int launch_averaging(pdf_ctx* c) {
    if (!c->avg_on) return PDF_OK;
    const int nt = c->m.nt, nn = c->m.nn, m = std::max(nt, nn);
    k_avg_accumulate<<<(m + 255) / 256, 256, 0, c->s>>>(nt, nn, c->emean, c->eR, c->epsivar, c->nmean, c->avg_sum,
                                                        c->avg_count);
    ++c->launches;
    if (c->cdf_n > 0) {
        const size_t smem = sizeof(unsigned) * c->cdf_bins;
        if (c->prec == 0)
            k_cdf_accumulate<double><<<c->cdf_n, 256, smem, c->s>>>(c->off, (const double*)c->stA[6], c->cdf_elem,
                                                                    c->cdf_bins, c->cdf_hist);
        else
            k_cdf_accumulate<float><<<c->cdf_n, 256, smem, c->s>>>(c->off, (const float*)c->stA[6], c->cdf_elem,
                                                                   c->cdf_bins, c->cdf_hist);
        ++c->launches;
    }
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

extern "C" {

int pdf_set_averaging(pdf_ctx* c, int32_t on, int32_t reset) {
    if (!c) return PDF_ERR_ARG;
    const int nt = c->m.nt, nn = c->m.nn;
    const size_t nsum = 12 * (size_t)nt + 4 * (size_t)nn;
    if (!c->avg_sum) {
        PDF_CUDA(c, cudaMalloc((void**)&c->avg_sum, sizeof(double) * nsum));
        PDF_CUDA(c, cudaMalloc((void**)&c->avg_count, sizeof(unsigned long long)));
        reset = 1;
    }
    if (reset) {
        PDF_CUDA(c, cudaMemsetAsync(c->avg_sum, 0, sizeof(double) * nsum, c->s));
        PDF_CUDA(c, cudaMemsetAsync(c->avg_count, 0, sizeof(unsigned long long), c->s));
        if (c->cdf_hist)
            PDF_CUDA(c, cudaMemsetAsync(c->cdf_hist, 0, sizeof(unsigned long long) * c->cdf_n * c->cdf_bins, c->s));
    }
    c->avg_on = on ? 1 : 0;
    return PDF_OK;
}

int64_t pdf_averaging_count(pdf_ctx* c) {
    if (!c || !c->avg_count) return 0;
    unsigned long long n = 0;
    if (cudaStreamSynchronize(c->s) != cudaSuccess) return -1;
    if (cudaMemcpy(&n, c->avg_count, sizeof(n), cudaMemcpyDeviceToHost) != cudaSuccess) return -1;
    return (int64_t)n;
}

int pdf_get_averages(pdf_ctx* c, int32_t which, double* out) {
    if (!c || !out || which < 0 || which > 3) return PDF_ERR_ARG;
    if (!c->avg_sum) return fail(c, PDF_ERR_STATE, "averaging was never enabled");
    const int nt = c->m.nt, nn = c->m.nn;
    const size_t nsum = 12 * (size_t)nt + 4 * (size_t)nn;
    std::vector<double> h(nsum);
    unsigned long long n = 0;
    PDF_CUDA(c, cudaStreamSynchronize(c->s));
    PDF_CUDA(c, cudaMemcpy(h.data(), c->avg_sum, sizeof(double) * nsum, cudaMemcpyDeviceToHost));
    PDF_CUDA(c, cudaMemcpy(&n, c->avg_count, sizeof(n), cudaMemcpyDeviceToHost));
    if (n == 0) return fail(c, PDF_ERR_STATE, "no averaged steps");
    const double inv = 1.0 / (double)n;
    const int width[4] = {5, 6, 1, 4}, first[4] = {0, 5, 11, 0};
    const int rows = which == 3 ? nn : nt;
    for (int r = 0; r < rows; ++r)
        for (int q = 0; q < width[which]; ++q)
            out[(size_t)width[which] * r + q] =
                (which == 3 ? h[12 * (size_t)nt + 4 * (size_t)r + q] : h[12 * (size_t)r + first[which] + q]) * inv;
    return PDF_OK;
}

int pdf_probe(pdf_ctx* c, int32_t which, int32_t comp, const double* x, const double* y, int32_t n, double* out,
              int32_t* elem_out) {
    if (!c || !x || !y || !out || n < 0) return PDF_ERR_ARG;
    const int width[6] = {4, 5, 6, 4, 5, 6};  // node mean, elem mean, elem R; then the time averages
    if (which < 0 || which > 5 || comp < 0 || comp >= width[which]) return fail(c, PDF_ERR_ARG, "bad probe field");
    if (n == 0) return PDF_OK;
    if (which >= 3 && !c->avg_sum) return fail(c, PDF_ERR_STATE, "averaging was never enabled");
    std::vector<int> el;
    std::vector<double> bary;
    TRY_OK(locate(c, x, y, n, el, bary));
    const int nt = c->m.nt, nn = c->m.nn;
    std::vector<int> tri(3 * (size_t)nt);
    PDF_CUDA(c, cudaMemcpy(tri.data(), c->m.tri, sizeof(int) * 3 * (size_t)nt, cudaMemcpyDeviceToHost));
    std::vector<double> field;
    if (which < 3) {
        const double* src = which == 0 ? c->nmean : (which == 1 ? c->emean : c->eR);
        const size_t cnt = (size_t)width[which] * (which == 0 ? nn : nt);
        field.resize(cnt);
        PDF_CUDA(c, cudaStreamSynchronize(c->s));
        PDF_CUDA(c, cudaMemcpy(field.data(), src, sizeof(double) * cnt, cudaMemcpyDeviceToHost));
    } else {
        field.resize((size_t)width[which] * (which == 3 ? nn : nt));
        const int st = pdf_get_averages(c, which == 3 ? 3 : (which == 4 ? 0 : 1), field.data());
        if (st != PDF_OK) return st;
    }
    for (int k = 0; k < n; ++k) {
        const int e = el[k];
        if (elem_out) elem_out[k] = e;
        if (which == 0 || which == 3) {  // node field, linear in the element
            double v = 0.0;
            for (int m = 0; m < 3; ++m) v += bary[3 * k + m] * field[4 * (size_t)tri[3 * e + m] + comp];
            out[k] = v;
        } else {
            out[k] = field[(size_t)width[which] * e + comp];
        }
    }
    return PDF_OK;
}

int pdf_set_cdf_probes(pdf_ctx* c, const double* x, const double* y, int32_t n, int32_t nbins) {
    if (!c || n < 0 || nbins < 1 || nbins > 4096 || (n > 0 && (!x || !y))) return PDF_ERR_ARG;
    cudaFree(c->cdf_elem);
    cudaFree(c->cdf_hist);
    c->cdf_elem = nullptr;
    c->cdf_hist = nullptr;
    c->cdf_n = 0;
    if (n == 0) return PDF_OK;
    std::vector<int> el;
    std::vector<double> bary;
    TRY_OK(locate(c, x, y, n, el, bary));
    PDF_CUDA(c, cudaMalloc((void**)&c->cdf_elem, sizeof(int) * n));
    PDF_CUDA(c, cudaMalloc((void**)&c->cdf_hist, sizeof(unsigned long long) * (size_t)n * nbins));
    PDF_CUDA(c, cudaMemcpy(c->cdf_elem, el.data(), sizeof(int) * n, cudaMemcpyHostToDevice));
    PDF_CUDA(c, cudaMemset(c->cdf_hist, 0, sizeof(unsigned long long) * (size_t)n * nbins));
    c->cdf_n = n;
    c->cdf_bins = nbins;
    return PDF_OK;
}

int pdf_get_cdf(pdf_ctx* c, double* out, int32_t* elem_out) {
    if (!c || !out) return PDF_ERR_ARG;
    if (c->cdf_n == 0) return fail(c, PDF_ERR_STATE, "no CDF probes");
    const size_t m = (size_t)c->cdf_n * c->cdf_bins;
    std::vector<unsigned long long> h(m);
    PDF_CUDA(c, cudaStreamSynchronize(c->s));
    PDF_CUDA(c, cudaMemcpy(h.data(), c->cdf_hist, sizeof(unsigned long long) * m, cudaMemcpyDeviceToHost));
    if (elem_out) PDF_CUDA(c, cudaMemcpy(elem_out, c->cdf_elem, sizeof(int) * c->cdf_n, cudaMemcpyDeviceToHost));
    for (int p = 0; p < c->cdf_n; ++p) {
        unsigned long long tot = 0, run = 0;
        for (int b = 0; b < c->cdf_bins; ++b) tot += h[(size_t)p * c->cdf_bins + b];
        for (int b = 0; b < c->cdf_bins; ++b) {
            run += h[(size_t)p * c->cdf_bins + b];
            out[(size_t)p * c->cdf_bins + b] = tot ? (double)run / (double)tot : 0.0;
        }
    }
    return PDF_OK;
}

}  // extern "C"
