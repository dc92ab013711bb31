// k_sort.cu -- keeps the particle state sorted by host element.
//
// The particle kernel leaves per-element counts; a grid-wide scan (block
// totals, then each block's offsets from the totals before it) turns them
// into segment offsets, then every particle claims a slot in its element's
// segment with a warp-aggregated atomic and moves its state there. The order
// inside a segment is not fixed; every later reduction orders the segment by
// (velocity, id) first, so results do not depend on it.
#include <mutex>

#include "pdf_internal.cuh"

namespace {

constexpr int SCAN_THREADS = 1024;

// exclusive scan of the element counts by one block (the allocation-free
// entry point, whose scratch holds no block totals): warp w owns a contiguous
// range of elements; pass 1 sums it with coalesced loads, warp 0 scans the 32
// totals, pass 2 scans the range 32 elements at a time with a running carry.
// Both passes load eight rows of 32 counts together, so a pass waits on
// memory once per 256 counts instead of once per row.
__global__ void __launch_bounds__(SCAN_THREADS) k_scan(const int* __restrict__ cnt, int nt, int* off,
                                                       int* cursor, uint32_t* bump) {
    if (bump != nullptr && threadIdx.x == 0) *bump += 1u;  // the step counter moves with the re-sort
    __shared__ int warp_ex[SCAN_THREADS / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    constexpr int NW = SCAN_THREADS / 32;
    const int per = (nt + NW - 1) / NW;
    const int b0 = min(nt, wid * per), b1 = min(nt, b0 + per);
    int s = 0;
    for (int e0 = b0 + lane; e0 < b1; e0 += 32 * 8) {
        int c8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) c8[k] = e0 + 32 * k < b1 ? cnt[e0 + 32 * k] : 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) s += c8[k];
    }
    s = __reduce_add_sync(0xffffffffu, s);
    if (lane == 0) warp_ex[wid] = s;
    __syncthreads();
    if (wid == 0) {
        const int v = lane < NW ? warp_ex[lane] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane < NW) warp_ex[lane] = incl - v;
        if (lane == 31) off[nt] = incl;
    }
    __syncthreads();
    int carry = warp_ex[wid];
    for (int e0 = b0; e0 < b1; e0 += 32 * 8) {
        int c8[8], i8[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = e0 + 32 * k + lane;
            c8[k] = e < b1 ? cnt[e] : 0;
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {  // eight independent row scans
            i8[k] = c8[k];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, i8[k], o);
                if (lane >= o) i8[k] += y;
            }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const int e = e0 + 32 * k + lane;
            if (e < b1) {
                off[e] = carry + i8[k] - c8[k];
                cursor[e] = carry + i8[k] - c8[k];
            }
            carry += __shfl_sync(0xffffffffu, i8[k], 31);
        }
    }
}

// grid-wide exclusive scan of the element counts in two launches, SCAN_CHUNK
// counts per block of 256 threads (four consecutive counts per thread), no
// block waiting on another: k_scan_part writes each block's total,
// k_scan_fin adds the totals of the blocks before its own and scans its chunk
__device__ __forceinline__ void load4(const int* __restrict__ p, int e0, int n, int (&c)[4]) {
    if (e0 + 3 < n) {
        const int4 v = *reinterpret_cast<const int4*>(p + e0);
        c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) c[k] = e0 + k < n ? p[e0 + k] : 0;
    }
}

__global__ void __launch_bounds__(256) k_scan_part(const int* __restrict__ cnt, int nt, int* part, uint32_t* bump) {
    __shared__ int ws[8];
    if (bump != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *bump += 1u;  // the step counter moves with the re-sort
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
    int c[4];
    load4(cnt, blockIdx.x * SCAN_CHUNK + 4 * t, nt, c);
    int s = __reduce_add_sync(0xffffffffu, c[0] + c[1] + c[2] + c[3]);
    if (lane == 0) ws[wid] = s;
    __syncthreads();
    if (t == 0) {
        s = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) s += ws[w];
        part[blockIdx.x] = s;
    }
}

__global__ void __launch_bounds__(256) k_scan_fin(const int* __restrict__ cnt, int nt, const int* __restrict__ part,
                                                  int* off, int* cursor) {
    __shared__ int ws[8];
    __shared__ int base;
    const int t = threadIdx.x, lane = t & 31, wid = t >> 5, b = blockIdx.x;
    if (wid == 0) {  // counts of the blocks before this one
        int s = 0;
        for (int k = lane; k < b; k += 32) s += part[k];
        s = __reduce_add_sync(0xffffffffu, s);
        if (lane == 0) base = s;
    }
    const int e0 = b * SCAN_CHUNK + 4 * t;
    int c[4];
    load4(cnt, e0, nt, c);
    const int loc = c[0] + c[1] + c[2] + c[3];
    int incl = loc;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[wid] = incl;
    __syncthreads();
    int run = base + incl - loc;
    for (int w = 0; w < wid; ++w) run += ws[w];
    int o4[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        o4[k] = run;
        run += c[k];
    }
    if (e0 + 3 < nt) {
        *reinterpret_cast<int4*>(off + e0) = make_int4(o4[0], o4[1], o4[2], o4[3]);
        *reinterpret_cast<int4*>(cursor + e0) = make_int4(o4[0], o4[1], o4[2], o4[3]);
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (e0 + k < nt) off[e0 + k] = cursor[e0 + k] = o4[k];
    }
    if (b == (int)gridDim.x - 1 && t == 255) off[nt] = run;  // the total (counts past nt are zeros)
}

__global__ void __launch_bounds__(256) k_count(int64_t n, const int* __restrict__ elem, int nt, int* cnt,
                                               int* status) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int e = elem[i];
    if (e < 0 || e >= nt) {
        set_status(status, ST_CAPACITY);
        e = 0;
    }
    const unsigned mask = __match_any_sync(__activemask(), e);
    if ((threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(&cnt[e], __popc(mask));
}

template <typename T>
__global__ void __launch_bounds__(512) k_scatter(int64_t n, const T* __restrict__ x, const T* __restrict__ y,
                                                 const T* __restrict__ u, const T* __restrict__ v,
                                                 const T* __restrict__ w, const T* __restrict__ om,
                                                 const T* __restrict__ psi, const uint32_t* __restrict__ id,
                                                 const int* __restrict__ elem, int nt, int* cursor, T* x2,
                                                 T* y2, T* u2, T* v2, T* w2, T* om2, T* psi2, uint32_t* id2,
                                                 int* elem2) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int e = elem[i];
    if (e < 0 || e >= nt) e = 0;  // reported by k_count
    const unsigned mask = __match_any_sync(__activemask(), e);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&cursor[e], __popc(mask));
    base = __shfl_sync(mask, base, leader);
    const int64_t slot = base + __popc(mask & ((1u << lane) - 1u));
    x2[slot] = x[i]; y2[slot] = y[i]; u2[slot] = u[i]; v2[slot] = v[i]; w2[slot] = w[i];
    om2[slot] = om[i]; psi2[slot] = psi[i]; id2[slot] = id[i]; elem2[slot] = e;
}

template <typename T>
void scatter(pdf_ctx* c, unsigned blocks, int threads) {
    T** A = (T**)c->stA;
    T** B = (T**)c->stB;
    k_scatter<T><<<blocks, threads, 0, c->s>>>(c->np, A[0], A[1], A[2], A[3], A[4], A[5], A[6], c->idA, c->elemA,
                                           c->m.nt, c->cursor, B[0], B[1], B[2], B[3], B[4], B[5], B[6],
                                           c->idB, c->elemB);
}

__global__ void __launch_bounds__(256) k_scatter_perm(int64_t n, const int* __restrict__ elem, int nt, int* cursor,
                                                      int* perm) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int e = elem[i];
    if (e < 0 || e >= nt) e = 0;  // reported by k_count
    const unsigned mask = __match_any_sync(__activemask(), e);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(&cursor[e], __popc(mask));
    base = __shfl_sync(mask, base, leader);
    perm[base + __popc(mask & ((1u << lane) - 1u))] = (int)i;
}

}  // namespace

// ---------------------------------------------------------------------------
// allocation-free sort: scratch in a fixed device array shared by every call
// ---------------------------------------------------------------------------
constexpr int STATIC_SORT_WORDS = 2 * PDF_SORT_STATIC_MAX_ELEMENTS + 64;  // counts, cursors, status (1 MiB)
static __device__ __align__(256) int g_static_sort_scratch[STATIC_SORT_WORDS];

namespace {
constexpr int STATIC_MAX_DEVICES = 64;
std::mutex g_static_mu;
int* g_static_ptr[STATIC_MAX_DEVICES] = {};

// device address of the scratch array on the current device, looked up once
// per device (with that device current)
int static_scratch(int** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(nullptr, PDF_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
    if (dev < 0 || dev >= STATIC_MAX_DEVICES) return fail(nullptr, PDF_ERR_CUDA, "device ordinal out of range");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_sort_scratch);
        if (e != cudaSuccess || !p)
            return fail(nullptr, PDF_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        g_static_ptr[dev] = (int*)p;
    }
    *out = g_static_ptr[dev];
    return PDF_OK;
}
}  // namespace

extern "C" int pdf_sort_by_element_static(const int32_t* elem, int64_t n, int32_t nt, int32_t* perm, int32_t* off,
                                          void* cuda_stream) {
    if (!off || nt < 1 || n < 0 || (n > 0 && (!elem || !perm)))
        return fail(nullptr, PDF_ERR_ARG, "pdf_sort_by_element_static: NULL array, nt < 1 or n < 0");
    if (nt > PDF_SORT_STATIC_MAX_ELEMENTS)
        return fail(nullptr, PDF_ERR_CAPACITY,
                    "pdf_sort_by_element_static: nt = " + std::to_string(nt) + " exceeds the maximum of " +
                        std::to_string(PDF_SORT_STATIC_MAX_ELEMENTS) + " elements");
    if (n > 0x7fffffffll)
        return fail(nullptr, PDF_ERR_CAPACITY, "pdf_sort_by_element_static: more than INT32_MAX particles");
    int* base = nullptr;
    const int st0 = static_scratch(&base);
    if (st0 != PDF_OK) return st0;
    int* cnt = base;
    int* cursor = base + PDF_SORT_STATIC_MAX_ELEMENTS;
    int* status = base + 2 * PDF_SORT_STATIC_MAX_ELEMENTS;
    cudaStream_t s = (cudaStream_t)cuda_stream;
#define STATIC_CUDA(call)                                                                              \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return fail(nullptr, PDF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
    STATIC_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * (size_t)nt, s));
    STATIC_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));
    const unsigned blocks = (unsigned)((n + 255) / 256);
    if (n > 0) k_count<<<blocks, 256, 0, s>>>(n, elem, nt, cnt, status);
    k_scan<<<1, SCAN_THREADS, 0, s>>>(cnt, nt, off, cursor, nullptr);
    if (n > 0) k_scatter_perm<<<blocks, 256, 0, s>>>(n, elem, nt, cursor, perm);
    STATIC_CUDA(cudaGetLastError());
    int h = 0;
    STATIC_CUDA(cudaMemcpyAsync(&h, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    STATIC_CUDA(cudaStreamSynchronize(s));
#undef STATIC_CUDA
    if (h & ST_CAPACITY) return fail(nullptr, PDF_ERR_ARG, "pdf_sort_by_element_static: element index outside [0, nt)");
    return PDF_OK;
}

int launch_sort(pdf_ctx* c, bool advance_step) {
    timing_begin(c, PDF_K_SORT);
    const int nb = scan_blocks(c->m.nt);
    k_scan_part<<<nb, 256, 0, c->s>>>(c->cnt, c->m.nt, c->scan_part, advance_step ? c->d_step : nullptr);
    k_scan_fin<<<nb, 256, 0, c->s>>>(c->cnt, c->m.nt, c->scan_part, c->off, c->cursor);
    c->launches += 2;
    if (c->np > 0) {
        const int th = c->scatter_threads;
        const unsigned blocks = (unsigned)((c->np + th - 1) / th);
        if (c->prec == 0) scatter<double>(c, blocks, th);
        else scatter<float>(c, blocks, th);
        ++c->launches;
    }
    timing_end(c, PDF_K_SORT);
    PDF_CUDA(c, cudaGetLastError());
    for (int k = 0; k < 7; ++k) std::swap(c->stA[k], c->stB[k]);
    std::swap(c->idA, c->idB);
    std::swap(c->elemA, c->elemB);
    return PDF_OK;
}

int launch_count_and_sort(pdf_ctx* c) {
    PDF_CUDA(c, cudaMemsetAsync(c->cnt, 0, sizeof(int) * c->m.nt, c->s));
    if (c->np > 0)
    {
        k_count<<<(unsigned)((c->np + 255) / 256), 256, 0, c->s>>>(c->np, c->elemA, c->m.nt, c->cnt,
                                                                   c->d_status);
        ++c->launches;
    }
    PDF_CUDA(c, cudaGetLastError());
    return launch_sort(c);
}
