// k_stats.cu -- element moments and velocity-conditioned scalar means.
//
// One block per element works on the element's contiguous segment of the
// sorted particle state. The segment's keys (velocity component, particle id)
// are sorted in shared memory with a bitonic network (global scratch for
// segments above STATS_CAP particles):
//  * after the first sort (by U, then id) the segment is in a canonical order,
//    and the ensemble averages of Section 2 (n, <U_i>, central <u_i u_j>,
//    <psi>, psi variance, <omega>) are reduced in that order, so the result
//    does not depend on where the sort put each particle;
//  * the equal-population bins of <phi|V> (Section 3, 2x2x2 by default) split
//    the sorted segment into nb1 groups, re-sort each group by (V, id) and
//    split into nb2, then by (W, id) into nb3; <phi|V> of a bin is its mean psi.
// Reductions are FP64 (or compensated FP32 with PDF_FP32_KAHAN).
//
// FP32 particle state with 2 x 2 x 2 bins, the production path, for elements
// of at most 512 particles: one warp per element computes the moments
// (k_moments_w: exact fixed-point sums for FP32, compensated FP32 sums for
// FP32 + Kahan) on a high-priority side stream; beside it, on a third
// stream, one warp per element (k_bins_med) keeps the segment in registers
// and shared memory and finds each split's median from a 256-bucket
// histogram (over the element's own value range) plus an exact rank of the
// few keys in the median's bucket, one pass over the keys per level (no
// sort). Only the next particle step reads the bins, so they run beside the
// moments and the field chain, which needs the moments alone. Crowded
// elements (more than 512 particles, listed by k_crowded) go to 256-thread
// teams, and elements above 4096 to the block kernel above, moments and bins
// together on the context stream. Other bin shapes take the warp bitonic
// kernel (k_moments_warp).
#include <algorithm>

#include "pdf_internal.cuh"
#include "exact_sum.cuh"

namespace {

struct AccD {
    double s = 0.0;
    __device__ void add(double x) { s += x; }
    __device__ void merge(const AccD& o) { s += o.s; }
    __device__ double value() const { return s; }
    __device__ AccD shfl_down(int o) const {
        AccD r;
        r.s = __shfl_down_sync(0xffffffffu, s, o);
        return r;
    }
};

// compensated FP32 sum: c accumulates the exact rounding error of every
// addition (Knuth's TwoSum, branch-free; the same error term as Neumaier's
// form), merges add the compensations
struct AccK {
    float s = 0.f, c = 0.f;
    __device__ void add(float x) {
        const float t = s + x;
        const float bp = t - s;
        c += (s - (t - bp)) + (x - bp);
        s = t;
    }
    __device__ void merge(const AccK& o) {
        add(o.s);
        c += o.c;
    }
    __device__ double value() const { return (double)s + (double)c; }
    __device__ AccK shfl_down(int o) const {
        AccK r;
        r.s = __shfl_down_sync(0xffffffffu, s, o);
        r.c = __shfl_down_sync(0xffffffffu, c, o);
        return r;
    }
};

template <typename T, bool KAHAN> struct AccSel { using type = AccD; using R = double; };
template <> struct AccSel<float, true> { using type = AccK; using R = float; };

__device__ __forceinline__ bool key_gt(const SortKey& a, const SortKey& b) {
    const uint32_t ga = a.gi >> 24, gb = b.gi >> 24;
    if (ga != gb) return ga > gb;
    if (a.v != b.v) return a.v > b.v;
    return a.id > b.id;
}

// ascending bitonic sort of K[0..N2), N2 a power of two
__device__ void bitonic(SortKey* K, int N2) {
    const int half = N2 >> 1;
    for (int k = 2; k <= N2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int p = threadIdx.x; p < half; p += blockDim.x) {
                const int i = 2 * j * (p / j) + (p % j);
                const int ixj = i + j;
                const SortKey A = K[i], Bk = K[ixj];
                const bool asc = (i & k) == 0;
                if (asc ? key_gt(A, Bk) : key_gt(Bk, A)) {
                    K[i] = Bk;
                    K[ixj] = A;
                }
            }
            __syncthreads();
        }
    }
}

// deterministic block reduction of NV accumulators (fixed tree)
template <typename Acc, int NV>
__device__ void block_reduce(Acc (&acc)[NV], double (&out)[NV]) {
    __shared__ Acc part[STATS_THREADS / 32][NV];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q].merge(acc[q].shfl_down(o));
    }
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) part[wid][q] = acc[q];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        Acc t = part[0][q];
        for (int w = 1; w < STATS_THREADS / 32; ++w) t.merge(part[w][q]);
        out[q] = t.value();
    }
    __syncthreads();
}

template <typename T>
struct MomArgs {
    const int* __restrict__ off;
    const T* __restrict__ u;
    const T* __restrict__ v;
    const T* __restrict__ w;
    const T* __restrict__ om;
    const T* __restrict__ psi;
    const uint32_t* __restrict__ id;
    int G0, G1, G2, B;
    int* en;
    double *emean, *eR, *epsivar, *ecm;
    T* ecmT;
    unsigned char* bin;
    SortKey* scratch;
    int64_t scratch_n;
    int* status;
    int min_n;  // the block kernel only takes elements with more particles than this
    // FP32 median path: elements too crowded for a warp, listed by k_crowded
    // (lcnt[0]: 512 < n <= 4096 in listA, lcnt[1]: n > 4096 in listB; lcnt[2],
    // lcnt[4]: the next listA entry a block of k_moments_sel_big takes for its
    // moments, for its bins; lcnt[3]: the next element of the warp bins kernel)
    int* lcnt;
    int* listA;
    int* listB;
};

__device__ __forceinline__ int chunk_of(int r, int m, int G) {
    const int base = m / G, rem = m % G;
    const int big = rem * (base + 1);
    return r < big ? r / (base + 1) : rem + (r - big) / base;
}

template <typename T, bool KAHAN>
__device__ void moments_element(const MomArgs<T>& a, const int e) {
    using Acc = typename AccSel<T, KAHAN>::type;
    using R = typename AccSel<T, KAHAN>::R;
    extern __shared__ SortKey skeys[];
    __shared__ int gstart[256], gsize[256], nstart[256], nsize[256];
    __shared__ double mean_s[5];
    const int s0 = a.off[e], n = a.off[e + 1] - s0;
    const int B = a.B;
    if (n <= a.min_n) return;  // done by the warp kernel
    if (n == 0) {
        if (threadIdx.x == 0) {
            a.en[e] = 0;
            for (int q = 0; q < 5; ++q) a.emean[5 * e + q] = 0.0;
            for (int q = 0; q < 6; ++q) a.eR[6 * e + q] = 0.0;
            a.epsivar[e] = 0.0;
        }
        for (int b = threadIdx.x; b < B; b += blockDim.x) {
            a.ecm[(size_t)B * e + b] = 0.0;
            a.ecmT[(size_t)B * e + b] = (T)0;
        }
        return;
    }
    int N2 = 1;
    while (N2 < n) N2 <<= 1;
    SortKey* K = skeys;
    if (N2 > STATS_CAP) {
        if ((int64_t)2 * s0 + N2 > a.scratch_n || n > (1 << 24)) {
            if (threadIdx.x == 0) set_status(a.status, ST_CAPACITY);
            return;
        }
        K = a.scratch + (size_t)2 * s0;
    }
    // level 0: (U, id)
    for (int q = threadIdx.x; q < N2; q += blockDim.x) {
        SortKey k;
        if (q < n) {
            k.v = ord_bits(a.u[s0 + q]);
            k.id = a.id[s0 + q];
            k.gi = (uint32_t)q;
        } else {
            k.v = ~0ull;
            k.id = 0xffffffffu;
            k.gi = 0xffffffffu;
        }
        K[q] = k;
    }
    __syncthreads();
    bitonic(K, N2);

    // ensemble averages in the canonical (U, id) order
    {
        Acc acc[5];
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            const int j = s0 + (int)(K[q].gi & 0xffffffu);
            acc[0].add((R)a.u[j]);
            acc[1].add((R)a.v[j]);
            acc[2].add((R)a.w[j]);
            acc[3].add((R)a.psi[j]);
            acc[4].add((R)a.om[j]);
        }
        double s[5];
        block_reduce<Acc, 5>(acc, s);
        if (threadIdx.x == 0)
            for (int q = 0; q < 5; ++q) mean_s[q] = s[q] / n;
        __syncthreads();
        const R mu = (R)mean_s[0], mv = (R)mean_s[1], mw = (R)mean_s[2], mp = (R)mean_s[3];
        Acc c2[7];
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            const int j = s0 + (int)(K[q].gi & 0xffffffu);
            const R du = (R)a.u[j] - mu, dv = (R)a.v[j] - mv, dw = (R)a.w[j] - mw, dp = (R)a.psi[j] - mp;
            c2[0].add(du * du);
            c2[1].add(dv * dv);
            c2[2].add(dw * dw);
            c2[3].add(du * dv);
            c2[4].add(du * dw);
            c2[5].add(dv * dw);
            c2[6].add(dp * dp);
        }
        double r2[7];
        block_reduce<Acc, 7>(c2, r2);
        if (threadIdx.x == 0) {
            a.en[e] = n;
            for (int q = 0; q < 5; ++q) a.emean[5 * e + q] = mean_s[q];
            for (int q = 0; q < 6; ++q) a.eR[6 * e + q] = r2[q] / n;
            a.epsivar[e] = r2[6] / n;
        }
    }

    // equal-population bins
    if (n < B) {
        for (int q = threadIdx.x; q < n; q += blockDim.x) a.bin[s0 + q] = 0;
        for (int b = threadIdx.x; b < B; b += blockDim.x) {
            a.ecm[(size_t)B * e + b] = mean_s[3];
            a.ecmT[(size_t)B * e + b] = (T)mean_s[3];
        }
        return;
    }
    const int G[3] = {a.G0, a.G1, a.G2};
    if (threadIdx.x == 0) { gstart[0] = 0; gsize[0] = n; }
    __syncthreads();
    int ngroups = 1;
    for (int d = 0; d < 3; ++d) {
        if (d > 0) {
            const T* comp = d == 1 ? a.v : a.w;
            for (int q = threadIdx.x; q < n; q += blockDim.x) K[q].v = ord_bits(comp[s0 + (K[q].gi & 0xffffffu)]);
            __syncthreads();
            bitonic(K, N2);
        }
        for (int q = threadIdx.x; q < n; q += blockDim.x) {
            const uint32_t gi = K[q].gi;
            const int g = (int)(gi >> 24);
            const int h = chunk_of(q - gstart[g], gsize[g], G[d]);
            K[q].gi = ((uint32_t)(g * G[d] + h) << 24) | (gi & 0xffffffu);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int t = 0;
            for (int g = 0; g < ngroups; ++g) {
                int st = gstart[g];
                const int m = gsize[g];
                for (int h = 0; h < G[d]; ++h, ++t) {
                    const int sz = m / G[d] + (h < m % G[d] ? 1 : 0);
                    nstart[t] = st;
                    nsize[t] = sz;
                    st += sz;
                }
            }
            for (int g = 0; g < t; ++g) { gstart[g] = nstart[g]; gsize[g] = nsize[g]; }
        }
        ngroups *= G[d];
        __syncthreads();
    }
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        const uint32_t gi = K[q].gi;
        a.bin[s0 + (gi & 0xffffffu)] = (unsigned char)(gi >> 24);
    }
    // <phi|V> per bin: one warp per bin over its contiguous sorted range
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int b = wid; b < B; b += STATS_THREADS / 32) {
        Acc acc;
        for (int q = gstart[b] + lane; q < gstart[b] + gsize[b]; q += 32)
            acc.add((R)a.psi[s0 + (K[q].gi & 0xffffffu)]);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc.merge(acc.shfl_down(o));
        if (lane == 0) {
            const double cm = acc.value() / gsize[b];
            a.ecm[(size_t)B * e + b] = cm;
            a.ecmT[(size_t)B * e + b] = (T)cm;
        }
    }
}

// one block per element (FP64 path, every element), or a persistent grid over
// the listed crowded elements (FP32 median path)
template <typename T, bool KAHAN>
__global__ void __launch_bounds__(STATS_THREADS) k_moments(const MomArgs<T> a) {
    if (a.listB == nullptr) {
        moments_element<T, KAHAN>(a, blockIdx.x);
        return;
    }
    const int cnt = a.lcnt[1];
    for (int j = blockIdx.x; j < cnt; j += gridDim.x) {
        moments_element<T, KAHAN>(a, a.listB[j]);
        __syncthreads();
    }
}


// ---------------------------------------------------------------------------
// warp-per-element variant for FP32 particle state (segments up to
// WARP_MAX_N particles): the keys (group|index, value bits, id) live in the
// warp's slice of shared memory as three word arrays and a bitonic network
// runs warp-synchronously over them; group ranges of each level are
// tabulated once per element.
// ---------------------------------------------------------------------------
constexpr int WARP_MAX_N = 512;
constexpr int WARPS_PER_BLOCK = 4;

struct WarpSmem {
    uint32_t gi[WARP_MAX_N];  // group << 16 | index in the segment
    uint32_t v[WARP_MAX_N];   // order-preserving value bits
    uint32_t id[WARP_MAX_N];
    float psi[WARP_MAX_N];
    short gst[256], gsz[256], nst[256], nsz[256];
};

__device__ __forceinline__ uint32_t ord32(float v) {
    v = v + 0.0f;
    const uint32_t b = __float_as_uint(v);
    return (b >> 31) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float ord32_inv(uint32_t k) {
    return (k >> 31) ? __uint_as_float(k & 0x7fffffffu) : __uint_as_float(~k);
}

__device__ __forceinline__ bool wgt(uint32_t ga, uint32_t va, uint32_t ia, uint32_t gb, uint32_t vb, uint32_t ib) {
    ga >>= 16;
    gb >>= 16;
    if (ga != gb) return ga > gb;
    if (va != vb) return va > vb;
    return ia > ib;
}

__device__ void warp_bitonic(WarpSmem& S, int N2, int lane) {
    const int half = N2 >> 1;
    for (int k = 2; k <= N2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            const int lj = __ffs(j) - 1;
            for (int p = lane; p < half; p += 32) {
                const int i = ((p >> lj) << (lj + 1)) + (p & (j - 1));
                const int q = i + j;
                const uint32_t ga = S.gi[i], va = S.v[i], ia = S.id[i];
                const uint32_t gb = S.gi[q], vb = S.v[q], ib = S.id[q];
                const bool asc = (i & k) == 0;
                if (asc == wgt(ga, va, ia, gb, vb, ib)) {
                    S.gi[i] = gb; S.v[i] = vb; S.id[i] = ib;
                    S.gi[q] = ga; S.v[q] = va; S.id[q] = ia;
                }
            }
            __syncwarp();
        }
    }
}

template <typename Acc>
__device__ __forceinline__ void warp_tree(Acc& a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a.merge(a.shfl_down(o));
}

template <bool KAHAN>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK) k_moments_warp(const MomArgs<float> a, int nt) {
    using Acc = typename AccSel<float, KAHAN>::type;
    using R = typename AccSel<float, KAHAN>::R;
    __shared__ WarpSmem sm[WARPS_PER_BLOCK];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int e = blockIdx.x * WARPS_PER_BLOCK + w;
    if (e >= nt) return;
    const int s0 = a.off[e], n = a.off[e + 1] - s0;
    if (n > WARP_MAX_N) return;  // the block kernel takes it
    const int B = a.B;
    WarpSmem& S = sm[w];
    if (n == 0) {
        if (lane == 0) {
            a.en[e] = 0;
            for (int q = 0; q < 5; ++q) a.emean[5 * e + q] = 0.0;
            for (int q = 0; q < 6; ++q) a.eR[6 * e + q] = 0.0;
            a.epsivar[e] = 0.0;
        }
        for (int b = lane; b < B; b += 32) {
            a.ecm[(size_t)B * e + b] = 0.0;
            a.ecmT[(size_t)B * e + b] = 0.f;
        }
        return;
    }
    int N2 = 32;
    while (N2 < n) N2 <<= 1;
    for (int q = lane; q < N2; q += 32) {
        if (q < n) {
            S.gi[q] = (uint32_t)q;
            S.v[q] = ord32(a.u[s0 + q]);
            S.id[q] = a.id[s0 + q];
        } else {
            S.gi[q] = 0xffffffffu; S.v[q] = 0xffffffffu; S.id[q] = 0xffffffffu;
        }
    }
    __syncwarp();
    warp_bitonic(S, N2, lane);
    // ensemble averages in the canonical (U, id) order, lane-strided
    Acc m[5];
    for (int q = lane; q < n; q += 32) {
        const int j = s0 + (int)(S.gi[q] & 0xffffu);
        m[0].add((R)a.u[j]); m[1].add((R)a.v[j]); m[2].add((R)a.w[j]);
        m[3].add((R)a.psi[j]); m[4].add((R)a.om[j]);
    }
    double mean[5];
#pragma unroll
    for (int q = 0; q < 5; ++q) {
        warp_tree(m[q]);
        mean[q] = __shfl_sync(0xffffffffu, m[q].value(), 0) / n;
    }
    const R mu = (R)mean[0], mv = (R)mean[1], mw = (R)mean[2], mp = (R)mean[3];
    Acc c2[7];
    for (int q = lane; q < n; q += 32) {
        const int j = s0 + (int)(S.gi[q] & 0xffffu);
        const R du = (R)a.u[j] - mu, dv = (R)a.v[j] - mv, dw = (R)a.w[j] - mw, dp = (R)a.psi[j] - mp;
        c2[0].add(du * du); c2[1].add(dv * dv); c2[2].add(dw * dw);
        c2[3].add(du * dv); c2[4].add(du * dw); c2[5].add(dv * dw); c2[6].add(dp * dp);
    }
#pragma unroll
    for (int q = 0; q < 7; ++q) warp_tree(c2[q]);
    if (lane == 0) {
        const double inv_n = 1.0 / n;
        a.en[e] = n;
        for (int q = 0; q < 5; ++q) a.emean[5 * e + q] = mean[q];
        for (int q = 0; q < 6; ++q) a.eR[6 * e + q] = c2[q].value() * inv_n;
        a.epsivar[e] = c2[6].value() * inv_n;
    }
    if (n < B) {
        for (int q = lane; q < n; q += 32) a.bin[s0 + q] = 0;
        for (int b = lane; b < B; b += 32) {
            a.ecm[(size_t)B * e + b] = mean[3];
            a.ecmT[(size_t)B * e + b] = (float)mean[3];
        }
        return;
    }
    const int G[3] = {a.G0, a.G1, a.G2};
    if (lane == 0) { S.gst[0] = 0; S.gsz[0] = (short)n; }
    __syncwarp();
    int ngroups = 1;
    for (int d = 0; d < 3; ++d) {
        const int Gd = G[d];
        if (d > 0) {
            const float* comp = d == 1 ? a.v : a.w;
            for (int q = lane; q < n; q += 32) S.v[q] = ord32(comp[s0 + (S.gi[q] & 0xffffu)]);
            __syncwarp();
            warp_bitonic(S, N2, lane);
        }
        // sub-group table of this level (lane-parallel over the groups)
        for (int g = lane; g < ngroups; g += 32) {
            const int st = S.gst[g], m = S.gsz[g], base = m / Gd, rem = m % Gd;
            int pos = st;
            for (int h = 0; h < Gd; ++h) {
                const int sz = base + (h < rem ? 1 : 0);
                S.nst[g * Gd + h] = (short)pos;
                S.nsz[g * Gd + h] = (short)sz;
                pos += sz;
            }
        }
        __syncwarp();
        for (int q = lane; q < n; q += 32) {
            const uint32_t gi = S.gi[q];
            const int g = (int)(gi >> 16);
            int h = Gd - 1;
            while (h > 0 && q < S.nst[g * Gd + h]) --h;
            S.gi[q] = ((uint32_t)(g * Gd + h) << 16) | (gi & 0xffffu);
        }
        ngroups *= Gd;
        for (int g = lane; g < ngroups; g += 32) { S.gst[g] = S.nst[g]; S.gsz[g] = S.nsz[g]; }
        __syncwarp();
    }
    for (int q = lane; q < n; q += 32) {
        const uint32_t gi = S.gi[q];
        const int j = s0 + (int)(gi & 0xffffu);
        a.bin[j] = (unsigned char)(gi >> 16);
        S.psi[q] = a.psi[j];
    }
    __syncwarp();
    for (int b = lane; b < B; b += 32) {
        const int st = S.gst[b], sz = S.gsz[b];
        Acc acc;
        for (int q = st; q < st + sz; ++q) acc.add((R)S.psi[q]);
        const double cm = acc.value() / sz;
        a.ecm[(size_t)B * e + b] = cm;
        a.ecmT[(size_t)B * e + b] = (float)cm;
    }
}


// ---------------------------------------------------------------------------
// median-split variant (every level halves its groups, as for the 2x2x2
// bins), one warp per element, compact code: the keys of the segment live in
// the warp's shared-memory slice and every pass is a rolled loop over the
// segment (element j handled by lane j % 32).
//  * moments: exact fixed-point sums of the values and their products
//    (integer pipes), correctly rounded to FP64 once per element;
//  * bins: per level and per group the boundary key -- the ceil(m/2)-th
//    smallest (value, id) -- from a 256-bucket histogram over the value range
//    (16-bit counts, two per word) and an exact ranking of the few keys in
//    the boundary bucket; a bisection over the value bits (then the ids) when
//    that bucket is crowded;
//  * <phi|V>: exact fixed-point psi sums per bin (shared-memory atomics).
// ---------------------------------------------------------------------------
// histogram buckets and boundary-bucket candidate cap of a size class (the
// block class ranks up to 64 keys of a crowded bucket before bisecting)
template <int NMAX>
struct SelCfg {
    static constexpr int NB = 256;  // at most 256: a key's bucket is kept in one byte
    static constexpr int CMAX = NMAX <= 512 ? 32 : 64;
};

template <int NMAX>
struct SelSmem {
    uint32_t kv[NMAX];  // order-preserving value bits of the current level
    unsigned char grp[NMAX];
    unsigned char bk8[NMAX];  // histogram bucket of each key at the current level (NB <= 256)
    unsigned hist[4][SelCfg<NMAX>::NB / 2];  // per-group histogram, two 16-bit counts per word
    uint32_t cv[4][SelCfg<NMAX>::CMAX], cid[4][SelCfg<NMAX>::CMAX];  // keys of each group's boundary bucket
    int nc[4], bkt[4], brank[4];
    int cbk[4];                // boundary bucket whose keys are ranked, or -1 (crowded: bisection)
    uint32_t bv[4], bid[4];    // boundary keys of the level's groups
    int ired[8];               // team reduction scratch
    unsigned ured[2][NMAX > 512 ? 8 : 1];
    unsigned long long xred[NMAX > 512 ? 8 : 1][24];  // per-warp exact sums (12 x 128 bit), block teams only
    float kred[NMAX > 512 ? 7 : 1][24];  // warps 1..7's compensated sums (s, c of 12), block teams only
    double mean[5];
    double rd[3];              // <uu>, <vv>, <ww> of the element (bucket ranges of the splits)
    unsigned long long binsum[8];  // sum of psi per bin, unit 2^-(63 - log2 NMAX) (psi in [0, 1])
    int bincnt[8];
};

template <int NMAX>
__device__ __forceinline__ int hcount(const SelSmem<NMAX>& S, int g, int b) {
    return (int)((S.hist[g][b >> 1] >> (16 * (b & 1))) & 0xffffu);
}

// NT threads work on one element: a warp (NT = 32) or a whole block
template <int NT>
struct Team {
    int tid, lane, wid;
    __device__ Team() : tid(threadIdx.x % NT), lane(threadIdx.x & 31), wid((threadIdx.x % NT) >> 5) {}
    __device__ void sync() const {
        if (NT == 32) __syncwarp();
        else __syncthreads();
    }
    template <int NMAX>
    __device__ int sum(int v, SelSmem<NMAX>& S) const {
        v = __reduce_add_sync(0xffffffffu, v);
        if (NT == 32) return v;
        if (lane == 0) S.ired[wid] = v;
        __syncthreads();
        int t = 0;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) t += S.ired[w];
        __syncthreads();
        return t;
    }
    template <int NMAX>
    __device__ void minmax(unsigned& mn, unsigned& mx, SelSmem<NMAX>& S) const {
        mn = __reduce_min_sync(0xffffffffu, mn);
        mx = __reduce_max_sync(0xffffffffu, mx);
        if (NT == 32) return;
        if (lane == 0) { S.ured[0][wid] = mn; S.ured[1][wid] = mx; }
        __syncthreads();
        mn = 0xffffffffu;
        mx = 0u;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) { mn = min(mn, S.ured[0][w]); mx = max(mx, S.ured[1][w]); }
        __syncthreads();
    }
};

__device__ __forceinline__ void x128_add_parts(Exact128& a, unsigned m, int e, bool neg) {
    unsigned long long lo, hi;
    x128_place((unsigned long long)m, e - 70, lo, hi);
    x128_add(a, lo, hi, neg);
}

// #{keys of group g with (v < cv) or (v == cv and id < cid)} over the segment
template <int NT, int NMAX>
__device__ __noinline__ int sel_count(SelSmem<NMAX>& S, const uint32_t* __restrict__ ids, int n, int g, uint32_t cv,
                                      uint32_t cid) {
    const Team<NT> T;
    int c = 0;
    for (int q = T.tid; q < n; q += NT) {
        const uint32_t v = S.kv[q];
        c += (S.grp[q] == g && (v < cv || (v == cv && ids[q] < cid))) ? 1 : 0;
    }
    return T.sum(c, S);
}

// boundary key of group g by bisection over the value bits (then id bits):
// the Tk-th smallest (value, id); used when the histogram leaves too many
// candidates in one bucket
template <int NT, int NMAX>
__device__ __noinline__ void sel_bisect(SelSmem<NMAX>& S, const uint32_t* __restrict__ ids, int n, int g, int Tk,
                                        int gsz, uint32_t prefix, int hb, uint32_t& ans, uint32_t& idb) {
    ans = prefix;
    for (int bit = hb; bit >= 0; --bit) {
        const uint32_t cand = ans | (1u << bit);
        if (sel_count<NT>(S, ids, n, g, cand, 0u) < Tk) ans = cand;
    }
    const int clt = sel_count<NT>(S, ids, n, g, ans, 0u);
    const int cle = ans == 0xffffffffu ? gsz : sel_count<NT>(S, ids, n, g, ans + 1u, 0u);
    idb = 0xffffffffu;
    if (cle - clt > 1 && Tk - clt < cle - clt) {
        uint32_t ia = 0u;
        for (int bit = 31; bit >= 0; --bit) {
            const uint32_t cand = ia | (1u << bit);
            if (sel_count<NT>(S, ids, n, g, ans, cand) - clt < Tk - clt) ia = cand;
        }
        idb = ia;
    }
}

// Bucket of a key for the histogram of one split level: 256 equal-width
// buckets over [mean - 4 sd, mean + 4 sd] of the element's component,
// clamped at both ends. The map is monotone, so the boundary (a median, always
// within one sd of the mean) falls into a bucket with few keys for any smooth
// distribution.
struct Buckets {
    float lo, sc;
    int top;  // number of buckets - 1
    __device__ int operator()(uint32_t k) const {
        return max(0, min(top, (int)((ord32_inv(k) - lo) * sc)));
    }
};

// 1/n for a count n >= 1 with few FP64 instructions (GB300's FP64 pipe is
// narrow): the FP32 reciprocal refined by one Newton step, relative error
// below 1e-14 (n < 2^24)
__device__ __forceinline__ double recip_n(int n) {
    const double r0 = (double)__frcp_rn((float)n), dn = (double)n;
    return fma(r0, fma(-dn, r0, 1.0), r0);
}

// (in FP32: any monotone map is exact for the selection, and FP64 on every
// lane of a warp would occupy GB300's narrow FP64 pipe)
__device__ __forceinline__ Buckets make_buckets(double mean, double var, int nb) {
    const float v = (float)var;
    const float sd = v > 0.f ? sqrtf(v) : 0.f;
    const float sc = sd > 0.f ? (float)nb / (8.f * sd) : 0.f;  // nb buckets over 8 sd
    Buckets b;
    b.top = nb - 1;
    b.lo = (float)mean - 4.f * sd;
    b.sc = (sc > 0.f && sc < 1e30f) ? sc : 0.f;
    return b;
}

// Boundary key of every group g < ng of the current level -- the Tk-th
// smallest (value, id), Tk = ceil(m/2) -- from the level's histogram: the
// bucket where the running count reaches Tk, then an exact rank of the keys
// in that bucket (bisection over the value bits when it holds more than 32).
template <int NT, int NMAX>
__device__ __forceinline__ void sel_boundaries(SelSmem<NMAX>& S, const uint32_t* __restrict__ ids, int n, int ng,
                                            const int (&gsize)[4], const Buckets bk) {
    const Team<NT> T;
    constexpr int NB = SelCfg<NMAX>::NB, PL = NB / 32, CMAX = SelCfg<NMAX>::CMAX;  // PL buckets per lane
    {  // boundary bucket of every group: a warp team scans the groups in
       // turn, a block team gives group g to its warp g
        const int lane = T.lane;
        const int g0 = NT == 32 ? 0 : T.wid, gstep = NT == 32 ? 1 : NT / 32;
        for (int g = g0; g < ng; g += gstep) {
            const int Tk = (gsize[g] + 1) / 2;
            int loc[PL], tot = 0;
#pragma unroll
            for (int k = 0; k < PL / 2; ++k) {
                const unsigned w2 = S.hist[g][(PL / 2) * lane + k];
                loc[2 * k] = (int)(w2 & 0xffffu);
                loc[2 * k + 1] = (int)(w2 >> 16);
                tot += loc[2 * k] + loc[2 * k + 1];
            }
            int incl = tot;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int excl = incl - tot;
            int mybucket = -1, mybelow = 0;
            if (excl < Tk && incl >= Tk) {
                int run = excl;
#pragma unroll
                for (int k = 0; k < PL; ++k) {
                    if (mybucket < 0 && run + loc[k] >= Tk) { mybucket = PL * lane + k; mybelow = run; }
                    run += loc[k];
                }
            }
            const unsigned who = __ballot_sync(0xffffffffu, mybucket >= 0);
            const int src = __ffs(who) - 1;
            const int bucket = __shfl_sync(0xffffffffu, mybucket, src);
            const int below = __shfl_sync(0xffffffffu, mybelow, src);
            if (lane == 0) {
                S.bkt[g] = bucket;
                S.brank[g] = Tk - below - 1;
                S.nc[g] = 0;
                S.cbk[g] = hcount(S, g, bucket) <= CMAX ? bucket : -1;
            }
        }
    }
    T.sync();
    for (int q = T.tid; q < n; q += NT) {  // candidates of all groups in one pass
        const int g = S.grp[q];
        if ((int)S.bk8[q] == S.cbk[g]) {
            const int slot = atomicAdd(&S.nc[g], 1);
            S.cv[g][slot] = S.kv[q];
            S.cid[g][slot] = ids[q];
        }
    }
    T.sync();
    for (int t = T.tid; t < CMAX * ng; t += NT) {  // exact rank among the bucket's keys
        const int g = t / CMAX, j0 = t % CMAX;
        const int kc = hcount(S, g, S.bkt[g]);
        if (kc <= CMAX && j0 < kc) {
            const uint32_t v = S.cv[g][j0], id = S.cid[g][j0];
            int r = 0;
            for (int j = 0; j < kc; ++j) {
                const uint32_t vj = S.cv[g][j];
                r += (vj < v || (vj == v && S.cid[g][j] < id)) ? 1 : 0;
            }
            if (r == S.brank[g]) { S.bv[g] = v; S.bid[g] = id; }
        }
    }
    T.sync();
    for (int g = 0; g < ng; ++g) {  // crowded bucket (rare): bisection over the value bits
        if (hcount(S, g, S.bkt[g]) > CMAX) {
            unsigned vmin = 0xffffffffu, vmax = 0u;
            for (int q = T.tid; q < n; q += NT) {
                vmin = min(vmin, S.kv[q]);
                vmax = max(vmax, S.kv[q]);
            }
            T.minmax(vmin, vmax, S);
            const uint32_t diff = vmin ^ vmax;
            const int hb = diff ? 31 - __clz(diff) : -1;
            const uint32_t prefix = hb >= 0 ? (vmin & ~((2u << hb) - 1u)) : vmin;
            uint32_t bv, bid;
            sel_bisect<NT>(S, ids, n, g, (gsize[g] + 1) / 2, gsize[g], prefix, hb, bv, bid);
            if (T.tid == 0) { S.bv[g] = bv; S.bid[g] = bid; }
            T.sync();
        }
    }
}

// exact moments of the segment; results of the 12 moments computed by warp 0
// (lanes 0..4 the means, 5..10 the central second moments, 11 psi variance)
template <int NT, int NMAX>
__device__ __noinline__ void exact_moments(const MomArgs<float>& a, int e, int s0, int n, SelSmem<NMAX>& S) {
    const Team<NT> T;
    Exact128 s1[5], s2[7];
    bool big = false;
    for (int q = T.tid; q < n; q += NT) {
        unsigned mu_, mv_, mw_, mp_, mo_;
        int eu, ev, ew, ep, eo;
        bool nu, nv, nw, np, no;
        f32_parts(a.u[s0 + q], mu_, eu, nu);
        f32_parts(a.v[s0 + q], mv_, ev, nv);
        f32_parts(a.w[s0 + q], mw_, ew, nw);
        f32_parts(a.psi[s0 + q], mp_, ep, np);
        f32_parts(a.om[s0 + q], mo_, eo, no);
        big |= max(max(max(eu, ev), max(ew, ep)), eo) > 145;  // |x| >= 2^19: outside the format
        x128_add_parts(s1[0], mu_, eu, nu);
        x128_add_parts(s1[1], mv_, ev, nv);
        x128_add_parts(s1[2], mw_, ew, nw);
        x128_add_parts(s1[3], mp_, ep, np);
        x128_add_parts(s1[4], mo_, eo, no);
        x128_add_prod(s2[0], mu_, eu, nu, mu_, eu, nu);
        x128_add_prod(s2[1], mv_, ev, nv, mv_, ev, nv);
        x128_add_prod(s2[2], mw_, ew, nw, mw_, ew, nw);
        x128_add_prod(s2[3], mu_, eu, nu, mv_, ev, nv);
        x128_add_prod(s2[4], mu_, eu, nu, mw_, ew, nw);
        x128_add_prod(s2[5], mv_, ev, nv, mw_, ew, nw);
        x128_add_prod(s2[6], mp_, ep, np, mp_, ep, np);
    }
    if (__any_sync(0xffffffffu, big) && T.lane == 0) set_status(a.status, ST_CAPACITY);
#pragma unroll
    for (int k = 0; k < 5; ++k) x128_warp_sum(s1[k]);
#pragma unroll
    for (int k = 0; k < 7; ++k) x128_warp_sum(s2[k]);
    if (NT > 32) {  // combine the warps' exact sums (exact, so in any order)
        if (T.lane == 0) {
#pragma unroll
            for (int k = 0; k < 5; ++k) { S.xred[T.wid][2 * k] = s1[k].lo; S.xred[T.wid][2 * k + 1] = s1[k].hi; }
#pragma unroll
            for (int k = 0; k < 7; ++k) { S.xred[T.wid][10 + 2 * k] = s2[k].lo; S.xred[T.wid][11 + 2 * k] = s2[k].hi; }
        }
        __syncthreads();
        if (T.wid == 0 && T.lane == 0) {
            for (int w = 1; w < NT / 32; ++w) {
#pragma unroll
                for (int k = 0; k < 5; ++k) x128_add(s1[k], S.xred[w][2 * k], S.xred[w][2 * k + 1], false);
#pragma unroll
                for (int k = 0; k < 7; ++k) x128_add(s2[k], S.xred[w][10 + 2 * k], S.xred[w][11 + 2 * k], false);
            }
        }
    }
    if (T.wid == 0) {
        const int lane = T.lane;
        Exact128 mine, xa, xb;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const unsigned long long lo = __shfl_sync(0xffffffffu, s1[k].lo, 0), hi = __shfl_sync(0xffffffffu, s1[k].hi, 0);
            if (lane == k) { mine.lo = lo; mine.hi = hi; }
            const int ia = lane == 5 || lane == 8 || lane == 9 ? 0 : (lane == 6 || lane == 10 ? 1 : (lane == 7 ? 2 : 3));
            const int ib = lane == 5 ? 0 : (lane == 6 || lane == 8 ? 1 : (lane == 7 || lane == 9 || lane == 10 ? 2 : 3));
            if (ia == k) { xa.lo = lo; xa.hi = hi; }
            if (ib == k) { xb.lo = lo; xb.hi = hi; }
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const unsigned long long lo = __shfl_sync(0xffffffffu, s2[k].lo, 0), hi = __shfl_sync(0xffffffffu, s2[k].hi, 0);
            if (lane == 5 + k) { mine.lo = lo; mine.hi = hi; }
        }
        double val = 0.0;
        if (lane < 5) val = x128_to_double(mine) / n;
        else if (lane < 12) val = x128_central(mine, xa, xb, (unsigned)n);
        if (lane < 5) { a.emean[5 * e + lane] = val; S.mean[lane] = val; }
        else if (lane < 11) a.eR[6 * e + lane - 5] = val;
        else if (lane == 11) a.epsivar[e] = val;
        if (lane >= 5 && lane < 8) S.rd[lane - 5] = val;
        if (lane == 0) a.en[e] = n;
    }
    T.sync();
}

// compensated-FP32 moments in one pass over the segment, on data shifted by
// the segment's first particle (x - s, whose sums stay small when the mean is
// large against the spread): sums of the shifted values and of their
// products, then mean = s + S1/n and central moments S2/n - (S1/n)^2. With
// NT > 32 every warp sums its share (particle q goes to thread q mod NT) and
// warp 0 merges the warps' sums in warp order.
template <int NT, int NMAX>
__device__ __forceinline__ void kahan_moments(const MomArgs<float>& a, int e, int s0, int n, SelSmem<NMAX>& S) {
    const Team<NT> T;
    {
        const int lane = T.lane;
        const float su = a.u[s0], sv = a.v[s0], sw = a.w[s0], sp = a.psi[s0];
        // 16 compensated sums (12 used): 0..4 the shifted u v w psi and omega,
        // 5..10 the products uu vv ww uv uw vw, 11 psi psi. Blocked: a lane
        // sums blocks of up to SEL_BLOCK of its particles in plain FP32 (the
        // products fused), and only the block sums enter the compensated
        // sums; the rounding error stays below (SEL_BLOCK + 2) u sum |x|.
        AccK acc[16];
        constexpr int SEL_BLOCK = 8;
        for (int b0 = T.tid; b0 < n; b0 += NT * SEL_BLOCK) {
            float blk[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) blk[k] = 0.f;
            // two particles at a time: their ten loads are issued together,
            // then added in particle order
#pragma unroll
            for (int h = 0; h < SEL_BLOCK; h += 2) {
                float x[2][5];
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const int q = b0 + NT * (h + r);
                    const bool in = q < n;
                    x[r][0] = in ? a.u[s0 + q] : su;
                    x[r][1] = in ? a.v[s0 + q] : sv;
                    x[r][2] = in ? a.w[s0 + q] : sw;
                    x[r][3] = in ? a.psi[s0 + q] : sp;
                    x[r][4] = in ? a.om[s0 + q] : 0.f;
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {  // a missing particle adds zeros
                    const float du = x[r][0] - su, dv = x[r][1] - sv, dw = x[r][2] - sw, dp = x[r][3] - sp;
                    blk[0] += du; blk[1] += dv; blk[2] += dw; blk[3] += dp; blk[4] += x[r][4];
                    blk[5] = fmaf(du, du, blk[5]); blk[6] = fmaf(dv, dv, blk[6]); blk[7] = fmaf(dw, dw, blk[7]);
                    blk[8] = fmaf(du, dv, blk[8]); blk[9] = fmaf(du, dw, blk[9]); blk[10] = fmaf(dv, dw, blk[10]);
                    blk[11] = fmaf(dp, dp, blk[11]);
                }
            }
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k].add(blk[k]);
        }
        // butterfly reduce-scatter over the warp: after the xor-16, 8, 4, 2
        // exchanges (each lane merging the half it keeps with the partner's)
        // lane l holds sum (l >> 1) of its lane pair, the xor-1 merge completes it
#pragma unroll
        for (int w = 8, o = 16; w >= 1; w >>= 1, o >>= 1) {
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int k = 0; k < w; ++k) {
                AccK send = upper ? acc[k] : acc[w + k];
                AccK keep = upper ? acc[w + k] : acc[k];
                AccK recv;
                recv.s = __shfl_xor_sync(0xffffffffu, send.s, o);
                recv.c = __shfl_xor_sync(0xffffffffu, send.c, o);
                keep.merge(recv);
                acc[k] = keep;
            }
        }
        {
            AccK recv;
            recv.s = __shfl_xor_sync(0xffffffffu, acc[0].s, 1);
            recv.c = __shfl_xor_sync(0xffffffffu, acc[0].c, 1);
            if (lane & 1) {  // the same order of operands in both lanes of the pair
                AccK mine = recv;
                mine.merge(acc[0]);
                acc[0] = mine;
            } else {
                acc[0].merge(recv);
            }
        }
        if constexpr (NT > 32) {  // warp 0 merges the other warps' sums, in warp order
            if (lane < 24 && T.wid > 0) {
                S.kred[T.wid - 1][lane] = (lane & 1) ? acc[0].c : acc[0].s;
            }
            __syncthreads();
            if (T.wid == 0 && lane < 24) {
#pragma unroll 1
                for (int w = 0; w < NT / 32 - 1; ++w) {
                    AccK o;
                    o.s = S.kred[w][lane & ~1];
                    o.c = S.kred[w][lane | 1];
                    acc[0].merge(o);
                }
            }
        }
        if (T.wid == 0) {  // finalisation
            // sum v sits in lanes 2v and 2v + 1: lane q < 12 finishes moment q (FP64,
            // all lanes at once): lanes 0..4 the means, 5..10 the central second
            // moments uu vv ww uv uw vw, 11 the psi variance
            int ia = 0, ib = 0, ic = 0;  // first-moment sums used by this lane; ic: its second-moment sum
            if (lane < 5) ia = lane;
            else if (lane < 11) {
                const int k = lane - 5;  // uu vv ww uv uw vw
                ia = k < 3 ? k : (k == 5 ? 1 : 0);
                ib = k < 3 ? k : (k == 3 ? 1 : 2);
                ic = 5 + k;
            } else {
                ia = ib = 3;
                ic = 11;
            }
            AccK A, Bq, Cq;
            A.s = __shfl_sync(0xffffffffu, acc[0].s, 2 * ia);
            A.c = __shfl_sync(0xffffffffu, acc[0].c, 2 * ia);
            Bq.s = __shfl_sync(0xffffffffu, acc[0].s, 2 * ib);
            Bq.c = __shfl_sync(0xffffffffu, acc[0].c, 2 * ib);
            Cq.s = __shfl_sync(0xffffffffu, acc[0].s, 2 * ic);
            Cq.c = __shfl_sync(0xffffffffu, acc[0].c, 2 * ic);
            if (lane < 12) {
                const double inv_n = recip_n(n);
                const double da = A.value() * inv_n;
                double val;
                if (lane < 5) {
                    const float shift = lane == 0 ? su : (lane == 1 ? sv : (lane == 2 ? sw : (lane == 3 ? sp : 0.f)));
                    val = shift + da;
                    a.emean[5 * e + lane] = val;
                    S.mean[lane] = val;
                } else {
                    val = Cq.value() * inv_n - da * (Bq.value() * inv_n);
                    if (lane < 11) a.eR[6 * e + lane - 5] = val;
                    else a.epsivar[e] = val;
                    if (lane < 8) S.rd[lane - 5] = val;
                }
            }
            if (lane == 0) a.en[e] = n;
        }
    }
    T.sync();
}

// one element per team of NT threads (a warp: WPB elements per block; a block).
// Passes over the segment: moments; then per split level one pass that
// applies the previous level's boundaries, loads the level's component and
// fills its histogram, and one candidate pass; a last pass applies the last
// level and sums psi per bin.
// PART selects the work: SEL_MOMENTS, SEL_BINS or both. The bins alone take
// the element means and variances (bucket ranges, the mean psi of an element
// with fewer particles than bins) from a moments launch that ran before.
constexpr int SEL_MOMENTS = 1, SEL_BINS = 2, SEL_ALL = 3;
constexpr int SEL_RANGES_GIVEN = 4;  // with SEL_BINS: S.mean[0..2], S.rd[0..2] already hold the bucket ranges
template <bool KAHAN, int NT, int NMAX, int PART = SEL_ALL>
__device__ void sel_element(const MomArgs<float>& a, int e, int s0, int n, SelSmem<NMAX>& S) {
    const Team<NT> T;
    const int B = a.B;
    const uint32_t* __restrict__ ids = a.id + s0;
    if constexpr ((PART & SEL_MOMENTS) != 0) {
        if constexpr (KAHAN) kahan_moments<NT>(a, e, s0, n, S);
        else exact_moments<NT>(a, e, s0, n, S);
    } else if constexpr ((PART & SEL_RANGES_GIVEN) == 0) {
        if (T.tid < 5) S.mean[T.tid] = a.emean[5 * e + T.tid];
        else if (T.tid < 8) S.rd[T.tid - 5] = a.eR[6 * e + T.tid - 5];
        T.sync();
    }
    if constexpr ((PART & SEL_BINS) == 0) return;
    if (n < B) {
        for (int q = T.tid; q < n; q += NT) a.bin[s0 + q] = 0;
        for (int b = T.tid; b < B; b += NT) {
            a.ecm[(size_t)B * e + b] = S.mean[3];
            a.ecmT[(size_t)B * e + b] = (float)S.mean[3];
        }
        return;
    }
    int gsize[4] = {n, 0, 0, 0};
    const int G[3] = {a.G0, a.G1, a.G2};
    int ng = 0;  // groups of the previous level (0: none yet)
    for (int d = 0; d < 3; ++d) {
        if (G[d] == 1) continue;
        const float* comp = d == 0 ? a.u : (d == 1 ? a.v : a.w);
        const Buckets bk = make_buckets(S.mean[d], S.rd[d], SelCfg<NMAX>::NB);
        const int ngl = ng == 0 ? 1 : 2 * ng;  // groups of this level
        for (int q = T.tid; q < ngl * (SelCfg<NMAX>::NB / 2); q += NT) (&S.hist[0][0])[q] = 0u;
        T.sync();
        // four keys per thread at a time: their component loads are issued
        // together (they come from L2), then the keys are assigned
        for (int q0 = T.tid; q0 < n; q0 += 4 * NT) {
            float c4[4];
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int q = q0 + r * NT;
                c4[r] = q < n ? comp[s0 + q] : 0.f;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int q = q0 + r * NT;
                if (q >= n) break;
                int g = 0;
                if (ng) {
                    const int gp = S.grp[q];
                    const uint32_t v = S.kv[q], bv = S.bv[gp];
                    g = 2 * gp + ((v < bv || (v == bv && ids[q] <= S.bid[gp])) ? 0 : 1);
                }
                S.grp[q] = (unsigned char)g;
                const uint32_t k = ord32(c4[r]);
                S.kv[q] = k;
                const int b = bk(k);
                S.bk8[q] = (unsigned char)b;
                atomicAdd(&S.hist[g][b >> 1], 1u << (16 * (b & 1)));
            }
        }
        if (ng) {  // sizes of the new groups: the lower half takes the extra key
            int ns[4] = {0, 0, 0, 0};
            for (int g = 0; g < ng; ++g) {
                ns[2 * g] = (gsize[g] + 1) / 2;
                ns[2 * g + 1] = gsize[g] - ns[2 * g];
            }
            for (int g = 0; g < 4; ++g) gsize[g] = ns[g];
        }
        ng = ngl;
        T.sync();
        sel_boundaries<NT>(S, ids, n, ng, gsize, bk);
    }
    // bins, and <phi|V> per bin: exact fixed-point sums of psi
    constexpr int UNIT = NMAX <= 512 ? 54 : 51;  // psi <= 1 and n <= NMAX keep the sums below 2^63
    if (T.tid < 8) { S.binsum[T.tid] = 0ull; S.bincnt[T.tid] = 0; }
    T.sync();
    for (int q0 = T.tid; q0 < n; q0 += 4 * NT) {
      float p4[4];  // the psi loads of four keys issued together
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int q = q0 + r * NT;
        p4[r] = q < n ? a.psi[s0 + q] : 0.f;
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int q = q0 + r * NT;
        if (q >= n) break;
        int bn = 0;
        if (ng) {
            const int gp = S.grp[q];
            const uint32_t v = S.kv[q], bv = S.bv[gp];
            bn = 2 * gp + ((v < bv || (v == bv && ids[q] <= S.bid[gp])) ? 0 : 1);
        }
        a.bin[s0 + q] = (unsigned char)bn;
        unsigned m;
        int ex;
        bool negp;
        f32_parts(fminf(fmaxf(p4[r], 0.f), 1.f), m, ex, negp);
        const int sh = ex - 150 + UNIT;  // m 2^(ex-150) = m 2^(ex-150+UNIT) 2^-UNIT
        const unsigned long long v = sh >= 0 ? ((unsigned long long)m << sh)
                                             : (-sh < 64 ? ((unsigned long long)m >> (-sh)) : 0ull);
        atomicAdd(&S.binsum[bn], v);
        atomicAdd(&S.bincnt[bn], 1);
      }
    }
    T.sync();
    for (int b = T.tid; b < B; b += NT) {
        const double cm = __ull2double_rn(S.binsum[b]) * (1.0 / (double)(1ull << UNIT)) * recip_n(S.bincnt[b]);
        a.ecm[(size_t)B * e + b] = cm;
        a.ecmT[(size_t)B * e + b] = (float)cm;
    }
}

__device__ void empty_moments(const MomArgs<float>& a, int e, int tid) {
    if (tid == 0) {
        a.en[e] = 0;
        for (int q = 0; q < 5; ++q) a.emean[5 * e + q] = 0.0;
        for (int q = 0; q < 6; ++q) a.eR[6 * e + q] = 0.0;
        a.epsivar[e] = 0.0;
    }
}

// ---------------------------------------------------------------------------
// 2 x 2 x 2 bins (median splits on U, then V in each U half, then W in each
// quarter), one warp per element of at most 512 particles. Lane l holds the
// keys q = l + 32 j: j < MRK in registers (u, v, w, psi, each loaded one level
// ahead of its use, so that at most two are live), MRK <= j < 16 in the warp's
// shared memory; the segment is read from memory once.
//  * moments: blocked compensated FP32 sums (KAHAN) or exact fixed-point
//    sums;
//  * every split level fills 256-bucket histograms of its component (value-
//    linear over mean +- 4 sd of the element); a scan of each group's
//    histogram gives the bucket holding the group's median and the median's
//    rank in it. In the next pass a key outside that bucket joins the lower
//    or the upper half by its bucket alone; the few keys inside it are
//    deferred to a candidate list, ranked exactly in the (value, id) order,
//    and join the next level's histograms once their half is known. Each
//    level costs one pass over the keys;
//  * the last pass writes the bins and sums psi per bin (exact fixed point);
//  * a level whose boundary buckets hold more than MCL keys (many equal or
//    clustered values) hands the element to the general selection path.
// ---------------------------------------------------------------------------
constexpr int MCL = 128;  // candidate list capacity
constexpr int MRK = 9;    // register key slots per lane: elements of up to 288 particles stay in registers
constexpr unsigned FULLW = 0xffffffffu;

struct __align__(16) MedSmem {
    unsigned hist[4][128];                       // per group: 256 buckets, two 16-bit counts per word (read as uint4)
    float ou[16 - MRK][32], ov[16 - MRK][32], ow[16 - MRK][32], op[16 - MRK][32];  // keys j >= MRK, slot j - MRK
    unsigned char ob[16 - MRK][32];              // their bucket at the current level
    uint32_t cv[MCL];                            // candidate: order bits of the resolved component
    uint32_t cid[MCL];                           // candidate: particle id (read where values tie)
    float cps[MCL];                              // candidate: psi (last level)
    unsigned short cq[MCL];                      // candidate: index in the segment
    unsigned short crank[MCL];                   // candidate: rank in its group's boundary bucket
    unsigned char cg[MCL], cb[MCL], ceq[MCL];    // group, next-level bucket, keys of equal value
    unsigned upb[16];                            // upper-half bit of every deferred key, by index
    int bkt[4], brank[4], ncand[4];
    int ncl;                                     // candidates listed at this level
    unsigned binpart[8][4];                      // sum of psi per bin, unit 2^-54, in 19-bit parts
};
static_assert(sizeof(MedSmem) % 16 == 0 && alignof(MedSmem) == 16, "per-warp slices keep hist 16-byte aligned");

__device__ __forceinline__ int bucket_of(const Buckets& bk, float x) {
    return max(0, min(bk.top, (int)((x + 0.0f - bk.lo) * bk.sc)));
}

// size of group g after `depth` halvings of n keys (the lower half takes the extra key)
__device__ __forceinline__ int split_size(int n, int g, int depth) {
    int m = n;
    for (int b = depth - 1; b >= 0; --b) m = ((g >> b) & 1) ? (m >> 1) : ((m + 1) >> 1);
    return m;
}

// byte j of the register keys' packed buckets (j a compile-time index after unrolling)
__device__ __forceinline__ int getbyte(const unsigned (&pb)[(MRK + 3) / 4], int j) {
    return (int)((pb[j >> 2] >> (8 * (j & 3))) & 0xffu);
}
__device__ __forceinline__ void setbyte(unsigned (&pb)[(MRK + 3) / 4], int j, int b) {
    unsigned& w = pb[j >> 2];
    w = (w & ~(0xffu << (8 * (j & 3)))) | ((unsigned)b << (8 * (j & 3)));
}

// register key j of x for a run-time j (a select chain: the array stays in registers)
__device__ __forceinline__ float pick(const float (&x)[MRK], int j) {
    float r = x[0];
#pragma unroll
    for (int k = 1; k < MRK; ++k) r = j == k ? x[k] : r;
    return r;
}
__device__ __forceinline__ int getbyte_rt(const unsigned (&pb)[(MRK + 3) / 4], int j) {
    unsigned w = pb[0];
#pragma unroll
    for (int k = 1; k < (MRK + 3) / 4; ++k) w = (j >> 2) == k ? pb[k] : w;
    return (int)((w >> (8 * (j & 3))) & 0xffu);
}

__device__ __forceinline__ unsigned hinc(int b) { return 1u << (16 * (b & 1)); }

// both bits of the 2-bit group field of every key flagged in m (register keys j < MRK)
__device__ __forceinline__ uint32_t med_spread(uint32_t m) {
    uint32_t r = 0u;
#pragma unroll
    for (int j = 0; j < MRK; ++j) r |= ((m >> j) & 1u) * (3u << (2 * j));
    return r;
}

// psi (clamped to [0, 1]) added to bin bn's sum: the fixed-point value
// (below 2^55) in three 19-bit parts, each part's sum over at most 512 keys
// below 2^28, so native 32-bit shared atomics keep the sum exact
__device__ __forceinline__ void med_binadd(MedSmem& S, int bn, unsigned long long v) {
    atomicAdd(&S.binpart[bn][0], (unsigned)(v & 0x7ffffull));
    atomicAdd(&S.binpart[bn][1], (unsigned)((v >> 19) & 0x7ffffull));
    atomicAdd(&S.binpart[bn][2], (unsigned)(v >> 38));
}

// psi (clamped to [0, 1]) in fixed point, unit 2^-54, truncated: the scaling
// by 2^54 is exact in FP32 (no overflow; subnormal inputs become normal) and
// the conversion truncates toward zero, as a right shift of the mantissa would
__device__ __forceinline__ unsigned long long psi_fixed(float p) {
    constexpr float SCALE = 18014398509481984.0f;  // 2^54: psi in [0, 1] and n <= 512 keep the bin sums below 2^63
    return __float2ull_rz(fminf(fmaxf(p, 0.f), 1.f) * SCALE);
}

// bucket of each group's median: NG groups, 32/NG lanes scan one group's
// histogram; writes bkt, brank (rank of the median in its bucket) and ncand
template <int NG>
__device__ __forceinline__ void med_scan(MedSmem& S, int n, int lane) {
    constexpr int LPG = 32 / NG, WPL = 128 / LPG, DEP = NG == 1 ? 0 : (NG == 2 ? 1 : 2);
    const int sub = lane & (LPG - 1), gl = lane / LPG;
    const int Tk = (split_size(n, gl, DEP) + 1) >> 1;
    const uint4* h4 = reinterpret_cast<const uint4*>(&S.hist[gl][sub * WPL]);
    unsigned hw[WPL];
#pragma unroll
    for (int k = 0; k < WPL / 4; ++k) {
        const uint4 x = h4[k];
        hw[4 * k] = x.x; hw[4 * k + 1] = x.y; hw[4 * k + 2] = x.z; hw[4 * k + 3] = x.w;
    }
    int tot = 0;
#pragma unroll
    for (int k = 0; k < WPL; ++k) tot += (int)(hw[k] & 0xffffu) + (int)(hw[k] >> 16);
    int incl = tot;
#pragma unroll
    for (int o = 1; o < LPG; o <<= 1) {
        const int y = __shfl_up_sync(FULLW, incl, o, LPG);
        if (sub >= o) incl += y;
    }
    const int excl = incl - tot;
    if (excl < Tk && incl >= Tk) {  // this lane's words hold the median: find the word, then the bucket
        int run = excl, k = 0;
        unsigned word = 0u;
        bool found = false;
#pragma unroll
        for (int i = 0; i < WPL; ++i) {
            const int c = (int)(hw[i] & 0xffffu) + (int)(hw[i] >> 16);
            if (!found) {
                if (run + c >= Tk) {
                    k = i;
                    word = hw[i];
                    found = true;
                } else {
                    run += c;
                }
            }
        }
        const int c0 = (int)(word & 0xffffu), c1 = (int)(word >> 16);
        const bool hi = run + c0 < Tk;
        S.bkt[gl] = 2 * (sub * WPL + k) + (hi ? 1 : 0);
        S.brank[gl] = Tk - (hi ? run + c0 : run) - 1;
        S.ncand[gl] = hi ? c1 : c0;
    }
}

// rank of every listed candidate in its group's boundary bucket, in the
// (value, id) order; ids are read only where two candidates of a group tie
__device__ __noinline__ void med_rank(MedSmem& S, const uint32_t* __restrict__ ids, int L, int lane) {
    int tied = 0;
    for (int t = lane; t < L; t += 32) {
        const uint32_t v = S.cv[t];
        const int g = S.cg[t];
        int r = 0, eq = 0;
        for (int u = 0; u < L; ++u) {
            if (S.cg[u] == g) {
                const uint32_t vu = S.cv[u];
                r += vu < v ? 1 : 0;
                eq += vu == v ? 1 : 0;
            }
        }
        S.crank[t] = (unsigned short)r;
        S.ceq[t] = (unsigned char)min(eq, 255);
        tied |= eq > 1 ? 1 : 0;
    }
    if (__any_sync(FULLW, tied)) {  // equal values: the ids decide (rare)
        __syncwarp();
        for (int t = lane; t < L; t += 32) S.cid[t] = ids[S.cq[t]];
        __syncwarp();
        for (int t = lane; t < L; t += 32) {
            if (S.ceq[t] > 1) {
                const uint32_t v = S.cv[t], it = S.cid[t];
                const int g = S.cg[t];
                int r = S.crank[t];
                for (int u = 0; u < L; ++u) r += (S.cg[u] == g && S.cv[u] == v && S.cid[u] < it) ? 1 : 0;
                S.crank[t] = (unsigned short)r;
            }
        }
    }
    __syncwarp();
}

// moments of the segment of at most 512 particles, read from memory in
// blocks of eight keys per lane (key q = lane + 32 j); lanes 0..11 write the
// means, the central second moments and the psi variance, lane 0 the count
template <bool KAHAN>
__device__ __forceinline__ void warp_moments(const MomArgs<float>& a, int e, int s0, int n, int lane) {
    const int kk = (n + 31) >> 5;
    double val = 0.0;
    if constexpr (KAHAN) {
        // sums of the values shifted by the segment's first particle and of
        // their products: a lane sums each block of eight of its keys in plain
        // FP32 (the products fused), the block sums enter compensated sums,
        // then a butterfly reduce-scatter merges the lanes
        const float su = a.u[s0], sv = a.v[s0], sw = a.w[s0], sp = a.psi[s0];
        AccK acc[16];
#pragma unroll
        for (int blkno = 0; blkno < 2; ++blkno) {
            if (blkno == 1 && kk <= 8) break;
            float tu[8], tv[8], tw[8], tp[8], to[8];
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int j = 8 * blkno + h, q = lane + 32 * j;
                const bool in = j < kk && q < n;
                tu[h] = in ? a.u[s0 + q] : su;
                tv[h] = in ? a.v[s0 + q] : sv;
                tw[h] = in ? a.w[s0 + q] : sw;
                tp[h] = in ? a.psi[s0 + q] : sp;
                to[h] = in ? a.om[s0 + q] : 0.f;
            }
            float blk[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) blk[k] = 0.f;
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int j = 8 * blkno + h, q = lane + 32 * j;
                const bool in = j < kk && q < n;
                const float du = in ? tu[h] - su : 0.f, dv = in ? tv[h] - sv : 0.f;
                const float dw = in ? tw[h] - sw : 0.f, dp = in ? tp[h] - sp : 0.f;
                blk[0] += du; blk[1] += dv; blk[2] += dw; blk[3] += dp; blk[4] += to[h];
                blk[5] = fmaf(du, du, blk[5]); blk[6] = fmaf(dv, dv, blk[6]); blk[7] = fmaf(dw, dw, blk[7]);
                blk[8] = fmaf(du, dv, blk[8]); blk[9] = fmaf(du, dw, blk[9]); blk[10] = fmaf(dv, dw, blk[10]);
                blk[11] = fmaf(dp, dp, blk[11]);
            }
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k].add(blk[k]);
        }
        // after the xor-16, 8, 4, 2 exchanges lane l holds sum (l >> 1) of
        // its lane pair; the xor-1 merge (same operand order in both lanes)
        // completes it
#pragma unroll
        for (int w = 8, o = 16; w >= 1; w >>= 1, o >>= 1) {
            const bool upper = (lane & o) != 0;
#pragma unroll
            for (int k = 0; k < w; ++k) {
                AccK send = upper ? acc[k] : acc[w + k];
                AccK keep = upper ? acc[w + k] : acc[k];
                AccK recv;
                recv.s = __shfl_xor_sync(FULLW, send.s, o);
                recv.c = __shfl_xor_sync(FULLW, send.c, o);
                keep.merge(recv);
                acc[k] = keep;
            }
        }
        {
            AccK recv;
            recv.s = __shfl_xor_sync(FULLW, acc[0].s, 1);
            recv.c = __shfl_xor_sync(FULLW, acc[0].c, 1);
            if (lane & 1) {
                AccK mine = recv;
                mine.merge(acc[0]);
                acc[0] = mine;
            } else {
                acc[0].merge(recv);
            }
        }
        // lane q < 12 finishes moment q: 0..4 the means, 5..10 the central
        // second moments uu vv ww uv uw vw, 11 the psi variance (sum v sits
        // in lanes 2v and 2v + 1)
        int ia = 0, ib = 0, ic = 0;
        if (lane < 5) ia = lane;
        else if (lane < 11) {
            const int k = lane - 5;
            ia = k < 3 ? k : (k == 5 ? 1 : 0);
            ib = k < 3 ? k : (k == 3 ? 1 : 2);
            ic = 5 + k;
        } else {
            ia = ib = 3;
            ic = 11;
        }
        AccK A, Bq, Cq;
        A.s = __shfl_sync(FULLW, acc[0].s, 2 * ia);
        A.c = __shfl_sync(FULLW, acc[0].c, 2 * ia);
        Bq.s = __shfl_sync(FULLW, acc[0].s, 2 * ib);
        Bq.c = __shfl_sync(FULLW, acc[0].c, 2 * ib);
        Cq.s = __shfl_sync(FULLW, acc[0].s, 2 * ic);
        Cq.c = __shfl_sync(FULLW, acc[0].c, 2 * ic);
        if (lane < 12) {
            const double inv_n = recip_n(n);
            const double da = A.value() * inv_n;
            if (lane < 5) {
                const float shift = lane == 0 ? su : (lane == 1 ? sv : (lane == 2 ? sw : (lane == 3 ? sp : 0.f)));
                val = shift + da;
            } else {
                val = Cq.value() * inv_n - da * (Bq.value() * inv_n);
            }
        }
    } else {
        // exact fixed-point sums (unit 2^-80) of the values and their products
        Exact128 s1[5], s2[7];
        bool big = false;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const int q = lane + 32 * j;
            if (j < kk && q < n) {
                const float x0 = a.u[s0 + q], x1 = a.v[s0 + q], x2 = a.w[s0 + q], x3 = a.psi[s0 + q];
                unsigned mu_, mv_, mw_, mp_, mo_;
                int eu, ev, ew, ep, eo;
                bool nu, nv, nw, np, no;
                f32_parts(x0, mu_, eu, nu);
                f32_parts(x1, mv_, ev, nv);
                f32_parts(x2, mw_, ew, nw);
                f32_parts(x3, mp_, ep, np);
                f32_parts(a.om[s0 + q], mo_, eo, no);
                big |= max(max(max(eu, ev), max(ew, ep)), eo) > 145;  // |x| >= 2^19: outside the format
                x128_add_parts(s1[0], mu_, eu, nu);
                x128_add_parts(s1[1], mv_, ev, nv);
                x128_add_parts(s1[2], mw_, ew, nw);
                x128_add_parts(s1[3], mp_, ep, np);
                x128_add_parts(s1[4], mo_, eo, no);
                x128_add_prod(s2[0], mu_, eu, nu, mu_, eu, nu);
                x128_add_prod(s2[1], mv_, ev, nv, mv_, ev, nv);
                x128_add_prod(s2[2], mw_, ew, nw, mw_, ew, nw);
                x128_add_prod(s2[3], mu_, eu, nu, mv_, ev, nv);
                x128_add_prod(s2[4], mu_, eu, nu, mw_, ew, nw);
                x128_add_prod(s2[5], mv_, ev, nv, mw_, ew, nw);
                x128_add_prod(s2[6], mp_, ep, np, mp_, ep, np);
            }
        }
        if (__any_sync(FULLW, big) && lane == 0) set_status(a.status, ST_CAPACITY);
#pragma unroll
        for (int k = 0; k < 5; ++k) x128_warp_sum(s1[k]);
#pragma unroll
        for (int k = 0; k < 7; ++k) x128_warp_sum(s2[k]);
        Exact128 mine, xa, xb;
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const unsigned long long lo = __shfl_sync(FULLW, s1[k].lo, 0), hi = __shfl_sync(FULLW, s1[k].hi, 0);
            if (lane == k) { mine.lo = lo; mine.hi = hi; }
            const int ia = lane == 5 || lane == 8 || lane == 9 ? 0 : (lane == 6 || lane == 10 ? 1 : (lane == 7 ? 2 : 3));
            const int ib = lane == 5 ? 0 : (lane == 6 || lane == 8 ? 1 : (lane == 7 || lane == 9 || lane == 10 ? 2 : 3));
            if (ia == k) { xa.lo = lo; xa.hi = hi; }
            if (ib == k) { xb.lo = lo; xb.hi = hi; }
        }
#pragma unroll
        for (int k = 0; k < 7; ++k) {
            const unsigned long long lo = __shfl_sync(FULLW, s2[k].lo, 0), hi = __shfl_sync(FULLW, s2[k].hi, 0);
            if (lane == 5 + k) { mine.lo = lo; mine.hi = hi; }
        }
        if (lane < 5) val = x128_to_double(mine) / n;
        else if (lane < 12) val = x128_central(mine, xa, xb, (unsigned)n);
    }
    if (lane < 5) a.emean[5 * e + lane] = val;
    else if (lane < 11) a.eR[6 * e + lane - 5] = val;
    else if (lane == 11) a.epsivar[e] = val;
    if (lane == 0) a.en[e] = n;
}

// the bucket map of one split level from the element's value range
// [lo, hi] (256 equal buckets; any monotone map keeps the selection exact)
__device__ __forceinline__ Buckets range_buckets(float lo, float hi) {
    Buckets b;
    b.top = 255;
    b.lo = lo;
    const float w = hi - lo;
    const float sc = w > 0.f ? 256.f / w : 0.f;
    b.sc = (sc > 0.f && sc < 1e30f) ? sc : 0.f;
    return b;
}

__device__ __forceinline__ float warp_min(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}
__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
    return x;
}

// append a key to the candidate list (a few keys per level; S.ncl counts them)
__device__ __forceinline__ void med_append(MedSmem& S, uint32_t key, int q, int g, int b, float ps) {
    const int slot = atomicAdd(&S.ncl, 1);
    if (slot < MCL) {
        S.cv[slot] = key;
        S.cq[slot] = (unsigned short)q;
        S.cg[slot] = (unsigned char)g;
        S.cb[slot] = (unsigned char)b;
        S.cps[slot] = ps;
    }
}

// the general selection path for an element whose boundary buckets are
// crowded (bins only: the moments are in memory)
__device__ __noinline__ void med_general(const MomArgs<float>& a, int e, int s0, int n, SelSmem<512>& S) {
    // the element's value ranges [lo, hi] (read again: the register passes
    // may not have reached every component), written as mean +- 4 sd, the
    // form sel_element reads
    const int lane = threadIdx.x % 32;
    const float* __restrict__ x[3] = {a.u + s0, a.v + s0, a.w + s0};
    for (int d = 0; d < 3; ++d) {
        float lo = 3.4e38f, hi = -3.4e38f;
        for (int q = lane; q < n; q += 32) {
            lo = fminf(lo, x[d][q]);
            hi = fmaxf(hi, x[d][q]);
        }
        lo = warp_min(lo);
        hi = warp_max(hi);
        if (lane == 0) {
            const double sd = ((double)hi - (double)lo) * 0.125;
            S.mean[d] = 0.5 * ((double)hi + (double)lo);
            S.rd[d] = sd * sd;
        }
    }
    __syncwarp();
    sel_element<true, 32, 512, SEL_BINS | SEL_RANGES_GIVEN>(a, e, s0, n, S);
}

// buckets over the element's value range of one component: register keys
// x[j < MRK] (slots 8.. only when rx) and the shared-memory keys xs[j - MRK]
__device__ __forceinline__ Buckets med_range(const float (&x)[MRK], const float (*xs)[32], bool rx, int kk, int n,
                                             int lane) {
    float lo = 3.4e38f, hi = -3.4e38f;
#pragma unroll
    for (int j = 0; j < MRK; ++j) {
        if (j >= 8 && !rx) break;
        if (j < kk && lane + 32 * j < n) {
            lo = fminf(lo, x[j]);
            hi = fmaxf(hi, x[j]);
        }
    }
    for (int j = MRK; j < kk; ++j) {
        if (lane + 32 * j < n) {
            lo = fminf(lo, xs[j - MRK][lane]);
            hi = fmaxf(hi, xs[j - MRK][lane]);
        }
    }
    return range_buckets(warp_min(lo), warp_max(hi));
}

__device__ __forceinline__ int upbit(const MedSmem& S, int q) { return (int)((S.upb[q >> 5] >> (q & 31)) & 1u); }

// The passes over the keys j >= MRK (shared memory, slot j - MRK), out of line:
// only elements above 32 MRK particles take them, and the register passes stay
// contiguous.
__device__ __noinline__ void med_tail0(MedSmem& S, Buckets bk, int n, int kk, int lane) {
    for (int j = MRK; j < kk; ++j) {
        if (lane + 32 * j < n) {
            const int b = bucket_of(bk, S.ou[j - MRK][lane]);
            S.ob[j - MRK][lane] = (unsigned char)b;
            atomicAdd(&S.hist[0][b >> 1], hinc(b));
        }
    }
}

__device__ __noinline__ uint2 med_tail1(MedSmem& S, Buckets bk, int c0, int n, int kk, int lane, uint32_t gw,
                                        uint32_t pend) {
    for (int j = MRK; j < kk; ++j) {
        const int q = lane + 32 * j;
        if (q < n) {
            const int b0 = S.ob[j - MRK][lane];
            const int b = bucket_of(bk, S.ov[j - MRK][lane]);
            S.ob[j - MRK][lane] = (unsigned char)b;
            if (b0 == c0) {
                pend |= 1u << j;
                med_append(S, ord32(S.ou[j - MRK][lane]), q, 0, b, 0.f);
            } else {
                const int g = b0 > c0 ? 1 : 0;
                gw |= (uint32_t)g << (2 * j);
                atomicAdd(&S.hist[g][b >> 1], hinc(b));
            }
        }
    }
    return make_uint2(gw, pend);
}

__device__ __noinline__ uint2 med_tail2(MedSmem& S, Buckets bk, int c0, int c1, int n, int kk, int lane, uint32_t gw,
                                        uint32_t pend, uint32_t pend2) {
    for (int j = MRK; j < kk; ++j) {
        const int q = lane + 32 * j;
        if (q < n) {
            int g = (int)((gw >> (2 * j)) & 3u);
            if ((pend >> j) & 1u) g = 2 * g + upbit(S, q);
            const int b1 = S.ob[j - MRK][lane], c = g ? c1 : c0;
            const int b = bucket_of(bk, S.ow[j - MRK][lane]);
            S.ob[j - MRK][lane] = (unsigned char)b;
            if (b1 == c) {
                pend2 |= 1u << j;
                gw = (gw & ~(3u << (2 * j))) | ((uint32_t)g << (2 * j));
                med_append(S, ord32(S.ov[j - MRK][lane]), q, g, b, 0.f);
            } else {
                const int g2 = 2 * g + (b1 > c ? 1 : 0);
                gw = (gw & ~(3u << (2 * j))) | ((uint32_t)g2 << (2 * j));
                atomicAdd(&S.hist[g2][b >> 1], hinc(b));
            }
        }
    }
    return make_uint2(gw, pend2);
}

__device__ __noinline__ void med_tail3(MedSmem& S, unsigned char* bins, int4 c4, int n, int kk, int lane, uint32_t gw,
                                       uint32_t pend) {
    for (int j = MRK; j < kk; ++j) {
        const int q = lane + 32 * j;
        if (q < n) {
            int g = (int)((gw >> (2 * j)) & 3u);
            if ((pend >> j) & 1u) g = 2 * g + upbit(S, q);
            const int b2 = S.ob[j - MRK][lane], c = g == 0 ? c4.x : (g == 1 ? c4.y : (g == 2 ? c4.z : c4.w));
            const float ps = S.op[j - MRK][lane];
            if (b2 == c) {
                med_append(S, ord32(S.ow[j - MRK][lane]), q, g, 0, ps);
            } else {
                const int bn = 2 * g + (b2 > c ? 1 : 0);
                bins[q] = (unsigned char)bn;
                med_binadd(S, bn, psi_fixed(ps));
            }
        }
    }
}

// moments of the elements of at most 512 particles, one warp per element
template <bool KAHAN>
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK) k_moments_w(const MomArgs<float> a, int nt) {
    const int lane = threadIdx.x & 31;
    const int e = blockIdx.x * WARPS_PER_BLOCK + (threadIdx.x >> 5);
    if (e >= nt) return;
    const int s0 = a.off[e], n = a.off[e + 1] - s0;
    if (n > 512) return;  // a block kernel takes it (listed by k_crowded)
    if (n == 0) {
        empty_moments(a, e, lane);
        return;
    }
    warp_moments<KAHAN>(a, e, s0, n, lane);
}

// the bins of element e (at most 512 particles: larger ones are left to the
// crowded-element kernels) by the warp
union __align__(16) MedUnion {
    MedSmem m;
    SelSmem<512> s;
};
static_assert(sizeof(MedUnion) % 16 == 0, "per-warp slices keep hist 16-byte aligned");

__device__ __forceinline__ void med_bins_element(const MomArgs<float>& a, int e, int lane, MedUnion& U) {
    const int s0 = a.off[e], n = a.off[e + 1] - s0;
    if (n > 512) return;  // a block kernel takes it (listed by k_crowded)
    if (n < 8) {  // no particles: <phi|V> = 0; fewer particles than bins: the element mean psi (IEM)
        double p = lane < n ? (double)a.psi[s0 + lane] : 0.0;
#pragma unroll
        for (int o = 4; o > 0; o >>= 1) p += __shfl_xor_sync(FULLW, p, o);  // lanes 0..7, a fixed order
        const double mean_psi = n == 0 ? 0.0 : p / n;
        if (lane < n) a.bin[s0 + lane] = 0;
        if (lane < 8) {
            a.ecm[(size_t)8 * e + lane] = mean_psi;
            a.ecmT[(size_t)8 * e + lane] = (float)mean_psi;
        }
        return;
    }
    MedSmem& S = U.m;
    const uint32_t* __restrict__ ids = a.id + s0;
    const int kk = (n + 31) >> 5;  // key slots in use (warp-uniform)
    float xu[MRK] = {}, xv[MRK] = {}, xw[MRK] = {}, xp[MRK] = {};
    const bool rx = kk > 8;  // the register slots 8.. are in use (warp-uniform: smaller elements skip them)
    // the register keys' components are loaded one level ahead of their use
    // (v during the first scan, w once u is spent, psi once v is spent), so
    // at most two of them are live at a time
#pragma unroll
    for (int j = 0; j < MRK; ++j) {
        if (j >= 8 && !rx) break;
        const int q = lane + 32 * j;
        xu[j] = j < kk && q < n ? a.u[s0 + q] : 0.f;
    }
    if (kk > MRK) {  // keys 32 MRK..511 into the warp's shared memory (all loads issued together)
        float tu[16 - MRK], tv[16 - MRK], tw[16 - MRK], tp[16 - MRK];
#pragma unroll
        for (int h = 0; h < 16 - MRK; ++h) {
            const int q = lane + 32 * (MRK + h);
            const bool in = MRK + h < kk && q < n;
            tu[h] = in ? a.u[s0 + q] : 0.f;
            tv[h] = in ? a.v[s0 + q] : 0.f;
            tw[h] = in ? a.w[s0 + q] : 0.f;
            tp[h] = in ? a.psi[s0 + q] : 0.f;
        }
#pragma unroll
        for (int h = 0; h < 16 - MRK; ++h) {
            S.ou[h][lane] = tu[h]; S.ov[h][lane] = tv[h]; S.ow[h][lane] = tw[h]; S.op[h][lane] = tp[h];
        }
    }
    // the bucket ranges: the element's own minimum and maximum of each
    // component (the bins need no moments, so they run beside the moments
    // kernel), taken when the component's level starts
    Buckets bk = med_range(xu, S.ou, rx, kk, n, lane);
    unsigned pb[(MRK + 3) / 4] = {};  // bucket of register key j at the current level (a byte each)
    // The passes over the register keys are branch-free (the key slot and the
    // segment bound predicate the stores and atomics), so the keys of a lane
    // interleave; keys deferred to the candidate list are flagged in a mask
    // and listed after the pass.
    // ---- level 0: U
    for (int t = lane; t < 128; t += 32) S.hist[0][t] = 0u;
    __syncwarp();
#pragma unroll
    for (int j = 0; j < MRK; ++j) {
        if (j >= 8 && !rx) break;
        const bool in = j < kk && lane + 32 * j < n;
        const int b = bucket_of(bk, xu[j]);
        setbyte(pb, j, b);
        if (in) atomicAdd(&S.hist[0][b >> 1], hinc(b));
    }
    if (kk > MRK) med_tail0(S, bk, n, kk, lane);
#pragma unroll
    for (int j = 0; j < MRK; ++j) {  // v of the register keys, in flight during the scan
        if (j >= 8 && !rx) break;
        const int q = lane + 32 * j;
        xv[j] = j < kk && q < n ? a.v[s0 + q] : 0.f;
    }
    __syncwarp();
    med_scan<1>(S, n, lane);
    __syncwarp();
    bool general = S.ncand[0] > MCL;
    uint32_t gw = 0u, pend = 0u;  // group of key j (2 bits each); keys deferred to the candidate list
    if (!general) {
        // ---- level 1: V; the U halves
        const int c0 = S.bkt[0];
        for (int t = lane; t < 256; t += 32) (&S.hist[0][0])[t] = 0u;
        if (lane < 16) S.upb[lane] = 0u;
        if (lane == 0) S.ncl = 0;
        bk = med_range(xv, S.ov, rx, kk, n, lane);
        __syncwarp();
#pragma unroll
        for (int j = 0; j < MRK; ++j) {
            if (j >= 8 && !rx) break;
            const bool in = j < kk && lane + 32 * j < n;
            const int b0 = getbyte(pb, j);
            const int b = bucket_of(bk, xv[j]);
            setbyte(pb, j, b);
            const int g = b0 > c0 ? 1 : 0;
            gw |= (uint32_t)g << (2 * j);
            const bool isc = in && b0 == c0;
            pend |= (isc ? 1u : 0u) << j;
            if (in && !isc) atomicAdd(&S.hist[g][b >> 1], hinc(b));
        }
        // the deferred register keys, lane by lane (a few per warp)
        for (uint32_t p = pend; p; p &= p - 1u) {
            const int j = __ffs(p) - 1;
            med_append(S, ord32(pick(xu, j)), lane + 32 * j, 0, getbyte_rt(pb, j), 0.f);
        }
#pragma unroll
        for (int j = 0; j < MRK; ++j) {  // u is spent: w of the register keys
            if (j >= 8 && !rx) break;
            const int q = lane + 32 * j;
            xw[j] = j < kk && q < n ? a.w[s0 + q] : 0.f;
        }
        gw &= ~med_spread(pend);  // deferred keys stay in group 0 until resolved
        if (kk > MRK) {
            const uint2 r = med_tail1(S, bk, c0, n, kk, lane, gw, pend);
            gw = r.x;
            pend = r.y;
        }
        __syncwarp();
        const int L = S.ncl;
        med_rank(S, ids, L, lane);
        for (int t = lane; t < L; t += 32) {  // the candidates join their U half
            const int g = S.cg[t], up = (int)S.crank[t] > S.brank[g] ? 1 : 0, b = S.cb[t];
            atomicAdd(&S.hist[2 * g + up][b >> 1], hinc(b));
            if (up) atomicOr(&S.upb[S.cq[t] >> 5], 1u << (S.cq[t] & 31));
        }
        __syncwarp();
        med_scan<2>(S, n, lane);
        __syncwarp();
        general = S.ncand[0] + S.ncand[1] > MCL;
    }
    if (!general) {
        // ---- level 2: W; the V halves of each U half
        const int c0 = S.bkt[0], c1 = S.bkt[1];
        for (int t = lane; t < 512; t += 32) (&S.hist[0][0])[t] = 0u;
        if (lane == 0) S.ncl = 0;
        bk = med_range(xw, S.ow, rx, kk, n, lane);
        __syncwarp();
        uint32_t pend2 = 0u;
#pragma unroll
        for (int j = 0; j < MRK; ++j) {
            if (j >= 8 && !rx) break;
            const bool in = j < kk && lane + 32 * j < n;
            int g = (int)((gw >> (2 * j)) & 3u);
            g = ((pend >> j) & 1u) ? 2 * g + upbit(S, lane + 32 * j) : g;
            const int b1 = getbyte(pb, j), c = g ? c1 : c0;
            const int b = bucket_of(bk, xw[j]);
            setbyte(pb, j, b);
            const bool isc = in && b1 == c;
            const int g2 = isc ? g : 2 * g + (b1 > c ? 1 : 0);
            gw = (gw & ~(3u << (2 * j))) | ((uint32_t)g2 << (2 * j));
            pend2 |= (isc ? 1u : 0u) << j;
            if (in && !isc) atomicAdd(&S.hist[g2][b >> 1], hinc(b));
        }
        for (uint32_t p = pend2; p; p &= p - 1u) {
            const int j = __ffs(p) - 1;
            med_append(S, ord32(pick(xv, j)), lane + 32 * j, (int)((gw >> (2 * j)) & 3u), getbyte_rt(pb, j), 0.f);
        }
#pragma unroll
        for (int j = 0; j < MRK; ++j) {  // v is spent: psi of the register keys (for the last pass)
            if (j >= 8 && !rx) break;
            const int q = lane + 32 * j;
            xp[j] = j < kk && q < n ? a.psi[s0 + q] : 0.f;
        }
        if (kk > MRK) {
            const uint2 r = med_tail2(S, bk, c0, c1, n, kk, lane, gw, pend, pend2);
            gw = r.x;
            pend2 = r.y;
        }
        pend = pend2;
        __syncwarp();
        const int L = S.ncl;
        if (lane < 16) S.upb[lane] = 0u;
        med_rank(S, ids, L, lane);  // (ends in a warp barrier before upb is written)
        for (int t = lane; t < L; t += 32) {  // the candidates join their V half
            const int g = S.cg[t], up = (int)S.crank[t] > S.brank[g] ? 1 : 0, b = S.cb[t];
            atomicAdd(&S.hist[2 * g + up][b >> 1], hinc(b));
            if (up) atomicOr(&S.upb[S.cq[t] >> 5], 1u << (S.cq[t] & 31));
        }
        __syncwarp();
        med_scan<4>(S, n, lane);
        __syncwarp();
        general = S.ncand[0] + S.ncand[1] + S.ncand[2] + S.ncand[3] > MCL;
    }
    if (general) {  // crowded boundary buckets: the general selection path
        __syncwarp();
        med_general(a, e, s0, n, U.s);
        return;
    }
    // ---- bins: the W halves; psi summed per bin
    const int c0 = S.bkt[0], c1 = S.bkt[1], c2 = S.bkt[2], c3 = S.bkt[3];
    (&S.binpart[0][0])[lane] = 0u;
    if (lane == 0) S.ncl = 0;
    __syncwarp();
    uint32_t pend3 = 0u;
#pragma unroll
    for (int j = 0; j < MRK; ++j) {
        if (j >= 8 && !rx) break;
        const int q = lane + 32 * j;
        const bool in = j < kk && q < n;
        int g = (int)((gw >> (2 * j)) & 3u);
        g = ((pend >> j) & 1u) ? 2 * g + upbit(S, q) : g;
        gw = (gw & ~(3u << (2 * j))) | ((uint32_t)g << (2 * j));
        const int b2 = getbyte(pb, j), c = g == 0 ? c0 : (g == 1 ? c1 : (g == 2 ? c2 : c3));
        const bool isc = in && b2 == c;
        pend3 |= (isc ? 1u : 0u) << j;
        const int bn = 2 * g + (b2 > c ? 1 : 0);
        if (in && !isc) {
            a.bin[s0 + q] = (unsigned char)bn;
            med_binadd(S, bn, psi_fixed(xp[j]));
        }
    }
    for (uint32_t p = pend3; p; p &= p - 1u) {
        const int j = __ffs(p) - 1;
        med_append(S, ord32(pick(xw, j)), lane + 32 * j, (int)((gw >> (2 * j)) & 3u), 0, pick(xp, j));
    }
    if (kk > MRK) med_tail3(S, a.bin + s0, make_int4(c0, c1, c2, c3), n, kk, lane, gw, pend);
    __syncwarp();
    const int L = S.ncl;
    med_rank(S, ids, L, lane);
    for (int t = lane; t < L; t += 32) {  // the candidates' bins
        const int g = S.cg[t], bn = 2 * g + ((int)S.crank[t] > S.brank[g] ? 1 : 0);
        a.bin[s0 + S.cq[t]] = (unsigned char)bn;
        med_binadd(S, bn, psi_fixed(S.cps[t]));
    }
    __syncwarp();
    if (lane < 8) {
        const unsigned long long sum = (unsigned long long)S.binpart[lane][0] +
                                       ((unsigned long long)S.binpart[lane][1] << 19) +
                                       ((unsigned long long)S.binpart[lane][2] << 38);
        const double cm = __ull2double_rn(sum) * (1.0 / (double)(1ull << 54)) * recip_n(split_size(n, lane, 3));
        a.ecm[(size_t)8 * e + lane] = cm;
        a.ecmT[(size_t)8 * e + lane] = (float)cm;
    }
}

// 2 x 2 x 2 bins and <phi|V> of the elements of at most 512 particles, one
// warp per element, independent of the moments (bucket ranges from the
// element's own value range, the mean psi of an element with fewer
// particles than bins from its particles). Six blocks per SM at most: 80
// registers (a few spilled: at 96, without spills, the kernel took more of
// the SM from the moments beside it and the step was no faster) and 36 KB of
// shared memory per 4-warp block. The grid may hold
// fewer blocks than element groups (the warps then take elements from the
// counter), leaving SM room for the kernels that run beside it.
__global__ void __launch_bounds__(32 * WARPS_PER_BLOCK, 6) k_bins_med(const MomArgs<float> a, int nt,
                                                                       int* next) {
    __shared__ MedUnion sm[WARPS_PER_BLOCK];
    const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
    // each warp takes the next element from a counter (zeroed before the
    // launch), so warps that drew large elements do not set the kernel's end
    for (;;) {
        int e = 0;
        if (lane == 0) e = atomicAdd(next, 1);
        e = __shfl_sync(FULLW, e, 0);
        if (e >= nt) break;
        med_bins_element(a, e, lane, sm[wq]);
        __syncwarp();  // the warp's shared memory is free for its next element
    }
}

// the crowded elements from the element offsets: 512 < n <= 4096 into listA,
// n > 4096 into listB (list order is free: every element is reduced by one
// team in a fixed order)
__global__ void k_crowded(const int* __restrict__ off, int nt, int* lcnt, int* listA, int* listB) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt) return;
    const int n = off[e + 1] - off[e];
    if (n > 4096) listB[atomicAdd(&lcnt[1], 1)] = e;
    else if (n > 512) listA[atomicAdd(&lcnt[0], 1)] = e;
}

// block of 256 threads per element: 512 < n <= 4096 (crowded elements). The
// blocks take the listed elements from a shared counter (lcnt[2]), so a block
// that drew large elements does not hold up the others.
template <bool KAHAN, int PART>
__global__ void __launch_bounds__(256) k_moments_sel_big(const MomArgs<float> a) {
    __shared__ SelSmem<4096> sm;
    __shared__ int jnext;
    const int cnt = a.lcnt[0];
    int* next = PART == SEL_BINS ? &a.lcnt[4] : &a.lcnt[2];
    for (;;) {
        if (threadIdx.x == 0) jnext = atomicAdd(next, 1);
        __syncthreads();
        const int j = jnext;
        if (j >= cnt) break;
        const int e = a.listA[j];
        const int s0 = a.off[e], n = a.off[e + 1] - s0;
        sel_element<KAHAN, 256, 4096, PART>(a, e, s0, n, sm);
        __syncthreads();  // the element's shared memory and jnext are free again
    }
}

template <typename T, bool KAHAN>
int run(pdf_ctx* c) {
    MomArgs<T> a;
    a.off = c->off;
    a.u = (const T*)c->stA[2]; a.v = (const T*)c->stA[3]; a.w = (const T*)c->stA[4];
    a.om = (const T*)c->stA[5]; a.psi = (const T*)c->stA[6];
    a.id = c->idA;
    a.G0 = c->p.nb1; a.G1 = c->p.nb2; a.G2 = c->p.nb3; a.B = c->B;
    a.en = c->en; a.emean = c->emean; a.eR = c->eR; a.epsivar = c->epsivar; a.ecm = c->ecm;
    a.ecmT = (T*)c->ecmT;
    a.bin = c->bin;
    a.scratch = c->sort_scratch;
    a.scratch_n = c->sort_scratch_n;
    a.status = c->d_status;
    a.min_n = -1;
    a.lcnt = a.listA = a.listB = nullptr;
    if constexpr (sizeof(T) == 4) {
        // warp-per-element kernels for segments up to WARP_MAX_N particles:
        // median splits for 2 x 2 x 2 bins, else a shared-memory bitonic sort
        a.min_n = WARP_MAX_N;
        const unsigned blocks = (unsigned)((c->m.nt + WARPS_PER_BLOCK - 1) / WARPS_PER_BLOCK);
        const bool medians = c->p.nb1 == 2 && c->p.nb2 == 2 && c->p.nb3 == 2;
        if (medians) {
            // crowded elements (particle density drifts during a run) get their
            // own size class with a larger shared-memory slice per warp
            // the warp kernel runs on the high-priority side stream; the block
            // kernels of the crowded elements (particle counts spread during a
            // run) run concurrently on the context stream and fill the SMs the
            // warp kernel's last waves leave
            a.min_n = 4096;
            // [0], [1]: list lengths; [2]: next element of listA for its moments,
            // [4] for its bins; [3]: next element of the warp bins kernel
            a.lcnt = c->elist;
            a.listA = c->elist + 8;
            a.listB = c->elist + 8 + c->m.nt;
            // Three streams from the sorted state on: the side stream takes the
            // moments of the elements of at most 512 particles, the bins
            // stream their bins (which need no moments: the bucket ranges are
            // each element's own value range, and only the next particle step
            // reads the bins), the context stream the crowded elements'
            // moments (the block kernel above 4096 particles takes moments and
            // bins together) and then the field chain, which waits for the
            // moments only. The crowded elements' bins follow the warp bins
            // on the bins stream, after the crowded moments (their bucket
            // ranges). pdf_step and pdf_estimate_stats join the bins stream
            // back before the step ends.
            PDF_CUDA(c, cudaMemsetAsync(a.lcnt, 0, 8 * sizeof(int), c->s));
            PDF_CUDA(c, cudaEventRecord(c->side_fork, c->s));
            PDF_CUDA(c, cudaStreamWaitEvent(c->s2, c->side_fork, 0));
            PDF_CUDA(c, cudaStreamWaitEvent(c->s3, c->side_fork, 0));
            k_moments_w<KAHAN><<<blocks, 32 * WARPS_PER_BLOCK, 0, c->s2>>>(a, c->m.nt);
            PDF_CUDA(c, cudaEventRecord(c->side_join, c->s2));
            timing_begin(c, PDF_K_BINS, c->s3);
            const unsigned bgrid = c->bins_bps > 0 ? std::min(blocks, (unsigned)(c->bins_bps * c->num_sms)) : blocks;
            k_bins_med<<<bgrid, 32 * WARPS_PER_BLOCK, 0, c->s3>>>(a, c->m.nt, a.lcnt + 3);
            k_crowded<<<(c->m.nt + 255) / 256, 256, 0, c->s>>>(c->off, c->m.nt, a.lcnt, a.listA, a.listB);
            const int big = std::min(c->m.nt, 3 * c->num_sms);
            k_moments_sel_big<KAHAN, SEL_MOMENTS><<<big, 256, 0, c->s>>>(a);
            const size_t smem = sizeof(SortKey) * STATS_CAP;
            k_moments<T, KAHAN><<<(unsigned)std::min(c->m.nt, c->num_sms), STATS_THREADS, smem, c->s>>>(a);
            PDF_CUDA(c, cudaEventRecord(c->crowd_done, c->s));
            PDF_CUDA(c, cudaStreamWaitEvent(c->s3, c->crowd_done, 0));
            k_moments_sel_big<KAHAN, SEL_BINS><<<big, 256, 0, c->s3>>>(a);
            timing_end(c, PDF_K_BINS, c->s3);
            PDF_CUDA(c, cudaEventRecord(c->bins_join, c->s3));
            c->bins_pending = true;
            PDF_CUDA(c, cudaStreamWaitEvent(c->s, c->side_join, 0));
            c->launches += 6;
            PDF_CUDA(c, cudaGetLastError());
            return PDF_OK;
        } else {
            k_moments_warp<KAHAN><<<blocks, 32 * WARPS_PER_BLOCK, 0, c->s>>>(a, c->m.nt);
            ++c->launches;
        }
    }
    const size_t smem = sizeof(SortKey) * STATS_CAP;
    const unsigned grid = a.listB ? (unsigned)std::min(c->m.nt, c->num_sms) : (unsigned)c->m.nt;
    k_moments<T, KAHAN><<<grid, STATS_THREADS, smem, c->s>>>(a);
    ++c->launches;
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

}  // namespace

int prepare_moments(pdf_ctx* c) {
    if (!c->s2) {
        int lo = 0, hi = 0;
        PDF_CUDA(c, cudaDeviceGetStreamPriorityRange(&lo, &hi));
        PDF_CUDA(c, cudaStreamCreateWithPriority(&c->s2, cudaStreamNonBlocking, hi));
        PDF_CUDA(c, cudaEventCreateWithFlags(&c->side_fork, cudaEventDisableTiming));
        PDF_CUDA(c, cudaEventCreateWithFlags(&c->side_join, cudaEventDisableTiming));
        PDF_CUDA(c, cudaEventCreateWithFlags(&c->side_join2, cudaEventDisableTiming));
        // the bins stream at the lowest priority: blocks of the field chain
        // take the SM slots the bins kernel frees first
        PDF_CUDA(c, cudaStreamCreateWithPriority(&c->s3, cudaStreamNonBlocking, lo));
        PDF_CUDA(c, cudaEventCreateWithFlags(&c->bins_join, cudaEventDisableTiming));
        PDF_CUDA(c, cudaEventCreateWithFlags(&c->crowd_done, cudaEventDisableTiming));
        PDF_CUDA(c, cudaStreamCreateWithFlags(&c->s_cond, cudaStreamNonBlocking));
    }
    const int smem = (int)(sizeof(SortKey) * STATS_CAP);
    PDF_CUDA(c, cudaFuncSetAttribute(k_moments<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    PDF_CUDA(c, cudaFuncSetAttribute(k_moments<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    PDF_CUDA(c, cudaFuncSetAttribute(k_moments<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    return PDF_OK;
}

int join_bins(pdf_ctx* c) {
    if (!c->bins_pending) return PDF_OK;
    c->bins_pending = false;
    PDF_CUDA(c, cudaStreamWaitEvent(c->s, c->bins_join, 0));
    return PDF_OK;
}

int launch_moments(pdf_ctx* c) {
    timing_begin(c, PDF_K_MOMENTS);
    int st;
    if (c->prec == 0) st = run<double, false>(c);
    else if (c->prec == 1) st = run<float, false>(c);
    else st = run<float, true>(c);
    timing_end(c, PDF_K_MOMENTS);
    return st;
}
