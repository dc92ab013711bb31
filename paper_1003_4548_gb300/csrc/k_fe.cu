// k_fe.cu -- elliptic relaxation of the GLM drift (Eqs. Gij, C0,
// elliptic-relaxation, H, L) by P1 finite elements.
//
// Per step: the right-hand side f_ij = 1/2 (1 - C1) k <omega> delta_ij +
// k H_ijkl d<U_k>/dx_l at the nodes (statistically two-dimensional field:
// in-plane wp_11, wp_12, wp_21, wp_22 and wp_33) and the wall values
// wp_ij = -er_wall eps n_i n_j (both formed in the node gradient kernel of
// k_fields.cu, from the node's own gradient), and the Galerkin system (M + K_{L^2}) wp = M f
// over the periodic-merged nodes, solved for the five components at once by
// Jacobi-preconditioned CG in FP64 (warm start from the previous step).
//
// The solver is one persistent cooperative kernel: the grid walks the matrix
// rows, and the reductions of each iteration go through per-block partials
// summed in block order by every block (deterministic), separated by a grid
// barrier whose spin is bounded (status ST_BARRIER on expiry).

#include <cooperative_groups.h>

#include "coop.cuh"
#include "ff.cuh"
#include "pdf_internal.cuh"

namespace {

constexpr int NC = 5;

// values of M + K_{L^2} (Eq. elliptic-relaxation in Galerkin form): each
// nonzero is its mass entry plus the L^2-weighted stiffness contributions of
// the elements that share the edge (L is an element constant, Eq. L);
// FP64, and the float-float pair for the compensated-FP32 CG
__global__ void k_fe_assemble(int64_t nnz, const double* __restrict__ mval, const int* __restrict__ kc_off,
                              const int* __restrict__ kc_elem, const double* __restrict__ kc_geo,
                              const double* __restrict__ eder, double* aval, float2* avf) {
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= nnz) return;
    double s = mval[q];
    for (int k = kc_off[q]; k < kc_off[q + 1]; ++k) {
        const double L = eder[9 * (size_t)kc_elem[k] + 8];
        s += L * L * kc_geo[k];
    }
    aval[q] = s;
    const ff v = ff_from_double(s);
    avf[q] = make_float2(v.hi, v.lo);
}

struct CGArgs {
    int nn;
    const int* __restrict__ rowptr;
    const int* __restrict__ colidx;
    const double* __restrict__ mval;
    const int* __restrict__ kc_off;
    const int* __restrict__ kc_elem;
    const double* __restrict__ kc_geo;
    const double* __restrict__ eder;  // L in column 8
    const int* __restrict__ rep;
    const unsigned char* __restrict__ is_wall;
    const double* __restrict__ f;
    const double* __restrict__ g;
    double* aval;
    float2* avf;   // aval as float-float (hi, lo), compensated-FP32 variant
    double* x;     // [nn][NC] node solution: warm start in, result out (canonical rows)
    double* zg;    // [nn][NC] preconditioned residual, shared between blocks for the SpMV
    double* part;  // [gridDim][PART_W]
    unsigned* bar;
    int* iters;
    int* status;
    const int* skip;       // surrogate: 1 = the network's wp passed the residual check, no solve
    const double* xprop;   // surrogate proposal (network at the free rows, Dirichlet values at the walls)
    double tol;
    int maxit;
    long long spin_max;  // polls of a grid barrier before it gives up (ST_BARRIER)
};

// the surrogate's check passed: take its proposal as the solution
__device__ __forceinline__ bool skip_solve(const CGArgs& a) {
    if (a.skip == nullptr || *(volatile const int*)a.skip == 0) return false;
    const int nc = blockDim.x / NC;  // rows per block
    const int c = threadIdx.x / nc, i = blockIdx.x * nc + threadIdx.x % nc;
    if (i < a.nn && a.rep[i] == i) a.x[NC * (size_t)i + c] = a.xprop[NC * (size_t)i + c];
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.iters = 0;
    return true;
}

constexpr int PART_W = 4 * NC;  // partial sums per block: 3 NC in phase A, NC in phase B

// Per-block sums over the rows of NV values per component (value v of
// component c of row t staged at red[(v * NC + c) * BS + t]); warp q sums
// value-component q in a fixed order and writes part[block][slot + q].
template <int BS>
__device__ void block_partial(const CGArgs& a, double* red, int nv, int slot) {
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = wid; q < nv * NC; q += (BS * NC) / 32) {
        double s = 0.0;
        for (int t = lane; t < BS; t += 32) s += red[q * BS + t];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) a.part[(size_t)blockIdx.x * PART_W + slot + q] = s;
    }
    __syncthreads();
}

// after a barrier: sums over all blocks of nv*NC partials (warp q: value q,
// fixed lane-strided order and shuffle tree; identical in every block)
__device__ void grid_sum(const CGArgs& a, int slot, int nvals, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = wid; q < nvals; q += blockDim.x / 32) {
        // the loads of a chunk of 4 x 32 blocks are issued together, then
        // summed in order
        double s = 0.0;
        for (int b0 = 0; b0 < (int)gridDim.x; b0 += 4 * 32) {
            double v[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int bl = b0 + 32 * k + lane;
                v[k] = bl < (int)gridDim.x ? a.part[(size_t)bl * PART_W + slot + q] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) s += v[k];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[q] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// z = Ainv_b r for the NC components of the block's rows, on the tensor
// cores: Z[BS x 8] = Ainv[BS x BS] R[BS x 8] (components padded to 8) with
// mma.sync m16n8k8 TF32 inputs and FP32 accumulation; warp w < BS/16 owns
// rows 16w..16w+15. Ainv is column-major in shared memory, R and Z are
// component-major (rv[c*BS + row]).
template <int BS>
__device__ __forceinline__ double block_precondition(const float* __restrict__ inv, float* rv, float* zv, int c,
                                                     int t, double r) {
    rv[c * BS + t] = (float)r;
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid < BS / 16) {
        const int g = lane >> 2, tq = lane & 3, m0 = 16 * wid;
        float d0 = 0.f, d1 = 0.f, d2 = 0.f, d3 = 0.f;
#pragma unroll 4
        for (int k0 = 0; k0 < BS; k0 += 8) {
            const uint32_t a0 = to_tf32(inv[(k0 + tq) * (BS + 4) + m0 + g]);
            const uint32_t a1 = to_tf32(inv[(k0 + tq) * (BS + 4) + m0 + g + 8]);
            const uint32_t a2 = to_tf32(inv[(k0 + tq + 4) * (BS + 4) + m0 + g]);
            const uint32_t a3 = to_tf32(inv[(k0 + tq + 4) * (BS + 4) + m0 + g + 8]);
            const uint32_t b0 = g < NC ? to_tf32(rv[g * BS + k0 + tq]) : 0u;
            const uint32_t b1 = g < NC ? to_tf32(rv[g * BS + k0 + tq + 4]) : 0u;
            asm volatile(
                "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                "{%0,%1,%2,%3};"
                : "+f"(d0), "+f"(d1), "+f"(d2), "+f"(d3)
                : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
        }
        // D(row, col): d0 (g, 2tq), d1 (g, 2tq+1), d2 (g+8, 2tq), d3 (g+8, 2tq+1)
        const int c0 = 2 * tq, c1 = 2 * tq + 1;
        if (c0 < NC) { zv[c0 * BS + m0 + g] = d0; zv[c0 * BS + m0 + g + 8] = d2; }
        if (c1 < NC) { zv[c1 * BS + m0 + g] = d1; zv[c1 * BS + m0 + g + 8] = d3; }
    }
    __syncthreads();
    return (double)zv[c * BS + t];
}

// Flexible (Polak-Ribiere) preconditioned CG in FP64 for the NC right-hand
// sides. One thread per (row, component); the rows of a block form the
// diagonal block of a block-Jacobi preconditioner whose FP32 explicit inverse
// (Gauss-Jordan without pivoting: the blocks are SPD) stays in shared memory
// for the whole solve. A p follows A p_{k+1} = A z_{k+1} + beta_k A p_k, so
// each iteration has one SpMV (on z) and two grid reductions.
template <int BS>
__global__ void __launch_bounds__(BS * NC) k_pcg(const CGArgs a) {
    if (skip_solve(a)) return;
    extern __shared__ float smem[];
    float* inv = smem;                                           // column j at inv[j*(BS+4) ..]
    float* rv = smem + BS * (BS + 4);                            // NC*BS
    float* zv = rv + NC * BS;                                    // NC*BS
    double* red = reinterpret_cast<double*>(zv + NC * BS);       // 3*NC*BS
    __shared__ double s_a[3 * NC], s_rz[NC], s_rr[NC], s_bn[NC], s_pap[NC], s_alpha[NC], s_beta[NC];
    __shared__ int s_active[NC];
    const int c = threadIdx.x / BS, t = threadIdx.x % BS;
    const int i = blockIdx.x * BS + t;
    const bool have = i < a.nn;
    const bool free_row = have && a.rep[i] == i && !a.is_wall[i];
    // b = M f and the Dirichlet values (the matrix was assembled by k_fe_assemble)
    double b = 0.0, x = 0.0;
    if (have) {
        for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) b += a.mval[q] * a.f[NC * (size_t)a.colidx[q] + c];
        x = a.is_wall[i] ? a.g[NC * (size_t)i + c] : a.x[NC * (size_t)i + c];
        a.x[NC * (size_t)i + c] = x;
    }
    for (int q = threadIdx.x; q < BS * (BS + 4); q += BS * NC) inv[q] = 0.f;
    __syncthreads();
    if (c == 0) {
        if (free_row) {
            for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
                const int j = a.colidx[q], jl = j - blockIdx.x * BS;
                if (jl >= 0 && jl < BS && a.rep[j] == j && !a.is_wall[j]) inv[jl * (BS + 4) + t] = (float)a.aval[q];
            }
        } else {
            inv[t * (BS + 4) + t] = 1.f;
        }
    }
    __syncthreads();
    for (int k = 0; k < BS; ++k) {  // in-place Gauss-Jordan inverse
        const float fk = inv[k * (BS + 4) + t];  // a[t][k]
        const float p = inv[k * (BS + 4) + k];
        __syncthreads();
        if (c == 0) {
            const float v = (t == k) ? 1.f : inv[t * (BS + 4) + k];  // a[k][t]
            inv[t * (BS + 4) + k] = v / p;
        }
        __syncthreads();
        if (t != k) {
            for (int j = c; j < BS; j += NC) {
                if (j == k) inv[k * (BS + 4) + t] = -fk * inv[k * (BS + 4) + k];
                else inv[j * (BS + 4) + t] -= fk * inv[j * (BS + 4) + k];
            }
        }
        __syncthreads();
    }
    grid_barrier(a.bar, a.status, a.spin_max);  // all x (warm start + Dirichlet) and matrix rows are in place
    // r = b - A x; z = Ainv r; p = z
    double r, z, p, ap;
    {
        double s = 0.0, b0 = b;
        if (free_row) {
            for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
                const int j = a.colidx[q];
                const double xv = a.aval[q] * a.x[NC * (size_t)j + c];
                s += xv;
                if (a.is_wall[j]) b0 -= xv;
            }
        }
        r = free_row ? b - s : 0.0;
        z = block_precondition<BS>(inv, rv, zv, c, t, r);
        if (!free_row) z = 0.0;
        p = z;
        if (have) a.zg[NC * (size_t)i + c] = z;
        red[(0 * NC + c) * BS + t] = r * z;
        red[(1 * NC + c) * BS + t] = r * r;
        red[(2 * NC + c) * BS + t] = free_row ? b0 * b0 : 0.0;
        block_partial<BS>(a, red, 3, 0);
    }
    grid_barrier(a.bar, a.status, a.spin_max);
    grid_sum(a, 0, 3 * NC, s_a);
    if (threadIdx.x < NC) {
        s_rz[threadIdx.x] = s_a[threadIdx.x];
        s_rr[threadIdx.x] = s_a[NC + threadIdx.x];
        s_bn[threadIdx.x] = sqrt(s_a[2 * NC + threadIdx.x]);
    }
    {  // A p_0
        double s = 0.0;
        if (free_row)
            for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) s += a.aval[q] * a.zg[NC * (size_t)a.colidx[q] + c];
        ap = free_row ? s : 0.0;
        red[c * BS + t] = p * ap;
        block_partial<BS>(a, red, 1, 3 * NC);
    }
    grid_barrier(a.bar, a.status, a.spin_max);
    grid_sum(a, 3 * NC, NC, s_pap);
    int it = 0;
    for (;; ++it) {
        if (threadIdx.x < NC) {
            const int k = threadIdx.x;
            s_active[k] = (s_bn[k] > 0.0) && (sqrt(s_rr[k]) > a.tol * s_bn[k]);
            s_alpha[k] = s_active[k] ? s_rz[k] / s_pap[k] : 0.0;
        }
        __syncthreads();
        bool any = false;
#pragma unroll
        for (int k = 0; k < NC; ++k) any |= s_active[k] != 0;
        if (!any) break;
        if (it >= a.maxit) {
            if (blockIdx.x == 0 && threadIdx.x == 0) set_status(a.status, ST_CG);
            break;
        }
        const bool act = s_active[c] != 0;
        // phase A: x += alpha p, r -= alpha Ap, z = Ainv r
        {
            const double rold = r;
            if (act) {
                x += s_alpha[c] * p;
                r -= s_alpha[c] * ap;
            }
            double zn = block_precondition<BS>(inv, rv, zv, c, t, r);
            if (!free_row) zn = 0.0;
            if (act) z = zn;
            if (have) a.zg[NC * (size_t)i + c] = z;
            red[(0 * NC + c) * BS + t] = r * z;
            red[(1 * NC + c) * BS + t] = rold * z;
            red[(2 * NC + c) * BS + t] = r * r;
            block_partial<BS>(a, red, 3, 0);
        }
        grid_barrier(a.bar, a.status, a.spin_max);
        grid_sum(a, 0, 3 * NC, s_a);
        if (threadIdx.x < NC) {
            const int k = threadIdx.x;
            s_beta[k] = s_active[k] ? (s_a[k] - s_a[NC + k]) / s_rz[k] : 0.0;
        }
        __syncthreads();
        // phase B: p = z + beta p (Polak-Ribiere); A p = A z + beta A p
        {
            double s = 0.0;
            if (free_row)
                for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q)
                    s += a.aval[q] * a.zg[NC * (size_t)a.colidx[q] + c];
            if (act) {
                p = z + s_beta[c] * p;
                ap = (free_row ? s : 0.0) + s_beta[c] * ap;
            }
            red[c * BS + t] = p * ap;
            block_partial<BS>(a, red, 1, 3 * NC);
        }
        grid_barrier(a.bar, a.status, a.spin_max);
        if (threadIdx.x < NC && s_active[threadIdx.x]) {
            s_rz[threadIdx.x] = s_a[threadIdx.x];
            s_rr[threadIdx.x] = s_a[2 * NC + threadIdx.x];
        }
        grid_sum(a, 3 * NC, NC, s_pap);
    }
    if (free_row) a.x[NC * (size_t)i + c] = x;
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.iters = it;
}


// ---------------------------------------------------------------------------
// Compensated-FP32 variant of the same flexible PCG: the iteration runs in
// float-float arithmetic (~48-bit significand: products by FMA TwoProduct,
// sums by TwoSum) -- the SpMV, the vector updates and the dot products with
// their block and grid reductions -- so no FP64 instruction sits in the
// loop; the initial residual, the CG coefficients and the stored solution
// are FP64. Its solution is checked against the FP64 CPU oracle.
// ---------------------------------------------------------------------------
template <int BS>
__device__ void block_partial_ff(const CGArgs& a, const float* rh, const float* rl, int nv, int slot) {
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float2* part = reinterpret_cast<float2*>(a.part);
    for (int q = wid; q < nv * NC; q += (BS * NC) / 32) {
        ff s = ff{0.f, 0.f};
        for (int t = lane; t < BS; t += 32) s = ff_add(s, ff{rh[q * BS + t], rl[q * BS + t]});
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = ff_add(s, ff_shfl_down(s, o));
        if (lane == 0) part[(size_t)blockIdx.x * PART_W + slot + q] = make_float2(s.hi, s.lo);
    }
    __syncthreads();
}

__device__ void grid_sum_ff(const CGArgs& a, int slot, int nvals, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const float2* part = reinterpret_cast<const float2*>(a.part);
    for (int q = wid; q < nvals; q += blockDim.x / 32) {
        ff s = ff{0.f, 0.f};
        for (int bl = lane; bl < (int)gridDim.x; bl += 32) {
            const float2 v = part[(size_t)bl * PART_W + slot + q];
            s = ff_add(s, ff{v.x, v.y});
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s = ff_add(s, ff_shfl_down(s, o));
        if (lane == 0) out[q] = ff_to_double(s);
    }
    __syncthreads();
}

template <int BS>
__global__ void __launch_bounds__(BS * NC) k_pcg_ff(const CGArgs a) {
    if (skip_solve(a)) return;
    extern __shared__ float smem[];
    float* inv = smem;
    float* rv = smem + BS * (BS + 4);
    float* zv = rv + NC * BS;
    float* redh = zv + NC * BS;      // 3*NC*BS
    float* redl = redh + 3 * NC * BS;
    __shared__ double s_a[3 * NC], s_rz[NC], s_rr[NC], s_bn[NC], s_pap[NC], s_alpha[NC], s_beta[NC];
    __shared__ int s_active[NC];
    const int c = threadIdx.x / BS, t = threadIdx.x % BS;
    const int i = blockIdx.x * BS + t;
    const bool have = i < a.nn;
    const bool free_row = have && a.rep[i] == i && !a.is_wall[i];
    double b = 0.0, x0 = 0.0;
    if (have) {
        for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) b += a.mval[q] * a.f[NC * (size_t)a.colidx[q] + c];
        x0 = a.is_wall[i] ? a.g[NC * (size_t)i + c] : a.x[NC * (size_t)i + c];
        a.x[NC * (size_t)i + c] = x0;
    }
    for (int q = threadIdx.x; q < BS * (BS + 4); q += BS * NC) inv[q] = 0.f;
    __syncthreads();
    if (c == 0) {
        if (free_row) {
            for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
                const int j = a.colidx[q], jl = j - blockIdx.x * BS;
                if (jl >= 0 && jl < BS && a.rep[j] == j && !a.is_wall[j]) inv[jl * (BS + 4) + t] = (float)a.aval[q];
            }
        } else {
            inv[t * (BS + 4) + t] = 1.f;
        }
    }
    __syncthreads();
    for (int k = 0; k < BS; ++k) {  // in-place Gauss-Jordan inverse (FP32)
        const float fk = inv[k * (BS + 4) + t];
        const float p = inv[k * (BS + 4) + k];
        __syncthreads();
        if (c == 0) {
            const float v = (t == k) ? 1.f : inv[t * (BS + 4) + k];
            inv[t * (BS + 4) + k] = v / p;
        }
        __syncthreads();
        if (t != k) {
            for (int j = c; j < BS; j += NC) {
                if (j == k) inv[k * (BS + 4) + t] = -fk * inv[k * (BS + 4) + k];
                else inv[j * (BS + 4) + t] -= fk * inv[j * (BS + 4) + k];
            }
        }
        __syncthreads();
    }
    grid_barrier(a.bar, a.status, a.spin_max);
    float* zg = reinterpret_cast<float*>(a.zg);
    ff x = ff_from_double(x0), r, p, ap;
    float z;
    {  // r = b - A x in FP64 once, then float-float
        double s = 0.0, b0 = b;
        if (free_row) {
            for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
                const int j = a.colidx[q];
                const double xv = a.aval[q] * a.x[NC * (size_t)j + c];
                s += xv;
                if (a.is_wall[j]) b0 -= xv;
            }
        }
        r = ff_from_double(free_row ? b - s : 0.0);
        z = (float)block_precondition<BS>(inv, rv, zv, c, t, (double)r.hi);
        if (!free_row) z = 0.f;
        p = ff_make(z);
        if (have) zg[NC * (size_t)i + c] = z;
        const ff rz = ff_mul_f(r, z), rr = ff_mul(r, r), bb = ff_from_double(free_row ? b0 * b0 : 0.0);
        redh[(0 * NC + c) * BS + t] = rz.hi; redl[(0 * NC + c) * BS + t] = rz.lo;
        redh[(1 * NC + c) * BS + t] = rr.hi; redl[(1 * NC + c) * BS + t] = rr.lo;
        redh[(2 * NC + c) * BS + t] = bb.hi; redl[(2 * NC + c) * BS + t] = bb.lo;
        block_partial_ff<BS>(a, redh, redl, 3, 0);
    }
    grid_barrier(a.bar, a.status, a.spin_max);
    grid_sum_ff(a, 0, 3 * NC, s_a);
    if (threadIdx.x < NC) {
        s_rz[threadIdx.x] = s_a[threadIdx.x];
        s_rr[threadIdx.x] = s_a[NC + threadIdx.x];
        s_bn[threadIdx.x] = sqrt(s_a[2 * NC + threadIdx.x]);
    }
    grid_barrier(a.bar, a.status, a.spin_max);  // the partials are reused below
    {  // A p_0
        ff s = ff{0.f, 0.f};
        if (free_row)
            for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
                const float2 av = a.avf[q];
                s = ff_add(s, ff_mul_f(ff{av.x, av.y}, zg[NC * (size_t)a.colidx[q] + c]));
            }
        ap = free_row ? s : ff{0.f, 0.f};
        const ff pap = ff_mul(p, ap);
        redh[c * BS + t] = pap.hi;
        redl[c * BS + t] = pap.lo;
        block_partial_ff<BS>(a, redh, redl, 1, 3 * NC);
    }
    grid_barrier(a.bar, a.status, a.spin_max);
    grid_sum_ff(a, 3 * NC, NC, s_pap);
    int it = 0;
    for (;; ++it) {
        if (threadIdx.x < NC) {
            const int k = threadIdx.x;
            s_active[k] = (s_bn[k] > 0.0) && (sqrt(s_rr[k]) > a.tol * s_bn[k]);
            s_alpha[k] = s_active[k] ? s_rz[k] / s_pap[k] : 0.0;
        }
        __syncthreads();
        bool any = false;
#pragma unroll
        for (int k = 0; k < NC; ++k) any |= s_active[k] != 0;
        if (!any) break;
        if (it >= a.maxit) {
            if (blockIdx.x == 0 && threadIdx.x == 0) set_status(a.status, ST_CG);
            break;
        }
        const bool act = s_active[c] != 0;
        {
            const ff rold = r;
            if (act) {
                const ff al = ff_from_double(s_alpha[c]);
                x = ff_add(x, ff_mul(al, p));
                r = ff_add(r, ff_neg(ff_mul(al, ap)));
            }
            float zn = (float)block_precondition<BS>(inv, rv, zv, c, t, (double)r.hi);
            if (!free_row) zn = 0.f;
            if (act) z = zn;
            if (have) zg[NC * (size_t)i + c] = z;
            const ff rz = ff_mul_f(r, z), roz = ff_mul_f(rold, z), rr = ff_mul(r, r);
            redh[(0 * NC + c) * BS + t] = rz.hi; redl[(0 * NC + c) * BS + t] = rz.lo;
            redh[(1 * NC + c) * BS + t] = roz.hi; redl[(1 * NC + c) * BS + t] = roz.lo;
            redh[(2 * NC + c) * BS + t] = rr.hi; redl[(2 * NC + c) * BS + t] = rr.lo;
            block_partial_ff<BS>(a, redh, redl, 3, 0);
        }
        grid_barrier(a.bar, a.status, a.spin_max);
        grid_sum_ff(a, 0, 3 * NC, s_a);
        if (threadIdx.x < NC) {
            const int k = threadIdx.x;
            s_beta[k] = s_active[k] ? (s_a[k] - s_a[NC + k]) / s_rz[k] : 0.0;
        }
        __syncthreads();
        {
            ff s = ff{0.f, 0.f};
            if (free_row)
                for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
                    const float2 av = a.avf[q];
                    s = ff_add(s, ff_mul_f(ff{av.x, av.y}, zg[NC * (size_t)a.colidx[q] + c]));
                }
            if (act) {
                const ff be = ff_from_double(s_beta[c]);
                p = ff_add(ff_make(z), ff_mul(be, p));
                ap = ff_add(free_row ? s : ff{0.f, 0.f}, ff_mul(be, ap));
            }
            const ff pap = ff_mul(p, ap);
            redh[c * BS + t] = pap.hi;
            redl[c * BS + t] = pap.lo;
            block_partial_ff<BS>(a, redh, redl, 1, 3 * NC);
        }
        grid_barrier(a.bar, a.status, a.spin_max);
        if (threadIdx.x < NC && s_active[threadIdx.x]) {
            s_rz[threadIdx.x] = s_a[threadIdx.x];
            s_rr[threadIdx.x] = s_a[2 * NC + threadIdx.x];
        }
        grid_sum_ff(a, 3 * NC, NC, s_pap);
    }
    if (free_row) a.x[NC * (size_t)i + c] = ff_to_double(x);
    if (blockIdx.x == 0 && threadIdx.x == 0) *a.iters = it;
}

template <int BS>
constexpr size_t pcg_ff_smem() {
    return sizeof(float) * (BS * (BS + 4) + 2 * NC * BS + 6 * NC * BS);
}

template <int BS>
constexpr size_t pcg_smem() {
    return sizeof(float) * (BS * (BS + 4) + 2 * NC * BS) + sizeof(double) * 3 * NC * BS;
}

}  // namespace

namespace {

template <int BS>
void* pcg_fn(bool ffv) { return ffv ? (void*)k_pcg_ff<BS> : (void*)k_pcg<BS>; }
template <int BS>
size_t pcg_bytes(bool ffv) { return ffv ? pcg_ff_smem<BS>() : pcg_smem<BS>(); }

template <int BS>
int try_blocks(pdf_ctx* c, int nn, int& per_sm, bool ffv) {
    const size_t smem = pcg_bytes<BS>(ffv);
    if (cudaFuncSetAttribute(pcg_fn<BS>(ffv), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return -1;
    per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pcg_fn<BS>(ffv), BS * NC, smem) != cudaSuccess)
        return -1;
    return (nn + BS - 1) / BS;
}

template <int BS>
cudaError_t launch_pcg(const CGArgs& a, int blocks, cudaStream_t s, bool ffv) {
    CGArgs aa = a;
    void* args[] = {&aa};
    return cudaLaunchCooperativeKernel(pcg_fn<BS>(ffv), dim3(blocks), dim3(BS * NC), args, pcg_bytes<BS>(ffv), s);
}

}  // namespace

// Lagged or surrogate wp inside a captured graph: the residual check decides
// on the device whether the FE solve runs. This gate takes the proposal as
// the solution where the check passed and sets the graph condition of the
// node that holds the cooperative CG, so a step that keeps its wp launches no
// cooperative grid (whose launch waits until the whole grid fits beside the
// kernels already running, e.g. the bins kernel beside the field chain).
__global__ void k_cg_gate(cudaGraphConditionalHandle h, const int* skip, const double* xprop, const int* rep,
                          double* x, int* iters, int nn) {
    const bool keep = *(volatile const int*)skip != 0;
    const size_t t = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (keep && t < (size_t)nn * NC) {
        const int i = (int)(t / NC);
        if (rep[i] == i) x[t] = xprop[t];
    }
    if (t == 0) {
        if (keep) *iters = 0;
        cudaGraphSetConditional(h, keep ? 0u : 1u);
    }
}

// grid of the cooperative CG for rows-per-block bs (0: the largest size whose
// grid is co-resident: fewer blocks and partial sums, a stronger block-Jacobi
// preconditioner)
namespace {

int choose_grid(pdf_ctx* c, int bs, bool ffv, int& chosen_bs, int& chosen_blocks);

}  // namespace

int prepare_elliptic(pdf_ctx* c, int bs) {
    int chosen = 0, blocks = 0;
    TRY_OK(choose_grid(c, bs, c->p.cg_precision == 1, chosen, blocks));
    c->fe_bs = chosen;
    c->fe_blocks = blocks;
    return PDF_OK;
}

namespace {

int choose_grid(pdf_ctx* c, int bs, bool ffv, int& chosen_bs, int& chosen_blocks) {
    const int nn = c->m.nn;
    int per_sm = 0, blocks = 0;
    const int order[3] = {192, 160, 128};
    int chosen = 0;
    for (int k = 0; k < 3 && !chosen; ++k) {
        const int b = order[k];
        if (bs && b != bs) continue;
        blocks = b == 192 ? try_blocks<192>(c, nn, per_sm, ffv)
                          : (b == 160 ? try_blocks<160>(c, nn, per_sm, ffv) : try_blocks<128>(c, nn, per_sm, ffv));
        if (blocks > 0 && blocks <= per_sm * c->num_sms) chosen = b;
    }
    if (!chosen) return fail(c, PDF_ERR_CAPACITY, "elliptic solver: mesh too large for one resident grid");
    if ((size_t)blocks * PART_W > (size_t)15 * 4096 || (blocks + 15) / 16 > 63)
        return fail(c, PDF_ERR_CAPACITY, "elliptic solver: partial-sum buffer too small");
    chosen_bs = chosen;
    chosen_blocks = blocks;
    return PDF_OK;
}

}  // namespace

int launch_fe_assemble(pdf_ctx* c, cudaStream_t s) {
    k_fe_assemble<<<(unsigned)((c->m.nnz + 255) / 256), 256, 0, s>>>(c->m.nnz, c->m.mval, c->m.kc_off, c->m.kc_elem,
                                                                    c->m.kc_geo, c->eder, c->m.aval, c->m.avf);
    ++c->launches;
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

int launch_elliptic(pdf_ctx* c) {
    const int nn = c->m.nn;
    timing_begin(c, PDF_K_ELLIPTIC);
    // the right-hand side (and the lagged proposal) was written by the node
    // gradient kernel; the assembly was launched on the side stream after the
    // element fields
    PDF_CUDA(c, cudaStreamWaitEvent(c->s, c->side_join, 0));
    PDF_CUDA(c, cudaGetLastError());
    if (c->sur_mode) {
        const int st = launch_surrogate(c);
        if (st != PDF_OK) return st;
    }
    if (c->fe_blocks == 0) {
        const int st = prepare_elliptic(c, 0);
        if (st != PDF_OK) return st;
    }
    CGArgs a;
    a.nn = nn;
    a.rowptr = c->m.rowptr; a.colidx = c->m.colidx; a.mval = c->m.mval;
    a.kc_off = c->m.kc_off; a.kc_elem = c->m.kc_elem; a.kc_geo = c->m.kc_geo;
    a.eder = c->eder; a.rep = c->m.rep; a.is_wall = c->m.is_wall;
    a.f = c->fe_f; a.g = c->fe_g; a.aval = c->m.aval; a.avf = c->m.avf;
    a.x = c->nwp;  // solution lives in the node array (canonical rows)
    a.zg = c->fe_z;
    a.part = c->fe_part; a.bar = c->fe_bar; a.iters = c->fe_iters; a.status = c->d_status;
    a.spin_max = c->wait_spins > 0 ? c->wait_spins : SPIN_DEFAULT;
    a.tol = c->p.cg_tol; a.maxit = c->p.cg_maxit;
    a.skip = c->sur_mode ? c->sur_skip : nullptr;
    a.xprop = c->fe_prop;
    cudaError_t err;
    const bool ffv = c->p.cg_precision == 1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaGraph_t graph = nullptr;
    if (c->sur_mode) PDF_CUDA(c, cudaStreamGetCaptureInfo(c->s, &cs, nullptr, &graph, nullptr, nullptr, nullptr));
    cudaStream_t cg_stream = c->s;
    if (c->sur_mode && cs == cudaStreamCaptureStatusActive) {
        // captured: the CG goes into the body of a conditional node that the
        // gate kernel opens only when the check rejected the proposal (the
        // condition defaults to 1: without the gate the CG runs and makes
        // the same decision itself)
        cudaGraphConditionalHandle h;
        PDF_CUDA(c, cudaGraphConditionalHandleCreate(&h, graph, 1, cudaGraphCondAssignDefault));
        const size_t tot = (size_t)nn * NC;
        k_cg_gate<<<(unsigned)((tot + 255) / 256), 256, 0, c->s>>>(h, c->sur_skip, c->fe_prop, c->m.rep, c->nwp,
                                                                    c->fe_iters, nn);
        ++c->launches;
        PDF_CUDA(c, cudaGetLastError());
        // cooperative grids of different contexts never run side by side (a
        // batch orders them in a chain): the chain joins the conditional node
        // only, so the gate and what precedes it do not wait for it
        if (c->coop_wait) PDF_CUDA(c, cudaStreamWaitEvent(c->s, c->coop_wait, 0));
        const cudaGraphNode_t* deps = nullptr;
        size_t nd = 0;
        PDF_CUDA(c, cudaStreamGetCaptureInfo(c->s, &cs, nullptr, &graph, &deps, nullptr, &nd));
        cudaGraphNodeParams np = {};
        np.type = cudaGraphNodeTypeConditional;
        np.conditional.handle = h;
        np.conditional.type = cudaGraphCondTypeIf;
        np.conditional.size = 1;
        cudaGraphNode_t node;
        PDF_CUDA(c, cudaGraphAddNode(&node, graph, deps, nullptr, nd, &np));
        PDF_CUDA(c, cudaStreamUpdateCaptureDependencies(c->s, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
        PDF_CUDA(c, cudaStreamBeginCaptureToGraph(c->s_cond, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                  cudaStreamCaptureModeRelaxed));
        cg_stream = c->s_cond;
    } else if (c->coop_wait) {
        // cooperative grids of different contexts never run side by side (a
        // batch orders them in a chain)
        PDF_CUDA(c, cudaStreamWaitEvent(c->s, c->coop_wait, 0));
    }
    if (c->fe_bs == 128) err = launch_pcg<128>(a, c->fe_blocks, cg_stream, ffv);
    else if (c->fe_bs == 160) err = launch_pcg<160>(a, c->fe_blocks, cg_stream, ffv);
    else err = launch_pcg<192>(a, c->fe_blocks, cg_stream, ffv);
    if (cg_stream != c->s) {
        cudaGraph_t body = nullptr;
        const cudaError_t end = cudaStreamEndCapture(cg_stream, &body);
        PDF_CUDA(c, err);
        PDF_CUDA(c, end);
    }
    PDF_CUDA(c, err);
    if (c->coop_done) PDF_CUDA(c, cudaEventRecord(c->coop_done, c->s));
    TRY_OK(launch_surrogate_rebase(c));
    // the periodic image rows take the canonical rows' solution in the node
    // pack kernel that follows
    ++c->launches;
    timing_end(c, PDF_K_ELLIPTIC);
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

