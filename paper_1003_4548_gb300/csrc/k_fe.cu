// k_fe.cu -- elliptic relaxation of the GLM drift (Eqs. Gij, C0,
// elliptic-relaxation, H, L) by P1 finite elements.
//
// Per step: the right-hand side f_ij = 1/2 (1 - C1) k <omega> delta_ij +
// k H_ijkl d<U_k>/dx_l at the nodes (statistically two-dimensional field:
// in-plane wp_11, wp_12, wp_21, wp_22 and wp_33), the wall values
// wp_ij = -er_wall eps n_i n_j, and the Galerkin system (M + K_{L^2}) wp = M f
// over the periodic-merged nodes, solved for the five components at once by
// Jacobi-preconditioned CG in FP64 (warm start from the previous step).
//
// The solver is one persistent cooperative kernel: the grid walks the matrix
// rows, and the reductions of each iteration go through per-block partials
// summed in block order by every block (deterministic), separated by a grid
// barrier whose spin is bounded (status ST_BARRIER on expiry).
#include <cooperative_groups.h>

#include "pdf_internal.cuh"

namespace {

constexpr int NC = 5;
constexpr int FE_THREADS = 256;

__global__ void k_fe_rhs(int nn, const double* __restrict__ nR, const double* __restrict__ ngrad,
                         const double* __restrict__ nke, const double* __restrict__ nmean,
                         const unsigned char* __restrict__ is_wall, const double* __restrict__ wn, pdf_params p,
                         double* f, double* g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const double* R = nR + 6 * (size_t)i;
    const double* gr = ngrad + 4 * (size_t)i;
    const double k = nke[2 * i];
    double om = nmean[4 * i + 3];
    om = om > p.floor_omega ? om : p.floor_omega;
    const double gg[2][2] = {{gr[0], gr[1]}, {gr[2], gr[3]}};
    const double Rm[2][2] = {{R[0], R[3]}, {R[3], R[1]}};
    const double tr = R[0] + R[1] + R[2];
    double b[2][2] = {{0, 0}, {0, 0}};
    if (tr > 0.0)
        for (int a = 0; a < 2; ++a)
            for (int c = 0; c < 2; ++c) b[a][c] = Rm[a][c] / tr - (a == c ? 1.0 / 3.0 : 0.0);
    const double det = R[2] * (R[0] * R[1] - R[3] * R[3]);
    const double tk = 2.0 / 3.0 * k;
    double Av = p.Cv * det / (tk * tk * tk);
    Av = Av < 1.0 ? Av : 1.0;
    const double iso = 0.5 * (1.0 - p.C1) * k * om;
    int q = 0;
    for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) {
            double t = (p.C2 * Av + p.gamma5 / 3.0) * gg[a][c] - p.gamma5 / 3.0 * gg[c][a];
            for (int m = 0; m < 2; ++m) t += p.gamma5 * b[a][m] * gg[m][c];
            for (int l = 0; l < 2; ++l) t -= p.gamma5 * b[a][l] * gg[c][l];
            f[NC * (size_t)i + q++] = (a == c ? iso : 0.0) + (p.rotta ? 0.0 : k * t);
        }
    f[NC * (size_t)i + 4] = iso;
    if (is_wall[i]) {
        const double eps = nke[2 * i + 1], nx = wn[2 * i], ny = wn[2 * i + 1];
        g[NC * (size_t)i + 0] = -p.er_wall * eps * nx * nx;
        g[NC * (size_t)i + 1] = -p.er_wall * eps * nx * ny;
        g[NC * (size_t)i + 2] = -p.er_wall * eps * ny * nx;
        g[NC * (size_t)i + 3] = -p.er_wall * eps * ny * ny;
        g[NC * (size_t)i + 4] = 0.0;
    }
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
    double* x;     // [nn][NC] node solution: warm start in, result out (canonical rows)
    double* zg;    // [nn][NC] preconditioned residual, shared between blocks for the SpMV
    double* part;  // [gridDim][PART_W]
    unsigned* bar;
    int* iters;
    int* status;
    double tol;
    int maxit;
};

constexpr int BS = 128;        // rows per block = size of the block-Jacobi diagonal blocks
constexpr int PART_W = 4 * NC; // partial sums per block: 3 NC in phase A, NC in phase B

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// grid-wide barrier of a cooperative launch: arrival by a release atomic,
// the last block bumps the generation word, the others poll it with acquire
// loads; the wait is bounded (ST_BARRIER, then the block proceeds)
__device__ void grid_barrier(const CGArgs& a) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g0 = ld_acquire(a.bar + 1);
        asm volatile("fence.acq_rel.gpu;" ::: "memory");  // the block's writes before the arrival
        unsigned arrived;
        asm volatile("atom.add.release.gpu.global.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(a.bar) : "memory");
        if (arrived + 1u == gridDim.x) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], 0;" ::"l"(a.bar) : "memory");
            asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(a.bar + 1) : "memory");
        } else {
            long long spins = 0;
            while (ld_acquire(a.bar + 1) == g0) {
                if (++spins > (1ll << 22)) {  // ~1-2 s of polling
                    set_status(a.status, ST_BARRIER);
                    break;
                }
            }
        }
        asm volatile("fence.acq_rel.gpu;" ::: "memory");  // other blocks' writes before the reads
    }
    __syncthreads();
}

// block sums of NV per-thread values into part[block][slot..slot+NV)
template <int NV>
__device__ void block_partial(const CGArgs& a, double (&v)[NV], int slot) {
    __shared__ double red[BS / 32][PART_W];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
    if (lane == 0)
#pragma unroll
        for (int q = 0; q < NV; ++q) red[wid][q] = v[q];
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < BS / 32; ++w) s += red[w][threadIdx.x];
        a.part[(size_t)blockIdx.x * PART_W + slot + threadIdx.x] = s;
    }
    __syncthreads();
}

// after a barrier: the sums over all blocks; value q is reduced by warp q % 4
// in a fixed lane-strided order and shuffle tree (the same in every block)
__device__ void grid_sum(const CGArgs& a, int slot, int nv, double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = wid; q < nv; q += BS / 32) {
        double s = 0.0;
        for (int bl = lane; bl < (int)gridDim.x; bl += 32) s += a.part[(size_t)bl * PART_W + slot + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[q] = s;
    }
    __syncthreads();
}

__device__ __forceinline__ void spmv_row(const CGArgs& a, int i, const double* __restrict__ v, double (&s)[NC]) {
#pragma unroll
    for (int k = 0; k < NC; ++k) s[k] = 0.0;
    for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
        const int j = a.colidx[q];
        const double A = a.aval[q];
#pragma unroll
        for (int k = 0; k < NC; ++k) s[k] += A * v[NC * (size_t)j + k];
    }
}

// z = Ainv_b r for the block's rows (FP32 dense product in shared memory)
__device__ __forceinline__ void block_precondition(const float* __restrict__ inv, float (*rv)[NC], int t,
                                                   const double (&r)[NC], double (&z)[NC]) {
#pragma unroll
    for (int k = 0; k < NC; ++k) rv[t][k] = (float)r[k];
    __syncthreads();
    float acc[NC] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 4
    for (int j = 0; j < BS; ++j) {
        const float m = inv[j * BS + t];
#pragma unroll
        for (int k = 0; k < NC; ++k) acc[k] += m * rv[j][k];
    }
#pragma unroll
    for (int k = 0; k < NC; ++k) z[k] = (double)acc[k];
    __syncthreads();
}

// Flexible (Polak-Ribiere) preconditioned CG in FP64 for the NC right-hand
// sides, block-Jacobi preconditioner with FP32 explicit inverses of the 128 x
// 128 diagonal blocks (one block of rows per thread block, inverted in shared
// memory by Gauss-Jordan without pivoting: the blocks are SPD). The vectors of
// a row live in the registers of its thread; the product A p follows the
// recurrence A p_{k+1} = A z_{k+1} + beta_k A p_k, so one SpMV (on z) and two
// grid reductions per iteration.
__global__ void __launch_bounds__(BS) k_pcg(const CGArgs a) {
    extern __shared__ float inv[];  // BS*BS, column j at inv[j*BS .. j*BS+BS)
    __shared__ float rv[BS][NC];
    __shared__ double s_a[PART_W];
    __shared__ double s_rz[NC], s_rr[NC], s_bn[NC], s_pap[NC], s_alpha[NC], s_beta[NC];
    __shared__ int s_active[NC];
    const int t = threadIdx.x;
    const int i = blockIdx.x * BS + t;
    const bool have = i < a.nn;
    const bool free_row = have && a.rep[i] == i && !a.is_wall[i];
    // assembly of M + K_{L^2}; b = M f; Dirichlet values
    double b[NC] = {0, 0, 0, 0, 0}, x[NC] = {0, 0, 0, 0, 0};
    if (have) {
        for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
            double s = a.mval[q];
            for (int c = a.kc_off[q]; c < a.kc_off[q + 1]; ++c) {
                const double L = a.eder[9 * (size_t)a.kc_elem[c] + 8];
                s += L * L * a.kc_geo[c];
            }
            a.aval[q] = s;
            const int j = a.colidx[q];
#pragma unroll
            for (int k = 0; k < NC; ++k) b[k] += a.mval[q] * a.f[NC * (size_t)j + k];
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            x[k] = a.is_wall[i] ? a.g[NC * (size_t)i + k] : a.x[NC * (size_t)i + k];
            a.x[NC * (size_t)i + k] = x[k];
        }
    }
    // diagonal block of the free rows (identity elsewhere), column-major
    for (int q = t; q < BS * BS; q += BS) inv[q] = 0.f;
    __syncthreads();
    if (have) {
        if (free_row) {
            for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
                const int j = a.colidx[q], jl = j - blockIdx.x * BS;
                if (jl >= 0 && jl < BS && a.rep[j] == j && !a.is_wall[j]) inv[jl * BS + t] = (float)a.aval[q];
            }
        } else {
            inv[t * BS + t] = 1.f;
        }
    } else {
        inv[t * BS + t] = 1.f;
    }
    __syncthreads();
    for (int k = 0; k < BS; ++k) {  // in-place Gauss-Jordan inverse
        const float fk = inv[k * BS + t];       // a[t][k]
        const float p = inv[k * BS + k];
        __syncthreads();
        {
            const float v = (t == k) ? 1.f : inv[t * BS + k];  // a[k][t]
            inv[t * BS + k] = v / p;
        }
        __syncthreads();
        if (t != k) {
            inv[k * BS + t] = 0.f;
            for (int j = 0; j < BS; ++j) inv[j * BS + t] -= fk * inv[j * BS + k];
        }
        __syncthreads();
    }
    grid_barrier(a);  // all x (warm start + Dirichlet) and matrix rows are in place
    // r = b - A x; z = Ainv r; p = z
    double r[NC], z[NC], p[NC], ap[NC];
    {
        double s[NC], b0[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) { s[k] = 0.0; b0[k] = b[k]; }
        if (free_row) {
            for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
                const int j = a.colidx[q];
                const double A = a.aval[q];
                const bool dj = a.is_wall[j];
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    const double xv = a.x[NC * (size_t)j + k];
                    s[k] += A * xv;
                    if (dj) b0[k] -= A * xv;
                }
            }
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) r[k] = free_row ? b[k] - s[k] : 0.0;
        block_precondition(inv, rv, t, r, z);
        double v[3 * NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            if (!free_row) z[k] = 0.0;
            p[k] = z[k];
            v[k] = r[k] * z[k];
            v[NC + k] = r[k] * r[k];
            v[2 * NC + k] = free_row ? b0[k] * b0[k] : 0.0;
            if (have) a.zg[NC * (size_t)i + k] = z[k];
        }
        block_partial<3 * NC>(a, v, 0);
    }
    grid_barrier(a);
    grid_sum(a, 0, 3 * NC, s_a);
    if (t < NC) {
        s_rz[t] = s_a[t];
        s_rr[t] = s_a[NC + t];
        s_bn[t] = sqrt(s_a[2 * NC + t]);
    }
    {  // A p_0
        double s[NC], v[NC];
        if (free_row) spmv_row(a, i, a.zg, s);
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            ap[k] = free_row ? s[k] : 0.0;
            v[k] = p[k] * ap[k];
        }
        block_partial<NC>(a, v, 3 * NC);
    }
    grid_barrier(a);
    grid_sum(a, 3 * NC, NC, s_pap);
    int it = 0;
    for (;; ++it) {
        if (t < NC) {
            s_active[t] = (s_bn[t] > 0.0) && (sqrt(s_rr[t]) > a.tol * s_bn[t]);
            s_alpha[t] = s_active[t] ? s_rz[t] / s_pap[t] : 0.0;
        }
        __syncthreads();
        bool any = false;
#pragma unroll
        for (int k = 0; k < NC; ++k) any |= s_active[k] != 0;
        if (!any) break;
        if (it >= a.maxit) {
            if (blockIdx.x == 0 && t == 0) set_status(a.status, ST_CG);
            break;
        }
        // phase A: x += alpha p, r -= alpha Ap, z = Ainv r
        {
            double rold[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                rold[k] = r[k];
                if (s_active[k]) {
                    const double alpha = s_alpha[k];
                    x[k] += alpha * p[k];
                    r[k] -= alpha * ap[k];
                }
            }
            double zn[NC];
            block_precondition(inv, rv, t, r, zn);
            double v[3 * NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                if (!free_row) zn[k] = 0.0;
                if (s_active[k]) z[k] = zn[k];
                v[k] = r[k] * z[k];
                v[NC + k] = rold[k] * z[k];
                v[2 * NC + k] = r[k] * r[k];
                if (have) a.zg[NC * (size_t)i + k] = z[k];
            }
            block_partial<3 * NC>(a, v, 0);
        }
        grid_barrier(a);
        grid_sum(a, 0, 3 * NC, s_a);
        if (t < NC) s_beta[t] = s_active[t] ? (s_a[t] - s_a[NC + t]) / s_rz[t] : 0.0;
        __syncthreads();
        // phase B: p = z + beta p (Polak-Ribiere); A p = A z + beta A p
        {
            double s[NC], v[NC];
            if (free_row) spmv_row(a, i, a.zg, s);
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                v[k] = 0.0;
                if (s_active[k]) {
                    const double beta = s_beta[k];
                    p[k] = z[k] + beta * p[k];
                    ap[k] = (free_row ? s[k] : 0.0) + beta * ap[k];
                }
                v[k] = p[k] * ap[k];
            }
            block_partial<NC>(a, v, 3 * NC);
        }
        grid_barrier(a);
        if (t < NC && s_active[t]) {
            s_rz[t] = s_a[t];
            s_rr[t] = s_a[2 * NC + t];
        }
        grid_sum(a, 3 * NC, NC, s_pap);
    }
    if (free_row)
#pragma unroll
        for (int k = 0; k < NC; ++k) a.x[NC * (size_t)i + k] = x[k];
    if (blockIdx.x == 0 && t == 0) *a.iters = it;
}

__global__ void k_fe_copy_out(int nn, const int* __restrict__ rep, const double* __restrict__ x, double* nwp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    const int r = rep[i];
#pragma unroll
    for (int k = 0; k < NC; ++k) nwp[NC * (size_t)i + k] = x[NC * (size_t)r + k];
}

}  // namespace

int launch_elliptic(pdf_ctx* c) {
    const int nn = c->m.nn;
    timing_begin(c, PDF_K_ELLIPTIC);
    k_fe_rhs<<<(nn + 127) / 128, 128, 0, c->s>>>(nn, c->nR, c->ngrad, c->nke, c->nmean, c->m.is_wall, c->m.wn,
                                                c->p, c->fe_f, c->fe_g);
    PDF_CUDA(c, cudaGetLastError());
    const int blocks = (nn + BS - 1) / BS;
    const size_t smem = sizeof(float) * BS * BS;
    if (c->fe_blocks == 0) {
        PDF_CUDA(c, cudaFuncSetAttribute(k_pcg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        PDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg, BS, smem));
        if (per_sm * c->num_sms < blocks)
            return fail(c, PDF_ERR_CAPACITY, "elliptic solver: mesh too large for one resident grid");
        if ((size_t)blocks * PART_W > (size_t)15 * 4096)
            return fail(c, PDF_ERR_CAPACITY, "elliptic solver: partial-sum buffer too small");
        c->fe_blocks = blocks;
    }
    CGArgs a;
    a.nn = nn;
    a.rowptr = c->m.rowptr; a.colidx = c->m.colidx; a.mval = c->m.mval;
    a.kc_off = c->m.kc_off; a.kc_elem = c->m.kc_elem; a.kc_geo = c->m.kc_geo;
    a.eder = c->eder; a.rep = c->m.rep; a.is_wall = c->m.is_wall;
    a.f = c->fe_f; a.g = c->fe_g; a.aval = c->m.aval;
    a.x = c->nwp;  // solution lives in the node array (canonical rows)
    a.zg = c->fe_z;
    a.part = c->fe_part; a.bar = c->fe_bar; a.iters = c->fe_iters; a.status = c->d_status;
    a.tol = c->p.cg_tol; a.maxit = c->p.cg_maxit;
    void* args[] = {&a};
    PDF_CUDA(c, cudaLaunchCooperativeKernel((void*)k_pcg, dim3(blocks), dim3(BS), args, smem, c->s));
    k_fe_copy_out<<<(nn + 127) / 128, 128, 0, c->s>>>(nn, c->m.rep, c->nwp, c->nwp);
    c->launches += 3;
    timing_end(c, PDF_K_ELLIPTIC);
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}
