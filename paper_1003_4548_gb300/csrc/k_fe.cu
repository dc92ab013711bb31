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
    const int* __restrict__ diag;
    const int* __restrict__ rep;
    const unsigned char* __restrict__ is_wall;
    const double* __restrict__ f;
    const double* __restrict__ g;
    double* aval;
    double *x, *b, *r, *z, *pv, *ap;  // [nn][NC]; x is the node solution (warm start in, result out)
    double* part;                      // [gridDim][3*NC]
    unsigned* bar;
    int* iters;
    int* status;
    double tol;
    int maxit;
};

__device__ void grid_barrier(const CGArgs& a) {
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = a.bar + 1;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(a.bar, 1u) + 1u;
        if (arrived == gridDim.x) {
            a.bar[0] = 0u;
            __threadfence();
            atomicAdd(a.bar + 1, 1u);
        } else {
            long long spins = 0;
            while (*gen == g0) {
                if (++spins > (1ll << 26)) {
                    set_status(a.status, ST_BARRIER);
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
}

// sum of NV per-thread values over the block, written to part[block][slot..]
template <int NV>
__device__ void block_partial(const CGArgs& a, double (&v)[NV], int slot) {
    __shared__ double red[FE_THREADS / 32][3 * NC];
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
        for (int w = 0; w < FE_THREADS / 32; ++w) s += red[w][threadIdx.x];
        a.part[(size_t)blockIdx.x * 3 * NC + slot + threadIdx.x] = s;
    }
    __syncthreads();
}

// after a barrier: every block sums the partials of all blocks; value q is
// reduced by warp q % 8 over a fixed lane-strided order and shuffle tree
// (deterministic, identical in every block)
__device__ void grid_sum(const CGArgs& a, int slot, int nv, double* out_shared) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int q = wid; q < nv; q += FE_THREADS / 32) {
        double s = 0.0;
        for (int bl = lane; bl < (int)gridDim.x; bl += 32) s += a.part[(size_t)bl * 3 * NC + slot + q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out_shared[q] = s;
    }
    __syncthreads();
}

// y = A v on the free canonical rows (0 elsewhere) for the NC components
__device__ __forceinline__ void spmv_row(const CGArgs& a, int i, const double* v, double (&s)[NC]) {
#pragma unroll
    for (int k = 0; k < NC; ++k) s[k] = 0.0;
    for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
        const int j = a.colidx[q];
        const double A = a.aval[q];
#pragma unroll
        for (int k = 0; k < NC; ++k) s[k] += A * v[NC * (size_t)j + k];
    }
}

// Jacobi-preconditioned CG with the product A p carried by the recurrence
// A p_{k+1} = A z_{k+1} + beta_k A p_k, so each iteration needs one SpMV and
// two grid-wide reductions (two barriers).
__global__ void __launch_bounds__(FE_THREADS) k_pcg(const CGArgs a) {
    __shared__ double s_rz[NC], s_rr[NC], s_bn[NC], s_pap[NC], s_new[3 * NC];
    __shared__ int s_active[NC];
    const int stride = gridDim.x * blockDim.x;
    const int t0 = blockIdx.x * blockDim.x + threadIdx.x;
    // assembly of M + K_{L^2}; b = M f; Dirichlet values into x
    for (int i = t0; i < a.nn; i += stride) {
        double bi[NC] = {0, 0, 0, 0, 0};
        for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
            double s = a.mval[q];
            for (int c = a.kc_off[q]; c < a.kc_off[q + 1]; ++c) {
                const double L = a.eder[9 * (size_t)a.kc_elem[c] + 8];
                s += L * L * a.kc_geo[c];
            }
            a.aval[q] = s;
            const int j = a.colidx[q];
#pragma unroll
            for (int k = 0; k < NC; ++k) bi[k] += a.mval[q] * a.f[NC * (size_t)j + k];
        }
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            a.b[NC * (size_t)i + k] = bi[k];
            if (a.is_wall[i]) a.x[NC * (size_t)i + k] = a.g[NC * (size_t)i + k];
        }
    }
    grid_barrier(a);
    // r = b - A x on free canonical rows; z = p = D^-1 r
    {
        double v[3 * NC] = {0};
        for (int i = t0; i < a.nn; i += stride) {
            const bool free_row = a.rep[i] == i && !a.is_wall[i];
            double ri[NC] = {0, 0, 0, 0, 0}, b0[NC] = {0, 0, 0, 0, 0};
            if (free_row) {
#pragma unroll
                for (int k = 0; k < NC; ++k) ri[k] = b0[k] = a.b[NC * (size_t)i + k];
                for (int q = a.rowptr[i]; q < a.rowptr[i + 1]; ++q) {
                    const int j = a.colidx[q];
                    const double A = a.aval[q];
                    const bool dj = a.is_wall[j];
#pragma unroll
                    for (int k = 0; k < NC; ++k) {
                        const double xv = a.x[NC * (size_t)j + k];
                        ri[k] -= A * xv;
                        if (dj) b0[k] -= A * xv;
                    }
                }
            }
            const double dg = (free_row && a.diag[i] >= 0) ? a.aval[a.diag[i]] : 1.0;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                const double zi = free_row ? ri[k] / dg : 0.0;
                a.r[NC * (size_t)i + k] = ri[k];
                a.z[NC * (size_t)i + k] = zi;
                a.pv[NC * (size_t)i + k] = zi;
                v[k] += ri[k] * zi;
                v[NC + k] += ri[k] * ri[k];
                v[2 * NC + k] += b0[k] * b0[k];
            }
        }
        block_partial<3 * NC>(a, v, 0);
    }
    grid_barrier(a);
    grid_sum(a, 0, 3 * NC, s_new);
    if (threadIdx.x < NC) {
        s_rz[threadIdx.x] = s_new[threadIdx.x];
        s_rr[threadIdx.x] = s_new[NC + threadIdx.x];
        s_bn[threadIdx.x] = sqrt(s_new[2 * NC + threadIdx.x]);
    }
    grid_barrier(a);  // all blocks have read the partials before they are reused
    // A p_0 and p_0.A p_0
    {
        double v[NC] = {0, 0, 0, 0, 0};
        for (int i = t0; i < a.nn; i += stride) {
            const bool free_row = a.rep[i] == i && !a.is_wall[i];
            double s[NC];
            spmv_row(a, i, a.pv, s);
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                const double ap = free_row ? s[k] : 0.0;
                a.ap[NC * (size_t)i + k] = ap;
                v[k] += a.pv[NC * (size_t)i + k] * ap;
            }
        }
        block_partial<NC>(a, v, 2 * NC);
    }
    grid_barrier(a);
    grid_sum(a, 2 * NC, NC, s_pap);
    int it = 0;
    for (;; ++it) {
        if (threadIdx.x < NC) {
            const int k = threadIdx.x;
            s_active[k] = (s_bn[k] > 0.0) && (sqrt(s_rr[k]) > a.tol * s_bn[k]);
        }
        __syncthreads();
        bool any = false;
        for (int k = 0; k < NC; ++k) any |= s_active[k] != 0;
        if (!any) break;
        if (it >= a.maxit) {
            if (t0 == 0) set_status(a.status, ST_CG);
            break;
        }
        // x += alpha p, r -= alpha Ap, z = D^-1 r; partial r.z, r.r
        {
            double v[2 * NC] = {0};
            for (int i = t0; i < a.nn; i += stride) {
                const bool free_row = a.rep[i] == i && !a.is_wall[i];
                const double dg = (free_row && a.diag[i] >= 0) ? a.aval[a.diag[i]] : 1.0;
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    if (!s_active[k]) continue;
                    const double alpha = s_rz[k] / s_pap[k];
                    const size_t o = NC * (size_t)i + k;
                    a.x[o] += alpha * a.pv[o];
                    const double rn = a.r[o] - alpha * a.ap[o];
                    a.r[o] = rn;
                    const double zn = free_row ? rn / dg : 0.0;
                    a.z[o] = zn;
                    v[k] += rn * zn;
                    v[NC + k] += rn * rn;
                }
            }
            block_partial<2 * NC>(a, v, 0);
        }
        grid_barrier(a);
        grid_sum(a, 0, 2 * NC, s_new);
        // p = z + beta p; A p = A z + beta A p; partial p.Ap
        {
            double v[NC] = {0, 0, 0, 0, 0};
            for (int i = t0; i < a.nn; i += stride) {
                const bool free_row = a.rep[i] == i && !a.is_wall[i];
                double s[NC];
                spmv_row(a, i, a.z, s);
#pragma unroll
                for (int k = 0; k < NC; ++k) {
                    if (!s_active[k]) continue;
                    const double beta = s_new[k] / s_rz[k];
                    const size_t o = NC * (size_t)i + k;
                    const double pn = a.z[o] + beta * a.pv[o];
                    const double apn = (free_row ? s[k] : 0.0) + beta * a.ap[o];
                    a.pv[o] = pn;
                    a.ap[o] = apn;
                    v[k] += pn * apn;
                }
            }
            block_partial<NC>(a, v, 2 * NC);
        }
        grid_barrier(a);
        if (threadIdx.x < NC && s_active[threadIdx.x]) {
            s_rz[threadIdx.x] = s_new[threadIdx.x];
            s_rr[threadIdx.x] = s_new[NC + threadIdx.x];
        }
        grid_sum(a, 2 * NC, NC, s_pap);
    }
    if (t0 == 0) *a.iters = it;
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
    if (c->fe_blocks == 0) {
        int per_sm = 0;
        PDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg, FE_THREADS, 0));
        if (per_sm < 1) return fail(c, PDF_ERR_CUDA, "elliptic solver cannot be made resident");
        int want = (nn + FE_THREADS - 1) / FE_THREADS;
        const int maxb = per_sm * c->num_sms;
        c->fe_blocks = want < maxb ? (want > 0 ? want : 1) : maxb;
    }
    CGArgs a;
    a.nn = nn;
    a.rowptr = c->m.rowptr; a.colidx = c->m.colidx; a.mval = c->m.mval;
    a.kc_off = c->m.kc_off; a.kc_elem = c->m.kc_elem; a.kc_geo = c->m.kc_geo;
    a.eder = c->eder; a.diag = c->m.diag; a.rep = c->m.rep; a.is_wall = c->m.is_wall;
    a.f = c->fe_f; a.g = c->fe_g; a.aval = c->m.aval;
    a.x = c->nwp;  // solution lives in the node array (canonical rows)
    a.b = c->fe_b; a.r = c->fe_r; a.z = c->fe_z; a.pv = c->fe_p; a.ap = c->fe_ap;
    a.part = c->fe_part; a.bar = c->fe_bar; a.iters = c->fe_iters; a.status = c->d_status;
    a.tol = c->p.cg_tol; a.maxit = c->p.cg_maxit;
    void* args[] = {&a};
    PDF_CUDA(c, cudaLaunchCooperativeKernel((void*)k_pcg, dim3(c->fe_blocks), dim3(FE_THREADS), args, 0, c->s));
    k_fe_copy_out<<<(nn + 127) / 128, 128, 0, c->s>>>(nn, c->m.rep, c->nwp, c->nwp);
    c->launches += 3;
    timing_end(c, PDF_K_ELLIPTIC);
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}
