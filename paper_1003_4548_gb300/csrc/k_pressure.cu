// k_pressure.cu -- mean-pressure projection (pressure = 1).
//
// The paper obtains the mean pressure by a projection scheme it cites but
// does not give; this is a first-principles P1 fractional step after every
// step's moments:
//   sum_e A_e grad N_i . grad N_j p_j = (1/dt) sum_e A_e grad N_i . <U>_e
// over the node classes (periodic partners merged; no mean flux through the
// walls and the top, imposed weakly; p = 0 at the lowest-id canonical node),
// then every particle's in-plane velocity and its element's mean lose
// dt grad p of the element (a uniform shift per element, so the Reynolds
// stresses, the velocity bins and <phi|V> are unchanged).
//
// The stiffness matrix is constant, so everything the preconditioner needs
// is built once: the FP32 inverses of its diagonal blocks of BS consecutive
// (Morton-ordered) rows, and the FP64 inverse of the coarse matrix
// A0 = P^T K P, P the block-wise constant prolongation. Each step one
// cooperative kernel runs a Chronopoulos-Gear CG with the two-level additive
// preconditioner u = Binv r + P A0^-1 P^T r: two grid barriers per
// iteration, the coarse residual of every block carried by recurrence.
#include <cmath>
#include <vector>

#include "coop.cuh"
#include "pdf_internal.cuh"

namespace {

constexpr int PR_W = 8;  // partial sums per block: 0 (r,u), 1 (r,r), 2 (w,u), 3 sum w, 4 (b,b), 5 sum r

// right-hand side at every canonical node i: (1/dt) sum over the elements
// around its class of A_e grad N_i . <U>_e
__global__ void k_pr_rhs(int nn, const int* __restrict__ rep, const int* __restrict__ n2e_off,
                         const int* __restrict__ n2e, const int* __restrict__ tri, const double* __restrict__ area,
                         const double* __restrict__ gradb, const double* __restrict__ emean, double idt,
                         double* __restrict__ b) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    double s = 0.0;
    if (rep[i] == i) {
        for (int q = n2e_off[i]; q < n2e_off[i + 1]; ++q) {
            const int e = n2e[q];
            int k = 0;
            while (k < 2 && rep[tri[3 * e + k]] != i) ++k;
            s += area[e] * (gradb[6 * e + 2 * k] * emean[5 * e + 0] + gradb[6 * e + 2 * k + 1] * emean[5 * e + 1]);
        }
        s *= idt;
    }
    b[i] = s;
}

// node pressure on every class member; element gradient; the element means
// of occupied elements shift by -dt grad p
__global__ void k_pr_grad(int nn, int nt, const int* __restrict__ rep, const double* __restrict__ x,
                          const int* __restrict__ tri, const double* __restrict__ gradb, const int* __restrict__ en,
                          double dt, double* __restrict__ pres, double* __restrict__ egp, double* __restrict__ emean) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nn) pres[t] = x[rep[t]];
    if (t >= nt) return;
    double gx = 0.0, gy = 0.0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double pk = x[rep[tri[3 * t + k]]];
        gx += pk * gradb[6 * t + 2 * k];
        gy += pk * gradb[6 * t + 2 * k + 1];
    }
    egp[2 * t] = gx;
    egp[2 * t + 1] = gy;
    if (en[t] > 0) {
        emean[5 * t + 0] -= dt * gx;
        emean[5 * t + 1] -= dt * gy;
    }
}

// U_p -= dt grad p of the host element: one warp per element over its
// particles (element-sorted state)
template <typename T>
__global__ void k_pr_correct(int nt, const int* __restrict__ off, const double* __restrict__ egp, double dt,
                             T* __restrict__ u, T* __restrict__ v) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int e = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); e < nt; e += nw) {
        const T du = (T)(dt * egp[2 * e]), dv = (T)(dt * egp[2 * e + 1]);
        const int s1 = off[e + 1];
        for (int q = off[e] + lane; q < s1; q += 32) {
            u[q] -= du;
            v[q] -= dv;
        }
    }
}

// FP32 inverse of the diagonal block of K over rows blk*BS .. blk*BS+BS-1
// (free rows and columns; identity elsewhere) by Gauss-Jordan without
// pivoting (the block is SPD); stored column-major with stride BS + 4:
// out[j*(BS+4) + t] = Binv[t][j]. One block of BS threads per diagonal block.
template <int BS>
__global__ void __launch_bounds__(BS) k_pr_blockinv(int nn, const int* __restrict__ rowptr,
                                                    const int* __restrict__ colidx, const double* __restrict__ val,
                                                    const int* __restrict__ rep, const unsigned char* __restrict__ pin,
                                                    float* __restrict__ out) {
    extern __shared__ float inv[];
    const int t = threadIdx.x, i = blockIdx.x * BS + t;
    const bool fr = i < nn && rep[i] == i && !pin[i];
    for (int q = t; q < BS * (BS + 4); q += BS) inv[q] = 0.f;
    __syncthreads();
    if (fr) {
        for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            const int j = colidx[q], jl = j - blockIdx.x * BS;
            if (jl >= 0 && jl < BS && rep[j] == j && !pin[j]) inv[jl * (BS + 4) + t] = (float)val[q];
        }
    } else {
        inv[t * (BS + 4) + t] = 1.f;
    }
    __syncthreads();
    for (int k = 0; k < BS; ++k) {
        const float fk = inv[k * (BS + 4) + t];  // a[t][k]
        const float p = inv[k * (BS + 4) + k];
        __syncthreads();
        const float v = (t == k) ? 1.f : inv[t * (BS + 4) + k];  // a[k][t]
        inv[t * (BS + 4) + k] = v / p;
        __syncthreads();
        if (t != k) {
            for (int j = 0; j < BS; ++j) {
                if (j == k) inv[k * (BS + 4) + t] = -fk * inv[k * (BS + 4) + k];
                else inv[j * (BS + 4) + t] -= fk * inv[j * (BS + 4) + k];
            }
        }
        __syncthreads();
    }
    // symmetrise (the same rounded average in both triangles), so that the
    // preconditioner is an exactly symmetric map
    float* dst = out + (size_t)blockIdx.x * BS * (BS + 4);
    for (int j = 0; j < BS; ++j) {
        const float sym = 0.5f * (inv[j * (BS + 4) + t] + inv[t * (BS + 4) + j]);
        dst[j * (BS + 4) + t] = sym;
    }
}

struct PrArgs {
    int nn, nb;
    const int* __restrict__ rowptr;
    const int* __restrict__ colidx;
    const double* __restrict__ val;
    const int* __restrict__ rep;
    const unsigned char* __restrict__ pin;
    const double* __restrict__ b;       // [nn] right-hand side (canonical rows)
    const float* __restrict__ binv;     // [nb][BS][BS + 4] block inverses
    const double* __restrict__ a0inv;   // [nb][nb] coarse inverse
    double* x;                          // [nn] warm start in, solution out (canonical rows)
    double* zg;                         // [nn] preconditioned residual, read by the SpMV
    double* part;                       // [nb][PR_W]
    unsigned* bar;
    int* iters;
    int* status;
    double tol;
    int maxit;
    long long spin_max;  // polls of a grid barrier before it gives up (ST_BARRIER)
};

constexpr int RMAX = 12;  // matrix entries per row staged in shared memory (the rest read from global)

template <int BS>
constexpr size_t pcg_p_smem(int nb) {
    return sizeof(float) * (size_t)(BS * (BS + 4) + BS) + sizeof(double) * (size_t)(3 * nb) +
           (sizeof(double) + sizeof(int)) * (size_t)(RMAX * BS);
}

// block sums of NV values published to this block's partial slots (fixed
// order: warp shuffle tree, then the warps in order)
template <int BS, int NV>
__device__ __forceinline__ void publish(const PrArgs& a, double (&v)[NV], const int (&slot)[NV], double* red) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {  // the NV trees interleaved
#pragma unroll
        for (int k = 0; k < NV; ++k) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) red[wid * NV + k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < NV) {
        double s = 0.0;
        for (int w = 0; w < BS / 32; ++w) s += red[w * NV + threadIdx.x];
        int sl = slot[0];
#pragma unroll
        for (int k = 1; k < NV; ++k) sl = (int)threadIdx.x == k ? slot[k] : sl;
        a.part[(size_t)blockIdx.x * PR_W + sl] = s;
    }
}

// after a grid barrier: sum over all blocks of NV slots (warp k: slot k, a
// fixed lane-strided order and shuffle tree, the same in every block)
template <int NV>
__device__ __forceinline__ void gather(const PrArgs& a, const int (&slot)[NV], double* out) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (wid < NV) {
        int sl = slot[0];
#pragma unroll
        for (int k = 1; k < NV; ++k) sl = wid == k ? slot[k] : sl;
        // the loads of a chunk are issued together (one L2 round trip per
        // chunk of 8 x 32 blocks), then summed in order
        double s = 0.0;
        for (int c0 = 0; c0 < a.nb; c0 += 8 * 32) {
            double v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const int c = c0 + 32 * k + lane;
                v[k] = c < a.nb ? a.part[(size_t)c * PR_W + sl] : 0.0;
            }
#pragma unroll
            for (int k = 0; k < 8; ++k) s += v[k];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) out[wid] = s;
    }
    __syncthreads();
}

// Two-level preconditioner of this block's rows, u = Binv r + (A0^-1 rc)_blk,
// rc = P^T r the coarse residual held (for every block) in shared memory.
// Binv is symmetrised at set-up, so the preconditioner is a fixed SPD map.
template <int BS>
__device__ __forceinline__ double precondition(const PrArgs& a, const float* inv, float* rv, const double* a0row,
                                               const double* rc, double* z0s, double r, bool fr) {
    const int t = threadIdx.x, lane = t & 31;
    rv[t] = (float)r;
    if (t < 32) {
        double s = 0.0, s1 = 0.0;  // two chains (the FP64 pipe's latency is long on GB300)
        int c = lane;
        for (; c + 32 < a.nb; c += 64) {
            s = fma(a0row[c], rc[c], s);
            s1 = fma(a0row[c + 32], rc[c + 32], s1);
        }
        if (c < a.nb) s = fma(a0row[c], rc[c], s);
        s += s1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) *z0s = s;
    }
    __syncthreads();
    float z0 = 0.f, z1 = 0.f, z2 = 0.f, z3 = 0.f;  // four chains, summed in a fixed order
#pragma unroll 4
    for (int k = 0; k < BS; k += 4) {
        z0 = fmaf(inv[k * (BS + 4) + t], rv[k], z0);
        z1 = fmaf(inv[(k + 1) * (BS + 4) + t], rv[k + 1], z1);
        z2 = fmaf(inv[(k + 2) * (BS + 4) + t], rv[k + 2], z2);
        z3 = fmaf(inv[(k + 3) * (BS + 4) + t], rv[k + 3], z3);
    }
    const float z = (z0 + z1) + (z2 + z3);
    const double out = fr ? (double)z + *z0s : 0.0;
    __syncthreads();  // rv and z0s are rewritten by the next call
    return out;
}

// row i of the stiffness matrix times the vector v (entries beyond RMAX from
// global memory)
__device__ __forceinline__ double row_times(const PrArgs& a, const int* scol, const double* sval, int BSn, int t,
                                            int i, int len, const double* v) {
    double s = 0.0, s1 = 0.0;  // two chains (the FP64 pipe's latency is long on GB300)
    const int m = len < RMAX ? len : RMAX;
    int k = 0;
    for (; k + 1 < m; k += 2) {
        s = fma(sval[k * BSn + t], v[scol[k * BSn + t]], s);
        s1 = fma(sval[(k + 1) * BSn + t], v[scol[(k + 1) * BSn + t]], s1);
    }
    if (k < m) s = fma(sval[k * BSn + t], v[scol[k * BSn + t]], s);
    s += s1;
    if (len > RMAX) {
        const int q0 = a.rowptr[i];
        for (int k = RMAX; k < len; ++k) s += a.val[q0 + k] * v[a.colidx[q0 + k]];
    }
    return s;
}

// Chronopoulos-Gear preconditioned CG (one fused reduction pair per
// iteration, two grid barriers): u = M r, w = A u,
//   gamma = (r, u), delta = (w, u), beta = gamma / gamma_old,
//   alpha = gamma / (delta - beta gamma / alpha_old),
//   p = u + beta p, s = w + beta s, x += alpha p, r -= alpha s.
// The coarse residual P^T r of every block follows the same recurrence from
// the published block sums of w, so the preconditioner needs no barrier of
// its own.
template <int BS>
__global__ void __launch_bounds__(BS) k_pcg_p(const PrArgs a) {
    extern __shared__ __align__(16) unsigned char smraw[];
    float* inv = reinterpret_cast<float*>(smraw);             // BS x (BS + 4)
    float* rv = inv + BS * (BS + 4);                           // BS
    double* a0row = reinterpret_cast<double*>(rv + BS);        // nb
    double* rc = a0row + a.nb;                                 // nb: P^T r
    double* psc = rc + a.nb;                                   // nb: P^T s
    double* sval = psc + a.nb;                                 // RMAX x BS
    int* scol = reinterpret_cast<int*>(sval + RMAX * BS);      // RMAX x BS
    __shared__ double red[(BS / 32) * 3];
    __shared__ double g[4];
    __shared__ double z0s;
    const int t = threadIdx.x, blk = blockIdx.x, i = blk * BS + t;
    const bool have = i < a.nn;
    const bool fr = have && a.rep[i] == i && !a.pin[i];
    int len = 0;
    {  // the block's inverse, coarse row and matrix rows into shared memory
        const float4* src = reinterpret_cast<const float4*>(a.binv + (size_t)blk * BS * (BS + 4));
        float4* dst = reinterpret_cast<float4*>(inv);
        for (int q = t; q < BS * (BS + 4) / 4; q += BS) dst[q] = src[q];
        for (int c = t; c < a.nb; c += BS) a0row[c] = a.a0inv[(size_t)blk * a.nb + c];
        if (fr) {
            const int q0 = a.rowptr[i];
            len = a.rowptr[i + 1] - q0;
            for (int k = 0; k < len && k < RMAX; ++k) {
                sval[k * BS + t] = a.val[q0 + k];
                scol[k * BS + t] = a.colidx[q0 + k];
            }
        }
    }
    unsigned gen = t == 0 ? coop_generation(a.bar) : 0u;  // before this launch's first barrier
    const double bi = fr ? a.b[i] : 0.0;
    double x = fr ? a.x[i] : 0.0;
    if (have && a.pin[i]) a.x[i] = 0.0;
    grid_barrier_gen(a.bar, a.status, gen, a.spin_max);  // warm start and the pinned zero in place
    double r = fr ? bi - row_times(a, scol, sval, BS, t, i, len, a.x) : 0.0;
    {
        double v[2] = {r, bi * bi};
        const int sl[2] = {5, 4};
        publish<BS, 2>(a, v, sl, red);
    }
    grid_barrier_gen(a.bar, a.status, gen, a.spin_max);
    {
        const int sl[1] = {4};
        gather<1>(a, sl, g);
    }
    const double bn = sqrt(g[0]);
    if (!(bn > 0.0)) {  // zero right-hand side: p = 0
        if (fr) a.x[i] = 0.0;
        if (blk == 0 && t == 0) *a.iters = 0;
        return;
    }
    for (int c = t; c < a.nb; c += BS) {
        rc[c] = a.part[(size_t)c * PR_W + 5];
        psc[c] = 0.0;
    }
    __syncthreads();
    double p = 0.0, s = 0.0, gamma_old = 1.0, alpha_old = 1.0;
    int it = 0;
    for (;; ++it) {
        const double u = precondition<BS>(a, inv, rv, a0row, rc, &z0s, r, fr);
        if (have) a.zg[i] = u;
        {
            double v[2] = {r * u, r * r};
            const int sl[2] = {0, 1};
            publish<BS, 2>(a, v, sl, red);
        }
        grid_barrier_gen(a.bar, a.status, gen, a.spin_max);  // A: u of every row, gamma and (r, r)
        {
            const int sl[2] = {0, 1};
            gather<2>(a, sl, g);
        }
        const double gamma = g[0], rr = g[1];
        if (!(sqrt(rr) > a.tol * bn)) break;
        if (it >= a.maxit) {
            if (blk == 0 && t == 0) set_status(a.status, ST_CG);
            break;
        }
        const double w = fr ? row_times(a, scol, sval, BS, t, i, len, a.zg) : 0.0;
        {
            double v[2] = {w * u, w};
            const int sl[2] = {2, 3};
            publish<BS, 2>(a, v, sl, red);
        }
        grid_barrier_gen(a.bar, a.status, gen, a.spin_max);  // B: delta and the block sums of w
        {
            const int sl[1] = {2};
            gather<1>(a, sl, g);
        }
        const double delta = g[0];
        const double beta = it == 0 ? 0.0 : gamma / gamma_old;
        const double alpha = it == 0 ? gamma / delta : gamma / (delta - beta * gamma / alpha_old);
        p = u + beta * p;
        s = w + beta * s;
        x += alpha * p;
        r -= alpha * s;
        for (int c = t; c < a.nb; c += BS) {
            psc[c] = a.part[(size_t)c * PR_W + 3] + beta * psc[c];
            rc[c] -= alpha * psc[c];
        }
        gamma_old = gamma;
        alpha_old = alpha;
        __syncthreads();
    }
    if (fr) a.x[i] = x;
    if (blk == 0 && t == 0) *a.iters = it;
}

template <int BS>
int try_grid(pdf_ctx* c, int& blocks) {
    const int nb = (c->m.nn + BS - 1) / BS;
    const size_t smem = pcg_p_smem<BS>(nb);
    if (cudaFuncSetAttribute(k_pcg_p<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_p<BS>, BS, smem) != cudaSuccess) return 0;
    if (nb > per_sm * c->num_sms || nb > 1024 || (size_t)nb * PR_W > (size_t)15 * 4096) return 0;
    blocks = nb;
    return BS;
}

// FP64 inverse of an SPD matrix by Cholesky (row-major n x n, in place)
bool spd_inverse(std::vector<double>& A, int n) {
    std::vector<double> L(A);
    for (int j = 0; j < n; ++j) {
        double d = L[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) d -= L[(size_t)j * n + k] * L[(size_t)j * n + k];
        if (!(d > 0.0)) return false;
        d = std::sqrt(d);
        L[(size_t)j * n + j] = d;
        for (int r = j + 1; r < n; ++r) {
            double s = L[(size_t)r * n + j];
            for (int k = 0; k < j; ++k) s -= L[(size_t)r * n + k] * L[(size_t)j * n + k];
            L[(size_t)r * n + j] = s / d;
        }
    }
    std::vector<double> y(n);
    for (int col = 0; col < n; ++col) {  // solve L L^T x = e_col
        for (int r = 0; r < n; ++r) {
            double s = r == col ? 1.0 : 0.0;
            for (int k = 0; k < r; ++k) s -= L[(size_t)r * n + k] * y[k];
            y[r] = s / L[(size_t)r * n + r];
        }
        for (int r = n - 1; r >= 0; --r) {
            double s = y[r];
            for (int k = r + 1; k < n; ++k) s -= L[(size_t)k * n + r] * A[(size_t)k * n + col];
            A[(size_t)r * n + col] = s / L[(size_t)r * n + r];
        }
    }
    return true;
}

}  // namespace

// Once per context: the grid (rows per block), the FP32 block inverses and the
// FP64 coarse inverse of the projection's preconditioner.
int prepare_pressure(pdf_ctx* c) {
    const int nn = c->m.nn;
    int blocks = 0;
    int bs = try_grid<192>(c, blocks);
    if (!bs) bs = try_grid<160>(c, blocks);
    if (!bs) bs = try_grid<128>(c, blocks);
    if (!bs) return fail(c, PDF_ERR_CAPACITY, "pressure projection: mesh too large for one resident grid");
    c->pr_bs = bs;
    c->pr_blocks = blocks;
    // coarse matrix A0 = P^T K P over the free rows, on the host
    const int nnz = c->m.nnz;
    std::vector<int> rowptr(nn + 1), colidx(nnz), rep(nn);
    std::vector<double> val(nnz);
    std::vector<unsigned char> pin(nn);
    PDF_CUDA(c, cudaMemcpy(rowptr.data(), c->m.rowptr, sizeof(int) * (nn + 1), cudaMemcpyDeviceToHost));
    PDF_CUDA(c, cudaMemcpy(colidx.data(), c->m.colidx, sizeof(int) * nnz, cudaMemcpyDeviceToHost));
    PDF_CUDA(c, cudaMemcpy(val.data(), c->m.pval, sizeof(double) * nnz, cudaMemcpyDeviceToHost));
    PDF_CUDA(c, cudaMemcpy(rep.data(), c->m.rep, sizeof(int) * nn, cudaMemcpyDeviceToHost));
    PDF_CUDA(c, cudaMemcpy(pin.data(), c->m.pin, nn, cudaMemcpyDeviceToHost));
    const int nb = blocks;
    std::vector<double> A0((size_t)nb * nb, 0.0);
    std::vector<int> nfree(nb, 0);
    for (int i = 0; i < nn; ++i) {
        if (rep[i] != i || pin[i]) continue;
        ++nfree[i / bs];
        for (int q = rowptr[i]; q < rowptr[i + 1]; ++q) {
            const int j = colidx[q];
            if (rep[j] != j || pin[j]) continue;
            A0[(size_t)(i / bs) * nb + j / bs] += val[q];
        }
    }
    for (int b = 0; b < nb; ++b)
        if (nfree[b] == 0) A0[(size_t)b * nb + b] = 1.0;  // a block without free rows is decoupled
    if (!spd_inverse(A0, nb)) return fail(c, PDF_ERR_CG_NOCONV, "pressure projection: coarse matrix not SPD");
    PDF_CUDA(c, cudaMalloc(&c->pr_a0inv, sizeof(double) * A0.size()));
    PDF_CUDA(c, cudaMemcpy(c->pr_a0inv, A0.data(), sizeof(double) * A0.size(), cudaMemcpyHostToDevice));
    const size_t nbinv = (size_t)nb * bs * (bs + 4);
    PDF_CUDA(c, cudaMalloc(&c->pr_binv, sizeof(float) * nbinv));
    const size_t sm = sizeof(float) * (size_t)bs * (bs + 4);
    if (bs == 192) {
        PDF_CUDA(c, cudaFuncSetAttribute(k_pr_blockinv<192>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_pr_blockinv<192><<<nb, 192, sm, c->s>>>(nn, c->m.rowptr, c->m.colidx, c->m.pval, c->m.rep, c->m.pin,
                                                 c->pr_binv);
    } else if (bs == 160) {
        PDF_CUDA(c, cudaFuncSetAttribute(k_pr_blockinv<160>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_pr_blockinv<160><<<nb, 160, sm, c->s>>>(nn, c->m.rowptr, c->m.colidx, c->m.pval, c->m.rep, c->m.pin,
                                                 c->pr_binv);
    } else {
        PDF_CUDA(c, cudaFuncSetAttribute(k_pr_blockinv<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        k_pr_blockinv<128><<<nb, 128, sm, c->s>>>(nn, c->m.rowptr, c->m.colidx, c->m.pval, c->m.rep, c->m.pin,
                                                 c->pr_binv);
    }
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

int launch_pressure(pdf_ctx* c, double dt) {
    const int nn = c->m.nn, nt = c->m.nt;
    if (c->pr_blocks == 0) return fail(c, PDF_ERR_STATE, "pressure projection not prepared");
    timing_begin(c, PDF_K_PRESSURE);
    k_pr_rhs<<<(nn + 127) / 128, 128, 0, c->s>>>(nn, c->m.rep, c->m.n2e_off, c->m.n2e, c->m.tri, c->m.area,
                                                c->m.gradb, c->emean, 1.0 / dt, c->pr_b);
    PrArgs a;
    a.nn = nn;
    a.nb = c->pr_blocks;
    a.rowptr = c->m.rowptr; a.colidx = c->m.colidx; a.val = c->m.pval;
    a.rep = c->m.rep; a.pin = c->m.pin;
    a.b = c->pr_b; a.binv = c->pr_binv; a.a0inv = c->pr_a0inv;
    a.x = c->pr_x;  // warm start from the previous step's pressure
    a.zg = c->fe_z;
    a.part = c->fe_part; a.bar = c->fe_bar; a.iters = c->pr_iters; a.status = c->d_status;
    a.spin_max = c->wait_spins > 0 ? c->wait_spins : SPIN_DEFAULT;
    a.tol = c->p.pressure_tol; a.maxit = c->p.cg_maxit;
    // cooperative grids of different contexts never run side by side (a
    // batch orders them in a chain)
    if (c->coop_wait) PDF_CUDA(c, cudaStreamWaitEvent(c->s, c->coop_wait, 0));
    void* args[] = {&a};
    const int bs = c->pr_bs;
    const size_t smem = bs == 192 ? pcg_p_smem<192>(a.nb) : (bs == 160 ? pcg_p_smem<160>(a.nb) : pcg_p_smem<128>(a.nb));
    void* fn = bs == 192 ? (void*)k_pcg_p<192> : (bs == 160 ? (void*)k_pcg_p<160> : (void*)k_pcg_p<128>);
    PDF_CUDA(c, cudaLaunchCooperativeKernel(fn, dim3(a.nb), dim3(bs), args, smem, c->s));
    if (c->coop_done) PDF_CUDA(c, cudaEventRecord(c->coop_done, c->s));
    const int mx = nn > nt ? nn : nt;
    k_pr_grad<<<(mx + 127) / 128, 128, 0, c->s>>>(nn, nt, c->m.rep, c->pr_x, c->m.tri, c->m.gradb, c->en, dt,
                                                 c->pres, c->egp, c->emean);
    const unsigned gw = (unsigned)((nt + 7) / 8);
    if (c->prec == 0)
        k_pr_correct<double><<<gw, 256, 0, c->s>>>(nt, c->off, c->egp, dt, (double*)c->stA[2], (double*)c->stA[3]);
    else
        k_pr_correct<float><<<gw, 256, 0, c->s>>>(nt, c->off, c->egp, dt, (float*)c->stA[2], (float*)c->stA[3]);
    c->launches += 4;
    timing_end(c, PDF_K_PRESSURE);
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}
