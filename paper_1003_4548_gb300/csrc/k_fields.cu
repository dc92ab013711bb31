// k_fields.cu -- node averages, derived element fields and the particle packs.
//
// FP64 (a few doubles per node and element; in the compensated-FP32 form the
// roots of t_m and L are taken in FP32):
//  * node statistics: particle-count weighted means over the incident
//    elements (periodic partners merged), k = <u_i u_i>/2 and
//    Eq. dissipation-from-frequency eps = <omega>(k + nu C_T^2 <omega>);
//  * element: P1 gradient of <U>, production P = -<u_i u_j> d<U_i>/dx_j,
//    Eq. frequency_source S_omega, Eq. micromixing-timescale t_m and the
//    length scale of Eq. L at the centroid;
//  * node gradient recovery (area-weighted), with elliptic relaxation the
//    node's FE right-hand side from it, and the element Laplacian;
//  * node pack for the particle kernel: <U>, <V>, <omega>, C0 eps and G_ij
//    (Eq. wall-GandC, or Eqs. Gij and C0 from the elliptic relaxation), and
//    the imposed mean driving force; then the same pack as an affine function
//    on each element (the record the particle kernel interpolates from);
//  * with the Section 4 frequency reflection: <omega u_i> and <omega u_i u_j>
//    (in-plane, fluctuations about the element mean) in the elements around
//    the wall nodes, then their count-weighted means at the wall nodes.
#include "pdf_internal.cuh"

namespace {

// frequency-weighted moments of the listed elements: one warp per element
// over its particles (element-sorted state), FP64 sums, divisor n
template <typename T>
__global__ void k_omw_elem(int nl, const int* __restrict__ list, const int* __restrict__ off,
                           const double* __restrict__ emean, const T* __restrict__ u, const T* __restrict__ v,
                           const T* __restrict__ om, double* __restrict__ eomw) {
    const int lane = threadIdx.x & 31;
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    for (int j = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); j < nl; j += nw) {
        const int e = list[j];
        const int s0 = off[e], s1 = off[e + 1];
        const double mu = emean[5 * e + 0], mv = emean[5 * e + 1];
        double acc[5] = {0, 0, 0, 0, 0};
        for (int q = s0 + lane; q < s1; q += 32) {
            const double du = (double)u[q] - mu, dv = (double)v[q] - mv, o = (double)om[q];
            const double ou = o * du, ov = o * dv;
            acc[0] += ou;
            acc[1] += ov;
            acc[2] += ou * du;
            acc[3] += ou * dv;
            acc[4] += ov * dv;
        }
#pragma unroll
        for (int k = 0; k < 5; ++k)
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) acc[k] += __shfl_xor_sync(0xffffffffu, acc[k], d);
        if (lane < 5) {
            const int n = s1 - s0;
            double a = acc[0];
#pragma unroll
            for (int k = 1; k < 5; ++k) a = lane == k ? acc[k] : a;
            eomw[5 * e + lane] = n > 0 ? a / (double)n : 0.0;
        }
    }
}

// count-weighted means at the listed wall nodes (periodic partners merged);
// a node without particles keeps its previous values
__global__ void k_omw_node(int nl, const int* __restrict__ list, const int* __restrict__ n2e_off,
                           const int* __restrict__ n2e, const int* __restrict__ en,
                           const double* __restrict__ eomw, double* __restrict__ nomw) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= nl) return;
    const int i = list[j];
    double wt = 0.0, W[5] = {0, 0, 0, 0, 0};
    for (int q = n2e_off[i]; q < n2e_off[i + 1]; ++q) {
        const int e = n2e[q];
        const double n = (double)en[e];
        wt += n;
#pragma unroll
        for (int k = 0; k < 5; ++k) W[k] += n * eomw[5 * e + k];
    }
    if (wt <= 0.0) return;
    const double iw = 1.0 / wt;
#pragma unroll
    for (int k = 0; k < 5; ++k) nomw[5 * i + k] = W[k] * iw;
}

__global__ void k_node_stats(int nn, const int* __restrict__ n2e_off, const int* __restrict__ n2e,
                             const int* __restrict__ en, const double* __restrict__ emean,
                             const double* __restrict__ eR, const double* __restrict__ epsivar,
                             pdf_params p, double* nwt, double* nmean, double* nR, double* npsivar,
                             double* nke) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    double wt = 0.0, m[4] = {0, 0, 0, 0}, R[6] = {0, 0, 0, 0, 0, 0}, pv = 0.0;
    const int q1 = n2e_off[i + 1];
    for (int q0 = n2e_off[i]; q0 < q1; q0 += 4) {
        // four elements at a time: their index loads, then their data loads,
        // are issued together (latency bounds this kernel); past the node's
        // last element the terms are zeros, so the sums equal the plain loop's
        int e4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) e4[k] = q0 + k < q1 ? n2e[q0 + k] : -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = e4[k];
            const bool in = e >= 0;
            const double n = in ? (double)en[e] : 0.0;
            wt += n;
            m[0] += n * (in ? emean[5 * e + 0] : 0.0);
            m[1] += n * (in ? emean[5 * e + 1] : 0.0);
            m[2] += n * (in ? emean[5 * e + 3] : 0.0);
            m[3] += n * (in ? emean[5 * e + 4] : 0.0);
#pragma unroll
            for (int j = 0; j < 6; ++j) R[j] += n * (in ? eR[6 * e + j] : 0.0);
            pv += n * (in ? epsivar[e] : 0.0);
        }
    }
    nwt[i] = wt;
    if (wt <= 0.0) return;  // keeps the previous node values
    const double iw = 1.0 / wt;  // one FP64 division (the FP64 pipe is narrow on GB300)
#pragma unroll
    for (int k = 0; k < 4; ++k) nmean[4 * i + k] = m[k] * iw;
#pragma unroll
    for (int k = 0; k < 6; ++k) nR[6 * i + k] = R[k] * iw;
    npsivar[i] = pv * iw;
    double kk = 0.5 * (nR[6 * i] + nR[6 * i + 1] + nR[6 * i + 2]);
    double Om = nmean[4 * i + 3];
    Om = Om > p.floor_omega ? Om : p.floor_omega;
    kk = kk > p.floor_k ? kk : p.floor_k;
    const double eps = Om * (kk + p.nu * p.CT * p.CT * Om);
    nke[2 * i] = kk;
    nke[2 * i + 1] = eps > p.floor_eps ? eps : p.floor_eps;
}

template <typename T>
__global__ void k_elem_derived(int nt, const int* __restrict__ tri, const double* __restrict__ gradb,
                               const double* __restrict__ cent, const double* __restrict__ nmean,
                               const double* __restrict__ nR, const double* __restrict__ nke, pdf_params p,
                               int fast, double* eder, T* epack) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt) return;
    double Ux = 0, Uy = 0, Vx = 0, Vy = 0, kc = 0, ec = 0, Uc = 0, Vc = 0;
    double Rc[6] = {0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int a = tri[3 * e + k];
        const double gx = gradb[6 * e + 2 * k], gy = gradb[6 * e + 2 * k + 1];
        Ux += nmean[4 * a] * gx; Uy += nmean[4 * a] * gy;
        Vx += nmean[4 * a + 1] * gx; Vy += nmean[4 * a + 1] * gy;
        kc += nke[2 * a]; ec += nke[2 * a + 1];
        Uc += nmean[4 * a]; Vc += nmean[4 * a + 1];
#pragma unroll
        for (int q = 0; q < 6; ++q) Rc[q] += nR[6 * a + q];
    }
    // centroid values: one multiply by 1/3 instead of a division per term
    const double third = 1.0 / 3.0;
    kc *= third; ec *= third; Uc *= third; Vc *= third;
#pragma unroll
    for (int q = 0; q < 6; ++q) Rc[q] *= third;
    double* d = eder + 9 * (size_t)e;
    d[0] = Ux; d[1] = Uy; d[2] = Vx; d[3] = Vy;
    const double P = -(Rc[0] * Ux + Rc[3] * Uy + Rc[3] * Vx + Rc[1] * Vy);
    const double iec = 1.0 / ec;
    d[6] = p.Comega2 - p.Comega1 * P * iec;
    double dx = cent[2 * e] - p.x0;
    dx -= p.period * floor(dx * (1.0 / p.period) + 0.5);
    const double dy = cent[2 * e + 1] - p.y0;
    const double Cxi = 1.0 + 1.3 * 1.0;  // C_xi = 1 + 1.3 n_i n_i with a unit normal
    const double t2a = kc * iec;
    if (fast) {
        // compensated-FP32 form: the roots of the mixing time scale and of
        // L in FP32 (relative error below 3e-7, inside that form's
        // statistical tolerance; GB300's FP64 pipe is narrow)
        const float iecf = (float)iec, kcf = (float)kc;
        const float Ucn = sqrtf((float)(Uc * Uc + Vc * Vc));
        const float dist = hypotf((float)dx, (float)dy);
        float t1 = (float)p.Cs * cbrtf((float)(p.r0 * p.r0 * iec));
        t1 += (Ucn > 0.f) ? (float)p.Ct * dist / Ucn : INFINITY;
        const float t2b = (float)p.CT * sqrtf((float)(p.nu * iec));
        const float t2 = fmaxf((float)t2a, t2b);
        d[7] = (double)(t1 < t2 ? t1 : t2);
        const float La = (float)Cxi * kcf * sqrtf(kcf) * iecf;
        const float Lb = (float)p.Ceta * sqrtf(sqrtf((float)(p.nu * p.nu * p.nu * iec)));
        d[8] = p.CL * (double)fmaxf(La, Lb);
    } else {
        const double Ucn = sqrt(Uc * Uc + Vc * Vc);
        const double dist = hypot(dx, dy);
        double t1 = p.Cs * cbrt(p.r0 * p.r0 * iec);
        t1 += (Ucn > 0.0) ? p.Ct * dist / Ucn : HUGE_VAL;
        const double t2b = p.CT * sqrt(p.nu * iec);
        const double t2 = t2a > t2b ? t2a : t2b;
        d[7] = t1 < t2 ? t1 : t2;
        const double La = Cxi * kc * sqrt(kc) * iec, Lb = p.Ceta * sqrt(sqrt(p.nu * p.nu * p.nu * iec));
        d[8] = p.CL * (La > Lb ? La : Lb);
    }
    T* ep = epack + (size_t)ELEM_PACK_W * e;
    ep[0] = (T)Ux; ep[1] = (T)Uy; ep[2] = (T)Vx; ep[3] = (T)Vy;
    ep[6] = (T)d[6]; ep[7] = (T)d[7];
}

// right-hand side of Eq. elliptic-relaxation at node i (the source f of the
// five components wp11, wp12, wp21, wp22, wp33 with Eq. H: the isotropic part
// and, unless the Rotta variant of Section 4 drops it, the H_ijkl term from
// the node's gradient gr), the Dirichlet value wp_ij = -er_wall eps n_i n_j at
// a wall node (the resolved-wall reading), and in the lagged FE mode the
// proposal (the previous solution at the free rows, the Dirichlet values at
// the walls)
struct RhsArgs {
    const double* __restrict__ nR;
    const double* __restrict__ nke;
    const double* __restrict__ nmean;
    const unsigned char* __restrict__ is_wall;
    const double* __restrict__ wn;
    double* f;     // NULL: no elliptic relaxation
    double* g;
    const double* __restrict__ prev;
    double* __restrict__ prop;  // NULL unless the lagged FE mode
};

__device__ __forceinline__ void fe_rhs_node(int i, const double (&gr)[4], const RhsArgs& r, const pdf_params& p) {
    constexpr int NC = 5;
    const double* R = r.nR + 6 * (size_t)i;
    const double k = r.nke[2 * i];
    double om = r.nmean[4 * i + 3];
    om = om > p.floor_omega ? om : p.floor_omega;
    const double gg[2][2] = {{gr[0], gr[1]}, {gr[2], gr[3]}};
    const double Rm[2][2] = {{R[0], R[3]}, {R[3], R[1]}};
    const double tr = R[0] + R[1] + R[2];
    double b[2][2] = {{0, 0}, {0, 0}};
    // one FP64 division per quotient at most (GB300's FP64 pipe is narrow):
    // the anisotropy from the reciprocal of the trace, gamma5 / 3 as a product
    if (tr > 0.0) {
        const double itr = 1.0 / tr;
        for (int a = 0; a < 2; ++a)
            for (int c = 0; c < 2; ++c) b[a][c] = Rm[a][c] * itr - (a == c ? 1.0 / 3.0 : 0.0);
    }
    const double det = R[2] * (R[0] * R[1] - R[3] * R[3]);
    const double tk = 2.0 / 3.0 * k;
    double Av = p.Cv * det / (tk * tk * tk);
    Av = Av < 1.0 ? Av : 1.0;
    const double iso = 0.5 * (1.0 - p.C1) * k * om;
    const double g3 = p.gamma5 * (1.0 / 3.0);
    int q = 0;
    for (int a = 0; a < 2; ++a)
        for (int c = 0; c < 2; ++c) {
            double t = (p.C2 * Av + g3) * gg[a][c] - g3 * gg[c][a];
            for (int m = 0; m < 2; ++m) t += p.gamma5 * b[a][m] * gg[m][c];
            for (int l = 0; l < 2; ++l) t -= p.gamma5 * b[a][l] * gg[c][l];
            r.f[NC * (size_t)i + q++] = (a == c ? iso : 0.0) + (p.rotta ? 0.0 : k * t);
        }
    r.f[NC * (size_t)i + 4] = iso;
    if (r.is_wall[i]) {
        const double eps = r.nke[2 * i + 1], nx = r.wn[2 * i], ny = r.wn[2 * i + 1];
        const double gw[NC] = {-p.er_wall * eps * nx * nx, -p.er_wall * eps * nx * ny, -p.er_wall * eps * ny * nx,
                               -p.er_wall * eps * ny * ny, 0.0};
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            r.g[NC * (size_t)i + c] = gw[c];
            if (r.prop != nullptr) r.prop[NC * (size_t)i + c] = gw[c];
        }
    } else if (r.prop != nullptr) {
#pragma unroll
        for (int c = 0; c < NC; ++c) r.prop[NC * (size_t)i + c] = r.prev[NC * (size_t)i + c];
    }
}

// node gradients of the mean velocity (area-weighted element gradients), and
// with elliptic relaxation the node's FE right-hand side from them, which
// needs nothing of other nodes
__global__ void k_node_grad(int nn, const int* __restrict__ n2e_off, const int* __restrict__ n2e,
                            const double* __restrict__ area, const double* __restrict__ eder, double* ngrad,
                            const RhsArgs rhs, const pdf_params p) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    double a = 0, g[4] = {0, 0, 0, 0};
    const int q1 = n2e_off[i + 1];
    for (int q0 = n2e_off[i]; q0 < q1; q0 += 4) {  // four elements at a time, as in k_node_stats
        int e4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) e4[k] = q0 + k < q1 ? n2e[q0 + k] : -1;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int e = e4[k];
            const bool in = e >= 0;
            const double A = in ? area[e] : 0.0;
            a += A;
#pragma unroll
            for (int j = 0; j < 4; ++j) g[j] += A * (in ? eder[9 * e + j] : 0.0);
        }
    }
    const double ia = 1.0 / a;
    double gr[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        gr[k] = g[k] * ia;
        ngrad[4 * i + k] = gr[k];
    }
    if (rhs.f != nullptr) fe_rhs_node(i, gr, rhs, p);
}

template <typename T>
__global__ void k_elem_lap(int nt, const int* __restrict__ tri, const double* __restrict__ gradb,
                           const double* __restrict__ ngrad, double* eder, T* epack) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nt) return;
    double lu = 0, lv = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int a = tri[3 * e + k];
        const double gx = gradb[6 * e + 2 * k], gy = gradb[6 * e + 2 * k + 1];
        lu += ngrad[4 * a] * gx + ngrad[4 * a + 1] * gy;
        lv += ngrad[4 * a + 2] * gx + ngrad[4 * a + 3] * gy;
    }
    eder[9 * (size_t)e + 4] = lu;
    eder[9 * (size_t)e + 5] = lv;
    epack[(size_t)ELEM_PACK_W * e + 4] = (T)lu;
    epack[(size_t)ELEM_PACK_W * e + 5] = (T)lv;
}

template <typename T>
__global__ void k_node_pack(int nn, const double* __restrict__ nmean, const double* __restrict__ nR,
                            const double* __restrict__ nke, const int* __restrict__ rep, double* nwp, pdf_params p,
                            double* npack, T* npackT) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nn) return;
    double q[NODE_PACK_W];
    const double kk = nke[2 * i], eps = nke[2 * i + 1];
    double Om = nmean[4 * i + 3];
    Om = Om > p.floor_omega ? Om : p.floor_omega;
    q[0] = nmean[4 * i]; q[1] = nmean[4 * i + 1]; q[2] = Om;
    if (p.wall_model == PDF_WALL_FUNCTIONS) {
        const double a = -(0.5 + 0.75 * p.C0) * Om;  // Eq. wall-GandC
        q[3] = p.C0 * eps;
        q[4] = a; q[5] = 0.0; q[6] = 0.0; q[7] = a; q[8] = a;
    } else {
        // Eqs. Gij and C0 with the solution of the node's canonical row; a
        // periodic image row takes that solution (canonical rows are only
        // read here, image rows only written)
        const int r = rep[i];
        const double* w = nwp + 5 * (size_t)r;
        if (r != i) {
#pragma unroll
            for (int k = 0; k < 5; ++k) nwp[5 * (size_t)i + k] = w[k];
        }
        const double* R = nR + 6 * (size_t)i;
        const double ik = 1.0 / kk, h2k = 0.5 * ik;
        q[4] = (2.0 * w[0] - eps) * h2k;
        q[5] = w[1] * ik;
        q[6] = w[2] * ik;
        q[7] = (2.0 * w[3] - eps) * h2k;
        q[8] = (2.0 * w[4] - eps) * h2k;
        const double s = w[0] * R[0] + w[1] * R[3] + w[2] * R[3] + w[3] * R[1] + w[4] * R[2];
        const double c0eps = -2.0 * s * ik * (1.0 / 3.0);
        q[3] = c0eps > 0.0 ? c0eps : 0.0;
    }
    q[9] = p.fx; q[10] = p.fy; q[11] = 0.0;
#pragma unroll
    for (int k = 0; k < 11; ++k) npack[11 * (size_t)i + k] = q[k];
#pragma unroll
    for (int k = 0; k < NODE_PACK_W; ++k) npackT[(size_t)NODE_PACK_W * i + k] = (T)q[k];
}

// the node pack written as an affine function on each element: with the
// barycentric coordinates l_k = a_k dx + b_k dy + c_k (dx, dy from the
// element's reference point), sum_k l_k F_k = dx sum_k a_k F_k +
// dy sum_k b_k F_k + sum_k c_k F_k, so a particle evaluates F0 + Fx dx + Fy dy
// from one record of its element instead of three node records
constexpr int AFF_THREADS = 128;  // elements per block of k_elem_affine

template <typename T>
__device__ __forceinline__ void load_row12(const T* __restrict__ p, T (&o)[12]) {
    if constexpr (sizeof(T) == 4) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 v = __ldg(q + k);
            o[4 * k] = v.x; o[4 * k + 1] = v.y; o[4 * k + 2] = v.z; o[4 * k + 3] = v.w;
        }
    } else {
        const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const double2 v = __ldg(q + k);
            o[2 * k] = v.x; o[2 * k + 1] = v.y;
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(AFF_THREADS) k_elem_affine(int nt, const int* __restrict__ tri,
                                                            const T* __restrict__ egeo,
                                                            const T* __restrict__ npackT, T* eaff) {
    // the block's records are assembled in shared memory, then written as one
    // contiguous run with 16-byte stores
    __shared__ __align__(16) T rec[AFF_THREADS * ELEM_AFF_W];
    const int e0 = blockIdx.x * AFF_THREADS, e = e0 + threadIdx.x;
    const int ne = min(AFF_THREADS, nt - e0);
    if (e < nt) {
        T g[12];
        load_row12(egeo + (size_t)EGEO_W * e, g);
        T F0[NODE_PACK_W], Fx[NODE_PACK_W], Fy[NODE_PACK_W];
#pragma unroll
        for (int q = 0; q < NODE_PACK_W; ++q) F0[q] = Fx[q] = Fy[q] = (T)0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            T P[12];
            load_row12(npackT + (size_t)NODE_PACK_W * tri[3 * e + k], P);
            const T ak = g[2 + 3 * k], bk = g[3 + 3 * k], ck = g[4 + 3 * k];
#pragma unroll
            for (int q = 0; q < NODE_PACK_W; ++q) {
                Fx[q] += ak * P[q];
                Fy[q] += bk * P[q];
                F0[q] += ck * P[q];
            }
        }
        T* o = rec + ELEM_AFF_W * threadIdx.x;
#pragma unroll
        for (int q = 0; q < NODE_PACK_W; ++q) {
            o[q] = F0[q];
            o[NODE_PACK_W + q] = Fx[q];
            o[2 * NODE_PACK_W + q] = Fy[q];
        }
    }
    __syncthreads();
    // ne records of ELEM_AFF_W values: 16-byte words (ELEM_AFF_W * sizeof(T) is a multiple of 16)
    constexpr int VW = 16 / sizeof(T);
    const int nwords = ne * ELEM_AFF_W / VW;
    const float4* src = reinterpret_cast<const float4*>(rec);
    float4* dst = reinterpret_cast<float4*>(eaff + (size_t)ELEM_AFF_W * e0);
    for (int w = threadIdx.x; w < nwords; w += AFF_THREADS) dst[w] = src[w];
}

template <typename T>
int run(pdf_ctx* c) {
    // one warp per block: these kernels are bound by GB300's FP64 pipe, and
    // with 20.5k nodes (40k elements) larger blocks leave some SMs with twice
    // the work of others
    const int nn = c->m.nn, nt = c->m.nt, tb = 32;
    const unsigned gn = (nn + tb - 1) / tb, ge = (nt + tb - 1) / tb;
    timing_begin(c, PDF_K_FIELDS);
    k_node_stats<<<gn, tb, 0, c->s>>>(nn, c->m.n2e_off, c->m.n2e, c->en, c->emean, c->eR, c->epsivar, c->p,
                                      c->nwt, c->nmean, c->nR, c->npsivar, c->nke);
    k_elem_derived<T><<<ge, tb, 0, c->s>>>(nt, c->m.tri, c->m.gradb, c->m.cent, c->nmean, c->nR, c->nke,
                                           c->p, c->prec == 2, c->eder, (T*)c->epackT);
    // elliptic relaxation: the FE assembly (it needs only L, column 8 of
    // eder) and then the element Laplacian (needed by the next particle step
    // only) run on the side stream, beside the node gradients, the right-hand
    // side and the residual check of the context stream; the Laplacian writes
    // columns 4 and 5 of eder, which nothing on the context stream reads
    // before the join at the end of this function
    const bool er = c->p.wall_model == PDF_ELLIPTIC_RELAXATION;
    if (er) {
        PDF_CUDA(c, cudaEventRecord(c->side_fork, c->s));
        PDF_CUDA(c, cudaStreamWaitEvent(c->s2, c->side_fork, 0));
        TRY_OK(launch_fe_assemble(c, c->s2));
        PDF_CUDA(c, cudaEventRecord(c->side_join, c->s2));
    }
    RhsArgs rhs;
    rhs.nR = c->nR; rhs.nke = c->nke; rhs.nmean = c->nmean; rhs.is_wall = c->m.is_wall; rhs.wn = c->m.wn;
    rhs.f = er ? c->fe_f : nullptr;
    rhs.g = c->fe_g;
    rhs.prev = c->nwp;
    rhs.prop = er && c->sur_mode == 5 ? c->fe_prop : nullptr;
    k_node_grad<<<gn, tb, 0, c->s>>>(nn, c->m.n2e_off, c->m.n2e, c->m.area, c->eder, c->ngrad, rhs, c->p);
    if (er) {
        PDF_CUDA(c, cudaEventRecord(c->side_fork, c->s));
        PDF_CUDA(c, cudaStreamWaitEvent(c->s2, c->side_fork, 0));
    }
    k_elem_lap<T><<<ge, tb, 0, er ? c->s2 : c->s>>>(nt, c->m.tri, c->m.gradb, c->ngrad, c->eder, (T*)c->epackT);
    if (er) PDF_CUDA(c, cudaEventRecord(c->side_join2, c->s2));
    c->launches += 4;
    if (c->m.n_owall_elem > 0) {
        const int nle = c->m.n_owall_elem, nln = c->m.n_owall_node;
        k_omw_elem<T><<<(nle + 7) / 8, 256, 0, c->s>>>(nle, c->m.owall_elem, c->off, c->emean,
                                                        (const T*)c->stA[2], (const T*)c->stA[3],
                                                        (const T*)c->stA[5], c->eomw);
        k_omw_node<<<(nln + tb - 1) / tb, tb, 0, c->s>>>(nln, c->m.owall_node, c->m.n2e_off, c->m.n2e, c->en,
                                                          c->eomw, c->nomw);
        c->launches += 2;
    }
    timing_end(c, PDF_K_FIELDS);
    PDF_CUDA(c, cudaGetLastError());
    if (c->p.wall_model == PDF_ELLIPTIC_RELAXATION) {
        const int st = launch_elliptic(c);
        if (st != PDF_OK) return st;
    }
    timing_begin(c, PDF_K_FIELDS);
    k_node_pack<T><<<gn, tb, 0, c->s>>>(nn, c->nmean, c->nR, c->nke, c->m.rep, c->nwp, c->p, c->npack,
                                        (T*)c->npackT);
    k_elem_affine<T><<<(nt + AFF_THREADS - 1) / AFF_THREADS, AFF_THREADS, 0, c->s>>>(
        nt, c->m.tri, (const T*)(sizeof(T) == 8 ? (const void*)c->m.egeo_d : (const void*)c->m.egeo_f),
        (const T*)c->npackT, (T*)c->eaffT);
    c->launches += 2;
    if (er) PDF_CUDA(c, cudaStreamWaitEvent(c->s, c->side_join2, 0));  // the side stream joins back
    timing_end(c, PDF_K_FIELDS);
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

}  // namespace

int launch_fields(pdf_ctx* c) { return c->prec == 0 ? run<double>(c) : run<float>(c); }
