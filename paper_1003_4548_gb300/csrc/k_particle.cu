// k_particle.cu -- seeding and the fused per-particle time step.
//
// One thread per particle, particles stored as structure-of-arrays sorted by
// host element so that the element and node data of a warp are the same few
// cache lines (broadcast loads). The step evaluates every right-hand side from
// the statistics S^n (forward Euler-Maruyama, end of Section 2.2):
//   Eq. IECM           psi <- psi - r (psi - <phi|V>_bin),  r = dt/t_m
//   Eq. frequency-model, Eq. frequency_source
//   Eq. Lagrangian-velocity (G_ij and C0 eps interpolated from the nodes,
//   through the element's affine record of the node pack)
//   Eq. Lagrangian-position with the velocity at step n
//   boundaries: periodic seams, symmetry top, wall reflections
//   (Eqs. wall-normal-velocity .. wall-omega, or specular no-slip), the
//   element walk to the new host element, and the continuous source.
#include <algorithm>

#include "mlp_tc.cuh"
#include "pdf_internal.cuh"

namespace {

// 12-wide packs (node pack, element geometry) and 8-wide packs, read with
// 128-bit loads in FP32 (64-bit pairs in FP64)
template <int W, typename T>
__device__ __forceinline__ void load_pack(const T* __restrict__ p, T (&o)[W]) {
    if constexpr (sizeof(T) == 4) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int k = 0; k < W / 4; ++k) {
            const float4 v = __ldg(q + k);
            o[4 * k] = v.x; o[4 * k + 1] = v.y; o[4 * k + 2] = v.z; o[4 * k + 3] = v.w;
        }
    } else {
        const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
        for (int k = 0; k < W / 2; ++k) {
            const double2 v = __ldg(q + k);
            o[2 * k] = v.x; o[2 * k + 1] = v.y;
        }
    }
}

// Gaussian pair from two uniforms in (0, 1]. FP64: Box & Muller with the
// accurate functions. FP32: the hardware logarithm, and the angle 2 pi ub
// taken as pi (2 ub - 1) in [-pi, pi], where the hardware sine/cosine are
// accurate to ~4e-7 absolute; z = -r cos(pi (2 ub - 1)) = r cos(2 pi ub)
// (same for the sine).
__device__ __forceinline__ void gauss_pair(double ua, double ub, double& za, double& zb) {
    box_muller(ua, ub, za, zb);
}
__device__ __forceinline__ float lg2_approx(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sin_approx(float x) {
    float y;
    asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float cos_approx(float x) {
    float y;
    asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
// the radius sqrt(-2 ln ua) of the FP32 pair: ua in [2^-32, 1] is normal, so
// the flush-to-zero hardware forms need no denormal handling; -2 ln ua =
// -2 ln(2) log2(ua)
__device__ __forceinline__ float bm_radius(float ua) {
    const float m2l = -1.3862943611198906f * lg2_approx(ua);
    return m2l > 0.f ? m2l * rsqrt_approx(m2l) : 0.f;
}
__device__ __forceinline__ void gauss_pair(float ua, float ub, float& za, float& zb) {
    const float r = bm_radius(ua);
    const float th = 3.14159265358979f * fmaf(2.0f, ub, -1.0f);
    za = -r * cos_approx(th);
    zb = -r * sin_approx(th);
}
// one member of a pair (the step uses six of its eight Gaussians)
__device__ __forceinline__ float gauss_cos(float ua, float ub) {
    return -bm_radius(ua) * cos_approx(3.14159265358979f * fmaf(2.0f, ub, -1.0f));
}
__device__ __forceinline__ float gauss_sin(float ua, float ub) {
    return -bm_radius(ua) * sin_approx(3.14159265358979f * fmaf(2.0f, ub, -1.0f));
}

template <typename T> __device__ __forceinline__ T t_div(T a, T b) { return a / b; }
template <> __device__ __forceinline__ float t_div<float>(float a, float b) { return __fdividef(a, b); }

template <typename T>
struct StepArgs {
    int64_t n;
    T dt, sdt, s2nu, nu;
    const uint32_t* stepp;  // step counter on the device (advanced by the sort after each step)
    uint2 key;
    PhiloxKeys rk;          // the key's ten round keys
    const int* __restrict__ tri;
    const int* __restrict__ nbr;
    const int* __restrict__ einfo;
    const T* __restrict__ egeo;
    const T* __restrict__ npack;
    const T* __restrict__ epack;
    const T* __restrict__ eaff;  // node pack fields as F0 + Fx dx + Fy dy on each element
    const T* __restrict__ ecm;
    const double* __restrict__ nmean;
    const double* __restrict__ nR;
    const double* __restrict__ nomw;  // Section 4 frequency reflection: wall-node <omega u_i>, <omega u_i u_j>
    T *x, *y, *u, *v, *w, *om, *psi;
    const uint32_t* __restrict__ id;
    int* elem;
    const unsigned char* __restrict__ bin;
    int* cnt;
    int* status;
    int B, wall_model, mix_exp, reflect_max;
    T C3, C4, C0, Cmu_half, kappa, E, yp, beta, fx, fy, x0, y0, r0, period, inv_period, floor_k, floor_om;
    // per-particle surrogate (FP32 state only)
    const float* __restrict__ nsur;   // node pack: 10 standardised features, k, eps, uu, vv, ww, uv
    const float* __restrict__ surw;   // bf16-rounded parameters, then the standardisation
    const int* __restrict__ sur_ok;   // the network passed this step's residual check
    float* pwp;                       // wp of every particle (mode 4), or NULL
};

// velocity and frequency at a boundary hit: tag 2 symmetry; tag 1 wall
// (wall functions in the wall-element frame, or specular no-slip); the hit
// lies at mu along the edge from node na to node nb
template <typename T>
__device__ void reflect(const StepArgs<T>& a, int tag, T nx, T ny, const double* st, int na, int nb, double mu,
                        T& u, T& v, T& w, T& om) {
    const T tx = ny, ty = -nx;
    const T Ut = u * tx + v * ty, Vn = u * nx + v * ny;
    if (tag == 2) {
        u = Ut * tx - Vn * nx;
        v = Ut * ty - Vn * ny;
        return;
    }
    if (a.wall_model == PDF_ELLIPTIC_RELAXATION) {
        u = -u; v = -v; w = -w;
        return;
    }
    const T Ump = (T)st[0] * tx + (T)st[1] * ty;
    const T R11 = (T)st[2], R22 = (T)st[3], R33 = (T)st[4], R12 = (T)st[5];
    T v2 = R11 * nx * nx + (T)2 * R12 * nx * ny + R22 * ny * ny;
    const T uv = R11 * tx * nx + R12 * (tx * ny + ty * nx) + R22 * ty * ny;
    v2 = v2 > a.floor_k ? v2 : a.floor_k;
    T kp = (T)0.5 * (R11 + R22 + R33);
    kp = kp > a.floor_k ? kp : a.floor_k;
    T Omp = (T)st[6];
    Omp = Omp > a.floor_om ? Omp : a.floor_om;
    const T dpdx = -(a.fx * tx + a.fy * ty);
    const T uhat2 = a.Cmu_half * kp;
    const T gam = (uv * dpdx > (T)0) ? (T)1 : (T)0;
    const T us = t_sqrt<T>(uhat2 + gam * fabs(a.yp * dpdx));
    const T Ue = us / a.kappa * t_log<T>(a.E * a.yp * us / a.nu);
    T Ue2 = Ue * Ue;
    Ue2 = Ue2 > a.floor_k ? Ue2 : a.floor_k;
    const T alpha = (T)2 * uhat2 * Ump * fabs(Ump) / (v2 * Ue2);
    const T VR = -Vn, UR = Ut + alpha * Vn;
    u = UR * tx + VR * nx;
    v = UR * ty + VR * ny;
    if (a.nomw) {
        // Section 4: omega_R = omega_I exp(-2 V_I <omega v>_p / <omega v^2>_p),
        // v the wall-normal fluctuation; <omega v^2> floored at floor_k <omega>_p
        const double* Wa = a.nomw + 5 * (size_t)na;
        const double* Wb = a.nomw + 5 * (size_t)nb;
        T W[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) W[k] = (T)((1 - mu) * Wa[k] + mu * Wb[k]);
        const T wv = W[0] * nx + W[1] * ny;
        T wv2 = W[2] * nx * nx + (T)2 * W[3] * nx * ny + W[4] * ny * ny;
        const T fl = a.floor_k * Omp;
        wv2 = wv2 > fl ? wv2 : fl;
        om = om * t_exp<T>((T)-2 * Vn * wv / wv2);
    } else {
        om = om * t_exp<T>(a.beta * Vn / (a.yp * Omp));
    }
}

// a particle between its SDEs and its boundaries: position at step n (P),
// the new position (Q), the new velocity, frequency and scalar (before the
// source), its element at step n
template <typename T>
struct Mid {
    int i, e0;
    T x, y, qx, qy, u, v, w, om, psi;
};

// first half of the particle-step of particle i whose state at step n was
// staged in shared memory: the mixing, frequency, velocity and position
// updates; `stays` reports whether Q lies in the particle's element (then
// the second half has no element walk to do)
template <typename T, bool SUR = false>
__device__ __forceinline__ Mid<T> step_sde(const StepArgs<T>& a, const uint32_t step, const int i, const T x,
                                           const T y, T u, T v, T w, T om, T psi, const uint32_t pid, const int e0,
                                           const int b, bool& stays, const float* ysur = nullptr) {

    // P1 interpolation of the node pack at the particle: the element's affine
    // record, F = F0 + Fx dx + Fy dy with (dx, dy) from the element's
    // reference point (the barycentric sum regrouped per element)
    T g[EGEO_W];
    load_pack<EGEO_W>(a.egeo + EGEO_W * e0, g);
    const T dx = x - g[0], dy = y - g[1];
    T lw[3] = {(T)0, (T)0, (T)0};  // barycentric coordinates, for the per-particle network's features
    if constexpr (SUR) {
        lw[0] = g[2] * dx + g[3] * dy + g[4];
        lw[1] = g[5] * dx + g[6] * dy + g[7];
        lw[2] = g[8] * dx + g[9] * dy + g[10];
    }
    T F[NODE_PACK_W];
    {
        T F0[NODE_PACK_W], Fx[NODE_PACK_W], Fy[NODE_PACK_W];
        const T* r = a.eaff + (size_t)ELEM_AFF_W * e0;
        load_pack<NODE_PACK_W>(r, F0);
        load_pack<NODE_PACK_W>(r + NODE_PACK_W, Fx);
        load_pack<NODE_PACK_W>(r + 2 * NODE_PACK_W, Fy);
#pragma unroll
        for (int q = 0; q < 11; ++q) F[q] = F0[q] + Fx[q] * dx + Fy[q] * dy;
    }
    if constexpr (SUR) {
        if (ysur != nullptr) {
            // wp of the network at this particle (standardised outputs in ysur),
            // then G_ij and C0 eps from it as Eqs. Gij and C0 do at the nodes,
            // with k, eps and the stresses interpolated to the particle
            float kk = 0.f, ee = 0.f, R[4] = {0.f, 0.f, 0.f, 0.f};
            const int nd[3] = {a.tri[3 * e0], a.tri[3 * e0 + 1], a.tri[3 * e0 + 2]};
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const float4 ke = __ldg(reinterpret_cast<const float4*>(a.nsur + 16 * (size_t)nd[m]) + 2);
                const float4 rr = __ldg(reinterpret_cast<const float4*>(a.nsur + 16 * (size_t)nd[m]) + 3);
                kk += lw[m] * ke.z;
                ee += lw[m] * ke.w;
                R[0] += lw[m] * rr.x; R[1] += lw[m] * rr.y; R[2] += lw[m] * rr.z; R[3] += lw[m] * rr.w;
            }
            kk = kk > (float)a.floor_k ? kk : (float)a.floor_k;
            const float* nm = a.surw + PDF_MLP_NPARAM;
            float wp[5];
#pragma unroll
            for (int o = 0; o < 5; ++o) wp[o] = ee * (ysur[o] * nm[25 + o] + nm[20 + o]);
            const float ik = 1.f / kk, h2k = 0.5f * ik;
            F[4] = (T)((2.f * wp[0] - ee) * h2k);
            F[5] = (T)(wp[1] * ik);
            F[6] = (T)(wp[2] * ik);
            F[7] = (T)((2.f * wp[3] - ee) * h2k);
            F[8] = (T)((2.f * wp[4] - ee) * h2k);
            const float s = wp[0] * R[0] + (wp[1] + wp[2]) * R[3] + wp[3] * R[1] + wp[4] * R[2];
            const float c0e = -2.f * s * ik * (1.f / 3.f);
            F[3] = (T)(c0e > 0.f ? c0e : 0.f);
            if (a.pwp != nullptr) {
#pragma unroll
                for (int o = 0; o < 5; ++o) a.pwp[5 * (size_t)i + o] = wp[o];
            }
        }
    }
    T ep[ELEM_PACK_W];
    load_pack<ELEM_PACK_W>(a.epack + ELEM_PACK_W * e0, ep);
    const T Ux = ep[0], Uy = ep[1], Vx = ep[2], Vy = ep[3], lapU = ep[4], lapV = ep[5];
    const T Som = ep[6], tm = ep[7];
    const T cm = a.ecm[a.B * e0 + b];

    // eight Gaussians: counter (id, step, call, 0); the step uses z[0], z[1]
    // (dW_1,2), z[3..5] (dW'), z[6] (dW for omega): z[2] (dW_3, paired with
    // the zero spanwise gradient) and z[7] are left out in FP32
    T z[8];
    {
        const uint4 r0 = philox4x32_10_rk(a.rk, make_uint4(pid, step, 0u, 0u));
        const uint4 r1 = philox4x32_10_rk(a.rk, make_uint4(pid, step, 1u, 0u));
        if constexpr (sizeof(T) == 4) {
            gauss_pair(unif<T>(r0.x), unif<T>(r0.y), z[0], z[1]);
            z[2] = (T)0;
            z[3] = gauss_sin(unif<T>(r0.z), unif<T>(r0.w));
            gauss_pair(unif<T>(r1.x), unif<T>(r1.y), z[4], z[5]);
            z[6] = gauss_cos(unif<T>(r1.z), unif<T>(r1.w));
            z[7] = (T)0;
        } else {
            gauss_pair(unif<T>(r0.x), unif<T>(r0.y), z[0], z[1]);
            gauss_pair(unif<T>(r0.z), unif<T>(r0.w), z[2], z[3]);
            gauss_pair(unif<T>(r1.x), unif<T>(r1.y), z[4], z[5]);
            gauss_pair(unif<T>(r1.z), unif<T>(r1.w), z[6], z[7]);
        }
    }
    const T dt = a.dt, sdt = a.sdt;

    // Eq. IECM
    const T r = a.mix_exp ? (T)1 - t_exp<T>(-t_div(dt, tm)) : t_div(dt, tm);
    if (!a.mix_exp && r > (T)1) set_status(a.status, ST_DT);
    const T psi1 = psi - r * (psi - cm);
    // Eq. frequency-model with Eq. frequency_source
    const T Om = F[2];
    T om1 = om - a.C3 * Om * (om - Om) * dt - Som * Om * om * dt +
            t_sqrt<T>((T)2 * a.C3 * a.C4 * Om * Om * om) * z[6] * sdt;
    om1 = fabs(om1);
    // Eq. Lagrangian-velocity
    const T du = u - F[0], dv = v - F[1], dw = w;
    const T cc = t_sqrt<T>(F[3] > (T)0 ? F[3] : (T)0);
    T u1 = u + (F[9] + (T)2 * a.nu * lapU + F[4] * du + F[5] * dv) * dt +
           a.s2nu * (Ux * z[0] + Uy * z[1]) * sdt + cc * z[3] * sdt;
    T v1 = v + (F[10] + (T)2 * a.nu * lapV + F[6] * du + F[7] * dv) * dt +
           a.s2nu * (Vx * z[0] + Vy * z[1]) * sdt + cc * z[4] * sdt;
    T w1 = w + (F[8] * dw) * dt + cc * z[5] * sdt;
    // Eq. Lagrangian-position with the velocity at step n
    T qx = x + u * dt + a.s2nu * z[0] * sdt;
    T qy = y + v * dt + a.s2nu * z[1] * sdt;

    // Most particles end the step in their own element: the walk's first
    // test (Q inside e0, the same arithmetic) decides that without the walk.
    {
        T ge[EGEO_W];
        load_pack<EGEO_W>(a.egeo + EGEO_W * e0, ge);
        const T qdx = qx - ge[0], qdy = qy - ge[1];
        const T lq0 = ge[2] * qdx + ge[3] * qdy + ge[4];
        const T lq1 = ge[5] * qdx + ge[6] * qdy + ge[7];
        const T lq2 = ge[8] * qdx + ge[9] * qdy + ge[10];
        stays = lq0 >= (T)0 && lq1 >= (T)0 && lq2 >= (T)0;
    }
    Mid<T> m;
    m.i = i; m.e0 = e0; m.x = x; m.y = y; m.qx = qx; m.qy = qy;
    m.u = u1; m.v = v1; m.w = w1; m.om = om1; m.psi = psi1;
    return m;
}

// second half: boundaries and the element walk along the straight path
// P -> Q (skipped when Q stays in e0), the source, the checks, the stores and
// the element histogram of the sort
template <typename T>
__device__ __forceinline__ void finish_particle(const StepArgs<T>& a, const Mid<T>& m, const bool stays) {
    const int i = m.i, e0 = m.e0;
    const T x = m.x, y = m.y;
    T qx = m.qx, qy = m.qy, u1 = m.u, v1 = m.v, w1 = m.w, om1 = m.om;
    const T psi1 = m.psi;
    T px = x, py = y;
    int e = e0, entry = -1, nref = 0, it = 0;
    for (; !stays && it < WALK_MAX; ++it) {
        T ge[EGEO_W];
        load_pack<EGEO_W>(a.egeo + EGEO_W * e, ge);
        const T qdx = qx - ge[0], qdy = qy - ge[1];
        const T lq0 = ge[2] * qdx + ge[3] * qdy + ge[4];
        const T lq1 = ge[5] * qdx + ge[6] * qdy + ge[7];
        const T lq2 = ge[8] * qdx + ge[9] * qdy + ge[10];
        const T pdx = px - ge[0], pdy = py - ge[1];
        int kx = -1;
        T tb = (T)2, lqk = (T)0;
        {
            const T lq[3] = {lq0, lq1, lq2};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                if (k != entry && lq[k] < (T)0) {
                    const T lp = ge[2 + 3 * k] * pdx + ge[3 + 3 * k] * pdy + ge[4 + 3 * k];
                    const T den = lp - lq[k];
                    const T t = den > (T)0 ? t_div(lp, den) : (T)0;
                    if (t < tb) { tb = t; kx = k; lqk = lq[k]; }
                }
            }
        }
        if (kx < 0) break;
        const int info = a.einfo[e];
        const int tag = (info >> (2 * kx)) & 3;
        T cx = px + tb * (qx - px), cy = py + tb * (qy - py);
        if (tag == 0 || tag == 3) {
            const int sh = (info >> (6 + 2 * kx)) & 3;
            if (sh) {
                const T d = sh == 1 ? a.period : -a.period;
                cx += d;
                qx += d;
            }
            entry = (info >> (12 + 2 * kx)) & 3;
            e = a.nbr[3 * e + kx];
            px = cx; py = cy;
        } else {
            if (++nref > a.reflect_max) {
                set_status(a.status, ST_WALL);
                qx = px; qy = py;
                break;
            }
            const T ax = ge[2 + 3 * kx], ay = ge[3 + 3 * kx];
            const T inv = (T)1 / t_sqrt<T>(ax * ax + ay * ay);
            const T nx = ax * inv, ny = ay * inv;
            const T sd = lqk * inv;  // signed distance of Q from the edge line (< 0)
            qx -= (T)2 * sd * nx;
            qy -= (T)2 * sd * ny;
            if (tag == 2 || a.wall_model == PDF_ELLIPTIC_RELAXATION) {
                // symmetry top, or the no-slip wall of the resolved case: no
                // wall statistics needed
                if (tag == 2) {  // the normal component reversed, as reflect<T> does
                    const T tx = ny, ty = -nx;
                    const T Ut = u1 * tx + v1 * ty, Vn = u1 * nx + v1 * ny;
                    u1 = Ut * tx - Vn * nx;
                    v1 = Ut * ty - Vn * ny;
                } else {
                    u1 = -u1; v1 = -v1; w1 = -w1;
                }
            } else {
                // wall functions: the statistics at the hit point, linear along the edge
                const int ka = (kx + 1) % 3, kb = (kx + 2) % 3;
                const T cdx = cx - ge[0], cdy = cy - ge[1];
                const T la = ge[2 + 3 * ka] * cdx + ge[3 + 3 * ka] * cdy + ge[4 + 3 * ka];
                const T lb = ge[2 + 3 * kb] * cdx + ge[3 + 3 * kb] * cdy + ge[4 + 3 * kb];
                const double mu = (double)(lb / (la + lb));
                const int na = a.tri[3 * e + ka], nb = a.tri[3 * e + kb];
                double st[7];
                st[0] = (1 - mu) * a.nmean[4 * na + 0] + mu * a.nmean[4 * nb + 0];
                st[1] = (1 - mu) * a.nmean[4 * na + 1] + mu * a.nmean[4 * nb + 1];
                st[2] = (1 - mu) * a.nR[6 * na + 0] + mu * a.nR[6 * nb + 0];
                st[3] = (1 - mu) * a.nR[6 * na + 1] + mu * a.nR[6 * nb + 1];
                st[4] = (1 - mu) * a.nR[6 * na + 2] + mu * a.nR[6 * nb + 2];
                st[5] = (1 - mu) * a.nR[6 * na + 3] + mu * a.nR[6 * nb + 3];
                st[6] = (1 - mu) * a.nmean[4 * na + 3] + mu * a.nmean[4 * nb + 3];
                reflect<T>(a, tag, nx, ny, st, na, nb, mu, u1, v1, w1, om1);
            }
            px = cx; py = cy;
            entry = kx;
        }
    }
    if (it == WALK_MAX) {
        set_status(a.status, ST_LOST);
        e = e0; qx = x; qy = y;
    }
    // continuous source (minimum-image distance in x; the image choice can
    // differ from an exact division only half a period from the source,
    // far outside the disc)
    T psi2 = psi1;
    {
        T ddx = qx - a.x0;
        ddx -= a.period * t_floor<T>(ddx * a.inv_period + (T)0.5);
        const T ddy = qy - a.y0;
        if (ddx * ddx + ddy * ddy < a.r0 * a.r0) psi2 = (T)1;
    }
    if (!isfinite(u1 + v1 + w1 + om1)) set_status(a.status, ST_NONFINITE);

    a.x[i] = qx; a.y[i] = qy;
    a.u[i] = u1; a.v[i] = v1; a.w[i] = w1; a.om[i] = om1; a.psi[i] = psi2;
    a.elem[i] = e;
    // element histogram for the sort (warp-aggregated)
    const unsigned mask = __match_any_sync(__activemask(), e);
    if ((threadIdx.x & 31) == __ffs(mask) - 1) atomicAdd(&a.cnt[e], __popc(mask));
}

// both halves of a particle-step
template <typename T, bool SUR = false>
__device__ __forceinline__ void advance_particle(const StepArgs<T>& a, const uint32_t step, const int i, const T x,
                                                 const T y, T u, T v, T w, T om, T psi, const uint32_t pid,
                                                 const int e0, const int b, const float* ysur = nullptr) {
    bool stays;
    const Mid<T> m = step_sde<T, SUR>(a, step, i, x, y, u, v, w, om, psi, pid, e0, b, stays, ysur);
    finish_particle(a, m, stays);
}

// ---------------------------------------------------------------------------
// The step kernel: a persistent grid over tiles of TILE consecutive particles.
// Thread 0 of a block stages the tile NSTAGE - 1 ahead (seven state arrays,
// id, element, bin) into shared memory with bulk asynchronous copies that
// complete on the stage's "full" mbarrier, while the block advances the
// current tile, so the load latency of the HBM-streamed state overlaps the
// arithmetic. A warp that has finished a tile arrives on the stage's "empty"
// mbarrier; only thread 0 waits for those arrivals, before it refills the
// stage, so the other warps never wait for the block's slowest particle (a
// wall reflection, a walk over several elements) at a block barrier. The
// arrays are allocated in whole tiles, so every copy starts 16-byte aligned
// and its size is rounded up to 16 bytes inside the allocation.
// ---------------------------------------------------------------------------
constexpr int TILE = 256;

template <typename T>
struct Stage {
    T s[7][TILE];  // x y u v w omega psi
    uint32_t id[TILE];
    int elem[TILE];
    unsigned char bin[TILE];
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    uint64_t g;
    asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(src));
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst)), "l"(g), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// bounded wait for a phase of the barrier (ST_BARRIER if it never completes)
__device__ __forceinline__ void mbar_wait(uint64_t* bar, unsigned parity, int* status) {
    for (int spin = 0; !mbar_try_wait(bar, parity); ++spin) {
        if (spin > (1 << 20)) {
            set_status(status, ST_BARRIER);
            break;
        }
    }
}

template <typename T>
__device__ __forceinline__ void stage_tile(const StepArgs<T>& a, Stage<T>& st, uint64_t* bar, int64_t base, int cnt) {
    const unsigned bt = (unsigned)(((size_t)cnt * sizeof(T) + 15) & ~(size_t)15);
    const unsigned b4 = (unsigned)(((size_t)cnt * 4 + 15) & ~(size_t)15);
    const unsigned b1 = (unsigned)((cnt + 15) & ~15);
    mbar_expect_tx(bar, 7 * bt + 2 * b4 + b1);
    const T* src[7] = {a.x, a.y, a.u, a.v, a.w, a.om, a.psi};
#pragma unroll
    for (int k = 0; k < 7; ++k) bulk_to_smem(st.s[k], src[k] + base, bt, bar);
    bulk_to_smem(st.id, a.id + base, b4, bar);
    bulk_to_smem(st.elem, a.elem + base, b4, bar);
    bulk_to_smem(st.bin, a.bin + base, b1, bar);
}

// stages of the particle kernel (FP32 state: 19 KB of static shared memory
// per block; a third or fourth stage measured no faster, or slower, as the
// staging takes L1 from the node and element gathers)
template <typename T> constexpr int NSTAGE = 2;

// Movers (particles whose new position leaves their element, a few per
// cent) would make a whole warp walk with them: in the FP32 kernel each warp
// queues its movers in shared memory and walks them 32 at a time, so the
// walk's cost follows the number of movers, not of warps holding one.
constexpr int QCAP = 64;  // queue entries per warp (fewer than 32 left plus at most 32 new)

template <typename T>
__global__ void __launch_bounds__(TILE) k_step(const StepArgs<T> a) {
    constexpr int NS = NSTAGE<T>, PD = NS - 1, NW = TILE / 32;  // PD: tiles staged ahead
    constexpr bool DEFER = sizeof(T) == 4;
    __shared__ __align__(128) Stage<T> st[NS];
    __shared__ __align__(8) uint64_t full[NS], empty[NS];
    __shared__ Mid<T> mq[DEFER ? NW : 1][DEFER ? QCAP : 1];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned ltmask = (1u << lane) - 1u;
    int qhead = 0, qn = 0;  // the warp's queue (warp-uniform)
    (void)wid; (void)ltmask; (void)qhead; (void)qn;
    const int64_t ntiles = (a.n + TILE - 1) / TILE;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < NS; ++q) {
            mbar_init(&full[q], 1);
            mbar_init(&empty[q], NW);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint32_t step = *a.stepp;
    const int64_t t0 = blockIdx.x, tstep = gridDim.x;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int q = 0; q < PD; ++q) {
            const int64_t tq = t0 + q * tstep;
            if (tq < ntiles) stage_tile(a, st[q], &full[q], tq * TILE, (int)min((int64_t)TILE, a.n - tq * TILE));
        }
    }
    int k = 0;
    for (int64_t t = t0; t < ntiles; t += tstep, ++k) {
        const int s = k % NS;
        const int64_t tn = t + PD * tstep;
        if (threadIdx.x == 0 && tn < ntiles) {
            // stage (k + PD) mod NS = (k - 1) mod NS: every warp has released
            // tile k - 1 from it (use (k - 1) / NS of that stage)
            const int sp = (k + PD) % NS;
            if (k >= 1) mbar_wait(&empty[sp], (unsigned)(((k - 1) / NS) & 1), a.status);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            stage_tile(a, st[sp], &full[sp], tn * TILE, (int)min((int64_t)TILE, a.n - tn * TILE));
        }
        mbar_wait(&full[s], (unsigned)((k / NS) & 1), a.status);
        const int64_t i = t * TILE + threadIdx.x;
        if constexpr (DEFER) {
            bool mover = false;
            Mid<T> m;
            if (i < a.n) {
                const Stage<T>& q = st[s];
                const int j = threadIdx.x;
                bool stays;
                m = step_sde<T>(a, step, (int)i, q.s[0][j], q.s[1][j], q.s[2][j], q.s[3][j], q.s[4][j], q.s[5][j],
                                q.s[6][j], q.id[j], q.elem[j], (int)q.bin[j], stays);
                if (stays) finish_particle(a, m, true);
                else mover = true;
            }
            // the warp's movers join its queue; the stage is free again
            const unsigned mv = __ballot_sync(0xffffffffu, mover);
            if (mover) mq[wid][(qhead + qn + __popc(mv & ltmask)) & (QCAP - 1)] = m;
            qn += __popc(mv);
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (qn >= 32) {  // a full warp of movers: their walks side by side
                const Mid<T> w = mq[wid][(qhead + lane) & (QCAP - 1)];
                __syncwarp();
                finish_particle(a, w, false);
                qhead = (qhead + 32) & (QCAP - 1);
                qn -= 32;
            }
        } else {
            if (i < a.n) {
                const Stage<T>& q = st[s];
                const int j = threadIdx.x;
                advance_particle(a, step, (int)i, q.s[0][j], q.s[1][j], q.s[2][j], q.s[3][j], q.s[4][j], q.s[5][j],
                                 q.s[6][j], q.id[j], q.elem[j], (int)q.bin[j]);
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);  // this warp is done with stage s
        }
    }
    if constexpr (DEFER) {
        if (lane < qn) finish_particle(a, mq[wid][(qhead + lane) & (QCAP - 1)], false);  // the last movers
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_seed(int64_t n, int ppe, uint2 key, const int* __restrict__ tri,
                                              const double* __restrict__ xy,
                                              const double* __restrict__ wdist, pdf_params p, T* x, T* y,
                                              T* u, T* v, T* w, T* om, T* psi, uint32_t* id, int* elem) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int e = (int)(i / ppe);
    const uint32_t pid = (uint32_t)i;
    const uint4 o0 = philox4x32_10(key, make_uint4(pid, 0u, 0u, 1u));
    const uint4 o1 = philox4x32_10(key, make_uint4(pid, 0u, 1u, 1u));
    const uint4 o2 = philox4x32_10(key, make_uint4(pid, 0u, 2u, 1u));
    const int a = tri[3 * e], b = tri[3 * e + 1], d = tri[3 * e + 2];
    const double s = sqrt(unif<double>(o0.x)), t = unif<double>(o0.y);
    const double l0 = 1.0 - s, l1 = s * (1.0 - t), l2 = s * t;
    const double px = l0 * xy[2 * a] + l1 * xy[2 * b] + l2 * xy[2 * d];
    const double py = l0 * xy[2 * a + 1] + l1 * xy[2 * b + 1] + l2 * xy[2 * d + 1];
    double z0, z1, z2, z3;
    box_muller(unif<double>(o0.z), unif<double>(o0.w), z0, z1);
    box_muller(unif<double>(o1.x), unif<double>(o1.y), z2, z3);
    const double dyr = py - p.y_roof;
    const double ulog = dyr >= p.yp ? p.ustar / p.kappa * log(p.E * dyr * p.ustar / p.nu) : 0.0;
    const double dw = l0 * wdist[a] + l1 * wdist[b] + l2 * wdist[d];
    const double om0 = sqrt(p.Cmu) * p.ustar / (p.kappa * (dw > p.yp ? dw : p.yp));
    const double gsum = -log(unif<double>(o1.z)) - log(unif<double>(o1.w)) - log(unif<double>(o2.x)) -
                        log(unif<double>(o2.y));
    const double sig = sqrt(2.0 / 3.0 * p.k0);
    double ddx = px - p.x0;
    ddx -= p.period * floor(ddx / p.period + 0.5);
    const double dd = hypot(ddx, py - p.y0);
    x[i] = (T)px; y[i] = (T)py;
    u[i] = (T)(ulog + sig * z0); v[i] = (T)(sig * z1); w[i] = (T)(sig * z2);
    om[i] = (T)(0.25 * om0 * gsum);
    psi[i] = dd < p.r0 ? (T)1 : (T)0;
    id[i] = pid;
    elem[i] = e;
}

template <typename T>
StepArgs<T> step_args(pdf_ctx* c, double dt) {
    const pdf_params& p = c->p;
    StepArgs<T> a;
    a.n = c->np;
    a.dt = (T)dt;
    a.sdt = (T)sqrt(dt);
    a.s2nu = (T)sqrt(2.0 * p.nu);
    a.nu = (T)p.nu;
    a.stepp = c->d_step;
    a.key = philox_key(p.seed, p.case_id);
    a.rk = philox_round_keys(a.key);
    a.tri = c->m.tri;
    a.nbr = c->m.nbr;
    a.einfo = c->m.einfo;
    a.egeo = (const T*)(sizeof(T) == 8 ? (const void*)c->m.egeo_d : (const void*)c->m.egeo_f);
    a.npack = (const T*)c->npackT;
    a.epack = (const T*)c->epackT;
    a.eaff = (const T*)c->eaffT;
    a.ecm = (const T*)c->ecmT;
    a.nmean = c->nmean;
    a.nR = c->nR;
    a.nomw = (p.wall_model == PDF_WALL_FUNCTIONS && p.omega_wall) ? c->nomw : nullptr;
    a.x = (T*)c->stA[0]; a.y = (T*)c->stA[1]; a.u = (T*)c->stA[2]; a.v = (T*)c->stA[3];
    a.w = (T*)c->stA[4]; a.om = (T*)c->stA[5]; a.psi = (T*)c->stA[6];
    a.id = c->idA;
    a.elem = c->elemA;
    a.bin = c->bin;
    a.cnt = c->cnt;
    a.status = c->d_status;
    a.B = c->B;
    a.wall_model = p.wall_model;
    a.mix_exp = p.mix_exp;
    a.reflect_max = p.reflect_max;
    a.C3 = (T)p.C3; a.C4 = (T)p.C4; a.C0 = (T)p.C0;
    a.Cmu_half = (T)sqrt(p.Cmu);
    a.kappa = (T)p.kappa; a.E = (T)p.E; a.yp = (T)p.yp;
    a.beta = (T)(-2.0 / (0.5 + 0.75 * p.C0 + p.C3 + p.Comega2 - p.Comega1));
    a.fx = (T)p.fx; a.fy = (T)p.fy;
    a.x0 = (T)p.x0; a.y0 = (T)p.y0; a.r0 = (T)p.r0; a.period = (T)p.period; a.inv_period = (T)(1.0 / p.period);
    a.floor_k = (T)p.floor_k; a.floor_om = (T)p.floor_omega;
    a.nsur = nullptr; a.surw = nullptr; a.sur_ok = nullptr; a.pwp = nullptr;
    return a;
}

}  // namespace

// ---------------------------------------------------------------------------
// Per-particle form of the surrogate (modes 3, 4): the staged step kernel
// with the network evaluated at every particle on the tensor cores. A block
// of 256 threads is two 128-row tiles; each particle's row holds the
// standardised node features interpolated to it. The outputs (wp / eps,
// standardised) go to shared memory, and advance_particle forms G_ij and
// C0 eps from them. When this step's residual check failed, the kernel
// takes G_ij from the node pack (the FE solve) and skips the network.
// ---------------------------------------------------------------------------
struct SurShared {
    __align__(128) uint16_t A[2 * mlptc::TILE_ELEMS];
    mlptc::Weights W;
    float Y[TILE][5];
    __align__(8) uint64_t bar;
    uint32_t tmem;
};

constexpr size_t SUR_STEP_SMEM = 2 * sizeof(Stage<float>) + sizeof(SurShared) + 128;

__global__ void __launch_bounds__(TILE) k_step_sur(const StepArgs<float> a) {
    extern __shared__ __align__(128) unsigned char dsm[];
    Stage<float>* st = reinterpret_cast<Stage<float>*>(dsm);
    SurShared& U = *reinterpret_cast<SurShared*>(dsm + 2 * sizeof(Stage<float>));
    __shared__ __align__(8) uint64_t bar[2];
    const int64_t ntiles = (a.n + TILE - 1) / TILE;
    const bool use_net = *a.sur_ok != 0;  // uniform over the grid
    const int warp = threadIdx.x >> 5;
    if (use_net) mlptc::load(U.W, a.surw, threadIdx.x, TILE);
    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        if (use_net) tc::mbar_init(&U.bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    if (use_net && warp == 0) tc::tmem_alloc(&U.tmem, 128);
    __syncthreads();
    const uint32_t tmem = use_net ? U.tmem : 0u;
    unsigned phase = 0;
    bool net_ok = true;
    const uint32_t step = *a.stepp;
    int64_t t = blockIdx.x;
    if (threadIdx.x == 0 && t < ntiles) stage_tile(a, st[0], &bar[0], t * TILE, (int)min((int64_t)TILE, a.n - t * TILE));
    for (int k = 0; t < ntiles; t += gridDim.x, ++k) {
        const int s = k & 1;
        const int64_t tn = t + gridDim.x;
        if (threadIdx.x == 0 && tn < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            stage_tile(a, st[s ^ 1], &bar[s ^ 1], tn * TILE, (int)min((int64_t)TILE, a.n - tn * TILE));
        }
        mbar_wait(&bar[s], (unsigned)((k >> 1) & 1), a.status);
        const int64_t i = t * TILE + threadIdx.x;
        const int j = threadIdx.x;
        const Stage<float>& q = st[s];
        if (use_net && net_ok) {
            // inputs: the node features interpolated to the particle
            float f[16] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
            if (i < a.n) {
                const int e0 = q.elem[j];
                float g[EGEO_W];
                load_pack<EGEO_W>(a.egeo + EGEO_W * e0, g);
                const float dx = q.s[0][j] - g[0], dy = q.s[1][j] - g[1];
                const float lw[3] = {g[2] * dx + g[3] * dy + g[4], g[5] * dx + g[6] * dy + g[7],
                                     g[8] * dx + g[9] * dy + g[10]};
#pragma unroll
                for (int m = 0; m < 3; ++m) {
                    const float4* np4 = reinterpret_cast<const float4*>(a.nsur + 16 * (size_t)a.tri[3 * e0 + m]);
                    const float4 f0 = __ldg(np4), f1 = __ldg(np4 + 1), f2 = __ldg(np4 + 2);
                    f[0] += lw[m] * f0.x; f[1] += lw[m] * f0.y; f[2] += lw[m] * f0.z; f[3] += lw[m] * f0.w;
                    f[4] += lw[m] * f1.x; f[5] += lw[m] * f1.y; f[6] += lw[m] * f1.z; f[7] += lw[m] * f1.w;
                    f[8] += lw[m] * f2.x; f[9] += lw[m] * f2.y;
                }
            }
            mlptc::put_inputs(U.A + (j >> 7) * mlptc::TILE_ELEMS, j & 127, f);
            float y[16];
            net_ok = mlptc::run(U.W, U.A, 2, tmem, &U.bar, phase, y);
#pragma unroll
            for (int o = 0; o < 5; ++o) U.Y[j][o] = y[o];
            if (!net_ok && threadIdx.x == 0) set_status(a.status, ST_BARRIER);
        }
        if (i < a.n)
            advance_particle<float, true>(a, step, (int)i, q.s[0][j], q.s[1][j], q.s[2][j], q.s[3][j], q.s[4][j],
                                          q.s[5][j], q.s[6][j], q.id[j], q.elem[j], (int)q.bin[j],
                                          (use_net && net_ok) ? U.Y[j] : nullptr);
        __syncthreads();
    }
    if (use_net) {
        tc::fence_before_sync();
        __syncthreads();
        if (warp == 0) {
            tc::fence_after_sync();
            tc::tmem_dealloc(tmem, 128);
        }
    }
}

// persistent grid of the particle kernel: per_sm blocks on every SM (0: as
// many as are resident)
int prepare_particle(pdf_ctx* c, int per_sm) {
    int occ = 0;
    if (c->prec == 0) PDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step<double>, TILE, 0));
    else PDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step<float>, TILE, 0));
    occ = std::max(1, occ);
    if (per_sm <= 0 || per_sm > occ) per_sm = occ;
    c->step_blocks = per_sm * c->num_sms;
    return PDF_OK;
}

int particle_occupancy(pdf_ctx* c) {
    int occ = 0;
    if (c->prec == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step<double>, TILE, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_step<float>, TILE, 0);
    return std::max(1, occ);
}

int launch_particle_step(pdf_ctx* c, double dt) {
    PDF_CUDA(c, cudaMemsetAsync(c->cnt, 0, sizeof(int) * c->m.nt, c->s));
    if (c->np == 0) return PDF_OK;
    if (c->step_blocks == 0) {
        const int st = prepare_particle(c, 0);
        if (st != PDF_OK) return st;
    }
    const int64_t ntiles = (c->np + TILE - 1) / TILE;
    timing_begin(c, PDF_K_PARTICLE);
    if ((c->sur_mode == 3 || c->sur_mode == 4) && c->prec != 0) {
        if (!c->step_sur_blocks) {
            int per_sm = 0;
            PDF_CUDA(c, cudaFuncSetAttribute(k_step_sur, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)SUR_STEP_SMEM));
            PDF_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_sur, TILE, SUR_STEP_SMEM));
            c->step_sur_blocks = std::max(1, std::min(per_sm, 4)) * c->num_sms;  // 128 TMEM columns each
        }
        StepArgs<float> sa = step_args<float>(c, dt);
        sa.nsur = c->nsurT;
        sa.surw = c->sur_w;
        sa.sur_ok = c->sur_skip;
        sa.pwp = (c->sur_mode == 4 && c->pwp_n >= c->np) ? c->pwp : nullptr;
        const unsigned blocks = (unsigned)std::min<int64_t>(ntiles, c->step_sur_blocks);
        k_step_sur<<<blocks, TILE, SUR_STEP_SMEM, c->s>>>(sa);
        ++c->launches;
        timing_end(c, PDF_K_PARTICLE);
        PDF_CUDA(c, cudaGetLastError());
        return PDF_OK;
    }
    const unsigned blocks = (unsigned)std::min<int64_t>(ntiles, c->step_blocks);
    if (c->prec == 0)
        k_step<double><<<blocks, TILE, 0, c->s>>>(step_args<double>(c, dt));
    else
        k_step<float><<<blocks, TILE, 0, c->s>>>(step_args<float>(c, dt));
    ++c->launches;
    timing_end(c, PDF_K_PARTICLE);
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

int launch_seed(pdf_ctx* c, int ppe) {
    if (c->np == 0) return PDF_OK;
    const int threads = 256;
    const unsigned blocks = (unsigned)((c->np + threads - 1) / threads);
    const uint2 key = philox_key(c->p.seed, c->p.case_id);
    if (c->prec == 0)
        k_seed<double><<<blocks, threads, 0, c->s>>>(
            c->np, ppe, key, c->m.tri, c->m.xy, c->m.wdist, c->p, (double*)c->stA[0], (double*)c->stA[1],
            (double*)c->stA[2], (double*)c->stA[3], (double*)c->stA[4], (double*)c->stA[5],
            (double*)c->stA[6], c->idA, c->elemA);
    else
        k_seed<float><<<blocks, threads, 0, c->s>>>(
            c->np, ppe, key, c->m.tri, c->m.xy, c->m.wdist, c->p, (float*)c->stA[0], (float*)c->stA[1],
            (float*)c->stA[2], (float*)c->stA[3], (float*)c->stA[4], (float*)c->stA[5],
            (float*)c->stA[6], c->idA, c->elemA);
    ++c->launches;
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}
