// pdf_internal.cuh -- context layout and device helpers shared by the CUDA
// translation units of the GB300 canyon PDF library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pdf_canyon.h"

// device status bits (pdf_sync maps the lowest set bit to a PDF_ERR_* code)
enum : int {
    ST_DT = 1,
    ST_LOST = 2,
    ST_WALL = 4,
    ST_NONFINITE = 8,
    ST_CG = 16,
    ST_CAPACITY = 32,
    ST_BARRIER = 64
};

constexpr int WALK_MAX = 256;       // element-walk steps per particle-step
constexpr int STATS_THREADS = 128;  // threads per element in the moments kernel
constexpr int STATS_CAP = 2048;     // particles per element held in shared memory
constexpr int NODE_PACK_W = 12;     // <U>,<V>,<omega>,C0eps,G11,G12,G21,G22,G33,Fx,Fy,0
constexpr int ELEM_PACK_W = 8;      // Ux,Uy,Vx,Vy,lapU,lapV,S_omega,t_m
constexpr int EGEO_W = 12;          // xref,yref,(ax,ay,c) x 3, area
constexpr int ELEM_AFF_W = 36;      // the node pack as an affine function on the element: F0, dF/dx, dF/dy

// element -> sort key of the velocity-bin construction (16 bytes)
struct SortKey {
    unsigned long long v;  // order-preserving bits of the velocity component
    uint32_t id;           // persistent particle id (tie-break)
    uint32_t gi;           // group (bits 24..31) | local index (bits 0..23)
};

struct DevMesh {
    int nn = 0, nt = 0;
    int* tri = nullptr;      // 3*nt
    int* nbr = nullptr;      // 3*nt neighbour across edge k (-1 on walls/top)
    int* einfo = nullptr;    // nt: tags (2 bits/edge), periodic shift codes, entry edges
    double* xy = nullptr;    // 2*nn
    double* egeo_d = nullptr;  // EGEO_W*nt
    float* egeo_f = nullptr;   // EGEO_W*nt
    double* gradb = nullptr;   // 6*nt gradients of the barycentric coordinates
    double* area = nullptr;    // nt
    double* cent = nullptr;    // 2*nt
    int* n2e_off = nullptr;    // nn+1
    int* n2e = nullptr;
    double* wdist = nullptr;   // nn
    double* wn = nullptr;      // 2*nn unit wall normal into the fluid (wall nodes)
    unsigned char* is_wall = nullptr;  // nn
    int* rep = nullptr;        // nn canonical node of the periodic class
    // finite elements over canonical nodes
    int nnz = 0;
    int* rowptr = nullptr;
    int* colidx = nullptr;
    double* mval = nullptr;    // consistent mass matrix values
    int* kc_off = nullptr;     // per nnz: contributions [kc_off[q], kc_off[q+1])
    int* kc_elem = nullptr;
    double* kc_geo = nullptr;  // A_e grad(l_k).grad(l_l)
    double* aval = nullptr;    // assembled M + K_{L^2}
    float2* avf = nullptr;     // the same as float-float (compensated-FP32 CG)
    int* diag = nullptr;       // position of the diagonal entry per row (-1 if none)
    // Section 4 frequency reflection (omega_wall = 1): wall nodes, elements around them
    int n_owall_node = 0, n_owall_elem = 0;
    int* owall_node = nullptr;
    int* owall_elem = nullptr;
    // mean-pressure projection (pressure = 1): stiffness values on the FE
    // pattern and the pinned node
    double* pval = nullptr;
    unsigned char* pin = nullptr;
};

struct Timing {
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev[PDF_K_COUNT];
    double total_ms[PDF_K_COUNT] = {0};
    int64_t launches[PDF_K_COUNT] = {0};
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
};

struct pdf_ctx {
    pdf_params p{};
    int B = 8;
    int prec = 0;  // 0 fp64 state, 1 fp32, 2 fp32 + compensated reductions
    cudaStream_t s = nullptr;
    DevMesh m;
    int64_t np = 0;
    int step = 0;
    uint32_t* d_step = nullptr;  // the step counter on the device (Philox counter word 1)
    bool seeded = false, stats_valid = false;
    // particle state, double-buffered for the element sort; T = double or float
    void* stA[7] = {nullptr};
    void* stB[7] = {nullptr};
    uint32_t *idA = nullptr, *idB = nullptr;
    int *elemA = nullptr, *elemB = nullptr;
    unsigned char* bin = nullptr;
    int64_t cap = 0;
    // element sort
    int* cnt = nullptr;
    int* off = nullptr;     // nt+1
    int* cursor = nullptr;  // nt
    int* scan_part = nullptr;  // per-block count totals of the grid-wide scan
    // statistics (FP64)
    int* en = nullptr;
    double *emean = nullptr, *eR = nullptr, *epsivar = nullptr, *ecm = nullptr;
    double *nwt = nullptr, *nmean = nullptr, *nR = nullptr, *nke = nullptr, *npsivar = nullptr;
    double *eder = nullptr, *ngrad = nullptr, *npack = nullptr, *nwp = nullptr;
    // frequency-weighted moments <omega u>,<omega v>,<omega uu>,<omega uv>,<omega vv>
    // of the Section 4 frequency reflection (omega_wall = 1 only)
    double *eomw = nullptr, *nomw = nullptr;
    // mean-pressure projection: right-hand side and solution (canonical
    // rows), node pressure, element gradient; the preconditioner's FP32 block
    // inverses and FP64 coarse inverse (built once)
    double *pr_b = nullptr, *pr_x = nullptr, *pres = nullptr, *egp = nullptr;
    float* pr_binv = nullptr;
    double* pr_a0inv = nullptr;
    int* pr_iters = nullptr;
    int pr_bs = 0, pr_blocks = 0;
    // particle-kernel copies in the state precision
    void* npackT = nullptr;
    void* epackT = nullptr;
    void* eaffT = nullptr;  // ELEM_AFF_W*nt in the state type: node pack fields affine on each element
    void* ecmT = nullptr;
    // crowded-element lists of the FP32 moments path: 2 counters, then 2 x nt ids
    int* elist = nullptr;
    // scratch of the moments kernel for elements above STATS_CAP particles
    SortKey* sort_scratch = nullptr;
    int64_t sort_scratch_n = 0;
    // elliptic relaxation work vectors (canonical nodes x 5)
    double *fe_f = nullptr, *fe_g = nullptr, *fe_z = nullptr, *fe_part = nullptr;
    double* fe_prop = nullptr;  // surrogate proposal for wp (canonical rows x 5)
    unsigned int* fe_bar = nullptr;  // grid barrier words
    int* fe_iters = nullptr;
    int fe_blocks = 0;
    int fe_bs = 0;  // rows per block of the elliptic solver (block-Jacobi block size)
    // learned surrogate of the elliptic solve (mode 0: off)
    int sur_mode = 0;
    double sur_tol = 0.0;
    float* sur_w = nullptr;               // PDF_MLP_NPARAM bf16-rounded parameters + PDF_MLP_NNORM
    int* sur_rows = nullptr;              // free canonical node ids
    int sur_nrows = 0;
    int* sur_skip = nullptr;              // 1: the network's wp passed the residual check this step
    unsigned long long* sur_cnt = nullptr;  // solves, fallbacks
    double* sur_part = nullptr;           // per-block residual partial sums, then the last residual
    float* nsurT = nullptr;               // per-particle form: node pack [nn][16] (10 standardised
                                          // features, k, eps, uu, vv, ww, uv)
    float* pwp = nullptr;                 // per-particle form, mode 4: wp of every particle [n][5]
    double* sur_base = nullptr;           // mode 6: wp of the last FE solve [nn][5] (canonical rows)
    double* sur_snap = nullptr;           // mode 6: eps y(x) at the last FE solve [nn][5]
    double* sur_y = nullptr;              // mode 6: eps y(x) of this step [nn][5]
    int64_t pwp_n = 0;
    // time averaging and probes
    int avg_on = 0;
    double* avg_sum = nullptr;                 // [nt][12] element sums, then [nn][4] node sums
    unsigned long long* avg_count = nullptr;   // averaged steps (on the device)
    int cdf_n = 0, cdf_bins = 0;
    int* cdf_elem = nullptr;
    unsigned long long* cdf_hist = nullptr;    // [cdf_n][cdf_bins]
    // status
    int* d_status = nullptr;
    int* h_status = nullptr;
    void* conv_buf = nullptr;
    size_t conv_bytes = 0;
    Timing tm;
    int timing = 0;
    int64_t launches = 0;  // kernels launched by this context
    long long wait_spins = 0;  // grid-barrier polls before a wait gives up (0: the default)
    int step_blocks = 0;   // persistent grid of the particle kernel
    int step_sur_blocks = 0;  // persistent grid of the per-particle surrogate form
    int scatter_threads = 256;  // block size of the re-sort scatter
    cudaEvent_t coop_wait = nullptr, coop_done = nullptr;  // batch: chain of the cooperative CG launches
    // side stream forked from and joined back into the context stream inside
    // each step: the warp moments kernel beside the crowded-element kernels;
    // the FE assembly and the element Laplacian beside the node gradients,
    // the right-hand side and the residual check (side_join2: the Laplacian)
    cudaStream_t s2 = nullptr;
    cudaEvent_t side_fork = nullptr, side_join = nullptr, side_join2 = nullptr;
    // bins stream: the velocity bins and <phi|V> of a step, forked after the
    // re-sort beside the moments, joined back into the context stream before
    // the step ends
    cudaStream_t s3 = nullptr;
    cudaEvent_t bins_join = nullptr;
    cudaEvent_t crowd_done = nullptr;  // the crowded elements' moments (bucket ranges of their bins)
    bool bins_pending = false;
    int bins_bps = 5;  // blocks per SM of the bins kernel (0: one block per four elements)
    // stream that captures the body of the conditional node around the
    // elliptic CG (lagged or surrogate wp in a captured graph); used for
    // nothing else
    cudaStream_t s_cond = nullptr;
    std::string err;
    int num_sms = 0;
};

// ---------------------------------------------------------------------------
// error helpers
// ---------------------------------------------------------------------------
int fail(pdf_ctx* c, int code, const std::string& msg);
#define TRY_OK(x)                        \
    do {                                 \
        const int st_ = (x);             \
        if (st_ != PDF_OK) return st_;   \
    } while (0)
#define PDF_CUDA(c, call)                                                              \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return fail((c), PDF_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// kernel-class timing brackets (no-ops unless timing is on)
void timing_begin(pdf_ctx* c, int k, cudaStream_t st = nullptr);  // st: the context stream if null
void timing_end(pdf_ctx* c, int k, cudaStream_t st = nullptr);

// ---------------------------------------------------------------------------
// launchers (one translation unit each)
// ---------------------------------------------------------------------------
int launch_seed(pdf_ctx* c, int ppe);
int launch_particle_step(pdf_ctx* c, double dt);
int launch_sort(pdf_ctx* c, bool advance_step = false);  // scan + scatter A -> B + swap (+ d_step += 1)
constexpr int SCAN_CHUNK = 1024;  // element counts per block of the grid-wide scan
inline int scan_blocks(int nt) { return (nt + SCAN_CHUNK - 1) / SCAN_CHUNK; }
int set_device_step(pdf_ctx* c);    // d_step = step
int launch_count_and_sort(pdf_ctx* c);  // histogram of elemA, then launch_sort
int launch_moments(pdf_ctx* c);
int join_bins(pdf_ctx* c);          // the context stream waits for the bins stream (no-op if nothing is pending)
int launch_fields(pdf_ctx* c);      // node stats, derived, recovery, ER solve, packs
int launch_elliptic(pdf_ctx* c);     // right-hand side, (wait for the assembly on side_join), check, CG
int launch_fe_assemble(pdf_ctx* c, cudaStream_t s);  // values of M + K_{L^2} from L (column 8 of eder)
int prepare_pressure(pdf_ctx* c);             // grid and preconditioner of the projection, once
int launch_pressure(pdf_ctx* c, double dt);  // projection after the moments (pressure = 1)
int prepare_particle(pdf_ctx* c, int per_sm);   // persistent grid (0: all resident blocks)
int particle_occupancy(pdf_ctx* c);
int prepare_elliptic(pdf_ctx* c, int bs);       // CG rows per block (0: largest co-resident)
int prepare_moments(pdf_ctx* c);
int launch_surrogate(pdf_ctx* c);   // network wp at the nodes + FE residual check (before the CG)
int launch_surrogate_rebase(pdf_ctx* c);  // mode 6: after the CG, a solve's wp and network values become the reference
int launch_averaging(pdf_ctx* c);   // running sums of the statistics and the CDF probes (when on)
int surrogate_rows(pdf_ctx* c);     // builds the free canonical row list once
int launch_to_double(pdf_ctx* c, const void* src, double* dst, int64_t n);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ void set_status(int* st, int bit) { atomicOr(st, bit); }

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw 2011): ten rounds of the
// multiply-xor round function, key bumped by the Weyl constants each round.
__device__ __forceinline__ uint4 philox4x32_10(uint2 key, uint4 c) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ key.x, lo1, hi0 ^ c.w ^ key.y, lo0);
        key.x += 0x9E3779B9u;
        key.y += 0xBB67AE85u;
    }
    return c;
}

__host__ __device__ inline uint2 philox_key(uint64_t seed, uint32_t case_id) {
    return make_uint2((uint32_t)seed, (uint32_t)(seed >> 32) ^ case_id);
}

// The ten round keys of Philox4x32-10 for one key (the Weyl schedule), made
// once on the host: the key is the same for every particle of a step, so a
// kernel that takes them as a parameter reads them from the constant bank
// instead of advancing the schedule per call.
struct PhiloxKeys {
    uint32_t k[20];  // round r: k[2 r], k[2 r + 1]
};

inline PhiloxKeys philox_round_keys(uint2 key) {
    PhiloxKeys rk;
    for (int r = 0; r < 10; ++r) {
        rk.k[2 * r] = key.x;
        rk.k[2 * r + 1] = key.y;
        key.x += 0x9E3779B9u;
        key.y += 0xBB67AE85u;
    }
    return rk;
}

// Philox4x32-10 from precomputed round keys; each round's two 32 x 32-bit
// products as 64-bit wide multiplies. Bit for bit philox4x32_10.
__device__ __forceinline__ uint4 philox4x32_10_rk(const PhiloxKeys& rk, uint4 c) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c.x;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c.z;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ rk.k[2 * r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ rk.k[2 * r + 1], (uint32_t)p0);
    }
    return c;
}

// uniform in (0, 1]: (w + 1) 2^-32, exact in double, rounded in float
template <typename T> __device__ __forceinline__ T unif(uint32_t w);
template <> __device__ __forceinline__ double unif<double>(uint32_t w) {
    return ((double)w + 1.0) * 2.3283064365386963e-10;
}
template <> __device__ __forceinline__ float unif<float>(uint32_t w) {
    return fmaf((float)w, 2.3283064365386963e-10f, 2.3283064365386963e-10f);
}

// Box & Muller (1958)
__device__ __forceinline__ void box_muller(double ua, double ub, double& za, double& zb) {
    const double r = sqrt(-2.0 * log(ua));
    double s, c;
    sincospi(2.0 * ub, &s, &c);
    za = r * c;
    zb = r * s;
}
__device__ __forceinline__ void box_muller(float ua, float ub, float& za, float& zb) {
    const float r = sqrtf(-2.0f * logf(ua));
    float s, c;
    sincospif(2.0f * ub, &s, &c);
    za = r * c;
    zb = r * s;
}

template <typename T> __device__ __forceinline__ T t_sqrt(T x);
template <> __device__ __forceinline__ double t_sqrt(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float t_sqrt(float x) { return sqrtf(x); }
template <typename T> __device__ __forceinline__ T t_exp(T x);
template <> __device__ __forceinline__ double t_exp(double x) { return exp(x); }
template <> __device__ __forceinline__ float t_exp(float x) { return expf(x); }
template <typename T> __device__ __forceinline__ T t_log(T x);
template <> __device__ __forceinline__ double t_log(double x) { return log(x); }
template <> __device__ __forceinline__ float t_log(float x) { return logf(x); }
template <typename T> __device__ __forceinline__ T t_floor(T x);
template <> __device__ __forceinline__ double t_floor(double x) { return floor(x); }
template <> __device__ __forceinline__ float t_floor(float x) { return floorf(x); }

// order-preserving unsigned bits of a float/double (-0 folded onto +0)
__device__ __forceinline__ unsigned long long ord_bits(double v) {
    v = v + 0.0;
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ unsigned long long ord_bits(float v) {
    v = v + 0.0f;
    uint32_t b = (uint32_t)__float_as_uint(v);
    return (unsigned long long)((b >> 31) ? ~b : (b | 0x80000000u));
}
