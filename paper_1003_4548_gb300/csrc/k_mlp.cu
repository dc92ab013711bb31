// k_mlp.cu -- learned surrogate of the elliptic-relaxation solve.
//
// The paper solves Eq. elliptic-relaxation for wp_ij by finite elements every
// step; wp_ij then gives the GLM drift G_ij and C0 eps (Eqs. Gij, C0). Here
// a 10 -> 64 -> 64 -> 64 -> 5 SiLU network maps local node quantities (wall
// distance, k, eps, the mean velocity gradient and the in-plane Reynolds
// stresses) to wp_ij / eps. This file holds:
//  * training: a tiled FP32 GEMM and the element-wise kernels of the forward
//    pass, the backward pass of the mean-squared error, and Adam;
//  * harvesting of (features, targets) at the free canonical nodes;
//  * node inference with bfloat16-rounded weights and FP32 accumulation, the
//    FE residual of its wp, and the device-side decision whether the CG runs;
//  * the lagged FE mode: the previous solution put under the same residual
//    check, so the FE solve runs only when the statistics have moved it.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "mlp_tc.cuh"
#include "pdf_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int IN = PDF_MLP_IN, H = PDF_MLP_HIDDEN, OUT = PDF_MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * H, OFF_W4 = OFF_B3 + H, OFF_B4 = OFF_W4 + OUT * H;
static_assert(OFF_B4 + OUT == PDF_MLP_NPARAM, "parameter layout");
constexpr int NC = 5;
constexpr int LOSS_BLOCKS = 1024;

__device__ __forceinline__ float sigm(float z) { return 1.f / (1.f + expf(-z)); }
__device__ __forceinline__ float silu(float z) { return z * sigm(z); }
__device__ __forceinline__ float silu_grad(float z) {
    const float s = sigm(z);
    return s * (1.f + z * (1.f - s));
}

// C[M][N] = op(A)[M][K] op(B)[K][N], row-major, FP32. op(A)(m, k) is
// A[m*lda + k] (or A[k*lda + m] with TA); op(B)(k, n) is B[k*ldb + n] (or
// B[n*ldb + k] with TB). 32x32 output tile per 256-thread block.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_sgemm(int M, int N, int K, const float* __restrict__ A, int lda,
                                               const float* __restrict__ B, int ldb, float* C, int ldc) {
    __shared__ float As[32][33], Bs[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int r = ty; r < 32; r += 8) {
            const int m = m0 + r, k = k0 + tx;
            As[r][tx] = (m < M && k < K) ? (TA ? A[(size_t)k * lda + m] : A[(size_t)m * lda + k]) : 0.f;
            const int kk = k0 + r, n = n0 + tx;
            Bs[r][tx] = (kk < K && n < N) ? (TB ? B[(size_t)n * ldb + kk] : B[(size_t)kk * ldb + n]) : 0.f;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            const float b = Bs[kk][tx];
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[j] = fmaf(As[ty + 8 * j][kk], b, acc[j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int m = m0 + ty + 8 * j, n = n0 + tx;
        if (m < M && n < N) C[(size_t)m * ldc + n] = acc[j];
    }
}

// Z[r][o] += b[o]; A = SiLU(Z) (act) or A = Z
__global__ void k_bias_act(float* Z, float* A, int64_t n, int d, const float* __restrict__ b, int act) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * d) return;
    const float z = Z[i] + b[i % d];
    Z[i] = z;
    if (A) A[i] = act ? silu(z) : z;
}

// dZ = dA * SiLU'(Z)
__global__ void k_silu_bwd(const float* __restrict__ dA, const float* __restrict__ Z, float* dZ, int64_t count) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dZ[i] = dA[i] * silu_grad(Z[i]);
}

// db[col] = sum over rows of dZ[row][col] (block per column, fixed order)
__global__ void __launch_bounds__(256) k_colsum(const float* __restrict__ dZ, int64_t n, int d, float* db) {
    __shared__ float red[256];
    const int col = blockIdx.x;
    float s = 0.f;
    for (int64_t r = threadIdx.x; r < n; r += 256) s += dZ[r * d + col];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[col] = red[0];
}

// dY = 2 (Y - T) / (5 n); per-block partial sums of (Y - T)^2
__global__ void __launch_bounds__(256) k_mse(const float* __restrict__ Y, const float* __restrict__ T, int64_t count,
                                             float scale, float* dY, float* part) {
    __shared__ float red[256];
    float s = 0.f;
    for (int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x; i < count; i += (int64_t)gridDim.x * 256) {
        const float e = Y[i] - T[i];
        dY[i] = 2.f * e * scale;
        s += e * e;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_loss_final(const float* __restrict__ part, int nb, float scale, float* loss) {
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int b = 0; b < nb; ++b) s += part[b];
        *loss = (float)(s * scale);
    }
}

__global__ void k_adam(float* p, const float* __restrict__ g, float* m, float* v, int count, float lr, float b1,
                       float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_bf16_round(const float* __restrict__ src, float* dst, int count) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) dst[i] = __bfloat162float(__float2bfloat16_rn(src[i]));
}

// column mean and standard deviation, FP64 sums in a fixed order
__global__ void __launch_bounds__(256) k_colstats(const float* __restrict__ X, int64_t n, int d, float* mean,
                                                  float* sd) {
    __shared__ double red[256];
    __shared__ double mu;
    const int col = blockIdx.x;
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += 256) s += X[r * d + col];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) mu = n > 0 ? red[0] / (double)n : 0.0;
    __syncthreads();
    const double m = mu;
    s = 0.0;
    for (int64_t r = threadIdx.x; r < n; r += 256) {
        const double e = X[r * d + col] - m;
        s += e * e;
    }
    __syncthreads();
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double sdev = n > 0 ? sqrt(red[0] / (double)n) : 0.0;
        mean[col] = (float)m;
        sd[col] = (float)(sdev > 1e-12 ? sdev : 1e-12);
    }
}

__global__ void k_gather_rows(const float* __restrict__ src, const int* __restrict__ idx, int n, int d, float* dst) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (int64_t)n * d) return;
    const int r = (int)(i / d), j = (int)(i % d);
    dst[i] = src[(size_t)idx[r] * d + j];
}

__global__ void k_standardize(float* X, int64_t n, int d, const float* __restrict__ mean,
                              const float* __restrict__ sd) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n * d) return;
    const int j = (int)(i % d);
    X[i] = (X[i] - mean[j]) / sd[j];
}

unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <bool TA, bool TB>
void gemm(int M, int N, int K, const float* A, int lda, const float* B, int ldb, float* C, int ldc, cudaStream_t s) {
    dim3 grid((N + 31) / 32, (M + 31) / 32);
    k_sgemm<TA, TB><<<grid, 256, 0, s>>>(M, N, K, A, lda, B, ldb, C, ldc);
}

struct Work {
    float *Z1, *A1, *Z2, *A2, *Z3, *A3, *Y, *dY, *dA, *dZ, *wq, *lpart;
    Work(float* w, int64_t n) {
        Z1 = w; A1 = Z1 + H * n; Z2 = A1 + H * n; A2 = Z2 + H * n; Z3 = A2 + H * n; A3 = Z3 + H * n;
        Y = A3 + H * n; dY = Y + OUT * n; dA = dY + OUT * n; dZ = dA + H * n;
        wq = dZ + H * n; lpart = wq + PDF_MLP_NPARAM + 3;
    }
};

void forward(const float* P, const float* X, int n, Work& w, float* Y, cudaStream_t s) {
    const unsigned bh = blocks_for((int64_t)n * H, 256);
    gemm<false, true>(n, H, IN, X, IN, P + OFF_W1, IN, w.Z1, H, s);
    k_bias_act<<<bh, 256, 0, s>>>(w.Z1, w.A1, n, H, P + OFF_B1, 1);
    gemm<false, true>(n, H, H, w.A1, H, P + OFF_W2, H, w.Z2, H, s);
    k_bias_act<<<bh, 256, 0, s>>>(w.Z2, w.A2, n, H, P + OFF_B2, 1);
    gemm<false, true>(n, H, H, w.A2, H, P + OFF_W3, H, w.Z3, H, s);
    k_bias_act<<<bh, 256, 0, s>>>(w.Z3, w.A3, n, H, P + OFF_B3, 1);
    gemm<false, true>(n, OUT, H, w.A3, H, P + OFF_W4, H, Y, OUT, s);
    k_bias_act<<<blocks_for((int64_t)n * OUT, 256), 256, 0, s>>>(Y, nullptr, n, OUT, P + OFF_B4, 0);
}

}  // namespace

extern "C" {

int64_t pdf_mlp_work_floats(int32_t n) {
    if (n < 0) return -1;
    return (int64_t)(6 * H + 2 * OUT + 2 * H) * n + PDF_MLP_NPARAM + 3 + LOSS_BLOCKS + 64;
}

int pdf_mlp_forward(const float* params, const float* X, int32_t n, float* Y, float* work, int32_t bf16_weights,
                    void* cuda_stream) {
    if (!params || !work || n < 0 || (n > 0 && (!X || !Y)))
        return fail(nullptr, PDF_ERR_ARG, "pdf_mlp_forward: NULL array or n < 0");
    if (n == 0) return PDF_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Work w(work, n);
    const float* P = params;
    if (bf16_weights) {
        k_bf16_round<<<blocks_for(PDF_MLP_NPARAM, 256), 256, 0, s>>>(params, w.wq, PDF_MLP_NPARAM);
        P = w.wq;
    }
    forward(P, X, n, w, Y, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, PDF_ERR_CUDA, std::string("pdf_mlp_forward: ") + cudaGetErrorString(e));
    return PDF_OK;
}

int pdf_mlp_loss_grad(const float* params, const float* X, const float* T, int32_t n, float* work, float* grad,
                      float* loss, void* cuda_stream) {
    if (!params || !work || !grad || !loss || n < 1 || !X || !T)
        return fail(nullptr, PDF_ERR_ARG, "pdf_mlp_loss_grad: NULL array or n < 1");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    Work w(work, n);
    const float* P = params;
    forward(P, X, n, w, w.Y, s);
    const int64_t ny = (int64_t)n * OUT;
    const int nb = (int)std::min<int64_t>(LOSS_BLOCKS, (ny + 255) / 256);
    const float scale = 1.f / (float)ny;
    k_mse<<<nb, 256, 0, s>>>(w.Y, T, ny, scale, w.dY, w.lpart);
    k_loss_final<<<1, 32, 0, s>>>(w.lpart, nb, (float)(1.0 / (double)ny), loss);
    // layer 4: dW4 = dY^T A3, db4 = colsum dY, dA3 = dY W4
    gemm<true, false>(OUT, H, n, w.dY, OUT, w.A3, H, grad + OFF_W4, H, s);
    k_colsum<<<OUT, 256, 0, s>>>(w.dY, n, OUT, grad + OFF_B4);
    gemm<false, false>(n, H, OUT, w.dY, OUT, P + OFF_W4, H, w.dA, H, s);
    const unsigned bh = blocks_for((int64_t)n * H, 256);
    // layer 3
    k_silu_bwd<<<bh, 256, 0, s>>>(w.dA, w.Z3, w.dZ, (int64_t)n * H);
    gemm<true, false>(H, H, n, w.dZ, H, w.A2, H, grad + OFF_W3, H, s);
    k_colsum<<<H, 256, 0, s>>>(w.dZ, n, H, grad + OFF_B3);
    gemm<false, false>(n, H, H, w.dZ, H, P + OFF_W3, H, w.dA, H, s);
    // layer 2
    k_silu_bwd<<<bh, 256, 0, s>>>(w.dA, w.Z2, w.dZ, (int64_t)n * H);
    gemm<true, false>(H, H, n, w.dZ, H, w.A1, H, grad + OFF_W2, H, s);
    k_colsum<<<H, 256, 0, s>>>(w.dZ, n, H, grad + OFF_B2);
    gemm<false, false>(n, H, H, w.dZ, H, P + OFF_W2, H, w.dA, H, s);
    // layer 1
    k_silu_bwd<<<bh, 256, 0, s>>>(w.dA, w.Z1, w.dZ, (int64_t)n * H);
    gemm<true, false>(H, IN, n, w.dZ, H, X, IN, grad + OFF_W1, IN, s);
    k_colsum<<<H, 256, 0, s>>>(w.dZ, n, H, grad + OFF_B1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, PDF_ERR_CUDA, std::string("pdf_mlp_loss_grad: ") + cudaGetErrorString(e));
    return PDF_OK;
}

int pdf_mlp_adam(float* params, const float* grad, float* m, float* v, int32_t t, float lr, float beta1,
                 float beta2, float eps, void* cuda_stream) {
    if (!params || !grad || !m || !v || t < 1) return fail(nullptr, PDF_ERR_ARG, "pdf_mlp_adam: bad argument");
    const float c1 = 1.f - powf(beta1, (float)t), c2 = 1.f - powf(beta2, (float)t);
    k_adam<<<blocks_for(PDF_MLP_NPARAM, 256), 256, 0, (cudaStream_t)cuda_stream>>>(
        params, grad, m, v, PDF_MLP_NPARAM, lr, beta1, beta2, eps, c1, c2);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, PDF_ERR_CUDA, std::string("pdf_mlp_adam: ") + cudaGetErrorString(e));
    return PDF_OK;
}

int pdf_mlp_column_stats(const float* X, int64_t n, int32_t d, float* mean, float* std, void* cuda_stream) {
    if (!X || !mean || !std || n < 1 || d < 1) return fail(nullptr, PDF_ERR_ARG, "pdf_mlp_column_stats: bad argument");
    k_colstats<<<d, 256, 0, (cudaStream_t)cuda_stream>>>(X, n, d, mean, std);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, PDF_ERR_CUDA, std::string("pdf_mlp_column_stats: ") + cudaGetErrorString(e));
    return PDF_OK;
}

int pdf_mlp_gather_rows(const float* src, const int32_t* idx, int32_t n, int32_t d, float* dst, void* cuda_stream) {
    if (!src || !idx || !dst || n < 0 || d < 1) return fail(nullptr, PDF_ERR_ARG, "pdf_mlp_gather_rows: bad argument");
    if (n == 0) return PDF_OK;
    k_gather_rows<<<blocks_for((int64_t)n * d, 256), 256, 0, (cudaStream_t)cuda_stream>>>(src, idx, n, d, dst);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, PDF_ERR_CUDA, std::string("pdf_mlp_gather_rows: ") + cudaGetErrorString(e));
    return PDF_OK;
}

int pdf_mlp_standardize(float* X, int64_t n, int32_t d, const float* mean, const float* std, void* cuda_stream) {
    if (!X || !mean || !std || n < 0 || d < 1) return fail(nullptr, PDF_ERR_ARG, "pdf_mlp_standardize: bad argument");
    if (n == 0) return PDF_OK;
    k_standardize<<<blocks_for(n * d, 256), 256, 0, (cudaStream_t)cuda_stream>>>(X, n, d, mean, std);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(nullptr, PDF_ERR_CUDA, std::string("pdf_mlp_standardize: ") + cudaGetErrorString(e));
    return PDF_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// the surrogate inside a context: features, node inference, FE residual check
// ---------------------------------------------------------------------------
namespace {


struct SurArgs {
    int nn;
    const int* __restrict__ rep;
    const unsigned char* __restrict__ is_wall;
    const double* __restrict__ wdist;
    const double* __restrict__ nke;
    const double* __restrict__ ngrad;
    const double* __restrict__ nR;
};

// features at node i: log d, log k, log eps, (k/eps) grad <U>, R/k. The
// network's inputs are FP32, so they are formed in FP32 from the FP64 node
// fields (one warp evaluates a node: FP64 work on every lane would saturate
// GB300's FP64 pipe).
__device__ void node_features(const SurArgs& a, int i, float f[IN], double& eps) {
    const double dd = a.wdist[i];
    const float d = dd > 1e-6 ? (float)dd : 1e-6f;
    const float k = (float)a.nke[2 * i];
    eps = a.nke[2 * i + 1];
    const float e = (float)eps;
    const float tau = k / e, ik = 1.f / k;
    f[0] = logf(d);
    f[1] = logf(k);
    f[2] = logf(e);
#pragma unroll
    for (int q = 0; q < 4; ++q) f[3 + q] = tau * (float)a.ngrad[4 * i + q];
    f[7] = (float)a.nR[6 * i + 0] * ik;
    f[8] = (float)a.nR[6 * i + 3] * ik;
    f[9] = (float)a.nR[6 * i + 1] * ik;
}

// node pack of the per-particle form: standardised features, then k, eps,
// uu, vv, ww, uv (every node: the particle kernel interpolates over elements)
__global__ void k_sur_featpack(SurArgs a, const float* __restrict__ nm, float* pack) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.nn) return;
    float f[IN];
    double eps;
    node_features(a, i, f, eps);
    float* o = pack + 16 * (size_t)i;
#pragma unroll
    for (int q = 0; q < IN; ++q) o[q] = (f[q] - nm[q]) / nm[IN + q];
    o[10] = (float)a.nke[2 * i];
    o[11] = (float)eps;
    o[12] = (float)a.nR[6 * i + 0];
    o[13] = (float)a.nR[6 * i + 1];
    o[14] = (float)a.nR[6 * i + 2];
    o[15] = (float)a.nR[6 * i + 3];
}

__global__ void k_sur_harvest(SurArgs a, int nrows, const int* __restrict__ rows, const double* __restrict__ wp,
                              float* X, float* T) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nrows) return;
    const int i = rows[r];
    float f[IN];
    double eps;
    node_features(a, i, f, eps);
#pragma unroll
    for (int q = 0; q < IN; ++q) X[(size_t)IN * r + q] = f[q];
#pragma unroll
    for (int q = 0; q < OUT; ++q) T[(size_t)OUT * r + q] = (float)(wp[NC * (size_t)i + q] / eps);
}

// wp at the canonical nodes: the network at the free ones (tensor cores, one
// CTA of 128 threads per 128 nodes, thread t: node row t), the Dirichlet value
// at the walls.
constexpr int TC_M = mlptc::TILE_ROWS;

struct TcSmem {
    __align__(128) uint16_t A[mlptc::TILE_ELEMS];
    mlptc::Weights W;
    __align__(8) uint64_t bar;
    uint32_t tmem;
};

// x = eps y(x) at the free canonical nodes (the Dirichlet values g at the
// walls); with base and snap (mode 6), x = base + eps y - snap, and eps y is
// also written to yout
__global__ void __launch_bounds__(TC_M) k_sur_nodes(SurArgs a, const float* __restrict__ wq,
                                                    const double* __restrict__ g, double* x, int* status,
                                                    const double* __restrict__ base = nullptr,
                                                    const double* __restrict__ snap = nullptr,
                                                    double* yout = nullptr) {
    __shared__ TcSmem S;
    const int t = threadIdx.x, warp = t >> 5;
    mlptc::load(S.W, wq, t, TC_M);
    if (t == 0) tc::mbar_init(&S.bar, 1);
    __syncwarp();
    if (warp == 0) tc::tmem_alloc(&S.tmem, 64);
    __syncthreads();
    const int i = blockIdx.x * TC_M + t;
    const bool row = i < a.nn && a.rep[i] == i;
    const bool net = row && !a.is_wall[i];
    double eps = 0.0;
    {
        float f[IN], in[16];
        if (net) node_features(a, i, f, eps);
#pragma unroll
        for (int k = 0; k < 16; ++k) in[k] = (net && k < IN) ? (f[k] - S.W.nm[k]) / S.W.nm[IN + k] : 0.f;
        mlptc::put_inputs(S.A, t, in);
    }
    const uint32_t tmem = S.tmem;
    unsigned phase = 0;
    float y[16];
    const bool ok = mlptc::run(S.W, S.A, 1, tmem, &S.bar, phase, y);
    if (ok && net) {
#pragma unroll
        for (int o = 0; o < OUT; ++o) {
            const double yo = (double)y[o] * S.W.nm[2 * IN + OUT + o] + S.W.nm[2 * IN + o];
            const size_t q = NC * (size_t)i + o;
            if (base) {
                yout[q] = eps * yo;
                x[q] = base[q] + (eps * yo - snap[q]);
            } else {
                x[q] = eps * yo;
            }
        }
    }
    if (!ok && t == 0) set_status(status, ST_BARRIER);
    if (row && !net) {
#pragma unroll
        for (int q = 0; q < NC; ++q) x[NC * (size_t)i + q] = g[NC * (size_t)i + q];
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem, 64);
    }
}

struct ResArgs {
    int nn;
    const int* __restrict__ rowptr;
    const int* __restrict__ colidx;
    const double* __restrict__ mval;
    const double* __restrict__ aval;  // assembled M + K_{L^2}
    const int* __restrict__ rep;
    const unsigned char* __restrict__ is_wall;
    const double* __restrict__ f;
    const double* __restrict__ x;
    double* part;  // [gridDim][4 NC]: sum r^2, sum b0^2, sum r, sum b0 per component
    unsigned* done;  // blocks finished (the last one decides, then resets it)
    int mode;
    double tol;
    int* skip;
    unsigned long long* cnt;
    double* last;
};

constexpr int RES_ROWS = 128;

// r = M f - A x over the free rows (x holds the Dirichlet values at the walls),
// b0 = M f - A_wall g; block partial sums of r^2, b0^2 (fine norm) and of r,
// b0 (the coarse residual: one aggregate per block of RES_ROWS Morton-ordered
// nodes, which averages out the node-to-node noise of the estimated
// statistics), in a fixed order
__global__ void __launch_bounds__(RES_ROWS) k_sur_residual(ResArgs a) {
    __shared__ double red[4 * NC][RES_ROWS / 32];
    const int t = threadIdx.x, i = blockIdx.x * RES_ROWS + t;
    // 32 slots per thread for the butterfly below: 0..4 r^2, 5..9 b0^2,
    // 10..14 r, 15..19 b0, 20..31 zero
    double val[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) val[k] = 0.0;
    if (i < a.nn && a.rep[i] == i && !a.is_wall[i]) {
        double b[NC] = {0, 0, 0, 0, 0}, s[NC] = {0, 0, 0, 0, 0}, sw[NC] = {0, 0, 0, 0, 0};
        const int qa = a.rowptr[i], q1 = a.rowptr[i + 1];
        bool touch = false;  // a column of the row is a wall node
        for (int q0 = qa; q0 < q1; q0 += 4) {
            // four entries at a time: their column loads, then their value
            // loads, are issued together (latency, not bandwidth, bounds this)
            int j4[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) j4[k] = q0 + k < q1 ? a.colidx[q0 + k] : -1;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (j4[k] < 0) break;
                const int j = j4[k];
                const double A = a.aval[q0 + k], M = a.mval[q0 + k];
                touch |= a.is_wall[j] != 0;
                // fused multiply-adds: GB300's FP64 pipe is narrow
#pragma unroll
                for (int c = 0; c < NC; ++c) {
                    b[c] = fma(M, a.f[NC * (size_t)j + c], b[c]);
                    s[c] = fma(A, a.x[NC * (size_t)j + c], s[c]);
                }
            }
        }
        if (touch) {  // the wall-column sum, on the few rows beside a wall
            for (int q = qa; q < q1; ++q) {
                const int j = a.colidx[q];
                if (!a.is_wall[j]) continue;
                const double A = a.aval[q];
#pragma unroll
                for (int c = 0; c < NC; ++c) sw[c] = fma(A, a.x[NC * (size_t)j + c], sw[c]);
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const double r = b[c] - s[c], b0 = b[c] - sw[c];
            val[c] = r * r;
            val[NC + c] = b0 * b0;
            val[2 * NC + c] = r;
            val[3 * NC + c] = b0;
        }
    }
    // warp sums of the 20 values by a butterfly reduce-scatter: at the xor-o
    // exchange a lane keeps the half of its w slots selected by its lane bit
    // o and adds the partner's copy of that half; lane l ends with the warp
    // sum of value l (a fixed order of additions)
    const int lane = t & 31, wid = t >> 5;
#pragma unroll
    for (int w = 16, o = 16; w >= 1; w >>= 1, o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int k = 0; k < w; ++k) {
            const double send = upper ? val[k] : val[w + k];
            const double keep = upper ? val[w + k] : val[k];
            val[k] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    if (lane < 4 * NC) red[lane][wid] = val[0];
    __syncthreads();
    if (t < 4 * NC) {
        double sum = 0.0;
#pragma unroll
        for (int w = 0; w < RES_ROWS / 32; ++w) sum += red[t][w];
        a.part[(size_t)blockIdx.x * 4 * NC + t] = sum;
    }
    // the last block to finish reduces all partials and takes the decision
    __shared__ bool last_block;
    __threadfence();
    __syncthreads();
    if (t == 0) last_block = atomicAdd(a.done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (last_block) {
        // 6 groups of 20 threads: thread (grp, v) sums value v over the blocks
        // b = grp, grp + 6, ... (squared for the coarse sums), in a fixed order
        __threadfence();
        __shared__ double acc6[6][4 * NC];
        const int grp = t / (4 * NC), v = t % (4 * NC);
        if (grp < 6) {
            // the partials of eight blocks are loaded together, then added in
            // block order
            double sacc = 0.0;
            const int nbk = (int)gridDim.x;
            for (int b0 = grp; b0 < nbk; b0 += 6 * 8) {
                double q8[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const int b = b0 + 6 * k;
                    q8[k] = b < nbk ? a.part[(size_t)b * 4 * NC + v] : 0.0;
                }
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    if (b0 + 6 * k >= nbk) break;
                    sacc += v < 2 * NC ? q8[k] : q8[k] * q8[k];
                }
            }
            acc6[grp][v] = sacc;
        }
        __syncthreads();
        __shared__ double tot[4 * NC];
        if (t < 4 * NC) {
            double sacc = 0.0;
#pragma unroll
            for (int g2 = 0; g2 < 6; ++g2) sacc += acc6[g2][t];
            tot[t] = sacc;
        }
        __syncthreads();
        if (t < 32) {
            // lane c < NC forms the squared fine and coarse ratios of
            // component c (every lane at once: a serial FP64 chain in one
            // thread costs tens of microseconds on the narrow FP64 pipe); the
            // largest ratio by shuffles, then one square root each, which
            // equals the largest of the square roots. A NaN fails the check.
            double xf = 0.0, xg = 0.0;
            if (t < NC) {
                const double rr = tot[t], bb = tot[NC + t], cr = tot[2 * NC + t], cb = tot[3 * NC + t];
                xf = bb > 0.0 ? rr / bb : rr;
                xg = cb > 0.0 ? cr / cb : cr;
            }
            const bool bad = __any_sync(0xffffffffu, !(xf == xf) || !(xg == xg));
#pragma unroll
            for (int o = 4; o >= 1; o >>= 1) {
                xf = fmax(xf, __shfl_xor_sync(0xffffffffu, xf, o));
                xg = fmax(xg, __shfl_xor_sync(0xffffffffu, xg, o));
            }
            const double qnan = __longlong_as_double(0x7ff8000000000000ll);
            const double fine = bad ? qnan : sqrt(xf), coarse = bad ? qnan : sqrt(xg);
            const int ok = (a.mode == 2) || (coarse <= a.tol);
            if (t == 0) {
                *a.skip = ok;
                a.last[0] = coarse;
                a.last[1] = fine;
                a.cnt[0] += 1ull;
                a.cnt[1] += ok ? 0ull : 1ull;
                *a.done = 0u;
            }
        }
    }
}

SurArgs sur_args(pdf_ctx* c) {
    SurArgs a;
    a.nn = c->m.nn; a.rep = c->m.rep; a.is_wall = c->m.is_wall; a.wdist = c->m.wdist;
    a.nke = c->nke; a.ngrad = c->ngrad; a.nR = c->nR;
    return a;
}

int sur_blocks(pdf_ctx* c) { return (c->m.nn + RES_ROWS - 1) / RES_ROWS; }

}  // namespace

int surrogate_rows(pdf_ctx* c) {
    if (c->sur_rows) return PDF_OK;
    const int nn = c->m.nn;
    std::vector<int> rep(nn);
    std::vector<unsigned char> wall(nn);
    PDF_CUDA(c, cudaStreamSynchronize(c->s));
    PDF_CUDA(c, cudaMemcpy(rep.data(), c->m.rep, sizeof(int) * nn, cudaMemcpyDeviceToHost));
    PDF_CUDA(c, cudaMemcpy(wall.data(), c->m.is_wall, nn, cudaMemcpyDeviceToHost));
    std::vector<int> rows;
    for (int i = 0; i < nn; ++i)
        if (rep[i] == i && !wall[i]) rows.push_back(i);
    PDF_CUDA(c, cudaMalloc((void**)&c->sur_rows, sizeof(int) * (rows.size() + 1)));
    PDF_CUDA(c, cudaMemcpy(c->sur_rows, rows.data(), sizeof(int) * rows.size(), cudaMemcpyHostToDevice));
    c->sur_nrows = (int)rows.size();
    return PDF_OK;
}

int launch_surrogate(pdf_ctx* c) {
    const int nn = c->m.nn;
    const SurArgs a = sur_args(c);
    // lagged FE mode: the right-hand-side kernel has written the proposal
    // (the previous solution, the Dirichlet values at the walls)
    if (c->sur_mode == 6) {
        k_sur_nodes<<<(nn + TC_M - 1) / TC_M, TC_M, 0, c->s>>>(a, c->sur_w, c->fe_g, c->fe_prop, c->d_status,
                                                               c->sur_base, c->sur_snap, c->sur_y);
        ++c->launches;
    } else if (c->sur_mode != 5) {
        k_sur_nodes<<<(nn + TC_M - 1) / TC_M, TC_M, 0, c->s>>>(a, c->sur_w, c->fe_g, c->fe_prop, c->d_status);
        ++c->launches;
    }
    ResArgs r;
    r.nn = nn; r.rowptr = c->m.rowptr; r.colidx = c->m.colidx; r.mval = c->m.mval; r.aval = c->m.aval;
    r.rep = c->m.rep; r.is_wall = c->m.is_wall;
    r.f = c->fe_f; r.x = c->fe_prop; r.part = c->sur_part;
    const int nb = sur_blocks(c);
    r.done = reinterpret_cast<unsigned*>(c->sur_part + (size_t)nb * 4 * NC + 2);
    r.mode = c->sur_mode;
    r.tol = c->sur_tol;
    r.skip = c->sur_skip;
    r.cnt = c->sur_cnt;
    r.last = c->sur_part + (size_t)nb * 4 * NC;
    k_sur_residual<<<nb, RES_ROWS, 0, c->s>>>(r);
    ++c->launches;
    if (c->sur_mode == 3 || c->sur_mode == 4) {
        k_sur_featpack<<<(nn + 127) / 128, 128, 0, c->s>>>(a, c->sur_w + PDF_MLP_NPARAM, c->nsurT);
        ++c->launches;
    }
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

// mode 6, after the CG: where the check rejected the proposal (the FE solve
// ran), that solution and this step's network values become the reference
__global__ void k_sur_rebase(const int* __restrict__ skip, const double* __restrict__ wp, const double* __restrict__ y,
                             double* base, double* snap, int64_t n) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n || *(volatile const int*)skip != 0) return;
    base[t] = wp[t];
    snap[t] = y[t];
}

int launch_surrogate_rebase(pdf_ctx* c) {
    if (c->sur_mode != 6) return PDF_OK;
    const int64_t n = (int64_t)NC * c->m.nn;
    k_sur_rebase<<<(unsigned)((n + 255) / 256), 256, 0, c->s>>>(c->sur_skip, c->nwp, c->sur_y, c->sur_base,
                                                                 c->sur_snap, n);
    ++c->launches;
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

extern "C" {

int32_t pdf_surrogate_rows(const pdf_ctx* c) {
    if (!c || c->p.wall_model != PDF_ELLIPTIC_RELAXATION) return -1;
    if (surrogate_rows(const_cast<pdf_ctx*>(c)) != PDF_OK) return -1;
    return c->sur_nrows;
}

int pdf_surrogate_harvest(pdf_ctx* c, float* X, float* T) {
    if (!c || !X || !T) return PDF_ERR_ARG;
    if (c->p.wall_model != PDF_ELLIPTIC_RELAXATION) return fail(c, PDF_ERR_ARG, "harvest needs elliptic relaxation");
    if (!c->stats_valid) return fail(c, PDF_ERR_STATE, "statistics not estimated");
    const int st = surrogate_rows(c);
    if (st != PDF_OK) return st;
    if (c->sur_nrows == 0) return PDF_OK;
    k_sur_harvest<<<(c->sur_nrows + 127) / 128, 128, 0, c->s>>>(sur_args(c), c->sur_nrows, c->sur_rows, c->nwp, X, T);
    ++c->launches;
    PDF_CUDA(c, cudaGetLastError());
    return PDF_OK;
}

int pdf_set_surrogate(pdf_ctx* c, int32_t mode, const float* params, const float* norm, double residual_tol) {
    if (!c) return PDF_ERR_ARG;
    if (mode < 0 || mode > 6) return fail(c, PDF_ERR_ARG, "surrogate mode must be 0 .. 6");
    if (mode == 6 && !c->stats_valid) return fail(c, PDF_ERR_STATE, "surrogate mode 6: statistics not estimated");
    if ((mode == 3 || mode == 4) && c->prec == 0) return fail(c, PDF_ERR_ARG, "the per-particle surrogate needs an FP32 state");
    if (mode == 0) {
        c->sur_mode = 0;
        return PDF_OK;
    }
    if (c->p.wall_model != PDF_ELLIPTIC_RELAXATION) return fail(c, PDF_ERR_ARG, "surrogate needs elliptic relaxation");
    if (!(residual_tol >= 0)) return fail(c, PDF_ERR_ARG, "surrogate: bad tolerance");
    if (mode != 5 && (!params || !norm)) return fail(c, PDF_ERR_ARG, "surrogate: NULL array");
    for (int q = 0; q < PDF_MLP_NNORM && mode != 5; ++q)
        if (!std::isfinite(norm[q]) || (((q >= IN && q < 2 * IN) || q >= 2 * IN + OUT) && !(norm[q] > 0.f)))
            return fail(c, PDF_ERR_ARG, "surrogate: standard deviations must be positive and finite");
    if ((mode == 3 || mode == 4) && !c->nsurT) PDF_CUDA(c, cudaMalloc((void**)&c->nsurT, sizeof(float) * 16 * (size_t)c->m.nn));
    if (mode == 4 && c->pwp_n < c->np) {
        cudaFree(c->pwp);
        c->pwp = nullptr;
        c->pwp_n = 0;
        PDF_CUDA(c, cudaMalloc((void**)&c->pwp, sizeof(float) * 5 * (size_t)std::max<int64_t>(c->np, 1)));
        c->pwp_n = c->np;
    }
    if (!c->sur_w) {
        PDF_CUDA(c, cudaMalloc((void**)&c->sur_w, sizeof(float) * (PDF_MLP_NPARAM + PDF_MLP_NNORM)));
        PDF_CUDA(c, cudaMalloc((void**)&c->sur_skip, sizeof(int)));
        PDF_CUDA(c, cudaMalloc((void**)&c->sur_cnt, 2 * sizeof(unsigned long long)));
        PDF_CUDA(c, cudaMalloc((void**)&c->sur_part, sizeof(double) * ((size_t)sur_blocks(c) * 4 * NC + 3)));
    }
    std::vector<float> h(PDF_MLP_NPARAM + PDF_MLP_NNORM, 0.f);
    for (int q = 0; q < PDF_MLP_NPARAM && mode != 5; ++q) h[q] = __bfloat162float(__float2bfloat16_rn(params[q]));
    for (int q = 0; q < PDF_MLP_NNORM && mode != 5; ++q) h[PDF_MLP_NPARAM + q] = norm[q];
    PDF_CUDA(c, cudaStreamSynchronize(c->s));
    PDF_CUDA(c, cudaMemcpy(c->sur_w, h.data(), sizeof(float) * h.size(), cudaMemcpyHostToDevice));
    PDF_CUDA(c, cudaMemset(c->sur_skip, 0, sizeof(int)));
    PDF_CUDA(c, cudaMemset(c->sur_cnt, 0, 2 * sizeof(unsigned long long)));
    PDF_CUDA(c, cudaMemset(c->sur_part, 0, sizeof(double) * ((size_t)sur_blocks(c) * 4 * NC + 3)));
    if (mode == 6) {
        // the first reference: the current wp and the network at the current statistics
        const size_t nb = sizeof(double) * NC * (size_t)c->m.nn;
        if (!c->sur_base) {
            PDF_CUDA(c, cudaMalloc((void**)&c->sur_base, nb));
            PDF_CUDA(c, cudaMalloc((void**)&c->sur_snap, nb));
            PDF_CUDA(c, cudaMalloc((void**)&c->sur_y, nb));
        }
        PDF_CUDA(c, cudaMemcpyAsync(c->sur_base, c->nwp, nb, cudaMemcpyDeviceToDevice, c->s));
        PDF_CUDA(c, cudaMemsetAsync(c->sur_snap, 0, nb, c->s));
        PDF_CUDA(c, cudaMemsetAsync(c->sur_y, 0, nb, c->s));
        const int nn = c->m.nn;
        k_sur_nodes<<<(nn + TC_M - 1) / TC_M, TC_M, 0, c->s>>>(sur_args(c), c->sur_w, c->fe_g, c->sur_snap,
                                                               c->d_status);
        ++c->launches;
        PDF_CUDA(c, cudaGetLastError());
        PDF_CUDA(c, cudaStreamSynchronize(c->s));
    }
    c->sur_mode = mode;
    c->sur_tol = residual_tol;
    return PDF_OK;
}

int pdf_surrogate_stats(pdf_ctx* c, int64_t* solves, int64_t* fallbacks, double last_residual[2]) {
    if (!c || !solves || !fallbacks || !last_residual) return PDF_ERR_ARG;
    *solves = *fallbacks = 0;
    last_residual[0] = last_residual[1] = 0.0;
    if (!c->sur_cnt) return PDF_OK;
    unsigned long long h[2];
    PDF_CUDA(c, cudaStreamSynchronize(c->s));
    PDF_CUDA(c, cudaMemcpy(h, c->sur_cnt, sizeof(h), cudaMemcpyDeviceToHost));
    PDF_CUDA(c, cudaMemcpy(last_residual, c->sur_part + (size_t)sur_blocks(c) * 4 * NC, 2 * sizeof(double),
                           cudaMemcpyDeviceToHost));
    *solves = (int64_t)h[0];
    *fallbacks = (int64_t)h[1];
    return PDF_OK;
}

}  // extern "C"
