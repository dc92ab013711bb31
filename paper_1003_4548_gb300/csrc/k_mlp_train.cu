// k_mlp_train.cu -- loss and gradient of the surrogate network on the
// 5th-generation tensor cores (bfloat16 operands, FP32 accumulation, FP32
// master weights), for training on the method's own harvested runs.
//
// One CTA of 128 threads takes a tile of 128 samples, thread r its row r. The
// forward pass is the inference chain (128 x N x 16 tcgen05 MMAs, FP32
// accumulators in tensor memory, bias and SiLU in the epilogue); the
// pre-activations Z1..Z3 stay in tensor memory for the backward pass. The
// backward pass per layer l (from 4 down to 1) issues two products:
//  * the weight gradient dW_l[o][i] = sum_r dZ_l[r][o] A_{l-1}[r][i] with the
//    tile's samples as the K dimension: A operand dZ_l stored by unit
//    (dZt[o][r], rows o >= out zero, M = 128), B operand A_{l-1} stored by
//    feature (A_{l-1}t[i][r]). A row of ones among the B rows (feature 10 of
//    the inputs, row 64 of the hidden activations) makes the same product
//    give the bias gradient sum_r dZ_l[r][o] in that column;
//  * the input gradient dA_{l-1} = dZ_l W_l (A operand dZ_l by sample, B
//    operand the transposed weights), whose epilogue forms
//    dZ_{l-1} = dA_{l-1} * SiLU'(Z_{l-1} + b_{l-1}).
// Operands are rounded to bfloat16 where they enter a product: the weights,
// the inputs, the hidden activations, dY and every dZ. The weight
// accumulators sit in tensor memory for the whole tile; the epilogue writes
// them as the tile's partial gradient, and a second kernel sums the tiles'
// partials in tile order (deterministic) into the gradient and the loss.
#include <cuda_bf16.h>

#include <string>

#include "mlp_tc.cuh"
#include "pdf_internal.cuh"
#include "tc.cuh"

namespace {

constexpr int IN = PDF_MLP_IN, H = PDF_MLP_HIDDEN, OUT = PDF_MLP_OUT, NP = PDF_MLP_NPARAM;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * H, OFF_W4 = OFF_B3 + H, OFF_B4 = OFF_W4 + OUT * H;
static_assert(OFF_B4 + OUT == NP, "parameter layout");
constexpr int R = 128;     // samples per tile (tensor-memory lanes)
constexpr int HB = H + 16;  // rows of a hidden layer's by-feature operand: 64 features, the ones row, zero padding
constexpr int ONES_IN = IN;  // input column that holds 1 (W1 is zero there)

// tensor-memory columns
constexpr uint32_t TM_Z1 = 0, TM_Z2 = 64, TM_Z3 = 128, TM_YDA = 192;
constexpr uint32_t TM_DW1 = 256, TM_DW2 = 272, TM_DW3 = 352, TM_DW4 = 432, TM_COLS = 512;

struct __align__(128) TrainSmem {
    // weights as B operands of the forward (K-major [out][in])
    __align__(128) uint16_t W1[H * 16];
    __align__(128) uint16_t W2[H * H];
    __align__(128) uint16_t W3[H * H];
    __align__(128) uint16_t W4[16 * H];
    // transposed weights as B operands of the input gradients ([in][out])
    __align__(128) uint16_t W2t[H * H];
    __align__(128) uint16_t W3t[H * H];
    __align__(128) uint16_t W4t[H * 16];
    // activations by sample (A operands of the forward)
    __align__(128) uint16_t A0[R * 16];
    __align__(128) uint16_t A1[R * H];
    __align__(128) uint16_t A2[R * H];
    __align__(128) uint16_t A3[R * H];
    // activations by feature (B operands of the weight gradients, K = sample)
    __align__(128) uint16_t A0t[16 * R];
    __align__(128) uint16_t A1t[HB * R];
    __align__(128) uint16_t A2t[HB * R];
    __align__(128) uint16_t A3t[HB * R];
    // output gradients by sample (A operand of the input gradient) and by unit
    // (A operand of the weight gradient, rows >= out zero)
    __align__(128) uint16_t dZ[R * H];
    __align__(128) uint16_t dZt[R * R];
    float bias[3 * H + 16];
    float lsum[4];
    uint64_t bar;
    uint32_t tmem;
};

__device__ __forceinline__ uint16_t bf(float x) { return mlptc::bf16_bits(x); }
__device__ __forceinline__ float sigmoid(float z) { return __fdividef(1.f, 1.f + __expf(-z)); }
__device__ __forceinline__ float silu_grad(float z) {
    const float s = sigmoid(z);
    return s * (1.f + z * (1.f - s));
}

// element (row, k) of a K-major operand with kc core matrices along K
__device__ __forceinline__ int at(int row, int k, int kc) { return tc::core_offset(row, k, kc); }

// issue the MMAs of one phase (thread 0) after the generic-proxy writes of
// every thread, then wait for them; false if the wait ran out
template <typename F>
__device__ __forceinline__ bool phase(TrainSmem& S, unsigned& ph, F issue) {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x == 0) {
        tc::fence_after_sync();
        issue();
        tc::commit(&S.bar);
    }
    const bool ok = __syncthreads_and(tc::mbar_wait(&S.bar, ph & 1u) ? 1 : 0) != 0;
    ++ph;
    tc::fence_after_sync();
    return ok;
}

// D (+)= A B^T over K = 16 ks, both K-major with kca / kcb core matrices along K
__device__ __forceinline__ void mma_k(uint32_t d, const uint16_t* A, int kca, const uint16_t* B, int kcb, int N, int ks,
                                      bool acc) {
    const uint32_t idesc = tc::idesc_bf16(R, N);
    for (int j = 0; j < ks; ++j) {
        const uint64_t ad = tc::smem_desc(A + j * 128, 128, (uint32_t)kca * 128);
        const uint64_t bd = tc::smem_desc(B + j * 128, 128, (uint32_t)kcb * 128);
        tc::mma_bf16(d, ad, bd, idesc, (acc || j > 0) ? 1u : 0u);
    }
}

// forward epilogue of hidden layer l (0-based): Z (+ bias) -> SiLU -> the
// activations by sample (next layer's A) and by feature (the weight gradient's B)
__device__ __forceinline__ void fwd_epilogue(const TrainSmem& S, uint32_t tz, const float* bias, uint16_t* Aout,
                                             uint16_t* Atout, int row) {
    for (int c0 = 0; c0 < H; c0 += 16) {
        float v[16];
        tc::ld16(tz + (uint32_t)c0, v);
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = mlptc::silu(v[k] + bias[c0 + k]);
        mlptc::put8(Aout, row, c0, 8, v);
        mlptc::put8(Aout, row, c0 + 8, 8, v + 8);
#pragma unroll
        for (int k = 0; k < 16; ++k) Atout[at(c0 + k, row, R / 8)] = bf(v[k]);
    }
}

// backward epilogue: dZ = dA * SiLU'(Z + b) into dZ (by sample, unless null)
// and dZt (by unit)
__device__ __forceinline__ void bwd_epilogue(TrainSmem& S, uint32_t tda, uint32_t tz, const float* bias, int row,
                                             bool by_sample) {
    for (int c0 = 0; c0 < H; c0 += 16) {
        float da[16], z[16];
        tc::ld16(tda + (uint32_t)c0, da);
        tc::ld16(tz + (uint32_t)c0, z);
#pragma unroll
        for (int k = 0; k < 16; ++k) da[k] *= silu_grad(z[k] + bias[c0 + k]);
        if (by_sample) {
            mlptc::put8(S.dZ, row, c0, 8, da);
            mlptc::put8(S.dZ, row, c0 + 8, 8, da + 8);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) S.dZt[at(c0 + k, row, R / 8)] = bf(da[k]);
    }
}

// read a weight-gradient accumulator (row = output unit, ncols columns: the
// in-unit gradients, then the bias column) into the tile's partial gradient
__device__ __forceinline__ void put_grad(uint32_t tw, int ncols, int nin, int nout, int ow, int ob, int row,
                                         float* part) {
    for (int c0 = 0; c0 < ncols; c0 += 16) {
        float v[16];
        tc::ld16(tw + (uint32_t)c0, v);
        if (row < nout) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
                const int i = c0 + k;
                if (i < nin) part[ow + nin * row + i] = v[k];
                else if (i == nin) part[ob + row] = v[k];
            }
        }
    }
}

__global__ void __launch_bounds__(R, 1) k_mlp_tc_grad(const float* __restrict__ P, const float* __restrict__ X,
                                                       const float* __restrict__ T, int n, float* part,
                                                       float* lpart, int* err) {
    extern __shared__ __align__(128) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    const int t = threadIdx.x, row = t, warp = t >> 5;
    const int r0 = blockIdx.x * R;
    const bool live = r0 + row < n;

    // weights (bf16), biases, constant rows and columns
    for (int q = t; q < H * 16; q += R) {
        const int o = q / 16, i = q % 16;
        S.W1[at(o, i, 2)] = bf(i < IN ? P[OFF_W1 + IN * o + i] : 0.f);
    }
    for (int q = t; q < H * H; q += R) {
        const int o = q / H, i = q % H;
        const uint16_t w2 = bf(P[OFF_W2 + q]), w3 = bf(P[OFF_W3 + q]);
        S.W2[at(o, i, 8)] = w2;
        S.W3[at(o, i, 8)] = w3;
        S.W2t[at(i, o, 8)] = w2;
        S.W3t[at(i, o, 8)] = w3;
    }
    for (int q = t; q < 16 * H; q += R) {
        const int o = q / H, i = q % H;
        const uint16_t w4 = bf(o < OUT ? P[OFF_W4 + H * o + i] : 0.f);
        S.W4[at(o, i, 8)] = w4;
        S.W4t[at(i, o, 2)] = w4;
    }
    for (int q = t; q < H; q += R) {
        S.bias[q] = P[OFF_B1 + q];
        S.bias[H + q] = P[OFF_B2 + q];
        S.bias[2 * H + q] = P[OFF_B3 + q];
    }
    if (t < 16) S.bias[3 * H + t] = t < OUT ? P[OFF_B4 + t] : 0.f;
    const uint16_t one = bf(1.f);
    for (int q = t; q < 16 * R; q += R) {  // by-feature rows 64..79 of the hidden layers: ones, then zeros
        const int k = H + q / R, r = q % R;
        const uint16_t v = k == H ? one : (uint16_t)0;
        S.A1t[at(k, r, R / 8)] = v;
        S.A2t[at(k, r, R / 8)] = v;
        S.A3t[at(k, r, R / 8)] = v;
    }
    for (int q = t; q < R * R; q += R) S.dZt[q] = 0;  // rows >= out stay zero
    // the tile's inputs (zero past n; feature 10 is the ones column)
    float tg[OUT];
    {
        float x[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) x[k] = (live && k < IN) ? X[(size_t)(r0 + row) * IN + k] : 0.f;
        x[ONES_IN] = 1.f;
        mlptc::put_inputs(S.A0, row, x);
#pragma unroll
        for (int k = 0; k < 16; ++k) S.A0t[at(k, row, R / 8)] = bf(x[k]);
#pragma unroll
        for (int o = 0; o < OUT; ++o) tg[o] = live ? T[(size_t)(r0 + row) * OUT + o] : 0.f;
    }
    if (t == 0) tc::mbar_init(&S.bar, 1);
    if (warp == 0) tc::tmem_alloc(&S.tmem, TM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tm = S.tmem;
    const uint32_t lanes = (uint32_t)((warp & 3) * 32) << 16;  // this warp's tensor-memory lanes
    const uint32_t tl = tm + lanes;
    unsigned ph = 0;
    bool ok = true;

    // ---- forward
    ok = ok && phase(S, ph, [&] { mma_k(tm + TM_Z1, S.A0, 2, S.W1, 2, H, 1, false); });
    if (ok) fwd_epilogue(S, tl + TM_Z1, S.bias, S.A1, S.A1t, row);
    ok = ok && phase(S, ph, [&] { mma_k(tm + TM_Z2, S.A1, 8, S.W2, 8, H, 4, false); });
    if (ok) fwd_epilogue(S, tl + TM_Z2, S.bias + H, S.A2, S.A2t, row);
    ok = ok && phase(S, ph, [&] { mma_k(tm + TM_Z3, S.A2, 8, S.W3, 8, H, 4, false); });
    if (ok) fwd_epilogue(S, tl + TM_Z3, S.bias + 2 * H, S.A3, S.A3t, row);
    ok = ok && phase(S, ph, [&] { mma_k(tm + TM_YDA, S.A3, 8, S.W4, 8, 16, 4, false); });
    // loss and dY = 2 (Y - T) / (5 n), by sample (16 columns) and by unit
    float l2 = 0.f;
    if (ok) {
        float y[16];
        tc::ld16(tl + TM_YDA, y);
        const float sc = 2.f / (5.f * (float)n);
#pragma unroll
        for (int o = 0; o < 16; ++o) {
            float dy = 0.f;
            if (o < OUT && live) {
                const float e = y[o] + S.bias[3 * H + o] - tg[o];
                l2 = fmaf(e, e, l2);
                dy = sc * e;
            }
            y[o] = dy;
            S.dZt[at(o, row, R / 8)] = bf(dy);
        }
        mlptc::put8(S.dZ, row, 0, 2, y);
        mlptc::put8(S.dZ, row, 8, 2, y + 8);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
    if ((t & 31) == 0) S.lsum[warp] = l2;

    // ---- backward: layer 4, then 3, 2, 1
    ok = ok && phase(S, ph, [&] {
        mma_k(tm + TM_DW4, S.dZt, R / 8, S.A3t, R / 8, HB, R / 16, false);
        mma_k(tm + TM_YDA, S.dZ, 2, S.W4t, 2, H, 1, false);
    });
    if (ok) bwd_epilogue(S, tl + TM_YDA, tl + TM_Z3, S.bias + 2 * H, row, true);
    ok = ok && phase(S, ph, [&] {
        mma_k(tm + TM_DW3, S.dZt, R / 8, S.A2t, R / 8, HB, R / 16, false);
        mma_k(tm + TM_YDA, S.dZ, 8, S.W3t, 8, H, 4, false);
    });
    if (ok) bwd_epilogue(S, tl + TM_YDA, tl + TM_Z2, S.bias + H, row, true);
    ok = ok && phase(S, ph, [&] {
        mma_k(tm + TM_DW2, S.dZt, R / 8, S.A1t, R / 8, HB, R / 16, false);
        mma_k(tm + TM_YDA, S.dZ, 8, S.W2t, 8, H, 4, false);
    });
    if (ok) bwd_epilogue(S, tl + TM_YDA, tl + TM_Z1, S.bias, row, false);
    ok = ok && phase(S, ph, [&] { mma_k(tm + TM_DW1, S.dZt, R / 8, S.A0t, R / 8, 16, R / 16, false); });

    // ---- the tile's partial gradient (rows = output units) and loss
    float* pt = part + (size_t)blockIdx.x * NP;
    if (ok) {
        put_grad(tl + TM_DW1, 16, IN, H, OFF_W1, OFF_B1, row, pt);
        put_grad(tl + TM_DW2, HB, H, H, OFF_W2, OFF_B2, row, pt);
        put_grad(tl + TM_DW3, HB, H, H, OFF_W3, OFF_B3, row, pt);
        put_grad(tl + TM_DW4, HB, H, OUT, OFF_W4, OFF_B4, row, pt);
    }
    if (t == 0) {
        lpart[blockIdx.x] = S.lsum[0] + S.lsum[1] + S.lsum[2] + S.lsum[3];
        if (!ok) atomicExch(err, 1);
    }
    if (!ok && t == 0) tc::mbar_wait(&S.bar, (ph - 1u) & 1u);  // one more bounded wait for MMAs in flight
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tm, TM_COLS);
    }
}

// gradient and loss: the tiles' partials summed in tile order
__global__ void k_mlp_tc_reduce(const float* __restrict__ part, const float* __restrict__ lpart, int ntiles,
                                const int* __restrict__ err, float* grad, float* loss, float lscale) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    const bool bad = *err != 0;
    if (p < NP) {
        float s = 0.f;
        for (int c = 0; c < ntiles; ++c) s += part[(size_t)c * NP + p];
        grad[p] = bad ? __int_as_float(0x7fc00000) : s;
    }
    if (p == 0) {
        float s = 0.f;
        for (int c = 0; c < ntiles; ++c) s += lpart[c];
        *loss = bad ? __int_as_float(0x7fc00000) : s * lscale;
    }
}

}  // namespace

extern "C" {

int pdf_mlp_loss_grad_bf16(const float* params, const float* X, const float* T, int32_t n, float* work, float* grad,
                           float* loss, void* cuda_stream) {
    if (!params || !work || !grad || !loss || n < 1 || !X || !T)
        return fail(nullptr, PDF_ERR_ARG, "pdf_mlp_loss_grad_bf16: NULL array or n < 1");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int ntiles = (n + R - 1) / R;
    float* part = work;
    float* lpart = part + (size_t)ntiles * NP;
    int* err = reinterpret_cast<int*>(lpart + ntiles);
    static_assert(sizeof(TrainSmem) <= 227 * 1024, "shared memory of the training tile");
    const int smem = (int)sizeof(TrainSmem) + 128;
    cudaError_t e = cudaFuncSetAttribute(k_mlp_tc_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(err, 0, sizeof(int), s);
    if (e == cudaSuccess) {
        k_mlp_tc_grad<<<ntiles, R, smem, s>>>(params, X, T, n, part, lpart, err);
        k_mlp_tc_reduce<<<(NP + 255) / 256, 256, 0, s>>>(part, lpart, ntiles, err, grad, loss,
                                                          (float)(1.0 / (5.0 * (double)n)));
        e = cudaGetLastError();
    }
    if (e != cudaSuccess)
        return fail(nullptr, PDF_ERR_CUDA, std::string("pdf_mlp_loss_grad_bf16: ") + cudaGetErrorString(e));
    return PDF_OK;
}

}  // extern "C"
