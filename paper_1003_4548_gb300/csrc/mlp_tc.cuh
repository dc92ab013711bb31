// mlp_tc.cuh -- the surrogate network (10 -> 64 -> 64 -> 64 -> 5, SiLU) on
// the 5th-generation tensor cores, for tiles of 128 rows (nodes or
// particles). Every layer is a chain of 128 x N x 16 tcgen05 MMAs: the
// activations A (bf16, K-major) and the weights W (bf16, stored out x in, so
// K-major as B) in shared memory, the FP32 accumulator in tensor memory. The
// thread of row r reads its row back (tensor-memory lane r), adds the bias,
// applies SiLU and writes the bf16 activations as the next layer's A. Shapes:
// 128x64x16 (inputs padded to 16), 128x64x64, 128x64x64, 128x16x64 (outputs
// padded to 16). Used by the node inference and the per-particle form.
#pragma once
#include <cuda_bf16.h>

#include "pdf_internal.cuh"
#include "tc.cuh"

namespace mlptc {

constexpr int IN = PDF_MLP_IN, H = PDF_MLP_HIDDEN, OUT = PDF_MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + H * IN, OFF_W2 = OFF_B1 + H, OFF_B2 = OFF_W2 + H * H;
constexpr int OFF_W3 = OFF_B2 + H, OFF_B3 = OFF_W3 + H * H, OFF_W4 = OFF_B3 + H, OFF_B4 = OFF_W4 + OUT * H;
constexpr int TILE_ROWS = 128;
constexpr int TILE_ELEMS = TILE_ROWS * H;  // bf16 elements of one activation tile

struct Weights {
    __align__(128) uint16_t W1[H * 16];  // 64 x 16
    __align__(128) uint16_t W2[H * H];
    __align__(128) uint16_t W3[H * H];
    __align__(128) uint16_t W4[16 * H];  // 16 x 64 (rows 5..15 zero)
    float bias[3 * H + 16];
    float nm[PDF_MLP_NNORM];  // in_mean in_std out_mean out_std
};

__device__ __forceinline__ uint16_t bf16_bits(float x) { return __bfloat16_as_ushort(__float2bfloat16_rn(x)); }
// SiLU with the hardware exponential and a fast divide: its error (a few
// ulp of FP32) is far below the bf16 rounding of the activation
__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.f + __expf(-z)); }

// 8 consecutive activations of one row (k = 8 j .. 8 j + 7) as one 16-byte
// store: they are contiguous in the canonical layout
__device__ __forceinline__ void put8(uint16_t* tile, int r, int k0, int kc, const float* v) {
    uint4 q;
    q.x = (uint32_t)bf16_bits(v[0]) | ((uint32_t)bf16_bits(v[1]) << 16);
    q.y = (uint32_t)bf16_bits(v[2]) | ((uint32_t)bf16_bits(v[3]) << 16);
    q.z = (uint32_t)bf16_bits(v[4]) | ((uint32_t)bf16_bits(v[5]) << 16);
    q.w = (uint32_t)bf16_bits(v[6]) | ((uint32_t)bf16_bits(v[7]) << 16);
    *reinterpret_cast<uint4*>(tile + tc::core_offset(r, k0, kc)) = q;
}

// weights (already bf16-rounded floats, parameter layout of the C ABI, then
// the standardisation) into the canonical layouts; threads t of nt
__device__ __forceinline__ void load(Weights& W, const float* __restrict__ wq, int t, int nt) {
    for (int q = t; q < H * 16; q += nt) {
        const int n = q / 16, k = q % 16;
        W.W1[tc::core_offset(n, k, 2)] = bf16_bits(k < IN ? wq[OFF_W1 + IN * n + k] : 0.f);
    }
    for (int q = t; q < H * H; q += nt) {
        const int n = q / H, k = q % H;
        W.W2[tc::core_offset(n, k, 8)] = bf16_bits(wq[OFF_W2 + q]);
        W.W3[tc::core_offset(n, k, 8)] = bf16_bits(wq[OFF_W3 + q]);
    }
    for (int q = t; q < 16 * H; q += nt) {
        const int n = q / H, k = q % H;
        W.W4[tc::core_offset(n, k, 8)] = bf16_bits(n < OUT ? wq[OFF_W4 + H * n + k] : 0.f);
    }
    for (int q = t; q < H; q += nt) {
        W.bias[q] = wq[OFF_B1 + q];
        W.bias[H + q] = wq[OFF_B2 + q];
        W.bias[2 * H + q] = wq[OFF_B3 + q];
    }
    for (int q = t; q < 16; q += nt) W.bias[3 * H + q] = q < OUT ? wq[OFF_B4 + q] : 0.f;
    for (int q = t; q < PDF_MLP_NNORM; q += nt) W.nm[q] = wq[PDF_MLP_NPARAM + q];
}

// the 16 standardised inputs (10 used, 6 zero) of row r of a tile (layer-1 layout)
__device__ __forceinline__ void put_inputs(uint16_t* tile, int r, const float (&f)[16]) {
    put8(tile, r, 0, 2, f);
    put8(tile, r, 8, 2, f + 8);
}

// The network on ntiles tiles of 128 rows: thread t is row t % 128 of tile
// t / 128 (blockDim = 128 ntiles); A holds the tiles back to back with the
// inputs already written; tmem has 64 ntiles columns; bar is an mbarrier of
// count 1 whose phase counter is carried in phase. Every thread of the block
// must call it. y: the 16 output columns of this thread's row, bias added
// (first OUT meaningful, standardised units). Returns false (on every
// thread) if an MMA completion wait ran out.
__device__ __forceinline__ bool run(const Weights& W, uint16_t* A, int ntiles, uint32_t tmem, uint64_t* bar,
                                    unsigned& phase, float (&y)[16]) {
    const int t = threadIdx.x, row = t & (TILE_ROWS - 1), warp = t >> 5;
    uint16_t* At = A + (t >> 7) * TILE_ELEMS;
    const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;  // this warp's tensor-memory lanes
    const uint32_t col0 = (uint32_t)((t >> 7) * H);                // this tile's columns
    for (int layer = 0; layer < 4; ++layer) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // A visible to the tensor cores
        tc::fence_before_sync();
        __syncthreads();
        if (t == 0) {
            tc::fence_after_sync();
            const int kc = layer == 0 ? 2 : 8;
            const int ksteps = layer == 0 ? 1 : 4;
            const uint16_t* Wl = layer == 0 ? W.W1 : (layer == 1 ? W.W2 : (layer == 2 ? W.W3 : W.W4));
            const uint32_t idesc = tc::idesc_bf16(TILE_ROWS, layer == 3 ? 16 : H);
            for (int tt = 0; tt < ntiles; ++tt)
                for (int j = 0; j < ksteps; ++j) {
                    const uint64_t ad = tc::smem_desc(A + tt * TILE_ELEMS + j * 128, 128, kc * 128);
                    const uint64_t bd = tc::smem_desc(Wl + j * 128, 128, kc * 128);
                    tc::mma_bf16(tmem + (uint32_t)(tt * H), ad, bd, idesc, j > 0 ? 1u : 0u);
                }
            tc::commit(bar);
        }
        const bool ok = __syncthreads_and(tc::mbar_wait(bar, phase & 1u) ? 1 : 0) != 0;
        ++phase;
        tc::fence_after_sync();
        if (!ok) return false;
        if (layer < 3) {
            const float* bias = W.bias + layer * H;
#pragma unroll
            for (int c0 = 0; c0 < H; c0 += 16) {
                float v[16];
                tc::ld16(tmem + lane_base + col0 + (uint32_t)c0, v);
#pragma unroll
                for (int k = 0; k < 16; ++k) v[k] = silu(v[k] + bias[c0 + k]);
                put8(At, row, c0, 8, v);
                put8(At, row, c0 + 8, 8, v + 8);
            }
            tc::fence_before_sync();
        } else {
            tc::ld16(tmem + lane_base + col0, y);
#pragma unroll
            for (int k = 0; k < 16; ++k) y[k] += W.bias[3 * H + k];
        }
    }
    return true;
}

}  // namespace mlptc
