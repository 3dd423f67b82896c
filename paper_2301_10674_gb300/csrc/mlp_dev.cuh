// Learned interface normal: a 27-64-64-4 perceptron with ReLU that maps the
// fill levels of a 3x3x3 block of cells (index q = (cx+1) + 3(cy+1) +
// 9(cz+1)) to a raw normal toward the gas and the curvature.
//
// On the tensor cores every product takes BF16 operands (weights, inputs,
// hidden activations) and accumulates in FP32 (mma.sync m16n8k16); biases
// are added in FP32. A warp evaluates 16 stencils at a time: row g of the
// 16-row tile is the stencil of lane group g (lanes 4g..4g+3), row g + 8
// the second stencil of the same group.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace fsl {

constexpr int MLP_IN = 27, MLP_H = 64, MLP_OUT = 4;
constexpr int MLP_NPARAM = MLP_H * MLP_IN + MLP_H + MLP_H * MLP_H + MLP_H + MLP_OUT * MLP_H + MLP_OUT;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + MLP_H * MLP_IN, OFF_W2 = OFF_B1 + MLP_H,
              OFF_B2 = OFF_W2 + MLP_H * MLP_H, OFF_W3 = OFF_B2 + MLP_H, OFF_B3 = OFF_W3 + MLP_OUT * MLP_H;
static_assert(MLP_NPARAM == 6212, "parameter count");

// Operand copies of the parameters. W1 is padded to 32 inputs and W3 to 16
// outputs (zeros); the transposes serve the backward pass.
struct MlpBf16 {
    __nv_bfloat16 w1[MLP_H * 32];       // (out, in)
    __nv_bfloat16 w2[MLP_H * MLP_H];    // (out, in)
    __nv_bfloat16 w2t[MLP_H * MLP_H];   // (in, out)
    __nv_bfloat16 w3[16 * MLP_H];       // (out, in)
    __nv_bfloat16 w3t[MLP_H * 16];      // (in, out)
    float b1[MLP_H], b2[MLP_H], b3[16];
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ uint32_t ld_pair(const __nv_bfloat16* p) {
    return *reinterpret_cast<const uint32_t*>(p);
}

// D += A (16x16, row-major fragments) * B (16x8, column-major fragments)
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Pre-activations of the two hidden layers (accumulator layout: n-tile nt,
// values for rows g, g, g+8, g+8 and columns 8 nt + 2t, 8 nt + 2t + 1) and
// the output (columns 2t, 2t + 1 of rows g and g + 8; lanes with t < 2 hold
// the four outputs).
struct MlpAct {
    float z1[8][4];
    float z2[8][4];
    float y[4];
};

// A fragment (16 x 16, k-tile kk) built from the accumulators of n-tiles
// 2 kk and 2 kk + 1, with ReLU applied
__device__ __forceinline__ void relu_frag(const float (&z)[8][4], int kk, uint32_t (&a)[4]) {
    const float* p = z[2 * kk];
    const float* q = z[2 * kk + 1];
    a[0] = pack_bf16(fmaxf(p[0], 0.f), fmaxf(p[1], 0.f));
    a[1] = pack_bf16(fmaxf(p[2], 0.f), fmaxf(p[3], 0.f));
    a[2] = pack_bf16(fmaxf(q[0], 0.f), fmaxf(q[1], 0.f));
    a[3] = pack_bf16(fmaxf(q[2], 0.f), fmaxf(q[3], 0.f));
}

// Forward pass from the input fragments x[kk] (k-tiles 0 and 1: inputs
// 0..15 and 16..31, inputs 27..31 zero). W may live in global or shared
// memory.
__device__ __forceinline__ void mlp_forward(const MlpBf16& W, const uint32_t (&x)[2][4], MlpAct& o) {
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float b0 = W.b1[8 * nt + 2 * t], b1 = W.b1[8 * nt + 2 * t + 1];
        float d[4] = {b0, b1, b0, b1};
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const __nv_bfloat16* row = W.w1 + (8 * nt + g) * 32 + 16 * kk + 2 * t;
            mma_bf16(d, x[kk][0], x[kk][1], x[kk][2], x[kk][3], ld_pair(row), ld_pair(row + 8));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) o.z1[nt][k] = d[k];
    }
    uint32_t a[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) relu_frag(o.z1, kk, a[kk]);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float b0 = W.b2[8 * nt + 2 * t], b1 = W.b2[8 * nt + 2 * t + 1];
        float d[4] = {b0, b1, b0, b1};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const __nv_bfloat16* row = W.w2 + (8 * nt + g) * MLP_H + 16 * kk + 2 * t;
            mma_bf16(d, a[kk][0], a[kk][1], a[kk][2], a[kk][3], ld_pair(row), ld_pair(row + 8));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) o.z2[nt][k] = d[k];
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) relu_frag(o.z2, kk, a[kk]);
    {
        const float b0 = W.b3[2 * t], b1 = W.b3[2 * t + 1];
        float d[4] = {b0, b1, b0, b1};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const __nv_bfloat16* row = W.w3 + g * MLP_H + 16 * kk + 2 * t;
            mma_bf16(d, a[kk][0], a[kk][1], a[kk][2], a[kk][3], ld_pair(row), ld_pair(row + 8));
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) o.y[k] = d[k];
    }
}

// Weight operands of the in-step forward pass in fragment order: entry
// [...][lane] is the register pair (b0, b1) that lane feeds one mma, so a
// warp reads one contiguous 256-byte row per mma. w1[m] is the first layer
// of mirror image m of R-17g (0 the network itself; 1, 2, 3 its input
// columns mirrored in x, in y, in both).
struct MlpFrag {
    uint2 w1[4][8][2][32];
    uint2 w2[8][4][32];
    uint2 w3[4][32];
};

// The forward pass of mlp_forward with the weights of G (first layer of
// mirror image m) and the biases of W
__device__ __forceinline__ void mlp_forward_frag(const MlpBf16& W, const MlpFrag& G, int m,
                                                 const uint32_t (&x)[2][4], MlpAct& o) {
    const int lane = threadIdx.x & 31, t = lane & 3;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float2 b = *reinterpret_cast<const float2*>(W.b1 + 8 * nt + 2 * t);
        float d[4] = {b.x, b.y, b.x, b.y};
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
            const uint2 w = G.w1[m][nt][kk][lane];
            mma_bf16(d, x[kk][0], x[kk][1], x[kk][2], x[kk][3], w.x, w.y);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) o.z1[nt][k] = d[k];
    }
    uint32_t a[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) relu_frag(o.z1, kk, a[kk]);
#pragma unroll
    for (int nt = 0; nt < 8; ++nt) {
        const float2 b = *reinterpret_cast<const float2*>(W.b2 + 8 * nt + 2 * t);
        float d[4] = {b.x, b.y, b.x, b.y};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint2 w = G.w2[nt][kk][lane];
            mma_bf16(d, a[kk][0], a[kk][1], a[kk][2], a[kk][3], w.x, w.y);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) o.z2[nt][k] = d[k];
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) relu_frag(o.z2, kk, a[kk]);
    {
        const float2 b = *reinterpret_cast<const float2*>(W.b3 + 2 * t);
        float d[4] = {b.x, b.y, b.x, b.y};
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const uint2 w = G.w3[kk][lane];
            mma_bf16(d, a[kk][0], a[kk][1], a[kk][2], a[kk][3], w.x, w.y);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) o.y[k] = d[k];
    }
}

// The four outputs of rows g and g + 8, gathered into every lane of group g
__device__ __forceinline__ void mlp_outputs(const MlpAct& o, float (&yg)[4], float (&yg8)[4]) {
    const int base = (threadIdx.x & 31) & ~3;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const int src = base + (c >> 1);
        yg[c] = __shfl_sync(0xffffffffu, o.y[c & 1], src);
        yg8[c] = __shfl_sync(0xffffffffu, o.y[2 + (c & 1)], src);
    }
}

// Input fragment entries of lane (g, t): column j of k-tile kk is
// 16 kk + {2t, 2t+1, 2t+8, 2t+9}[j]
__device__ __forceinline__ int frag_col(int kk, int j, int t) {
    return 16 * kk + 2 * t + (j & 1) + ((j >> 1) << 3);
}

// Input fragments from two stencils' values v(row, column) supplied by f
template <class F>
__device__ __forceinline__ void input_frags(F f, uint32_t (&x)[2][4]) {
    const int t = threadIdx.x & 3;
#pragma unroll
    for (int kk = 0; kk < 2; ++kk) {
        const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
        x[kk][0] = pack_bf16(f(0, c0), f(0, c0 + 1));
        x[kk][1] = pack_bf16(f(1, c0), f(1, c0 + 1));
        x[kk][2] = pack_bf16(f(0, c1), f(0, c1 + 1));
        x[kk][3] = pack_bf16(f(1, c1), f(1, c1 + 1));
    }
}

}  // namespace fsl
