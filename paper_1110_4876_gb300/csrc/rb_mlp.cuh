// rb_mlp.cuh -- tensor-core pieces of the learned far-field correction (not
// in the paper) shared by the training kernels (rb_mlp.cu) and the learned
// gravity walk (rb_walk.cu): the padded parameter layout, BF16 packing, the
// mma.sync.m16n8k16 wrapper, the GELU (tanh form) and the inference forward
// pass over weights stored as pre-packed B fragments.
//
// Network: 12 -> 64 -> 64 -> 64 -> 3, GELU after each hidden layer.  Padded
// layout ("padded", 9928 floats): W1 16x64 (rows 12..15 zero), b1 64,
// W2 64x64, b2 64, W3 64x64, b3 64, W4 64x8 (cols 3..7 zero), b4 8; W is
// row-major input x output.
#pragma once
#include <cuda_bf16.h>

#include <cstdint>

namespace rb {
namespace mlp {

constexpr int kW1 = 0, kB1 = kW1 + 16 * 64, kW2 = kB1 + 64, kB2 = kW2 + 64 * 64;
constexpr int kW3 = kB2 + 64, kB3 = kW3 + 64 * 64, kW4 = kB3 + 64, kB4 = kW4 + 64 * 8;
constexpr int kPad = kB4 + 8;   // 9928

// Inference weights as mma B fragments: entry [t][j][lane] holds the two
// 32-bit registers lane (g = lane / 4, q = lane % 4) passes for the 16 x 8
// tile of W at rows 16 t .., columns 8 j ..: {W[k][n], W[k+1][n]} and
// {W[k+8][n], W[k+9][n]} with k = 16 t + 2 q, n = 8 j + g (BF16, round to
// nearest even).  One 8-byte shared load per lane and MMA, no bank conflict.
struct Packed {
    uint2 B1[1][8][32];
    uint2 B2[4][8][32];
    uint2 B3[4][8][32];
    uint2 B4[4][1][32];
    float b1[64], b2[64], b3[64], b4[8];
};
static_assert(sizeof(Packed) % 16 == 0, "Packed is copied in 16-byte words");

#ifdef __CUDACC__
namespace {

constexpr float kGeluC = 0.7978845608028654f;   // sqrt(2 / pi)

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack2h(__nv_bfloat16 lo, __nv_bfloat16 hi) {
    __nv_bfloat162 v;
    v.x = lo;
    v.y = hi;
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ float gelu(float z) {
    return 0.5f * z * (1.f + tanhf(kGeluC * (z + 0.044715f * z * z * z)));
}

// GELU for inference: the same tanh form with the hardware tanh
// (tanh.approx.f32, relative error about 2^-11), below the BF16 rounding
// (2^-9) the activation gets next.
__device__ __forceinline__ float gelu_fast(float z) {
    const float u = kGeluC * fmaf(0.044715f * z, z * z, z);
    float t;
    asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(u));
    const float h = 0.5f * z;
    return fmaf(h, t, h);
}

// A fragment (16 x 16 tile at (r0, c0)) of a row-major BF16 matrix in shared
// memory with ld columns (lane l: g = l / 4, q = l % 4).
__device__ __forceinline__ void ldA(uint32_t (&a)[4], const __nv_bfloat16* M, int ld, int r0, int c0,
                                    int g, int q) {
    a[0] = *reinterpret_cast<const uint32_t*>(&M[(r0 + g) * ld + c0 + 2 * q]);
    a[1] = *reinterpret_cast<const uint32_t*>(&M[(r0 + g + 8) * ld + c0 + 2 * q]);
    a[2] = *reinterpret_cast<const uint32_t*>(&M[(r0 + g) * ld + c0 + 8 + 2 * q]);
    a[3] = *reinterpret_cast<const uint32_t*>(&M[(r0 + g + 8) * ld + c0 + 8 + 2 * q]);
}

// Hidden layer: c = bias + A W (K = 16 kt, N = 64), then GELU, repacked as the
// next layer's A fragments (the accumulator tile of columns 8 j .. is half of
// the A tile t = j / 2).
template <int KT>
__device__ __forceinline__ void hidden_layer(uint32_t (&a)[4][4], const uint2 (&B)[KT][8][32],
                                             const float* bias, int lane, int q) {
    float c[8][4];
#pragma unroll
    for (int j = 0; j < 8; j++) {
        c[j][0] = c[j][2] = bias[8 * j + 2 * q];
        c[j][1] = c[j][3] = bias[8 * j + 2 * q + 1];
    }
#pragma unroll
    for (int t = 0; t < KT; t++)
#pragma unroll
        for (int j = 0; j < 8; j++) {
            const uint2 b = B[t][j][lane];
            mma(c[j], a[t], b.x, b.y);
        }
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const int t = j >> 1;
        const uint32_t lo = pack2(gelu_fast(c[j][0]), gelu_fast(c[j][1]));
        const uint32_t hi = pack2(gelu_fast(c[j][2]), gelu_fast(c[j][3]));
        if ((j & 1) == 0) {
            a[t][0] = lo;
            a[t][1] = hi;
        } else {
            a[t][2] = lo;
            a[t][3] = hi;
        }
    }
}

// Network outputs for 16 rows held by one warp: X is BF16 [16][16] (inputs
// in columns 0..11, zeros after); out holds rows g and g + 8, columns 2 q and
// 2 q + 1 of the 16 x 8 output tile (columns 0..2 are the outputs).
__device__ __forceinline__ void forward_packed(const Packed& w, const __nv_bfloat16* X, float (&out)[4]) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    uint32_t a[4][4];
    ldA(a[0], X, 16, 0, 0, g, q);
    hidden_layer<1>(a, w.B1, w.b1, lane, q);
    hidden_layer<4>(a, w.B2, w.b2, lane, q);
    hidden_layer<4>(a, w.B3, w.b3, lane, q);
    out[0] = out[2] = w.b4[2 * q];
    out[1] = out[3] = w.b4[2 * q + 1];
#pragma unroll
    for (int t = 0; t < 4; t++) {
        const uint2 b = w.B4[t][0][lane];
        mma(out, a[t], b.x, b.y);
    }
}

}  // namespace
#endif

// Writes the inference layout of the padded FP32 weights w (device) to
// packed (device); async on s.
void pack_async(const float* w, Packed* packed, cudaStream_t s);

}  // namespace mlp
}  // namespace rb
