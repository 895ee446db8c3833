// rb_mlp.cu -- learned far-field correction (not in the paper): a small MLP
// (12 -> 64 -> 64 -> 64 -> 3, GELU tanh form) predicts the residual between
// an accepted cell's exact force (Eq. 1 over its particles) and its
// multipole force (Sect. 4.2), in units of G M / R^2, so the walk can open
// cells at a wider theta and add the predicted residual.
//
// This file holds the training side (residual labels, the tensor-core
// gradient kernel, Adam) and the packing of trained weights for inference;
// inference itself runs inside the gravity walk (rb_walk.cu).
//
// Tensor cores: every layer of the forward and backward pass is a BF16
// mma.sync.m16n8k16 with FP32 accumulation on 16-row tiles per warp.  The
// hidden activations stay in registers between forward layers (the FP32
// accumulator fragment of one layer is the BF16 A fragment of the next).
// Training keeps FP32 master weights (Adam) and hands BF16 copies to the
// kernels.
//
// Parameter layout used inside the library ("padded"): W1 16x64 (rows 12..15
// zero), b1 64, W2 64x64, b2 64, W3 64x64, b3 64, W4 64x8 (cols 3..7 zero),
// b4 8 -- 9928 values; the C ABI exchanges the unpadded 9347 values in the
// order W1 (12x64), b1, W2, b2, W3, b3, W4 (64x3), b4 (row-major, input x
// output).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <vector>

#include "rb_internal.cuh"
#include "rb_mlp.cuh"

namespace rb {
namespace mlp {
namespace {

constexpr int kWarps = 4;       // warps per block of the training kernel (16 rows each)

__device__ __forceinline__ float gelu_grad(float z) {
    const float t = tanhf(kGeluC * (z + 0.044715f * z * z * z));
    return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * kGeluC * (1.f + 3.f * 0.044715f * z * z);
}

// Fragment loads from row-major BF16 matrices in shared memory (lane l:
// g = l / 4, q = l % 4); ldA is shared with the inference path.
// A tile of M^T: A[m][k] = M[k][m], m in [r0, r0+16), k in [c0, c0+16).
__device__ __forceinline__ void ldAT(uint32_t (&a)[4], const __nv_bfloat16* M, int ld, int r0, int c0,
                                     int g, int q) {
    const int k0 = c0 + 2 * q, m0 = r0 + g;
    a[0] = pack2h(M[k0 * ld + m0], M[(k0 + 1) * ld + m0]);
    a[1] = pack2h(M[k0 * ld + m0 + 8], M[(k0 + 1) * ld + m0 + 8]);
    a[2] = pack2h(M[(k0 + 8) * ld + m0], M[(k0 + 9) * ld + m0]);
    a[3] = pack2h(M[(k0 + 8) * ld + m0 + 8], M[(k0 + 9) * ld + m0 + 8]);
}
// B tile (16 x 8) of M: B[k][n] = M[k][n], k in [k0, k0+16), n in [n0, n0+8).
__device__ __forceinline__ void ldB(uint32_t& b0, uint32_t& b1, const __nv_bfloat16* M, int ld, int k0,
                                    int n0, int g, int q) {
    const int k = k0 + 2 * q, n = n0 + g;
    b0 = pack2h(M[k * ld + n], M[(k + 1) * ld + n]);
    b1 = pack2h(M[(k + 8) * ld + n], M[(k + 9) * ld + n]);
}
// B tile of M^T: B[k][n] = M[n][k].
__device__ __forceinline__ void ldBT(uint32_t& b0, uint32_t& b1, const __nv_bfloat16* M, int ld, int k0,
                                     int n0, int g, int q) {
    b0 = *reinterpret_cast<const uint32_t*>(&M[(n0 + g) * ld + k0 + 2 * q]);
    b1 = *reinterpret_cast<const uint32_t*>(&M[(n0 + g) * ld + k0 + 8 + 2 * q]);
}

// Shared-memory weights of one block: BF16 W (padded row-major) + FP32 biases.
struct SW {
    __nv_bfloat16 W1[16 * 64], W2[64 * 64], W3[64 * 64], W4[64 * 8];
    float b1[64], b2[64], b3[64], b4[8];
};

__device__ void load_weights(SW& s, const __nv_bfloat16* __restrict__ wbf, const float* __restrict__ wf) {
    for (int i = threadIdx.x; i < 16 * 64; i += blockDim.x) s.W1[i] = wbf[kW1 + i];
    for (int i = threadIdx.x; i < 64 * 64; i += blockDim.x) {
        s.W2[i] = wbf[kW2 + i];
        s.W3[i] = wbf[kW3 + i];
    }
    for (int i = threadIdx.x; i < 64 * 8; i += blockDim.x) s.W4[i] = wbf[kW4 + i];
    for (int i = threadIdx.x; i < 64; i += blockDim.x) {
        s.b1[i] = wf[kB1 + i];
        s.b2[i] = wf[kB2 + i];
        s.b3[i] = wf[kB3 + i];
    }
    if (threadIdx.x < 8) s.b4[threadIdx.x] = wf[kB4 + threadIdx.x];
}

// Forward pass of 16 rows held by one warp.  X: BF16 [16][16] (features in
// columns 0..11).  If Z/H are given, the hidden pre-activations (FP32) and
// activations (BF16) of layers 1..3 are stored as [3][16][64] for backward.
// out: the output fragment (rows g and g+8, columns 2q and 2q+1).
__device__ void forward(const SW& w, const __nv_bfloat16* X, float (&out)[4], float* Z,
                        __nv_bfloat16* H) {
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    uint32_t a[4][4];
    ldA(a[0], X, 16, 0, 0, g, q);
    int kt = 1;
    const __nv_bfloat16* Ws[3] = {w.W1, w.W2, w.W3};
    const float* bs[3] = {w.b1, w.b2, w.b3};
    for (int L = 0; L < 3; L++) {
        float c[8][4];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            c[j][0] = c[j][2] = bs[L][8 * j + 2 * q];
            c[j][1] = c[j][3] = bs[L][8 * j + 2 * q + 1];
        }
        for (int t = 0; t < kt; t++)
#pragma unroll
            for (int j = 0; j < 8; j++) {
                uint32_t b0, b1;
                ldB(b0, b1, Ws[L], 64, 16 * t, 8 * j, g, q);
                mma(c[j], a[t], b0, b1);
            }
#pragma unroll
        for (int j = 0; j < 8; j++) {
            float h[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int row = g + ((e >> 1) << 3), col = 8 * j + 2 * q + (e & 1);
                if (Z) Z[(L * 16 + row) * 64 + col] = c[j][e];
                h[e] = gelu(c[j][e]);
                if (H) H[(L * 16 + row) * 64 + col] = __float2bfloat16_rn(h[e]);
            }
            const int t = j >> 1;
            if ((j & 1) == 0) {
                a[t][0] = pack2(h[0], h[1]);
                a[t][1] = pack2(h[2], h[3]);
            } else {
                a[t][2] = pack2(h[0], h[1]);
                a[t][3] = pack2(h[2], h[3]);
            }
        }
        kt = 4;
    }
    out[0] = out[2] = w.b4[2 * q];
    out[1] = out[3] = w.b4[2 * q + 1];
#pragma unroll
    for (int t = 0; t < 4; t++) {
        uint32_t b0, b1;
        ldB(b0, b1, w.W4, 8, 16 * t, 0, g, q);
        mma(out, a[t], b0, b1);
    }
}

// Per-warp scratch of the training kernel.
struct WarpScratch {
    __nv_bfloat16 X[16 * 16];
    float Z[3 * 16 * 64];
    __nv_bfloat16 H[3 * 16 * 64];
    __nv_bfloat16 D[16 * 64];    // current layer's output gradient (BF16)
    __nv_bfloat16 D4[16 * 16];   // dY padded to 16 columns
};

struct TrainSmem {
    SW w;
    float grad[kPad];
    WarpScratch ws[kWarps];
    float loss[kWarps];
};

// Add a 16x8 fragment tile of a weight gradient (rows r0.., cols c0..) to
// the block's gradient (row-major, ld columns).
__device__ __forceinline__ void add_tile(float* G, int ld, int r0, int c0, const float (&c)[4], int g,
                                         int q) {
    atomicAdd(&G[(r0 + g) * ld + c0 + 2 * q], c[0]);
    atomicAdd(&G[(r0 + g) * ld + c0 + 2 * q + 1], c[1]);
    atomicAdd(&G[(r0 + g + 8) * ld + c0 + 2 * q], c[2]);
    atomicAdd(&G[(r0 + g + 8) * ld + c0 + 2 * q + 1], c[3]);
}

// Sum over the 16 rows of a column pair (rows g and g+8 of every lane with
// the same q): shuffle-reduce over g.
__device__ __forceinline__ float rows_sum(float v) {
    v += __shfl_xor_sync(0xffffffffu, v, 4);
    v += __shfl_xor_sync(0xffffffffu, v, 8);
    v += __shfl_xor_sync(0xffffffffu, v, 16);
    return v;
}

// Gradient of the mean squared error over the rows idx[0..n) (all rows of a
// batch of size n_total): forward, then backward through the three hidden
// layers; weight gradients are MMAs of activations^T x output gradients.
__global__ void __launch_bounds__(kWarps * 32) k_mlp_grad(const __nv_bfloat16* __restrict__ wbf,
                                                          const float* __restrict__ wf,
                                                          const float* __restrict__ X,
                                                          const float* __restrict__ Y,
                                                          const int32_t* __restrict__ idx, int n,
                                                          int n_total, float* __restrict__ grad,
                                                          float* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
    load_weights(S.w, wbf, wf);
    for (int i = threadIdx.x; i < kPad; i += blockDim.x) S.grad[i] = 0.f;
    if (threadIdx.x < kWarps) S.loss[threadIdx.x] = 0.f;
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    WarpScratch& W = S.ws[warp];
    const float scale = 2.f / (3.f * (float)n_total);
    const int ntiles = (n + 15) / 16;
    for (int tile = blockIdx.x * kWarps + warp; tile < ntiles; tile += gridDim.x * kWarps) {
        // inputs
        for (int e = lane; e < 16 * 16; e += 32) {
            const int r = e >> 4, c = e & 15, row = tile * 16 + r;
            const float v = (row < n && c < 12) ? X[(size_t)idx[row] * 12 + c] : 0.f;
            W.X[e] = __float2bfloat16_rn(v);
        }
        __syncwarp();
        float out[4];
        forward(S.w, W.X, out, W.Z, W.H);
        __syncwarp();
        // output gradient dY = 2 (P - Y) / (3 n_total), zero outside
        float dy[4], lsum = 0.f;
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int r = g + ((e >> 1) << 3), c = 2 * q + (e & 1), row = tile * 16 + r;
            float d = 0.f;
            if (row < n && c < 3) {
                const float diff = out[e] - Y[(size_t)idx[row] * 3 + c];
                d = scale * diff;
                lsum += diff * diff;
            }
            dy[e] = d;
            W.D4[r * 16 + c] = __float2bfloat16_rn(d);
            W.D4[r * 16 + c + 8] = __float2bfloat16_rn(0.f);
        }
        for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
        if (lane == 0) S.loss[warp] += lsum;
        __syncwarp();
        // layer 4: b4, W4 (64 x 8) += H3^T dY
        {
            const float s0 = rows_sum(dy[0] + dy[2]), s1 = rows_sum(dy[1] + dy[3]);
            if (g == 0) {
                atomicAdd(&S.grad[kB4 + 2 * q], s0);
                atomicAdd(&S.grad[kB4 + 2 * q + 1], s1);
            }
            for (int mt = 0; mt < 4; mt++) {
                float c[4] = {0.f, 0.f, 0.f, 0.f};
                uint32_t a[4], b0, b1;
                ldAT(a, W.H + 2 * 16 * 64, 64, 16 * mt, 0, g, q);
                ldB(b0, b1, W.D4, 16, 0, 0, g, q);
                mma(c, a, b0, b1);
                add_tile(S.grad + kW4, 8, 16 * mt, 0, c, g, q);
            }
        }
        // dH3 = dY W4^T; hidden layers 3, 2, 1
        const __nv_bfloat16* Wl[3] = {S.w.W1, S.w.W2, S.w.W3};
        const int offW[3] = {kW1, kW2, kW3}, offB[3] = {kB1, kB2, kB3};
        for (int L = 2; L >= 0; L--) {
            float dh[8][4];
            // output gradient of layer L (16 x 64) from the layer above
#pragma unroll
            for (int j = 0; j < 8; j++) {
                dh[j][0] = dh[j][1] = dh[j][2] = dh[j][3] = 0.f;
                if (L == 2) {
                    uint32_t a[4], b0, b1;
                    ldA(a, W.D4, 16, 0, 0, g, q);
                    // B[k = output o][n = hidden h] = W4[h][o]; rows o >= 8 are zero
                    b0 = *reinterpret_cast<const uint32_t*>(&S.w.W4[(8 * j + g) * 8 + 2 * q]);
                    b1 = 0u;
                    mma(dh[j], a, b0, b1);
                } else {
                    for (int t = 0; t < 4; t++) {
                        uint32_t a[4], b0, b1;
                        ldA(a, W.D, 64, 0, 16 * t, g, q);
                        ldBT(b0, b1, Wl[L + 1], 64, 16 * t, 8 * j, g, q);
                        mma(dh[j], a, b0, b1);
                    }
                }
            }
            __syncwarp();
            // dZ = dH * gelu'(Z); bias gradient; keep dZ in BF16 for the MMAs
#pragma unroll
            for (int j = 0; j < 8; j++) {
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int r = g + ((e >> 1) << 3), c = 8 * j + 2 * q + (e & 1);
                    dh[j][e] *= gelu_grad(W.Z[(L * 16 + r) * 64 + c]);
                    W.D[r * 64 + c] = __float2bfloat16_rn(dh[j][e]);
                }
                const float s0 = rows_sum(dh[j][0] + dh[j][2]), s1 = rows_sum(dh[j][1] + dh[j][3]);
                if (g == 0) {
                    atomicAdd(&S.grad[offB[L] + 8 * j + 2 * q], s0);
                    atomicAdd(&S.grad[offB[L] + 8 * j + 2 * q + 1], s1);
                }
            }
            __syncwarp();
            // W_L += (input of layer L)^T dZ
            const __nv_bfloat16* in = L == 0 ? W.X : W.H + (L - 1) * 16 * 64;
            const int ldin = L == 0 ? 16 : 64;
            const int mts = L == 0 ? 1 : 4;
            for (int mt = 0; mt < mts; mt++)
#pragma unroll
                for (int j = 0; j < 8; j++) {
                    float c[4] = {0.f, 0.f, 0.f, 0.f};
                    uint32_t a[4], b0, b1;
                    ldAT(a, in, ldin, 16 * mt, 0, g, q);
                    ldB(b0, b1, W.D, 64, 0, 8 * j, g, q);
                    mma(c, a, b0, b1);
                    add_tile(S.grad + offW[L], 64, 16 * mt, 8 * j, c, g, q);
                }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kPad; i += blockDim.x)
        if (S.grad[i] != 0.f) atomicAdd(&grad[i], S.grad[i]);
    if (threadIdx.x == 0) {
        float l = 0.f;
        for (int w = 0; w < kWarps; w++) l += S.loss[w];
        atomicAdd(loss, l);
    }
}

// Adam on the padded FP32 master weights (padding stays zero), then the
// BF16 copies the kernels read.
__global__ void k_mlp_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v,
                           const float* __restrict__ grad, __nv_bfloat16* __restrict__ wbf, float lr,
                           float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= kPad) return;
    const bool pad = (i < kB1 && (i - kW1) / 64 >= 12) || (i >= kW4 && i < kB4 && (i - kW4) % 8 >= 3) ||
                     (i >= kB4 && i - kB4 >= 3);
    if (pad) {
        w[i] = 0.f;
        wbf[i] = __float2bfloat16_rn(0.f);
        return;
    }
    const float gi = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + 1e-8f);
    w[i] = wi;
    wbf[i] = __float2bfloat16_rn(wi);
}

__global__ void k_mlp_to_bf16(const float* __restrict__ w, __nv_bfloat16* __restrict__ wbf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kPad) wbf[i] = __float2bfloat16_rn(w[i]);
}

// ---- FP32 debug gradient (canonical layout, no BF16 rounding) ----
// One thread per row: forward and backward of the network in plain FP32
// (inputs, weights, activations and accumulation), products summed in index
// order; the row's gradient of the mean squared error goes to G[row][9347].
// A second launch sums the rows in row order, one thread per parameter, so
// the result does not depend on scheduling.
constexpr int kCW1 = 0, kCB1 = 12 * 64, kCW2 = kCB1 + 64, kCB2 = kCW2 + 64 * 64, kCW3 = kCB2 + 64,
              kCB3 = kCW3 + 64 * 64, kCW4 = kCB3 + 64, kCB4 = kCW4 + 64 * 3, kCN = kCB4 + 3;
static_assert(kCN == 9347, "canonical parameter count");

__device__ __forceinline__ float gelu_grad_f32(float z) {
    const float t = tanhf(kGeluC * (z + 0.044715f * z * z * z));
    return 0.5f * (1.f + t) + 0.5f * z * (1.f - t * t) * kGeluC * (1.f + 3.f * 0.044715f * z * z);
}

__global__ void __launch_bounds__(64) k_mlp_grad_rows_f32(const float* __restrict__ w,
                                                           const float* __restrict__ X,
                                                           const float* __restrict__ Y, int n,
                                                           float* __restrict__ G,
                                                           float* __restrict__ lrow) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float x[12], z1[64], z2[64], z3[64], h1[64], h2[64], h3[64], pr[3], dy[3];
    for (int k = 0; k < 12; k++) x[k] = X[(size_t)r * 12 + k];
    const int inW[3] = {kCW1, kCW2, kCW3}, inB[3] = {kCB1, kCB2, kCB3}, fan[3] = {12, 64, 64};
    float* zs[3] = {z1, z2, z3};
    float* hs[3] = {h1, h2, h3};
    const float* in = x;
    for (int L = 0; L < 3; L++) {
        for (int j = 0; j < 64; j++) {
            float a = w[inB[L] + j];
            for (int k = 0; k < fan[L]; k++) a = fmaf(in[k], w[inW[L] + k * 64 + j], a);
            zs[L][j] = a;
            hs[L][j] = gelu(a);
        }
        in = hs[L];
    }
    float ls = 0.f;
    for (int c = 0; c < 3; c++) {
        float a = w[kCB4 + c];
        for (int k = 0; k < 64; k++) a = fmaf(h3[k], w[kCW4 + k * 3 + c], a);
        pr[c] = a;
        const float d = a - Y[(size_t)r * 3 + c];
        ls = fmaf(d, d, ls);
        dy[c] = 2.f * d / (3.f * (float)n);
    }
    lrow[r] = ls;
    float* g = G + (size_t)r * kCN;
    for (int c = 0; c < 3; c++) g[kCB4 + c] = dy[c];
    for (int k = 0; k < 64; k++)
        for (int c = 0; c < 3; c++) g[kCW4 + k * 3 + c] = h3[k] * dy[c];
    // layer 3: dZ3 = (W4 dy) * gelu'(Z3), kept in z3
    for (int j = 0; j < 64; j++) {
        float a = 0.f;
        for (int c = 0; c < 3; c++) a = fmaf(w[kCW4 + j * 3 + c], dy[c], a);
        z3[j] = a * gelu_grad_f32(z3[j]);
    }
    // layers 3, 2, 1: weight and bias gradients, then the previous layer's dZ
    const float* dz = z3;
    for (int L = 2; L >= 0; L--) {
        const float* prev = L == 0 ? x : hs[L - 1];
        for (int j = 0; j < 64; j++) g[inB[L] + j] = dz[j];
        for (int k = 0; k < fan[L]; k++)
            for (int j = 0; j < 64; j++) g[inW[L] + k * 64 + j] = prev[k] * dz[j];
        if (L > 0) {
            float* zp = zs[L - 1];
            for (int k = 0; k < 64; k++) {
                float a = 0.f;
                for (int j = 0; j < 64; j++) a = fmaf(w[inW[L] + k * 64 + j], dz[j], a);
                zp[k] = a * gelu_grad_f32(zp[k]);
            }
            dz = zp;
        }
    }
}

__global__ void __launch_bounds__(256) k_mlp_grad_sum_f32(const float* __restrict__ G,
                                                          const float* __restrict__ lrow, int n,
                                                          float* __restrict__ grad, float* __restrict__ loss) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < kCN) {
        float a = 0.f;
        for (int r = 0; r < n; r++) a += G[(size_t)r * kCN + j];
        grad[j] = a;
    }
    if (j == 0) {
        float l = 0.f;
        for (int r = 0; r < n; r++) l += lrow[r];
        *loss = l / (3.f * (float)n);
    }
}

// ---- requests (target slot, image, cell entry) ----

struct CellView {
    double px, py, pz;      // target point (target minus image offset)
    double cx, cy, cz, M, w;
    double Q[6];
    int first, count, level, slot, code;
};

__device__ void req_view(const ReqArgs& A, uint64_t r, CellView& v) {
    v.slot = (int)(r >> 40);
    v.code = (int)((r >> 28) & 0xFFFull);
    const int e = (int)(r & 0xFFFFFFFull);
    const int gx = (v.code & 15) - 7, gy = ((v.code >> 4) & 15) - 7, gz = ((v.code >> 8) & 15) - 7;
    const BoxP bp = A.boxes[A.box[v.slot]];
    const double s = shear_offset(bp, time_of(A.ctl, A.t0, A.half_dt, A.hs));
    double ox, oy, oz;
    image_offset(bp, s, gx, gy, gz, ox, oy, oz);
    v.px = A.x[v.slot] - ox;
    v.py = A.y[v.slot] - oy;
    v.pz = A.z[v.slot] - oz;
    const double4_32a a = A.d_a[e], q0 = A.d_q0[e], q1 = A.d_q1[e];
    v.cx = a.x; v.cy = a.y; v.cz = a.z;
    v.M = q0.x;
    v.Q[0] = q0.y; v.Q[1] = q0.z; v.Q[2] = q0.w; v.Q[3] = q1.x; v.Q[4] = q1.y; v.Q[5] = q1.z;
    v.w = q1.w;
    v.first = A.e_first[e];
    v.count = A.e_count[e];
    v.level = A.e_level[e];
}

// The 12 network inputs (see the oracle's definition) and R^2 = |p - com|^2.
__device__ void req_features(const ReqArgs& A, const CellView& v, float* f, double& R2) {
    const double rx = v.px - v.cx, ry = v.py - v.cy, rz = v.pz - v.cz;
    R2 = rx * rx + ry * ry + rz * rz;
    const double R = sqrt(R2);
    const double hx = rx / R, hy = ry / R, hz = rz / R;
    const BoxP bp = A.boxes[A.box[v.first]];
    const double lo = -0.5 * bp.L;
    const uint64_t key = A.key[v.first];
    const int sh = kMaxDepth - v.level;
    const double ix = (double)(morton_compact3(key >> 2) >> sh);
    const double iy = (double)(morton_compact3(key >> 1) >> sh);
    const double iz = (double)(morton_compact3(key) >> sh);
    const double ccx = lo + (ix + 0.5) * v.w, ccy = lo + (iy + 0.5) * v.w, ccz = lo + (iz + 0.5) * v.w;
    const double sc = 1.0 / (v.M * v.w * v.w);
    const double qxx = v.Q[0] * sc, qyy = v.Q[1] * sc, qzz = v.Q[2] * sc;
    const double qxy = v.Q[3] * sc, qxz = v.Q[4] * sc, qyz = v.Q[5] * sc;
    const double ux = qxx * hx + qxy * hy + qxz * hz;
    const double uy = qxy * hx + qyy * hy + qyz * hz;
    const double uz = qxz * hx + qyz * hy + qzz * hz;
    f[0] = (float)hx; f[1] = (float)hy; f[2] = (float)hz;
    f[3] = (float)(v.w / R);
    f[4] = (float)log10((double)v.count);
    f[5] = (float)((v.cx - ccx) / v.w); f[6] = (float)((v.cy - ccy) / v.w); f[7] = (float)((v.cz - ccz) / v.w);
    f[8] = (float)(hx * ux + hy * uy + hz * uz);
    f[9] = (float)sqrt(ux * ux + uy * uy + uz * uz);
    f[10] = (float)(qxx * qxx + qyy * qyy + qzz * qzz + 2.0 * (qxy * qxy + qxz * qxz + qyz * qyz));
    f[11] = (float)(qxx * (qyy * qzz - qyz * qyz) - qxy * (qxy * qzz - qyz * qxz) +
                    qxz * (qxy * qyz - qyy * qxz));
}

// Residual labels: (exact cell force - multipole force) / (G M / R^2); the
// exact force is Eq. 1 summed over the cell's particles by one warp.
__global__ void __launch_bounds__(256) k_mlp_label(ReqArgs A, float* __restrict__ X,
                                                   float* __restrict__ Y, int64_t* __restrict__ meta) {
    const int nreq = min(*A.req_count, A.req_cap);
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int r = warp; r < nreq; r += nwarps) {
        CellView v;
        req_view(A, A.req[r], v);
        double sx = 0.0, sy = 0.0, sz = 0.0;
        int minid = 0x7fffffff;
        for (int j = v.first + lane; j < v.first + v.count; j += 32) {
            const double dx = A.x[j] - v.px, dy = A.y[j] - v.py, dz = A.z[j] - v.pz;
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double inv = 1.0 / sqrt(r2);
            const double f = source_mass(A.boxes[A.box[j]], A.id[j], A.m[j]) * inv * inv * inv;
            sx += f * dx;
            sy += f * dy;
            sz += f * dz;
            minid = min(minid, A.id[j]);
        }
        for (int o = 16; o > 0; o >>= 1) {
            sx += __shfl_down_sync(0xffffffffu, sx, o);
            sy += __shfl_down_sync(0xffffffffu, sy, o);
            sz += __shfl_down_sync(0xffffffffu, sz, o);
            minid = min(minid, __shfl_down_sync(0xffffffffu, minid, o));
        }
        if (lane == 0) {
            float f[12];
            double R2;
            req_features(A, v, f, R2);
            // multipole force of the cell (monopole + quadrupole, unsoftened)
            const double dx = v.cx - v.px, dy = v.cy - v.py, dz = v.cz - v.pz;
            const double inv = 1.0 / sqrt(R2);
            const double inv3 = inv * inv * inv, inv5 = inv3 * inv * inv;
            const double qx = v.Q[0] * dx + v.Q[3] * dy + v.Q[4] * dz;
            const double qy = v.Q[3] * dx + v.Q[1] * dy + v.Q[5] * dz;
            const double qz = v.Q[4] * dx + v.Q[5] * dy + v.Q[2] * dz;
            const double dqd = dx * qx + dy * qy + dz * qz;
            const double c = 2.5 * dqd * inv5 * inv * inv;
            const double mx = v.M * inv3 * dx + c * dx - inv5 * qx;
            const double my = v.M * inv3 * dy + c * dy - inv5 * qy;
            const double mz = v.M * inv3 * dz + c * dz - inv5 * qz;
            const double unit = v.M / R2;   // G cancels
            for (int k = 0; k < 12; k++) X[(size_t)r * 12 + k] = f[k];
            Y[(size_t)r * 3 + 0] = (float)((sx - mx) / unit);
            Y[(size_t)r * 3 + 1] = (float)((sy - my) / unit);
            Y[(size_t)r * 3 + 2] = (float)((sz - mz) / unit);
            if (meta) {
                meta[(size_t)r * 5 + 0] = A.id[v.slot];
                meta[(size_t)r * 5 + 1] = v.code;
                meta[(size_t)r * 5 + 2] = v.level;
                meta[(size_t)r * 5 + 3] = minid;
                meta[(size_t)r * 5 + 4] = v.count;
            }
        }
    }
}

// Inference layout (Packed) of the padded FP32 weights: one thread per B
// fragment entry, then the biases.
__global__ void k_mlp_pack(const float* __restrict__ w, Packed* __restrict__ P) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    constexpr int n1 = 8 * 32, n2 = 32 * 32, n4 = 4 * 32;
    if (i < n1 + 2 * n2 + n4) {
        int k = i, off, ld, nt;
        uint2* dst;
        if (k < n1) {
            off = kW1; ld = 64; nt = 8; dst = &P->B1[0][0][0];
        } else if ((k -= n1) < n2) {
            off = kW2; ld = 64; nt = 8; dst = &P->B2[0][0][0];
        } else if ((k -= n2) < n2) {
            off = kW3; ld = 64; nt = 8; dst = &P->B3[0][0][0];
        } else {
            k -= n2;
            off = kW4; ld = 8; nt = 1; dst = &P->B4[0][0][0];
        }
        const int lane = k & 31, tile = k >> 5, t = tile / nt, j = tile % nt;
        const int g = lane >> 2, q = lane & 3, r = 16 * t + 2 * q, c = 8 * j + g;
        const float* W = w + off;
        uint2 b;
        b.x = pack2(W[r * ld + c], W[(r + 1) * ld + c]);
        b.y = pack2(W[(r + 8) * ld + c], W[(r + 9) * ld + c]);
        dst[k] = b;
    } else if ((i -= n1 + 2 * n2 + n4) < 200) {
        if (i < 64) P->b1[i] = w[kB1 + i];
        else if (i < 128) P->b2[i - 64] = w[kB2 + i - 64];
        else if (i < 192) P->b3[i - 128] = w[kB3 + i - 128];
        else P->b4[i - 192] = w[kB4 + i - 192];
    }
}

}  // namespace

void label_async(const ReqArgs& A, float* X, float* Y, int64_t* meta, int max_req, cudaStream_t s) {
    const int blocks = std::max(1, std::min((max_req + 7) / 8, 8 * 152));
    k_mlp_label<<<blocks, 256, 0, s>>>(A, X, Y, meta);
}

void pack_async(const float* w, Packed* packed, cudaStream_t s) {
    constexpr int n = 8 * 32 + 2 * 32 * 32 + 4 * 32 + 200;
    k_mlp_pack<<<(n + 255) / 256, 256, 0, s>>>(w, packed);
}

// ---- host helpers ----

int padded_size() { return kPad; }

// canonical (9347) <-> padded (9928)
void to_padded(const float* c, float* p) {
    std::fill(p, p + kPad, 0.f);
    int k = 0;
    const int in[4] = {12, 64, 64, 64}, out[4] = {64, 64, 64, 3};
    const int offw[4] = {kW1, kW2, kW3, kW4}, offb[4] = {kB1, kB2, kB3, kB4};
    const int ldp[4] = {64, 64, 64, 8};
    for (int L = 0; L < 4; L++) {
        for (int i = 0; i < in[L]; i++)
            for (int o = 0; o < out[L]; o++) p[offw[L] + i * ldp[L] + o] = c[k++];
        for (int o = 0; o < out[L]; o++) p[offb[L] + o] = c[k++];
    }
}

void from_padded(const float* p, float* c) {
    int k = 0;
    const int in[4] = {12, 64, 64, 64}, out[4] = {64, 64, 64, 3};
    const int offw[4] = {kW1, kW2, kW3, kW4}, offb[4] = {kB1, kB2, kB3, kB4};
    const int ldp[4] = {64, 64, 64, 8};
    for (int L = 0; L < 4; L++) {
        for (int i = 0; i < in[L]; i++)
            for (int o = 0; o < out[L]; o++) c[k++] = p[offw[L] + i * ldp[L] + o];
        for (int o = 0; o < out[L]; o++) c[k++] = p[offb[L] + o];
    }
}

size_t train_smem_bytes() { return sizeof(TrainSmem); }

// Gradient (padded; zeroed first) of the mean squared error of the rows
// idx[0..n) with n_total as the mean's denominator; the summed squared
// error is added to *loss.  Device pointers; async on s.
cudaError_t grad_async(const void* wbf, const float* wf, const float* X, const float* Y,
                       const int32_t* idx, int n, int n_total, float* grad, float* loss,
                       cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(TrainSmem));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    cudaMemsetAsync(grad, 0, sizeof(float) * kPad, s);
    const int tiles = (n + 15) / 16;
    const int blocks = std::max(1, std::min((tiles + kWarps - 1) / kWarps, 2 * 152));
    k_mlp_grad<<<blocks, kWarps * 32, sizeof(TrainSmem), s>>>(
        static_cast<const __nv_bfloat16*>(wbf), wf, X, Y, idx, n, n_total, grad, loss);
    return cudaGetLastError();
}

cudaError_t grad_f32_async(const float* w, const float* X, const float* Y, int n, float* G, float* lrow,
                           float* grad, float* loss, cudaStream_t s) {
    k_mlp_grad_rows_f32<<<(n + 63) / 64, 64, 0, s>>>(w, X, Y, n, G, lrow);
    k_mlp_grad_sum_f32<<<(kCN + 255) / 256, 256, 0, s>>>(G, lrow, n, grad, loss);
    return cudaGetLastError();
}

void adam_async(float* w, float* m, float* v, const float* grad, void* wbf, float lr, int step,
                cudaStream_t s) {
    const float c1 = 1.f - powf(0.9f, (float)step), c2 = 1.f - powf(0.999f, (float)step);
    k_mlp_adam<<<(kPad + 255) / 256, 256, 0, s>>>(w, m, v, grad, static_cast<__nv_bfloat16*>(wbf),
                                                  lr, c1, c2);
}

void to_bf16_async(const float* w, void* wbf, cudaStream_t s) {
    k_mlp_to_bf16<<<(kPad + 255) / 256, 256, 0, s>>>(w, static_cast<__nv_bfloat16*>(wbf));
}

}  // namespace mlp
}  // namespace rb
