// sdm_surrogate.cuh -- learned stand-in for the gravitational collision kernel.
//
// Not in the paper: a small multilayer perceptron maps the pair's radii to the
// kernel value, trained on the GPU by the kernels below on pairs whose targets
// come from the plain FP64 kernel, with the plain kernel kept as the fallback
// wherever the network's relative error on a validation grid exceeds a threshold.
//
//   z = ((ln R - c0) / c1, (ln r - c0) / c1)      R >= r the pair's radii,
//       c0, c1 the centre and half-width of ln r over the training range
//   h1 = silu(W1 z + b1), h2 = silu(W2 h1 + b2), h3 = silu(W3 h2 + b3)   (64 each)
//   y  = w4 . h3 + b4
//   K^ = exp(mu + sigma y) - K_floor, clamped at 0  (the network fits the
//        standardised ln(K + K_floor); K_floor keeps the target finite where
//        vt(R) = vt(r) makes K vanish)
//
// Weights are kept in FP32 for the optimiser and used rounded to BF16 (round to
// nearest even) in every forward and backward pass; activations and sums are FP32.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace sdm {

constexpr int SURR_H = 64;                 // hidden width
constexpr int SURR_W1 = 0;                 // [64][2]
constexpr int SURR_B1 = SURR_W1 + SURR_H * 2;
constexpr int SURR_W2 = SURR_B1 + SURR_H;  // [64][64], row j = inputs of unit j
constexpr int SURR_B2 = SURR_W2 + SURR_H * SURR_H;
constexpr int SURR_W3 = SURR_B2 + SURR_H;
constexpr int SURR_B3 = SURR_W3 + SURR_H * SURR_H;
constexpr int SURR_W4 = SURR_B3 + SURR_H;  // [64]
constexpr int SURR_B4 = SURR_W4 + SURR_H;
constexpr int SURR_NPARAM = SURR_B4 + 1;   // 8577
constexpr int SURR_NPS = (SURR_NPARAM + 3) & ~3;   // stride of the parameter-sized device arrays
constexpr int SURR_TILES = 256;            // fallback mask: tiles per input axis over [-1, 1]

// What a step needs of a trained surrogate (device pointers).
struct SurrogateDev {
    const float* w;          // [SURR_NPARAM] BF16-rounded parameters, stored as float
    const uint8_t* mask;     // [SURR_TILES][SURR_TILES] 1: use the network, 0: plain kernel
    float c0, c1;            // input normalisation of ln r
    float mu, sigma;         // target standardisation
    float k_floor;           // [m^3/s]
    float r_min, r_max;      // training range of the radii [m]
};

__device__ __forceinline__ float silu_f(float x) { return x / (1.0f + __expf(-x)); }

// silu'(x) = s (1 + x (1 - s)), s = 1 / (1 + e^-x)
__device__ __forceinline__ float silu_grad_f(float x)
{
    const float s = 1.0f / (1.0f + __expf(-x));
    return s * (1.0f + x * (1.0f - s));
}

__device__ __forceinline__ float bf16_round(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// Network output y for inputs (z0, z1); w are the BF16-rounded parameters in global
// memory (read through L1).  Rolled loops keep the code small.
__device__ __noinline__ float surr_forward(const float* __restrict__ w, float z0, float z1)
{
    float h[SURR_H], g[SURR_H];
#pragma unroll 4
    for (int j = 0; j < SURR_H; ++j)
        h[j] = silu_f(fmaf(__ldg(w + SURR_W1 + 2 * j), z0, fmaf(__ldg(w + SURR_W1 + 2 * j + 1), z1, __ldg(w + SURR_B1 + j))));
#pragma unroll 1
    for (int j = 0; j < SURR_H; ++j) {
        const float* row = w + SURR_W2 + SURR_H * j;
        float acc = __ldg(w + SURR_B2 + j);
#pragma unroll
        for (int k = 0; k < SURR_H; ++k) acc = fmaf(__ldg(row + k), h[k], acc);
        g[j] = silu_f(acc);
    }
#pragma unroll 1
    for (int j = 0; j < SURR_H; ++j) {
        const float* row = w + SURR_W3 + SURR_H * j;
        float acc = __ldg(w + SURR_B3 + j);
#pragma unroll
        for (int k = 0; k < SURR_H; ++k) acc = fmaf(__ldg(row + k), g[k], acc);
        h[j] = silu_f(acc);
    }
    float y = __ldg(w + SURR_B4);
#pragma unroll
    for (int k = 0; k < SURR_H; ++k) y = fmaf(__ldg(w + SURR_W4 + k), h[k], y);
    return y;
}

// Surrogate kernel value for radii R >= r, or a negative number when the pair must use
// the plain kernel (outside the training range or in a masked tile).
__device__ __forceinline__ float surr_kernel(const SurrogateDev& S, float R, float r)
{
    if (!(r >= S.r_min) || !(R <= S.r_max)) return -1.0f;
    const float z0 = (__logf(R) - S.c0) / S.c1, z1 = (__logf(r) - S.c0) / S.c1;
    const int a = min(SURR_TILES - 1, max(0, (int)((z0 + 1.0f) * (0.5f * SURR_TILES))));
    const int b = min(SURR_TILES - 1, max(0, (int)((z1 + 1.0f) * (0.5f * SURR_TILES))));
    if (!S.mask[a * SURR_TILES + b]) return -1.0f;
    const float y = surr_forward(S.w, z0, z1);
    return fmaxf(__expf(fmaf(S.sigma, y, S.mu)) - S.k_floor, 0.0f);
}

// ---------------------------------------------------------------------------
// Training: samples are pairs of radii drawn log-uniform in [r_min, r_max] by
// Philox (counter (i, 0, 0, 3), key = seed; two words per radius), with
// targets from the plain FP64 kernel.
// ---------------------------------------------------------------------------
struct SurrTrainArgs {
    float* w32;              // FP32 master parameters
    float* wbf;              // BF16-rounded copy used by the passes
    float* grad;             // [SURR_NPARAM] accumulated gradient of the loss
    float* m;                // Adam moments
    float* v;
    float* loss;             // [1] accumulated loss of the current step
    uint32_t seed_lo, seed_hi;
    double ln_rmin, ln_rmax;
    float c0, c1, mu, sigma;
    double k_floor;
    uint64_t n_train;        // size of the training set (sample index modulo n_train)
};

// pair i of the training set: radii R >= r, features and target
__device__ __forceinline__ void surr_sample(const SurrTrainArgs& A, uint64_t i, float& z0, float& z1, float& t,
                                            double& K)
{
    const U4 x = philox((uint32_t)i, (uint32_t)(i >> 32), 0u, 3u, A.seed_lo, A.seed_hi);
    const double u1 = ((double)(x.x >> 8) + 0.5) * 0x1p-24, u2 = ((double)(x.y >> 8) + 0.5) * 0x1p-24;
    double l1 = A.ln_rmin + (A.ln_rmax - A.ln_rmin) * u1, l2 = A.ln_rmin + (A.ln_rmax - A.ln_rmin) * u2;
    if (l2 > l1) { const double s = l1; l1 = l2; l2 = s; }
    const double R = exp(l1), r = exp(l2);
    const double c = 4.0 / 3.0 * PI_D;
    K = kernel_grav_d(c * R * R * R, c * r * r * r);
    z0 = (float)((l1 - A.c0) / A.c1);
    z1 = (float)((l2 - A.c0) / A.c1);
    t = (float)((log(K + A.k_floor) - A.mu) / A.sigma);
}

__global__ void surr_targets_kernel(SurrTrainArgs A, uint64_t n, double* K_out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        float z0, z1, t;
        double K;
        surr_sample(A, i, z0, z1, t, K);
        K_out[i] = K;
    }
}

// ---------------------------------------------------------------------------
// Inference on the tensor cores for a warp's 32 pairs at once (the queued pairs a
// step evaluates together).  The samples are the rows of the activation matrix
// (M = 32: two m16 tiles), the 64 hidden units its columns; the 64 x 64 layers are
// mma.sync m16n8k16 products with BF16 operands and FP32 accumulation.  An FP32
// activation x enters as hi + lo with hi = bf16(x), lo = bf16(x - hi), two products
// per tile, so that the result keeps ~16 bits of each activation (the weights are
// BF16 already).  The accumulator layout of two adjacent n8 tiles is the operand
// layout of one k16 slab, so a layer's output feeds the next layer from registers.
//   fragments (lane = 4 g + t): A regs {(g, 2t..2t+1), (g+8, 2t..), (g, 2t+8..),
//   (g+8, 2t+8..)}; B regs {(k = 2t..2t+1, n = g), (k = 2t+8.., n = g)};
//   C/D {(g, 2t), (g, 2t+1), (g+8, 2t), (g+8, 2t+1)}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t bf16x2_bits(float lo_elem, float hi_elem)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo_elem, hi_elem);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// hi and lo BF16 operand registers of four FP32 values laid out as one A register pair set
__device__ __forceinline__ void split_bf16(float x0, float x1, uint32_t& hi, uint32_t& lo)
{
    const float h0 = bf16_round(x0), h1 = bf16_round(x1);
    hi = bf16x2_bits(h0, h1);
    lo = bf16x2_bits(x0 - h0, x1 - h1);
}

constexpr int SURR_TB = 64;                // samples per CTA of the training pass
constexpr int SURR_THREADS = 256;

constexpr int SURR_ZS = SURR_H + 1;         // row stride of the activation arrays (no bank conflicts)

// dynamic shared memory of the training pass
struct SurrSmem {
    float w[SURR_NPARAM];
    float z[SURR_TB][2];
    float t[SURR_TB];
    float y[SURR_TB];
    float Z1[SURR_TB][SURR_ZS], Z2[SURR_TB][SURR_ZS], Z3[SURR_TB][SURR_ZS];   // pre-activations
    float D[SURR_TB][SURR_ZS];                                             // dL/dZ of the current layer
    float E[SURR_TB][SURR_ZS];                                             // dL/dZ of the layer below
};

// The 64 x 64 products of the training pass on the tensor cores (mma.sync m16n8k16, BF16
// operands, FP32 sums).  Each product's output is 4 m16 x 8 n8 tiles; warp w of the 8 takes row
// tile w & 3 and column tiles 4 (w >> 2) .. + 3.  An FP32 operand x enters as hi + lo (hi =
// bf16(x), lo = bf16(x - hi)); the weights are BF16 already.  Fragment layout (lane = 4 g + t):
// A regs (row g, cols 2t..2t+1), (g + 8, 2t..), (g, 2t + 8..), (g + 8, 2t + 8..); B regs
// (k = 2t..2t+1, col g), (k = 2t + 8.., col g); C (g, 2t), (g, 2t+1), (g + 8, 2t), (g + 8, 2t+1).

// Zout[s][j] = b[j] + sum_k W[j][k] silu(Zin[s][k])  (forward of a hidden layer; rows: samples)
__device__ __forceinline__ void surr_tc_forward(const float* __restrict__ W, const float* __restrict__ b,
                                                const float (*Zin)[SURR_ZS], float (*Zout)[SURR_ZS], int warp,
                                                int lane)
{
    const int g = lane >> 2, t = lane & 3, r0 = 16 * (warp & 3) + g, n0 = 32 * (warp >> 2);
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const float b0 = b[n0 + 8 * j + 2 * t], b1 = b[n0 + 8 * j + 2 * t + 1];
        acc[j][0] = b0; acc[j][1] = b1; acc[j][2] = b0; acc[j][3] = b1;
    }
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        const int c = 16 * ks + 2 * t;
        uint32_t ahi[4], alo[4];
        split_bf16(silu_f(Zin[r0][c]), silu_f(Zin[r0][c + 1]), ahi[0], alo[0]);
        split_bf16(silu_f(Zin[r0 + 8][c]), silu_f(Zin[r0 + 8][c + 1]), ahi[1], alo[1]);
        split_bf16(silu_f(Zin[r0][c + 8]), silu_f(Zin[r0][c + 9]), ahi[2], alo[2]);
        split_bf16(silu_f(Zin[r0 + 8][c + 8]), silu_f(Zin[r0 + 8][c + 9]), ahi[3], alo[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float* row = W + SURR_H * (n0 + 8 * j + g);          // B(k, n) = W[n][k]
            const uint32_t b0 = bf16x2_bits(row[c], row[c + 1]), b1 = bf16x2_bits(row[c + 8], row[c + 9]);
            mma_bf16_16816(acc[j], ahi, b0, b1);
            mma_bf16_16816(acc[j], alo, b0, b1);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = n0 + 8 * j + 2 * t;
        Zout[r0][col] = acc[j][0];
        Zout[r0][col + 1] = acc[j][1];
        Zout[r0 + 8][col] = acc[j][2];
        Zout[r0 + 8][col + 1] = acc[j][3];
    }
}

// E[s][k] = (sum_j D[s][j] W[j][k]) silu'(Zb[s][k])  (dL/dZ of the layer below)
__device__ __forceinline__ void surr_tc_backprop(const float* __restrict__ W, const float (*D)[SURR_ZS],
                                                 const float (*Zb)[SURR_ZS], float (*E)[SURR_ZS], int warp, int lane)
{
    const int g = lane >> 2, t = lane & 3, r0 = 16 * (warp & 3) + g, n0 = 32 * (warp >> 2);
    float acc[4][4] = {};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        const int c = 16 * ks + 2 * t;
        uint32_t ahi[4], alo[4];
        split_bf16(D[r0][c], D[r0][c + 1], ahi[0], alo[0]);
        split_bf16(D[r0 + 8][c], D[r0 + 8][c + 1], ahi[1], alo[1]);
        split_bf16(D[r0][c + 8], D[r0][c + 9], ahi[2], alo[2]);
        split_bf16(D[r0 + 8][c + 8], D[r0 + 8][c + 9], ahi[3], alo[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + 8 * j + g;                                 // B(k = j', n) = W[j'][n]
            const uint32_t b0 = bf16x2_bits(W[SURR_H * c + n], W[SURR_H * (c + 1) + n]);
            const uint32_t b1 = bf16x2_bits(W[SURR_H * (c + 8) + n], W[SURR_H * (c + 9) + n]);
            mma_bf16_16816(acc[j], ahi, b0, b1);
            mma_bf16_16816(acc[j], alo, b0, b1);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = n0 + 8 * j + 2 * t;
        E[r0][col] = acc[j][0] * silu_grad_f(Zb[r0][col]);
        E[r0][col + 1] = acc[j][1] * silu_grad_f(Zb[r0][col + 1]);
        E[r0 + 8][col] = acc[j][2] * silu_grad_f(Zb[r0 + 8][col]);
        E[r0 + 8][col + 1] = acc[j][3] * silu_grad_f(Zb[r0 + 8][col + 1]);
    }
}

// grad[j][k] += sum_s D[s][j] silu(Zb[s][k])  (the layer's weight gradient; K = the 64 samples)
__device__ __forceinline__ void surr_tc_weight_grad(float* __restrict__ grad, const float (*D)[SURR_ZS],
                                                    const float (*Zb)[SURR_ZS], int warp, int lane)
{
    const int g = lane >> 2, t = lane & 3, m0 = 16 * (warp & 3), n0 = 32 * (warp >> 2);
    float acc[4][4] = {};
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        const int s = 16 * ks + 2 * t;                                   // sample (the K index)
        uint32_t ahi[4], alo[4];                                          // A(m = j, k = s) = D[s][j]
        split_bf16(D[s][m0 + g], D[s + 1][m0 + g], ahi[0], alo[0]);
        split_bf16(D[s][m0 + g + 8], D[s + 1][m0 + g + 8], ahi[1], alo[1]);
        split_bf16(D[s + 8][m0 + g], D[s + 9][m0 + g], ahi[2], alo[2]);
        split_bf16(D[s + 8][m0 + g + 8], D[s + 9][m0 + g + 8], ahi[3], alo[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + 8 * j + g;                                 // B(k = s, n) = silu(Zb[s][n])
            uint32_t bhi0, blo0, bhi1, blo1;
            split_bf16(silu_f(Zb[s][n]), silu_f(Zb[s + 1][n]), bhi0, blo0);
            split_bf16(silu_f(Zb[s + 8][n]), silu_f(Zb[s + 9][n]), bhi1, blo1);
            mma_bf16_16816(acc[j], ahi, bhi0, bhi1);
            mma_bf16_16816(acc[j], ahi, blo0, blo1);
            mma_bf16_16816(acc[j], alo, bhi0, bhi1);
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int col = n0 + 8 * j + 2 * t;
        atomicAdd(grad + SURR_H * (m0 + g) + col, acc[j][0]);
        atomicAdd(grad + SURR_H * (m0 + g) + col + 1, acc[j][1]);
        atomicAdd(grad + SURR_H * (m0 + g + 8) + col, acc[j][2]);
        atomicAdd(grad + SURR_H * (m0 + g + 8) + col + 1, acc[j][3]);
    }
}

// One CTA: forward and backward of SURR_TB samples; adds the loss and the gradient of
// mean((y - t)^2) over the whole batch (n_batch samples) to A.loss and A.grad.  The
// samples are given either by index (training set, x_ext == nullptr) or by features
// and targets in device memory (x_ext [n][2], t_ext [n]; the gradient check).  The two
// 64 x 64 layers' products (forward, backward, weight gradients) run on the tensor cores.
__global__ void __launch_bounds__(SURR_THREADS) surr_pass_kernel(SurrTrainArgs A, uint64_t first, uint64_t n_batch,
                                                                 const float* x_ext, const float* t_ext)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SurrSmem& S = *reinterpret_cast<SurrSmem*>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int k = tid; k < SURR_NPARAM; k += SURR_THREADS) S.w[k] = A.wbf[k];
    const uint64_t s0 = (uint64_t)blockIdx.x * SURR_TB;
    if (tid < SURR_TB) {
        float z0 = 0.f, z1 = 0.f, t = 0.f;
        if (s0 + tid < n_batch) {
            if (x_ext) {
                z0 = x_ext[2 * (s0 + tid)];
                z1 = x_ext[2 * (s0 + tid) + 1];
                t = t_ext[s0 + tid];
            } else {
                double K;
                surr_sample(A, (first + s0 + tid) % A.n_train, z0, z1, t, K);
            }
        }
        S.z[tid][0] = z0;
        S.z[tid][1] = z1;
        S.t[tid] = t;
    }
    __syncthreads();
    // forward: the first layer (two inputs) on the FP32 pipe, the others on the tensor cores
    const int s = tid >> 2, jq = tid & 3;
    for (int j = jq; j < SURR_H; j += 4)
        S.Z1[s][j] = fmaf(S.w[SURR_W1 + 2 * j], S.z[s][0], fmaf(S.w[SURR_W1 + 2 * j + 1], S.z[s][1], S.w[SURR_B1 + j]));
    __syncthreads();
    surr_tc_forward(S.w + SURR_W2, S.w + SURR_B2, S.Z1, S.Z2, warp, lane);
    __syncthreads();
    surr_tc_forward(S.w + SURR_W3, S.w + SURR_B3, S.Z2, S.Z3, warp, lane);
    __syncthreads();
    if (tid < SURR_TB) {
        float y = S.w[SURR_B4];
        for (int k = 0; k < SURR_H; ++k) y = fmaf(S.w[SURR_W4 + k], silu_f(S.Z3[tid][k]), y);
        const bool in = s0 + tid < n_batch;
        const float d = in ? y - S.t[tid] : 0.0f;
        S.y[tid] = in ? 2.0f * d / (float)n_batch : 0.0f;        // dL/dy
        float l = d * d / (float)n_batch;
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if ((tid & 31) == 0) atomicAdd(A.loss, l);
    }
    __syncthreads();
    // output layer: dL/dZ3 = dy w4 silu'(Z3); gradients of w4, b4
    for (int j = jq; j < SURR_H; j += 4) S.D[s][j] = S.y[s] * S.w[SURR_W4 + j] * silu_grad_f(S.Z3[s][j]);
    if (tid < SURR_H) {
        float g = 0.f;
        for (int q = 0; q < SURR_TB; ++q) g = fmaf(S.y[q], silu_f(S.Z3[q][tid]), g);
        atomicAdd(A.grad + SURR_W4 + tid, g);
    } else if (tid == SURR_H) {
        float g = 0.f;
        for (int q = 0; q < SURR_TB; ++q) g += S.y[q];
        atomicAdd(A.grad + SURR_B4, g);
    }
    __syncthreads();
    // hidden layers 3 and 2: dW = D^T silu(Zbelow), dZbelow = (D W) silu'(Zbelow), both on the
    // tensor cores; the bias gradients are column sums of D
    for (int layer = 3; layer >= 2; --layer) {
        const int OW = layer == 3 ? SURR_W3 : SURR_W2, OB = layer == 3 ? SURR_B3 : SURR_B2;
        const float (*Zb)[SURR_ZS] = layer == 3 ? S.Z2 : S.Z1;
        surr_tc_weight_grad(A.grad + OW, S.D, Zb, warp, lane);
        if (tid < SURR_H) {
            float g = 0.f;
            for (int q = 0; q < SURR_TB; ++q) g += S.D[q][tid];
            atomicAdd(A.grad + OB + tid, g);
        }
        surr_tc_backprop(S.w + OW, S.D, Zb, S.E, warp, lane);
        __syncthreads();
        for (int k = jq; k < SURR_H; k += 4) S.D[s][k] = S.E[s][k];
        __syncthreads();
    }
    // first layer: dW1[j][i] = sum_s D[s][j] z[s][i]
    if (tid < SURR_H * 2) {
        const int j = tid >> 1, i = tid & 1;
        float g = 0.f;
        for (int q = 0; q < SURR_TB; ++q) g = fmaf(S.D[q][j], S.z[q][i], g);
        atomicAdd(A.grad + SURR_W1 + tid, g);
    } else if (tid < SURR_H * 3) {
        const int j = tid - 2 * SURR_H;
        float g = 0.f;
        for (int q = 0; q < SURR_TB; ++q) g += S.D[q][j];
        atomicAdd(A.grad + SURR_B1 + j, g);
    }
}

// Adam step t (1-based) on every parameter, then the BF16 copy and a cleared gradient.
__global__ void surr_adam_kernel(SurrTrainArgs A, float lr, uint32_t t)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = 1.0f - powf(b1, (float)t), c2 = 1.0f - powf(b2, (float)t);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < SURR_NPARAM; k += gridDim.x * blockDim.x) {
        const float g = A.grad[k];
        const float m = b1 * A.m[k] + (1.0f - b1) * g;
        const float v = b2 * A.v[k] + (1.0f - b2) * g * g;
        A.m[k] = m;
        A.v[k] = v;
        const float w = A.w32[k] - lr * (m / c1) / (sqrtf(v / c2) + eps);
        A.w32[k] = w;
        A.wbf[k] = bf16_round(w);
        A.grad[k] = 0.0f;
    }
}

__global__ void surr_round_kernel(const float* w32, float* wbf)
{
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < SURR_NPARAM; k += gridDim.x * blockDim.x)
        wbf[k] = bf16_round(w32[k]);
}

// Fallback mask: tile (a, b) of the (z0, z1) grid uses the network when, at 4 x 4
// points inside it, |K^ - K| <= tol K with K from the FP64 kernel (K > 0).  Tiles
// with r > R only, or where K vanishes, keep the plain kernel.
__global__ void surr_mask_kernel(SurrogateDev S, double ln_rmin, double ln_rmax, float tol, uint8_t* mask,
                                 float* max_err)
{
    const int tile = blockIdx.x * (blockDim.x / 16) + threadIdx.x / 16;
    if (tile >= SURR_TILES * SURR_TILES) return;
    const int a = tile / SURR_TILES, b = tile % SURR_TILES, q = threadIdx.x % 16;
    const double za = -1.0 + 2.0 * (a + ((q & 3) + 0.5) / 4.0) / SURR_TILES;
    const double zb = -1.0 + 2.0 * (b + ((q >> 2) + 0.5) / 4.0) / SURR_TILES;
    const double c0 = 0.5 * (ln_rmin + ln_rmax), c1 = 0.5 * (ln_rmax - ln_rmin);
    const double R = exp(c0 + c1 * za), r = exp(c0 + c1 * zb);
    float err = INFINITY;
    if (r <= R) {
        const double c = 4.0 / 3.0 * PI_D;
        const double K = kernel_grav_d(c * R * R * R, c * r * r * r);
        const float y = surr_forward(S.w, (float)za, (float)zb);
        const double Kh = fmax(exp((double)S.mu + (double)S.sigma * (double)y) - (double)S.k_floor, 0.0);
        if (K > 0.0) err = (float)(fabs(Kh - K) / K);
    }
    for (int o = 8; o > 0; o >>= 1) err = fmaxf(err, __shfl_xor_sync(0xffffffffu, err, o, 16));
    if (q == 0) {
        mask[tile] = err <= tol ? 1u : 0u;
        max_err[tile] = err;
    }
}

// K^ of a pair of volumes (or -1: use the plain kernel); out of line so that the
// network's working set stays out of the register allocation of the step kernels
__device__ __noinline__ float surr_pair_kernel(const SurrogateDev* __restrict__ S, double v1, double v2)
{
    const float c = 0.238732414637843f;   // 3 / (4 pi)
    const float r1 = cbrtf((float)v1 * c), r2 = cbrtf((float)v2 * c);
    const SurrogateDev D = *S;
    return surr_kernel(D, fmaxf(r1, r2), fminf(r1, r2));
}

// One 64 x 64 layer for one m16 tile: out = silu(W in + b), in given as hi/lo A operand
// registers per k16 slab, out as FP32 accumulators per n8 tile.
__device__ __forceinline__ void surr_layer_mma(const float* __restrict__ W, const float* __restrict__ bias,
                                               const uint32_t (&ahi)[4][4], const uint32_t (&alo)[4][4],
                                               float (&out)[8][4], uint32_t g, uint32_t t)
{
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float2 bb = __ldg(reinterpret_cast<const float2*>(bias + 8 * j + 2 * t));
        out[j][0] = bb.x; out[j][1] = bb.y; out[j][2] = bb.x; out[j][3] = bb.y;
        const float* row = W + SURR_H * (8 * j + g);               // unit n = 8 j + g
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
            const float2 w0 = __ldg(reinterpret_cast<const float2*>(row + 16 * ks + 2 * t));
            const float2 w1 = __ldg(reinterpret_cast<const float2*>(row + 16 * ks + 2 * t + 8));
            const uint32_t b0 = bf16x2_bits(w0.x, w0.y), b1 = bf16x2_bits(w1.x, w1.y);   // exact: BF16 values
            mma_bf16_16816(out[j], ahi[ks], b0, b1);
            mma_bf16_16816(out[j], alo[ks], b0, b1);
        }
#pragma unroll
        for (int e = 0; e < 4; ++e) out[j][e] = silu_f(out[j][e]);
    }
}

// accumulators of the n8 tiles 2 ks, 2 ks + 1 -> hi/lo operands of k16 slab ks
__device__ __forceinline__ void acc_to_operand(const float (&d)[8][4], uint32_t (&ahi)[4][4], uint32_t (&alo)[4][4])
{
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
        split_bf16(d[2 * ks][0], d[2 * ks][1], ahi[ks][0], alo[ks][0]);          // (g, 2t..)
        split_bf16(d[2 * ks][2], d[2 * ks][3], ahi[ks][1], alo[ks][1]);          // (g+8, 2t..)
        split_bf16(d[2 * ks + 1][0], d[2 * ks + 1][1], ahi[ks][2], alo[ks][2]);  // (g, 2t+8..)
        split_bf16(d[2 * ks + 1][2], d[2 * ks + 1][3], ahi[ks][3], alo[ks][3]);  // (g+8, 2t+8..)
    }
}

// Network output y of the sample (z0, z1) of every lane; all 32 lanes take part.
__device__ __noinline__ float surr_forward_warp(const float* __restrict__ w, float z0, float z1)
{
    const uint32_t lane = threadIdx.x & 31u, g = lane >> 2, t = lane & 3u;
    float ysel[2][2];
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
        // layer 1 in operand layout: rows 16 mt + g and 16 mt + g + 8 of h1 = silu(W1 z + b1)
        const float za0 = __shfl_sync(0xffffffffu, z0, 16 * mt + g), za1 = __shfl_sync(0xffffffffu, z1, 16 * mt + g);
        const float zb0 = __shfl_sync(0xffffffffu, z0, 16 * mt + g + 8),
                    zb1 = __shfl_sync(0xffffffffu, z1, 16 * mt + g + 8);
        uint32_t ahi[4][4], alo[4][4];
#pragma unroll
        for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {               // columns 16 ks + 2t (+8 half)
                const int k = 16 * ks + 2 * t + 8 * half;
                const float4 wk = __ldg(reinterpret_cast<const float4*>(w + SURR_W1 + 2 * k));   // units k, k+1
                const float2 bk = __ldg(reinterpret_cast<const float2*>(w + SURR_B1 + k));
                const float pa0 = silu_f(fmaf(wk.x, za0, fmaf(wk.y, za1, bk.x)));
                const float pa1 = silu_f(fmaf(wk.z, za0, fmaf(wk.w, za1, bk.y)));
                const float pb0 = silu_f(fmaf(wk.x, zb0, fmaf(wk.y, zb1, bk.x)));
                const float pb1 = silu_f(fmaf(wk.z, zb0, fmaf(wk.w, zb1, bk.y)));
                split_bf16(pa0, pa1, ahi[ks][2 * half], alo[ks][2 * half]);
                split_bf16(pb0, pb1, ahi[ks][2 * half + 1], alo[ks][2 * half + 1]);
            }
        }
        float d[8][4];
        surr_layer_mma(w + SURR_W2, w + SURR_B2, ahi, alo, d, g, t);
        acc_to_operand(d, ahi, alo);
        surr_layer_mma(w + SURR_W3, w + SURR_B3, ahi, alo, d, g, t);
        // output unit: partial dot products over this lane's 16 columns, summed over the group
        float ya = 0.0f, yb = 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float2 w4 = __ldg(reinterpret_cast<const float2*>(w + SURR_W4 + 8 * j + 2 * t));
            ya = fmaf(w4.x, d[j][0], fmaf(w4.y, d[j][1], ya));
            yb = fmaf(w4.x, d[j][2], fmaf(w4.y, d[j][3], yb));
        }
        ya += __shfl_xor_sync(0xffffffffu, ya, 1);
        ya += __shfl_xor_sync(0xffffffffu, ya, 2);
        yb += __shfl_xor_sync(0xffffffffu, yb, 1);
        yb += __shfl_xor_sync(0xffffffffu, yb, 2);
        ysel[mt][0] = ya;                                        // sample 16 mt + g
        ysel[mt][1] = yb;                                        // sample 16 mt + g + 8
    }
    // sample `lane` = 16 mt + 8 h + g' sits in lanes 4 g' .. 4 g' + 3
    const uint32_t src = 4u * (lane & 7u);
    const float y00 = __shfl_sync(0xffffffffu, ysel[0][0], src), y01 = __shfl_sync(0xffffffffu, ysel[0][1], src);
    const float y10 = __shfl_sync(0xffffffffu, ysel[1][0], src), y11 = __shfl_sync(0xffffffffu, ysel[1][1], src);
    const uint32_t mt = lane >> 4, h = (lane >> 3) & 1u;
    const float y = mt ? (h ? y11 : y10) : (h ? y01 : y00);
    return y + __ldg(w + SURR_B4);
}

// K^ of each lane's pair of volumes (or -1: the plain kernel is used, also for inactive lanes);
// every lane of the warp calls it, converged
__device__ __forceinline__ float surr_pair_kernel_warp(const SurrogateDev* __restrict__ Sp, double v1, double v2,
                                                       bool active)
{
    const float c = 0.238732414637843f;   // 3 / (4 pi)
    const SurrogateDev S = *Sp;
    float z0 = 0.0f, z1 = 0.0f;
    bool use = false;
    if (active) {
        const float r1 = cbrtf((float)v1 * c), r2 = cbrtf((float)v2 * c);
        const float R = fmaxf(r1, r2), r = fminf(r1, r2);
        if (r >= S.r_min && R <= S.r_max) {
            z0 = (__logf(R) - S.c0) / S.c1;
            z1 = (__logf(r) - S.c0) / S.c1;
            const int ta = min(SURR_TILES - 1, max(0, (int)((z0 + 1.0f) * (0.5f * SURR_TILES))));
            const int tb = min(SURR_TILES - 1, max(0, (int)((z1 + 1.0f) * (0.5f * SURR_TILES))));
            use = S.mask[ta * SURR_TILES + tb] != 0;
        }
    }
    if (!__any_sync(0xffffffffu, use)) return -1.0f;
    const float y = surr_forward_warp(S.w, use ? z0 : 0.0f, use ? z1 : 0.0f);
    return use ? fmaxf(__expf(fmaf(S.sigma, y, S.mu)) - S.k_floor, 0.0f) : -1.0f;
}

// Device-side evaluation through the step's tensor-core path: K^ (or -1) per pair, one warp per
// 32 pairs.
__global__ void surr_eval_warp_kernel(SurrogateDev S, const double* R, const double* r, uint64_t n, float* K)
{
    __shared__ SurrogateDev Ss;
    if (threadIdx.x == 0) Ss = S;
    __syncthreads();
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x >> 5);
    for (uint64_t base = ((uint64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * 32; base < n; base += 32 * nw) {
        const uint64_t i = base + (threadIdx.x & 31u);
        const bool act = i < n;
        const double Ri = act ? fmax(R[i], r[i]) : 1.0, ri = act ? fmin(R[i], r[i]) : 1.0;
        const double c = 4.0 / 3.0 * 3.14159265358979311600;
        const float k = surr_pair_kernel_warp(&Ss, c * Ri * Ri * Ri, c * ri * ri * ri, act);
        if (act) K[i] = k;
    }
}

// Device-side evaluation for tests: K^ (or -1 where the plain kernel is used) per pair.
__global__ void surr_eval_kernel(SurrogateDev S, const double* R, const double* r, uint64_t n, float* K)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        K[i] = surr_kernel(S, (float)fmax(R[i], r[i]), (float)fmin(R[i], r[i]));
}

}  // namespace sdm
