// Proposal network 12 -> 64 -> 64 -> 1 (ReLU) on the tensor cores: BF16
// operands, FP32 accumulation (mma.sync m16n8k16), FP32 master weights, Adam.
//
// Fragment layout of mma.m16n8k16 (g = lane / 4, q = lane % 4):
//   A 16x16 row-major: a0 = A[g][2q..2q+1], a1 = A[g+8][2q..], a2 = A[g][2q+8..], a3 = A[g+8][2q+8..]
//   B 16x8  (k x n):   b0 = B[2q..2q+1][g], b1 = B[2q+8..2q+9][g]
//   C 16x8:            c0,c1 = C[g][2q..2q+1], c2,c3 = C[g+8][2q..2q+1]
// so the C fragments of two adjacent n-tiles are exactly the A fragment of
// the next layer's k-step: hidden activations never leave registers.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/snap.h"
#include "snap_mlp.h"

namespace snap {

namespace {

constexpr int NF = kMlpFeatures;   // 12
constexpr int KP = 16;             // padded input width
constexpr int HD = 64;             // hidden width

// parameter offsets in the packed FP32 vector
constexpr int OW1 = 0, OB1 = OW1 + KP * HD, OW2 = OB1 + HD, OB2 = OW2 + HD * HD, OW3 = OB2 + HD,
              OB3 = OW3 + HD, NPAR = OB3 + 1;
static_assert(NPAR == kMlpParams, "parameter count");

__device__ __forceinline__ uint32_t pack2(float lo, float hi)
{
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

__device__ __forceinline__ void mma16816(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// Shared-memory copy of the weights: W1T[n][k] and W2T[n][k] (so that a B
// fragment's k pair is one 32-bit word), W2 row-major [k][n] for the
// backward product with W2^T, biases and w3 in FP32.
struct SmemW {
    __nv_bfloat16 w1t[HD][KP];
    __nv_bfloat16 w2t[HD][HD];
    __nv_bfloat16 w2[HD][HD];
    float b1[HD], b2[HD], w3[HD];
    float b3;
};

__device__ void load_weights(SmemW &s, const MlpDev &M)
{
    for (int t = threadIdx.x; t < HD * KP; t += blockDim.x) {
        const int n = t / KP, k = t % KP;
        s.w1t[n][k] = __float2bfloat16_rn(M.w[OW1 + k * HD + n]);
    }
    for (int t = threadIdx.x; t < HD * HD; t += blockDim.x) {
        const int a = t / HD, b = t % HD;            // W2[a][b]: a input, b output
        const __nv_bfloat16 v = __float2bfloat16_rn(M.w[OW2 + t]);
        s.w2[a][b] = v;
        s.w2t[b][a] = v;
    }
    for (int t = threadIdx.x; t < HD; t += blockDim.x) {
        s.b1[t] = M.w[OB1 + t];
        s.b2[t] = M.w[OB2 + t];
        s.w3[t] = M.w[OW3 + t];
    }
    if (threadIdx.x == 0) s.b3 = M.w[OB3];
    __syncthreads();
}

__device__ __forceinline__ uint32_t lds32(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ float feat(const float *X, long long rows, long long r, int k)
{
    return (r < rows && k < NF) ? X[r * NF + k] : 0.f;
}

// Forward of one 16-row tile held by a warp.  Outputs the layer-1 and
// layer-2 pre-activations in C layout (z1[8][4], z2[8][4]) and the logits of
// rows g and g+8 (valid on every lane after the quad reduction).
__device__ __forceinline__ void tile_forward(const SmemW &s, const float *X, long long rows, long long r0,
                                             float (&z1)[8][4], float (&z2)[8][4], float &y_lo, float &y_hi)
{
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const long long ra = r0 + g, rb = r0 + g + 8;
    const uint32_t a0 = pack2(feat(X, rows, ra, 2 * q), feat(X, rows, ra, 2 * q + 1));
    const uint32_t a1 = pack2(feat(X, rows, rb, 2 * q), feat(X, rows, rb, 2 * q + 1));
    const uint32_t a2 = pack2(feat(X, rows, ra, 2 * q + 8), feat(X, rows, ra, 2 * q + 9));
    const uint32_t a3 = pack2(feat(X, rows, rb, 2 * q + 8), feat(X, rows, rb, 2 * q + 9));
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
        mma16816(c, a0, a1, a2, a3, lds32(&s.w1t[8 * t + g][2 * q]), lds32(&s.w1t[8 * t + g][2 * q + 8]));
        const float bl = s.b1[8 * t + 2 * q], bh = s.b1[8 * t + 2 * q + 1];
        z1[t][0] = c[0] + bl; z1[t][1] = c[1] + bh; z1[t][2] = c[2] + bl; z1[t][3] = c[3] + bh;
    }
    uint32_t h[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        h[k][0] = pack2(fmaxf(z1[2 * k][0], 0.f), fmaxf(z1[2 * k][1], 0.f));
        h[k][1] = pack2(fmaxf(z1[2 * k][2], 0.f), fmaxf(z1[2 * k][3], 0.f));
        h[k][2] = pack2(fmaxf(z1[2 * k + 1][0], 0.f), fmaxf(z1[2 * k + 1][1], 0.f));
        h[k][3] = pack2(fmaxf(z1[2 * k + 1][2], 0.f), fmaxf(z1[2 * k + 1][3], 0.f));
    }
    float ylo = 0.f, yhi = 0.f;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 4; ++k)
            mma16816(c, h[k][0], h[k][1], h[k][2], h[k][3], lds32(&s.w2t[8 * t + g][16 * k + 2 * q]),
                     lds32(&s.w2t[8 * t + g][16 * k + 2 * q + 8]));
        const int n0 = 8 * t + 2 * q;
        z2[t][0] = c[0] + s.b2[n0]; z2[t][1] = c[1] + s.b2[n0 + 1];
        z2[t][2] = c[2] + s.b2[n0]; z2[t][3] = c[3] + s.b2[n0 + 1];
        ylo += fmaxf(z2[t][0], 0.f) * s.w3[n0] + fmaxf(z2[t][1], 0.f) * s.w3[n0 + 1];
        yhi += fmaxf(z2[t][2], 0.f) * s.w3[n0] + fmaxf(z2[t][3], 0.f) * s.w3[n0 + 1];
    }
    ylo += __shfl_xor_sync(0xFFFFFFFFu, ylo, 1);
    ylo += __shfl_xor_sync(0xFFFFFFFFu, ylo, 2);
    yhi += __shfl_xor_sync(0xFFFFFFFFu, yhi, 1);
    yhi += __shfl_xor_sync(0xFFFFFFFFu, yhi, 2);
    y_lo = ylo + s.b3;
    y_hi = yhi + s.b3;
}

// rows_dev (nullable): the row count is read on the device (rows is then only
// the capacity the grid was sized for); blocks without a tile return before
// staging the weights.
__global__ void __launch_bounds__(128) k_mlp_forward(MlpDev M, const float *X, long long rows, float *y,
                                                     const int32_t *rows_dev)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemW &s = *reinterpret_cast<SmemW *>(smem_raw);
    if (rows_dev) rows = min(rows, (long long)*rows_dev);
    const long long ntile = (rows + 15) / 16;
    if ((long long)blockIdx.x * (blockDim.x >> 5) >= ntile) return;   // uniform over the block
    load_weights(s, M);
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3;
    const long long wid = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long tile = wid; tile < ntile; tile += nw) {
        float z1[8][4], z2[8][4], ylo, yhi;
        tile_forward(s, X, rows, tile * 16, z1, z2, ylo, yhi);
        if (q == 0) {
            if (tile * 16 + g < rows) y[tile * 16 + g] = ylo;
            if (tile * 16 + g + 8 < rows) y[tile * 16 + g + 8] = yhi;
        }
    }
}

// Listwise softmax cross-entropy per event (candidate rows off[e]..off[e+1]).
__global__ void k_mlp_loss(const float *y, const int32_t *off, int32_t row_base, const int32_t *label,
                           long long events, float *dy, double *loss_sum)
{
    const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double l = 0.0;
    if (e < events) {
        const int a = off[e] - row_base, b = off[e + 1] - row_base;
        float m = -3.0e38f;
        for (int r = a; r < b; ++r) m = fmaxf(m, y[r]);
        float z = 0.f;
        for (int r = a; r < b; ++r) z += __expf(y[r] - m);
        const float inv = 1.f / (z * (float)events);
        for (int r = a; r < b; ++r) dy[r] = __expf(y[r] - m) * inv;
        const int lab = a + label[e];
        dy[lab] -= 1.f / (float)events;
        l = -((double)(y[lab] - m) - log((double)z));
    }
    for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
    if ((threadIdx.x & 31) == 0 && l != 0.0) atomicAdd(loss_sum, l);
}

// Backward: each block walks 64-row chunks (four warps x 16 rows).  Per chunk
// the warps recompute their tile's forward pass, form dZ2 = dy w3 [Z2 > 0]
// and dZ1 = (dZ2 W2^T) [Z1 > 0] (tensor cores, register-local fragments), and
// park H1, dZ2, X and dZ1 tiles in shared memory.  Then warp w accumulates the
// weight gradients it owns over the chunk's 64 rows on the tensor cores:
// dW2 rows 16w..16w+15 (all 64 columns) and dW1 columns 16w..16w+15.
struct SmemB {
    __nv_bfloat16 h1[64][HD];     // rows x hidden
    __nv_bfloat16 dz2[64][HD];
    __nv_bfloat16 dz1[64][HD];
    __nv_bfloat16 x[64][KP];
};

__global__ void __launch_bounds__(128) k_mlp_backward(MlpDev M, const float *X, const float *dy_in,
                                                      long long rows)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    SmemW &s = *reinterpret_cast<SmemW *>(smem_raw);
    SmemB &b = *reinterpret_cast<SmemB *>(smem_raw + ((sizeof(SmemW) + 15) & ~size_t(15)));
    load_weights(s, M);
    const int lane = threadIdx.x & 31, g = lane >> 2, q = lane & 3, w = threadIdx.x >> 5;
    float gw2[8][4], gw1[2][4];
#pragma unroll
    for (int t = 0; t < 8; ++t) gw2[t][0] = gw2[t][1] = gw2[t][2] = gw2[t][3] = 0.f;
#pragma unroll
    for (int t = 0; t < 2; ++t) gw1[t][0] = gw1[t][1] = gw1[t][2] = gw1[t][3] = 0.f;
    float gb1[1] = {0.f}, gb2[1] = {0.f};   // bias column 16w + lane (lanes 0..15)
    float gw3[16], gb3 = 0.f;
#pragma unroll
    for (int k = 0; k < 16; ++k) gw3[k] = 0.f;
    const long long nchunk = (rows + 63) / 64;
    for (long long ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
        const long long r0 = ch * 64 + 16 * w;
        float z1[8][4], z2[8][4], ylo, yhi;
        tile_forward(s, X, rows, r0, z1, z2, ylo, yhi);
        const float dlo = (r0 + g < rows) ? dy_in[r0 + g] : 0.f;
        const float dhi = (r0 + g + 8 < rows) ? dy_in[r0 + g + 8] : 0.f;
        // dZ2 in C layout, H2 contributions to dw3/db3, and the tiles to smem
        float dz2[8][4];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int n0 = 8 * t + 2 * q;
            dz2[t][0] = z2[t][0] > 0.f ? dlo * s.w3[n0] : 0.f;
            dz2[t][1] = z2[t][1] > 0.f ? dlo * s.w3[n0 + 1] : 0.f;
            dz2[t][2] = z2[t][2] > 0.f ? dhi * s.w3[n0] : 0.f;
            dz2[t][3] = z2[t][3] > 0.f ? dhi * s.w3[n0 + 1] : 0.f;
            gw3[2 * t] += dlo * fmaxf(z2[t][0], 0.f) + dhi * fmaxf(z2[t][2], 0.f);
            gw3[2 * t + 1] += dlo * fmaxf(z2[t][1], 0.f) + dhi * fmaxf(z2[t][3], 0.f);
            const int rl = 16 * w + g;
            *reinterpret_cast<uint32_t *>(&b.dz2[rl][n0]) = pack2(dz2[t][0], dz2[t][1]);
            *reinterpret_cast<uint32_t *>(&b.dz2[rl + 8][n0]) = pack2(dz2[t][2], dz2[t][3]);
            *reinterpret_cast<uint32_t *>(&b.h1[rl][n0]) = pack2(fmaxf(z1[t][0], 0.f), fmaxf(z1[t][1], 0.f));
            *reinterpret_cast<uint32_t *>(&b.h1[rl + 8][n0]) = pack2(fmaxf(z1[t][2], 0.f), fmaxf(z1[t][3], 0.f));
        }
        if (q == 0) gb3 += dlo + dhi;
        {
            const int rl = 16 * w + g;
            const long long ra = r0 + g, rb = r0 + g + 8;
            *reinterpret_cast<uint32_t *>(&b.x[rl][2 * q]) = pack2(feat(X, rows, ra, 2 * q), feat(X, rows, ra, 2 * q + 1));
            *reinterpret_cast<uint32_t *>(&b.x[rl][2 * q + 8]) = pack2(feat(X, rows, ra, 2 * q + 8), feat(X, rows, ra, 2 * q + 9));
            *reinterpret_cast<uint32_t *>(&b.x[rl + 8][2 * q]) = pack2(feat(X, rows, rb, 2 * q), feat(X, rows, rb, 2 * q + 1));
            *reinterpret_cast<uint32_t *>(&b.x[rl + 8][2 * q + 8]) = pack2(feat(X, rows, rb, 2 * q + 8), feat(X, rows, rb, 2 * q + 9));
        }
        // dH1 = dZ2 W2^T  (A = dZ2 from registers, B[k][n] = W2[n][k])
        uint32_t ad[4][4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            ad[k][0] = pack2(dz2[2 * k][0], dz2[2 * k][1]);
            ad[k][1] = pack2(dz2[2 * k][2], dz2[2 * k][3]);
            ad[k][2] = pack2(dz2[2 * k + 1][0], dz2[2 * k + 1][1]);
            ad[k][3] = pack2(dz2[2 * k + 1][2], dz2[2 * k + 1][3]);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            float c[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                mma16816(c, ad[k][0], ad[k][1], ad[k][2], ad[k][3], lds32(&s.w2[8 * t + g][16 * k + 2 * q]),
                         lds32(&s.w2[8 * t + g][16 * k + 2 * q + 8]));
            const int n0 = 8 * t + 2 * q, rl = 16 * w + g;
            const float d0 = z1[t][0] > 0.f ? c[0] : 0.f, d1 = z1[t][1] > 0.f ? c[1] : 0.f;
            const float d2 = z1[t][2] > 0.f ? c[2] : 0.f, d3 = z1[t][3] > 0.f ? c[3] : 0.f;
            *reinterpret_cast<uint32_t *>(&b.dz1[rl][n0]) = pack2(d0, d1);
            *reinterpret_cast<uint32_t *>(&b.dz1[rl + 8][n0]) = pack2(d2, d3);
        }
        __syncthreads();
        // dW2[16w + m][n] += sum_r H1[r][16w + m] dZ2[r][n]   (A = H1^T, B = dZ2, K = 64 rows)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int rr = 16 * k + 2 * q;
            const int m = 16 * w + g;
            const uint32_t a0 = pack2(__bfloat162float(b.h1[rr][m]), __bfloat162float(b.h1[rr + 1][m]));
            const uint32_t a1 = pack2(__bfloat162float(b.h1[rr][m + 8]), __bfloat162float(b.h1[rr + 1][m + 8]));
            const uint32_t a2 = pack2(__bfloat162float(b.h1[rr + 8][m]), __bfloat162float(b.h1[rr + 9][m]));
            const uint32_t a3 = pack2(__bfloat162float(b.h1[rr + 8][m + 8]), __bfloat162float(b.h1[rr + 9][m + 8]));
#pragma unroll
            for (int t = 0; t < 8; ++t) {
                const int n = 8 * t + g;
                const uint32_t b0 = pack2(__bfloat162float(b.dz2[rr][n]), __bfloat162float(b.dz2[rr + 1][n]));
                const uint32_t b1 = pack2(__bfloat162float(b.dz2[rr + 8][n]), __bfloat162float(b.dz2[rr + 9][n]));
                mma16816(gw2[t], a0, a1, a2, a3, b0, b1);
            }
        }
        // dW1[m][16w + n] += sum_r X[r][m] dZ1[r][16w + n]   (A = X^T, m < 16)
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int rr = 16 * k + 2 * q;
            const uint32_t a0 = pack2(__bfloat162float(b.x[rr][g]), __bfloat162float(b.x[rr + 1][g]));
            const uint32_t a1 = pack2(__bfloat162float(b.x[rr][g + 8]), __bfloat162float(b.x[rr + 1][g + 8]));
            const uint32_t a2 = pack2(__bfloat162float(b.x[rr + 8][g]), __bfloat162float(b.x[rr + 9][g]));
            const uint32_t a3 = pack2(__bfloat162float(b.x[rr + 8][g + 8]), __bfloat162float(b.x[rr + 9][g + 8]));
#pragma unroll
            for (int t = 0; t < 2; ++t) {
                const int n = 16 * w + 8 * t + g;
                const uint32_t b0 = pack2(__bfloat162float(b.dz1[rr][n]), __bfloat162float(b.dz1[rr + 1][n]));
                const uint32_t b1 = pack2(__bfloat162float(b.dz1[rr + 8][n]), __bfloat162float(b.dz1[rr + 9][n]));
                mma16816(gw1[t], a0, a1, a2, a3, b0, b1);
            }
        }
        // bias gradients: lanes 0..15 of warp w own hidden column 16w + lane
        if (lane < 16) {
            const int n = 16 * w + lane;
            float s1 = 0.f, s2 = 0.f;
            for (int r = 0; r < 64; ++r) {
                s1 += __bfloat162float(b.dz1[r][n]);
                s2 += __bfloat162float(b.dz2[r][n]);
            }
            gb1[0] += s1;
            gb2[0] += s2;
        }
        __syncthreads();
    }
    // flush this block's partial gradients
    float *G = M.grad;
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int m = 16 * w + g, n = 8 * t + 2 * q;
        atomicAdd(&G[OW2 + m * HD + n], gw2[t][0]);
        atomicAdd(&G[OW2 + m * HD + n + 1], gw2[t][1]);
        atomicAdd(&G[OW2 + (m + 8) * HD + n], gw2[t][2]);
        atomicAdd(&G[OW2 + (m + 8) * HD + n + 1], gw2[t][3]);
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int n = 16 * w + 8 * t + 2 * q;
        if (g < NF) {
            atomicAdd(&G[OW1 + g * HD + n], gw1[t][0]);
            atomicAdd(&G[OW1 + g * HD + n + 1], gw1[t][1]);
        }
        if (g + 8 < NF) {
            atomicAdd(&G[OW1 + (g + 8) * HD + n], gw1[t][2]);
            atomicAdd(&G[OW1 + (g + 8) * HD + n + 1], gw1[t][3]);
        }
    }
    if (lane < 16) {
        atomicAdd(&G[OB1 + 16 * w + lane], gb1[0]);
        atomicAdd(&G[OB2 + 16 * w + lane], gb2[0]);
    }
    // w3 / b3: lane (g, q) holds columns 8t + 2q + {0,1} summed over its rows; reduce over g
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        float v = gw3[k];
        v += __shfl_xor_sync(0xFFFFFFFFu, v, 4);
        v += __shfl_xor_sync(0xFFFFFFFFu, v, 8);
        v += __shfl_xor_sync(0xFFFFFFFFu, v, 16);
        if (g == 0) atomicAdd(&G[OW3 + 8 * (k / 2) + 2 * q + (k & 1)], v);
    }
    {
        float v = gb3;
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
        if (lane == 0) atomicAdd(&G[OB3], v);
    }
}

__global__ void k_mlp_adam(MlpDev M, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= NPAR) return;
    if (k >= OW1 + NF * HD && k < OB1) {   // padded input rows stay zero
        M.w[k] = 0.f;
        M.grad[k] = 0.f;
        return;
    }
    const float gk = M.grad[k];
    const float m = b1 * M.m[k] + (1.f - b1) * gk;
    const float v = b2 * M.v[k] + (1.f - b2) * gk * gk;
    M.m[k] = m;
    M.v[k] = v;
    M.w[k] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    M.grad[k] = 0.f;
}

}  // namespace

size_t mlp_forward_smem() { return sizeof(SmemW); }
size_t mlp_backward_smem() { return ((sizeof(SmemW) + 15) & ~size_t(15)) + sizeof(SmemB); }

cudaError_t mlp_forward(const MlpDev &M, const float *X, long long rows, float *y, cudaStream_t s)
{
    if (rows <= 0) return cudaSuccess;
    const long long tiles = (rows + 15) / 16;
    int blocks = (int)std::min<long long>((tiles + 3) / 4, 148 * 8);
    k_mlp_forward<<<blocks, 128, mlp_forward_smem(), s>>>(M, X, rows, y, nullptr);
    return cudaGetLastError();
}

cudaError_t mlp_forward_counted(const MlpDev &M, const float *X, const int32_t *rows_dev, long long max_rows,
                                float *y, cudaStream_t s)
{
    if (max_rows <= 0) return cudaSuccess;
    const long long tiles = (max_rows + 15) / 16;
    int blocks = (int)std::min<long long>((tiles + 3) / 4, 148 * 8);
    k_mlp_forward<<<blocks, 128, mlp_forward_smem(), s>>>(M, X, max_rows, y, rows_dev);
    return cudaGetLastError();
}

cudaError_t mlp_loss_grad(const MlpDev &M, const float *X, long long rows, const int32_t *off, int32_t row_base,
                          const int32_t *label, long long events, float *y, float *dy, double *loss_sum,
                          cudaStream_t s)
{
    cudaError_t e = mlp_forward(M, X, rows, y, s);
    if (e != cudaSuccess) return e;
    if (events > 0)
        k_mlp_loss<<<(unsigned)((events + 255) / 256), 256, 0, s>>>(y, off, row_base, label, events, dy, loss_sum);
    const long long chunks = (rows + 63) / 64;
    const int blocks = (int)std::min<long long>(chunks, 148 * 4);
    if (blocks > 0) k_mlp_backward<<<blocks, 128, mlp_backward_smem(), s>>>(M, X, dy, rows);
    return cudaGetLastError();
}

cudaError_t mlp_adam(const MlpDev &M, float lr, int t, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.f - std::pow(b1, (float)t), c2 = 1.f - std::pow(b2, (float)t);
    k_mlp_adam<<<(NPAR + 255) / 256, 256, 0, s>>>(M, lr, b1, b2, 1e-8f, c1, c2);
    return cudaGetLastError();
}

cudaError_t mlp_configure()
{
    cudaError_t e = cudaFuncSetAttribute(k_mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mlp_forward_smem());
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_mlp_backward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)mlp_backward_smem());
}

}  // namespace snap
