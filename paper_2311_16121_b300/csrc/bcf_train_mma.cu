// bcf_train_mma.cu -- the training step (Sec. 4.1-4.3, Eq. 5-9) with the MLP
// of Eq. 3 on the tensor cores, for three-layer decoders K0 <= 16 -> 32 -> 32
// -> C <= 16 (the 13-32-32-9 materials); other shapes use k_train.  The
// features are either block parameters through the emulated BC6 mode-10
// decompression, or (FREE) unconstrained per-texel values, the first stage
// of Sec. 5.1.
//
// One warp owns 32 queries.  The per-query work (batch draw, emulated BC6
// taps, reference sample, gradient scatter) runs one query per lane exactly as
// in k_train.  The MLP runs on mma.sync m16n8k16 BF16 with FP32 accumulation:
//  * forward: A = the BF16-rounded inputs / hidden activations, B = the
//    BF16-rounded weights -- the operands the method rounds anyway, so the
//    products are exact and only the FP32 summation order differs;
//  * backward: the FP32 output gradient g enters as two BF16 terms
//    g_hi + g_lo (g_hi = bf16(g), g_lo = bf16(g - g_hi)), so every product
//    carries 16 significant bits of g (relative error <= 2^-17) and the sums
//    stay FP32: dL/dh = (g W) * relu'(h), dW = g^T a, db = column sums of g;
//  * the transposed operands of dW = g^T a come from the forward and backward
//    fragments themselves (movmatrix transposes 8 x 8 BF16 blocks in
//    registers), so no activation is written to shared memory.
// Weight gradients are accumulated per CTA in shared memory and added to the
// global gradients once at the end, as in k_train.
//
// The phases of a tile (features, MLP forward and backward, scatter) are long
// stretches of distinct code, and warps that drift into different phases
// thrash the instruction cache ("no instruction" was the top stall): the
// CTA's eight warps take their tiles together and meet at a barrier before
// the MLP and before the scatter (measured A/B: 1.87 ms per 2^20 step with
// free-running CTAs of 4 warps, 1.60 ms with the two barriers, 1.54 ms with
// CTAs of 8 warps; 16 warps 1.57 ms, a barrier at every phase 1.56 ms).
#include <cuda_bf16.h>
#include <math.h>

#include "bcf_kernels.h"
#include "bcf_train.h"
#include "bcf_train_sample.cuh"

namespace bcf {
namespace {

constexpr int kWarps = 8, kThreads = 32 * kWarps;
constexpr int K0P = 16, N1 = 32, N2 = 32, NOP = 16;
constexpr int S16 = 24, S32 = 40; // row strides (BF16) of [n][k] tiles with K = 16 / 32: 12 / 20 words
constexpr int kRowF = NOP + 1;    // FP32 staging row stride
constexpr int kMaxW = N1 * K0P + N2 * N1 + NOP * N2, kMaxB = N1 + N2 + NOP;
// The coarsest levels (at most 16 x 16 texels: 16 + 4 + 1 blocks) of the first textures collect the gradient
// contributions of most queries on a handful of blocks; they are accumulated in shared memory per CTA
// instead of by contended global atomics, and added to the global gradients once at the end.
constexpr int kCoarseTex = 4, kCoarseBlocks = 21;

typedef __nv_bfloat16 bf16;

struct MmaSmem {
    bf16 W1[N1 * S16], W2[N2 * S32], W3[NOP * S32];    // forward B: [out][in]
    bf16 W1T[K0P * S32], W2T[N1 * S32], W3T[N2 * S16]; // backward B: [in][out]
    float b1[N1], b2[N2], b3[NOP];
    float dW[kMaxW], db[kMaxB];
    bf16 X[kWarps][32 * S16]; // the warp's BF16 input rows
    float R[kWarps][32 * kRowF]; // row <-> fragment staging: outputs, output gradients, input gradients
    float coarse[kCoarseTex][kCoarseBlocks * 32];
};

// First block of the coarse tail (levels of at most 16 x 16 texels) of a texture's block array.
__device__ __forceinline__ int64_t coarse_start(const TrainTexDev &T)
{
    int lg = 0;
    while ((2 << lg) <= T.res)
        ++lg;
    const int lc = max(lg - 4, 0);
    if (lc >= T.levels)
        return T.blocks;
    const uint32_t wb0 = (uint32_t)(T.res >> 2), wbl = (uint32_t)((T.res >> lc) >> 2);
    return (int64_t)((wb0 * wb0 - wbl * wbl) * 4u / 3u);
}

__device__ __forceinline__ uint32_t ld32(const bf16 *p) { return *reinterpret_cast<const uint32_t *>(p); }

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&h);
}

// g = hi + lo with hi = bf16(g), lo = bf16(g - hi), two elements per register.
__device__ __forceinline__ void split_bf16(float x0, float x1, uint32_t &hi, uint32_t &lo)
{
    __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
    const float2 f = __bfloat1622float2(h);
    hi = *reinterpret_cast<uint32_t *>(&h);
    lo = pack_bf16(x0 - f.x, x1 - f.y);
}

// relu'(h) > 0 for element `half` of a packed pair of BF16 post-ReLU values (+0 and -0 give 0)
__device__ __forceinline__ bool positive(uint32_t pair, int half) { return (int16_t)(pair >> (16 * half)) > 0; }

__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t trans8(uint32_t x)
{
    uint32_t y;
    asm("movmatrix.sync.aligned.m8n8.trans.b16 %0, %1;" : "=r"(y) : "r"(x));
    return y;
}

// Fragments of m16n8k16 (row.col): A [m][k] row-major, B from an [n][k] tile, C/D FP32.
template <int S>
__device__ __forceinline__ void frag_a(const bf16 *A, int m0, int g, int t, uint32_t a[4])
{
    const bf16 *p = A + (m0 + g) * S + 2 * t;
    a[0] = ld32(p);
    a[1] = ld32(p + 8 * S);
    a[2] = ld32(p + 8);
    a[3] = ld32(p + 8 * S + 8);
}

template <int S>
__device__ __forceinline__ void frag_b(const bf16 *W, int n0, int k0, int g, int t, uint32_t b[2])
{
    const bf16 *p = W + (n0 + g) * S + k0 + 2 * t;
    b[0] = ld32(p);
    b[1] = ld32(p + 8);
}

// The A fragment of the transposed 16 x 16 block: its 8 x 8 quarters swap across the diagonal and transpose.
__device__ __forceinline__ void trans_a(const uint32_t a[4], uint32_t at[4])
{
    at[0] = trans8(a[0]);
    at[1] = trans8(a[2]);
    at[2] = trans8(a[1]);
    at[3] = trans8(a[3]);
}

// B fragment (k = the 16 rows of an A fragment, n = its columns 8 nh .. 8 nh + 7) of an A-layout block.
__device__ __forceinline__ void a_as_b(const uint32_t a[4], int nh, uint32_t b[2])
{
    b[0] = trans8(a[2 * nh]);
    b[1] = trans8(a[2 * nh + 1]);
}

// C fragments of n-tiles (2 kt, 2 kt + 1) -> the A fragment of k-tile kt, with bias + ReLU + BF16 rounding.
template <int NT>
__device__ __forceinline__ void hidden_a(const float (&c)[2][NT][4], const float *bias, int t, uint32_t (&a)[2][NT / 2][4])
{
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int r = 0; r < NT * 2; ++r) {
            const int kt = r >> 2, reg = r & 3;
            const int nt = 2 * kt + (reg >> 1), ci = (reg & 1) * 2;
            const float b0 = bias[nt * 8 + 2 * t], b1 = bias[nt * 8 + 2 * t + 1];
            a[mt][kt][reg] = pack_bf16(fmaxf(c[mt][nt][ci] + b0, 0.0f), fmaxf(c[mt][nt][ci + 1] + b1, 0.0f));
        }
}

// relu' mask from the forward activations, then the two-term BF16 split as A fragments.
template <int NT>
__device__ __forceinline__ void grad_a(float (&d)[2][NT][4], const uint32_t (&act)[2][NT / 2][4],
                                       uint32_t (&hi)[2][NT / 2][4], uint32_t (&lo)[2][NT / 2][4])
{
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if (!positive(act[mt][nt >> 1][(nt & 1) * 2 + (c >> 1)], c & 1))
                    d[mt][nt][c] = 0.0f;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int r = 0; r < NT * 2; ++r) {
            const int kt = r >> 2, reg = r & 3;
            const int nt = 2 * kt + (reg >> 1), ci = (reg & 1) * 2;
            split_bf16(d[mt][nt][ci], d[mt][nt][ci + 1], hi[mt][kt][reg], lo[mt][kt][reg]);
        }
}

// Column sums of the warp's 32 rows of C fragments, added to db (lanes 0..3 hold the totals).
template <int NT>
__device__ __forceinline__ void add_bias_grad(const float (&d)[2][NT][4], float *db, int lane, int t)
{
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        float s0 = d[0][nt][0] + d[0][nt][2] + d[1][nt][0] + d[1][nt][2];
        float s1 = d[0][nt][1] + d[0][nt][3] + d[1][nt][1] + d[1][nt][3];
#pragma unroll
        for (int off = 4; off < 32; off <<= 1) {
            s0 += __shfl_xor_sync(0xffffffffu, s0, off);
            s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        }
        if (lane < 4) {
            atomicAdd(db + nt * 8 + 2 * t, s0);
            atomicAdd(db + nt * 8 + 2 * t + 1, s1);
        }
    }
}

// dW[m][n] += sum over the warp's rows of g[row][m] a[row][n]: A = g^T (two terms), B = a^T, K = the rows.
// g: A fragments [row tile][m tile], a: A fragments [row tile][n k-tile]; dW row-major with `ld` columns,
// only m < m_lim and n < n_lim stored.
template <int MT, int NT>
__device__ __forceinline__ void weight_grad(const uint32_t (&ghi)[2][MT][4], const uint32_t (&glo)[2][MT][4],
                                            const uint32_t (&act)[2][(NT + 1) / 2][4], float *dW, int ld, int m_lim,
                                            int n_lim, int g, int t)
{
    float w[MT][NT][4];
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c)
                w[mi][nt][c] = 0.0f;
#pragma unroll
    for (int kr = 0; kr < 2; ++kr) {
        uint32_t ah[MT][4], al[MT][4];
#pragma unroll
        for (int mi = 0; mi < MT; ++mi) {
            trans_a(ghi[kr][mi], ah[mi]);
            trans_a(glo[kr][mi], al[mi]);
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            uint32_t b[2];
            a_as_b(act[kr][nt >> 1], nt & 1, b);
#pragma unroll
            for (int mi = 0; mi < MT; ++mi) {
                mma_bf16(w[mi][nt], ah[mi], b);
                mma_bf16(w[mi][nt], al[mi], b);
            }
        }
    }
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int nt = 0; nt < NT; ++nt)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int m = mi * 16 + g + (c >> 1) * 8, n = nt * 8 + 2 * t + (c & 1);
                if (m < m_lim && n < n_lim)
                    atomicAdd(dW + m * ld + n, w[mi][nt][c]);
            }
}

template <bool FREE, int EMU, bool GRID, bool TWO>
__global__ void __launch_bounds__(kThreads, 2) k_train_mma(TrainDev D, int mode, int64_t batch, uint32_t seed_lo,
                                                        uint32_t seed_hi, uint32_t step_lo, uint32_t step_hi,
                                                        const float *__restrict__ qu, const float *__restrict__ qv,
                                                        const float *__restrict__ qs, float *__restrict__ out,
                                                        const float *__restrict__ grad_out, float *loss, float gscale)
{
    __shared__ __align__(16) MmaSmem S;
    // TWO: the paper's two-layer decoder K0 <= 16 -> 16 -> C (Sec. 5.1): its hidden layer takes the first 16
    // rows of the W1 tiles, its output layer the W3 tiles (K = 16 of their 32 columns), its biases b1 and b3
    constexpr int H1 = TWO ? 16 : N1; // first hidden width
    const int K0 = D.dims[0], C = D.dims[TWO ? 2 : 3];
    const int wout = TWO ? 1 : 2;     // layer index of the output layer
    // weights as BF16 operand tiles (zero padded), biases, zeroed gradient accumulators
    for (int e = threadIdx.x; e < N1 * K0P; e += kThreads) {
        const int o = e / K0P, i = e % K0P;
        const bf16 w = __float2bfloat16_rn(i < K0 && o < H1 ? D.W[D.w_off[0] + o * K0 + i] : 0.0f);
        S.W1[o * S16 + i] = w;
        S.W1T[i * S32 + o] = w;
    }
    if constexpr (!TWO)
        for (int e = threadIdx.x; e < N2 * N1; e += kThreads) {
            const int o = e / N1, i = e % N1;
            const bf16 w = __float2bfloat16_rn(D.W[D.w_off[1] + o * N1 + i]);
            S.W2[o * S32 + i] = w;
            S.W2T[i * S32 + o] = w;
        }
    constexpr int KO = TWO ? H1 : N2; // inputs of the output layer
    for (int e = threadIdx.x; e < NOP * N2; e += kThreads) {
        const int o = e / N2, i = e % N2;
        const bf16 w = __float2bfloat16_rn(o < C && i < KO ? D.W[D.w_off[wout] + o * KO + i] : 0.0f);
        S.W3[o * S32 + i] = w;
        if (i < 16 || !TWO)
            S.W3T[i * S16 + o] = w;
    }
    for (int e = threadIdx.x; e < kMaxB; e += kThreads) {
        if (e < N1)
            S.b1[e] = e < H1 ? D.b[D.b_off[0] + e] : 0.0f;
        else if (e < N1 + N2)
            S.b2[e - N1] = TWO ? 0.0f : D.b[D.b_off[1] + e - N1];
        else
            S.b3[e - N1 - N2] = e - N1 - N2 < C ? D.b[D.b_off[wout] + e - N1 - N2] : 0.0f;
        S.db[e] = 0.0f;
    }
    for (int e = threadIdx.x; e < kMaxW; e += kThreads)
        S.dW[e] = 0.0f;
    for (int e = threadIdx.x; e < kCoarseTex * kCoarseBlocks * 32; e += kThreads)
        (&S.coarse[0][0])[e] = 0.0f;
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    bf16 *X = S.X[warp];
    float *R = S.R[warp];
    float loss_acc = 0.0f;
    const int64_t wtiles = (batch + 31) / 32;
    for (int64_t wt0 = (int64_t)blockIdx.x * kWarps; wt0 < wtiles; wt0 += (int64_t)gridDim.x * kWarps) {
        const int64_t wt = wt0 + warp; // every warp of the CTA takes the same iterations (barriers below)
        const int64_t q = wt * 32 + lane;
        const bool active = q < batch;
        float u = 0.0f, v = 0.0f, s = 0.0f;
        if (active) {
            if (qu) {
                u = qu[q];
                v = qv[q];
                s = qs[q];
            } else {
                if (D.batch_grid > 0)
                    draw_query_grid(q, D.batch_grid, seed_lo, seed_hi, step_lo, step_hi, D.s_max, u, v, s);
                else
                    draw_query(q, seed_lo, seed_hi, step_lo, step_hi, D.s_max, u, v, s);
            }
            u = isfinite(u) ? u - floorf(u) : 0.0f;
            v = isfinite(v) ? v - floorf(v) : 0.0f;
        }
        // ---- features (emulated BC6 + trilinear) -> the lane's BF16 input row
        bf16 *xr = X + lane * S16;
        for (int tx = 0; tx < D.n_tex; ++tx) {
            float f[3] = {0.0f, 0.0f, 0.0f};
            if (active && FREE) {
                for_each_side_free<true>(D.tex[tx], u, v, s,
                                         [&](const int64_t(&)[4], const float(&wt)[4], const float4(&val)[4]) {
#pragma unroll
                                             for (int j = 0; j < 4; ++j) {
                                                 f[0] = fmaf(wt[j], val[j].x, f[0]);
                                                 f[1] = fmaf(wt[j], val[j].y, f[1]);
                                                 f[2] = fmaf(wt[j], val[j].z, f[2]);
                                             }
                                         });
            } else if (active) {
                const TrainTexDev &T = D.tex[tx];
                for_each_side(T, u, v, s, [&](const Tap(&tp)[4], const TexelParams(&P)[4]) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        SteTexel tt;
                        ste_from_v<EMU>(P[j], tt);
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            f[c] = fmaf(tp[j].weight, tt.v[c], f[c]);
                    }
                });
            }
#pragma unroll
            for (int c = 0; c < 3; ++c)
                xr[3 * tx + c] = __float2bfloat16_rn(f[c]);
        }
        for (int i = 3 * D.n_tex; i < K0P; ++i)
            xr[i] = __float2bfloat16_rn(i == 3 * D.n_tex && D.lod_input && active ? (isnan(s) ? 0.0f : fmaxf(s, 0.0f))
                                                                                  : 0.0f);
        __syncwarp();
        uint32_t xa[2][1][4];
        frag_a<S16>(X, 0, g, t, xa[0][0]);
        frag_a<S16>(X, 16, g, t, xa[1][0]);

        __syncthreads(); // the CTA's warps enter the MLP together (instruction-cache locality)
        // ---- forward: h1 = relu(x W1^T + b1), h2 = relu(h1 W2^T + b2) (both rounded to BF16), y = h2 W3^T + b3;
        // two layers: h1 (16 wide) = relu(x W1^T + b1), y = h1 W3^T + b3
        uint32_t a1[2][2][4], a2[2][2][4];
        if constexpr (TWO) {
            {
                float c[2][2][4] = {};
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    uint32_t b[2];
                    frag_b<S16>(S.W1, nt * 8, 0, g, t, b);
                    mma_bf16(c[0][nt], xa[0][0], b);
                    mma_bf16(c[1][nt], xa[1][0], b);
                }
                uint32_t h[2][1][4];
                hidden_a<2>(c, S.b1, t, h);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                    for (int r = 0; r < 4; ++r)
                        a1[mt][0][r] = h[mt][0][r];
            }
            float c[2][2][4] = {};
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                uint32_t b[2];
                frag_b<S32>(S.W3, nt * 8, 0, g, t, b);
                mma_bf16(c[0][nt], a1[0][0], b);
                mma_bf16(c[1][nt], a1[1][0], b);
            }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        const int row = mt * 16 + g + (cc >> 1) * 8, col = nt * 8 + 2 * t + (cc & 1);
                        R[row * kRowF + col] = c[mt][nt][cc] + S.b3[col];
                    }
        } else {
        {
            float c[2][4][4] = {};
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                uint32_t b[2];
                frag_b<S16>(S.W1, nt * 8, 0, g, t, b);
                mma_bf16(c[0][nt], xa[0][0], b);
                mma_bf16(c[1][nt], xa[1][0], b);
            }
            hidden_a<4>(c, S.b1, t, a1);
        }
        {
            float c[2][4][4] = {};
#pragma unroll
            for (int kt = 0; kt < 2; ++kt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    uint32_t b[2];
                    frag_b<S32>(S.W2, nt * 8, kt * 16, g, t, b);
                    mma_bf16(c[0][nt], a1[0][kt], b);
                    mma_bf16(c[1][nt], a1[1][kt], b);
                }
            hidden_a<4>(c, S.b2, t, a2);
        }
        {
            float c[2][2][4] = {};
#pragma unroll
            for (int kt = 0; kt < 2; ++kt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    uint32_t b[2];
                    frag_b<S32>(S.W3, nt * 8, kt * 16, g, t, b);
                    mma_bf16(c[0][nt], a2[0][kt], b);
                    mma_bf16(c[1][nt], a2[1][kt], b);
                }
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc) {
                        const int row = mt * 16 + g + (cc >> 1) * 8, col = nt * 8 + 2 * t + (cc & 1);
                        R[row * kRowF + col] = c[mt][nt][cc] + S.b3[col];
                    }
        }
        }
        __syncwarp();
        float *rr = R + lane * kRowF;
        if (mode == kModeForward) {
            if (active)
#pragma unroll
                for (int o = 0; o < NOP; ++o)
                    if (o < C)
                        out[q * C + o] = rr[o];
            __syncwarp();
            continue;
        }
        // ---- output gradient: given, or from the MSE against the reference (Eq. 5, mean over batch x C)
        {
            float gl[NOP];
            if (mode == kModeBackward) {
#pragma unroll
                for (int o = 0; o < NOP; ++o)
                    gl[o] = active && o < C ? grad_out[q * C + o] : 0.0f;
            } else {
                float tg[9];
                if (active)
                    target_sample(D, u, v, s, tg);
#pragma unroll
                for (int o = 0; o < NOP; ++o) {
                    const float d = active && o < C ? rr[o] - tg[o < 9 ? o : 0] : 0.0f;
                    loss_acc = fmaf(d, d, loss_acc);
                    gl[o] = gscale * d;
                }
            }
            __syncwarp();
#pragma unroll
            for (int o = 0; o < NOP; ++o)
                rr[o] = gl[o];
#pragma unroll
            for (int o = 0; o < NOP; ++o) {
                if (o >= C)
                    break;
                float sum = gl[o];
#pragma unroll
                for (int off = 16; off > 0; off >>= 1)
                    sum += __shfl_xor_sync(0xffffffffu, sum, off);
                if (lane == 0)
                    atomicAdd(S.db + N1 + N2 + o, sum);
            }
        }
        __syncwarp();
        uint32_t g3h[2][1][4], g3l[2][1][4];
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
            const float *p = R + (mt * 16 + g) * kRowF + 2 * t;
            split_bf16(p[0], p[1], g3h[mt][0][0], g3l[mt][0][0]);
            split_bf16(p[8 * kRowF], p[8 * kRowF + 1], g3h[mt][0][1], g3l[mt][0][1]);
            split_bf16(p[8], p[9], g3h[mt][0][2], g3l[mt][0][2]);
            split_bf16(p[8 * kRowF + 8], p[8 * kRowF + 9], g3h[mt][0][3], g3l[mt][0][3]);
        }
        if constexpr (TWO) {
            // ---- output layer: dW3 = g3^T h1; dh1 = g3 W3, masked by relu'
            uint32_t h1[2][1][4];
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int r = 0; r < 4; ++r)
                    h1[mt][0][r] = a1[mt][0][r];
            weight_grad<1, 2>(g3h, g3l, h1, S.dW + D.w_off[1], H1, C, H1, g, t);
            uint32_t g1h[2][1][4], g1l[2][1][4];
            {
                float d[2][2][4] = {};
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    uint32_t b[2];
                    frag_b<S16>(S.W3T, nt * 8, 0, g, t, b);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma_bf16(d[mt][nt], g3h[mt][0], b);
                        mma_bf16(d[mt][nt], g3l[mt][0], b);
                    }
                }
                grad_a<2>(d, h1, g1h, g1l);
                add_bias_grad<2>(d, S.db, lane, t);
            }
            // ---- hidden layer: dW1 = g1^T x; dx = g1 W1, staged per row for the scatter
            weight_grad<1, 2>(g1h, g1l, xa, S.dW + D.w_off[0], K0, H1, K0, g, t);
            float d[2][2][4] = {};
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                uint32_t b[2];
                frag_b<S32>(S.W1T, nt * 8, 0, g, t, b);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_bf16(d[mt][nt], g1h[mt][0], b);
                    mma_bf16(d[mt][nt], g1l[mt][0], b);
                }
            }
            __syncwarp();
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc)
                        R[(mt * 16 + g + (cc >> 1) * 8) * kRowF + nt * 8 + 2 * t + (cc & 1)] = d[mt][nt][cc];
        } else {
        // ---- layer 3: dW3 = g3^T h2; dh2 = g3 W3, masked by relu'
        weight_grad<1, 4>(g3h, g3l, a2, S.dW + D.w_off[2], N2, C, N2, g, t);
        uint32_t g2h[2][2][4], g2l[2][2][4];
        {
            float d[2][4][4] = {};
#pragma unroll
            for (int nt = 0; nt < 4; ++nt) {
                uint32_t b[2];
                frag_b<S16>(S.W3T, nt * 8, 0, g, t, b);
#pragma unroll
                for (int mt = 0; mt < 2; ++mt) {
                    mma_bf16(d[mt][nt], g3h[mt][0], b);
                    mma_bf16(d[mt][nt], g3l[mt][0], b);
                }
            }
            grad_a<4>(d, a2, g2h, g2l);
            add_bias_grad<4>(d, S.db + N1, lane, t);
        }
        // ---- layer 2: dW2 = g2^T h1; dh1 = g2 W2, masked by relu'
        weight_grad<2, 4>(g2h, g2l, a1, S.dW + D.w_off[1], N1, N2, N1, g, t);
        uint32_t g1h[2][2][4], g1l[2][2][4];
        {
            float d[2][4][4] = {};
#pragma unroll
            for (int kt = 0; kt < 2; ++kt)
#pragma unroll
                for (int nt = 0; nt < 4; ++nt) {
                    uint32_t b[2];
                    frag_b<S32>(S.W2T, nt * 8, kt * 16, g, t, b);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma_bf16(d[mt][nt], g2h[mt][kt], b);
                        mma_bf16(d[mt][nt], g2l[mt][kt], b);
                    }
                }
            grad_a<4>(d, a1, g1h, g1l);
            add_bias_grad<4>(d, S.db, lane, t);
        }
        // ---- layer 1: dW1 = g1^T x; dx = g1 W1 (no relu on the inputs), staged per row for the scatter
        weight_grad<2, 2>(g1h, g1l, xa, S.dW + D.w_off[0], K0, N1, K0, g, t);
        {
            float d[2][2][4] = {};
#pragma unroll
            for (int kt = 0; kt < 2; ++kt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt) {
                    uint32_t b[2];
                    frag_b<S32>(S.W1T, nt * 8, kt * 16, g, t, b);
#pragma unroll
                    for (int mt = 0; mt < 2; ++mt) {
                        mma_bf16(d[mt][nt], g1h[mt][kt], b);
                        mma_bf16(d[mt][nt], g1l[mt][kt], b);
                    }
                }
            __syncwarp();
#pragma unroll
            for (int mt = 0; mt < 2; ++mt)
#pragma unroll
                for (int nt = 0; nt < 2; ++nt)
#pragma unroll
                    for (int cc = 0; cc < 4; ++cc)
                        R[(mt * 16 + g + (cc >> 1) * 8) * kRowF + nt * 8 + 2 * t + (cc & 1)] = d[mt][nt][cc];
        }
        }
        __syncwarp();
        __syncthreads(); // and the scatter (the forward-only mode leaves the loop above, uniformly)
        // ---- the scatter of the input gradient into the block parameters (straight-through, Eq. 7-9)
        // Grid batches (one scale per step, neighbouring lanes on neighbouring texels): with every lane active,
        // the lanes' paths through the taps are uniform, and lanes that update the same block record and region
        // add their endpoint gradients first (below).
        const bool agg = GRID && __all_sync(0xffffffffu, active); // (a separate kernel: no cost to random batches)
        if (active) {
            for (int tx = 0; tx < D.n_tex; ++tx) {
                const float dxf[3] = {rr[3 * tx], rr[3 * tx + 1], rr[3 * tx + 2]};
                const TrainTexDev &T = D.tex[tx];
                if (FREE) {
                    for_each_side_free<false>(T, u, v, s,
                                              [&](const int64_t(&idx)[4], const float(&wt)[4], const float4(&)[4]) {
#pragma unroll
                                                  for (int j = 0; j < 4; ++j)
                                                      red_add_v4(T.grad + idx[j] * 4, dxf[0] * wt[j], dxf[1] * wt[j],
                                                                 dxf[2] * wt[j], 0.0f);
                                              });
                    continue;
                }
                const int64_t cst = tx < kCoarseTex ? coarse_start(T) : T.blocks;
                for_each_side(T, u, v, s, [&](const Tap(&tps)[4], const TexelParams(&P)[4]) {
                    // per tap: the region's endpoint gradients (6) and the index gradient
                    float g[4][6], gx[4];
                    int reg[4];
                    bool inx[4];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        SteTexel tt;
                        ste_from_v<EMU>(P[j], tt);
                        reg[j] = tt.region;
                        inx[j] = tt.inx;
                        gx[j] = 0.0f;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float dv = dxf[c] * tps[j].weight;
                            g[j][c] = tt.ina[c] ? dv * tt.dea[c] : 0.0f;
                            g[j][3 + c] = tt.inb[c] ? dv * tt.deb[c] : 0.0f;
                            gx[j] = fmaf(dv, tt.dx[c], gx[j]);
                        }
                    }
                    // taps of the footprint in the same block and region share one endpoint update
                    bool own[4] = {true, true, true, true};
#pragma unroll
                    for (int j = 1; j < 4; ++j)
#pragma unroll
                        for (int k = 0; k < j; ++k)
                            if (own[j] && own[k] && tps[k].block == tps[j].block && reg[k] == reg[j]) {
#pragma unroll
                                for (int c = 0; c < 6; ++c)
                                    g[k][c] += g[j][c];
                                own[j] = false;
                            }
                    if (agg) {
                        // a segmented scan over runs of lanes with equal (block, region): the run's last lane
                        // carries the run's sum (lanes that do not own an update have keys of their own)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const long long key = own[j] ? tps[j].block * 2 + reg[j] : -1 - lane;
                            // every lane executes every shuffle (none sits behind a short-circuit operator)
                            const long long kprev = __shfl_up_sync(0xffffffffu, key, 1);
                            const long long knext = __shfl_down_sync(0xffffffffu, key, 1);
                            const bool head = lane == 0 || kprev != key;
                            const unsigned heads = __ballot_sync(0xffffffffu, head);
                            const int start = 31 - __clz(heads & (0xffffffffu >> (31 - lane)));
#pragma unroll
                            for (int off = 1; off < 32; off <<= 1) {
                                float pv[6];
#pragma unroll
                                for (int c = 0; c < 6; ++c)
                                    pv[c] = __shfl_up_sync(0xffffffffu, g[j][c], off);
                                if (lane - off >= start) {
#pragma unroll
                                    for (int c = 0; c < 6; ++c)
                                        g[j][c] += pv[c];
                                }
                            }
                            const bool tail = lane == 31 || knext != key;
                            own[j] = own[j] && tail;
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const Tap &tp = tps[j];
                        // horizontal neighbours in one block with an even first texel: one 8-byte index update
                        const bool pair_lo = (j == 0 || j == 2) && tps[j + (j < 3 ? 1 : 0)].block == tp.block &&
                                             tps[j + (j < 3 ? 1 : 0)].texel == tp.texel + 1 && (tp.texel & 1) == 0;
                        const bool pair_hi = (j == 1 || j == 3) && tps[j - 1].block == tp.block &&
                                             tp.texel == tps[j - 1].texel + 1 && (tps[j - 1].texel & 1) == 0;
                        if (tp.block >= cst) {
                            float *cp = S.coarse[tx] + (tp.block - cst) * 32;
                            if (own[j]) {
#pragma unroll
                                for (int c = 0; c < 6; ++c)
                                    atomicAdd(cp + 8 * reg[j] + c, g[j][c]);
                            }
                            if (inx[j])
                                atomicAdd(cp + 16 + tp.texel, gx[j]);
                        } else {
                            float *gp = T.grad + tp.block * 32;
                            if (own[j]) {
                                red_add_v4(gp + 8 * reg[j], g[j][0], g[j][1], g[j][2], g[j][3]);
                                red_add_v2(gp + 8 * reg[j] + 4, g[j][4], g[j][5]);
                            }
                            if (pair_lo)
                                red_add_v2(gp + 16 + tp.texel, inx[j] ? gx[j] : 0.0f,
                                           inx[j + 1] ? gx[j + 1] : 0.0f);
                            else if (!pair_hi && inx[j])
                                atomicAdd(gp + 16 + tp.texel, gx[j]);
                        }
                    }
                });
            }
        }
        __syncwarp(); // the staging rows are rewritten by the warp's next tile
    }
    // ---- flush the CTA's weight gradients and loss
    if (mode != kModeForward) {
        __syncthreads();
        const int w_total = D.w_total;
        for (int i = threadIdx.x; i < w_total; i += kThreads)
            if (S.dW[i] != 0.0f)
                atomicAdd(D.Wg + i, S.dW[i]);
        // S.db holds b1 at [0, N1), b2 at [N1, N1 + N2), the output bias at [N1 + N2, N1 + N2 + C); two layers:
        // b1 (H1) and the output bias, which the caller stores as b_off 0 and b_off 1
        for (int i = threadIdx.x; i < N1 + N2 + C; i += kThreads) {
            const int dst = !TWO ? i : (i < H1 ? i : (i >= N1 + N2 ? H1 + (i - N1 - N2) : -1));
            if (dst >= 0 && S.db[i] != 0.0f)
                atomicAdd(D.bg + dst, S.db[i]);
        }
        for (int tx = 0; tx < (FREE ? 0 : min(D.n_tex, kCoarseTex)); ++tx) {
            const TrainTexDev &T = D.tex[tx];
            const int64_t cst = coarse_start(T);
            for (int i = threadIdx.x; i < (int)(T.blocks - cst) * 32; i += kThreads)
                if (S.coarse[tx][i] != 0.0f)
                    atomicAdd(T.grad + cst * 32 + i, S.coarse[tx][i]);
        }
    }
    if (mode == kModeStep) {
        for (int off = 16; off > 0; off >>= 1)
            loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
        if (lane == 0 && loss_acc != 0.0f)
            atomicAdd(loss, loss_acc * (gscale * 0.5f));
    }
}

} // namespace

static bool train_mma_two_layer(const TrainDev &D)
{
    return D.n_layers == 2 && D.dims[0] <= K0P && D.dims[1] == 16 && D.dims[2] <= 9 && D.b_off[1] == 16;
}

bool train_mma_supported(const TrainDev &D)
{
    return train_mma_two_layer(D) || (D.n_layers == 3 && D.dims[0] <= K0P && D.dims[1] == N1 && D.dims[2] == N2 &&
                                      D.dims[3] <= NOP && D.dims[3] <= 9 && D.b_off[1] == N1 &&
                                      D.b_off[2] == N1 + N2);
}

cudaError_t launch_train_mma(const TrainDev &D, int mode, int64_t batch, uint64_t seed, int64_t step,
                             const float *u, const float *v, const float *s, float *out, const float *grad_out,
                             float *loss, int sms, cudaStream_t st)
{
    static void (*const kernels[18])(TrainDev, int, int64_t, uint32_t, uint32_t, uint32_t, uint32_t, const float *,
                                     const float *, const float *, float *, const float *, float *, float) = {
        k_train_mma<false, 0, false, false>, k_train_mma<false, 1, false, false>, k_train_mma<false, 2, false, false>,
        k_train_mma<false, 3, false, false>, k_train_mma<true, 0, false, false>,  k_train_mma<false, 0, true, false>,
        k_train_mma<false, 1, true, false>,  k_train_mma<false, 2, true, false>,  k_train_mma<false, 3, true, false>,
        k_train_mma<false, 0, false, true>,  k_train_mma<false, 1, false, true>,  k_train_mma<false, 2, false, true>,
        k_train_mma<false, 3, false, true>,  k_train_mma<true, 0, false, true>,   k_train_mma<false, 0, true, true>,
        k_train_mma<false, 1, true, true>,   k_train_mma<false, 2, true, true>,   k_train_mma<false, 3, true, true>};
    const auto kern = kernels[(train_mma_two_layer(D) ? 9 : 0) +
                              (D.unconstrained ? 4 : (D.batch_grid > 0 ? 5 : 0) + emulation_variant(D))];
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    const int64_t tiles = (batch + kThreads - 1) / kThreads;
    const int64_t grid = min(tiles, (int64_t)sms * max(per_sm, 1));
    const float gscale = 2.0f / ((float)batch * (float)D.dims[D.n_layers]);
    kern<<<(unsigned)grid, kThreads, 0, st>>>(D, mode, batch, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)step,
                                              (uint32_t)((uint64_t)step >> 32), u, v, s, out, grad_out, loss, gscale);
    return cudaGetLastError();
}

} // namespace bcf
