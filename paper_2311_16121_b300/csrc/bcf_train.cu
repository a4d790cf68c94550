// bcf_train.cu -- training of a block-compressed neural material through the
// emulated BC6 decompression (Sec. 4.1-4.3, Eq. 5-9) and its optimiser.
//
// k_train: one persistent kernel for forward / backward / full step.  Per
// query (one thread): Philox batch draw or given (u, v, s); trilinear taps
// (Eq. 10, Eq. 11 bias) over the block parameters with the straight-through
// mode-10 emulation; MLP forward with BF16-rounded weights and inputs (FP32
// accumulation); Catmull-Rom reference F(M); MSE; FP32 backward through the
// MLP; tap gradients scattered with vector atomics.  MLP weight gradients are
// reduced per CTA: the tile's layer inputs and output gradients are staged in
// shared memory and contracted over the tile's queries, accumulated in
// shared memory across the CTA's tiles, and added to the global gradients
// once at the end.
// k_adam: Adam with exponentially decayed learning rate, box projection of
// the block parameters, and zeroing of the gradients.
// k_export: trained blocks -> BC6H mode-10 bitstreams, weights -> FP16.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include "bc6h_pack.cuh"
#include "bc6h_unpack.cuh"
#include "bcf_kernels.h"
#include "bcf_train.h"
#include "bcf_train_sample.cuh"

namespace bcf {

// ------------------------------------------------------------ the kernel

constexpr int kTrainThreads = 128;

struct TrainSmem {
    float *Wbf, *bias, *dW, *db;
    float *act[BCF_MAX_LAYERS];  // layer inputs A[l] [threads][stride]
    float *grd[BCF_MAX_LAYERS];  // dL/d(output of layer l) [threads][stride]
    int stride[BCF_MAX_LAYERS + 1];
};

__host__ __device__ inline int64_t train_smem_floats(const TrainDev &D)
{
    int64_t f = 2 * (int64_t)(D.w_total + D.b_total);
    for (int l = 0; l <= D.n_layers; ++l) {
        const int st = D.dims[l] | 1; // odd row stride: conflict-free column access
        if (l < D.n_layers)
            f += (int64_t)kTrainThreads * st; // act[l]
        if (l > 0)
            f += (int64_t)kTrainThreads * st; // grd[l-1]
    }
    return f;
}

// EMU: the emulation variant of the block features (compile-time: one variant's code per kernel keeps the
// instruction footprint small; with the variant chosen at run time "no instruction" was the second stall)
template <int EMU>
__global__ void __launch_bounds__(kTrainThreads) k_train(TrainDev D, int mode, int64_t batch, uint32_t seed_lo,
                                                         uint32_t seed_hi, uint32_t step_lo, uint32_t step_hi,
                                                         const float *__restrict__ qu, const float *__restrict__ qv,
                                                         const float *__restrict__ qs, float *__restrict__ out,
                                                         const float *__restrict__ grad_out, float *loss,
                                                         float gscale)
{
    extern __shared__ __align__(16) float tsm[];
    const int L = D.n_layers;
    TrainSmem S;
    {
        float *p = tsm;
        S.Wbf = p;
        p += D.w_total;
        S.bias = p;
        p += D.b_total;
        S.dW = p;
        p += D.w_total;
        S.db = p;
        p += D.b_total;
        for (int l = 0; l <= L; ++l)
            S.stride[l] = D.dims[l] | 1;
        for (int l = 0; l < L; ++l) {
            S.act[l] = p;
            p += kTrainThreads * S.stride[l];
        }
        for (int l = 0; l < L; ++l) {
            S.grd[l] = p;
            p += kTrainThreads * S.stride[l + 1];
        }
    }
    for (int i = threadIdx.x; i < D.w_total; i += blockDim.x) {
        S.Wbf[i] = bf16r(D.W[i]);
        S.dW[i] = 0.0f;
    }
    for (int i = threadIdx.x; i < D.b_total; i += blockDim.x) {
        S.bias[i] = D.b[i];
        S.db[i] = 0.0f;
    }
    __syncthreads();
    const int tid = threadIdx.x;
    const int nout = D.dims[L];
    float loss_acc = 0.0f;
    const int64_t tiles = (batch + kTrainThreads - 1) / kTrainThreads;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t q = tile * kTrainThreads + tid;
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
        // ---- features (emulated BC6 + trilinear), rounded MLP input row
        float *a0 = S.act[0] + tid * S.stride[0];
        for (int t = 0; t < D.n_tex; ++t) {
            float f[3] = {0.0f, 0.0f, 0.0f};
            if (active) {
                const TrainTexDev &T = D.tex[t];
                for_each_side(T, u, v, s, [&](const Tap(&tps)[4], const TexelParams(&P)[4]) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        SteTexel tx;
                        ste_from_v<EMU>(P[j], tx);
#pragma unroll
                        for (int c = 0; c < 3; ++c)
                            f[c] = fmaf(tps[j].weight, tx.v[c], f[c]);
                    }
                });
            }
            a0[3 * t] = bf16r(f[0]);
            a0[3 * t + 1] = bf16r(f[1]);
            a0[3 * t + 2] = bf16r(f[2]);
        }
        if (D.lod_input)
            a0[3 * D.n_tex] = bf16r(active ? (isnan(s) ? 0.0f : fmaxf(s, 0.0f)) : 0.0f);
        // ---- MLP forward (hidden: ReLU then BF16 rounding; output: FP32)
        float y[64];
        for (int l = 0; l < L; ++l) {
            const int ni = D.dims[l], no = D.dims[l + 1];
            const float *W = S.Wbf + D.w_off[l];
            const float *b = S.bias + D.b_off[l];
            const float *xin = S.act[l] + tid * S.stride[l];
            float *xout = l + 1 < L ? S.act[l + 1] + tid * S.stride[l + 1] : nullptr;
            for (int o = 0; o < no; ++o) {
                float acc = 0.0f;
                for (int i = 0; i < ni; ++i)
                    acc = fmaf(W[o * ni + i], xin[i], acc);
                acc += b[o];
                if (xout)
                    xout[o] = bf16r(fmaxf(acc, 0.0f));
                else
                    y[o] = acc;
            }
        }
        if (mode == kModeForward) {
            if (active)
                for (int o = 0; o < nout; ++o)
                    out[q * nout + o] = y[o];
            continue;
        }
        // ---- output gradient: given, or from the MSE against the reference (Eq. 5, mean over batch x C)
        float *gL = S.grd[L - 1] + tid * S.stride[L];
        if (mode == kModeBackward) {
            for (int o = 0; o < nout; ++o)
                gL[o] = active ? grad_out[q * nout + o] : 0.0f;
        } else {
            float tg[9];
            if (active)
                target_sample(D, u, v, s, tg);
            for (int o = 0; o < nout; ++o) {
                const float d = active ? y[o] - tg[o] : 0.0f;
                loss_acc = fmaf(d, d, loss_acc);
                gL[o] = gscale * d;
            }
        }
        // ---- MLP backward: grd[l-1] = (act[l] > 0) * W_l^T grd[l]
        for (int l = L - 1; l >= 1; --l) {
            const int ni = D.dims[l], no = D.dims[l + 1];
            const float *W = S.Wbf + D.w_off[l];
            const float *g = S.grd[l] + tid * S.stride[l + 1];
            const float *a = S.act[l] + tid * S.stride[l];
            float *gp = S.grd[l - 1] + tid * S.stride[l];
            for (int i = 0; i < ni; ++i) {
                float acc = 0.0f;
                if (a[i] > 0.0f)
                    for (int o = 0; o < no; ++o)
                        acc = fmaf(W[o * ni + i], g[o], acc);
                gp[i] = acc;
            }
        }
        __syncthreads();
        // ---- weight gradients of the tile: dW_l += sum_q grd[l][q] (x) act[l][q], db_l += sum_q grd[l][q]
        for (int l = 0; l < L; ++l) {
            const int ni = D.dims[l], no = D.dims[l + 1];
            const int sa = S.stride[l], sg = S.stride[l + 1];
            for (int e = tid; e < no * (ni + 1); e += kTrainThreads) {
                const int o = e / (ni + 1), i = e - o * (ni + 1);
                float acc = 0.0f;
                const float *g = S.grd[l] + o;
                if (i < ni) {
                    const float *a = S.act[l] + i;
                    for (int r = 0; r < kTrainThreads; ++r)
                        acc = fmaf(g[r * sg], a[r * sa], acc);
                    S.dW[D.w_off[l] + o * ni + i] += acc;
                } else {
                    for (int r = 0; r < kTrainThreads; ++r)
                        acc += g[r * sg];
                    S.db[D.b_off[l] + o] += acc;
                }
            }
        }
        // ---- input gradient and the scatter into the block parameters
        if (active) {
            const float *g1 = S.grd[0] + tid * S.stride[1];
            const float *W0 = S.Wbf + D.w_off[0];
            const int n1 = D.dims[1], n0 = D.dims[0];
            for (int t = 0; t < D.n_tex; ++t) {
                float dxf[3];
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    float acc = 0.0f;
                    for (int o = 0; o < n1; ++o)
                        acc = fmaf(W0[o * n0 + 3 * t + c], g1[o], acc);
                    dxf[c] = acc;
                }
                const TrainTexDev &T = D.tex[t];
                for_each_side(T, u, v, s, [&](const Tap(&tps)[4], const TexelParams(&P)[4]) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const Tap &tp = tps[j];
                        SteTexel tx;
                        ste_from_v<EMU>(P[j], tx);
                        float *gp = T.grad + tp.block * 32;
                        float ga[3], gb[3], gx = 0.0f;
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            const float dv = dxf[c] * tp.weight;
                            ga[c] = tx.ina[c] ? dv * tx.dea[c] : 0.0f;
                            gb[c] = tx.inb[c] ? dv * tx.deb[c] : 0.0f;
                            gx = fmaf(dv, tx.dx[c], gx);
                        }
                        red_add_v4(gp + 8 * tx.region, ga[0], ga[1], ga[2], gb[0]);
                        red_add_v2(gp + 8 * tx.region + 4, gb[1], gb[2]);
                        if (tx.inx)
                            atomicAdd(gp + 16 + tp.texel, gx);
                    }
                });
            }
        }
        __syncthreads(); // the staged rows are rewritten by the next tile
    }
    // ---- flush the CTA's weight gradients and loss
    if (mode != kModeForward) {
        __syncthreads();
        for (int i = threadIdx.x; i < D.w_total; i += blockDim.x)
            if (S.dW[i] != 0.0f)
                atomicAdd(D.Wg + i, S.dW[i]);
        for (int i = threadIdx.x; i < D.b_total; i += blockDim.x)
            if (S.db[i] != 0.0f)
                atomicAdd(D.bg + i, S.db[i]);
    }
    if (mode == kModeStep) {
        for (int off = 16; off > 0; off >>= 1)
            loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, off);
        if ((threadIdx.x & 31) == 0 && loss_acc != 0.0f)
            atomicAdd(loss, loss_acc * (gscale * 0.5f));
    }
}

// ------------------------------------------------------------------ Adam

struct AdamSeg {
    float *p, *g, *m, *v;
    int64_t n;
    float lr;
    int blocks_layout; // 1: block parameters (clamp endpoints to [elo, ehi], x to [0, 1], skip unused)
    float elo, ehi;
    const uint8_t *part; // block parameters: the partition ids, checked for ids above 31
    unsigned *check;
};

struct AdamArgs {
    AdamSeg seg[BCF_MAX_TEX + 2];
    int64_t chunk_start[BCF_MAX_TEX + 3];
    int nseg;
    float beta1, beta2, eps, bc1, bc2;
};

constexpr int kAdamChunk = 1024;  // elements per CTA: 256 threads x 1 float4 (more CTAs in flight; 4096: 1% slower step)
constexpr int kAdamVec = kAdamChunk / (256 * 4);

__device__ __forceinline__ float adam_one(const AdamArgs &A, float lr, float &p, float g, float &m, float &v)
{
    m = A.beta1 * m + (1.0f - A.beta1) * g;
    v = A.beta2 * v + (1.0f - A.beta2) * g * g;
    p = p - lr * (m / A.bc1) / (sqrtf(v / A.bc2) + A.eps);
    return p;
}

// Block-parameter records: element e of a 32-float record is an endpoint channel (e < 16, box [0, 63]) or an
// index coordinate (e >= 16, box [0, 1]); elements 6, 7, 14, 15 are padding and are left untouched.
__device__ __forceinline__ bool record_pad(int e) { return e == 6 || e == 7 || e == 14 || e == 15; }
__device__ __forceinline__ float record_clamp(int e, float p, float elo, float ehi)
{
    return e < 16 ? fminf(fmaxf(p, elo), ehi) : fminf(fmaxf(p, 0.0f), 1.0f);
}

// One Adam step over the segments (feature records of every texture, MLP weights, MLP biases), with the
// learning rate lr_0 gamma^step and the gradients zeroed for the next step.  Each CTA streams a 4096-element
// chunk of one segment with 16-byte accesses, all four of a thread's groups loaded before any is written so
// that 16 loads per thread are in flight; ragged or unaligned segments take the scalar path.
__global__ void __launch_bounds__(256) k_adam(AdamArgs A)
{
    int k = 0;
    while (k + 1 < A.nseg && (int64_t)blockIdx.x >= A.chunk_start[k + 1])
        ++k;
    const AdamSeg &S = A.seg[k];
    const int64_t i0 = ((int64_t)blockIdx.x - A.chunk_start[k]) * kAdamChunk;
    const int64_t i1 = min(i0 + kAdamChunk, S.n);
    if (S.part && threadIdx.x < kAdamChunk / 32) { // the chunk's block records: their partition ids
        const int64_t r = i0 / 32 + threadIdx.x;
        if (r < S.n / 32 && S.part[r] > 31 && S.check)
            atomicOr(S.check, BCF_CHECK_PARTITION);
    }
    const bool aligned = ((reinterpret_cast<uintptr_t>(S.p) | reinterpret_cast<uintptr_t>(S.g) |
                           reinterpret_cast<uintptr_t>(S.m) | reinterpret_cast<uintptr_t>(S.v)) & 15) == 0;
    if (aligned && i1 - i0 == kAdamChunk) {
        float4 *__restrict__ P = reinterpret_cast<float4 *>(S.p + i0);
        float4 *__restrict__ G = reinterpret_cast<float4 *>(S.g + i0);
        float4 *__restrict__ M = reinterpret_cast<float4 *>(S.m + i0);
        float4 *__restrict__ V = reinterpret_cast<float4 *>(S.v + i0);
        float4 p[kAdamVec], g[kAdamVec], m[kAdamVec], v[kAdamVec];
#pragma unroll
        for (int j = 0; j < kAdamVec; ++j) {
            const int x = threadIdx.x + 256 * j;
            g[j] = G[x];
            m[j] = __ldcs(M + x);
            v[j] = __ldcs(V + x);
            p[j] = P[x];
        }
#pragma unroll
        for (int j = 0; j < kAdamVec; ++j) {
            const int x = threadIdx.x + 256 * j;
            float *pp = &p[j].x, *gg = &g[j].x, *mm = &m[j].x, *vv = &v[j].x;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int e = (4 * x + c) & 31;
                if (S.blocks_layout && record_pad(e))
                    continue;
                float pn = pp[c], mn = mm[c], vn = vv[c];
                adam_one(A, S.lr, pn, gg[c], mn, vn);
                pp[c] = S.blocks_layout ? record_clamp(e, pn, S.elo, S.ehi) : pn;
                mm[c] = mn;
                vv[c] = vn;
            }
            G[x] = make_float4(0.0f, 0.0f, 0.0f, 0.0f); // parameters and gradients stay in L2 for the next
            P[x] = p[j];                               // step; the moments stream
            __stcs(M + x, m[j]);
            __stcs(V + x, v[j]);
        }
        return;
    }
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const float g = S.g[i];
        S.g[i] = 0.0f;
        const int e = (int)(i & 31);
        if (S.blocks_layout && record_pad(e))
            continue;
        float p = S.p[i], m = S.m[i], v = S.v[i];
        adam_one(A, S.lr, p, g, m, v);
        S.m[i] = m;
        S.v[i] = v;
        S.p[i] = S.blocks_layout ? record_clamp(e, p, S.elo, S.ehi) : p;
    }
}

// ---------------------------------------------------------------- export

__global__ void k_export_blocks(const float *__restrict__ params, const uint8_t *__restrict__ part, int64_t nblocks,
                                int is_signed, unsigned *__restrict__ check, uint4 *__restrict__ out)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nblocks)
        return;
    const float *p = params + b * 32;
    int k = part[b];
    if (k > 31) { // the same reading as training: id & 31
        if (check)
            atomicOr(check, BCF_CHECK_PARTITION);
        k &= 31;
    }
    int q[4][3], idx[16];
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            q[e][c] = (int)rintf(fminf(fmaxf(p[(e >> 1) * 8 + (e & 1) * 3 + c], is_signed ? -32.0f : 0.0f),
                                       is_signed ? 31.0f : 63.0f)); // SF16: the low 6 bits hold the two's complement
#pragma unroll
    for (int t = 0; t < 16; ++t)
        idx[t] = (int)rintf(7.0f * fminf(fmaxf(p[16 + t], 0.0f), 1.0f));
    out[b] = bc6h_pack_mode10(q, idx, k);
}

__global__ void k_export_weights(const float *__restrict__ W, int64_t n, uint16_t *__restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n)
        out[i] = __half_as_ushort(__float2half_rn(W[i]));
}

// -------------------------------------------------------------- launchers

static int train_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0)
            sms = 148;
    }
    return sms;
}

int64_t train_smem_bytes(const TrainDev &D) { return train_smem_floats(D) * 4; }

cudaError_t launch_train(const TrainDev &D, int mode, int64_t batch, uint64_t seed, int64_t step, const float *u,
                         const float *v, const float *s, float *out, const float *grad_out, float *loss,
                         cudaStream_t st)
{
    if (batch <= 0)
        return cudaSuccess;
    if (train_mma_supported(D))
        return launch_train_mma(D, mode, batch, seed, step, u, v, s, out, grad_out, loss, train_sms(), st);
    const int64_t smem = train_smem_bytes(D);
    static void (*const kernels[4])(TrainDev, int, int64_t, uint32_t, uint32_t, uint32_t, uint32_t, const float *,
                                    const float *, const float *, float *, const float *, float *, float) = {
        k_train<0>, k_train<1>, k_train<2>, k_train<3>};
    const int emu = emulation_variant(D);
    const auto kern = kernels[emu];
    static int configured[4] = {0, 0, 0, 0};
    if (!configured[emu]) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        configured[emu] = 1;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTrainThreads, (size_t)smem);
    const int64_t tiles = (batch + kTrainThreads - 1) / kTrainThreads;
    const int64_t grid = min(tiles, (int64_t)train_sms() * max(per_sm, 1));
    const float gscale = 2.0f / ((float)batch * (float)D.dims[D.n_layers]);
    kern<<<(unsigned)grid, kTrainThreads, (size_t)smem, st>>>(
        D, mode, batch, (uint32_t)seed, (uint32_t)(seed >> 32), (uint32_t)step, (uint32_t)((uint64_t)step >> 32), u, v,
        s, out, grad_out, loss, gscale);
    return cudaGetLastError();
}

cudaError_t launch_adam(const TrainDev &D, const TrainHyper &H, int64_t step, cudaStream_t st)
{
    AdamArgs A;
    memset(&A, 0, sizeof A);
    const double decay = pow((double)H.gamma, (double)step);
    int k = 0;
    for (int t = 0; t < D.n_tex; ++t) {
        A.seg[k] = {D.tex[t].params, D.tex[t].grad, D.tex[t].m, D.tex[t].v, feature_floats(D, t),
                    (float)(H.lr_features * decay), D.unconstrained ? 0 : 1, D.is_signed ? -32.0f : 0.0f,
                    D.is_signed ? 31.0f : 63.0f, D.unconstrained ? nullptr : D.tex[t].part, D.tex[t].check};
        ++k;
    }
    A.seg[k++] = {D.W, D.Wg, D.Wm, D.Wv, D.w_total, (float)(H.lr_mlp * decay), 0, 0.0f, 0.0f, nullptr, nullptr};
    A.seg[k++] = {D.b, D.bg, D.bm, D.bv, D.b_total, (float)(H.lr_mlp * decay), 0, 0.0f, 0.0f, nullptr, nullptr};
    A.nseg = k;
    int64_t chunks = 0;
    for (int i = 0; i < k; ++i) {
        A.chunk_start[i] = chunks;
        chunks += (A.seg[i].n + kAdamChunk - 1) / kAdamChunk;
    }
    A.chunk_start[k] = chunks;
    A.beta1 = H.beta1;
    A.beta2 = H.beta2;
    A.eps = H.eps;
    A.bc1 = (float)(1.0 - pow((double)H.beta1, (double)(step + 1)));
    A.bc2 = (float)(1.0 - pow((double)H.beta2, (double)(step + 1)));
    if (chunks == 0)
        return cudaSuccess;
    k_adam<<<(unsigned)chunks, 256, 0, st>>>(A);
    return cudaGetLastError();
}

cudaError_t launch_export_blocks(const float *params, const uint8_t *part, int64_t nblocks, int is_signed,
                                 unsigned *check, void *out, cudaStream_t st)
{
    if (nblocks > 0)
        k_export_blocks<<<(unsigned)((nblocks + 127) / 128), 128, 0, st>>>(params, part, nblocks, is_signed, check,
                                                                           (uint4 *)out);
    return cudaGetLastError();
}

cudaError_t launch_export(const TrainDev &D, void *const *blocks_out, uint16_t *weights_fp16, cudaStream_t st)
{
    for (int t = 0; t < D.n_tex; ++t) {
        const cudaError_t e = launch_export_blocks(D.tex[t].params, D.tex[t].part, D.tex[t].blocks, D.is_signed,
                                                   D.tex[t].check, blocks_out[t], st);
        if (e != cudaSuccess)
            return e;
    }
    if (weights_fp16)
        k_export_weights<<<(unsigned)((D.w_total + 255) / 256), 256, 0, st>>>(D.W, D.w_total, weights_fp16);
    return cudaGetLastError();
}

} // namespace bcf
