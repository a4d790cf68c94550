// bcf_mlp.cuh -- the MLP decoder f_eta of Eq. 3 (ReLU hidden layers, linear
// output) for the fused decode kernels.
//
// Low precision: one warp evaluates 32 queries as a [32 x K] activation tile
// on the tensor cores (mma.sync m16n8k16 for FP16 / BF16, m16n8k32 for
// OCP E4M3), FP32 accumulation, bias + ReLU + rounding to the next layer's
// operand type in the epilogue.  Operands and activations live in shared
// memory with padded row strides (conflict-free fragment loads).
//
// FP32: one thread per query on the SIMT cores with weights broadcast from
// shared memory (the plain reference evaluation).
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "bcf_internal.h"

namespace bcf {

// ----------------------------------------------------------------- MMA ops

__device__ __forceinline__ void mma_f16(float d[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_bf16(float d[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile("mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void mma_e4m3(float d[4], const uint32_t a[4], const uint32_t b[2])
{
    asm volatile("mma.sync.aligned.m16n8k32.row.col.f32.e4m3.e4m3.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
                 "{%0,%1,%2,%3};\n"
                 : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
                 : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Operand traits: element size, K per MMA, conversions.
template <int PREC>
struct Op;

template <>
struct Op<BCF_FP16> {
    static constexpr int kBytes = 2, kK = 16;
    __device__ static uint32_t pack2(float a, float b)
    {
        __half2 h = __floats2half2_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __device__ static void mma(float d[4], const uint32_t a[4], const uint32_t b[2]) { mma_f16(d, a, b); }
};

template <>
struct Op<BCF_BF16> {
    static constexpr int kBytes = 2, kK = 16;
    __device__ static uint32_t pack2(float a, float b)
    {
        __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        return *reinterpret_cast<uint32_t *>(&h);
    }
    __device__ static void mma(float d[4], const uint32_t a[4], const uint32_t b[2]) { mma_bf16(d, a, b); }
};

template <>
struct Op<BCF_FP8_E4M3> {
    static constexpr int kBytes = 1, kK = 32;
    // two E4M3 (round to nearest even, saturating): a in the low byte
    __device__ static uint32_t pack2(float a, float b)
    {
        return (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    }
    __device__ static void mma(float d[4], const uint32_t a[4], const uint32_t b[2]) { mma_e4m3(d, a, b); }
};

// Row stride (bytes) of an activation / weight tile with `k` operand columns:
// padded by 16 bytes so that the 8 fragment rows hit distinct banks.
template <int PREC>
__host__ __device__ constexpr int tile_stride_bytes(int k)
{
    return k * (PREC == BCF_FP8_E4M3 ? 1 : 2) + 16;
}

// Shared-memory image of the MLP for the tensor-core path: per layer the
// padded weights W[npad][kpad] in the operand type, then the padded biases.
struct MlpSmem {
    int w_off[BCF_MAX_LAYERS]; // byte offsets of each layer's weight tile
    int b_off[BCF_MAX_LAYERS]; // float offsets of each layer's biases
};

// Load the caller-layout weights into the padded shared tiles (zeros in the
// padding).  Called by all threads of the CTA, followed by __syncthreads().
template <int PREC>
__device__ void load_mlp_smem(const MlpDev &P, unsigned char *sw, float *sb)
{
    int woff = 0, boff = 0;
    for (int l = 0; l < P.n_layers; ++l) {
        const int kin = P.dims[l], nout = P.dims[l + 1];
        const int kp = P.kpad[l], np = P.npad[l];
        const int stride = tile_stride_bytes<PREC>(kp);
        for (int e = threadIdx.x; e < np * kp; e += blockDim.x) {
            const int n = e / kp, k = e % kp;
            unsigned char *dst = sw + woff + n * stride + k * Op<PREC>::kBytes;
            const bool in = n < nout && k < kin;
            const int64_t src = P.w_off[l] + (int64_t)n * kin + k;
            if (PREC == BCF_FP8_E4M3)
                *dst = in ? ((const unsigned char *)P.weights)[src] : 0;
            else
                *(uint16_t *)dst = in ? ((const uint16_t *)P.weights)[src] : 0;
        }
        for (int e = threadIdx.x; e < np; e += blockDim.x)
            sb[boff + e] = e < nout ? P.biases[P.b_off[l] + e] : 0.0f;
        woff += np * stride;
        boff += np;
    }
}

template <int PREC>
__host__ __device__ inline int mlp_smem_weight_bytes(const MlpDev &P)
{
    int b = 0;
    for (int l = 0; l < P.n_layers; ++l)
        b += P.npad[l] * tile_stride_bytes<PREC>(P.kpad[l]);
    return b;
}

__host__ __device__ inline int mlp_smem_bias_floats(const MlpDev &P)
{
    int b = 0;
    for (int l = 0; l < P.n_layers; ++l)
        b += P.npad[l];
    return b;
}

// Evaluate the MLP for the warp's 32 queries.  act0 holds the quantised
// layer-0 input rows (row = lane), act1 is scratch of the same size; the FP32
// outputs [32][n_out] are written to `out` (row-major, stride n_out).
template <int PREC>
__device__ void warp_mlp(const MlpDev &P, const unsigned char *sw, const float *sb, unsigned char *act0,
                         unsigned char *act1, float *out)
{
    const int lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    constexpr int EB = Op<PREC>::kBytes;
    constexpr int KK = Op<PREC>::kK;
    unsigned char *ain = act0, *aout = act1;
    int woff = 0, boff = 0;
    for (int l = 0; l < P.n_layers; ++l) {
        const int kp = P.kpad[l], np = P.npad[l];
        const int astride = tile_stride_bytes<PREC>(kp);
        const int wstride = astride;
        const bool last = l + 1 == P.n_layers;
        const int ostride = last ? 0 : tile_stride_bytes<PREC>(P.kpad[l + 1]);
        const float oscale = PREC == BCF_FP8_E4M3 ? P.act_scale[l] * P.w_scale[l] : 1.0f;
        const float next_inv = (PREC == BCF_FP8_E4M3 && !last) ? P.inv_act_scale[l + 1] : 1.0f;
        for (int m = 0; m < 2; ++m) {
            for (int n0 = 0; n0 < np; n0 += 8) {
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                for (int k0 = 0; k0 < kp; k0 += KK) {
                    uint32_t a[4], b[2];
                    const unsigned char *ar0 = ain + (m * 16 + g) * astride + k0 * EB;
                    const unsigned char *ar1 = ar0 + 8 * astride;
                    const int kc = (PREC == BCF_FP8_E4M3 ? 4 : 2) * t * EB; // byte column of this lane
                    const int kh = (KK / 2) * EB;                           // byte offset of the upper K half
                    a[0] = *(const uint32_t *)(ar0 + kc);
                    a[1] = *(const uint32_t *)(ar1 + kc);
                    a[2] = *(const uint32_t *)(ar0 + kc + kh);
                    a[3] = *(const uint32_t *)(ar1 + kc + kh);
                    const unsigned char *br = sw + woff + (n0 + g) * wstride + k0 * EB;
                    b[0] = *(const uint32_t *)(br + kc);
                    b[1] = *(const uint32_t *)(br + kc + kh);
                    Op<PREC>::mma(d, a, b);
                }
                // epilogue: rows m*16+g and m*16+g+8, columns n0+2t, n0+2t+1
                const int c0 = n0 + 2 * t;
                const float b0 = sb[boff + c0], b1 = sb[boff + c0 + 1];
                float v00 = d[0] * oscale + b0, v01 = d[1] * oscale + b1;
                float v10 = d[2] * oscale + b0, v11 = d[3] * oscale + b1;
                const int r0 = m * 16 + g, r1 = r0 + 8;
                if (last) {
                    const int C = P.dims[P.n_layers];
                    if (c0 < C) {
                        out[r0 * C + c0] = v00;
                        out[r1 * C + c0] = v10;
                    }
                    if (c0 + 1 < C) {
                        out[r0 * C + c0 + 1] = v01;
                        out[r1 * C + c0 + 1] = v11;
                    }
                } else {
                    v00 = fmaxf(v00, 0.f) * next_inv;
                    v01 = fmaxf(v01, 0.f) * next_inv;
                    v10 = fmaxf(v10, 0.f) * next_inv;
                    v11 = fmaxf(v11, 0.f) * next_inv;
                    const uint32_t p0 = Op<PREC>::pack2(v00, v01), p1 = Op<PREC>::pack2(v10, v11);
                    if (EB == 2) {
                        *(uint32_t *)(aout + r0 * ostride + c0 * 2) = p0;
                        *(uint32_t *)(aout + r1 * ostride + c0 * 2) = p1;
                    } else {
                        *(uint16_t *)(aout + r0 * ostride + c0) = (uint16_t)p0;
                        *(uint16_t *)(aout + r1 * ostride + c0) = (uint16_t)p1;
                    }
                }
            }
        }
        __syncwarp();
        woff += np * wstride;
        boff += np;
        unsigned char *tmp = ain;
        ain = aout;
        aout = tmp;
    }
}

// Write one query's layer-0 input row (features [n_in], zero padded to kpad)
// in the operand type; FP8 divides by the layer's activation scale first
// (scales are powers of two, so the multiply by the reciprocal is exact).
template <int PREC>
__device__ __forceinline__ void store_input_row(const MlpDev &P, const float *x, int n_in, unsigned char *row)
{
    const float inv = PREC == BCF_FP8_E4M3 ? P.inv_act_scale[0] : 1.0f;
    const int kp = P.kpad[0];
    for (int k = 0; k < kp; k += 2) {
        const float a = k < n_in ? x[k] * inv : 0.0f;
        const float b = k + 1 < n_in ? x[k + 1] * inv : 0.0f;
        const uint32_t p = Op<PREC>::pack2(a, b);
        if (Op<PREC>::kBytes == 2)
            *(uint32_t *)(row + 2 * k) = p;
        else
            *(uint16_t *)(row + k) = (uint16_t)p;
    }
}

// ----------------------------------------------------------- FP32 SIMT MLP

// Fully unrolled dense layer y = W x + b (W row-major [NO][NI] in shared
// memory, broadcast reads), optional ReLU.
template <int NI, int NO, bool RELU>
__device__ __forceinline__ void dense_fp32(const float *W, const float *b, const float (&x)[NI], float (&y)[NO])
{
#pragma unroll
    for (int o = 0; o < NO; ++o) {
        float acc = b[o];
#pragma unroll
        for (int i = 0; i < NI; ++i)
            acc = fmaf(W[o * NI + i], x[i], acc);
        y[o] = RELU ? fmaxf(acc, 0.0f) : acc;
    }
}

} // namespace bcf
