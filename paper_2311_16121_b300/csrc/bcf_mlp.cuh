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
    // max(a, 0), max(b, 0) rounded to nearest-even halves in one conversion (a in the low half)
    __device__ static uint32_t pack2_relu(float a, float b)
    {
        uint32_t d;
        asm("cvt.rn.relu.f16x2.f32 %0, %2, %1;" : "=r"(d) : "f"(a), "f"(b));
        return d;
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
    __device__ static uint32_t pack2_relu(float a, float b)
    {
        uint32_t d;
        asm("cvt.rn.relu.bf16x2.f32 %0, %2, %1;" : "=r"(d) : "f"(a), "f"(b));
        return d;
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
// padding) by threads tid = 0 .. nthreads - 1 of a group (the CTA, followed by
// __syncthreads(), or one warp, followed by __syncwarp()).
template <int PREC>
__device__ void load_mlp_smem(const MlpDev &P, unsigned char *sw, float *sb, int tid, int nthreads)
{
    int woff = 0, boff = 0;
    for (int l = 0; l < P.n_layers; ++l) {
        const int kin = P.dims[l], nout = P.dims[l + 1];
        const int kp = P.kpad[l], np = P.npad[l];
        const int stride = tile_stride_bytes<PREC>(kp);
        for (int e = tid; e < np * kp; e += nthreads) {
            const int n = e / kp, k = e % kp;
            unsigned char *dst = sw + woff + n * stride + k * Op<PREC>::kBytes;
            const bool in = n < nout && k < kin;
            const int64_t src = P.w_off[l] + (int64_t)n * kin + k;
            if (PREC == BCF_FP8_E4M3)
                *dst = in ? ((const unsigned char *)P.weights)[src] : 0;
            else
                *(uint16_t *)dst = in ? ((const uint16_t *)P.weights)[src] : 0;
        }
        for (int e = tid; e < np; e += nthreads)
            sb[boff + e] = e < nout ? P.biases[P.b_off[l] + e] : 0.0f;
        woff += np * stride;
        boff += np;
    }
}

// The whole CTA loads the weights and biases.
template <int PREC>
__device__ void load_mlp_smem(const MlpDev &P, unsigned char *sw, float *sb)
{
    load_mlp_smem<PREC>(P, sw, sb, threadIdx.x, blockDim.x);
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

// One MLP input feature written in the operand format (FP8: scaled by the layer's inverse activation scale).
template <int PREC>
__device__ __forceinline__ void store_feature(unsigned char *row, int col, float x, float inv_scale)
{
    if constexpr (PREC == BCF_FP8_E4M3) {
        row[col] = (unsigned char)__nv_cvt_float_to_fp8(x * inv_scale, __NV_SATFINITE, __NV_E4M3);
    } else if constexpr (PREC == BCF_BF16) {
        *(__nv_bfloat16 *)(row + 2 * col) = __float2bfloat16_rn(x);
    } else {
        *(__half *)(row + 2 * col) = __float2half_rn(x);
    }
}

// Coalesced store of a warp's rows [q0, q0 + rows) from the FP32 staging tile ost[rows][C]: FP16 output in
// 16-byte chunks of 8 values (q0 is a multiple of 32, so a chunk never straddles the 16-byte alignment of out),
// the tail value by value; FP32 output in chunks of 4.
__device__ __forceinline__ void store_warp_rows(const float *ost, void *out, int64_t q0, int rows, int C, int out_fp16,
                                                int lane)
{
    const int tot = rows * C;
    if (out_fp16) {
        __half *o = (__half *)out + q0 * C;
        const int full = tot >> 3;
        for (int k = lane; k < full; k += 32) {
            const float4 a = *reinterpret_cast<const float4 *>(ost + 8 * k);
            const float4 b = *reinterpret_cast<const float4 *>(ost + 8 * k + 4);
            const __half2 h0 = __floats2half2_rn(a.x, a.y), h1 = __floats2half2_rn(a.z, a.w);
            const __half2 h2 = __floats2half2_rn(b.x, b.y), h3 = __floats2half2_rn(b.z, b.w);
            uint4 w;
            w.x = *reinterpret_cast<const uint32_t *>(&h0);
            w.y = *reinterpret_cast<const uint32_t *>(&h1);
            w.z = *reinterpret_cast<const uint32_t *>(&h2);
            w.w = *reinterpret_cast<const uint32_t *>(&h3);
            *reinterpret_cast<uint4 *>(o + 8 * k) = w;
        }
        for (int i = (full << 3) + lane; i < tot; i += 32)
            o[i] = __float2half_rn(ost[i]);
    } else {
        float *o = (float *)out + q0 * C;
        const int full = tot >> 2;
        for (int k = lane; k < full; k += 32)
            *reinterpret_cast<float4 *>(o + 4 * k) = *reinterpret_cast<const float4 *>(ost + 4 * k);
        for (int i = (full << 2) + lane; i < tot; i += 32)
            o[i] = ost[i];
    }
}

// store_warp_rows for rows starting anywhere (material-set ranges): the 16-byte path when the first output
// element is 16-byte aligned, element by element otherwise.
__device__ __forceinline__ void store_rows_any(const float *ost, void *out, int64_t q0, int rows, int C, int out_fp16,
                                               int lane)
{
    if (((q0 * C * (out_fp16 ? 2 : 4)) & 15) == 0) {
        store_warp_rows(ost, out, q0, rows, C, out_fp16, lane);
        return;
    }
    const int tot = rows * C;
    if (out_fp16) {
        __half *o = (__half *)out + q0 * C;
        for (int i = lane; i < tot; i += 32)
            o[i] = __float2half_rn(ost[i]);
    } else {
        float *o = (float *)out + q0 * C;
        for (int i = lane; i < tot; i += 32)
            o[i] = ost[i];
    }
}

// Writes a query's MLP input row column by column, in increasing column order: 16-bit operands go out in
// pairs (one 4-byte store per two columns), E4M3 bytes one by one.
template <int PREC>
struct RowWriter {
    unsigned char *row;
    float inv; // FP8: the first layer's inverse activation scale
    float pend; // the value of an even column waiting for its odd neighbour
    __device__ __forceinline__ void put(int col, float x)
    {
        if constexpr (PREC == BCF_FP8_E4M3) {
            store_feature<PREC>(row, col, x, inv);
        } else if (col & 1) {
            *reinterpret_cast<uint32_t *>(row + 2 * (col - 1)) = Op<PREC>::pack2(pend, x);
        } else {
            pend = x;
        }
    }
    // after the last column: an unpaired even column is written alone
    __device__ __forceinline__ void finish(int ncols)
    {
        if constexpr (PREC != BCF_FP8_E4M3)
            if (ncols & 1)
                store_feature<PREC>(row, ncols - 1, pend, inv);
    }
};

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

namespace bcf {

// ------------------------------------------ register-chained 3-layer MLP

__device__ __forceinline__ uint32_t lds32(const unsigned char *p) { return *reinterpret_cast<const uint32_t *>(p); }

// B fragment (k0..k0+KK, n0..n0+8) of a padded weight tile W[npad][kpad]
// (row stride `stride` bytes) for MMA K size KK and element size EB.
template <int EB, int KK>
__device__ __forceinline__ void load_b(const unsigned char *W, int stride, int k0, int n0, int g, int t, uint32_t b[2])
{
    const unsigned char *r = W + (n0 + g) * stride + k0 * EB;
    const int kc = (EB == 1 ? 4 : 2) * t * EB;
    b[0] = lds32(r + kc);
    b[1] = lds32(r + kc + (KK / 2) * EB);
}

// A fragment (rows r0..r0+16, k0..k0+KK) of a row-major tile (row stride `stride` bytes).
template <int EB, int KK>
__device__ __forceinline__ void load_a(const unsigned char *A, int stride, int r0, int k0, int g, int t, uint32_t a[4])
{
    const unsigned char *p0 = A + (r0 + g) * stride + k0 * EB;
    const unsigned char *p1 = p0 + 8 * stride;
    const int kc = (EB == 1 ? 4 : 2) * t * EB;
    const int kh = (KK / 2) * EB;
    a[0] = lds32(p0 + kc);
    a[1] = lds32(p1 + kc);
    a[2] = lds32(p0 + kc + kh);
    a[3] = lds32(p1 + kc + kh);
}

// Dense layer on MT 16-row tiles: D[m][NP/8][4] = A_m(16 x KP) * W^T; each B
// fragment is loaded once and used for all MT row tiles.
template <int PREC, int MT, int KP, int NP>
__device__ __forceinline__ void mma_layer(const uint32_t (&a)[MT][KP / Op<PREC>::kK][4], const unsigned char *W,
                                          int stride, int g, int t, float (&d)[MT][NP / 8][4],
                                          const float *bias = nullptr)
{
    constexpr int KK = Op<PREC>::kK, EB = Op<PREC>::kBytes;
#pragma unroll
    for (int nt = 0; nt < NP / 8; ++nt) {
        // accumulators start at the bias (columns 8 nt + 2 t, + 1) when one is given, else at 0
        const float c0 = bias ? bias[nt * 8 + 2 * t] : 0.0f, c1 = bias ? bias[nt * 8 + 2 * t + 1] : 0.0f;
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            d[m][nt][0] = d[m][nt][2] = c0;
            d[m][nt][1] = d[m][nt][3] = c1;
        }
#pragma unroll
        for (int kt = 0; kt < KP / KK; ++kt) {
            uint32_t b[2];
            load_b<EB, KK>(W, stride, kt * KK, nt * 8, g, t, b);
#pragma unroll
            for (int m = 0; m < MT; ++m)
                Op<PREC>::mma(d[m][nt], a[m][kt], b);
        }
    }
}

// Hidden epilogue for 16-bit operands: the accumulators already hold bias + sum (mma_layer with a bias); ReLU
// and rounding in one conversion, straight into the next layer's A fragments (D tile columns 8 nt + 2 t map
// onto A fragment nt / 2, registers 0/1 for even nt and 2/3 for odd nt).
template <int PREC, int MT, int NP>
__device__ __forceinline__ void hidden_to_a16(const float (&d)[MT][NP / 8][4], uint32_t (&a)[MT][NP / 16][4])
{
#pragma unroll
    for (int nt = 0; nt < NP / 8; ++nt) {
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            a[m][nt >> 1][(nt & 1) * 2 + 0] = Op<PREC>::pack2_relu(d[m][nt][0], d[m][nt][1]);
            a[m][nt >> 1][(nt & 1) * 2 + 1] = Op<PREC>::pack2_relu(d[m][nt][2], d[m][nt][3]);
        }
    }
}

// Hidden epilogue for FP8: bias + ReLU after the scale, divided by the next
// layer's activation scale, rounded to E4M3 into a byte tile (16 MT rows),
// from which the next layer's (K = 32) A fragments are loaded.
template <int MT, int NP>
__device__ __forceinline__ void hidden_to_tile8(const float (&d)[MT][NP / 8][4], const float *bias, float oscale,
                                                float next_inv, int g, int t, unsigned char *tile, int stride)
{
#pragma unroll
    for (int nt = 0; nt < NP / 8; ++nt) {
        const int c = nt * 8 + 2 * t;
        const float b0 = bias[c], b1 = bias[c + 1];
#pragma unroll
        for (int m = 0; m < MT; ++m) {
            const uint32_t lo = Op<BCF_FP8_E4M3>::pack2(fmaxf(d[m][nt][0] * oscale + b0, 0.f) * next_inv,
                                                        fmaxf(d[m][nt][1] * oscale + b1, 0.f) * next_inv);
            const uint32_t hi = Op<BCF_FP8_E4M3>::pack2(fmaxf(d[m][nt][2] * oscale + b0, 0.f) * next_inv,
                                                        fmaxf(d[m][nt][3] * oscale + b1, 0.f) * next_inv);
            *reinterpret_cast<uint16_t *>(tile + (m * 16 + g) * stride + c) = (uint16_t)lo;
            *reinterpret_cast<uint16_t *>(tile + (m * 16 + g + 8) * stride + c) = (uint16_t)hi;
        }
    }
}

// Rows processed together by warp_mlp3.  One 16-row tile per pass: two
// tiles would let each weight fragment feed two MMAs, but under the decode
// kernel's 80-register budget the extra accumulators spill.
template <int N1, int N2>
struct MlpRows {
    static constexpr int kMT = 1;
};

// K0 -> N1 -> N2 -> NO (all padded) MLP for the warp's 32 rows.  in: the
// quantised input tile [32][K0] (row stride in_stride bytes).  The FP32
// outputs go to ost[32][C]; all A fragments of a pass are loaded before its
// outputs are written.  tmp8: FP8 scratch tile (16 kMT rows, stride
// tmp_stride) for the FP8 layer chaining.
template <int PREC, int K0, int N1, int N2, int NO>
__device__ __forceinline__ void warp_mlp3(const MlpDev &P, const unsigned char *sw, const float *sb,
                                          const unsigned char *in, int in_stride, unsigned char *tmp8,
                                          int tmp_stride, float *ost, int C)
{
    constexpr int KK = Op<PREC>::kK, EB = Op<PREC>::kBytes;
    constexpr int MT = MlpRows<N1, N2>::kMT;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int s0 = tile_stride_bytes<PREC>(K0), s1 = tile_stride_bytes<PREC>(N1), s2 = tile_stride_bytes<PREC>(N2);
    const unsigned char *W0 = sw;
    const unsigned char *W1 = W0 + N1 * s0;
    const unsigned char *W2 = W1 + N2 * s1;
    const float *b0 = sb, *b1 = sb + N1, *b2 = sb + N1 + N2;
    float sc0 = 1.f, sc1 = 1.f, sc2 = 1.f, in1 = 1.f, in2 = 1.f;
    if constexpr (PREC == BCF_FP8_E4M3) {
        sc0 = P.act_scale[0] * P.w_scale[0];
        sc1 = P.act_scale[1] * P.w_scale[1];
        sc2 = P.act_scale[2] * P.w_scale[2];
        in1 = P.inv_act_scale[1];
        in2 = P.inv_act_scale[2];
    }
#pragma unroll 1
    for (int m0 = 0; m0 < 2; m0 += MT) {
        uint32_t a0[MT][K0 / KK][4];
#pragma unroll
        for (int m = 0; m < MT; ++m)
#pragma unroll
            for (int kt = 0; kt < K0 / KK; ++kt)
                load_a<EB, KK>(in, in_stride, (m0 + m) * 16, kt * KK, g, t, a0[m][kt]);
        float d1[MT][N1 / 8][4];
        mma_layer<PREC, MT, K0, N1>(a0, W0, s0, g, t, d1, PREC == BCF_FP8_E4M3 ? nullptr : b0);
        uint32_t a1[MT][N1 / KK][4];
        if constexpr (PREC == BCF_FP8_E4M3) {
            hidden_to_tile8<MT, N1>(d1, b0, sc0, in1, g, t, tmp8, tmp_stride);
            __syncwarp();
#pragma unroll
            for (int m = 0; m < MT; ++m)
#pragma unroll
                for (int kt = 0; kt < N1 / KK; ++kt)
                    load_a<EB, KK>(tmp8, tmp_stride, m * 16, kt * KK, g, t, a1[m][kt]);
            __syncwarp();
        } else {
            hidden_to_a16<PREC, MT, N1>(d1, a1);
        }
        float d2[MT][N2 / 8][4];
        mma_layer<PREC, MT, N1, N2>(a1, W1, s1, g, t, d2, PREC == BCF_FP8_E4M3 ? nullptr : b1);
        uint32_t a2[MT][N2 / KK][4];
        if constexpr (PREC == BCF_FP8_E4M3) {
            hidden_to_tile8<MT, N2>(d2, b1, sc1, in2, g, t, tmp8, tmp_stride);
            __syncwarp();
#pragma unroll
            for (int m = 0; m < MT; ++m)
#pragma unroll
                for (int kt = 0; kt < N2 / KK; ++kt)
                    load_a<EB, KK>(tmp8, tmp_stride, m * 16, kt * KK, g, t, a2[m][kt]);
            __syncwarp();
        } else {
            hidden_to_a16<PREC, MT, N2>(d2, a2);
        }
        float d3[MT][NO / 8][4];
        mma_layer<PREC, MT, N2, NO>(a2, W2, s2, g, t, d3, PREC == BCF_FP8_E4M3 ? nullptr : b2);
#pragma unroll
        for (int nt = 0; nt < NO / 8; ++nt) {
            const int c = nt * 8 + 2 * t;
#pragma unroll
            for (int m = 0; m < MT; ++m) {
                const int r0 = (m0 + m) * 16 + g, r1 = r0 + 8;
                if constexpr (PREC == BCF_FP8_E4M3) {
                    if (c < C) {
                        ost[r0 * C + c] = d3[m][nt][0] * sc2 + b2[c];
                        ost[r1 * C + c] = d3[m][nt][2] * sc2 + b2[c];
                    }
                    if (c + 1 < C) {
                        ost[r0 * C + c + 1] = d3[m][nt][1] * sc2 + b2[c + 1];
                        ost[r1 * C + c + 1] = d3[m][nt][3] * sc2 + b2[c + 1];
                    }
                } else { // the bias is in the accumulators
                    if (c < C) {
                        ost[r0 * C + c] = d3[m][nt][0];
                        ost[r1 * C + c] = d3[m][nt][2];
                    }
                    if (c + 1 < C) {
                        ost[r0 * C + c + 1] = d3[m][nt][1];
                        ost[r1 * C + c + 1] = d3[m][nt][3];
                    }
                }
            }
        }
    }
}

// K0 -> N1 -> NO (padded) MLP with one hidden layer -- the paper's decoder shape (12 inputs, one hidden layer
// of 16, Sec. 5.1) -- for 16-bit operands, layers chained through registers as in warp_mlp3.
template <int PREC, int K0, int N1, int NO>
__device__ __forceinline__ void warp_mlp2(const unsigned char *sw, const float *sb, const unsigned char *in,
                                          int in_stride, float *ost, int C)
{
    static_assert(PREC != BCF_FP8_E4M3, "FP8 pads the hidden layer's K to 32: the generic MLP covers it");
    constexpr int KK = Op<PREC>::kK, EB = Op<PREC>::kBytes;
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int s0 = tile_stride_bytes<PREC>(K0), s1 = tile_stride_bytes<PREC>(N1);
    const unsigned char *W0 = sw;
    const unsigned char *W1 = W0 + N1 * s0;
    const float *b0 = sb, *b1 = sb + N1;
#pragma unroll 1
    for (int m0 = 0; m0 < 2; ++m0) {
        uint32_t a0[1][K0 / KK][4];
#pragma unroll
        for (int kt = 0; kt < K0 / KK; ++kt)
            load_a<EB, KK>(in, in_stride, m0 * 16, kt * KK, g, t, a0[0][kt]);
        float d1[1][N1 / 8][4];
        mma_layer<PREC, 1, K0, N1>(a0, W0, s0, g, t, d1, b0);
        uint32_t a1[1][N1 / KK][4];
        hidden_to_a16<PREC, 1, N1>(d1, a1);
        float d2[1][NO / 8][4];
        mma_layer<PREC, 1, N1, NO>(a1, W1, s1, g, t, d2, b1);
#pragma unroll
        for (int nt = 0; nt < NO / 8; ++nt) {
            const int c = nt * 8 + 2 * t;
            const int r0 = m0 * 16 + g, r1 = r0 + 8;
            if (c < C) {
                ost[r0 * C + c] = d2[0][nt][0];
                ost[r1 * C + c] = d2[0][nt][2];
            }
            if (c + 1 < C) {
                ost[r0 * C + c + 1] = d2[0][nt][1];
                ost[r1 * C + c + 1] = d2[0][nt][3];
            }
        }
    }
}

} // namespace bcf
