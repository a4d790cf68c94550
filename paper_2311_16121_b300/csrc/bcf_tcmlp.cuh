// bcf_tcmlp.cuh -- the MLP decoder f_eta of Eq. 3 on the fifth-generation tensor cores (tcgen05) for a CTA tile
// of 32 NW queries (NW = 4, 8 or 16 warps).
//
// Every thread first writes the layer's FP32 bias into its own row's accumulator columns in tensor memory
// (tcgen05.st; for E4M3 the bias divided by the layer's power-of-two product scale, which is exact); one
// thread then issues the layer's MMAs (M = 128 rows per instruction, one per 128-row part of the tile, K = 16
// for FP16 / BF16 and 32 for E4M3 per instruction), which accumulate onto the bias in FP32; every thread reads
// its own row's accumulators back (tcgen05.ld, 32 lanes x 32-bit columns per warp), applies ReLU and rounds to
// the next layer's operand type straight into that layer's A tile in shared memory.  The part of the tile a
// row lies in owns one block of MAXN accumulator columns for all three layers (the parts share the 128 lanes).
// Operand tiles use the canonical K-major layout without swizzling: 8-row groups of 16-byte
// core matrices, core matrices along K 128 bytes apart (the descriptor's leading byte offset), 8-row groups
// (K bytes / 16) x 128 bytes apart (its stride byte offset).
//
// Synchronisation per layer: every thread waits for its bias stores (tcgen05.wait::st) and orders them, and
// its reads of the previous layer's accumulators, before the barrier (tcgen05.fence::before_thread_sync); the
// A tile's writers fence their generic-proxy stores for the async proxy; all meet at a CTA barrier (which also
// keeps the A tiles in y, aliasing the caller's texel arena, from being written before every warp's filter is
// done); the issuing thread orders the MMAs after it (tcgen05.fence::after_thread_sync) and commits them to an
// mbarrier; every thread waits on that mbarrier (a bounded wait: when it runs out, the caller's check word gets
// BCF_CHECK_TIMEOUT and the kernel stops taking tiles) and reads the accumulators.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "bcf_internal.h"
#include "bcf_mlp.cuh"

namespace bcf {

// ---------------------------------------------------------------- PTX wrappers

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.b32 %0, 1, 0, p;\n\t}\n"
                 : "=r"(ok)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the mbarrier to complete, at most `limit` polls; false when the limit ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int limit)
{
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// Tensor-memory allocation (one full warp): the column base is written to *dst (shared memory).
__device__ __forceinline__ void tc_alloc(uint32_t *dst, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(dst)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory matrix descriptor: start address, leading byte offset (between core matrices along K), stride
// byte offset (between 8-row groups), the descriptor version bits 46-48 = 0b001, base offset 0, no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Instruction descriptor of a dense MMA with FP32 accumulation: A and B formats (kind::f16: 0 = F16, 1 = BF16;
// kind::f8f6f4: 0 = E4M3), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n, uint32_t ab_fmt)
{
    return (1u << 4) | (ab_fmt << 7) | (ab_fmt << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc)
{
    if constexpr (PREC == BCF_FP8_E4M3)
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
                     "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
                     : "memory");
    else
        asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
                     "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
                     : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

// Store 16 consecutive 32-bit columns of the calling thread's tensor-memory lane (completion: tc_wait_st).
__device__ __forceinline__ void tc_st16(uint32_t taddr, const float (&v)[16])
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15, %16};" ::"r"(taddr),
                 "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
                 "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
                 "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
                 "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
                 "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
                 "r"(__float_as_uint(v[15]))
                 : "memory");
}

__device__ __forceinline__ void tc_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// 16 consecutive 32-bit accumulator columns of the calling thread's tensor-memory lane.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                 "%13, %14, %15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                   "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
                   "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i)
        v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------- the CTA MLP

__host__ __device__ constexpr int tc_pow2_cols(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : 256; }

template <int PREC, int NW, int K0, int N1, int N2, int NO>
struct TcMlp {
    static_assert(NW == 4 || NW == 8 || NW == 16 || NW == 32, "whole 128-row MMA quarters of the tile");
    static constexpr int EB = PREC == BCF_FP8_E4M3 ? 1 : 2;
    static constexpr int KS = PREC == BCF_FP8_E4M3 ? 32 : 16; // K per MMA instruction
    static constexpr int ROWS = 32 * NW, HALVES = NW / 4;
    static constexpr uint32_t FMT = PREC == BCF_BF16 ? 1u : 0u;
    static_assert(K0 % KS == 0 && N1 % KS == 0 && N2 % KS == 0, "K of every layer a multiple of the MMA K");
    static_assert(N1 % 16 == 0 && N2 % 16 == 0 && NO % 16 == 0 && NO >= 16, "N a multiple of 16 for M = 128");
    static constexpr int MAXN = N1 > N2 ? (N1 > NO ? N1 : NO) : (N2 > NO ? N2 : NO);
    static constexpr int NCOLS = tc_pow2_cols(MAXN * HALVES); // tensor-memory columns per CTA
    // bytes of a canonical tile with `rows` rows and K columns, and its 8-row group stride
    __host__ __device__ static constexpr int tile_bytes(int rows, int k) { return rows * k * EB; }
    __host__ __device__ static constexpr int sbo(int k) { return k * EB / 16 * 128; }
    static constexpr int W0B = tile_bytes(N1, K0), W1B = tile_bytes(N2, N1), W2B = tile_bytes(NO, N2);
    static constexpr int W_BYTES = W0B + W1B + W2B;            // B tiles of the three layers
    static constexpr int X_BYTES = tile_bytes(ROWS, K0);                // A0
    static constexpr int Y_BYTES = tile_bytes(ROWS, N1 > N2 ? N1 : N2); // A1, then A2, then the output staging
    // byte offset of element (r, k) in a canonical tile with K columns
    __device__ __forceinline__ static int off(int r, int k, int K)
    {
        const int kb = k * EB;
        return (r >> 3) * sbo(K) + (kb >> 4) * 128 + (r & 7) * 16 + (kb & 15);
    }
};

// Load the caller-layout weights (W_l [out][in] row-major in the material's precision) into the canonical B
// tiles (zero padding) and the biases (zero padding); all threads, followed by a CTA barrier.
template <int PREC, int NW, int K0, int N1, int N2, int NO>
__device__ void tc_load_weights(const MlpDev &P, unsigned char *w, float *sb)
{
    using T = TcMlp<PREC, NW, K0, N1, N2, NO>;
    const int kp[3] = {K0, N1, N2}, np[3] = {N1, N2, NO};
    int woff = 0, boff = 0;
    for (int l = 0; l < 3; ++l) {
        const int kin = P.dims[l], nout = P.dims[l + 1];
        for (int e = threadIdx.x; e < np[l] * kp[l]; e += blockDim.x) {
            const int n = e / kp[l], k = e % kp[l];
            const bool in = n < nout && k < kin;
            const int64_t src = P.w_off[l] + (int64_t)n * kin + k;
            unsigned char *dst = w + woff + T::off(n, k, kp[l]);
            if constexpr (PREC == BCF_FP8_E4M3)
                *dst = in ? ((const unsigned char *)P.weights)[src] : 0;
            else
                *(uint16_t *)dst = in ? ((const uint16_t *)P.weights)[src] : 0;
        }
        for (int e = threadIdx.x; e < np[l]; e += blockDim.x)
            sb[boff + e] = e < nout ? P.biases[P.b_off[l] + e] : 0.0f;
        woff += np[l] * kp[l] * T::EB;
        boff += np[l];
    }
}

// Write one input feature of row r (column col) into the canonical A0 tile: 16-bit operands in pairs (the
// even column's value waits in `pend`), E4M3 bytes one by one (x already scaled by the inverse activation scale).
template <int PREC, int NW, int K0, int N1, int N2, int NO>
struct TcRowWriter {
    unsigned char *a0;
    int r;
    float inv;
    float pend;        // 16-bit: the value of an even column waiting for its odd neighbour
    uint32_t word = 0; // E4M3: the bytes of the current group of four columns
    // columns in increasing order from 0; each group of two (16-bit) or four (E4M3) columns is one 4-byte store
    __device__ __forceinline__ void put(int col, float x)
    {
        using T = TcMlp<PREC, NW, K0, N1, N2, NO>;
        if constexpr (PREC == BCF_FP8_E4M3) {
            word |= (uint32_t)(unsigned char)__nv_cvt_float_to_fp8(x * inv, __NV_SATFINITE, __NV_E4M3)
                    << (8 * (col & 3));
            if ((col & 3) == 3) {
                *reinterpret_cast<uint32_t *>(a0 + T::off(r, col - 3, K0)) = word;
                word = 0u;
            }
        } else if (col & 1) {
            *reinterpret_cast<uint32_t *>(a0 + T::off(r, col - 1, K0)) = Op<PREC>::pack2(pend, x);
        } else {
            pend = x;
        }
    }
    // after the last column written: its partial group, then zeros up to the padded width K0
    __device__ __forceinline__ void finish(int ncols)
    {
        using T = TcMlp<PREC, NW, K0, N1, N2, NO>;
        constexpr int G = PREC == BCF_FP8_E4M3 ? 4 : 2; // columns per 4-byte store
        int c = ncols & ~(G - 1);
        if (ncols & (G - 1)) {
            if constexpr (PREC == BCF_FP8_E4M3)
                *reinterpret_cast<uint32_t *>(a0 + T::off(r, c, K0)) = word;
            else
                *reinterpret_cast<uint32_t *>(a0 + T::off(r, c, K0)) = Op<PREC>::pack2(pend, 0.0f);
            c += G;
        }
        for (; c < K0; c += G)
            *reinterpret_cast<uint32_t *>(a0 + T::off(r, c, K0)) = 0u;
    }
};

// Issue one layer: for every 128-row part h of the tile, K / KS MMAs accumulating A (rows of that part, K
// columns) x B^T onto tensor-memory columns [h CS, h CS + N) (which hold the bias), then commit them to the
// mbarrier.
template <int PREC, int NW, int K, int N, int CS>
__device__ __forceinline__ void tc_issue_layer(uint32_t tmem, const unsigned char *a, const unsigned char *b,
                                               uint64_t *bar)
{
    constexpr int EB = PREC == BCF_FP8_E4M3 ? 1 : 2, KS = PREC == BCF_FP8_E4M3 ? 32 : 16;
    constexpr uint32_t FMT = PREC == BCF_BF16 ? 1u : 0u;
    constexpr int SBO = K * EB / 16 * 128;
    constexpr uint32_t idesc = tc_idesc(128, N, FMT);
    tc_fence_after();
#pragma unroll
    for (int h = 0; h < NW / 4; ++h)
#pragma unroll
        for (int s = 0; s < K / KS; ++s) {
            // K step s covers KS elements = 2 core matrices along K (2 x 128 bytes)
            const uint64_t ad = tc_smem_desc(smem_addr(a) + h * 16 * SBO + s * 256, 128, SBO);
            const uint64_t bd = tc_smem_desc(smem_addr(b) + s * 256, 128, SBO);
            tc_mma<PREC>(tmem + (uint32_t)(h * CS), ad, bd, idesc, 1u);
        }
    tc_commit(bar);
}

// Write the bias of a layer (N columns; multiplied by inv, the inverse of the layer's product scale) into the
// calling thread's accumulator columns starting at trow, and wait for the stores.
template <int N>
__device__ __forceinline__ void tc_bias_init(uint32_t trow, const float *bias, float inv)
{
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
#pragma unroll
        for (int j = 0; j < 16; j += 4) {
            const float4 b4 = *reinterpret_cast<const float4 *>(bias + c0 + j);
            v[j] = b4.x * inv;
            v[j + 1] = b4.y * inv;
            v[j + 2] = b4.z * inv;
            v[j + 3] = b4.w * inv;
        }
        tc_st16(trow + (uint32_t)c0, v);
    }
    tc_wait_st();
}

// Hidden epilogue of one layer for the calling thread's row: accumulators (N columns, bias included), ReLU,
// rounding to the operand type (E4M3: after the product scale and the next layer's inverse activation scale)
// into the next A tile (row r, N columns), 16 bytes at a time.
template <int PREC, int NW, int K0, int N1, int N2, int NO, int N>
__device__ __forceinline__ void tc_hidden(uint32_t trow, float oscale, float next_inv, unsigned char *anext, int r)
{
    using T = TcMlp<PREC, NW, K0, N1, N2, NO>;
#pragma unroll
    for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tc_ld16(trow + (uint32_t)c0, v);
        if constexpr (PREC == BCF_FP8_E4M3) {
            uint32_t w[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float x0 = fmaxf(v[4 * j] * oscale, 0.f) * next_inv;
                const float x1 = fmaxf(v[4 * j + 1] * oscale, 0.f) * next_inv;
                const float x2 = fmaxf(v[4 * j + 2] * oscale, 0.f) * next_inv;
                const float x3 = fmaxf(v[4 * j + 3] * oscale, 0.f) * next_inv;
                w[j] = Op<PREC>::pack2(x0, x1) | (Op<PREC>::pack2(x2, x3) << 16);
            }
            *reinterpret_cast<uint4 *>(anext + T::off(r, c0, N)) = make_uint4(w[0], w[1], w[2], w[3]);
        } else {
            uint32_t w[8];
#pragma unroll
            for (int j = 0; j < 8; ++j)
                w[j] = Op<PREC>::pack2_relu(v[2 * j], v[2 * j + 1]);
            *reinterpret_cast<uint4 *>(anext + T::off(r, c0, N)) = make_uint4(w[0], w[1], w[2], w[3]);
            *reinterpret_cast<uint4 *>(anext + T::off(r, c0 + 8, N)) = make_uint4(w[4], w[5], w[6], w[7]);
        }
    }
}

// The three layers for the CTA tile whose A0 tile (x) every thread has written.  Called by all threads; the
// FP32 outputs of row r (C values) go to ost[r * C + c] (ost may alias y, not x: the next tile's features may
// be written into x while other warps still read their outputs).  A1 and then A2 live in y: each layer's MMA has
// completed before the next epilogue overwrites its operand.  Returns false when a bounded wait ran out (the
// tile's outputs are then undefined).  phase: the mbarrier parity, flipped per layer.
template <int PREC, int NW, int K0, int N1, int N2, int NO>
__device__ __forceinline__ bool tc_mlp3(const MlpDev &P, const unsigned char *w, const float *sb, unsigned char *x,
                                        unsigned char *y, float *ost, int C, uint64_t *bar, uint32_t &phase,
                                        uint32_t tmem, int wait_limit)
{
    using T = TcMlp<PREC, NW, K0, N1, N2, NO>;
    constexpr int CS = T::MAXN; // accumulator columns of one 128-row part
    const int warp = threadIdx.x >> 5, r = threadIdx.x;
    const int half = warp >> 2;
    // this thread's tensor-memory lane (lane quarter warp % 4 of the CTA's allocation) and its part's columns
    const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(half * CS);
    const unsigned char *W0 = w, *W1 = w + T::W0B, *W2 = W1 + T::W1B;
    const float *b0 = sb, *b1 = sb + N1, *b2 = sb + N1 + N2;
    float sc0 = 1.f, sc1 = 1.f, sc2 = 1.f, in1 = 1.f, in2 = 1.f;
    if constexpr (PREC == BCF_FP8_E4M3) {
        sc0 = P.act_scale[0] * P.w_scale[0];
        sc1 = P.act_scale[1] * P.w_scale[1];
        sc2 = P.act_scale[2] * P.w_scale[2];
        in1 = P.inv_act_scale[1];
        in2 = P.inv_act_scale[2];
    }
    // the products of an E4M3 layer are scaled by sc after the sum: its bias enters the sum as b / sc (exact:
    // the scales are powers of two)
    const float ib0 = PREC == BCF_FP8_E4M3 ? 1.0f / sc0 : 1.0f, ib1 = PREC == BCF_FP8_E4M3 ? 1.0f / sc1 : 1.0f,
                ib2 = PREC == BCF_FP8_E4M3 ? 1.0f / sc2 : 1.0f;
    bool ok = true;
    // layer 1: bias, then A0 (x) accumulated onto it
    tc_bias_init<N1>(trow, b0, ib0);
    tc_fence_before();
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0)
        tc_issue_layer<PREC, NW, K0, N1, CS>(tmem, x, W0, bar);
    ok = mbar_wait_bounded(bar, phase, wait_limit) && ok;
    phase ^= 1u;
    tc_fence_after();
    tc_hidden<PREC, NW, K0, N1, N2, NO, N1>(trow, sc0, in1, y, r);
    // layer 2 into the same columns (read above); A2 then overwrites A1 in y
    tc_bias_init<N2>(trow, b1, ib1);
    tc_fence_before();
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0)
        tc_issue_layer<PREC, NW, N1, N2, CS>(tmem, y, W1, bar);
    ok = mbar_wait_bounded(bar, phase, wait_limit) && ok;
    phase ^= 1u;
    tc_fence_after();
    tc_hidden<PREC, NW, K0, N1, N2, NO, N2>(trow, sc1, in2, y, r);
    // layer 3: A2 (y) -> outputs
    tc_bias_init<NO>(trow, b2, ib2);
    tc_fence_before();
    fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0)
        tc_issue_layer<PREC, NW, N2, NO, CS>(tmem, y, W2, bar);
    ok = mbar_wait_bounded(bar, phase, wait_limit) && ok;
    phase ^= 1u;
    tc_fence_after();
#pragma unroll
    for (int c0 = 0; c0 < NO; c0 += 16) {
        float v[16];
        tc_ld16(trow + (uint32_t)c0, v);
#pragma unroll
        for (int j = 0; j < 16; ++j)
            if (c0 + j < C)
                ost[r * C + c0 + j] = PREC == BCF_FP8_E4M3 ? v[j] * sc2 : v[j];
    }
    tc_fence_before();
    return ok;
}

} // namespace bcf
