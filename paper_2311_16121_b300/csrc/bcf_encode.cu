// bcf_encode.cu -- BC6H mode-10 block encoder: partition selection and the
// initial block parameters from free per-texel features (Sec. 5.1: the
// unconstrained features of a short first training stage are compressed with
// the BC6 algorithm, which fixes each block's partition and initialises its
// endpoints and indices).
//
// One warp per block, one lane per partition k = 0..31.  Each lane fits a
// line to each of its two regions in the format's interpolation domain (the
// binary16 bit pattern of the value): mean, 3 x 3 scatter matrix, principal
// axis by 8 power iterations started from the scatter column of the largest
// diagonal entry, segment between the smallest and largest projections.  The
// segment ends are quantised to 6-bit endpoints (inverting unquantise
// 1024 e + 512 and finish x 31/64), each texel takes the 3-bit index whose
// decoded value is closest (squared RGB error in value space), and the warp
// keeps the partition with the smallest total error (ties: smaller k).
//
// Every floating-point quantity here decides an integer (an endpoint, an
// index, the partition), so it is computed in IEEE single precision with
// explicitly rounded operations in one fixed order -- no contraction into
// fused multiply-adds -- which makes the choice reproducible and independent
// of compiler scheduling.
#include <cuda_fp16.h>
#include <math.h>

#include "bc6h_unpack.cuh"
#include "bcf_kernels.h"

namespace bcf {
namespace {

constexpr int kEncWarps = 8;

__device__ __forceinline__ float fmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float fdiv(float a, float b) { return __fdiv_rn(a, b); }

// interpolation-domain coordinate of a target value: its half bit pattern (0 for v <= 0 or NaN, 0x7BFF above
// the finite half range)
__device__ __forceinline__ float enc_coord(float v)
{
    if (!(v > 0.0f))
        return 0.0f;
    const unsigned bits = __half_as_ushort(__float2half_rn(v));
    return bits >= 0x7C00u ? 31743.0f : (float)bits;
}

__device__ __forceinline__ int unq6(int e) { return e == 0 ? 0 : (e == 63 ? 0xFFFF : (e << 10) + 512); }

// decoded value of a mode-10 channel from the unquantised endpoints and weight w
__device__ __forceinline__ float mode10_value(int ua, int ub, int w)
{
    const int yi = (ua * (64 - w) + ub * w + 32) >> 6;
    return __half2float(__ushort_as_half((unsigned short)((yi * 31) >> 6)));
}

__device__ __forceinline__ int enc_quantise(float y)
{
    const float q = rintf(fdiv(fsub(fmul(y, 64.0f / 31.0f), 512.0f), 1024.0f));
    return q < 0.0f ? 0 : (q > 63.0f ? 63 : (int)q);
}

// line fit of region r of the partition with texel mask pm (bit t set: texel t in region 1)
__device__ void fit_region(const float *y, uint32_t pm, int r, int e[2][3])
{
    float sum[3] = {0.0f, 0.0f, 0.0f};
    int n = 0;
    for (int t = 0; t < 16; ++t)
        if ((int)((pm >> t) & 1) == r) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                sum[c] = fadd(sum[c], y[3 * t + c]);
            ++n;
        }
    float m[3];
#pragma unroll
    for (int c = 0; c < 3; ++c)
        m[c] = n ? fdiv(sum[c], (float)n) : 0.0f;
    float C00 = 0.0f, C01 = 0.0f, C02 = 0.0f, C11 = 0.0f, C12 = 0.0f, C22 = 0.0f;
    for (int t = 0; t < 16; ++t)
        if ((int)((pm >> t) & 1) == r) {
            const float d0 = fsub(y[3 * t], m[0]), d1 = fsub(y[3 * t + 1], m[1]), d2 = fsub(y[3 * t + 2], m[2]);
            C00 = fadd(C00, fmul(d0, d0));
            C01 = fadd(C01, fmul(d0, d1));
            C02 = fadd(C02, fmul(d0, d2));
            C11 = fadd(C11, fmul(d1, d1));
            C12 = fadd(C12, fmul(d1, d2));
            C22 = fadd(C22, fmul(d2, d2));
        }
    const float C[3][3] = {{C00, C01, C02}, {C01, C11, C12}, {C02, C12, C22}};
    int jm = 0;
    if (C[1][1] > C[jm][jm])
        jm = 1;
    if (C[2][2] > C[jm][jm])
        jm = 2;
    float A[3], B[3];
    if (C[jm][jm] > 0.0f) {
        float a[3] = {C[0][jm], C[1][jm], C[2][jm]};
        for (int it = 0; it < 8; ++it) {
            float b[3];
#pragma unroll
            for (int i = 0; i < 3; ++i)
                b[i] = fadd(fadd(fmul(C[i][0], a[0]), fmul(C[i][1], a[1])), fmul(C[i][2], a[2]));
            float s = fabsf(b[0]);
            if (fabsf(b[1]) > s)
                s = fabsf(b[1]);
            if (fabsf(b[2]) > s)
                s = fabsf(b[2]);
            if (!(s > 0.0f))
                break;
#pragma unroll
            for (int i = 0; i < 3; ++i)
                a[i] = fdiv(b[i], s);
        }
        const float aa = fadd(fadd(fmul(a[0], a[0]), fmul(a[1], a[1])), fmul(a[2], a[2]));
        float pmin = INFINITY, pmax = -INFINITY;
        for (int t = 0; t < 16; ++t)
            if ((int)((pm >> t) & 1) == r) {
                const float d0 = fsub(y[3 * t], m[0]), d1 = fsub(y[3 * t + 1], m[1]), d2 = fsub(y[3 * t + 2], m[2]);
                const float p = fadd(fadd(fmul(d0, a[0]), fmul(d1, a[1])), fmul(d2, a[2]));
                if (p < pmin)
                    pmin = p;
                if (p > pmax)
                    pmax = p;
            }
        const float s0 = fdiv(pmin, aa), s1 = fdiv(pmax, aa);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            A[c] = fadd(m[c], fmul(s0, a[c]));
            B[c] = fadd(m[c], fmul(s1, a[c]));
        }
    } else {
#pragma unroll
        for (int c = 0; c < 3; ++c)
            A[c] = B[c] = m[c];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        e[0][c] = enc_quantise(A[c]);
        e[1][c] = enc_quantise(B[c]);
    }
}

__global__ void __launch_bounds__(32 * kEncWarps) k_encode_mode10(const float *__restrict__ texels, int stride, int res, int levels,
                                                                 int64_t nblocks, float *__restrict__ params,
                                                                 uint8_t *__restrict__ part, float *__restrict__ err)
{
    __shared__ float sv[kEncWarps][48], sy[kEncWarps][48];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * kEncWarps + warp;
    if (b >= nblocks) // warp-uniform
        return;
    // the block's level and position; texel offset of the level
    int l = 0;
    int64_t boff = 0, toff = 0;
    for (; l < levels - 1; ++l) {
        const int64_t wb = (res >> l) >> 2;
        if (b < boff + wb * wb)
            break;
        boff += wb * wb;
        toff += (int64_t)(res >> l) * (res >> l) * stride;
    }
    const int W = res >> l, wb = W >> 2;
    const int64_t bl = b - boff;
    const int by = (int)(bl / wb), bx = (int)(bl % wb);
    float *v = sv[warp], *y = sy[warp];
    for (int e = lane; e < 48; e += 32) {
        const int t = e / 3, c = e % 3;
        const float x = texels[toff + ((int64_t)(4 * by + (t >> 2)) * W + 4 * bx + (t & 3)) * stride + c];
        v[e] = x;
        y[e] = enc_coord(x);
    }
    __syncwarp();

    const int k = lane;
    const uint32_t pm = partition_mask(k);
    int e[2][2][3];
    fit_region(y, pm, 0, e[0]);
    fit_region(y, pm, 1, e[1]);
    int ua[2][3], ub[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ua[r][c] = unq6(e[r][0][c]);
            ub[r][c] = unq6(e[r][1][c]);
        }
    float total = 0.0f;
    uint32_t idx_bits = 0, idx_hi = 0; // 3 bits per texel: texels 0-7, 8-15
    for (int t = 0; t < 16; ++t) {
        const int r = (int)((pm >> t) & 1);
        float be = INFINITY;
        int bi = 0;
        for (int i = 0; i < 8; ++i) {
            const int w = weight3(i);
            float q[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float d = fsub(mode10_value(r ? ua[1][c] : ua[0][c], r ? ub[1][c] : ub[0][c], w), v[3 * t + c]);
                q[c] = fmul(d, d);
            }
            const float er = fadd(fadd(q[0], q[1]), q[2]);
            if (er < be) {
                be = er;
                bi = i;
            }
        }
        if (t < 8)
            idx_bits |= (uint32_t)bi << (3 * t);
        else
            idx_hi |= (uint32_t)bi << (3 * (t - 8));
        total = fadd(total, be);
    }
    // smallest total error over the warp; a NaN total never wins over a number, ties go to the smaller k
    float key = isnan(total) ? INFINITY : total;
    int best = k;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ok = __shfl_xor_sync(0xffffffffu, key, off);
        const int obest = __shfl_xor_sync(0xffffffffu, best, off);
        if (ok < key || (ok == key && obest < best)) {
            key = ok;
            best = obest;
        }
    }
    if (k != best)
        return;
    float *pr = params + b * 32;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pr[8 * r + c] = (float)e[r][0][c];
            pr[8 * r + 3 + c] = (float)e[r][1][c];
        }
    pr[6] = pr[7] = pr[14] = pr[15] = 0.0f;
    for (int t = 0; t < 16; ++t) {
        const int i = t < 8 ? (int)((idx_bits >> (3 * t)) & 7) : (int)((idx_hi >> (3 * (t - 8))) & 7);
        pr[16 + t] = (float)i / 7.0f;
    }
    part[b] = (uint8_t)k;
    if (err)
        err[b] = total;
}

} // namespace

cudaError_t launch_encode_mode10(const float *texels, int stride, int res, int levels, int64_t nblocks,
                                 float *params, uint8_t *part, float *err, cudaStream_t st)
{
    if (nblocks <= 0)
        return cudaSuccess;
    const int64_t grid = (nblocks + kEncWarps - 1) / kEncWarps;
    k_encode_mode10<<<(unsigned)grid, 32 * kEncWarps, 0, st>>>(texels, stride, res, levels, nblocks, params, part,
                                                              err);
    return cudaGetLastError();
}

} // namespace bcf
