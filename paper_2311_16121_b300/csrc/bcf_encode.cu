// bcf_encode.cu -- BC6H block encoders of RGB textures.
//
// k_encode_mode10: partition selection and the initial block parameters from
// free per-texel features (Sec. 5.1: the unconstrained features of a short
// first training stage are compressed with the BC6 algorithm, which fixes
// each block's partition and initialises its endpoints and indices).
// k_compress_bc6h: the same mode-10 search against a mode-11 candidate, the
// better one written as a BC6H block -- a plain texture compressor, used to
// store a material's channels directly (the material without the network).
//
// One warp per block, one lane per partition k = 0..31.  Each lane fits a
// line to each of its two regions in the format's interpolation domain (the
// binary16 bit pattern of the value): mean, 3 x 3 scatter matrix, principal
// axis by 8 power iterations started from the scatter column of the largest
// diagonal entry, segment between the smallest and largest projections.  The
// segment ends are quantised to 6-bit endpoints (inverting unquantise
// 1024 e + 512 and finish x 31/64), each texel takes the 3-bit index whose
// decoded value is closest (squared RGB error in value space), and the warp
// keeps the partition with the smallest total error (ties: smaller k).  The
// mode-11 candidate fits one line to all sixteen texels, quantises its ends
// to 10 bits (unquantise 64 e + 32) and picks 4-bit indices the same way.
// The line fit's quantised ends are not always the best codes (rounding each
// end on its own ignores the decoder's floors and the other texels), so the
// winner is refined: the 24 (mode 11: 12) moves of one endpoint code by one
// are tried in parallel, one per lane, and the best is taken while it lowers
// the error.
//
// Every floating-point quantity here decides an integer (an endpoint, an
// index, the partition, the mode), so it is computed in IEEE single
// precision with explicitly rounded operations in one fixed order -- no
// contraction into fused multiply-adds -- which makes the choice
// reproducible and independent of compiler scheduling.
#include <cuda_fp16.h>
#include <math.h>

#include "bc6h_pack.cuh"
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

// decoded UF16 value of a channel (modes 10 and 11) from the unquantised endpoints and weight w
__device__ __forceinline__ float texel_value(int ua, int ub, int w)
{
    const int yi = (ua * (64 - w) + ub * w + 32) >> 6;
    return __half2float(__ushort_as_half((unsigned short)((yi * 31) >> 6)));
}

__device__ __forceinline__ int enc_quantise6(float y)
{
    const float q = rintf(fdiv(fsub(fmul(y, 64.0f / 31.0f), 512.0f), 1024.0f));
    return q < 0.0f ? 0 : (q > 63.0f ? 63 : (int)q);
}

// 10-bit endpoints (mode 11): unquantise 64 e + 32, finish x 31/64
__device__ __forceinline__ int unq10(int e) { return e == 0 ? 0 : (e == 1023 ? 0xFFFF : (e << 6) + 32); }

__device__ __forceinline__ int enc_quantise10(float y)
{
    const float q = rintf(fdiv(fsub(fmul(y, 64.0f / 31.0f), 32.0f), 64.0f));
    return q < 0.0f ? 0 : (q > 1023.0f ? 1023 : (int)q);
}

// Line fit of region r of the partition with texel mask pm (bit t set: texel t in region 1; pm = 0, r = 0: all
// sixteen texels): the segment [A, B] between the extreme projections on the principal axis.
__device__ void fit_segment(const float *y, uint32_t pm, int r, float A[3], float B[3])
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
}

// squared RGB error (value space) of texel target v[0..2] against the value of weight w between ua and ub
__device__ __forceinline__ float texel_error(const int ua[3], const int ub[3], int w, const float *v)
{
    float q[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float d = fsub(texel_value(ua[c], ub[c], w), v[c]);
        q[c] = fmul(d, d);
    }
    return fadd(fadd(q[0], q[1]), q[2]);
}

// Indices and total squared error of the mode-10 segments e[region][end][c] for the partition with texel mask
// pm: each texel the best of the 8 indices (ties: the smaller), texels 0-7 in idx_lo, 8-15 in idx_hi, the
// total summed in texel order.
__device__ float mode10_assign(const float *v, uint32_t pm, const int e[2][2][3], uint32_t &idx_lo,
                               uint32_t &idx_hi)
{
    int ua[2][3], ub[2][3];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ua[r][c] = unq6(e[r][0][c]);
            ub[r][c] = unq6(e[r][1][c]);
        }
    float total = 0.0f;
    idx_lo = idx_hi = 0;
    for (int t = 0; t < 16; ++t) {
        const int r = (int)((pm >> t) & 1);
        float be = INFINITY;
        int bi = 0;
        for (int i = 0; i < 8; ++i) {
            const float er = texel_error(r ? ua[1] : ua[0], r ? ub[1] : ub[0], weight3(i), v + 3 * t);
            if (er < be) {
                be = er;
                bi = i;
            }
        }
        if (t < 8)
            idx_lo |= (uint32_t)bi << (3 * t);
        else
            idx_hi |= (uint32_t)bi << (3 * (t - 8));
        total = fadd(total, be);
    }
    return total;
}

// Mode-10 candidate of partition k (one lane): the line fit of both regions quantised to 6-bit endpoints
// e[region][end][c], then mode10_assign.
__device__ float mode10_candidate(const float *v, const float *y, int k, int e[2][2][3], uint32_t &idx_lo,
                                  uint32_t &idx_hi)
{
    const uint32_t pm = partition_mask(k);
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        float A[3], B[3];
        fit_segment(y, pm, r, A, B);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            e[r][0][c] = enc_quantise6(A[c]);
            e[r][1][c] = enc_quantise6(B[c]);
        }
    }
    return mode10_assign(v, pm, e, idx_lo, idx_hi);
}

// smallest key over the warp (a NaN total never wins over a number; ties go to the smaller k)
__device__ __forceinline__ int warp_best_partition(float total, int k, float &key)
{
    key = isnan(total) ? INFINITY : total;
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
    return best;
}

// Smallest key over the warp with ties to the smaller lane: the winning lane.
__device__ __forceinline__ int warp_argmin(float key, float &best)
{
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const float ok = __shfl_xor_sync(0xffffffffu, key, off);
        const int ol = __shfl_xor_sync(0xffffffffu, lane, off);
        if (ok < key || (ok == key && ol < lane)) {
            key = ok;
            lane = ol;
        }
    }
    best = key;
    return lane;
}

constexpr int kRefineRounds = 16;

// Improve the segments e (the same on every lane) of the partition with mask pm whose total error is `cur`:
// in each round lane j < 2 n_codes moves endpoint code j / 2 down (j even) or up (j odd) by one, re-assigns the
// indices and sums the error; the best move is taken while it lowers the error (ties: the lower lane), for at
// most kRefineRounds rounds.  Every lane returns the final segments and error.  Codes stay in [0, top].
template <int NE, class Assign>
__device__ float refine_codes(int *e, float cur, int top, Assign assign)
{
    const int lane = threadIdx.x & 31;
    for (int round = 0; round < kRefineRounds; ++round) {
        const int j = lane >> 1, dir = (lane & 1) ? 1 : -1;
        float key = INFINITY;
        if (lane < 2 * NE) {
            int trial[NE];
#pragma unroll
            for (int i = 0; i < NE; ++i)
                trial[i] = e[i];
            const int nv = trial[j] + dir;
            if (nv >= 0 && nv <= top) {
                trial[j] = nv;
                const float tot = assign(trial);
                key = isnan(tot) ? INFINITY : tot;
            }
        }
        float best;
        const int win = warp_argmin(key, best);
        if (!(best < cur))
            break; // warp-uniform: every lane holds the same best and cur
        const int wj = win >> 1, wd = (win & 1) ? 1 : -1;
        e[wj] += wd;
        cur = best;
    }
    return cur;
}

__device__ __forceinline__ int mode10_index(uint32_t idx_lo, uint32_t idx_hi, int t)
{
    return t < 8 ? (int)((idx_lo >> (3 * t)) & 7) : (int)((idx_hi >> (3 * (t - 8))) & 7);
}

// The winning partition's segments broadcast from lane `best` (whose total error is `total`) and refined by
// refine_codes; every lane returns the refined segments in e, their indices and total error.
__device__ float refine_mode10(const float *v, int best, int e[2][2][3], float total, uint32_t &idx_lo,
                               uint32_t &idx_hi)
{
    int flat[12];
#pragma unroll
    for (int i = 0; i < 12; ++i)
        flat[i] = __shfl_sync(0xffffffffu, e[i / 6][(i / 3) & 1][i % 3], best);
    const uint32_t pm = partition_mask(best);
    const auto assign = [&](const int *f) {
        int t[2][2][3];
        uint32_t lo, hi;
#pragma unroll
        for (int i = 0; i < 12; ++i)
            t[i / 6][(i / 3) & 1][i % 3] = f[i];
        return mode10_assign(v, pm, t, lo, hi);
    };
    refine_codes<12>(flat, total, 63, assign);
#pragma unroll
    for (int i = 0; i < 12; ++i)
        e[i / 6][(i / 3) & 1][i % 3] = flat[i];
    return mode10_assign(v, pm, e, idx_lo, idx_hi);
}

// Indices (best of 16, ties: the smaller) and total squared error, in texel order, of the mode-11 segment
// e[end][c] over all sixteen texels.
__device__ float mode11_assign(const float *v, const int e[2][3], int idx[16])
{
    int ua[3], ub[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        ua[c] = unq10(e[0][c]);
        ub[c] = unq10(e[1][c]);
    }
    float total = 0.0f;
    for (int t = 0; t < 16; ++t) {
        float be = INFINITY;
        int bi = 0;
        for (int i = 0; i < 16; ++i) {
            const float er = texel_error(ua, ub, weight4(i), v + 3 * t);
            if (er < be) {
                be = er;
                bi = i;
            }
        }
        idx[t] = bi;
        total = fadd(total, be);
    }
    return total;
}

// The block b of a mipmapped texture: its 48 targets (v) and their interpolation-domain coordinates (y) in the
// warp's shared rows.
__device__ void load_block(const float *__restrict__ texels, int stride, int res, int levels, int64_t b, float *v,
                           float *y, int lane)
{
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
    for (int e = lane; e < 48; e += 32) {
        const int t = e / 3, c = e % 3;
        const float x = texels[toff + ((int64_t)(4 * by + (t >> 2)) * W + 4 * bx + (t & 3)) * stride + c];
        v[e] = x;
        y[e] = enc_coord(x);
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32 * kEncWarps) k_encode_mode10(const float *__restrict__ texels, int stride, int res,
                                                                 int levels, int64_t nblocks,
                                                                 float *__restrict__ params,
                                                                 uint8_t *__restrict__ part, float *__restrict__ err)
{
    __shared__ float sv[kEncWarps][48], sy[kEncWarps][48];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * kEncWarps + warp;
    if (b >= nblocks) // warp-uniform
        return;
    float *v = sv[warp], *y = sy[warp];
    load_block(texels, stride, res, levels, b, v, y, lane);
    const int k = lane;
    int e[2][2][3];
    uint32_t idx_lo, idx_hi;
    float total = mode10_candidate(v, y, k, e, idx_lo, idx_hi);
    float key;
    const int best = warp_best_partition(total, k, key);
    total = refine_mode10(v, best, e, __shfl_sync(0xffffffffu, total, best), idx_lo, idx_hi);
    if (lane != 0)
        return;
    const int kb = best;
    float *pr = params + b * 32;
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            pr[8 * r + c] = (float)e[r][0][c];
            pr[8 * r + 3 + c] = (float)e[r][1][c];
        }
    pr[6] = pr[7] = pr[14] = pr[15] = 0.0f;
    for (int t = 0; t < 16; ++t)
        pr[16 + t] = (float)mode10_index(idx_lo, idx_hi, t) / 7.0f;
    part[b] = (uint8_t)kb;
    if (err)
        err[b] = total;
}

// Two-mode compressor: the mode-10 encoding above against a mode-11 encoding (one region over all sixteen
// texels, 10-bit endpoints, 4-bit indices); the smaller total error is written as a BC6H block (ties and NaN
// totals: mode 10).  The mode-11 line fit runs on every lane alike; its index search takes texel lane & 15.
__global__ void __launch_bounds__(32 * kEncWarps) k_compress_bc6h(const float *__restrict__ texels, int stride, int res,
                                                                 int levels, int64_t nblocks, uint4 *__restrict__ out,
                                                                 float *__restrict__ err, uint8_t *__restrict__ modes)
{
    __shared__ float sv[kEncWarps][48], sy[kEncWarps][48];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = (int64_t)blockIdx.x * kEncWarps + warp;
    if (b >= nblocks) // warp-uniform
        return;
    float *v = sv[warp], *y = sy[warp];
    load_block(texels, stride, res, levels, b, v, y, lane);
    const int k = lane;
    int e[2][2][3];
    uint32_t idx_lo, idx_hi;
    float total10 = mode10_candidate(v, y, k, e, idx_lo, idx_hi);
    float key10;
    const int best = warp_best_partition(total10, k, key10);
    total10 = refine_mode10(v, best, e, __shfl_sync(0xffffffffu, total10, best), idx_lo, idx_hi);
    key10 = isnan(total10) ? INFINITY : total10;

    float A[3], B[3];
    fit_segment(y, 0u, 0, A, B);
    int e11[2][3], ua[3], ub[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        e11[0][c] = enc_quantise10(A[c]);
        e11[1][c] = enc_quantise10(B[c]);
        ua[c] = unq10(e11[0][c]);
        ub[c] = unq10(e11[1][c]);
    }
    const int tl = lane & 15;
    float be = INFINITY;
    for (int i = 0; i < 16; ++i) {
        const float er = texel_error(ua, ub, weight4(i), v + 3 * tl);
        if (er < be)
            be = er;
    }
    float total11 = 0.0f;
#pragma unroll
    for (int t = 0; t < 16; ++t) // texel order, as a sequential sum would take it
        total11 = fadd(total11, __shfl_sync(0xffffffffu, be, t));
    int flat11[6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
        flat11[i] = e11[i / 3][i % 3];
    const auto assign11 = [&](const int *f) {
        int t[2][3], idx[16];
#pragma unroll
        for (int i = 0; i < 6; ++i)
            t[i / 3][i % 3] = f[i];
        return mode11_assign(v, t, idx);
    };
    refine_codes<6>(flat11, total11, 1023, assign11);
    if (lane != 0)
        return;
#pragma unroll
    for (int i = 0; i < 6; ++i)
        e11[i / 3][i % 3] = flat11[i];
    int idx11[16];
    total11 = mode11_assign(v, e11, idx11);
    const float key11 = isnan(total11) ? INFINITY : total11;
    if (key11 < key10) {
        out[b] = bc6h_pack_mode11(e11, idx11);
        if (err)
            err[b] = total11;
        if (modes)
            modes[b] = 11;
        return;
    }
    int q[4][3], idx[16];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            q[2 * r][c] = e[r][0][c];
            q[2 * r + 1][c] = e[r][1][c];
        }
#pragma unroll
    for (int t = 0; t < 16; ++t)
        idx[t] = mode10_index(idx_lo, idx_hi, t);
    out[b] = bc6h_pack_mode10(q, idx, best);
    if (err)
        err[b] = total10;
    if (modes)
        modes[b] = 10;
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

namespace bcf {

cudaError_t launch_compress_bc6h(const float *texels, int stride, int res, int levels, int64_t nblocks, void *out,
                                 float *err, uint8_t *modes, cudaStream_t st)
{
    if (nblocks <= 0)
        return cudaSuccess;
    const int64_t grid = (nblocks + kEncWarps - 1) / kEncWarps;
    k_compress_bc6h<<<(unsigned)grid, 32 * kEncWarps, 0, st>>>(texels, stride, res, levels, nblocks, (uint4 *)out,
                                                              err, modes);
    return cudaGetLastError();
}

} // namespace bcf
