// bcf_train_sample.cuh -- per-query pieces of the training step shared by the
// training kernels: the Philox4x32-10 batch draw, the straight-through mode-10
// texel (Sec. 4.2, Eq. 7-9), the trilinear taps over the block parameters
// (Eq. 10, Eq. 11 bias), the Catmull-Rom reference sample, and vector atomics.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "bc6h_unpack.cuh"
#include "bcf_train.h"

namespace bcf {

enum { kModeForward = 0, kModeBackward = 1, kModeStep = 2 };

// ------------------------------------------------------------ Philox4x32-10

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = lo1;
        c[2] = n2;
        c[3] = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

// --------------------------------------------------- emulated BC6 mode 10

// One texel of the block-based features: value (half reinterpretation of the
// exact integer decode of the rounded parameters, Eq. 9) and the partials of
// the relaxed pipeline at that point.
struct SteTexel {
    float v[3];
    float dea[3], deb[3], dx[3];
    int region;
    int ina[3], inb[3], inx;
};

__device__ __forceinline__ int unq6(float e)
{
    const int q = (int)rintf(fminf(fmaxf(e, 0.0f), 63.0f));
    return q == 0 ? 0 : (q == 63 ? 0xFFFF : q * 1024 + 512);
}

// The parameters one texel reads: its region's endpoints (e_a, e_b) and its index coordinate x.
struct TexelParams {
    float4 a; // e_a RGB, e_b R
    float2 b; // e_b G, B
    float x;
    int region;
};

// Partition id of block b, read as id & 31 (an id above 31 sets the partition check bit in the optimiser and the
// export, which see every block once; a branch here, per texel read, cost 6% of a training step).
__device__ __forceinline__ int read_partition(const TrainTexDev &T, int64_t b) { return T.part[b] & 31; }

__device__ __forceinline__ void load_texel(const float *p, int k, int t, TexelParams &P)
{
    P.region = (int)((partition_mask(k) >> t) & 1);
    P.a = *reinterpret_cast<const float4 *>(p + 8 * P.region);
    P.b = *reinterpret_cast<const float2 *>(p + 8 * P.region + 4);
    P.x = p[16 + t];
}

// SF16 unquantisation of a 6-bit two's complement code (sign carried, saturating at |e| >= 31)
__device__ __forceinline__ int unq6s(int q)
{
    const int m = q < 0 ? -q : q;
    const int u = m == 0 ? 0 : (m >= 31 ? 0x7FFF : m * 1024 + 512);
    return q < 0 ? -u : u;
}

// Eq. 9 on a real coordinate (sign carried): 2^(h - 14) (|y| / 1024 - h), h = max(floor((|y| - 1) / 1024) - 1, 0);
// its slope 2^(h - 24) through `slope`
__device__ __forceinline__ float eq9_real(float y, float &slope)
{
    const float a = fabsf(y);
    const int h = max((int)floorf((a - 1.0f) * (1.0f / 1024.0f)) - 1, 0);
    slope = ldexpf(1.0f, h - 24);
    const float w = ldexpf(a * (1.0f / 1024.0f) - (float)h, h - 14);
    return y < 0.0f ? -w : w;
}

// The emulated texel (Sec. 4.2) for the four variants EMU = signed (bit 0) | literal (bit 1):
//  exact:   the format's integer steps on the rounded codes (UF16: unquantise 1024 e + 512 with 0 and 63
//           special, >> 6 interpolation, x 31/64; SF16: sign-magnitude, saturating, x 31/32), the result read
//           as a half (Eq. 9 on the integer), so the value is the decode of the exported block;
//  literal: Eq. 7-8 as printed on the rounded codes ((a 2^16 e + 2^15) / 2^6, real interpolation), Eq. 9 on
//           the real result.
// Partials: the relaxed pipeline's (a 1024 per endpoint unit times the interpolation weight, the index
// coordinate through w / 64, the slope of Eq. 9) at the forward values.
template <int EMU>
__device__ __forceinline__ void ste_from_v(const TexelParams &P, SteTexel &o)
{
    constexpr bool SGN = (EMU & 1) != 0, LIT = (EMU & 2) != 0;
    constexpr float lo = SGN ? -32.0f : 0.0f, hi = SGN ? 31.0f : 63.0f;
    o.region = P.region;
    const float ea[3] = {P.a.x, P.a.y, P.a.z}, eb[3] = {P.a.w, P.b.x, P.b.y};
    const float x = P.x;
    o.inx = x >= 0.0f && x <= 1.0f;
    const int w = weight3((int)rintf(7.0f * fminf(fmaxf(x, 0.0f), 1.0f)));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        o.ina[c] = ea[c] >= lo && ea[c] <= hi;
        o.inb[c] = eb[c] >= lo && eb[c] <= hi;
        const int qa = (int)rintf(fminf(fmaxf(ea[c], lo), hi)), qb = (int)rintf(fminf(fmaxf(eb[c], lo), hi));
        float slope, span;
        if (!LIT) {
            const int ua = SGN ? unq6s(qa) : (qa == 0 ? 0 : (qa == 63 ? 0xFFFF : qa * 1024 + 512));
            const int ub = SGN ? unq6s(qb) : (qb == 0 ? 0 : (qb == 63 ? 0xFFFF : qb * 1024 + 512));
            const int yi = (64 * ua + 32 + (ub - ua) * w) >> 6; // arithmetic shift: floor for SF16 too
            const bool neg = SGN && yi < 0;
            const int mag = SGN ? (((neg ? -yi : yi) * 31) >> 5) : ((yi * 31) >> 6);
            const float v = __half2float(__ushort_as_half((unsigned short)mag));
            o.v[c] = neg && mag ? -v : v;
            // slope of Eq. 9 at the integer magnitude, times a
            const int h = max(((mag - 1) >> 10) - 1, 0);
            slope = ldexpf(31.0f, h - (SGN ? 29 : 30));
            span = (float)(ub - ua);
        } else {
            constexpr float a = SGN ? 31.0f / 32.0f : 31.0f / 64.0f;
            const float ua = a * 1024.0f * (float)qa + 512.0f, ub = a * 1024.0f * (float)qb + 512.0f;
            const float y = ua + ((float)w * (1.0f / 64.0f)) * (ub - ua);
            float s9;
            o.v[c] = eq9_real(y, s9);
            slope = s9 * a;
            span = (ub - ua) * (1.0f / a);
        }
        o.dea[c] = slope * (float)((64 - w) * 16);
        o.deb[c] = slope * (float)(w * 16);
        o.dx[c] = slope * span;
    }
}

__device__ __forceinline__ void ste_from(const TexelParams &P, SteTexel &o) { ste_from_v<0>(P, o); }

__device__ __forceinline__ void ste_texel(const float *p, int k, int t, SteTexel &o)
{
    TexelParams P;
    load_texel(p, k, t, P);
    ste_from(P, o);
}

// compile-time variant
template <int EMU>
__device__ __forceinline__ void ste_texel_e(const float *p, int k, int t, SteTexel &o)
{
    TexelParams P;
    load_texel(p, k, t, P);
    ste_from_v<EMU>(P, o);
}

// Fire-and-forget vector reductions into the gradient arrays.  The kernels never read a gradient they add
// to, so the reductions carry no memory clobber: later parameter loads may be issued ahead of them.
__device__ __forceinline__ void red_add_v4(float *p, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(a), "f"(b), "f"(c), "f"(d));
}
__device__ __forceinline__ void red_add_v2(float *p, float a, float b)
{
    asm volatile("red.global.add.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(a), "f"(b));
}

// Trilinear taps of texture T at (u, v, s): per side (level floor(s_t) and
// the next, weights 1 - lambda and lambda) the 2 x 2 bilinear footprint.
struct Tap {
    int64_t block;
    int texel;
    float weight;
};

// The parameters of a 2x2 footprint's four taps (0: (i, j), 1: (i+1, j), 2: (i, j+1), 3: (i+1, j+1)).  Taps in
// one block share its partition read, and taps in one block and region share the endpoint loads; the loads
// are predicated off lane by lane, which saves L1 wavefronts in the L1-bound training kernel (most footprints
// lie in one or two blocks; measured 1.3% of a step).  Every texel's index x is loaded on its own.
__device__ __forceinline__ void load_footprint(const TrainTexDev &T, const Tap (&tp)[4], TexelParams (&P)[4])
{
    const bool s10 = tp[1].block == tp[0].block, s20 = tp[2].block == tp[0].block;
    const bool s32 = tp[3].block == tp[2].block, s31 = tp[3].block == tp[1].block;
    int k[4];
    k[0] = read_partition(T, tp[0].block);
    k[1] = k[0];
    if (!s10)
        k[1] = read_partition(T, tp[1].block);
    k[2] = k[0];
    if (!s20)
        k[2] = read_partition(T, tp[2].block);
    k[3] = s32 ? k[2] : k[1];
    if (!s32 && !s31)
        k[3] = read_partition(T, tp[3].block);
    const float *p[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        p[c] = T.params + tp[c].block * 32;
        P[c].region = (int)((partition_mask(k[c]) >> tp[c].texel) & 1);
        P[c].x = p[c][16 + tp[c].texel];
    }
    P[0].a = *reinterpret_cast<const float4 *>(p[0] + 8 * P[0].region);
    P[0].b = *reinterpret_cast<const float2 *>(p[0] + 8 * P[0].region + 4);
    const bool e10 = s10 && P[1].region == P[0].region, e20 = s20 && P[2].region == P[0].region;
    const bool e32 = s32 && P[3].region == P[2].region, e31 = s31 && P[3].region == P[1].region;
    P[1].a = P[0].a;
    P[1].b = P[0].b;
    if (!e10) {
        P[1].a = *reinterpret_cast<const float4 *>(p[1] + 8 * P[1].region);
        P[1].b = *reinterpret_cast<const float2 *>(p[1] + 8 * P[1].region + 4);
    }
    P[2].a = P[0].a;
    P[2].b = P[0].b;
    if (!e20) {
        P[2].a = *reinterpret_cast<const float4 *>(p[2] + 8 * P[2].region);
        P[2].b = *reinterpret_cast<const float2 *>(p[2] + 8 * P[2].region + 4);
    }
    P[3].a = e32 ? P[2].a : P[1].a;
    P[3].b = e32 ? P[2].b : P[1].b;
    if (!e32 && !e31) {
        P[3].a = *reinterpret_cast<const float4 *>(p[3] + 8 * P[3].region);
        P[3].b = *reinterpret_cast<const float2 *>(p[3] + 8 * P[3].region + 4);
    }
}

// The trilinear taps grouped by side: f(taps[4], params[4]) once per side with a non-zero weight.  The
// partition bytes and then the parameter records of a side's four taps are loaded together (two memory
// latencies per side).
template <class F>
__device__ __forceinline__ void for_each_side(const TrainTexDev &T, float u, float v, float s, F f)
{
    float st = (isnan(s) ? 0.0f : s) + (float)T.lod_bias;
    st = fminf(fmaxf(st, 0.0f), (float)(T.levels - 1));
    const float fl = floorf(st);
    const int l0 = (int)fl;
    const int l1 = min(l0 + 1, T.levels - 1);
    const float lam = st - fl;
#pragma unroll 1 // one copy of the side body (instruction-fetch bound kernels)
    for (int side = 0; side < 2; ++side) {
        const int level = side ? l1 : l0;
        const float lw = side ? lam : 1.0f - lam;
        if (lw == 0.0f)
            continue;
        const int W = T.res >> level, wb = W >> 2;
        const int64_t lbase = (int64_t)((((uint32_t)(T.res >> 2) * (uint32_t)(T.res >> 2)) -
                                         ((uint32_t)wb * (uint32_t)wb)) * 4u / 3u);
        const float x = u * (float)W - 0.5f, y = v * (float)W - 0.5f;
        const float fx0 = floorf(x), fy0 = floorf(y);
        const float fx = x - fx0, fy = y - fy0;
        const int i0 = (int)fx0, j0 = (int)fy0;
        Tap tp[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = (i0 + (c & 1)) & (W - 1), j = (j0 + (c >> 1)) & (W - 1);
            tp[c].block = lbase + (int64_t)(j >> 2) * wb + (i >> 2);
            tp[c].texel = ((j & 3) << 2) | (i & 3);
            tp[c].weight = lw * ((c & 1) ? fx : 1.0f - fx) * ((c >> 1) ? fy : 1.0f - fy);
        }
        TexelParams P[4];
        load_footprint(T, tp, P);
        f(tp, P);
    }
}

// Unconstrained features ([texels][4], levels concatenated): per side with a non-zero weight,
// f(texel indices[4], tap weights[4], texel values[4]); the values are loaded only when LOAD is set.
template <bool LOAD, class F>
__device__ __forceinline__ void for_each_side_free(const TrainTexDev &T, float u, float v, float s, F f)
{
    float st = (isnan(s) ? 0.0f : s) + (float)T.lod_bias;
    st = fminf(fmaxf(st, 0.0f), (float)(T.levels - 1));
    const float fl = floorf(st);
    const int l0 = (int)fl;
    const int l1 = min(l0 + 1, T.levels - 1);
    const float lam = st - fl;
#pragma unroll 1
    for (int side = 0; side < 2; ++side) {
        const int level = side ? l1 : l0;
        const float lw = side ? lam : 1.0f - lam;
        if (lw == 0.0f)
            continue;
        const int W = T.res >> level;
        const int64_t lbase = (int64_t)(((uint64_t)T.res * (uint64_t)T.res - (uint64_t)W * (uint64_t)W) * 4u / 3u);
        const float x = u * (float)W - 0.5f, y = v * (float)W - 0.5f;
        const float fx0 = floorf(x), fy0 = floorf(y);
        const float fx = x - fx0, fy = y - fy0;
        const int i0 = (int)fx0, j0 = (int)fy0;
        int64_t idx[4];
        float wt[4];
        float4 val[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int i = (i0 + (c & 1)) & (W - 1), j = (j0 + (c >> 1)) & (W - 1);
            idx[c] = lbase + (int64_t)j * W + i;
            wt[c] = lw * ((c & 1) ? fx : 1.0f - fx) * ((c >> 1) ? fy : 1.0f - fy);
        }
        if (LOAD) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                val[c] = *reinterpret_cast<const float4 *>(T.params + idx[c] * 4);
        }
        f(idx, wt, val);
    }
}

// ----------------------------------------------------- reference material

__device__ __forceinline__ void catmull_rom(float f, float w[4])
{
    const float f2 = f * f, f3 = f2 * f;
    w[0] = 0.5f * (-f3 + 2.0f * f2 - f);
    w[1] = 0.5f * (3.0f * f3 - 5.0f * f2 + 2.0f);
    w[2] = 0.5f * (-3.0f * f3 + 4.0f * f2 + f);
    w[3] = 0.5f * (f3 - f2);
}

__device__ __forceinline__ void target_level(const TrainDev &D, int level, float u, float v, float scale, float out[9])
{
    const int W = D.tres >> level;
    int64_t base = 0;
    for (int l = 0; l < level; ++l)
        base += (int64_t)(D.tres >> l) * (D.tres >> l);
    const float x = u * (float)W - 0.5f, y = v * (float)W - 0.5f;
    const float fx0 = floorf(x), fy0 = floorf(y);
    float wx[4], wy[4];
    catmull_rom(x - fx0, wx);
    catmull_rom(y - fy0, wy);
    const int i0 = (int)fx0, j0 = (int)fy0;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int j = (j0 - 1 + b) & (W - 1);
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int i = (i0 - 1 + a) & (W - 1);
            const int64_t idx = base + (int64_t)j * W + i;
            const float wgt = wx[a] * wy[b] * scale;
            const uint4 c8 = __ldg(reinterpret_cast<const uint4 *>(D.t8) + idx);
            const uint32_t w4[4] = {c8.x, c8.y, c8.z, c8.w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w4[q]));
                out[2 * q] = fmaf(wgt, f.x, out[2 * q]);
                out[2 * q + 1] = fmaf(wgt, f.y, out[2 * q + 1]);
            }
            out[8] = fmaf(wgt, __half2float(__ushort_as_half(__ldg(D.t1 + idx))), out[8]);
        }
    }
}

__device__ __forceinline__ void target_sample(const TrainDev &D, float u, float v, float s, float out[9])
{
    float sq = isnan(s) ? 0.0f : s;
    sq = fminf(fmaxf(sq, 0.0f), (float)(D.tlevels - 1));
    const float fl = floorf(sq);
    const int l0 = (int)fl;
    const int l1 = min(l0 + 1, D.tlevels - 1);
    const float lam = sq - fl;
#pragma unroll
    for (int c = 0; c < 9; ++c)
        out[c] = 0.0f;
    const int nside = (l1 != l0 && lam > 0.0f) ? 2 : 1;
#pragma unroll 1 // one copy of the 16-tap body: the kernels that inline it are instruction-fetch bound
    for (int side = 0; side < nside; ++side)
        target_level(D, side ? l1 : l0, u, v, nside == 1 ? 1.0f : (side ? lam : 1.0f - lam), out);
}

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// One batch draw (u, v, s) of query q at the given step: Philox4x32-10 with the
// counter (q, step, q >> 32) and the seed as key; 24-bit uniforms.
__device__ __forceinline__ void draw_query(int64_t q, uint32_t seed_lo, uint32_t seed_hi, uint32_t step_lo,
                                           uint32_t step_hi, float s_max, float &u, float &v, float &s)
{
    uint32_t c[4] = {(uint32_t)q, step_lo, step_hi, (uint32_t)((uint64_t)q >> 32)};
    philox4x32_10(c, seed_lo, seed_hi);
    u = (float)(c[0] >> 8) * 0x1p-24f;
    v = (float)(c[1] >> 8) * 0x1p-24f;
    s = ((float)(c[2] >> 8) * 0x1p-24f) * s_max;
}

// The paper's batch form (Sec. 5.1): query q of a grid x grid batch at ((i + o_u) / grid, (j + o_v) / grid),
// i = q mod grid, j = q / grid, with one offset and one s per step from the Philox counter
// (2^32 - 1, step, 2^32 - 1), which no per-query draw uses.
__device__ __forceinline__ void draw_query_grid(int64_t q, int grid, uint32_t seed_lo, uint32_t seed_hi,
                                                uint32_t step_lo, uint32_t step_hi, float s_max, float &u, float &v,
                                                float &s)
{
    uint32_t c[4] = {0xFFFFFFFFu, step_lo, step_hi, 0xFFFFFFFFu};
    philox4x32_10(c, seed_lo, seed_hi);
    const float ou = (float)(c[0] >> 8) * 0x1p-24f, ov = (float)(c[1] >> 8) * 0x1p-24f;
    const int i = (int)(q % grid), j = (int)(q / grid);
    const float inv = 1.0f / (float)grid;
    u = __fmul_rn(__fadd_rn((float)i, ou), inv);
    v = __fmul_rn(__fadd_rn((float)j, ov), inv);
    s = ((float)(c[2] >> 8) * 0x1p-24f) * s_max;
}

} // namespace bcf
