// bcf_sample.cuh -- per-query feature sampling: LOD selection (Eq. 11 bias),
// texel addressing, BC6H unpack of the texels a bilinear footprint needs, and
// exact FP32 trilinear filtering (Eq. 10).
//
// The loops over textures, levels and footprint corners are kept rolled so
// that a kernel holds a single copy of the BC6H decode path; a block header
// is decoded once and reused for the footprint texels it contains.
#pragma once
#include <cuda_fp16.h>

#include "bc6h_unpack.cuh"
#include "bcf_internal.h"

namespace bcf {

// Block offset of mip level l in a chain whose level 0 is wb0 x wb0 blocks
// (wb0 a power of two): sum_{k<l} (wb0 >> k)^2 = 4 (wb0^2 - (wb0 >> l)^2) / 3.
__device__ __forceinline__ uint32_t level_offset(uint32_t wb0, int l)
{
    uint32_t wbl = wb0 >> l;
    return ((wb0 * wb0 - wbl * wbl) * 4u) / 3u;
}

__device__ __forceinline__ float sanitize(float c, int wrap)
{
    if (!isfinite(c))
        c = 0.0f;
    return wrap ? c - floorf(c) : fminf(fmaxf(c, 0.0f), 1.0f);
}

__device__ __forceinline__ int address(int i, int W, int wrap)
{
    return wrap ? (i & (W - 1)) : min(max(i, 0), W - 1);
}

// T_t(u, v, s) of one texture: bilinear on levels floor(s_t) and
// floor(s_t) + 1 (when the fraction is non-zero and the level exists),
// lerped by the fraction; s_t = clamp(s + lod_bias, 0, L - 1).
__device__ __forceinline__ float3 sample_texture(const TexDev &T, int wrap, bool sgn, float u, float v, float s)
{
    float st = (isnan(s) ? 0.0f : s) + (float)T.lod_bias;
    st = fminf(fmaxf(st, 0.0f), (float)(T.levels - 1));
    const float fl = floorf(st);
    const int l0 = (int)fl;
    const float lam = st - fl;
    const int nlev = (lam > 0.0f && l0 + 1 < T.levels) ? 2 : 1;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
#pragma unroll 1
    for (int side = 0; side < nlev; ++side) {
        const int level = l0 + side;
        const float scale = nlev == 1 ? 1.0f : (side ? lam : 1.0f - lam);
        const int W = T.res >> level;
        const int wb = W >> 2;
        const uint4 *base = T.blocks + level_offset((uint32_t)(T.res >> 2), level);
        const float x = u * (float)W - 0.5f, y = v * (float)W - 0.5f;
        const float fx0 = floorf(x), fy0 = floorf(y);
        const float fx = x - fx0, fy = y - fy0;
        const int i0 = (int)fx0, j0 = (int)fy0;
        const int ia = address(i0, W, wrap), ib = address(i0 + 1, W, wrap);
        const int ja = address(j0, W, wrap), jb = address(j0 + 1, W, wrap);
        uint32_t cur = 0xFFFFFFFFu;
        Bc6hBlock blk;
        Bc6hHeader H;
#pragma unroll 1
        for (int c = 0; c < 4; ++c) {
            const int i = (c & 1) ? ib : ia;
            const int j = (c & 2) ? jb : ja;
            const float w = ((c & 1) ? fx : 1.0f - fx) * ((c & 2) ? fy : 1.0f - fy) * scale;
            const uint32_t bidx = (uint32_t)(j >> 2) * (uint32_t)wb + (uint32_t)(i >> 2);
            if (bidx != cur) {
                blk = load_block(base + bidx);
                bc6h_header(blk, sgn, H);
                cur = bidx;
            }
            uint32_t r, g, b;
            bc6h_texel(blk, H, ((j & 3) << 2) | (i & 3), sgn, r, g, b);
            a0 = fmaf(w, __half2float(__ushort_as_half((unsigned short)r)), a0);
            a1 = fmaf(w, __half2float(__ushort_as_half((unsigned short)g)), a1);
            a2 = fmaf(w, __half2float(__ushort_as_half((unsigned short)b)), a2);
        }
    }
    return make_float3(a0, a1, a2);
}

// All features of one query written to `row` ([3 T] then the LOD input);
// `row` may be shared or global memory.
__device__ __forceinline__ void query_features(const MaterialDev &M, float u, float v, float s, float *row)
{
    const float uu = sanitize(u, M.wrap), vv = sanitize(v, M.wrap);
    const bool sgn = M.is_signed != 0;
#pragma unroll 1
    for (int t = 0; t < M.n_tex; ++t) {
        const float3 f = sample_texture(M.tex[t], M.wrap, sgn, uu, vv, s);
        row[3 * t] = f.x;
        row[3 * t + 1] = f.y;
        row[3 * t + 2] = f.z;
    }
    if (M.lod_input)
        row[3 * M.n_tex] = isnan(s) ? 0.0f : fmaxf(s, 0.0f);
}

// The same features through the texture unit (the render-time design of Sec. 5.2): hardware trilinear
// filtering of the BC6H textures at the per-texture LOD of Eq. 11.  The hardware's filter weights are low-
// precision fixed point, so these features differ from query_features by a bounded filtering error.
__device__ __forceinline__ float3 texture_trilinear_hw(const TexDev &X, unsigned long long tex, float u, float v,
                                                       float s)
{
    const float lod = fminf(fmaxf((isnan(s) ? 0.0f : s) + (float)X.lod_bias, 0.0f), (float)(X.levels - 1));
    const float4 f = tex2DLod<float4>((cudaTextureObject_t)tex, u, v, lod);
    return make_float3(f.x, f.y, f.z);
}

__device__ __forceinline__ void query_features_hw(const MaterialDev &M, const TexUnitObjs &T, float u, float v,
                                                  float s, float *row)
{
    const float uu = sanitize(u, M.wrap), vv = sanitize(v, M.wrap);
#pragma unroll 1
    for (int t = 0; t < M.n_tex; ++t) {
        const float3 f = texture_trilinear_hw(M.tex[t], T.tex[t], uu, vv, s);
        row[3 * t] = f.x;
        row[3 * t + 1] = f.y;
        row[3 * t + 2] = f.z;
    }
    if (M.lod_input)
        row[3 * M.n_tex] = isnan(s) ? 0.0f : fmaxf(s, 0.0f);
}

// The exact features with the texels decoded by the texture unit: each footprint texel is fetched with point
// filtering at its centre (the hardware BC6H decoder, bit-exact with bc6h_texel) and filtered here with the
// same FP32 operations in the same order as sample_texture, so the features are identical to it.
__device__ __forceinline__ float3 sample_texture_hwpoint(const TexDev &T, unsigned long long tex, int wrap, float u,
                                                         float v, float s)
{
    float st = (isnan(s) ? 0.0f : s) + (float)T.lod_bias;
    st = fminf(fmaxf(st, 0.0f), (float)(T.levels - 1));
    const float fl = floorf(st);
    const int l0 = (int)fl;
    const float lam = st - fl;
    const int nlev = (lam > 0.0f && l0 + 1 < T.levels) ? 2 : 1;
    // both levels' eight texels are fetched before any is used (the fetch latency is paid once)
    float fxs[2], fys[2];
    float4 c4[2][4];
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        if (side < nlev) {
            const int level = l0 + side;
            const int W = T.res >> level;
            const float x = u * (float)W - 0.5f, y = v * (float)W - 0.5f;
            const float fx0 = floorf(x), fy0 = floorf(y);
            fxs[side] = x - fx0;
            fys[side] = y - fy0;
            const int i0 = (int)fx0, j0 = (int)fy0;
            const int ia = address(i0, W, wrap), ib = address(i0 + 1, W, wrap);
            const int ja = address(j0, W, wrap), jb = address(j0 + 1, W, wrap);
            const float rw = 1.0f / (float)W; // exact: W is a power of two
#pragma unroll
            for (int c = 0; c < 4; ++c) // texel centres (i + 1/2) / W are exact in FP32
                c4[side][c] = tex2DLod<float4>((cudaTextureObject_t)tex, ((float)((c & 1) ? ib : ia) + 0.5f) * rw,
                                               ((float)((c & 2) ? jb : ja) + 0.5f) * rw, (float)level);
        }
    }
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f;
#pragma unroll
    for (int side = 0; side < 2; ++side) {
        if (side < nlev) {
            const float scale = nlev == 1 ? 1.0f : (side ? lam : 1.0f - lam);
            const float fx = fxs[side], fy = fys[side];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const float w = ((c & 1) ? fx : 1.0f - fx) * ((c & 2) ? fy : 1.0f - fy) * scale;
                a0 = fmaf(w, c4[side][c].x, a0);
                a1 = fmaf(w, c4[side][c].y, a1);
                a2 = fmaf(w, c4[side][c].z, a2);
            }
        }
    }
    return make_float3(a0, a1, a2);
}

__device__ __forceinline__ void query_features_hwpoint(const MaterialDev &M, const TexUnitObjs &T, float u, float v,
                                                       float s, float *row)
{
    const float uu = sanitize(u, M.wrap), vv = sanitize(v, M.wrap);
#pragma unroll 1
    for (int t = 0; t < M.n_tex; ++t) {
        const float3 f = sample_texture_hwpoint(M.tex[t], T.texp[t], M.wrap, uu, vv, s);
        row[3 * t] = f.x;
        row[3 * t + 1] = f.y;
        row[3 * t + 2] = f.z;
    }
    if (M.lod_input)
        row[3 * M.n_tex] = isnan(s) ? 0.0f : fmaxf(s, 0.0f);
}

} // namespace bcf
