// bcf_texunit.cu -- the GPU texture unit on BC6H data: the blocks are copied
// into CUDA arrays of 16-byte elements and viewed as BC6H textures (resource
// views with a block-compressed format).
//  * texunit_decode: every texel centre fetched with point filtering -- an
//    independent statement of the format, used to check the integer decoder
//    and the CPU oracle; not a hot path.
//  * texunit_create: a material's feature textures as mipmapped CUDA arrays
//    of the BC6H channel format with hardware trilinear filtering (the
//    render-time design of Sec. 5.2), sampled by the texture-unit decode
//    variant.
#include <cuda_fp16.h>

#include "bcf_kernels.h"

namespace bcf {

__global__ void k_texunit_fetch(cudaTextureObject_t tex, int W, int H, uint16_t *__restrict__ out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= W || y >= H)
        return;
    const float4 c = tex2D<float4>(tex, (float)x + 0.5f, (float)y + 0.5f);
    uint16_t *o = out + ((size_t)y * W + x) * 3;
    o[0] = __half_as_ushort(__float2half_rn(c.x));
    o[1] = __half_as_ushort(__float2half_rn(c.y));
    o[2] = __half_as_ushort(__float2half_rn(c.z));
}

cudaError_t texunit_decode(const void *d_blocks, int bw, int bh, int is_signed, uint16_t *d_out, cudaStream_t st)
{
    cudaArray_t arr = nullptr;
    cudaTextureObject_t tex = 0;
    cudaChannelFormatDesc cd = cudaCreateChannelDesc(32, 32, 32, 32, cudaChannelFormatKindUnsigned);
    cudaError_t e = cudaMallocArray(&arr, &cd, (size_t)bw, (size_t)bh);
    if (e != cudaSuccess) {
        set_error("cudaMallocArray: %s", cudaGetErrorString(e));
        return e;
    }
    e = cudaMemcpy2DToArrayAsync(arr, 0, 0, d_blocks, (size_t)bw * 16, (size_t)bw * 16, (size_t)bh,
                                 cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypeArray;
        rd.res.array.array = arr;
        cudaTextureDesc td = {};
        td.addressMode[0] = td.addressMode[1] = cudaAddressModeClamp;
        td.filterMode = cudaFilterModePoint;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 0;
        cudaResourceViewDesc vd = {};
        vd.format = is_signed ? cudaResViewFormatSignedBlockCompressed6H : cudaResViewFormatUnsignedBlockCompressed6H;
        vd.width = (size_t)bw * 4;
        vd.height = (size_t)bh * 4;
        vd.depth = 0;
        e = cudaCreateTextureObject(&tex, &rd, &td, &vd);
        if (e != cudaSuccess)
            set_error("cudaCreateTextureObject (BC6H view): %s", cudaGetErrorString(e));
    } else {
        set_error("cudaMemcpy2DToArrayAsync: %s", cudaGetErrorString(e));
    }
    if (e == cudaSuccess) {
        dim3 grid((bw * 4 + 127) / 128, bh * 4);
        k_texunit_fetch<<<grid, 128, 0, st>>>(tex, bw * 4, bh * 4, d_out);
        e = cudaGetLastError();
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(st);
        if (e != cudaSuccess)
            set_error("texture fetch: %s", cudaGetErrorString(e));
    }
    if (tex)
        cudaDestroyTextureObject(tex);
    if (arr)
        cudaFreeArray(arr);
    return e;
}

void texunit_destroy(TexUnitObjs &T, void **arrays, int n_tex)
{
    for (int t = 0; t < n_tex; ++t) {
        if (T.tex[t])
            cudaDestroyTextureObject((cudaTextureObject_t)T.tex[t]);
        if (T.texp[t])
            cudaDestroyTextureObject((cudaTextureObject_t)T.texp[t]);
        T.texp[t] = 0;
        if (arrays[t])
            cudaFreeMipmappedArray((cudaMipmappedArray_t)arrays[t]);
        T.tex[t] = 0;
        arrays[t] = nullptr;
    }
}

cudaError_t texunit_create(const MaterialDev &M, TexUnitObjs &T, void **arrays)
{
    for (int t = 0; t < BCF_MAX_TEX; ++t) {
        T.tex[t] = 0;
        T.texp[t] = 0;
        arrays[t] = nullptr;
    }
    // arrays of the BC6H channel format itself (texels as the extent): the texture unit filters them as floats
    const cudaChannelFormatDesc cd = cudaCreateChannelDesc(
        16, 16, 16, 0,
        M.is_signed ? cudaChannelFormatKindSignedBlockCompressed6H : cudaChannelFormatKindUnsignedBlockCompressed6H);
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < M.n_tex && e == cudaSuccess; ++t) {
        const TexDev &X = M.tex[t];
        const int wb0 = X.res / 4;
        cudaMipmappedArray_t mip = nullptr;
        e = cudaMallocMipmappedArray(&mip, &cd, make_cudaExtent((size_t)X.res, (size_t)X.res, 0), (unsigned)X.levels);
        if (e != cudaSuccess) {
            set_error("cudaMallocMipmappedArray: %s", cudaGetErrorString(e));
            break;
        }
        arrays[t] = mip;
        for (int l = 0; l < X.levels && e == cudaSuccess; ++l) {
            cudaArray_t lvl = nullptr;
            e = cudaGetMipmappedArrayLevel(&lvl, mip, (unsigned)l);
            const size_t wb = (size_t)max(wb0 >> l, 1);
            // block-compressed arrays are copied as rows of blocks: 16 bytes per block, one row per 4 texel rows
            if (e == cudaSuccess)
                e = cudaMemcpy2DToArray(lvl, 0, 0, X.blocks + X.level_off[l], wb * 16, wb * 16, wb,
                                        cudaMemcpyDeviceToDevice);
            if (e != cudaSuccess)
                set_error("texture level %d of texture %d: %s", l, t, cudaGetErrorString(e));
        }
        if (e != cudaSuccess)
            break;
        cudaResourceDesc rd = {};
        rd.resType = cudaResourceTypeMipmappedArray;
        rd.res.mipmap.mipmap = mip;
        cudaTextureDesc td = {};
        const cudaTextureAddressMode am = M.wrap ? cudaAddressModeWrap : cudaAddressModeClamp;
        td.addressMode[0] = td.addressMode[1] = am;
        td.filterMode = cudaFilterModeLinear;
        td.mipmapFilterMode = cudaFilterModeLinear;
        td.readMode = cudaReadModeElementType;
        td.normalizedCoords = 1;
        td.minMipmapLevelClamp = 0.0f;
        td.maxMipmapLevelClamp = (float)(X.levels - 1);
        cudaTextureObject_t tex = 0;
        e = cudaCreateTextureObject(&tex, &rd, &td, nullptr);
        if (e != cudaSuccess) {
            set_error("cudaCreateTextureObject (mipmapped BC6H): %s", cudaGetErrorString(e));
            break;
        }
        T.tex[t] = (unsigned long long)tex;
        // the same arrays sampled texel by texel: point filtering, point mip selection (integer LODs)
        td.filterMode = cudaFilterModePoint;
        td.mipmapFilterMode = cudaFilterModePoint;
        tex = 0;
        e = cudaCreateTextureObject(&tex, &rd, &td, nullptr);
        if (e != cudaSuccess) {
            set_error("cudaCreateTextureObject (mipmapped BC6H, point): %s", cudaGetErrorString(e));
            break;
        }
        T.texp[t] = (unsigned long long)tex;
    }
    if (e != cudaSuccess)
        texunit_destroy(T, arrays, M.n_tex);
    return e;
}

// Copy the caller's block arrays into the material's mipmapped arrays again, level by level, ordered on `st`
// (after the caller's rewrite of the blocks when issued on the same stream, before later decodes on it).
cudaError_t texunit_refresh(const MaterialDev &M, void *const *arrays, cudaStream_t st)
{
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < M.n_tex && e == cudaSuccess; ++t) {
        const TexDev &X = M.tex[t];
        const int wb0 = X.res / 4;
        for (int l = 0; l < X.levels && e == cudaSuccess; ++l) {
            cudaArray_t lvl = nullptr;
            e = cudaGetMipmappedArrayLevel(&lvl, (cudaMipmappedArray_t)arrays[t], (unsigned)l);
            const size_t wb = (size_t)max(wb0 >> l, 1);
            if (e == cudaSuccess)
                e = cudaMemcpy2DToArrayAsync(lvl, 0, 0, X.blocks + X.level_off[l], wb * 16, wb * 16, wb,
                                             cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess)
                set_error("refresh of level %d of texture %d: %s", l, t, cudaGetErrorString(e));
        }
    }
    return e;
}

// Point-fetch rate probe (measurement only): every lane fetches the 2 x 2 footprint around its own texel of one
// level, as a query's bilinear taps do, with the 32 lanes of a warp on an 8 x 4 patch of neighbouring texels
// (a warp of screen-coherent queries) and the warps' patches in row-major order over the level; each of the
// `rounds` rounds moves the footprint one texel along x.  The fetched values are summed into sink[thread] so
// that no fetch can be dropped.
__global__ void __launch_bounds__(128) k_texfetch_probe(cudaTextureObject_t tex, int W, int level, int64_t n,
                                                        int rounds, float *__restrict__ sink)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n)
        return;
    const int lane = threadIdx.x & 31;
    const int64_t patch = t >> 5;
    const int per_row = max(W / 8, 1);
    const int px = (int)((patch % per_row) * 8) + (lane & 7);
    const int py = (int)(((patch / per_row) * 4) % W) + (lane >> 3);
    const float rw = 1.0f / (float)W;
    const float lod = (float)level;
    float acc = 0.0f;
    for (int r = 0; r < rounds; ++r) {
        const float x0 = (float)((px + r) & (W - 1)) + 0.5f, x1 = (float)((px + r + 1) & (W - 1)) + 0.5f;
        const float y0 = (float)(py & (W - 1)) + 0.5f, y1 = (float)((py + 1) & (W - 1)) + 0.5f;
        const float4 a = tex2DLod<float4>(tex, x0 * rw, y0 * rw, lod);
        const float4 b = tex2DLod<float4>(tex, x1 * rw, y0 * rw, lod);
        const float4 c = tex2DLod<float4>(tex, x0 * rw, y1 * rw, lod);
        const float4 d = tex2DLod<float4>(tex, x1 * rw, y1 * rw, lod);
        acc += (a.x + b.y) + (c.z + d.x);
    }
    sink[t] = acc;
}

cudaError_t launch_texfetch_probe(unsigned long long tex, int W, int level, int64_t n, int rounds, float *sink,
                                  cudaStream_t st)
{
    if (n <= 0)
        return cudaSuccess;
    k_texfetch_probe<<<(unsigned)((n + 127) / 128), 128, 0, st>>>((cudaTextureObject_t)tex, W, level, n, rounds,
                                                                  sink);
    return cudaGetLastError();
}

} // namespace bcf
