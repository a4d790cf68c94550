// bcf_texunit.cu -- BC6H decode by the GPU texture unit: the blocks are
// copied into a CUDA array of 16-byte elements and viewed as a BC6H texture
// (a resource view with a block-compressed format), then every texel centre
// is fetched with point filtering.  An independent statement of the format,
// used to check the integer decoder and the CPU oracle; not a hot path.
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

} // namespace bcf
