// bcf_internal.h -- structures shared by the libbcf host code and kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bcf.h"

namespace bcf {

// One feature texture as the kernels see it.
struct TexDev {
    const uint4 *blocks;               // level 0 first, row-major blocks, mips concatenated
    int32_t res;                       // level-0 width
    int32_t log2res;
    int32_t levels;
    int32_t lod_bias;                  // log2(res) - log2(res_ref): the b_i of Eq. 11 in levels
    uint32_t level_off[BCF_MAX_LEVELS]; // block offset of each level
};

// Padded MLP geometry for the tensor-core path: K and N of every layer are
// rounded up to the MMA tile (16 for 16-bit operands, 32 for FP8 K).
struct MlpDev {
    int32_t n_layers;
    int32_t dims[BCF_MAX_LAYERS + 1];
    int32_t kpad[BCF_MAX_LAYERS];      // padded input width per layer
    int32_t npad[BCF_MAX_LAYERS];      // padded output width per layer
    int32_t precision;
    const void *weights;               // caller layout: W_l [out][in] row-major, concatenated
    const float *biases;
    float act_scale[BCF_MAX_LAYERS];
    float w_scale[BCF_MAX_LAYERS];
    float inv_act_scale[BCF_MAX_LAYERS];
    int32_t w_off[BCF_MAX_LAYERS];     // element offset of W_l in the caller layout
    int32_t b_off[BCF_MAX_LAYERS];
    int32_t smem_w_bytes;              // padded weights in shared memory (MMA operand type)
    int32_t smem_b_floats;             // padded biases
};

// Texture objects of a material's feature textures for the texture-unit decodes: mipmapped CUDA arrays of
// the BC6H format (cudaTextureObject_t values); `tex` filters trilinearly in hardware, `texp` samples single
// texels (point filtering at texel centres: the hardware's exact BC6H decode).
struct TexUnitObjs {
    unsigned long long tex[BCF_MAX_TEX];
    unsigned long long texp[BCF_MAX_TEX];
};

struct MaterialDev {
    int32_t n_tex;
    int32_t is_signed;
    int32_t wrap;
    int32_t lod_input;
    int32_t n_in;                      // 3 T + lod_input
    int32_t n_out;
    // textures with the same resolution and level count sample the same texel
    // footprints: they form one geometry group
    int32_t n_groups;
    int32_t tex_group[BCF_MAX_TEX];    // group of each texture
    int32_t group_first[BCF_MAX_TEX];  // a texture of each group (its geometry)
    TexDev tex[BCF_MAX_TEX];
    MlpDev mlp;
    int32_t mlp_engine;                // BCF_MLP_MMA_SYNC or BCF_MLP_TCGEN05 (bcf_set_mlp_engine)
};

// The current device's check word (include/bcf.h, BCF_CHECK_*), created on the first call; nullptr if that
// allocation failed.  Kernels set its bits with atomicOr; bcf_device_check reads and clears it.
unsigned *check_word();

} // namespace bcf

#ifndef BCF_MAX_SET
#define BCF_MAX_SET 256 // materials per material set
#endif

// Buffers of bcf_decode_material_host's pipeline (each holds one chunk's queries and outputs).
#ifndef BCF_PIPE_BUFS
#define BCF_PIPE_BUFS 3
#endif

struct bcf_material_s {
    bcf::MaterialDev host;   // host copy (passed by value to single-material kernels)
    bcf::MaterialDev *dev;   // device copy (batched kernels)
    int device;
    int variant;             // tensor-core decode: 0 tile-cooperative, 1 per-lane, 2 texture unit (hardware
                             // trilinear), 3 texture-unit texels with the exact FP32 filter
    bcf::TexUnitObjs hw;     // variant 2: BC6H texture objects with hardware trilinear filtering
    void *hw_arrays[BCF_MAX_TEX];
    int hw_ready;
    // bcf_decode_material_host's pipeline: upload, decode and download streams and their events, created by
    // the first such call and released with the material
    cudaStream_t pipe_streams[3];
    cudaEvent_t pipe_events[2 + 3 * BCF_PIPE_BUFS];
    int pipe_ready;
};
