// bcf_kernels.h -- launchers of the libbcf kernels (internal, C++).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "bcf_internal.h"

namespace bcf {

cudaError_t launch_encode_mode10(const float *texels, int stride, int res, int levels, int64_t nblocks,
                                 float *params, uint8_t *part, float *err, cudaStream_t st);
cudaError_t launch_compress_bc6h(const float *texels, int stride, int res, int levels, int64_t nblocks, void *out,
                                 float *err, uint8_t *modes, cudaStream_t st);
cudaError_t launch_decode_fp32_texunit(const MaterialDev &M, const TexUnitObjs &T, const float *u, const float *v,
                                       const float *s, int64_t n, void *out, int out_fp16, cudaStream_t st);
bool set_tex_supported(const MaterialDev &M0);
cudaError_t launch_decode_texunit(const MaterialDev &M, const TexUnitObjs &T, int exact_filter, const float *u,
                                  const float *v, const float *s, int64_t n, void *out, int out_fp16, cudaStream_t st);
cudaError_t texunit_create(const MaterialDev &M, TexUnitObjs &T, void **arrays);
cudaError_t launch_texfetch_probe(unsigned long long tex, int W, int level, int64_t n, int rounds, float *sink,
                                  cudaStream_t st);
void texunit_destroy(TexUnitObjs &T, void **arrays, int n_tex);
cudaError_t texunit_refresh(const MaterialDev &M, void *const *arrays, cudaStream_t st);
cudaError_t launch_unpack_image(const void *blocks, int bw, int bh, int is_signed, uint16_t *out, cudaStream_t st);
cudaError_t launch_sample_features(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                                   float *feat, cudaStream_t st);
cudaError_t launch_decode_fp32(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                               void *out, int out_fp16, cudaStream_t st);
cudaError_t launch_decode_mma(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                              void *out, int out_fp16, cudaStream_t st);
int64_t decode_mma_smem_bytes(const MlpDev &P);
cudaError_t launch_decode_tiled(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                                void *out, int out_fp16, cudaStream_t st);
int64_t decode_tiled_smem_bytes(const MlpDev &P);

// Launch configuration of a material-set decode (picked by the autotuner).
struct SetConfig {
    int cap;          // shared-memory block arena (256 or 320 blocks; the software set kernel)
    int ctas_per_sm;  // persistent CTAs per SM (capped by occupancy)
    int chunk;        // consecutive tiles taken per work-counter grab
};
cudaError_t launch_decode_set_tex(const MaterialDev &M0, const MaterialDev *mats, const TexUnitObjs *texs, int nmat,
                                  const int64_t *offsets, const float *u, const float *v, const float *s, int64_t n,
                                  void *out, int out_fp16, int *counter, unsigned *check, const SetConfig &cfg,
                                  cudaStream_t st);
cudaError_t launch_decode_set(const MaterialDev &M0, const MaterialDev *mats, int nmat, const int64_t *offsets,
                              const float *u, const float *v, const float *s, int64_t n, void *out, int out_fp16,
                              int *counter, unsigned *check, const SetConfig &cfg, bool single_geometry,
                              cudaStream_t st);
cudaError_t texunit_decode(const void *d_blocks, int bw, int bh, int is_signed, uint16_t *d_out, cudaStream_t st);

// thread-local error text
void set_error(const char *fmt, ...);

} // namespace bcf
