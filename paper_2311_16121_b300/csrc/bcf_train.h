// bcf_train.h -- trainer structures shared by the training kernels and the C ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/bcf.h"

namespace bcf {

struct TrainTexDev {
    float *params;        // [blocks][32]
    float *grad;          // [blocks][32]
    float *m, *v;         // Adam moments
    const uint8_t *part;  // [blocks]
    unsigned *check;      // the device's check word (BCF_CHECK_PARTITION)
    int32_t res, levels, lod_bias;
    int64_t blocks;       // block records, or texels when the features are unconstrained
};

struct TrainDev {
    int32_t n_tex, lod_input, n_layers;
    int32_t dims[BCF_MAX_LAYERS + 1];
    int32_t w_off[BCF_MAX_LAYERS], b_off[BCF_MAX_LAYERS];
    int32_t w_total, b_total;
    TrainTexDev tex[BCF_MAX_TEX];
    float *W, *b, *Wg, *bg, *Wm, *Wv, *bm, *bv;
    int32_t tres, tlevels;
    const uint16_t *t8, *t1;
    float s_max;
    int32_t unconstrained; // free per-texel features [texels][4] instead of block records [blocks][32]
    int32_t is_signed;     // SF16 block features (endpoints in [-32, 31], a = 31/32)
    int32_t literal;       // Eq. 7-8 as printed instead of the format's exact steps
    int32_t batch_grid;    // > 0: batches are batch_grid x batch_grid uv grids with one scale (the paper's form)
};

// emulation variant of the block features: bit 0 signed, bit 1 literal
__host__ __device__ inline int emulation_variant(const TrainDev &D) { return (D.is_signed ? 1 : 0) | (D.literal ? 2 : 0); }

// floats of one texture's feature array
inline int64_t feature_floats(const TrainDev &D, int t) { return D.tex[t].blocks * (D.unconstrained ? 4 : 32); }

struct TrainHyper {
    float lr_features, lr_mlp, gamma, beta1, beta2, eps;
};

int64_t train_smem_bytes(const TrainDev &D);
cudaError_t launch_train(const TrainDev &D, int mode, int64_t batch, uint64_t seed, int64_t step, const float *u,
                         const float *v, const float *s, float *out, const float *grad_out, float *loss,
                         cudaStream_t st);
bool train_mma_supported(const TrainDev &D);
cudaError_t launch_train_mma(const TrainDev &D, int mode, int64_t batch, uint64_t seed, int64_t step,
                             const float *u, const float *v, const float *s, float *out, const float *grad_out,
                             float *loss, int sms, cudaStream_t st);
cudaError_t launch_adam(const TrainDev &D, const TrainHyper &H, int64_t step, cudaStream_t st);
cudaError_t launch_export(const TrainDev &D, void *const *blocks_out, uint16_t *weights_fp16, cudaStream_t st);
cudaError_t launch_export_blocks(const float *params, const uint8_t *part, int64_t nblocks, int is_signed,
                                 unsigned *check, void *out, cudaStream_t st);

} // namespace bcf

struct bcf_trainer_s {
    bcf::TrainDev dev;
    bcf::TrainHyper hyper;
};
