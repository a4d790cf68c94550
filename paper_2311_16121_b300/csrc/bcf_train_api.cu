// bcf_train_api.cu -- C ABI of the training path (include/bcf.h): validation
// of the trainer descriptor and the launches of a step.
#include <math.h>
#include <new>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "bcf_kernels.h"
#include "bcf_train.h"

namespace bcf {

static bcf_status tfail(bcf_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    set_error("%s", buf);
    return st;
}

static bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
static int lg2(int64_t v)
{
    int r = 0;
    while ((1ll << r) < v)
        ++r;
    return r;
}
static bool al16(const void *p) { return p && ((uintptr_t)p & 15) == 0; }

} // namespace bcf

using namespace bcf;

extern "C" {

bcf_status bcf_trainer_create(const bcf_trainer_desc *d, bcf_trainer *out)
{
    if (!d || !out)
        return tfail(BCF_ERR_INVALID_ARG, "bcf_trainer_create: null argument");
    *out = nullptr;
    TrainDev D;
    memset(&D, 0, sizeof D);
    if (d->num_textures < 1 || d->num_textures > BCF_MAX_TEX)
        return tfail(BCF_ERR_INVALID_ARG, "num_textures %d not in [1, %d]", d->num_textures, BCF_MAX_TEX);
    if (!pow2(d->res_ref))
        return tfail(BCF_ERR_INVALID_ARG, "res_ref %d is not a power of two", d->res_ref);
    D.n_tex = d->num_textures;
    D.lod_input = d->lod_input != 0;
    D.unconstrained = d->unconstrained != 0;
    D.is_signed = d->is_signed != 0;
    D.literal = d->literal != 0;
    if (d->batch_grid < 0 || d->batch_grid > 65535)
        return tfail(BCF_ERR_INVALID_ARG, "batch_grid %d not in [0, 65535]", d->batch_grid);
    D.batch_grid = d->batch_grid;
    if (D.unconstrained && (D.is_signed || D.literal))
        return tfail(BCF_ERR_INVALID_ARG, "unconstrained features have no BC6 emulation variant");
    for (int t = 0; t < D.n_tex; ++t) {
        const int res = d->res[t];
        if (!pow2(res) || res < 4 || res > 32768)
            return tfail(BCF_ERR_INVALID_ARG, "texture %d: res %d is not a power of two in [4, 32768]", t, res);
        if (d->levels[t] < 1 || d->levels[t] > lg2(res) - 1)
            return tfail(BCF_ERR_INVALID_ARG, "texture %d: levels %d not in [1, %d]", t, d->levels[t], lg2(res) - 1);
        if (!al16(d->d_params[t]) || !al16(d->d_grad[t]) || !al16(d->d_adam_m[t]) || !al16(d->d_adam_v[t]) ||
            (!d->d_partition[t] && !D.unconstrained))
            return tfail(BCF_ERR_INVALID_ARG, "texture %d: null or non-16-byte-aligned array", t);
        TrainTexDev &T = D.tex[t];
        T.params = d->d_params[t];
        T.grad = d->d_grad[t];
        T.m = d->d_adam_m[t];
        T.v = d->d_adam_v[t];
        T.part = d->d_partition[t];
        T.res = res;
        T.levels = d->levels[t];
        T.lod_bias = lg2(res) - lg2(d->res_ref);
        int64_t nb = 0;
        for (int l = 0; l < T.levels; ++l)
            nb += D.unconstrained ? (int64_t)(res >> l) * (res >> l) : (int64_t)((res >> l) / 4) * ((res >> l) / 4);
        T.blocks = nb;
    }
    if (d->n_layers < 1 || d->n_layers > BCF_MAX_LAYERS)
        return tfail(BCF_ERR_INVALID_ARG, "n_layers %d not in [1, %d]", d->n_layers, BCF_MAX_LAYERS);
    if (d->dims[0] != 3 * D.n_tex + D.lod_input)
        return tfail(BCF_ERR_INVALID_ARG, "dims[0] = %d but 3 * textures + lod_input = %d", d->dims[0],
                     3 * D.n_tex + D.lod_input);
    D.n_layers = d->n_layers;
    for (int l = 0; l <= D.n_layers; ++l) {
        if (d->dims[l] < 1 || d->dims[l] > 64)
            return tfail(d->dims[l] < 1 ? BCF_ERR_INVALID_ARG : BCF_ERR_UNSUPPORTED, "dims[%d] = %d not in [1, 64]",
                         l, d->dims[l]);
        D.dims[l] = d->dims[l];
    }
    if (D.dims[D.n_layers] != 9)
        return tfail(BCF_ERR_UNSUPPORTED, "the reference material has 9 channels; the MLP outputs %d",
                     D.dims[D.n_layers]);
    for (int l = 0; l < D.n_layers; ++l) {
        D.w_off[l] = D.w_total;
        D.b_off[l] = D.b_total;
        D.w_total += D.dims[l] * D.dims[l + 1];
        D.b_total += D.dims[l + 1];
    }
    const void *mlp[] = {d->d_W, d->d_b, d->d_W_grad, d->d_b_grad, d->d_W_m, d->d_W_v, d->d_b_m, d->d_b_v};
    for (const void *p : mlp)
        if (!al16(p))
            return tfail(BCF_ERR_INVALID_ARG, "null or non-16-byte-aligned MLP array");
    D.W = d->d_W;
    D.b = d->d_b;
    D.Wg = d->d_W_grad;
    D.bg = d->d_b_grad;
    D.Wm = d->d_W_m;
    D.Wv = d->d_W_v;
    D.bm = d->d_b_m;
    D.bv = d->d_b_v;
    if (!pow2(d->target_res) || d->target_res < 4 || d->target_levels < 1 ||
        d->target_levels > lg2(d->target_res) - 1 || !al16(d->d_target8) || !d->d_target1)
        return tfail(BCF_ERR_INVALID_ARG, "reference material: res %d levels %d or arrays invalid", d->target_res,
                     d->target_levels);
    D.tres = d->target_res;
    D.tlevels = d->target_levels;
    D.t8 = d->d_target8;
    D.t1 = d->d_target1;
    if (!(d->s_max >= 0.0f) || !(d->gamma > 0.0f) || !(d->beta1 >= 0.0f && d->beta1 < 1.0f) ||
        !(d->beta2 >= 0.0f && d->beta2 < 1.0f) || !(d->eps > 0.0f))
        return tfail(BCF_ERR_INVALID_ARG, "invalid hyper-parameters");
    D.s_max = d->s_max;
    if (D.unconstrained && !train_mma_supported(D))
        return tfail(BCF_ERR_UNSUPPORTED, "unconstrained features need a dims[0] <= 16 -> 32 -> 32 -> C or "
                                          "dims[0] <= 16 -> 16 -> C MLP (C <= 9)");
    if (train_smem_bytes(D) > 227 * 1024)
        return tfail(BCF_ERR_UNSUPPORTED, "MLP too wide for the training kernel's shared memory");
    unsigned *check = check_word(); // after every argument check: the first call allocates on the device
    if (!check)
        return tfail(BCF_ERR_OOM, "bcf_trainer_create: the device check word could not be created");
    for (int t = 0; t < D.n_tex; ++t)
        D.tex[t].check = check;
    bcf_trainer tr = new (std::nothrow) bcf_trainer_s;
    if (!tr)
        return tfail(BCF_ERR_OOM, "host allocation failed");
    tr->dev = D;
    tr->hyper = {d->lr_features, d->lr_mlp, d->gamma, d->beta1, d->beta2, d->eps};
    *out = tr;
    return BCF_OK;
}

bcf_status bcf_trainer_destroy(bcf_trainer tr)
{
    delete tr;
    return BCF_OK;
}

static bcf_status check_queries(const float *u, const float *v, const float *s, int64_t n, const char *what)
{
    if (n < 0)
        return tfail(BCF_ERR_INVALID_ARG, "%s: n < 0", what);
    if (n > 0 && (!u || !v || !s))
        return tfail(BCF_ERR_INVALID_ARG, "%s: null query arrays", what);
    return BCF_OK;
}

bcf_status bcf_train_step(bcf_trainer tr, int64_t batch, uint64_t seed, int64_t step, const float *d_u,
                          const float *d_v, const float *d_s, float *d_loss_out, bcf_stream stream)
{
    if (!tr || batch < 0 || step < 0 || !d_loss_out)
        return tfail(BCF_ERR_INVALID_ARG, "bcf_train_step: null trainer / loss, or negative batch / step");
    if ((d_u != nullptr) != (d_v != nullptr) || (d_u != nullptr) != (d_s != nullptr))
        return tfail(BCF_ERR_INVALID_ARG, "bcf_train_step: give all of u, v, s or none");
    if (!d_u && tr->dev.batch_grid > 0 && batch != (int64_t)tr->dev.batch_grid * tr->dev.batch_grid)
        return tfail(BCF_ERR_INVALID_ARG, "bcf_train_step: grid batches need batch = %d^2",
                     tr->dev.batch_grid);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync(d_loss_out, 0, sizeof(float), st);
    if (e == cudaSuccess)
        e = launch_train(tr->dev, 2, batch, seed, step, d_u, d_v, d_s, nullptr, nullptr, d_loss_out, st);
    if (e == cudaSuccess)
        e = launch_adam(tr->dev, tr->hyper, step, st);
    if (e != cudaSuccess)
        return tfail(BCF_ERR_CUDA, "bcf_train_step: %s", cudaGetErrorString(e));
    return BCF_OK;
}

bcf_status bcf_train_forward(bcf_trainer tr, const float *d_u, const float *d_v, const float *d_s, int64_t n,
                             float *d_out, bcf_stream stream)
{
    if (!tr)
        return tfail(BCF_ERR_INVALID_ARG, "bcf_train_forward: null trainer");
    bcf_status st = check_queries(d_u, d_v, d_s, n, "bcf_train_forward");
    if (st != BCF_OK)
        return st;
    if (n > 0 && !d_out)
        return tfail(BCF_ERR_INVALID_ARG, "bcf_train_forward: null output");
    cudaError_t e = launch_train(tr->dev, 0, n, 0, 0, d_u, d_v, d_s, d_out, nullptr, nullptr, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return tfail(BCF_ERR_CUDA, "bcf_train_forward: %s", cudaGetErrorString(e));
    return BCF_OK;
}

bcf_status bcf_train_backward(bcf_trainer tr, const float *d_u, const float *d_v, const float *d_s, int64_t n,
                              const float *d_grad_out, bcf_stream stream)
{
    if (!tr)
        return tfail(BCF_ERR_INVALID_ARG, "bcf_train_backward: null trainer");
    bcf_status st = check_queries(d_u, d_v, d_s, n, "bcf_train_backward");
    if (st != BCF_OK)
        return st;
    if (n > 0 && !d_grad_out)
        return tfail(BCF_ERR_INVALID_ARG, "bcf_train_backward: null gradient");
    cudaError_t e =
        launch_train(tr->dev, 1, n, 0, 0, d_u, d_v, d_s, nullptr, d_grad_out, nullptr, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return tfail(BCF_ERR_CUDA, "bcf_train_backward: %s", cudaGetErrorString(e));
    return BCF_OK;
}

bcf_status bcf_train_export(bcf_trainer tr, void *const *d_blocks_out, uint16_t *d_weights_fp16, bcf_stream stream)
{
    if (!tr || !d_blocks_out)
        return tfail(BCF_ERR_INVALID_ARG, "bcf_train_export: null argument");
    if (tr->dev.unconstrained)
        return tfail(BCF_ERR_UNSUPPORTED, "bcf_train_export: unconstrained features have no block encoding "
                                          "(compress them with bcf_encode_mode10)");
    for (int t = 0; t < tr->dev.n_tex; ++t)
        if (!al16(d_blocks_out[t]))
            return tfail(BCF_ERR_INVALID_ARG, "bcf_train_export: texture %d output null or misaligned", t);
    cudaError_t e = launch_export(tr->dev, d_blocks_out, d_weights_fp16, (cudaStream_t)stream);
    if (e != cudaSuccess)
        return tfail(BCF_ERR_CUDA, "bcf_train_export: %s", cudaGetErrorString(e));
    return BCF_OK;
}

bcf_status bcf_pack_mode10(const float *d_params, const uint8_t *d_partitions, int64_t n_blocks, int32_t is_signed,
                           void *d_blocks_out, bcf_stream stream)
{
    if (n_blocks < 0)
        return tfail(BCF_ERR_INVALID_ARG, "bcf_pack_mode10: n_blocks %lld < 0", (long long)n_blocks);
    if (n_blocks == 0)
        return BCF_OK;
    if (!al16(d_params) || !d_partitions || !al16(d_blocks_out))
        return tfail(BCF_ERR_INVALID_ARG, "bcf_pack_mode10: null or misaligned pointer");
    unsigned *check = check_word();
    if (!check)
        return tfail(BCF_ERR_OOM, "bcf_pack_mode10: the device check word could not be created");
    cudaError_t e = launch_export_blocks(d_params, d_partitions, n_blocks, is_signed ? 1 : 0, check, d_blocks_out,
                                         (cudaStream_t)stream);
    if (e != cudaSuccess)
        return tfail(BCF_ERR_CUDA, "bcf_pack_mode10: %s", cudaGetErrorString(e));
    return BCF_OK;
}

} // extern "C"
