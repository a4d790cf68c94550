// bcf_train_noalloc.cu -- the training step without any device allocation,
// for callers that cannot allocate device memory (engines with their own
// budgeted allocator, frame loops that must not call cudaMalloc).
//
// The gradient accumulators, which only live between the gradient kernel
// and the optimiser kernel, are placed in a file-scope device array of
// BCF_NOALLOC_MAX_GRAD_FLOATS floats.  Host code cannot use the array's name
// as a device address, so its address is looked up once per device with
// cudaGetSymbolAddress and passed to the kernels.
#include <mutex>
#include <stdio.h>

#include "bcf_kernels.h"
#include "bcf_train.h"

namespace bcf {

static __device__ __align__(256) float g_train_grad_scratch[BCF_NOALLOC_MAX_GRAD_FLOATS];

constexpr int kMaxDevices = 64;
static std::mutex g_scratch_mu;
static float *g_scratch_ptr[kMaxDevices];

// Device address of the scratch array on the current device (looked up on
// the first call made with that device current).  The address stays valid
// for the life of the device's primary context: a cudaDeviceReset ends it,
// as it ends every material and trainer created before it.
static cudaError_t scratch_address(float **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return e;
    if (dev < 0 || dev >= kMaxDevices)
        return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_train_grad_scratch);
        if (e != cudaSuccess)
            return e;
        g_scratch_ptr[dev] = static_cast<float *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

static int64_t round32(int64_t n) { return (n + 31) / 32 * 32; }

} // namespace bcf

using namespace bcf;

extern "C" bcf_status bcf_train_step_noalloc(bcf_trainer tr, int64_t batch, uint64_t seed, int64_t step,
                                             const float *d_u, const float *d_v, const float *d_s, float *d_loss_out,
                                             bcf_stream stream)
{
    if (!tr || batch < 0 || step < 0 || !d_loss_out) {
        set_error("bcf_train_step_noalloc: null trainer / loss, or negative batch / step");
        return BCF_ERR_INVALID_ARG;
    }
    if ((d_u != nullptr) != (d_v != nullptr) || (d_u != nullptr) != (d_s != nullptr)) {
        set_error("bcf_train_step_noalloc: give all of u, v, s or none");
        return BCF_ERR_INVALID_ARG;
    }
    if (!d_u && tr->dev.batch_grid > 0 && batch != (int64_t)tr->dev.batch_grid * tr->dev.batch_grid) {
        set_error("bcf_train_step_noalloc: grid batches need batch = %d^2", tr->dev.batch_grid);
        return BCF_ERR_INVALID_ARG;
    }
    TrainDev D = tr->dev;
    int64_t need = 0;
    for (int t = 0; t < D.n_tex; ++t)
        need += round32(feature_floats(D, t));
    need += round32(D.w_total) + round32(D.b_total);
    if (need > BCF_NOALLOC_MAX_GRAD_FLOATS) {
        set_error("bcf_train_step_noalloc: %lld gradient values exceed the %d of the library's scratch array",
                  (long long)need, BCF_NOALLOC_MAX_GRAD_FLOATS);
        return BCF_ERR_UNSUPPORTED;
    }
    float *base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) {
        set_error("bcf_train_step_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        return BCF_ERR_CUDA;
    }
    int64_t off = 0;
    for (int t = 0; t < D.n_tex; ++t) {
        D.tex[t].grad = base + off;
        off += round32(feature_floats(D, t));
    }
    D.Wg = base + off;
    off += round32(D.w_total);
    D.bg = base + off;
    cudaStream_t st = (cudaStream_t)stream;
    e = cudaMemsetAsync(base, 0, (size_t)need * sizeof(float), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(d_loss_out, 0, sizeof(float), st);
    if (e == cudaSuccess)
        e = launch_train(D, 2, batch, seed, step, d_u, d_v, d_s, nullptr, nullptr, d_loss_out, st);
    if (e == cudaSuccess)
        e = launch_adam(D, tr->hyper, step, st);
    if (e != cudaSuccess) {
        set_error("bcf_train_step_noalloc: %s", cudaGetErrorString(e));
        return BCF_ERR_CUDA;
    }
    return BCF_OK;
}
