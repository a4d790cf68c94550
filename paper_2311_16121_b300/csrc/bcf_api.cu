// bcf_api.cu -- the libbcf C ABI (include/bcf.h): argument validation, the
// material metadata and the kernel launches.  No entry point allocates on
// the decode path; bcf_create_material allocates the small device metadata.
#include <math.h>
#include <algorithm>
#include <mutex>
#include <new>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "bcf_kernels.h"

namespace bcf {

static thread_local char g_err[512];

void set_error(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

static bcf_status fail(bcf_status st, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

static bcf_status cuda_status(cudaError_t e, const char *what)
{
    if (e == cudaSuccess)
        return BCF_OK;
    return fail(BCF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

static bool is_pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
static int ilog2(int64_t v)
{
    int r = 0;
    while ((1ll << r) < v)
        ++r;
    return r;
}
static bool aligned(const void *p, int a) { return ((uintptr_t)p % (uintptr_t)a) == 0; }
static int round_up(int v, int m) { return (v + m - 1) / m * m; }

constexpr int kMaxDevices = 64;
static std::mutex g_check_mu;
static unsigned *g_check[kMaxDevices];

unsigned *check_word()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return nullptr;
    std::lock_guard<std::mutex> lock(g_check_mu);
    if (!g_check[dev]) {
        unsigned *p = nullptr;
        const unsigned zero = 0;
        if (cudaMalloc(&p, sizeof(unsigned)) != cudaSuccess)
            return nullptr;
        if (cudaMemcpy(p, &zero, sizeof zero, cudaMemcpyHostToDevice) != cudaSuccess) { // synchronous
            cudaFree(p);
            return nullptr;
        }
        g_check[dev] = p;
    }
    return g_check[dev];
}

} // namespace bcf

using namespace bcf;

extern "C" {

const char *bcf_status_string(bcf_status s)
{
    switch (s) {
    case BCF_OK: return "ok";
    case BCF_ERR_INVALID_ARG: return "invalid argument";
    case BCF_ERR_UNSUPPORTED: return "unsupported";
    case BCF_ERR_CUDA: return "CUDA error";
    case BCF_ERR_OOM: return "out of memory";
    case BCF_ERR_TIMEOUT: return "device wait timed out";
    case BCF_ERR_DEVICE_CHECK: return "device-side check failed";
    }
    return "unknown status";
}

const char *bcf_last_error(void) { return g_err; }

int bcf_version(void) { return 100; }

bcf_status bcf_device_check(uint32_t *h_word)
{
    if (h_word)
        *h_word = 0;
    unsigned *w = check_word();
    if (!w)
        return fail(BCF_ERR_OOM, "bcf_device_check: the device check word could not be created");
    unsigned h = 0;
    cudaError_t e = cudaDeviceSynchronize(); // every stream: no kernel can set a bit between the read and the clear
    if (e == cudaSuccess)
        e = cudaMemcpy(&h, w, sizeof h, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemset(w, 0, sizeof h);
    if (e == cudaSuccess)
        e = cudaDeviceSynchronize();
    if (e != cudaSuccess)
        return cuda_status(e, "bcf_device_check");
    if (h_word)
        *h_word = h;
    if (!h)
        return BCF_OK;
    return fail(BCF_ERR_DEVICE_CHECK, "device checks fired (word 0x%x):%s%s%s", h,
                (h & BCF_CHECK_PARTITION) ? " a training block's partition id is above 31 (read as id & 31);" : "",
                (h & BCF_CHECK_OFFSETS) ? " material-set query offsets decrease (that range was decoded as empty);"
                                        : "",
                (h & BCF_CHECK_TIMEOUT) ? " a decode's bounded wait for its tensor-core MMAs ran out (output "
                                          "incomplete);"
                                        : "");
}

bcf_status bcf_decode_bc6h(const void *d_blocks, int32_t blocks_w, int32_t blocks_h, int32_t is_signed, uint16_t *d_out,
                           bcf_stream stream)
{
    if (blocks_w < 0 || blocks_h < 0)
        return fail(BCF_ERR_INVALID_ARG, "bcf_decode_bc6h: negative size %d x %d", blocks_w, blocks_h);
    if ((int64_t)blocks_w * blocks_h == 0)
        return BCF_OK;
    if ((int64_t)blocks_w * blocks_h > (1ll << 31))
        return fail(BCF_ERR_INVALID_ARG, "bcf_decode_bc6h: more than 2^31 blocks");
    if (!d_blocks || !d_out || !aligned(d_blocks, 16) || !aligned(d_out, 8))
        return fail(BCF_ERR_INVALID_ARG, "bcf_decode_bc6h: null or misaligned pointer");
    return cuda_status(launch_unpack_image(d_blocks, blocks_w, blocks_h, is_signed != 0, d_out, (cudaStream_t)stream),
                       "bcf_decode_bc6h launch");
}

bcf_status bcf_texunit_decode_bc6h(const void *d_blocks, int32_t blocks_w, int32_t blocks_h, int32_t is_signed,
                                   uint16_t *d_out, bcf_stream stream)
{
    if (blocks_w <= 0 || blocks_h <= 0 || blocks_w > 16384 || blocks_h > 16384)
        return fail(BCF_ERR_INVALID_ARG, "bcf_texunit_decode_bc6h: size %d x %d out of range", blocks_w, blocks_h);
    if (!d_blocks || !d_out || !aligned(d_blocks, 16) || !aligned(d_out, 8))
        return fail(BCF_ERR_INVALID_ARG, "bcf_texunit_decode_bc6h: null or misaligned pointer");
    cudaError_t e = texunit_decode(d_blocks, blocks_w, blocks_h, is_signed != 0, d_out, (cudaStream_t)stream);
    return e == cudaSuccess ? BCF_OK : BCF_ERR_CUDA;
}

bcf_status bcf_create_material(const bcf_material_desc *d, bcf_material *out)
{
    if (!d || !out)
        return fail(BCF_ERR_INVALID_ARG, "bcf_create_material: null argument");
    *out = nullptr;
    if (d->num_textures < 1 || d->num_textures > BCF_MAX_TEX)
        return fail(BCF_ERR_INVALID_ARG, "num_textures %d not in [1, %d]", d->num_textures, BCF_MAX_TEX);
    if (!is_pow2(d->res_ref))
        return fail(BCF_ERR_INVALID_ARG, "res_ref %d is not a power of two", d->res_ref);
    MaterialDev M;
    memset(&M, 0, sizeof M);
    M.n_tex = d->num_textures;
    M.is_signed = d->is_signed != 0;
    M.wrap = d->wrap != 0;
    M.lod_input = d->lod_input != 0;
    for (int t = 0; t < M.n_tex; ++t) {
        const int res = d->res[t];
        if (!is_pow2(res) || res < 4 || res > 32768)
            return fail(BCF_ERR_INVALID_ARG, "texture %d: res %d is not a power of two in [4, 32768]", t, res);
        const int maxl = ilog2(res) - 1;
        if (d->levels[t] < 1 || d->levels[t] > maxl || d->levels[t] > BCF_MAX_LEVELS)
            return fail(BCF_ERR_INVALID_ARG, "texture %d: levels %d not in [1, %d]", t, d->levels[t], maxl);
        if (!d->d_blocks[t] || !aligned(d->d_blocks[t], 16))
            return fail(BCF_ERR_INVALID_ARG, "texture %d: null or non-16-byte-aligned block pointer", t);
        TexDev &T = M.tex[t];
        T.blocks = (const uint4 *)d->d_blocks[t];
        T.res = res;
        T.log2res = ilog2(res);
        T.levels = d->levels[t];
        T.lod_bias = ilog2(res) - ilog2(d->res_ref);
        uint32_t off = 0;
        for (int l = 0; l < BCF_MAX_LEVELS; ++l) {
            T.level_off[l] = off;
            if (l < T.levels) {
                const uint32_t wb = (uint32_t)(res >> l) / 4;
                off += wb * wb;
            }
        }
    }
    M.n_in = 3 * M.n_tex + M.lod_input;
    M.n_groups = 0;
    for (int t = 0; t < M.n_tex; ++t) {
        int g = 0;
        while (g < M.n_groups && !(M.tex[M.group_first[g]].res == M.tex[t].res &&
                                   M.tex[M.group_first[g]].levels == M.tex[t].levels))
            ++g;
        if (g == M.n_groups)
            M.group_first[M.n_groups++] = t;
        M.tex_group[t] = g;
    }
    MlpDev &P = M.mlp;
    if (d->n_layers < 1 || d->n_layers > BCF_MAX_LAYERS)
        return fail(BCF_ERR_INVALID_ARG, "n_layers %d not in [1, %d]", d->n_layers, BCF_MAX_LAYERS);
    if (d->dims[0] != M.n_in)
        return fail(BCF_ERR_INVALID_ARG, "dims[0] = %d but 3 * textures + lod_input = %d", d->dims[0], M.n_in);
    if (d->precision < BCF_FP32 || d->precision > BCF_FP8_E4M3)
        return fail(BCF_ERR_INVALID_ARG, "unknown precision %d", (int)d->precision);
    if (!d->d_weights || !d->d_biases || !aligned(d->d_weights, 4) || !aligned(d->d_biases, 4))
        return fail(BCF_ERR_INVALID_ARG, "null or misaligned weights / biases");
    P.n_layers = d->n_layers;
    P.precision = d->precision;
    P.weights = d->d_weights;
    P.biases = d->d_biases;
    int woff = 0, boff = 0;
    const int kq = d->precision == BCF_FP8_E4M3 ? 32 : 16;
    for (int l = 0; l <= P.n_layers; ++l) {
        if (d->dims[l] < 1 || d->dims[l] > BCF_MAX_WIDTH)
            return fail(d->dims[l] < 1 ? BCF_ERR_INVALID_ARG : BCF_ERR_UNSUPPORTED, "dims[%d] = %d not in [1, %d]", l,
                        d->dims[l], BCF_MAX_WIDTH);
        P.dims[l] = d->dims[l];
    }
    for (int l = 0; l < P.n_layers; ++l) {
        P.w_off[l] = woff;
        P.b_off[l] = boff;
        woff += P.dims[l] * P.dims[l + 1];
        boff += P.dims[l + 1];
        P.kpad[l] = round_up(P.dims[l], kq);
    }
    for (int l = 0; l < P.n_layers; ++l)
        P.npad[l] = l + 1 < P.n_layers ? P.kpad[l + 1] : round_up(P.dims[l + 1], 8);
    for (int l = 0; l < P.n_layers; ++l) {
        P.act_scale[l] = 1.0f;
        P.w_scale[l] = 1.0f;
        P.inv_act_scale[l] = 1.0f;
        if (d->precision == BCF_FP8_E4M3) {
            const float a = d->act_scale[l], w = d->w_scale[l];
            int ea, ew;
            if (!(a > 0.0f) || !(w > 0.0f) || frexpf(a, &ea) != 0.5f || frexpf(w, &ew) != 0.5f)
                return fail(BCF_ERR_UNSUPPORTED, "layer %d: FP8 scales must be positive powers of two (got %g, %g)", l,
                            (double)a, (double)w);
            P.act_scale[l] = a;
            P.w_scale[l] = w;
            P.inv_act_scale[l] = 1.0f / a;
        }
    }
    M.n_out = P.dims[P.n_layers];
    if (d->precision != BCF_FP32) {
        P.smem_w_bytes = 0;
        if (decode_mma_smem_bytes(P) > 200 * 1024 || decode_tiled_smem_bytes(P) > 227 * 1024)
            return fail(BCF_ERR_UNSUPPORTED, "MLP too large for the shared-memory tensor-core path");
    }
    bcf_material m = new (std::nothrow) bcf_material_s;
    if (!m)
        return fail(BCF_ERR_OOM, "host allocation failed");
    m->host = M;
    m->dev = nullptr;
    m->variant = 0;
    m->hw = TexUnitObjs{};
    for (int t = 0; t < BCF_MAX_TEX; ++t)
        m->hw_arrays[t] = nullptr;
    m->hw_ready = 0;
    m->pipe_ready = 0;
    for (cudaStream_t &x : m->pipe_streams)
        x = nullptr;
    for (cudaEvent_t &x : m->pipe_events)
        x = nullptr;
    cudaGetDevice(&m->device);
    cudaError_t e = cudaMalloc(&m->dev, sizeof(MaterialDev));
    if (e != cudaSuccess) {
        delete m;
        return fail(BCF_ERR_OOM, "cudaMalloc(material metadata): %s", cudaGetErrorString(e));
    }
    e = cudaMemcpy(m->dev, &m->host, sizeof(MaterialDev), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(m->dev);
        delete m;
        return cuda_status(e, "cudaMemcpy(material metadata)");
    }
    *out = m;
    return BCF_OK;
}

bcf_status bcf_set_decode_variant(bcf_material m, int32_t variant)
{
    if (!m || variant < 0 || variant > 3)
        return fail(BCF_ERR_INVALID_ARG, "bcf_set_decode_variant: null material or variant not in {0, 1, 2, 3}");
    if (variant >= 2) {
        if (m->host.mlp.precision == BCF_FP32 && variant == 2)
            return fail(BCF_ERR_UNSUPPORTED, "bcf_set_decode_variant: the hardware-trilinear variant needs a "
                                             "tensor-core (FP16 / BF16 / FP8) material");
        if (!m->hw_ready) {
            cudaError_t e = texunit_create(m->host, m->hw, m->hw_arrays);
            if (e != cudaSuccess)
                return cuda_status(e, "bcf_set_decode_variant: texture-unit textures");
            m->hw_ready = 1;
        }
    }
    m->variant = variant;
    return BCF_OK;
}

bcf_status bcf_material_refresh(bcf_material m, bcf_stream stream)
{
    if (!m)
        return fail(BCF_ERR_INVALID_ARG, "bcf_material_refresh: null material");
    if (!m->hw_ready)
        return BCF_OK;
    return cuda_status(texunit_refresh(m->host, m->hw_arrays, (cudaStream_t)stream), "bcf_material_refresh");
}

bcf_status bcf_set_mlp_engine(bcf_material m, int32_t engine)
{
    if (!m || (engine != BCF_MLP_MMA_SYNC && engine != BCF_MLP_TCGEN05))
        return fail(BCF_ERR_INVALID_ARG, "bcf_set_mlp_engine: null material or engine not in {0, 1}");
    if (engine == BCF_MLP_TCGEN05) {
        const MlpDev &P = m->host.mlp;
        const bool shape = P.n_layers == 3 && P.npad[2] == 16 &&
                           ((P.npad[0] == 32 && P.npad[1] == 32 &&
                             P.kpad[0] == (P.precision == BCF_FP8_E4M3 ? 32 : 16)) ||
                            (P.npad[0] == 64 && P.npad[1] == 64 && P.kpad[0] == 32));
        if (P.precision == BCF_FP32 || !shape)
            return fail(BCF_ERR_UNSUPPORTED, "bcf_set_mlp_engine: tcgen05 covers FP16 / BF16 / FP8 MLPs of three "
                                             "layers K0 -> 32 -> 32 -> C or 32 -> 64 -> 64 -> C (C <= 16)");
    }
    m->host.mlp_engine = engine;
    cudaError_t e = cudaMemcpy(&m->dev->mlp_engine, &m->host.mlp_engine, sizeof(int32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess)
        return cuda_status(e, "bcf_set_mlp_engine");
    return BCF_OK;
}

bcf_status bcf_texunit_fetch_probe(bcf_material m, int32_t texture, int32_t level, int64_t n_threads,
                                   int32_t rounds, float *d_sink, bcf_stream stream)
{
    if (!m || texture < 0 || texture >= m->host.n_tex || level < 0 || level >= m->host.tex[texture].levels ||
        n_threads < 0 || n_threads > (1ll << 40) || rounds < 1 || rounds > 4096 || (n_threads > 0 && !d_sink) ||
        !aligned(d_sink, 4))
        return fail(BCF_ERR_INVALID_ARG, "bcf_texunit_fetch_probe: invalid material, texture, level, size or sink");
    if (!m->hw_ready)
        return fail(BCF_ERR_UNSUPPORTED, "bcf_texunit_fetch_probe: the material has no texture objects "
                                         "(select decode variant 2 or 3 first)");
    return cuda_status(launch_texfetch_probe(m->hw.texp[texture], m->host.tex[texture].res >> level, level,
                                             n_threads, rounds, d_sink, (cudaStream_t)stream),
                       "bcf_texunit_fetch_probe launch");
}

bcf_status bcf_destroy_material(bcf_material m)
{
    if (!m)
        return BCF_OK;
    if (m->hw_ready)
        texunit_destroy(m->hw, m->hw_arrays, m->host.n_tex);
    if (m->pipe_ready) { // released once their pending work completes
        for (cudaStream_t x : m->pipe_streams)
            cudaStreamDestroy(x);
        for (cudaEvent_t x : m->pipe_events)
            cudaEventDestroy(x);
    }
    cudaError_t e = cudaFree(m->dev);
    delete m;
    return cuda_status(e, "cudaFree(material metadata)");
}

bcf_status bcf_sample_features(bcf_material m, const float *d_u, const float *d_v, const float *d_s, int64_t n,
                               float *d_feat, bcf_stream stream)
{
    if (!m || n < 0)
        return fail(BCF_ERR_INVALID_ARG, "bcf_sample_features: null material or n < 0");
    if (n == 0)
        return BCF_OK;
    if (!d_u || !d_v || !d_feat || !aligned(d_u, 4) || !aligned(d_v, 4) || !aligned(d_feat, 4) ||
        (d_s && !aligned(d_s, 4)))
        return fail(BCF_ERR_INVALID_ARG, "bcf_sample_features: null or misaligned pointer");
    return cuda_status(launch_sample_features(m->host, d_u, d_v, d_s, n, d_feat, (cudaStream_t)stream),
                       "bcf_sample_features launch");
}

bcf_status bcf_decode_material(bcf_material m, const float *d_u, const float *d_v, const float *d_s, int64_t n,
                               void *d_out, bcf_precision out_precision, bcf_stream stream)
{
    if (!m || n < 0)
        return fail(BCF_ERR_INVALID_ARG, "bcf_decode_material: null material or n < 0");
    if (out_precision != BCF_FP32 && out_precision != BCF_FP16)
        return fail(BCF_ERR_INVALID_ARG, "bcf_decode_material: out_precision must be FP32 or FP16");
    if (n == 0)
        return BCF_OK;
    if (!d_u || !d_v || !d_out || !aligned(d_u, 4) || !aligned(d_v, 4) || !aligned(d_out, 16) ||
        (d_s && !aligned(d_s, 4)))
        return fail(BCF_ERR_INVALID_ARG, "bcf_decode_material: null or misaligned pointer");
    const int fp16 = out_precision == BCF_FP16;
    cudaError_t e;
    if (m->host.mlp.precision == BCF_FP32)
        e = m->variant == 3 ? launch_decode_fp32_texunit(m->host, m->hw, d_u, d_v, d_s, n, d_out, fp16,
                                                          (cudaStream_t)stream)
                            : launch_decode_fp32(m->host, d_u, d_v, d_s, n, d_out, fp16, (cudaStream_t)stream);
    else if (m->variant == 1)
        e = launch_decode_mma(m->host, d_u, d_v, d_s, n, d_out, fp16, (cudaStream_t)stream);
    else if (m->variant >= 2)
        e = launch_decode_texunit(m->host, m->hw, m->variant == 3, d_u, d_v, d_s, n, d_out, fp16,
                                  (cudaStream_t)stream);
    else
        e = launch_decode_tiled(m->host, d_u, d_v, d_s, n, d_out, fp16, (cudaStream_t)stream);
    return cuda_status(e, "bcf_decode_material launch");
}

// ------------------------------------------------------------ host-resident queries

// The decode of queries and outputs that live in host memory, pipelined in chunks over three streams: the
// upload of chunk i + 1, the decode of chunk i and the download of chunk i - 1 overlap.  BCF_PIPE_BUFS (three)
// chunk buffers rotate in the caller's device scratch; per buffer an event marks when its download has
// finished so the next upload into it may start.
bcf_status bcf_decode_material_host(bcf_material m, const float *h_u, const float *h_v, const float *h_s, int64_t n,
                                    void *h_out, bcf_precision out_precision, void *d_scratch, int64_t scratch_bytes,
                                    bcf_stream stream)
{
    if (!m || n < 0)
        return fail(BCF_ERR_INVALID_ARG, "bcf_decode_material_host: null material or n < 0");
    if (out_precision != BCF_FP32 && out_precision != BCF_FP16)
        return fail(BCF_ERR_INVALID_ARG, "bcf_decode_material_host: out_precision must be FP32 or FP16");
    if (n == 0)
        return BCF_OK;
    if (!h_u || !h_v || !h_out || !d_scratch || !aligned(d_scratch, 256))
        return fail(BCF_ERR_INVALID_ARG, "bcf_decode_material_host: null pointer or scratch not 256-byte aligned");
    const int C = m->host.mlp.dims[m->host.mlp.n_layers];
    const int64_t out_b = (int64_t)C * (out_precision == BCF_FP16 ? 2 : 4);
    const int64_t per_q = (h_s ? 12 : 8) + out_b;
    constexpr int NB = BCF_PIPE_BUFS;
    int64_t chunk = (scratch_bytes - 1024 * (NB + 1)) / (NB * per_q) / 256 * 256; // each array 256-aligned
    if (chunk < 256)
        return fail(BCF_ERR_INVALID_ARG, "bcf_decode_material_host: scratch of %lld bytes holds no 256-query chunk",
                    (long long)scratch_bytes);
    // at least about four chunks; three buffers let chunk i + 1 upload while chunk i decodes and chunk i - 1
    // downloads (measured on the 3840x2160 frame with 128 MB of scratch, 6 chunks: 3.60 ms, against 3.85 ms
    // with two buffers; about 16 smaller chunks, or a short first and last chunk, were slower)
    chunk = std::min<int64_t>(chunk, std::max<int64_t>(256, (n / 4 + 255) / 256 * 256));
    auto up = [](int64_t b) { return (b + 255) / 256 * 256; };
    const int64_t buf = up(chunk * 4) * (h_s ? 3 : 2) + up(chunk * out_b);
    char *base[NB];
    for (int b = 0; b < NB; ++b)
        base[b] = (char *)d_scratch + b * buf;
    cudaError_t e = cudaSuccess;
    if (!m->pipe_ready) { // the material's pipeline streams and events, created once
        for (int i = 0; i < 3 && e == cudaSuccess; ++i)
            e = cudaStreamCreateWithFlags(&m->pipe_streams[i], cudaStreamNonBlocking);
        for (int i = 0; i < 2 + 3 * NB && e == cudaSuccess; ++i)
            e = cudaEventCreateWithFlags(&m->pipe_events[i], cudaEventDisableTiming);
        if (e != cudaSuccess)
            return cuda_status(e, "bcf_decode_material_host: pipeline streams and events");
        m->pipe_ready = 1;
    }
    cudaStream_t cs = (cudaStream_t)stream, sin = m->pipe_streams[0], scomp = m->pipe_streams[1],
                 sout = m->pipe_streams[2];
    cudaEvent_t start = m->pipe_events[0], done = m->pipe_events[1];
    const cudaEvent_t *in_done = m->pipe_events + 2, *comp_done = in_done + NB, *free_ev = comp_done + NB;
    if (e == cudaSuccess)
        e = cudaEventRecord(start, cs); // the pipeline starts after the caller's earlier work
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(sin, start, 0);
    bcf_status st = BCF_OK;
    int64_t q0 = 0;
    for (int64_t i = 0; q0 < n && e == cudaSuccess && st == BCF_OK; ++i) {
        const int b = (int)(i % NB);
        const int64_t nq = std::min(chunk, n - q0);
        float *du = (float *)base[b], *dv = (float *)(base[b] + up(chunk * 4));
        float *ds = h_s ? (float *)(base[b] + 2 * up(chunk * 4)) : nullptr;
        void *dout = base[b] + up(chunk * 4) * (h_s ? 3 : 2);
        if (i >= NB) // the buffer's previous chunk has been downloaded
            e = cudaStreamWaitEvent(sin, free_ev[b], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(du, h_u + q0, nq * 4, cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dv, h_v + q0, nq * 4, cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess && h_s)
            e = cudaMemcpyAsync(ds, h_s + q0, nq * 4, cudaMemcpyHostToDevice, sin);
        if (e == cudaSuccess)
            e = cudaEventRecord(in_done[b], sin);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(scomp, in_done[b], 0);
        if (e == cudaSuccess)
            st = bcf_decode_material(m, du, dv, ds, nq, dout, out_precision, (bcf_stream)scomp);
        if (e == cudaSuccess && st == BCF_OK)
            e = cudaEventRecord(comp_done[b], scomp);
        if (e == cudaSuccess && st == BCF_OK)
            e = cudaStreamWaitEvent(sout, comp_done[b], 0);
        if (e == cudaSuccess && st == BCF_OK)
            e = cudaMemcpyAsync((char *)h_out + q0 * out_b, dout, nq * out_b, cudaMemcpyDeviceToHost, sout);
        if (e == cudaSuccess && st == BCF_OK)
            e = cudaEventRecord(free_ev[b], sout);
        q0 += nq;
    }
    if (e == cudaSuccess && st == BCF_OK)
        e = cudaEventRecord(done, sout);
    if (e == cudaSuccess && st == BCF_OK)
        e = cudaStreamWaitEvent(cs, done, 0); // the caller's stream continues after the last download
    if (st != BCF_OK)
        return st;
    return cuda_status(e, "bcf_decode_material_host");
}

// ------------------------------------------------------------ partition selection encoder

bcf_status bcf_encode_mode10(const float *d_texels, int32_t texel_stride, int32_t res, int32_t levels,
                             float *d_params, uint8_t *d_partitions, float *d_errors, bcf_stream stream)
{
    if (texel_stride != 3 && texel_stride != 4)
        return fail(BCF_ERR_INVALID_ARG, "bcf_encode_mode10: texel_stride %d is not 3 or 4", texel_stride);
    if (!is_pow2(res) || res < 4 || res > 32768)
        return fail(BCF_ERR_INVALID_ARG, "bcf_encode_mode10: res %d is not a power of two in [4, 32768]", res);
    int lg = 0;
    while ((2 << lg) <= res)
        ++lg;
    if (levels < 1 || levels > lg - 1)
        return fail(BCF_ERR_INVALID_ARG, "bcf_encode_mode10: levels %d not in [1, %d]", levels, lg - 1);
    if (!d_texels || !d_params || !d_partitions || !aligned(d_texels, 4) || !aligned(d_params, 16) ||
        (d_errors && !aligned(d_errors, 4)))
        return fail(BCF_ERR_INVALID_ARG, "bcf_encode_mode10: null or misaligned pointer");
    int64_t nb = 0;
    for (int l = 0; l < levels; ++l)
        nb += (int64_t)((res >> l) / 4) * ((res >> l) / 4);
    return cuda_status(launch_encode_mode10(d_texels, texel_stride, res, levels, nb, d_params, d_partitions,
                                            d_errors, (cudaStream_t)stream),
                       "bcf_encode_mode10 launch");
}

bcf_status bcf_compress_bc6h(const float *d_texels, int32_t texel_stride, int32_t res, int32_t levels,
                             void *d_blocks, float *d_errors, uint8_t *d_modes, bcf_stream stream)
{
    if (texel_stride != 3 && texel_stride != 4)
        return fail(BCF_ERR_INVALID_ARG, "bcf_compress_bc6h: texel_stride %d is not 3 or 4", texel_stride);
    if (!is_pow2(res) || res < 4 || res > 32768)
        return fail(BCF_ERR_INVALID_ARG, "bcf_compress_bc6h: res %d is not a power of two in [4, 32768]", res);
    if (levels < 1 || levels > ilog2(res) - 1)
        return fail(BCF_ERR_INVALID_ARG, "bcf_compress_bc6h: levels %d not in [1, %d]", levels, ilog2(res) - 1);
    if (!d_texels || !d_blocks || !aligned(d_texels, 4) || !aligned(d_blocks, 16) ||
        (d_errors && !aligned(d_errors, 4)))
        return fail(BCF_ERR_INVALID_ARG, "bcf_compress_bc6h: null or misaligned pointer");
    int64_t nb = 0;
    for (int l = 0; l < levels; ++l)
        nb += (int64_t)((res >> l) / 4) * ((res >> l) / 4);
    return cuda_status(launch_compress_bc6h(d_texels, texel_stride, res, levels, nb, d_blocks, d_errors, d_modes,
                                            (cudaStream_t)stream),
                       "bcf_compress_bc6h launch");
}

// ------------------------------------------------------------ material sets

} // extern "C"

struct bcf_material_set_s {
    int n;
    bcf::MaterialDev first; // host copy of material 0 (MLP shape and layout of the set)
    bcf::MaterialDev *table; // device table
    int *counter;            // device work counter
    bcf::SetConfig cfg;
    bcf::TexUnitObjs *tex_table; // device table of the materials' texture objects (texture-unit sets)
    int texunit;             // 1: every material was on decode variant 3 at creation
    bool single_geometry;    // decoded by the single-material tile kernel: one geometry group per material and an
                             // MLP shape that kernel has an instance for
    unsigned *check;         // the device's check word (BCF_CHECK_OFFSETS)
};

// The MLP shapes the single-material tile kernel has instances for (launch_tiled_prec): three layers
// K0 -> 32 -> 32 -> C or 32 -> 64 -> 64 -> C (K0 padded to 16, or 32 for E4M3; C padded to 16), or two 16-bit
// layers 16 -> 16 -> C.
static bool geo_shape(const MlpDev &P)
{
    const int kq = P.precision == BCF_FP8_E4M3 ? 32 : 16;
    if (P.n_layers == 3)
        return P.npad[2] == 16 && ((P.kpad[0] == kq && P.npad[0] == 32 && P.npad[1] == 32) ||
                                   (P.kpad[0] == 32 && P.npad[0] == 64 && P.npad[1] == 64));
    return P.n_layers == 2 && P.precision != BCF_FP8_E4M3 && P.kpad[0] == 16 && P.npad[0] == 16 && P.npad[1] == 16;
}

extern "C" {

bcf_status bcf_create_material_set(const bcf_material *mats, int32_t n, bcf_material_set *out)
{
    if (!mats || !out || n < 1 || n > BCF_MAX_SET)
        return fail(BCF_ERR_INVALID_ARG, "bcf_create_material_set: null argument or n = %d not in [1, %d]", n,
                    BCF_MAX_SET);
    *out = nullptr;
    for (int m = 0; m < n; ++m) {
        if (!mats[m])
            return fail(BCF_ERR_INVALID_ARG, "bcf_create_material_set: material %d is null", m);
        const MaterialDev &A = mats[0]->host, &B = mats[m]->host;
        bool same = A.n_tex == B.n_tex && A.lod_input == B.lod_input && A.mlp.n_layers == B.mlp.n_layers &&
                    A.mlp.precision == B.mlp.precision;
        for (int l = 0; same && l <= A.mlp.n_layers; ++l)
            same = A.mlp.dims[l] == B.mlp.dims[l];
        if (!same)
            return fail(BCF_ERR_INVALID_ARG, "bcf_create_material_set: material %d does not share the MLP / textures",
                        m);
    }
    if (mats[0]->host.mlp.precision == BCF_FP32)
        return fail(BCF_ERR_UNSUPPORTED, "bcf_create_material_set: FP32 materials use bcf_decode_material");
    bcf_material_set set = new (std::nothrow) bcf_material_set_s;
    if (!set)
        return fail(BCF_ERR_OOM, "host allocation failed");
    set->n = n;
    set->first = mats[0]->host;
    set->table = nullptr;
    set->counter = nullptr;
    set->cfg = {320, 3, 2};
    set->tex_table = nullptr;
    set->texunit = set_tex_supported(mats[0]->host);
    for (int m = 0; m < n; ++m)
        set->texunit = set->texunit && mats[m]->hw_ready && mats[m]->variant == 3;
    set->single_geometry = geo_shape(mats[0]->host.mlp);
    for (int m = 0; m < n; ++m)
        set->single_geometry = set->single_geometry && mats[m]->host.n_groups == 1;
    if (set->texunit)
        set->cfg = {320, 6, 32}; // the autotuner's pick on the 64-material benchmark workload
    else if (set->single_geometry)
        set->cfg = {0, 2, 2}; // the single-geometry kernel (arena fixed by its tile): two CTAs of 512 queries per SM
    MaterialDev *host = new (std::nothrow) MaterialDev[n];
    if (!host) {
        delete set;
        return fail(BCF_ERR_OOM, "host allocation failed");
    }
    for (int m = 0; m < n; ++m)
        host[m] = mats[m]->host;
    set->check = check_word();
    cudaError_t e = set->check ? cudaMalloc(&set->table, sizeof(MaterialDev) * n) : cudaErrorMemoryAllocation;
    if (e == cudaSuccess)
        e = cudaMalloc(&set->counter, sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemcpy(set->table, host, sizeof(MaterialDev) * n, cudaMemcpyHostToDevice);
    delete[] host;
    if (e == cudaSuccess && set->texunit) {
        TexUnitObjs *th = new (std::nothrow) TexUnitObjs[n];
        if (!th)
            e = cudaErrorMemoryAllocation;
        for (int m = 0; th && m < n; ++m)
            th[m] = mats[m]->hw;
        if (e == cudaSuccess)
            e = cudaMalloc(&set->tex_table, sizeof(TexUnitObjs) * n);
        if (e == cudaSuccess)
            e = cudaMemcpy(set->tex_table, th, sizeof(TexUnitObjs) * n, cudaMemcpyHostToDevice);
        delete[] th;
    }
    if (e != cudaSuccess) {
        cudaFree(set->table);
        cudaFree(set->counter);
        cudaFree(set->tex_table);
        delete set;
        return fail(BCF_ERR_OOM, "bcf_create_material_set: %s", cudaGetErrorString(e));
    }
    *out = set;
    return BCF_OK;
}

bcf_status bcf_destroy_material_set(bcf_material_set set)
{
    if (!set)
        return BCF_OK;
    cudaError_t e = cudaFree(set->table);
    cudaError_t e2 = cudaFree(set->counter);
    cudaFree(set->tex_table);
    delete set;
    return cuda_status(e != cudaSuccess ? e : e2, "bcf_destroy_material_set");
}

static bcf_status check_set_args(bcf_material_set set, const int64_t *d_offsets, const float *d_u, const float *d_v,
                                 const float *d_s, int64_t n, void *d_out, bcf_precision out_precision)
{
    if (!set || n < 0 || !d_offsets)
        return fail(BCF_ERR_INVALID_ARG, "material set decode: null set / offsets or n < 0");
    if (out_precision != BCF_FP32 && out_precision != BCF_FP16)
        return fail(BCF_ERR_INVALID_ARG, "material set decode: out_precision must be FP32 or FP16");
    if (n > 0 && (!d_u || !d_v || !d_out || !aligned(d_u, 4) || !aligned(d_v, 4) || !aligned(d_out, 16) ||
                  (d_s && !aligned(d_s, 4)) || !aligned(d_offsets, 8)))
        return fail(BCF_ERR_INVALID_ARG, "material set decode: null or misaligned pointer");
    return BCF_OK;
}

bcf_status bcf_decode_material_set(bcf_material_set set, const int64_t *d_offsets, const float *d_u, const float *d_v,
                                   const float *d_s, int64_t n_queries, void *d_out, bcf_precision out_precision,
                                   bcf_stream stream)
{
    bcf_status st = check_set_args(set, d_offsets, d_u, d_v, d_s, n_queries, d_out, out_precision);
    if (st != BCF_OK || n_queries == 0)
        return st;
    if (set->texunit)
        return cuda_status(launch_decode_set_tex(set->first, set->table, set->tex_table, set->n, d_offsets, d_u, d_v,
                                                 d_s, n_queries, d_out, out_precision == BCF_FP16, set->counter,
                                                 set->check, set->cfg, (cudaStream_t)stream),
                           "bcf_decode_material_set launch");
    return cuda_status(launch_decode_set(set->first, set->table, set->n, d_offsets, d_u, d_v, d_s, n_queries, d_out,
                                         out_precision == BCF_FP16, set->counter, set->check, set->cfg,
                                         set->single_geometry, (cudaStream_t)stream),
                       "bcf_decode_material_set launch");
}

bcf_status bcf_material_set_config(bcf_material_set set, int32_t *cap, int32_t *ctas_per_sm, int32_t *chunk)
{
    if (!set)
        return fail(BCF_ERR_INVALID_ARG, "bcf_material_set_config: null set");
    if (cap)
        *cap = set->cfg.cap;
    if (ctas_per_sm)
        *ctas_per_sm = set->cfg.ctas_per_sm;
    if (chunk)
        *chunk = set->cfg.chunk;
    return BCF_OK;
}

bcf_status bcf_autotune_material_set(bcf_material_set set, const int64_t *d_offsets, const float *d_u,
                                     const float *d_v, const float *d_s, int64_t n_queries, void *d_out,
                                     bcf_precision out_precision, bcf_stream stream, int32_t *cap,
                                     int32_t *ctas_per_sm, int32_t *chunk)
{
    bcf_status st = check_set_args(set, d_offsets, d_u, d_v, d_s, n_queries, d_out, out_precision);
    if (st != BCF_OK)
        return st;
    cudaStream_t cs = (cudaStream_t)stream;
    if (n_queries > 0) {
        cudaEvent_t a = nullptr, b = nullptr;
        cudaError_t e = cudaEventCreate(&a);
        if (e == cudaSuccess)
            e = cudaEventCreate(&b);
        float best = 1e30f;
        SetConfig best_cfg = set->cfg;
        // the software set kernel: arena size x CTAs per SM x tiles per grab; the texture-unit set kernel
        // (128-query tiles): CTAs per SM x tiles per grab
        // tiles per grab: the texture-unit kernel's tiles are one warp's 32 queries
        const int caps[2] = {256, 320}, ctas_sw[3] = {1, 2, 3}, ctas_tex[3] = {4, 6, 8}, chunks_sw[4] = {1, 2, 4, 8},
                  chunks_tex[4] = {8, 16, 32, 64};
        const int ncap = set->texunit || set->single_geometry ? 1 : 2; // the tile kernel's arena is fixed
        for (int ic = 0; e == cudaSuccess && ic < ncap; ++ic)
            for (int ir = 0; e == cudaSuccess && ir < 3; ++ir)
                for (int ik = 0; e == cudaSuccess && ik < 4; ++ik) {
                    const SetConfig cfg = {set->single_geometry && !set->texunit ? 0 : caps[ic],
                                           set->texunit ? ctas_tex[ir] : ctas_sw[ir],
                                           set->texunit ? chunks_tex[ik] : chunks_sw[ik]};
                    float ms = 0.0f;
                    for (int rep = 0; e == cudaSuccess && rep < 3; ++rep) { // first run warms up
                        e = cudaEventRecord(a, cs);
                        if (e == cudaSuccess)
                            e = set->texunit
                                    ? launch_decode_set_tex(set->first, set->table, set->tex_table, set->n, d_offsets,
                                                            d_u, d_v, d_s, n_queries, d_out, out_precision == BCF_FP16,
                                                            set->counter, set->check, cfg, cs)
                                    : launch_decode_set(set->first, set->table, set->n, d_offsets, d_u, d_v, d_s,
                                                        n_queries, d_out, out_precision == BCF_FP16, set->counter,
                                                        set->check, cfg, set->single_geometry, cs);
                        if (e == cudaSuccess)
                            e = cudaEventRecord(b, cs);
                        if (e == cudaSuccess)
                            e = cudaEventSynchronize(b);
                        float t = 0.0f;
                        if (e == cudaSuccess)
                            e = cudaEventElapsedTime(&t, a, b);
                        if (rep > 0)
                            ms += t;
                    }
                    if (e == cudaSuccess && ms < best) {
                        best = ms;
                        best_cfg = cfg;
                    }
                }
        if (a)
            cudaEventDestroy(a);
        if (b)
            cudaEventDestroy(b);
        if (e != cudaSuccess)
            return cuda_status(e, "bcf_autotune_material_set");
        set->cfg = best_cfg;
    }
    return bcf_material_set_config(set, cap, ctas_per_sm, chunk);
}

} // extern "C"
