/*
 * bcf.h -- C ABI of libbcf, a B300 (sm_103a) implementation of the decode and
 * training hot path of "Real-Time Neural Materials using Block-Compressed
 * Features" (Weinreich, de Oliveira, Houdard, Nader; arXiv 2311.16121).
 *
 * A neural material is a set of BC6H-compressed feature textures T_i with
 * mip chains plus a small MLP f_eta (Eq. 3, Sec. 3).  For a query (u, v, s)
 * the library unpacks the BC6H blocks it needs (Sec. 4.1-4.2 and the BC6H
 * format they reference), filters every texture trilinearly at a per-texture
 * LOD (Eq. 10, Eq. 11), concatenates the filtered features (and the query
 * LOD) and evaluates the MLP (ReLU hidden layers, linear output).  Training
 * emulates BC6 mode-10 decompression on per-block parameters (Eq. 6-9) with
 * a hand-written forward and backward pass.
 *
 * Conventions shared by every entry point:
 *   - Every pointer named d_* is a device pointer on the current CUDA device;
 *     the caller allocates and owns it.  Pointers named h_* are host memory.
 *   - Every call is asynchronous on the given stream (0 = legacy default
 *     stream) and performs no device allocation, no host synchronisation and
 *     no implicit copy, except where a function says otherwise.  Results are
 *     visible after the stream is synchronised.
 *   - Every function returns a bcf_status and never aborts.  Invalid
 *     arguments are detected on the host before anything is launched; a
 *     failed launch returns BCF_ERR_CUDA.  bcf_last_error() gives a
 *     thread-local text for the last failure.
 *   - Textures are square, power-of-two sized (>= 4 texels) and store their
 *     mip levels concatenated from level 0, each level as row-major 16-byte
 *     BC6H blocks; level l is (res >> l) texels wide.  Block pointers must be
 *     16-byte aligned.
 *   - Texel centres sit at ((i + 0.5) / W, (j + 0.5) / W); u selects the
 *     column, v the row.
 */
#ifndef BCF_H_
#define BCF_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BCF_MAX_TEX 16    /* feature textures per material */
#define BCF_MAX_LEVELS 16 /* mip levels per texture */
#define BCF_MAX_LAYERS 8  /* MLP layers */
#define BCF_MAX_WIDTH 128 /* MLP layer width (inputs, hidden, outputs) */

typedef enum {
    BCF_OK = 0,
    BCF_ERR_INVALID_ARG = 1,  /* a size, pointer, alignment or descriptor field is invalid */
    BCF_ERR_UNSUPPORTED = 2,  /* valid but outside what this build implements */
    BCF_ERR_CUDA = 3,         /* a CUDA runtime call or kernel launch failed */
    BCF_ERR_OOM = 4,          /* a create-time allocation failed */
    BCF_ERR_TIMEOUT = 5,      /* a bounded device-side wait ran out */
    BCF_ERR_DEVICE_CHECK = 6  /* a device-side consistency check failed */
} bcf_status;

typedef enum {
    BCF_FP32 = 0,     /* plain FP32 SIMT evaluation */
    BCF_FP16 = 1,     /* FP16 operands on tensor cores, FP32 accumulation */
    BCF_BF16 = 2,     /* BF16 operands on tensor cores, FP32 accumulation */
    BCF_FP8_E4M3 = 3  /* OCP E4M3 operands with per-layer scales, FP32 accumulation */
} bcf_precision;

typedef void *bcf_stream; /* a cudaStream_t */

/* ------------------------------------------------------------------ status */

const char *bcf_status_string(bcf_status s);
/* Text of the last failure on the calling thread ("" if none). */
const char *bcf_last_error(void);
/* Library version as major * 10000 + minor * 100 + patch. */
int bcf_version(void);

/* ------------------------------------------------------------ BC6H unpack */

/*
 * bcf_decode_bc6h -- decode a whole BC6H image (Sec. 4.1-4.2: the paper's
 * block format, whose exact bitstream the BC6H definition it cites fixes).
 *
 * d_blocks : blocks_h rows of blocks_w 16-byte BC6H blocks, row-major,
 *            16-byte aligned, blocks_w * blocks_h * 16 bytes.
 * is_signed: 0 = BC6H unsigned half (UF16), 1 = signed half (SF16).
 * d_out    : [4 * blocks_h][4 * blocks_w][3] uint16 IEEE half bit patterns
 *            (R, G, B per texel), 8-byte aligned.
 * All 14 modes are decoded bit-exactly; the four reserved mode values
 * decode to zero.  blocks_w * blocks_h == 0 is a no-op.
 * Errors: BCF_ERR_INVALID_ARG for negative sizes, null or misaligned
 * pointers, or more than 2^31 blocks.
 */
bcf_status bcf_decode_bc6h(const void *d_blocks, int32_t blocks_w, int32_t blocks_h, int32_t is_signed, uint16_t *d_out,
                           bcf_stream stream);

/*
 * bcf_texunit_decode_bc6h -- the same image decoded by the GPU's texture
 * unit (a BC6H texture object sampled at texel centres with point
 * filtering).  It is an independent statement of the format used to check
 * bcf_decode_bc6h and the CPU oracle; it allocates and frees a CUDA array
 * and synchronises the stream, so it is not for hot paths.
 * Arguments and output as bcf_decode_bc6h.
 */
bcf_status bcf_texunit_decode_bc6h(const void *d_blocks, int32_t blocks_w, int32_t blocks_h, int32_t is_signed,
                                   uint16_t *d_out, bcf_stream stream);

/* ----------------------------------------------------------------- material */

typedef struct bcf_material_s *bcf_material;

typedef struct {
    int32_t num_textures;           /* 1 <= T <= BCF_MAX_TEX */
    int32_t res[BCF_MAX_TEX];       /* level-0 width = height, power of two, >= 4 */
    int32_t levels[BCF_MAX_TEX];    /* 1 <= L_t <= log2(res) - 1 (the last level is one 4x4 block) */
    int32_t res_ref;                /* power of two; the query LOD s is in units of this resolution, and
                                       texture t is sampled at s_t = s + log2(res_t / res_ref) (Eq. 11) */
    int32_t is_signed;              /* 0 = BC6H UF16, 1 = SF16 */
    int32_t wrap;                   /* 1 = repeat addressing, 0 = clamp to edge */
    int32_t lod_input;              /* 1 = the query LOD max(s, 0) is the last MLP input */
    const void *d_blocks[BCF_MAX_TEX]; /* texture blocks, mips concatenated from level 0 */
    int32_t n_layers;               /* 1 <= n <= BCF_MAX_LAYERS */
    int32_t dims[BCF_MAX_LAYERS + 1]; /* dims[0] = 3 T + lod_input, ..., dims[n] = output channels C */
    bcf_precision precision;        /* storage format of d_weights and arithmetic of the MLP */
    const void *d_weights;          /* per layer W_l [dims[l+1]][dims[l]] row-major, layers concatenated, in
                                       `precision` (FP32 / FP16 / BF16 / E4M3 bytes) */
    const float *d_biases;          /* per layer b_l [dims[l+1]], FP32, concatenated */
    float act_scale[BCF_MAX_LAYERS]; /* FP8 only: layer l's input is quantised as E4M3(x / act_scale[l]) */
    float w_scale[BCF_MAX_LAYERS];   /* FP8 only: layer l's weights are E4M3(W / w_scale[l]) */
} bcf_material_desc;

/*
 * bcf_create_material -- validate a material (Eq. 3: feature textures plus
 * the MLP decoder) and build its metadata (per-level block offsets, LOD
 * biases, padded weight layouts).  Allocates a small device metadata block
 * (freed by bcf_destroy_material) and copies it synchronously.  Texture
 * blocks, weights and biases stay caller-owned and must outlive the
 * material.  Errors: BCF_ERR_INVALID_ARG (any field out of range, dims[0]
 * != 3 T + lod_input, misaligned pointers), BCF_ERR_UNSUPPORTED (a layer
 * wider than BCF_MAX_WIDTH, or an FP8 scale that is not a power of two),
 * BCF_ERR_OOM / BCF_ERR_CUDA.
 */
bcf_status bcf_create_material(const bcf_material_desc *desc, bcf_material *out);
bcf_status bcf_destroy_material(bcf_material mat);

/*
 * bcf_sample_features -- T_t(u, v, s) for every texture t of the material,
 * concatenated (Eq. 10 with the per-texture LOD of Eq. 11): BC6H unpack
 * plus exact FP32 bilinear filtering on levels floor(s_t) and floor(s_t)+1,
 * lerped by the fractional part; s_t is clamped to [0, L_t - 1].
 * d_u, d_v, d_s: n FP32 each (d_s may be NULL: s = 0).  NaN coordinates
 * read as 0; with repeat addressing u and v wrap to [0, 1).
 * d_feat: [n][3 T] FP32, 16-byte aligned.  n == 0 is a no-op.
 */
bcf_status bcf_sample_features(bcf_material mat, const float *d_u, const float *d_v, const float *d_s, int64_t n,
                               float *d_feat, bcf_stream stream);

/*
 * bcf_decode_material -- G(u, v, s) = f_eta(T_0, ..., T_{T-1}[, s]) (Eq. 3)
 * for n queries of one material: BC6H unpack, trilinear filtering and the
 * MLP in one kernel.  The MLP runs in the material's precision: FP32 on the
 * SIMT cores, FP16 / BF16 / FP8 E4M3 on the tensor cores with FP32
 * accumulation (each layer's input rounded to the precision, FP8 divided by
 * the layer's act_scale first; products scaled back by act_scale * w_scale;
 * FP32 bias; ReLU on hidden layers).
 * d_out: [n][C] in out_precision (BCF_FP32 or BCF_FP16), 16-byte aligned.
 * Errors: BCF_ERR_INVALID_ARG for null / misaligned pointers, n < 0, or an
 * out_precision other than FP32 / FP16.
 */
bcf_status bcf_decode_material(bcf_material mat, const float *d_u, const float *d_v, const float *d_s, int64_t n,
                               void *d_out, bcf_precision out_precision, bcf_stream stream);

/*
 * bcf_set_decode_variant -- choose the kernel bcf_decode_material uses for a
 * tensor-core (FP16 / BF16 / FP8) material.  0 (default): tile-cooperative
 * decode -- 256 screen-coherent queries share one decode of each BC6H block
 * their footprints touch (blocks mode-sorted, texels staged in shared
 * memory); falls back per tile to 1 when the tile's blocks do not fit.
 * 1: per-lane decode -- every query decodes the blocks of its own
 * footprints.  Both compute the same values.  FP32 materials always use the
 * per-lane SIMT path.  Errors: BCF_ERR_INVALID_ARG for a null material or
 * another variant.
 */
bcf_status bcf_set_decode_variant(bcf_material mat, int32_t variant);

#ifdef __cplusplus
}
#endif
#endif /* BCF_H_ */
