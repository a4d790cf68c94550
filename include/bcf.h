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
    BCF_ERR_UNSUPPORTED = 2,  /* valid but outside what the library implements */
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

/*
 * Device-side checks.  Some conditions can only be seen by the kernels, on
 * data that lives on the device: those kernels set a bit of a 32-bit check
 * word (one per device, created with the first material set or trainer)
 * with an atomic OR, take the documented safe reading of the data and carry
 * on.  Nothing is reported until the caller asks:
 *
 *   BCF_CHECK_PARTITION  a training block's partition id (d_partition) is
 *                        above 31; the block is read, trained and exported
 *                        with id & 31.  Checked by the optimiser of
 *                        bcf_train_step / bcf_train_step_noalloc and by
 *                        the export (bcf_train_forward / _backward only
 *                        mask).
 *   BCF_CHECK_OFFSETS    material-set query offsets decrease
 *                        (d_offsets[m+1] < d_offsets[m]); that material's
 *                        range is decoded as empty.
 *   BCF_CHECK_TIMEOUT    a bounded wait of a decode for its tcgen05 MMAs
 *                        ran out (bcf_set_mlp_engine, BCF_MLP_TCGEN05); the
 *                        kernel stopped taking tiles, so part of the output
 *                        is missing.
 */
#define BCF_CHECK_PARTITION 0x1u
#define BCF_CHECK_OFFSETS 0x2u
#define BCF_CHECK_TIMEOUT 0x4u

/*
 * bcf_device_check -- wait for all work on the current device (every
 * stream), then read and clear its check word.  Returns BCF_OK if no check
 * fired, else BCF_ERR_DEVICE_CHECK with bcf_last_error() naming the checks.
 * h_word (may be NULL) receives the word.  Like cudaDeviceSynchronize, this
 * blocks the host; launches made by other host threads while it runs may
 * land on either side of the read.
 */
bcf_status bcf_device_check(uint32_t *h_word);

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
 * bcf_decode_material_host -- bcf_decode_material for queries and outputs in
 * host memory (page-locked memory gives overlapped copies; pageable memory
 * works but serialises).  The n queries are processed in chunks through three
 * rotating buffers carved from the caller's device scratch; the upload of
 * the next chunk, the decode of the current one and the download of the
 * previous one run concurrently on three library streams, ordered after the
 * work already on `stream`, and `stream` waits for the last download, so the
 * call is asynchronous like the others (h_out is complete once `stream`
 * reaches that point).  Each chunk is a multiple of 256 queries: a chunk needs
 * 3 x (8 + 4 [with s] + C x out bytes) per query plus 1 KB per buffer of
 * alignment; the chunk size is the largest the scratch allows, up to n / 4
 * (a 128 MB scratch gives six chunks for a 3840 x 2160 frame of FP16
 * outputs).
 * h_u, h_v, h_s (may be NULL when the material has no LOD input): n floats;
 * h_out: [n][C] in out_precision.  The three streams and eleven events of
 * the pipeline belong to the material: the first call creates them (the
 * only allocation), bcf_destroy_material releases them.  Calls on one
 * material therefore must not overlap (issue them from one host thread, or
 * serialise them); later calls create nothing.
 * Errors: BCF_ERR_INVALID_ARG for null pointers, scratch not 256-byte aligned
 * or too small for one 256-query chunk; the errors of bcf_decode_material;
 * BCF_ERR_CUDA.
 */
bcf_status bcf_decode_material_host(bcf_material mat, const float *h_u, const float *h_v, const float *h_s, int64_t n,
                                    void *h_out, bcf_precision out_precision, void *d_scratch, int64_t scratch_bytes,
                                    bcf_stream stream);

/* ------------------------------------------------------------ material sets */

/*
 * A material set decodes many materials in one launch (Sec. 5.2: several
 * materials' networks in one buffer, indexed by material id).  All
 * materials of a set must share the MLP (precision, layer count and
 * widths, LOD input) and the texture count; textures may differ in
 * resolution and levels.  At most BCF_MAX_SET materials.
 */
#define BCF_MAX_SET 256
typedef struct bcf_material_set_s *bcf_material_set;

/*
 * bcf_create_material_set -- copy the materials' metadata into one device
 * table and allocate the set's work counter (freed by
 * bcf_destroy_material_set; synchronous).  The materials must outlive the
 * set.  When every material is on decode variant 3 at creation (see
 * bcf_set_decode_variant) and the MLP is one of the register-chained shapes
 * (three layers, K0 <= 16 (FP8: 32) -> 32 -> 32 -> C <= 16, or
 * K0 <= 32 -> 64 -> 64 -> C <= 16), the set decodes through the texture unit
 * the same way (texture-unit texels, exact FP32 filter) with a persistent
 * kernel whose warps each take 32-query tiles (bcf_autotune_material_set
 * picks its CTAs per SM and tiles per grab); otherwise it uses the library's own BC6H decode:
 * for the register-chained shapes, the tile kernel of bcf_decode_material
 * (tiles of 512 queries, 256 for 16-bit 64-wide MLPs; each material's
 * textures of one resolution and level count), else the multi-group tile
 * decode (256-query tiles).
 * Errors: BCF_ERR_INVALID_ARG (n out of [1, BCF_MAX_SET], null
 * materials, materials that do not share the MLP / texture count),
 * BCF_ERR_UNSUPPORTED (FP32 materials: the set path is the tensor-core
 * path), BCF_ERR_OOM / BCF_ERR_CUDA.
 */
bcf_status bcf_create_material_set(const bcf_material *mats, int32_t n, bcf_material_set *out);
bcf_status bcf_destroy_material_set(bcf_material_set set);

/*
 * bcf_decode_material_set -- bcf_decode_material for every material of the
 * set in one persistent launch.  The queries of all materials are
 * concatenated: material m's queries are [d_offsets[m], d_offsets[m+1]) of
 * d_u / d_v / d_s (and of the rows of d_out [n_queries][C]).  d_offsets:
 * n + 1 non-decreasing int64 on the device (entries are clipped to
 * [0, n_queries]; a decreasing pair sets BCF_CHECK_OFFSETS).  Queries are
 * processed in tiles (see bcf_create_material_set; a tile never spans two
 * materials) taken from an
 * atomic work counter that a memset before the launch resets, so the call
 * can be captured into a CUDA graph and replayed.  Calls on one set must
 * not overlap on the GPU (they share the counter).  Errors as
 * bcf_decode_material.
 */
bcf_status bcf_decode_material_set(bcf_material_set set, const int64_t *d_offsets, const float *d_u, const float *d_v,
                                   const float *d_s, int64_t n_queries, void *d_out, bcf_precision out_precision,
                                   bcf_stream stream);

/*
 * bcf_autotune_material_set -- time the set-decode launch configurations
 * (sets on the tile kernel of bcf_decode_material: 1-3 persistent CTAs per
 * SM, capped by residency, *cap = 0 since its arena is fixed by its tile;
 * multi-group software sets: shared-memory block arena 256 / 320 blocks,
 * 1-3 CTAs per SM; texture-unit sets: 4 / 6 / 8 CTAs per SM, capped by
 * occupancy, and 8 / 16 / 32 / 64 warp tiles per grab; the others: 1 / 2 / 4 /
 * 8 tiles per work-counter grab) on the given
 * workload with
 * CUDA events (synchronises the stream; the output is overwritten), keep the
 * fastest for the set, and return it in *cap, *ctas_per_sm, *chunk (any may
 * be NULL).  bcf_material_set_config reads the current configuration.
 */
bcf_status bcf_autotune_material_set(bcf_material_set set, const int64_t *d_offsets, const float *d_u,
                                     const float *d_v, const float *d_s, int64_t n_queries, void *d_out,
                                     bcf_precision out_precision, bcf_stream stream, int32_t *cap,
                                     int32_t *ctas_per_sm, int32_t *chunk);
bcf_status bcf_material_set_config(bcf_material_set set, int32_t *cap, int32_t *ctas_per_sm, int32_t *chunk);

/* ----------------------------------------------------------------- training */

/*
 * Training of a block-compressed neural material (Sec. 4.1-4.3, Sec. 5.1,
 * Eq. 4-9): per-block parameters theta (Eq. 6) and the MLP eta are fitted to
 * a filtered reference F(M) with the MSE of Eq. 5 and Adam (Sec. 6.1).
 *
 * Block parameter layout (one 128-byte record per block, mips concatenated
 * from level 0, blocks row-major per level), 32 floats:
 *   [0..2]  e1 RGB, [3..5] e2 RGB   endpoints of region 0, in 6-bit units [0, 63]
 *   [6..7]  unused (kept 0)
 *   [8..10] e3 RGB, [11..13] e4 RGB endpoints of region 1
 *   [14..15] unused (kept 0)
 *   [16..31] x_1..x_16             per-texel positions on the segment, [0, 1]
 * plus one partition id k in [0, 31] per block (uint8, fixed during training;
 * a larger id sets BCF_CHECK_PARTITION and reads as k & 31).
 *
 * Forward (the emulated BC6 decompression of Sec. 4.2 at the exported
 * precision of Sec. 5.2, i.e. BC6H mode 10): endpoints and x are rounded to
 * the 6-bit / 3-bit lattice (straight-through), unquantised, interpolated
 * with the 3-bit weights and scaled by 31/64 exactly as the BC6H decoder
 * does, and the 15-bit result is read as a half float (Eq. 9), so the
 * forward equals the decode of the exported block bit for bit.  Backward:
 * the exact derivatives of the relaxed pipeline (Eq. 7 slope 1024 per
 * endpoint unit, Eq. 8 linear in w/64 ~ x, 31/64, slope of Eq. 9) at the
 * rounded forward values; zero outside [0, 63] / [0, 1].
 * The MLP evaluates with weights and layer inputs rounded to bfloat16 and
 * FP32 accumulation; its backward is FP32 with respect to those rounded
 * values.
 *
 * Signed features (is_signed = 1, Sec. 4.2 with a = 31/32): endpoints are
 * 6-bit two's complement codes in [-32, 31] (the box of the optimiser),
 * unquantised and finished as the BC6H signed format does (sign carried,
 * Eq. 9 on the magnitude), exported as SF16 mode-10 blocks.
 *
 * Literal emulation (literal = 1): the forward evaluates Eq. 7 and Eq. 8
 * exactly as printed on the rounded codes -- unquantisation
 * (a 2^16 e + 2^15) / 2^6 with no special cases for the smallest and
 * largest codes, real interpolation with weight w / 64, no floors -- and
 * Eq. 9 on that real value; the backward is that function's derivative.
 * It differs from the decode of the exported block (the 2^15 term is not
 * scaled by a), which is why the exact form is the default.
 *
 * Unconstrained features (unconstrained = 1; the first training stage of
 * Sec. 5.1, whose result bcf_encode_mode10 compresses into the initial block
 * parameters and partitions): each texture holds free RGB values per texel,
 * [texels][4] floats (R, G, B, unused 0), mips concatenated from level 0,
 * texels row-major per level; d_params, d_grad, d_adam_m, d_adam_v have
 * that layout, d_partition is ignored, the texel values are filtered
 * trilinearly (Eq. 10) without any compression emulation or bound, and
 * bcf_train_export does not apply.  Supported for MLPs dims[0] <= 16 ->
 * 32 -> 32 -> C and for the paper's two-layer dims[0] <= 16 -> 16 -> C
 * (C <= 9; BCF_ERR_UNSUPPORTED otherwise).
 *
 * Kernels: those two MLP shapes train on the tensor cores (BF16 products,
 * FP32 sums, the output gradient split into two BF16 terms); other shapes
 * on a SIMT kernel with the same rounding of weights and layer inputs.
 *
 * Reference material F(M) (Sec. 5.1): 9 channels, FP16, a mip chain from
 * target_res down to 4 x 4 (level l is target_res >> l), channels 0..7
 * interleaved [texels][8] and channel 8 in its own array [texels]; sampled
 * with Catmull-Rom bicubic filtering on levels floor(s) and floor(s) + 1,
 * lerped, repeat addressing.
 */
typedef struct bcf_trainer_s *bcf_trainer;

typedef struct {
    int32_t num_textures;                   /* T */
    int32_t res[BCF_MAX_TEX];
    int32_t levels[BCF_MAX_TEX];
    int32_t res_ref;                        /* query LOD s is in units of res_ref (the reference's resolution) */
    int32_t lod_input;                      /* 1: max(s, 0) is the last MLP input */
    float *d_params[BCF_MAX_TEX];           /* [blocks][32] block parameters, updated in place by the optimiser */
    const uint8_t *d_partition[BCF_MAX_TEX]; /* [blocks] partition ids */
    float *d_grad[BCF_MAX_TEX];             /* [blocks][32] gradient accumulators (zeroed by the optimiser) */
    float *d_adam_m[BCF_MAX_TEX];           /* [blocks][32] Adam first moments */
    float *d_adam_v[BCF_MAX_TEX];           /* [blocks][32] Adam second moments */
    int32_t n_layers;                       /* 1 <= n <= BCF_MAX_LAYERS, widths <= 64 */
    int32_t dims[BCF_MAX_LAYERS + 1];       /* dims[0] = 3 T + lod_input */
    float *d_W, *d_b;                       /* FP32 master weights (layers concatenated, W_l [out][in]) */
    float *d_W_grad, *d_b_grad;             /* their gradient accumulators */
    float *d_W_m, *d_W_v, *d_b_m, *d_b_v;   /* Adam moments */
    int32_t target_res, target_levels;
    const uint16_t *d_target8;              /* FP16 channels 0..7 of the reference, [texels][8] */
    const uint16_t *d_target1;              /* FP16 channel 8, [texels] */
    float lr_features, lr_mlp;              /* initial learning rates (Sec. 6.1: 1e-2 and 1e-3) */
    float gamma;                            /* exponential decay per step (Sec. 6.1: 0.9999) */
    float beta1, beta2, eps;                /* Adam constants */
    float s_max;                            /* batch draws: s ~ U[0, s_max) in res_ref units */
    int32_t unconstrained;                  /* 1: free per-texel features (see below) instead of block parameters */
    int32_t is_signed;                      /* 1: BC6H signed (SF16) features: endpoints in [-32, 31], a = 31/32 */
    int32_t literal;                        /* 1: Eq. 7-8 as printed instead of the format's exact steps (below) */
    int32_t batch_grid;                     /* > 0: step batches are batch_grid^2 uv grids (below); 0: random */
} bcf_trainer_desc;

/*
 * bcf_trainer_create -- validate a trainer (sizes, alignment: every array
 * 16-byte aligned) and copy its metadata to the device (a small allocation
 * freed by bcf_trainer_destroy).  All parameter, gradient, moment and
 * target arrays stay caller-owned.  Errors: BCF_ERR_INVALID_ARG,
 * BCF_ERR_UNSUPPORTED (a layer wider than 64, a target not 9 channels),
 * BCF_ERR_OOM / BCF_ERR_CUDA.
 */
bcf_status bcf_trainer_create(const bcf_trainer_desc *desc, bcf_trainer *out);
bcf_status bcf_trainer_destroy(bcf_trainer tr);

/*
 * bcf_train_step -- one optimisation step (Eq. 5 on one batch, then Adam):
 *   queries: (d_u, d_v, d_s) of length `batch` if given, otherwise drawn with
 *   Philox4x32-10: counter (q, step low, step high, q high), key (seed low,
 *   seed high); u, v, s = top 24 bits of output words 0, 1, 2 times 2^-24
 *   (s also times s_max).  With batch_grid = G > 0 (the paper's batches,
 *   Sec. 5.1: a uniformly sampled uv grid with one scale per batch) the batch
 *   must be G^2 and query q = j G + i sits at ((i + o_u) / G, (j + o_v) / G)
 *   with one (o_u, o_v, s) per step from the counter (2^32 - 1, step low,
 *   step high, 2^32 - 1), single-precision arithmetic;
 *   loss: mean over batch and channels of (G - F(M))^2, written to
 *   d_loss_out (one float, device; overwritten);
 *   gradients accumulated into the trainer's grad arrays, then Adam with
 *   lr_t = lr0 gamma^step, bias correction with step + 1, endpoints clamped
 *   to [0, 63] and x to [0, 1]; gradients are zeroed afterwards.
 * batch == 0 only runs the optimiser on zero gradients.  Errors:
 * BCF_ERR_INVALID_ARG for batch < 0, step < 0, a null loss pointer, or a
 * grid trainer's batch other than G^2.
 */
bcf_status bcf_train_step(bcf_trainer tr, int64_t batch, uint64_t seed, int64_t step, const float *d_u,
                          const float *d_v, const float *d_s, float *d_loss_out, bcf_stream stream);

/*
 * bcf_train_forward -- G(u, v, s) of the current parameters for n queries
 * (the emulated forward above), d_out [n][C] FP32.
 * bcf_train_backward -- given dL/dG [n][C] FP32 for the same queries,
 * accumulate dL/dtheta and dL/deta into the trainer's gradient arrays
 * (nothing is zeroed and no optimiser step is taken).
 * Together they are the forward / backward of a torch.autograd.Function.
 */
bcf_status bcf_train_forward(bcf_trainer tr, const float *d_u, const float *d_v, const float *d_s, int64_t n,
                             float *d_out, bcf_stream stream);
bcf_status bcf_train_backward(bcf_trainer tr, const float *d_u, const float *d_v, const float *d_s, int64_t n,
                              const float *d_grad_out, bcf_stream stream);

/*
 * bcf_train_step_noalloc -- bcf_train_step for callers that cannot allocate
 * device memory: engines and real-time hosts that own every device byte
 * through their own budgeted allocator, or whose frame loop must not call
 * cudaMalloc (it can synchronise the device and fails once the budget is
 * reached).  The paper has no counterpart; this is a property of the
 * library's interface.
 *
 * It computes the same step as bcf_train_step (same arguments, same loss,
 * parameter, weight and moment updates), but the gradient accumulators --
 * scratch that lives only between the gradient kernel and the optimiser
 * kernel -- are kept in one library-owned device array of
 * BCF_NOALLOC_MAX_GRAD_FLOATS floats (4 MiB) that every GPU which loads
 * the library holds until the process exits.  The trainer's own gradient
 * arrays are neither read nor written.  Nothing is allocated: the array's
 * device address is looked up once per device (cudaGetSymbolAddress) on the
 * first call made with that device current, so make that first call before
 * any stream capture.  Every call zeroes the part of the array it uses
 * before accumulating (the array keeps the last call's contents).  All calls
 * on a device share the one array: calls whose work overlaps on the GPU
 * (different streams, or different threads) race and give wrong results.
 * The looked-up address belongs to the device's primary context: after a
 * cudaDeviceReset (which also invalidates every material and trainer made
 * before it) the library must not be called again in that process.
 * Errors: those of bcf_train_step; BCF_ERR_UNSUPPORTED when the trainer has
 * more gradient values than the array holds (each texture's block records
 * and the weights and biases, each rounded up to 32 floats); BCF_ERR_CUDA
 * when the address lookup fails.
 */
#define BCF_NOALLOC_MAX_GRAD_FLOATS (1 << 20)
bcf_status bcf_train_step_noalloc(bcf_trainer tr, int64_t batch, uint64_t seed, int64_t step, const float *d_u,
                                  const float *d_v, const float *d_s, float *d_loss_out, bcf_stream stream);

/*
 * bcf_train_export -- write the trained features as BC6H mode-10 blocks
 * (Sec. 5.2: endpoints rounded to 6 bits, indices to 3 bits; where a
 * region's anchor texel would need the top index bit, the region's
 * endpoints are swapped and its indices mirrored, which keeps every texel
 * value) and the MLP weights as FP16 (biases stay FP32 in d_b).
 * d_blocks_out[t]: [blocks][16] bytes per texture, 16-byte aligned;
 * d_weights_fp16: [sum of W_l sizes] (may be NULL).
 */
bcf_status bcf_train_export(bcf_trainer tr, void *const *d_blocks_out, uint16_t *d_weights_fp16, bcf_stream stream);

/* ---------------------------------------------- partition selection encoder */

/*
 * bcf_encode_mode10 -- compress a mipmapped RGB feature texture into BC6H
 * mode-10 block parameters (Sec. 5.1: after a short training of unconstrained
 * features, compressing them with the BC6 algorithm fixes each block's
 * partition and initialises its endpoints and indices).
 *
 * Per block, every one of the 32 two-region partitions is tried: a line is
 * fitted to each region in the format's interpolation domain (the half bit
 * pattern of the value; principal axis of the region's scatter matrix, the
 * segment between the extreme projections), its ends are quantised to 6-bit
 * endpoints, every texel takes the 3-bit index with the smallest squared RGB
 * error of the decoded value, and the partition with the smallest total
 * error is kept (ties: the smaller partition number).  The winner's endpoint
 * codes are then improved: while moving one code up or down by one lowers
 * the total error, the best such move is taken (at most 16 moves).  All
 * decisions are computed in IEEE single precision in a fixed order, so the
 * result is reproducible.
 *
 * d_texels : level 0 .. levels-1 concatenated, each [W][W][texel_stride]
 *            float32 with W = res >> level (R, G, B first per texel,
 *            row-major), 4-byte aligned.
 * texel_stride: floats per texel, 3 (RGB) or 4 (the unconstrained features
 *            of bcf_trainer_desc).
 * res      : level-0 width, a power of two in [4, 32768]; levels in
 *            [1, log2(res) - 1] (down to at most one 4 x 4 block).
 * d_params : [blocks][32] float32, the block-parameter record of
 *            bcf_trainer_desc ([0..5] region-0 endpoints e_a RGB, e_b RGB,
 *            [8..13] region 1, [16..31] index / 7 per texel, pads 0);
 *            blocks = sum over levels of (W / 4)^2, in the trainer's order
 *            (per level, row-major).  16-byte aligned.
 * d_partitions: [blocks] partition numbers (0..31).
 * d_errors : [blocks] float32 total squared error of the chosen encoding,
 *            or NULL.
 * Caller-owned buffers; asynchronous on `stream`; no allocation.
 * Errors: BCF_ERR_INVALID_ARG for an invalid size, level count or texel
 * stride, or a null or misaligned pointer.
 */
bcf_status bcf_encode_mode10(const float *d_texels, int32_t texel_stride, int32_t res, int32_t levels,
                             float *d_params, uint8_t *d_partitions, float *d_errors, bcf_stream stream);

/*
 * bcf_compress_bc6h -- compress a mipmapped RGB texture into BC6H UF16
 * blocks, for storing channels directly (the material without the network,
 * as a comparison).  Per block two candidates: the mode-10 encoding of
 * bcf_encode_mode10 (written as bcf_pack_mode10 writes it) and a mode-11
 * encoding (one region over all sixteen texels: the same line fit, its ends
 * quantised to 10-bit endpoints, each texel the best of the 16 indices,
 * then the same one-code moves of its six endpoint codes);
 * the one with the smaller total squared error is written (ties, or a NaN
 * total: mode 10).  Decisions in IEEE single precision in a fixed order, as
 * in bcf_encode_mode10.
 * d_texels, texel_stride, res, levels: as bcf_encode_mode10.
 * d_blocks : [blocks][16] bytes, levels concatenated (per level,
 *            row-major), 16-byte aligned -- a texture bcf_create_material
 *            takes as is.
 * d_errors : [blocks] float32 total squared error of the written block,
 *            or NULL.
 * d_modes  : [blocks] uint8, 10 or 11, or NULL.
 * Caller-owned buffers; asynchronous on `stream`; no allocation.  Errors:
 * as bcf_encode_mode10.
 */
bcf_status bcf_compress_bc6h(const float *d_texels, int32_t texel_stride, int32_t res, int32_t levels, void *d_blocks,
                             float *d_errors, uint8_t *d_modes, bcf_stream stream);

/*
 * bcf_pack_mode10 -- write block-parameter records as BC6H mode-10 blocks:
 * the step bcf_train_export applies to a trainer's features, for any array
 * of records (with bcf_encode_mode10 in front, a complete mode-10
 * compressor).  Endpoints are rounded to 6-bit codes (clamped to [0, 63], or
 * to [-32, 31] two's complement when is_signed), positions to 3-bit indices
 * (round(7 x), x clamped to [0, 1]); where a region's anchor texel would
 * need the top index bit, the region's endpoints are swapped and its indices
 * mirrored, which keeps every texel value (Sec. 5.2).
 * d_params    : [n_blocks][32] float32 records as in bcf_trainer_desc,
 *               16-byte aligned.
 * d_partitions: [n_blocks] ids in [0, 31] (a larger id sets
 *               BCF_CHECK_PARTITION and reads as id & 31).
 * d_blocks_out: [n_blocks][16] bytes, 16-byte aligned.
 * n_blocks = 0 is a no-op.  The first call on a device creates its check
 * word; otherwise no allocation.  Errors: BCF_ERR_INVALID_ARG for
 * n_blocks < 0 or a null or misaligned pointer.
 */
bcf_status bcf_pack_mode10(const float *d_params, const uint8_t *d_partitions, int64_t n_blocks, int32_t is_signed,
                           void *d_blocks_out, bcf_stream stream);

/*
 * bcf_set_decode_variant -- choose the kernel bcf_decode_material uses for a
 * tensor-core (FP16 / BF16 / FP8) material.  0 (default): tile-cooperative
 * decode -- 512 screen-coherent queries (256 for textures of several
 * resolutions, or a 64-wide 16-bit MLP) share one decode of each BC6H block
 * their footprints touch (blocks mode-sorted, texels staged in shared
 * memory); falls back per tile to 1 when the tile's blocks do not fit.
 * 1: per-lane decode -- every query decodes the blocks of its own
 * footprints.  Both compute the same values.
 * 2: texture unit -- the render-time design of Sec. 5.2: the feature
 * textures are sampled through BC6H texture objects with hardware trilinear
 * filtering (mipmapped CUDA arrays; the hardware decodes the blocks), then
 * the same tensor-core MLP.  The hardware's filter and LOD weights are
 * low-precision fixed point, so its outputs differ from variants 0 and 1 by
 * a bounded filtering error: a comparison path, not a parity one.
 * 3: texture-unit texels with the exact filter -- every footprint texel is
 * fetched from the same BC6H texture objects with point filtering at its
 * centre (the hardware's BC6H decoder, bit-exact with the software one) and
 * filtered in FP32 with the software path's operations in the same order:
 * the outputs equal those of variants 0 and 1 bit for bit.  The fastest
 * exact variant.
 * Setting variant 2 or 3 allocates the mipmapped arrays and copies the
 * blocks into them (synchronously, once per material); they are freed with
 * the material.  This is the one exception to caller-owned bulk memory: the
 * arrays are a library-owned second copy of every texture's blocks (as many
 * bytes as the blocks: 179 MB for eight 4096^2 textures), because the
 * texture unit reads block-compressed data only from CUDA arrays.  The copy
 * does not follow later changes of the caller's block arrays: after
 * rewriting them, call bcf_material_refresh.  FP32 materials use the per-lane SIMT MLP; on variant 3
 * their texels come from the texture unit as above (same features), on the
 * other variants from the software decoder.
 * Errors: BCF_ERR_INVALID_ARG for a null material or another variant;
 * BCF_ERR_UNSUPPORTED for variant 2 on an FP32 material; BCF_ERR_CUDA if the
 * texture objects cannot be created.
 */
bcf_status bcf_set_decode_variant(bcf_material mat, int32_t variant);

/*
 * bcf_material_refresh -- copy the caller's block arrays into the material's
 * texture-unit arrays again (decode variants 2 and 3 sample those arrays, a
 * copy made when the variant was first set).  Asynchronous on `stream`:
 * issue it after the rewrite of the blocks (on the stream that wrote them,
 * or after synchronising it) and before the decodes that must see the new
 * blocks.  A no-op for a material without texture-unit arrays.
 * Errors: BCF_ERR_INVALID_ARG (null material), BCF_ERR_CUDA.
 */
bcf_status bcf_material_refresh(bcf_material mat, bcf_stream stream);

/*
 * bcf_set_mlp_engine -- choose the tensor-core instructions of a material's
 * MLP (Eq. 3) in its single-material decodes: decode variants 1, 2 and 3,
 * and variant 0 for materials whose textures share one resolution and
 * level count (material sets keep the warp-level MMAs).
 * BCF_MLP_MMA_SYNC (default): every warp evaluates its 32 queries with
 * warp-level MMAs, layers chained through registers.
 * BCF_MLP_TCGEN05: the CTA's tile of queries (512 on variant 0, 256 there
 * for the 64-wide 16-bit MLPs, 128 on the others) goes through the fifth-generation tensor cores -- one thread
 * issues 128-row MMAs per layer (FP16 / BF16
 * kind::f16, E4M3 kind::f8f6f4) from operand tiles in shared memory, FP32
 * accumulators in tensor memory, read back per row for the bias / ReLU /
 * rounding epilogue.  Both evaluate the same arithmetic (FP32 sums of exact
 * products, FP32 bias, rounding to the operand type between layers); the
 * summation order inside the tensor cores may differ, so outputs agree
 * within FP32 rounding (and its operand-rounding flips), not bit for bit.
 * A decode whose bounded wait for its MMAs runs out sets BCF_CHECK_TIMEOUT.
 * Errors: BCF_ERR_INVALID_ARG (null material, another engine),
 * BCF_ERR_UNSUPPORTED (FP32 materials; MLPs other than three layers
 * K0 -> 32 -> 32 -> C or 32 -> 64 -> 64 -> C with C <= 16).
 */
#define BCF_MLP_MMA_SYNC 0
#define BCF_MLP_TCGEN05 1
bcf_status bcf_set_mlp_engine(bcf_material mat, int32_t engine);

/*
 * bcf_texunit_fetch_probe -- measurement only: the rate at which the texture
 * unit point-fetches this material's BC6H texels, the path decode variant 3
 * is bound by.  n_threads threads each fetch, `rounds` times, the 2 x 2
 * footprint around their own texel of level `level` of feature texture
 * `texture` (4 x rounds x n_threads fetches in all), the 32 lanes of a warp
 * on an 8 x 4 patch of neighbouring texels and the patches in row-major
 * order over the level, as screen-coherent queries access it; the summed
 * values go to d_sink[n_threads] (float32).  The material must have texture
 * objects (decode variant 2 or 3 selected).  Asynchronous; no allocation.
 * Errors: BCF_ERR_INVALID_ARG (texture, level, rounds in [1, 4096],
 * n_threads in [0, 2^40], null or misaligned sink), BCF_ERR_UNSUPPORTED
 * (no texture objects).
 */
bcf_status bcf_texunit_fetch_probe(bcf_material mat, int32_t texture, int32_t level, int64_t n_threads, int32_t rounds,
                                   float *d_sink, bcf_stream stream);


#ifdef __cplusplus
}
#endif
#endif /* BCF_H_ */
