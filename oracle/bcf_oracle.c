/*
 * bcf_oracle.c -- plain, slow, CPU reference ("the oracle") for the BCf
 * decode and training path of "Real-Time Neural Materials using
 * Block-Compressed Features" (Weinreich et al., arXiv 2311.16121).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the libbcf C-ABI,
 * its CUDA kernels or its Python binding) may link, import or call this
 * file.  It is used by tests/, by __graft_entry__.smoke() and by the
 * cpu_baseline / reference leg of bench.py.  It shares no code, header,
 * table or constant with the CUDA path: every table below is written out
 * here, in its own notation, from the public format definition.
 *
 * Arithmetic: FP64 for every floating-point step, integers for the BC6H
 * bitstream, which the format defines exactly.
 *
 * What each part follows:
 *   - IEEE-754 binary16 / bfloat16 / OCP E4M3 codecs: the format definitions.
 *   - BC6H decode (all 14 modes, unsigned and signed): the Direct3D 11
 *     "BC6H format" definition that Sec. 4.1 and Sec. 4.2 defer to
 *     (mode table, per-mode bit layouts, 32 two-region partitions, anchor
 *     indices, unquantise / interpolate / finish steps; Eq. 7 and Eq. 8 are
 *     the paper's restatement of the latter).
 *   - Eq. 9: the continuous half-float reinterpretation.
 *   - Trilinear filtering (Eq. 10) with the per-texture LOD offset of
 *     Eq. 11, bilinear per mip level.
 *   - The MLP decoder f_eta of Eq. 3 (ReLU hidden layers, linear output),
 *     in FP64, optionally rounding at the same points as a low-precision
 *     tensor-core evaluation ("quantisation-aware").
 *   - Training (Sec. 4.1-4.3, Sec. 5.1): per-block parameters of Eq. 6,
 *     the emulated BC6 mode-10 decompression (6-bit endpoints, 3-bit
 *     indices, Sec. 5.2) with straight-through quantisation, its gradient,
 *     the relaxed continuous forward used for finite differences, the
 *     bicubic reference sampling of Sec. 5.1, the MSE loss of Eq. 5 and an
 *     Adam step (Sec. 6.1).
 *   - Philox4x32-10 (Salmon et al., SC'11) for the training batch draws.
 *   - BC6H mode-10 block encoder for partition selection and the initial
 *     block parameters (Sec. 5.1: compress unconstrained features with the
 *     BC6 algorithm): per-partition principal-axis line fit, 6-bit / 3-bit
 *     quantisation, minimum-error partition; and a plain two-mode BC6H
 *     compressor (that mode-10 encoding against a one-region mode-11 fit
 *     with 10-bit endpoints and 4-bit indices, the smaller error kept) that
 *     stores a material's channels directly, the comparison without the
 *     network.
 *
 * Parity unpinned: the bicubic kernel choice (Catmull-Rom) for the
 * reference sampling and the LOD-input convention are readings of text the
 * paper leaves open; they are internally consistent but no printed value
 * fixes them.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_TEX 16
#define OR_MAX_LAYERS 8

/* ------------------------------------------------------------------------- */
/* Number formats, from their definitions                                     */
/* ------------------------------------------------------------------------- */

/* IEEE-754 binary16: 1 sign bit, 5 exponent bits (bias 15), 10 fraction bits. */
double oracle_half_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int e = (h >> 10) & 31;
    int m = h & 1023;
    double v;
    if (e == 0)
        v = ldexp((double)m, -24); /* subnormal: m/1024 * 2^-14 */
    else if (e == 31)
        v = m ? NAN : INFINITY;
    else
        v = ldexp(1.0 + m / 1024.0, e - 15);
    return sign ? -v : v;
}

/* bfloat16: the upper 16 bits of an IEEE-754 binary32. */
double oracle_bf16_to_double(uint16_t h)
{
    int sign = (h >> 15) & 1;
    int e = (h >> 7) & 255;
    int m = h & 127;
    double v;
    if (e == 0)
        v = ldexp((double)m, -133); /* m/128 * 2^-126 */
    else if (e == 255)
        v = m ? NAN : INFINITY;
    else
        v = ldexp(1.0 + m / 128.0, e - 127);
    return sign ? -v : v;
}

/* OCP FP8 E4M3 ("fn"): bias 7, no infinities, S.1111.111 is NaN, max 448. */
double oracle_e4m3_to_double(uint8_t b)
{
    int sign = (b >> 7) & 1;
    int e = (b >> 3) & 15;
    int m = b & 7;
    double v;
    if (e == 0)
        v = ldexp((double)m, -9); /* m/8 * 2^-6 */
    else if (e == 15 && m == 7)
        v = NAN;
    else
        v = ldexp(1.0 + m / 8.0, e - 7);
    return sign ? -v : v;
}

/* Round x to the nearest value of a binary floating-point format with
 * `mant` fraction bits and minimum normal exponent `emin`, ties to even.
 * Magnitudes above `maxv` either saturate (sat=1) or become infinite. */
static double round_to_format(double x, int mant, int emin, double maxv, int sat, double overflow_at)
{
    if (x == 0.0 || isnan(x) || isinf(x))
        return x;
    double a = fabs(x);
    int e;
    frexp(a, &e); /* a = f * 2^e with f in [0.5, 1) -> exponent of a is e-1 */
    int exp2 = e - 1;
    if (exp2 < emin)
        exp2 = emin;
    double quantum = ldexp(1.0, exp2 - mant);
    double r = nearbyint(a / quantum) * quantum; /* default mode: ties to even */
    if (sat) {
        if (r > maxv)
            r = maxv;
    } else if (a >= overflow_at) {
        r = INFINITY;
    }
    return x < 0 ? -r : r;
}

double oracle_round_half(double x) { return round_to_format(x, 10, -14, 65504.0, 0, 65520.0); }
double oracle_round_bf16(double x) { return round_to_format(x, 7, -126, 3.3895313892515355e38, 0, 3.3961775292304611e38); }
double oracle_round_e4m3(double x) { return round_to_format(x, 3, -6, 448.0, 1, 0.0); }
double oracle_round_f32(double x) { return (double)(float)x; }

/* ------------------------------------------------------------------------- */
/* BC6H format tables (Direct3D 11 BC6H definition)                          */
/* ------------------------------------------------------------------------- */

/* Endpoint naming of the format definition: w, x are the two endpoints of
 * region 0 and y, z those of region 1; r, g, b the channels.  A field
 * "rw[9:0]" occupies the next 10 bit positions of the block, the lowest
 * position holding bit 0 of rw; "rw[10:15]" is stored reversed, the lowest
 * position holding bit 15.  "m" is the mode field and "d" the partition
 * (shape) index. */
typedef struct {
    int code;      /* value of the mode field */
    int mode_bits; /* 2 or 5 */
    int regions;   /* 1 or 2 */
    int transformed;
    int epb;       /* endpoint precision */
    int delta[3];  /* bits of the delta-coded endpoints, per channel */
    const char *layout;
} bc6h_mode_def;

static const bc6h_mode_def k_modes[14] = {
    /* mode 1 */ {0, 2, 2, 1, 10, {5, 5, 5},
        "m[1:0] gy[4] by[4] bz[4] rw[9:0] gw[9:0] bw[9:0] rx[4:0] gz[4] gy[3:0] gx[4:0] bz[0] "
        "gz[3:0] bx[4:0] bz[1] by[3:0] ry[4:0] bz[2] rz[4:0] bz[3] d[4:0]"},
    /* mode 2 */ {1, 2, 2, 1, 7, {6, 6, 6},
        "m[1:0] gy[5] gz[4] gz[5] rw[6:0] bz[0] bz[1] by[4] gw[6:0] by[5] bz[2] gy[4] bw[6:0] "
        "bz[3] bz[5] bz[4] rx[5:0] gy[3:0] gx[5:0] gz[3:0] bx[5:0] by[3:0] ry[5:0] rz[5:0] d[4:0]"},
    /* mode 3 */ {2, 5, 2, 1, 11, {5, 4, 4},
        "m[4:0] rw[9:0] gw[9:0] bw[9:0] rx[4:0] rw[10] gy[3:0] gx[3:0] gw[10] bz[0] gz[3:0] "
        "bx[3:0] bw[10] bz[1] by[3:0] ry[4:0] bz[2] rz[4:0] bz[3] d[4:0]"},
    /* mode 4 */ {6, 5, 2, 1, 11, {4, 5, 4},
        "m[4:0] rw[9:0] gw[9:0] bw[9:0] rx[3:0] rw[10] gz[4] gy[3:0] gx[4:0] gw[10] gz[3:0] "
        "bx[3:0] bw[10] bz[1] by[3:0] ry[3:0] bz[0] bz[2] rz[3:0] gy[4] bz[3] d[4:0]"},
    /* mode 5 */ {10, 5, 2, 1, 11, {4, 4, 5},
        "m[4:0] rw[9:0] gw[9:0] bw[9:0] rx[3:0] rw[10] by[4] gy[3:0] gx[3:0] gw[10] bz[0] "
        "gz[3:0] bx[4:0] bw[10] by[3:0] ry[3:0] bz[1] bz[2] rz[3:0] bz[4] bz[3] d[4:0]"},
    /* mode 6 */ {14, 5, 2, 1, 9, {5, 5, 5},
        "m[4:0] rw[8:0] by[4] gw[8:0] gy[4] bw[8:0] bz[4] rx[4:0] gz[4] gy[3:0] gx[4:0] bz[0] "
        "gz[3:0] bx[4:0] bz[1] by[3:0] ry[4:0] bz[2] rz[4:0] bz[3] d[4:0]"},
    /* mode 7 */ {18, 5, 2, 1, 8, {6, 5, 5},
        "m[4:0] rw[7:0] gz[4] by[4] gw[7:0] bz[2] gy[4] bw[7:0] bz[3] bz[4] rx[5:0] gy[3:0] "
        "gx[4:0] bz[0] gz[3:0] bx[4:0] bz[1] by[3:0] ry[5:0] rz[5:0] d[4:0]"},
    /* mode 8 */ {22, 5, 2, 1, 8, {5, 6, 5},
        "m[4:0] rw[7:0] bz[0] by[4] gw[7:0] gy[5] gy[4] bw[7:0] gz[5] bz[4] rx[4:0] gz[4] "
        "gy[3:0] gx[5:0] gz[3:0] bx[4:0] bz[1] by[3:0] ry[4:0] bz[2] rz[4:0] bz[3] d[4:0]"},
    /* mode 9 */ {26, 5, 2, 1, 8, {5, 5, 6},
        "m[4:0] rw[7:0] bz[1] by[4] gw[7:0] by[5] gy[4] bw[7:0] bz[5] bz[4] rx[4:0] gz[4] "
        "gy[3:0] gx[4:0] bz[0] gz[3:0] bx[5:0] by[3:0] ry[4:0] bz[2] rz[4:0] bz[3] d[4:0]"},
    /* mode 10 */ {30, 5, 2, 0, 6, {6, 6, 6},
        "m[4:0] rw[5:0] gz[4] bz[0] bz[1] by[4] gw[5:0] gy[5] by[5] bz[2] gy[4] bw[5:0] gz[5] "
        "bz[3] bz[5] bz[4] rx[5:0] gy[3:0] gx[5:0] gz[3:0] bx[5:0] by[3:0] ry[5:0] rz[5:0] d[4:0]"},
    /* mode 11 */ {3, 5, 1, 0, 10, {10, 10, 10},
        "m[4:0] rw[9:0] gw[9:0] bw[9:0] rx[9:0] gx[9:0] bx[9:0]"},
    /* mode 12 */ {7, 5, 1, 1, 11, {9, 9, 9},
        "m[4:0] rw[9:0] gw[9:0] bw[9:0] rx[8:0] rw[10] gx[8:0] gw[10] bx[8:0] bw[10]"},
    /* mode 13 */ {11, 5, 1, 1, 12, {8, 8, 8},
        "m[4:0] rw[9:0] gw[9:0] bw[9:0] rx[7:0] rw[10:11] gx[7:0] gw[10:11] bx[7:0] bw[10:11]"},
    /* mode 14 */ {15, 5, 1, 1, 16, {4, 4, 4},
        "m[4:0] rw[9:0] gw[9:0] bw[9:0] rx[3:0] rw[10:15] gx[3:0] gw[10:15] bx[3:0] bw[10:15]"},
};

/* The 32 two-region partitions: region of texel 0..15 (row-major 4x4). */
static const char *k_partitions[32] = {
    "0011001100110011", "0001000100010001", "0111011101110111", "0001001100110111",
    "0000000100010011", "0011011101111111", "0001001101111111", "0000000100110111",
    "0000000000010011", "0011011111111111", "0000000101111111", "0000000000010111",
    "0001011111111111", "0000000011111111", "0000111111111111", "0000000000001111",
    "0000100011101111", "0111000100000000", "0000000010001110", "0111001100010000",
    "0011000100000000", "0000100011001110", "0000000010001100", "0111001100110001",
    "0011000100010000", "0000100010001100", "0110011001100110", "0011011001101100",
    "0001011111101000", "0000111111110000", "0111000110001110", "0011100110011100",
};

/* Anchor texel of region 1 for each two-region partition (region 0's anchor
 * is texel 0).  An anchor texel stores its index with the top bit omitted. */
static const int k_anchor2[32] = {
    15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15, 15,
    15, 2, 8, 2, 2, 8, 8, 15, 2, 8, 2, 2, 8, 8, 2, 2,
};

/* Interpolation weights for 3-bit and 4-bit indices (out of 64). */
static const int k_weights3[8] = {0, 9, 18, 27, 37, 46, 55, 64};
static const int k_weights4[16] = {0, 4, 9, 13, 17, 21, 26, 30, 34, 38, 43, 47, 51, 55, 60, 64};

int oracle_bc6h_partition_region(int k, int texel) { return k_partitions[k][texel] - '0'; }
int oracle_bc6h_anchor2(int k) { return k_anchor2[k]; }
int oracle_bc6h_weight(int index_bits, int index) { return index_bits == 3 ? k_weights3[index] : k_weights4[index]; }

/* One parsed layout field: `count` consecutive block bits starting at
 * `pos`, bit j of which is bit (first + j*step) of value `target`.
 * target: 0..11 = endpoint (w,x,y,z) * 3 + channel (r,g,b), 12 = d, 13 = m. */
typedef struct {
    int pos, count, target, first, step;
} layout_field;

typedef struct {
    int n;
    layout_field f[40];
    int total_bits;
} parsed_layout;

static parsed_layout g_layouts[14];
static int g_layouts_ready = 0;
static pthread_once_t g_layout_once = PTHREAD_ONCE_INIT;

static void parse_layouts(void)
{
    for (int m = 0; m < 14; ++m) {
        const char *p = k_modes[m].layout;
        parsed_layout *L = &g_layouts[m];
        L->n = 0;
        int pos = 0;
        while (*p) {
            while (*p == ' ')
                ++p;
            if (!*p)
                break;
            int target;
            if (p[0] == 'm') {
                target = 13;
                p += 1;
            } else if (p[0] == 'd') {
                target = 12;
                p += 1;
            } else {
                int ch = p[0] == 'r' ? 0 : p[0] == 'g' ? 1 : 2;
                int ep = p[1] == 'w' ? 0 : p[1] == 'x' ? 1 : p[1] == 'y' ? 2 : 3;
                target = ep * 3 + ch;
                p += 2;
            }
            /* "[a:b]" or "[a]" */
            ++p; /* '[' */
            int a = (int)strtol(p, (char **)&p, 10);
            int b = a;
            if (*p == ':') {
                ++p;
                b = (int)strtol(p, (char **)&p, 10);
            }
            ++p; /* ']' */
            layout_field *F = &L->f[L->n++];
            F->pos = pos;
            F->count = abs(a - b) + 1;
            F->target = target;
            F->first = b;
            F->step = a >= b ? 1 : -1;
            pos += F->count;
        }
        L->total_bits = pos;
    }
    g_layouts_ready = 1;
}

static void ensure_layouts(void) { pthread_once(&g_layout_once, parse_layouts); }

/* Total header bits (mode + endpoints + partition) of BC6H mode 1..14:
 * 82 for two-region modes, 65 for one-region modes. */
int oracle_bc6h_header_bits(int mode)
{
    ensure_layouts();
    return g_layouts[mode - 1].total_bits;
}

static int block_bit(const uint8_t blk[16], int i) { return (blk[i >> 3] >> (i & 7)) & 1; }

static int sign_extend(int v, int bits)
{
    int s = 1 << (bits - 1);
    v &= (1 << bits) - 1;
    return (v ^ s) - s;
}

/* Unquantise an endpoint of `bits` precision to 16 bits (format definition). */
static int bc6h_unquantize(int comp, int bits, int is_signed)
{
    if (!is_signed) {
        if (bits >= 15)
            return comp;
        if (comp == 0)
            return 0;
        if (comp == (1 << bits) - 1)
            return 0xFFFF;
        return ((comp << 16) + 0x8000) >> bits;
    }
    if (bits >= 16)
        return comp;
    int neg = comp < 0;
    int mag = neg ? -comp : comp;
    int unq;
    if (mag == 0)
        unq = 0;
    else if (mag >= (1 << (bits - 1)) - 1)
        unq = 0x7FFF;
    else
        unq = ((mag << 15) + 0x4000) >> (bits - 1);
    return neg ? -unq : unq;
}

static int floor_div64(int v) { return v >= 0 ? v / 64 : -((-v + 63) / 64); }

/* Final scaling to half bits: 31/64 (unsigned) or 31/32 of the magnitude
 * (signed).  For signed values the magnitude is scaled first and the sign
 * bit is taken from the scaled integer, so a value that scales to 0 gives
 * +0, never -0. */
static uint16_t bc6h_finish(int comp, int is_signed)
{
    if (!is_signed)
        return (uint16_t)((comp * 31) >> 6);
    int scaled = comp < 0 ? -(((-comp) * 31) >> 5) : (comp * 31) >> 5;
    if (scaled < 0)
        return (uint16_t)(0x8000 | -scaled);
    return (uint16_t)scaled;
}

/* Identify the mode (1..14) of a block, or 0 for the four reserved codes. */
int oracle_bc6h_block_mode(const uint8_t blk[16])
{
    int m2 = block_bit(blk, 0) | (block_bit(blk, 1) << 1);
    int code = m2;
    if (m2 >= 2) {
        code = 0;
        for (int i = 0; i < 5; ++i)
            code |= block_bit(blk, i) << i;
    }
    for (int m = 0; m < 14; ++m)
        if (k_modes[m].code == code && (k_modes[m].mode_bits == 2) == (m2 < 2))
            return m + 1;
    return 0;
}

/* Decode one BC6H block into 16 texels x RGB half-float bit patterns.
 * Texel t = 4*row + column.  Returns the mode (1..14), or 0 for a reserved
 * mode, whose texels the definition sets to zero. */
int oracle_bc6h_decode_block(const uint8_t blk[16], int is_signed, uint16_t out[48])
{
    ensure_layouts();
    int mode = oracle_bc6h_block_mode(blk);
    if (mode == 0) {
        memset(out, 0, 48 * sizeof(uint16_t));
        return 0;
    }
    const bc6h_mode_def *M = &k_modes[mode - 1];
    const parsed_layout *L = &g_layouts[mode - 1];

    int raw[4][3] = {{0}};
    int partition = 0;
    for (int fi = 0; fi < L->n; ++fi) {
        const layout_field *F = &L->f[fi];
        for (int j = 0; j < F->count; ++j) {
            int bit = block_bit(blk, F->pos + j);
            int dst = F->first + j * F->step;
            if (F->target == 12)
                partition |= bit << dst;
            else if (F->target < 12)
                raw[F->target / 3][F->target % 3] |= bit << dst;
        }
    }

    int n_ep = 2 * M->regions;
    int e[4][3];
    for (int c = 0; c < 3; ++c) {
        e[0][c] = raw[0][c];
        if (is_signed)
            e[0][c] = sign_extend(raw[0][c], M->epb);
        for (int i = 1; i < n_ep; ++i) {
            e[i][c] = raw[i][c];
            if (is_signed || M->transformed)
                e[i][c] = sign_extend(raw[i][c], M->transformed ? M->delta[c] : M->epb);
        }
        if (M->transformed) {
            int mask = (1 << M->epb) - 1;
            for (int i = 1; i < n_ep; ++i) {
                e[i][c] = (e[0][c] + e[i][c]) & mask;
                if (is_signed)
                    e[i][c] = sign_extend(e[i][c], M->epb);
            }
        }
    }

    int unq[4][3];
    for (int i = 0; i < n_ep; ++i)
        for (int c = 0; c < 3; ++c)
            unq[i][c] = bc6h_unquantize(e[i][c], M->epb, is_signed);

    int index_bits = M->regions == 2 ? 3 : 4;
    int pos = L->total_bits; /* indices follow the header */
    for (int t = 0; t < 16; ++t) {
        int region = M->regions == 2 ? oracle_bc6h_partition_region(partition, t) : 0;
        int anchor = (t == 0) || (M->regions == 2 && t == k_anchor2[partition]);
        int nb = index_bits - anchor;
        int index = 0;
        for (int j = 0; j < nb; ++j)
            index |= block_bit(blk, pos + j) << j;
        pos += nb;
        int w = oracle_bc6h_weight(index_bits, index);
        for (int c = 0; c < 3; ++c) {
            int a = unq[2 * region][c], b = unq[2 * region + 1][c];
            int v = floor_div64(a * (64 - w) + b * w + 32);
            out[t * 3 + c] = bc6h_finish(v, is_signed);
        }
    }
    return mode;
}

/* Decode a blocks_w x blocks_h image of row-major blocks into
 * [4*blocks_h][4*blocks_w][3] half bits. */
void oracle_bc6h_decode_image(const uint8_t *blocks, int blocks_w, int blocks_h, int is_signed, uint16_t *out)
{
    int W = 4 * blocks_w;
    for (int by = 0; by < blocks_h; ++by)
        for (int bx = 0; bx < blocks_w; ++bx) {
            uint16_t tex[48];
            oracle_bc6h_decode_block(blocks + 16 * ((size_t)by * blocks_w + bx), is_signed, tex);
            for (int t = 0; t < 16; ++t) {
                int x = 4 * bx + (t & 3), y = 4 * by + (t >> 2);
                for (int c = 0; c < 3; ++c)
                    out[((size_t)y * W + x) * 3 + c] = tex[t * 3 + c];
            }
        }
}

/* Write one block field by field from the same layout description (used by
 * tests to build blocks with known endpoints; the inverse of the field
 * extraction above). raw: endpoint values already in stored form. */
void oracle_bc6h_encode_fields(int mode, const int raw[12], int partition, const int *indices, uint8_t blk[16])
{
    ensure_layouts();
    const bc6h_mode_def *M = &k_modes[mode - 1];
    const parsed_layout *L = &g_layouts[mode - 1];
    memset(blk, 0, 16);
    for (int fi = 0; fi < L->n; ++fi) {
        const layout_field *F = &L->f[fi];
        for (int j = 0; j < F->count; ++j) {
            int src = F->first + j * F->step;
            int val;
            if (F->target == 13)
                val = (M->code >> src) & 1;
            else if (F->target == 12)
                val = (partition >> src) & 1;
            else
                val = (raw[F->target] >> src) & 1;
            int p = F->pos + j;
            blk[p >> 3] |= (uint8_t)(val << (p & 7));
        }
    }
    int index_bits = M->regions == 2 ? 3 : 4;
    int pos = L->total_bits;
    for (int t = 0; t < 16; ++t) {
        int anchor = (t == 0) || (M->regions == 2 && t == k_anchor2[partition]);
        int nb = index_bits - anchor;
        for (int j = 0; j < nb; ++j) {
            int bit = (indices[t] >> j) & 1;
            blk[(pos + j) >> 3] |= (uint8_t)(bit << ((pos + j) & 7));
        }
        pos += nb;
    }
}

/* Per-mode facts, for tests: code, regions, transformed, endpoint bits, delta bits. */
void oracle_bc6h_mode_info(int mode, int info[7])
{
    const bc6h_mode_def *M = &k_modes[mode - 1];
    info[0] = M->code;
    info[1] = M->regions;
    info[2] = M->transformed;
    info[3] = M->epb;
    info[4] = M->delta[0];
    info[5] = M->delta[1];
    info[6] = M->delta[2];
}

/* ------------------------------------------------------------------------- */
/* Eq. 9: half-float bit reinterpretation as a continuous function            */
/* ------------------------------------------------------------------------- */

static double eq9_h(double y)
{
    double h = floor((y - 1.0) / 1024.0) - 1.0;
    return h > 0.0 ? h : 0.0;
}

/* w(y) = 2^(h(y)-14) (y/1024 - h(y)) for y >= 0, odd extension for y < 0. */
double oracle_eq9(double y)
{
    double a = fabs(y);
    double h = eq9_h(a);
    double w = ldexp(a / 1024.0 - h, (int)h - 14);
    return y < 0 ? -w : w;
}

/* Slope of Eq. 9: 2^(h(y)-14) / 1024 (piecewise constant). */
double oracle_eq9_slope(double y)
{
    double h = eq9_h(fabs(y));
    return ldexp(1.0, (int)h - 14) / 1024.0;
}

/* ------------------------------------------------------------------------- */
/* Textures, filtering (Eq. 10, Eq. 11)                                       */
/* ------------------------------------------------------------------------- */

typedef struct {
    int n_tex;
    int res[OR_MAX_TEX];    /* level-0 width = height, power of two >= 4 */
    int levels[OR_MAX_TEX]; /* mip levels stored, level l is res >> l */
    const uint8_t *blocks[OR_MAX_TEX]; /* mips concatenated from level 0, row-major blocks */
    int res_ref;   /* resolution the query LOD s is expressed in */
    int is_signed; /* 0: BC6H unsigned half, 1: signed */
    int wrap;      /* 1: repeat addressing, 0: clamp to edge */
    int lod_input; /* 1: append the query LOD as the last MLP input */
} oracle_material;

static int64_t level_block_offset(int res, int level)
{
    int64_t off = 0;
    for (int l = 0; l < level; ++l) {
        int64_t bw = (res >> l) / 4;
        off += bw * bw;
    }
    return off;
}

/* Decoded texel (i, j) = (column, row) of one mip level, as three doubles. */
static void texel_value(const oracle_material *M, int t, int level, int i, int j, double out[3])
{
    int W = M->res[t] >> level;
    int bw = W / 4;
    const uint8_t *blk = M->blocks[t] + 16 * (level_block_offset(M->res[t], level) + (int64_t)(j / 4) * bw + (i / 4));
    uint16_t tex[48];
    oracle_bc6h_decode_block(blk, M->is_signed, tex);
    int tt = (j % 4) * 4 + (i % 4);
    for (int c = 0; c < 3; ++c)
        out[c] = oracle_half_to_double(tex[tt * 3 + c]);
}

static int address(int i, int W, int wrap)
{
    if (wrap) {
        i %= W;
        return i < 0 ? i + W : i;
    }
    return i < 0 ? 0 : (i >= W ? W - 1 : i);
}

static double sanitize_coord(float c, int wrap)
{
    double x = isnan(c) || isinf(c) ? 0.0 : (double)c;
    if (wrap)
        return x - floor(x);
    return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x);
}

/* Bilinear sample of level `level` of texture t at (u, v); texel centres at
 * (i + 0.5) / W. */
static void bilinear(const oracle_material *M, int t, int level, double u, double v, double out[3])
{
    int W = M->res[t] >> level;
    double x = u * W - 0.5, y = v * W - 0.5;
    double fx0 = floor(x), fy0 = floor(y);
    double fx = x - fx0, fy = y - fy0;
    int i0 = (int)fx0, j0 = (int)fy0;
    double a[3], b[3], c[3], d[3];
    texel_value(M, t, level, address(i0, W, M->wrap), address(j0, W, M->wrap), a);
    texel_value(M, t, level, address(i0 + 1, W, M->wrap), address(j0, W, M->wrap), b);
    texel_value(M, t, level, address(i0, W, M->wrap), address(j0 + 1, W, M->wrap), c);
    texel_value(M, t, level, address(i0 + 1, W, M->wrap), address(j0 + 1, W, M->wrap), d);
    for (int k = 0; k < 3; ++k)
        out[k] = (1 - fx) * (1 - fy) * a[k] + fx * (1 - fy) * b[k] + (1 - fx) * fy * c[k] + fx * fy * d[k];
}

static int ilog2(int v)
{
    int r = 0;
    while ((1 << r) < v)
        ++r;
    return r;
}

/* Per-texture LOD: the query's s is in units of res_ref; texture t is
 * sampled at s_t = s + log2(res_t / res_ref) (the bias b_i of Eq. 11),
 * clamped to the stored levels. */
static void texture_lod(const oracle_material *M, int t, float s, int *l0, int *l1, double *lambda)
{
    double sq = isnan(s) ? 0.0 : (double)s;
    double st = sq + (double)(ilog2(M->res[t]) - ilog2(M->res_ref));
    double smax = (double)(M->levels[t] - 1);
    if (st < 0.0)
        st = 0.0;
    if (st > smax)
        st = smax;
    double fl = floor(st);
    *l0 = (int)fl;
    *l1 = *l0 + 1 < M->levels[t] ? *l0 + 1 : *l0;
    *lambda = st - fl;
}

/* T_t(u, v, s) of Eq. 10 for every texture, concatenated: feat[3 * n_tex]. */
void oracle_features_one(const oracle_material *M, float u, float v, float s, double *feat)
{
    double uu = sanitize_coord(u, M->wrap), vv = sanitize_coord(v, M->wrap);
    for (int t = 0; t < M->n_tex; ++t) {
        int l0, l1;
        double lam;
        texture_lod(M, t, s, &l0, &l1, &lam);
        double f0[3], f1[3];
        bilinear(M, t, l0, uu, vv, f0);
        if (l1 != l0 && lam > 0.0)
            bilinear(M, t, l1, uu, vv, f1);
        else
            memcpy(f1, f0, sizeof f0);
        for (int c = 0; c < 3; ++c)
            feat[3 * t + c] = lam * f1[c] + (1.0 - lam) * f0[c];
    }
}

void oracle_sample_features(const oracle_material *M, int64_t n, const float *u, const float *v, const float *s, double *feat)
{
    for (int64_t q = 0; q < n; ++q)
        oracle_features_one(M, u[q], v[q], s ? s[q] : 0.0f, feat + q * 3 * M->n_tex);
}

/* ------------------------------------------------------------------------- */
/* MLP decoder f_eta (Eq. 3)                                                  */
/* ------------------------------------------------------------------------- */

enum { OR_FP32 = 0, OR_FP16 = 1, OR_BF16 = 2, OR_FP8 = 3 };

typedef struct {
    int n_layers;
    int dims[OR_MAX_LAYERS + 1]; /* dims[0] inputs ... dims[n_layers] outputs */
    int precision;               /* storage format of `weights` */
    const void *weights;         /* per layer W[out][in] row-major, layers concatenated, in `precision` */
    const float *biases;         /* per layer b[out], FP32, concatenated */
    const float *act_scale;      /* FP8 only: per-layer input scale */
    const float *w_scale;        /* FP8 only: per-layer weight scale */
} oracle_mlp;

static double weight_value(const oracle_mlp *P, int64_t idx)
{
    switch (P->precision) {
    case OR_FP16: return oracle_half_to_double(((const uint16_t *)P->weights)[idx]);
    case OR_BF16: return oracle_bf16_to_double(((const uint16_t *)P->weights)[idx]);
    case OR_FP8: return oracle_e4m3_to_double(((const uint8_t *)P->weights)[idx]);
    default: return (double)((const float *)P->weights)[idx];
    }
}

static double quantize_input(int precision, double x)
{
    switch (precision) {
    case OR_FP16: return oracle_round_half(x);
    case OR_BF16: return oracle_round_bf16(x);
    case OR_FP8: return oracle_round_e4m3(x);
    default: return x;
    }
}

/* Forward one input vector.  quant_aware = 1 rounds each layer's input to
 * the storage precision (after dividing by the layer's activation scale
 * for FP8) and multiplies the FP8 product sums back by both scales; with
 * quant_aware = 0 the stored weights (times w_scale for FP8) are used as
 * exact reals and nothing else is rounded. */
void oracle_mlp_one(const oracle_mlp *P, const double *x_in, int quant_aware, double *y_out)
{
    double buf0[256], buf1[256];
    double *x = buf0, *y = buf1;
    memcpy(x, x_in, sizeof(double) * P->dims[0]);
    int64_t woff = 0, boff = 0;
    for (int l = 0; l < P->n_layers; ++l) {
        int nin = P->dims[l], nout = P->dims[l + 1];
        double as = P->precision == OR_FP8 ? (double)P->act_scale[l] : 1.0;
        double ws = P->precision == OR_FP8 ? (double)P->w_scale[l] : 1.0;
        double xq[256];
        for (int i = 0; i < nin; ++i) {
            if (quant_aware)
                xq[i] = P->precision == OR_FP8 ? quantize_input(OR_FP8, x[i] / as) : quantize_input(P->precision, x[i]);
            else
                xq[i] = P->precision == OR_FP8 ? x[i] / as : x[i];
        }
        for (int o = 0; o < nout; ++o) {
            double acc = 0.0;
            for (int i = 0; i < nin; ++i)
                acc += weight_value(P, woff + (int64_t)o * nin + i) * xq[i];
            double h = acc * as * ws + (double)P->biases[boff + o];
            if (l + 1 < P->n_layers && h < 0.0)
                h = 0.0;
            y[o] = h;
        }
        woff += (int64_t)nin * nout;
        boff += nout;
        double *tmp = x;
        x = y;
        y = tmp;
    }
    memcpy(y_out, x, sizeof(double) * P->dims[P->n_layers]);
}

/* MLP input of one query: the features, then (optionally) the query LOD
 * clamped at 0, NaN read as 0. */
static int mlp_input(const oracle_material *M, float s, const double *feat, double *x)
{
    int n = 3 * M->n_tex;
    memcpy(x, feat, sizeof(double) * n);
    if (M->lod_input) {
        double sq = isnan(s) ? 0.0 : (double)s;
        x[n++] = sq > 0.0 ? sq : 0.0;
    }
    return n;
}

/* G(u, v, s) = f_eta(T_0(u,v,s), ..., T_n(u,v,s)) (Eq. 3) for queries
 * [q0, q1): out[q][dims[n_layers]] in FP64. */
void oracle_decode_range(const oracle_material *M, const oracle_mlp *P, int64_t q0, int64_t q1, const float *u, const float *v,
                         const float *s, int quant_aware, double *out)
{
    int nout = P->dims[P->n_layers];
    for (int64_t q = q0; q < q1; ++q) {
        double feat[3 * OR_MAX_TEX], x[3 * OR_MAX_TEX + 1];
        float sq = s ? s[q] : 0.0f;
        oracle_features_one(M, u[q], v[q], sq, feat);
        mlp_input(M, sq, feat, x);
        oracle_mlp_one(P, x, quant_aware, out + q * nout);
    }
}

void oracle_decode(const oracle_material *M, const oracle_mlp *P, int64_t n, const float *u, const float *v, const float *s,
                   int quant_aware, double *out)
{
    oracle_decode_range(M, P, 0, n, u, v, s, quant_aware, out);
}

typedef struct {
    const oracle_material *M;
    const oracle_mlp *P;
    int64_t q0, q1;
    const float *u, *v, *s;
    int quant_aware;
    double *out;
} decode_job;

static void *decode_worker(void *arg)
{
    decode_job *J = (decode_job *)arg;
    oracle_decode_range(J->M, J->P, J->q0, J->q1, J->u, J->v, J->s, J->quant_aware, J->out);
    return NULL;
}

/* The same computation split over `threads` POSIX threads (timing only). */
void oracle_decode_mt(const oracle_material *M, const oracle_mlp *P, int64_t n, const float *u, const float *v, const float *s,
                      int quant_aware, double *out, int threads)
{
    ensure_layouts();
    if (threads < 1)
        threads = 1;
    if (threads > 512)
        threads = 512;
    pthread_t th[512];
    decode_job jobs[512];
    for (int i = 0; i < threads; ++i) {
        jobs[i] = (decode_job){M, P, n * i / threads, n * (i + 1) / threads, u, v, s, quant_aware, out};
        pthread_create(&th[i], NULL, decode_worker, &jobs[i]);
    }
    for (int i = 0; i < threads; ++i)
        pthread_join(th[i], NULL);
}

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)                          */
/* ------------------------------------------------------------------------- */

void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0;
        c1 = n1;
        c2 = n2;
        c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0;
    out[1] = c1;
    out[2] = c2;
    out[3] = c3;
}

/* Training batch draw for query q of step t: counter (q, t_lo, t_hi, 0),
 * key (seed_lo, seed_hi); u, v in [0, 1) and s in [0, s_max) from the top
 * 24 bits of the first three output words. */
/* The paper's batch form (Sec. 5.1: a uniformly sampled uv grid with one scale per batch): query q of a
 * grid x grid batch sits at ((i + o_u) / grid, (j + o_v) / grid), i = q mod grid, j = q / grid, with one
 * offset (o_u, o_v) and one s per step, drawn from the Philox counter (2^32 - 1, step, 2^32 - 1), which no
 * per-query draw uses.  Single-precision arithmetic, as on the device. */
void oracle_train_query_grid(uint64_t seed, uint64_t step, int64_t q, int grid, float s_max, float *u, float *v,
                             float *s)
{
    uint32_t ctr[4] = {0xFFFFFFFFu, (uint32_t)step, (uint32_t)(step >> 32), 0xFFFFFFFFu};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    oracle_philox4x32_10(ctr, key, o);
    float ou = (float)ldexp((double)(o[0] >> 8), -24), ov = (float)ldexp((double)(o[1] >> 8), -24);
    int i = (int)(q % grid), j = (int)(q / grid);
    float inv = 1.0f / (float)grid;
    float xu = (float)i + ou, xv = (float)j + ov;
    *u = xu * inv;
    *v = xv * inv;
    *s = (float)(ldexp((double)(o[2] >> 8), -24) * (double)s_max);
}

void oracle_train_query(uint64_t seed, uint64_t step, int64_t q, float s_max, float *u, float *v, float *s)
{
    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)step, (uint32_t)(step >> 32), (uint32_t)((uint64_t)q >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    oracle_philox4x32_10(ctr, key, o);
    *u = (float)ldexp((double)(o[0] >> 8), -24);
    *v = (float)ldexp((double)(o[1] >> 8), -24);
    *s = (float)(ldexp((double)(o[2] >> 8), -24) * (double)s_max);
}

/* ------------------------------------------------------------------------- */
/* Training: block-based features (Eq. 6) with emulated BC6 mode 10           */
/* ------------------------------------------------------------------------- */

/* Per block: 28 parameters = endpoints e1, e2 (region 0), e3, e4 (region 1)
 * as RGB triples in 6-bit quantisation units [0, 63], then 16 per-texel
 * positions x in [0, 1] (Eq. 6); plus one partition id k per block.  The
 * oracle holds them in FP64 (the device keeps FP32, converted exactly). */
#define OR_BLOCK_PARAMS 28

typedef struct {
    int n_tex;
    int res[OR_MAX_TEX];
    int levels[OR_MAX_TEX];
    const double *params[OR_MAX_TEX];     /* [blocks][28] per texture, mips concatenated */
    const uint8_t *partition[OR_MAX_TEX]; /* [blocks] */
    int res_ref;
    int lod_input;
    int free_texels; /* 1: unconstrained features, params[t] = [texels][3] values (mips concatenated), no
                      * partition -- the first training stage of Sec. 5.1 */
    int is_signed;   /* block features: BC6H signed (SF16) emulation */
    int literal;     /* block features: Eq. 7 and Eq. 8 as printed instead of the format's exact steps */
} oracle_train_features;

static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* One texel of the block-based features with the partial derivatives of
 * its value with respect to the two endpoints of its region and its x. */
typedef struct {
    int region;
    double value[3];
    double d_ea[3], d_eb[3], d_x[3];
    int e_in_a[3], e_in_b[3]; /* 1 where the endpoint lies inside [0, 63] */
    int x_in;                 /* 1 where x lies inside [0, 1] */
} texel_eval;

/* Emulated decompression (Sec. 4.2), straight-through form: endpoints and
 * index quantised to the exported mode-10 lattice (6-bit endpoints, 3-bit
 * indices, Sec. 5.2), then the value.  Variants:
 *   sgn = 0: BC6H unsigned (UF16): endpoints in [0, 63], a = 31/64;
 *   sgn = 1: BC6H signed (SF16): endpoints are 6-bit two's complement
 *            values in [-32, 31], a = 31/32, the value carries the sign and
 *            Eq. 9 acts on its magnitude;
 *   lit = 0: the format's exact integer steps (unquantise with its special
 *            cases for 0 and the largest code, interpolate with the >> 6
 *            floor, finish with a), so the value equals the decode of the
 *            exported block bit for bit;
 *   lit = 1: Eq. 7 and Eq. 8 as printed ("paper_literal"): the real
 *            unquantisation (a 2^16 e + 2^15) / 2^6 with no special cases,
 *            real interpolation with weight w / 64, no floors, then Eq. 9 on
 *            the real result.
 * The partials are those of the relaxed pipeline (Eq. 7 slope a 2^16 / 2^6
 * per endpoint unit, interpolation linear in w / 64 with w / 64 standing for
 * x, slope of Eq. 9) evaluated at the quantised forward values. */
static void texel_ste_v(const double *p, int k, int texel, int sgn, int lit, texel_eval *T)
{
    int region = oracle_bc6h_partition_region(k, texel);
    T->region = region;
    double x = p[12 + texel];
    T->x_in = x >= 0.0 && x <= 1.0;
    int idx = (int)nearbyint(7.0 * clampd(x, 0.0, 1.0));
    int w = k_weights3[idx];
    double lo = sgn ? -32.0 : 0.0, hi = sgn ? 31.0 : 63.0;
    double a = sgn ? 31.0 / 32.0 : 31.0 / 64.0;
    for (int c = 0; c < 3; ++c) {
        double ea = p[(2 * region) * 3 + c], eb = p[(2 * region + 1) * 3 + c];
        T->e_in_a[c] = ea >= lo && ea <= hi;
        T->e_in_b[c] = eb >= lo && eb <= hi;
        int qa = (int)nearbyint(clampd(ea, lo, hi)), qb = (int)nearbyint(clampd(eb, lo, hi));
        double slope, span;
        if (!lit) {
            int ua = bc6h_unquantize(qa, 6, sgn), ub = bc6h_unquantize(qb, 6, sgn);
            int yi = floor_div64(ua * (64 - w) + ub * w + 32);
            uint16_t bits = bc6h_finish(yi, sgn);
            T->value[c] = oracle_half_to_double(bits);
            slope = oracle_eq9_slope((double)(bits & 0x7FFF)) * a;
            span = (double)(ub - ua);
        } else {
            double ua = (a * 65536.0 * qa + 32768.0) / 64.0, ub = (a * 65536.0 * qb + 32768.0) / 64.0;
            double y = ua + (w / 64.0) * (ub - ua);
            T->value[c] = oracle_eq9(y);
            slope = oracle_eq9_slope(y) * a; /* a is inside the unquantisation here */
            span = (ub - ua) / a;
        }
        T->d_ea[c] = slope * (64.0 - w) / 64.0 * 1024.0;
        T->d_eb[c] = slope * w / 64.0 * 1024.0;
        T->d_x[c] = slope * span;
    }
}

static void texel_ste(const double *p, int k, int texel, texel_eval *T) { texel_ste_v(p, k, texel, 0, 0, T); }

/* Relaxed (continuous) texel: no rounding and no floors.  Exact form: the
 * unquantisation e -> 1024 e + 512 (signed: 1024 e + 512 sign(e)), weight
 * w = 64 x, scale a, then Eq. 9 (on the magnitude, sign restored); literal
 * form: Eq. 7 and Eq. 8 as printed with the real e and w = 64 x.  Exact
 * partials of that function. */
static void texel_relaxed_v(const double *p, int k, int texel, int sgn, int lit, texel_eval *T)
{
    int region = oracle_bc6h_partition_region(k, texel);
    T->region = region;
    T->x_in = 1;
    double w = 64.0 * p[12 + texel];
    double a = sgn ? 31.0 / 32.0 : 31.0 / 64.0;
    for (int c = 0; c < 3; ++c) {
        T->e_in_a[c] = T->e_in_b[c] = 1;
        double e0 = p[(2 * region) * 3 + c], e1 = p[(2 * region + 1) * 3 + c];
        double ea, eb, y, de;
        if (!lit) {
            ea = 1024.0 * e0 + 512.0 * (sgn && e0 < 0.0 ? -1.0 : 1.0);
            eb = 1024.0 * e1 + 512.0 * (sgn && e1 < 0.0 ? -1.0 : 1.0);
            y = ((64.0 - w) * ea + w * eb) / 64.0 * a;
            de = 1024.0 * a;
        } else {
            ea = (a * 65536.0 * e0 + 32768.0) / 64.0;
            eb = (a * 65536.0 * e1 + 32768.0) / 64.0;
            y = ((64.0 - w) * ea + w * eb) / 64.0;
            de = a * 1024.0;
        }
        T->value[c] = oracle_eq9(y);
        double sl = oracle_eq9_slope(y);
        T->d_ea[c] = sl * (64.0 - w) / 64.0 * de;
        T->d_eb[c] = sl * w / 64.0 * de;
        T->d_x[c] = sl * (lit ? (eb - ea) : (eb - ea) * a);
    }
}

static void texel_relaxed(const double *p, int k, int texel, texel_eval *T) { texel_relaxed_v(p, k, texel, 0, 0, T); }

double oracle_train_texel_v(const double *p, int k, int texel, int channel, int sgn, int lit, int relaxed)
{
    texel_eval T;
    if (relaxed)
        texel_relaxed_v(p, k, texel, sgn, lit, &T);
    else
        texel_ste_v(p, k, texel, sgn, lit, &T);
    return T.value[channel];
}

void oracle_train_texel_grad_v(const double *p, int k, int texel, int channel, int sgn, int lit, int relaxed,
                               double grad[28])
{
    texel_eval T;
    if (relaxed)
        texel_relaxed_v(p, k, texel, sgn, lit, &T);
    else
        texel_ste_v(p, k, texel, sgn, lit, &T);
    memset(grad, 0, sizeof(double) * 28);
    if (T.e_in_a[channel])
        grad[(2 * T.region) * 3 + channel] = T.d_ea[channel];
    if (T.e_in_b[channel])
        grad[(2 * T.region + 1) * 3 + channel] = T.d_eb[channel];
    if (T.x_in)
        grad[12 + texel] = T.d_x[channel];
}

double oracle_train_texel(const double *p, int k, int texel, int channel)
{
    texel_eval T;
    texel_ste(p, k, texel, &T);
    return T.value[channel];
}

double oracle_train_texel_relaxed(const double *p, int k, int texel, int channel)
{
    texel_eval T;
    texel_relaxed(p, k, texel, &T);
    return T.value[channel];
}

/* Partials of one texel channel with respect to the 28 block parameters. */
void oracle_train_texel_grad(const double *p, int k, int texel, int channel, int relaxed, double grad[28])
{
    texel_eval T;
    if (relaxed)
        texel_relaxed(p, k, texel, &T);
    else
        texel_ste(p, k, texel, &T);
    memset(grad, 0, sizeof(double) * 28);
    if (T.e_in_a[channel])
        grad[(2 * T.region) * 3 + channel] = T.d_ea[channel];
    if (T.e_in_b[channel])
        grad[(2 * T.region + 1) * 3 + channel] = T.d_eb[channel];
    if (T.x_in)
        grad[12 + texel] = T.d_x[channel];
}

static int64_t train_block_index(const oracle_train_features *F, int t, int level, int i, int j)
{
    int W = F->res[t] >> level;
    if (F->free_texels) { /* the texel itself: levels of W^2 texels concatenated */
        int64_t off = 0;
        for (int l = 0; l < level; ++l)
            off += (int64_t)(F->res[t] >> l) * (F->res[t] >> l);
        return off + (int64_t)j * W + i;
    }
    return level_block_offset(F->res[t], level) + (int64_t)(j / 4) * (W / 4) + (i / 4);
}

/* An unconstrained texel: its value, with derivative 1 (carried in d_ea) per channel. */
static void texel_free(const double *p, texel_eval *T)
{
    memset(T, 0, sizeof *T);
    for (int c = 0; c < 3; ++c) {
        T->value[c] = p[c];
        T->d_ea[c] = 1.0;
        T->e_in_a[c] = 1;
    }
}

typedef struct {
    int n;                 /* texel taps used */
    int tex[64];
    int64_t block[64];
    int texel[64];
    double weight[64];     /* filter weight of the tap in its feature */
} tap_list;

/* Trilinear taps of every texture for one query (repeat addressing). */
static void train_taps(const oracle_train_features *F, float u, float v, float s, tap_list *L)
{
    oracle_material M;
    memset(&M, 0, sizeof M);
    M.n_tex = F->n_tex;
    for (int t = 0; t < F->n_tex; ++t) {
        M.res[t] = F->res[t];
        M.levels[t] = F->levels[t];
    }
    M.res_ref = F->res_ref;
    M.wrap = 1;
    double uu = sanitize_coord(u, 1), vv = sanitize_coord(v, 1);
    L->n = 0;
    for (int t = 0; t < F->n_tex; ++t) {
        int l0, l1;
        double lam;
        texture_lod(&M, t, s, &l0, &l1, &lam);
        for (int side = 0; side < 2; ++side) {
            int level = side ? l1 : l0;
            double lw = side ? lam : 1.0 - lam;
            int W = F->res[t] >> level;
            double x = uu * W - 0.5, y = vv * W - 0.5;
            double fx0 = floor(x), fy0 = floor(y);
            double fx = x - fx0, fy = y - fy0;
            int i0 = (int)fx0, j0 = (int)fy0;
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    int i = address(i0 + di, W, 1), j = address(j0 + dj, W, 1);
                    double bw = (di ? fx : 1.0 - fx) * (dj ? fy : 1.0 - fy);
                    int n = L->n++;
                    L->tex[n] = t;
                    L->block[n] = train_block_index(F, t, level, i, j);
                    L->texel[n] = (j % 4) * 4 + (i % 4);
                    L->weight[n] = lw * bw;
                }
        }
    }
}

/* Features of the block-parameterised textures (Eq. 10 over emulated BC6). */
void oracle_train_features_one(const oracle_train_features *F, float u, float v, float s, int relaxed, double *feat)
{
    tap_list L;
    train_taps(F, u, v, s, &L);
    memset(feat, 0, sizeof(double) * 3 * F->n_tex);
    for (int n = 0; n < L.n; ++n) {
        int t = L.tex[n];
        texel_eval T;
        if (F->free_texels) {
            texel_free(F->params[t] + L.block[n] * 3, &T);
            for (int c = 0; c < 3; ++c)
                feat[3 * t + c] += L.weight[n] * T.value[c];
            continue;
        }
        const double *p = F->params[t] + L.block[n] * OR_BLOCK_PARAMS;
        if (relaxed)
            texel_relaxed_v(p, F->partition[t][L.block[n]], L.texel[n], F->is_signed, F->literal, &T);
        else
            texel_ste_v(p, F->partition[t][L.block[n]], L.texel[n], F->is_signed, F->literal, &T);
        for (int c = 0; c < 3; ++c)
            feat[3 * t + c] += L.weight[n] * T.value[c];
    }
}

/* --- reference material F(M): bicubic on two mips, then lerp (Sec. 5.1) --- */

typedef struct {
    int res;      /* level-0 resolution */
    int levels;   /* levels stored, level l is res >> l */
    const uint16_t *rgba8; /* per texel channels 0..7 (FP16 bits), mips concatenated */
    const uint16_t *ch8;   /* per texel channel 8 (FP16 bits), mips concatenated */
} oracle_target;

static int64_t level_texel_offset(int res, int level)
{
    int64_t off = 0;
    for (int l = 0; l < level; ++l) {
        int64_t w = res >> l;
        off += w * w;
    }
    return off;
}

/* Catmull-Rom weights (cubic convolution with a = -1/2) for taps -1..2. */
static void catmull_rom(double f, double w[4])
{
    double f2 = f * f, f3 = f2 * f;
    w[0] = 0.5 * (-f3 + 2.0 * f2 - f);
    w[1] = 0.5 * (3.0 * f3 - 5.0 * f2 + 2.0);
    w[2] = 0.5 * (-3.0 * f3 + 4.0 * f2 + f);
    w[3] = 0.5 * (f3 - f2);
}

static void bicubic_level(const oracle_target *T, int level, double u, double v, double out[9])
{
    int W = T->res >> level;
    double x = u * W - 0.5, y = v * W - 0.5;
    double fx0 = floor(x), fy0 = floor(y);
    double wx[4], wy[4];
    catmull_rom(x - fx0, wx);
    catmull_rom(y - fy0, wy);
    int i0 = (int)fx0, j0 = (int)fy0;
    int64_t base = level_texel_offset(T->res, level);
    for (int c = 0; c < 9; ++c)
        out[c] = 0.0;
    for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
            int i = address(i0 - 1 + a, W, 1), j = address(j0 - 1 + b, W, 1);
            int64_t idx = base + (int64_t)j * W + i;
            double wgt = wx[a] * wy[b];
            for (int c = 0; c < 8; ++c)
                out[c] += wgt * oracle_half_to_double(T->rgba8[idx * 8 + c]);
            out[8] += wgt * oracle_half_to_double(T->ch8[idx]);
        }
}

/* F(M)(u, v, s): bicubic on levels floor(s) and floor(s)+1, lerp by the
 * fractional part; s clamped to the stored levels; repeat addressing. */
void oracle_target_sample(const oracle_target *T, float u, float v, float s, double out[9])
{
    double uu = sanitize_coord(u, 1), vv = sanitize_coord(v, 1);
    double sq = isnan(s) ? 0.0 : (double)s;
    sq = clampd(sq, 0.0, (double)(T->levels - 1));
    double fl = floor(sq);
    int l0 = (int)fl;
    int l1 = l0 + 1 < T->levels ? l0 + 1 : l0;
    double lam = sq - fl;
    double a[9], b[9];
    bicubic_level(T, l0, uu, vv, a);
    if (l1 != l0 && lam > 0.0)
        bicubic_level(T, l1, uu, vv, b);
    else
        memcpy(b, a, sizeof a);
    for (int c = 0; c < 9; ++c)
        out[c] = lam * b[c] + (1.0 - lam) * a[c];
}

/* --- one training step: forward, MSE (Eq. 5), backward --- */

/* MLP of the training path: master weights, evaluated with the weights and
 * each layer's input rounded to bfloat16 when bf16 = 1 (accumulation in
 * FP64 here, FP32 on the device).  The backward is taken with respect to
 * the rounded weights and rounded activations (rounding is passed
 * straight through). */
typedef struct {
    int n_layers;
    int dims[OR_MAX_LAYERS + 1];
    const double *W; /* per layer [out][in], concatenated */
    const double *b; /* per layer [out], concatenated */
    int bf16;
} oracle_train_mlp;

typedef struct {
    double *feat_grad[OR_MAX_TEX]; /* same layout as params, accumulated */
    double *W_grad;
    double *b_grad;
} oracle_train_grads;

static double rnd_t(const oracle_train_mlp *P, double x) { return P->bf16 ? oracle_round_bf16(x) : x; }

/* Forward and backward of one query; returns the query's squared error
 * summed over channels.  Gradients of the mean loss (gscale = 2 / (B C))
 * are accumulated into G when G != NULL. */
static double train_query_ext(const oracle_train_features *F, const oracle_train_mlp *P, const oracle_target *Tg, float u,
                              float v, float s, int relaxed, double gscale, oracle_train_grads *G, const double *dy_ext,
                              double *y_out);

static double train_query(const oracle_train_features *F, const oracle_train_mlp *P, const oracle_target *Tg, float u, float v,
                          float s, int relaxed, double gscale, oracle_train_grads *G)
{
    return train_query_ext(F, P, Tg, u, v, s, relaxed, gscale, G, NULL, NULL);
}

/* One query: forward; then either the MSE gradient against the reference
 * (dy_ext == NULL) or the given output gradient dy_ext; y_out receives the
 * MLP outputs when non-NULL. */
static double train_query_ext(const oracle_train_features *F, const oracle_train_mlp *P, const oracle_target *Tg, float u,
                              float v, float s, int relaxed, double gscale, oracle_train_grads *G, const double *dy_ext,
                              double *y_out)
{
    tap_list L;
    train_taps(F, u, v, s, &L);
    texel_eval taps[64];
    int nin = 3 * F->n_tex + (F->lod_input ? 1 : 0);
    double x[64];
    memset(x, 0, sizeof x);
    for (int n = 0; n < L.n; ++n) {
        int t = L.tex[n];
        const double *p = F->params[t] + L.block[n] * (F->free_texels ? 3 : OR_BLOCK_PARAMS);
        if (F->free_texels)
            texel_free(p, &taps[n]);
        else if (relaxed)
            texel_relaxed_v(p, F->partition[t][L.block[n]], L.texel[n], F->is_signed, F->literal, &taps[n]);
        else
            texel_ste_v(p, F->partition[t][L.block[n]], L.texel[n], F->is_signed, F->literal, &taps[n]);
        for (int c = 0; c < 3; ++c)
            x[3 * t + c] += L.weight[n] * taps[n].value[c];
    }
    if (F->lod_input) {
        double sq = isnan(s) ? 0.0 : (double)s;
        x[3 * F->n_tex] = sq > 0.0 ? sq : 0.0;
    }
    /* forward, keeping every layer's (rounded) input */
    double act[OR_MAX_LAYERS + 1][64];
    double pre[OR_MAX_LAYERS][64];
    for (int i = 0; i < nin; ++i)
        act[0][i] = rnd_t(P, x[i]);
    int64_t woff = 0, boff = 0;
    int64_t woffs[OR_MAX_LAYERS], boffs[OR_MAX_LAYERS];
    for (int l = 0; l < P->n_layers; ++l) {
        int ni = P->dims[l], no = P->dims[l + 1];
        woffs[l] = woff;
        boffs[l] = boff;
        for (int o = 0; o < no; ++o) {
            double acc = 0.0;
            for (int i = 0; i < ni; ++i)
                acc += rnd_t(P, P->W[woff + (int64_t)o * ni + i]) * act[l][i];
            pre[l][o] = acc + P->b[boff + o];
            double h = pre[l][o];
            if (l + 1 < P->n_layers)
                act[l + 1][o] = rnd_t(P, h > 0.0 ? h : 0.0);
            else
                act[l + 1][o] = h;
        }
        woff += (int64_t)ni * no;
        boff += no;
    }
    int nout = P->dims[P->n_layers];
    if (y_out)
        for (int c = 0; c < nout; ++c)
            y_out[c] = act[P->n_layers][c];
    double err = 0.0;
    double dy[64];
    if (dy_ext) {
        for (int c = 0; c < nout; ++c)
            dy[c] = dy_ext[c];
    } else if (Tg) {
        double tgt[9];
        oracle_target_sample(Tg, u, v, s, tgt);
        for (int c = 0; c < nout; ++c) {
            double d = act[P->n_layers][c] - tgt[c];
            err += d * d;
            dy[c] = gscale * d;
        }
    }
    if (!G)
        return err;
    /* backward through the MLP (ReLU passes gradient where its input > 0) */
    for (int l = P->n_layers - 1; l >= 0; --l) {
        int ni = P->dims[l], no = P->dims[l + 1];
        double dx[64];
        for (int i = 0; i < ni; ++i)
            dx[i] = 0.0;
        for (int o = 0; o < no; ++o) {
            double g = dy[o];
            if (l + 1 < P->n_layers && !(pre[l][o] > 0.0))
                g = 0.0;
            G->b_grad[boffs[l] + o] += g;
            for (int i = 0; i < ni; ++i) {
                G->W_grad[woffs[l] + (int64_t)o * ni + i] += g * act[l][i];
                dx[i] += g * rnd_t(P, P->W[woffs[l] + (int64_t)o * ni + i]);
            }
        }
        for (int i = 0; i < ni; ++i)
            dy[i] = dx[i];
    }
    /* dy holds dL/d(MLP input); the LOD input has no parameters.  Backward
     * through the filter weights and the texel partials. */
    for (int n = 0; n < L.n; ++n) {
        int t = L.tex[n];
        texel_eval *T = &taps[n];
        if (F->free_texels) {
            double *g = G->feat_grad[t] + L.block[n] * 3;
            for (int c = 0; c < 3; ++c)
                g[c] += dy[3 * t + c] * L.weight[n] * T->d_ea[c];
            continue;
        }
        double *g = G->feat_grad[t] + L.block[n] * OR_BLOCK_PARAMS;
        for (int c = 0; c < 3; ++c) {
            double dv = dy[3 * t + c] * L.weight[n];
            if (T->e_in_a[c])
                g[(2 * T->region) * 3 + c] += dv * T->d_ea[c];
            if (T->e_in_b[c])
                g[(2 * T->region + 1) * 3 + c] += dv * T->d_eb[c];
            if (T->x_in)
                g[12 + L.texel[n]] += dv * T->d_x[c];
        }
    }
    return err;
}

/* Loss (mean over batch and channels, Eq. 5 normalised) and, if G != NULL,
 * its gradient, for a batch of explicit queries.  relaxed = 1 evaluates
 * the relaxed continuous forward (finite-difference checks). */
double oracle_train_loss_grad(const oracle_train_features *F, const oracle_train_mlp *P, const oracle_target *Tg, int64_t batch,
                              const float *u, const float *v, const float *s, int relaxed, oracle_train_grads *G)
{
    int nout = P->dims[P->n_layers];
    double gscale = 2.0 / ((double)batch * nout);
    double sum = 0.0;
    for (int64_t q = 0; q < batch; ++q)
        sum += train_query(F, P, Tg, u[q], v[q], s[q], relaxed, gscale, G);
    return sum / ((double)batch * nout);
}

typedef struct {
    const oracle_train_features *F;
    const oracle_train_mlp *P;
    const oracle_target *Tg;
    int64_t q0, q1;
    const float *u, *v, *s;
    double sum;
} loss_job;

static void *loss_worker(void *arg)
{
    loss_job *J = (loss_job *)arg;
    double sum = 0.0;
    for (int64_t q = J->q0; q < J->q1; ++q)
        sum += train_query(J->F, J->P, J->Tg, J->u[q], J->v[q], J->s[q], 0, 0.0, NULL);
    J->sum = sum;
    return NULL;
}

/* The loss alone (no gradients) over `threads` POSIX threads, each summing a contiguous range of queries;
 * the partial sums are added in range order (the same value as the sequential loop up to that order). */
double oracle_train_loss_mt(const oracle_train_features *F, const oracle_train_mlp *P, const oracle_target *Tg,
                            int64_t batch, const float *u, const float *v, const float *s, int threads)
{
    ensure_layouts();
    if (threads < 1)
        threads = 1;
    if (threads > 512)
        threads = 512;
    pthread_t th[512];
    loss_job jobs[512];
    for (int i = 0; i < threads; ++i) {
        jobs[i] = (loss_job){F, P, Tg, batch * i / threads, batch * (i + 1) / threads, u, v, s, 0.0};
        pthread_create(&th[i], NULL, loss_worker, &jobs[i]);
    }
    double sum = 0.0;
    for (int i = 0; i < threads; ++i) {
        pthread_join(th[i], NULL);
        sum += jobs[i].sum;
    }
    return sum / ((double)batch * P->dims[P->n_layers]);
}

/* --- Adam with exponentially decayed learning rate (Sec. 6.1) --- */

/* Step t (0-based): lr_t = lr0 * gamma^t, bias correction with t + 1;
 * afterwards the parameter is clamped to [lo, hi] (lo > hi: no clamp). */
void oracle_adam(int64_t n, double *p, const double *g, double *m, double *v, int64_t t, double lr0, double gamma, double beta1,
                 double beta2, double eps, double lo, double hi)
{
    double lr = lr0 * pow(gamma, (double)t);
    double bc1 = 1.0 - pow(beta1, (double)(t + 1));
    double bc2 = 1.0 - pow(beta2, (double)(t + 1));
    for (int64_t i = 0; i < n; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        double mh = m[i] / bc1, vh = v[i] / bc2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
        if (lo <= hi)
            p[i] = clampd(p[i], lo, hi);
    }
}

/* ------------------------------------------------------------------------- */
/* Storage model and export (Sec. 5.2)                                        */
/* ------------------------------------------------------------------------- */

/* Blocks stored for a square texture of `res` with `levels` mip levels. */
int64_t oracle_texture_blocks(int res, int levels) { return level_block_offset(res, levels); }

/* Export one trained block as a BC6H mode-10 block (6-bit endpoints, 3-bit
 * indices, Sec. 5.2).  Where a region's anchor texel would need the top
 * index bit, the region's two endpoints are swapped and its indices
 * mirrored (index -> 7 - index), which leaves every texel value unchanged
 * because the 3-bit weights satisfy W(7 - i) = 64 - W(i). */
void oracle_train_export_block_v(const double *p, int k, int sgn, uint8_t blk[16])
{
    int q[4][3], idx[16];
    for (int e = 0; e < 4; ++e)
        for (int c = 0; c < 3; ++c)
            q[e][c] = (int)nearbyint(sgn ? clampd(p[e * 3 + c], -32.0, 31.0) : clampd(p[e * 3 + c], 0.0, 63.0));
    for (int t = 0; t < 16; ++t)
        idx[t] = (int)nearbyint(7.0 * clampd(p[12 + t], 0.0, 1.0));
    for (int r = 0; r < 2; ++r) {
        int anchor = r == 0 ? 0 : k_anchor2[k];
        if (idx[anchor] >= 4) {
            for (int c = 0; c < 3; ++c) {
                int tmp = q[2 * r][c];
                q[2 * r][c] = q[2 * r + 1][c];
                q[2 * r + 1][c] = tmp;
            }
            for (int t = 0; t < 16; ++t)
                if (oracle_bc6h_partition_region(k, t) == r)
                    idx[t] = 7 - idx[t];
        }
    }
    int raw[12];
    for (int e = 0; e < 4; ++e)
        for (int c = 0; c < 3; ++c)
            raw[e * 3 + c] = q[e][c] & 63; /* 6-bit field (two's complement for SF16) */
    oracle_bc6h_encode_fields(10, raw, k, idx, blk);
}

void oracle_train_export_block(const double *p, int k, uint8_t blk[16]) { oracle_train_export_block_v(p, k, 0, blk); }

/* MLP outputs of the block-parameterised material for explicit queries
 * (out[n][C]), and the gradients for a given output gradient grad_out[n][C]
 * accumulated into G (the forward / backward pair of an autograd function). */
void oracle_train_outputs(const oracle_train_features *F, const oracle_train_mlp *P, int64_t n, const float *u, const float *v,
                          const float *s, double *out)
{
    int nout = P->dims[P->n_layers];
    for (int64_t q = 0; q < n; ++q)
        train_query_ext(F, P, NULL, u[q], v[q], s[q], 0, 0.0, NULL, NULL, out + q * nout);
}

void oracle_train_backward_given(const oracle_train_features *F, const oracle_train_mlp *P, int64_t n, const float *u,
                                 const float *v, const float *s, const double *grad_out, oracle_train_grads *G)
{
    int nout = P->dims[P->n_layers];
    for (int64_t q = 0; q < n; ++q)
        train_query_ext(F, P, NULL, u[q], v[q], s[q], 0, 0.0, G, grad_out + q * nout, NULL);
}

/* ------------------------------------------------------------------------- */
/* Rounding flips of the low-precision networks (test support)               */
/* ------------------------------------------------------------------------- */
/*
 * A low-precision evaluation rounds every layer input to its storage format.
 * The quantisation-aware forward above computes the value that is rounded in
 * FP64; the device computes it in FP32 (filter, accumulation, scale, bias).
 * Where that value lies within the device's FP32 error of a rounding
 * boundary, the two sides may round it to neighbouring representable values
 * (a flip), and the outputs then differ by the effect of one operand unit in
 * the last place, which for E4M3 and bfloat16 can exceed the absolute output
 * tolerance.  The functions below decide whether a device output that misses
 * the tolerance is such a case, and nothing else: they enumerate every
 * combination of roundings that the FP32 error windows allow (layer by
 * layer, through the ReLU) and report whether one combination reproduces the
 * device output within the tolerance on every channel.
 *
 * Error windows, bounds on |device value - exact value| before a rounding:
 *   layer-0 inputs: x_err[i], from the caller (the FP32 filter's bound);
 *   a hidden or output pre-activation: 4 (n_in + 2) 2^-24 (|scale| sum_i
 *   |w_i x_i| + |b|), the worst case of an FP32 sum of n_in products, one
 *   scaling and one bias addition (with a factor 2 for truncating adders).
 */
typedef struct {
    int n_layers;
    const int *dims;
    const double *W;      /* per layer [out][in]: the operand values the device multiplies */
    const double *b;      /* per layer [out] */
    const double *scale;  /* per layer: factor of the product sums (E4M3: act_scale * w_scale, else 1) */
    const double *in_div; /* per layer: the layer input is divided by this before rounding (E4M3: act_scale) */
    int precision;        /* rounding of every layer input (OR_FP16 / OR_BF16 / OR_FP8; OR_FP32: none) */
    const double *y_dev;  /* the device's outputs */
    double tol;
    int out_half;         /* the device output was stored as binary16 */
    long leaves, max_leaves;
    int64_t woff[OR_MAX_LAYERS], boff[OR_MAX_LAYERS];
} flip_ctx;

static double flip_round(const flip_ctx *C, int l, double h) { return quantize_input(C->precision, h / C->in_div[l]); }

/* the rounded values an input of layer l can take when its exact value is v and the device's lies within e */
static int flip_candidates(const flip_ctx *C, int l, double v, double e, int relu, double out[3])
{
    double lo = v - e, hi = v + e;
    if (relu) {
        lo = lo > 0.0 ? lo : 0.0;
        hi = hi > 0.0 ? hi : 0.0;
        v = v > 0.0 ? v : 0.0;
    }
    double a = flip_round(C, l, lo), m = flip_round(C, l, v), z = flip_round(C, l, hi);
    int n = 0;
    out[n++] = m;
    if (a != m)
        out[n++] = a;
    if (z != m && z != a)
        out[n++] = z;
    return n;
}

static int flip_layer(flip_ctx *C, int l, const double *xq);

/* fix inputs i .. n_in - 1 of layer l to each of their candidates in turn, then evaluate the layer */
static int flip_choose(flip_ctx *C, int l, double *xq, double (*cand)[3], const int *nc, int i, int n_in)
{
    while (i < n_in && nc[i] == 1) {
        xq[i] = cand[i][0];
        ++i;
    }
    if (i == n_in) {
        if (++C->leaves > C->max_leaves)
            return -1;
        return flip_layer(C, l, xq);
    }
    for (int k = 0; k < nc[i]; ++k) {
        xq[i] = cand[i][k];
        int r = flip_choose(C, l, xq, cand, nc, i + 1, n_in);
        if (r != 0)
            return r;
    }
    return 0;
}

/* layer l with rounded inputs xq: 1 when some rounding of the later layers matches the device, 0 when none,
 * -1 when the enumeration exceeds its limit */
static int flip_layer(flip_ctx *C, int l, const double *xq)
{
    int ni = C->dims[l], no = C->dims[l + 1];
    double pre[256], err[256];
    for (int o = 0; o < no; ++o) {
        double acc = 0.0, mag = 0.0;
        for (int i = 0; i < ni; ++i) {
            double p = C->W[C->woff[l] + (int64_t)o * ni + i] * xq[i];
            acc += p;
            mag += fabs(p);
        }
        double bb = C->b[C->boff[l] + o];
        pre[o] = acc * C->scale[l] + bb;
        err[o] = 4.0 * (ni + 2) * ldexp(1.0, -24) * (mag * fabs(C->scale[l]) + fabs(bb));
    }
    if (l + 1 == C->n_layers) {
        for (int c = 0; c < no; ++c) {
            double y = pre[c], t = C->tol + err[c];
            if (C->out_half) {
                y = oracle_round_half(y);
                t += fabs(y) * ldexp(1.0, -11);
            }
            if (!(fabs(C->y_dev[c] - y) <= t))
                return 0;
        }
        return 1;
    }
    double cand[256][3], xn[256];
    int nc[256];
    for (int o = 0; o < no; ++o)
        nc[o] = flip_candidates(C, l + 1, pre[o], err[o], 1, cand[o]);
    return flip_choose(C, l + 1, xn, cand, nc, 0, no);
}

static int flip_run(flip_ctx *C, const double *x, const double *x_err)
{
    int64_t wo = 0, bo = 0;
    for (int l = 0; l < C->n_layers; ++l) {
        C->woff[l] = wo;
        C->boff[l] = bo;
        wo += (int64_t)C->dims[l] * C->dims[l + 1];
        bo += C->dims[l + 1];
    }
    double cand[256][3], xq[256];
    int nc[256];
    for (int i = 0; i < C->dims[0]; ++i)
        nc[i] = flip_candidates(C, 0, x[i], x_err[i], 0, cand[i]);
    C->leaves = 0;
    return flip_choose(C, 0, xq, cand, nc, 0, C->dims[0]);
}

/* Decode network: x[dims[0]] = the exact (FP64) MLP input of one query, x_err[dims[0]] its device error bound,
 * y_dev[C] the device's outputs.  Returns 1 if a combination of roundings within the error windows gives
 * outputs within tol (plus half an FP16 unit of the output when out_half) of y_dev, 0 if none does, -1 if more
 * than max_leaves combinations would have to be tried. */
int oracle_mlp_explain(const oracle_mlp *P, const double *x, const double *x_err, const double *y_dev, double tol,
                       int out_half, long max_leaves)
{
    int64_t nw = 0, nb = 0;
    for (int l = 0; l < P->n_layers; ++l) {
        nw += (int64_t)P->dims[l] * P->dims[l + 1];
        nb += P->dims[l + 1];
    }
    double *W = malloc(sizeof(double) * (size_t)nw), *b = malloc(sizeof(double) * (size_t)nb);
    double scale[OR_MAX_LAYERS], in_div[OR_MAX_LAYERS];
    for (int64_t i = 0; i < nw; ++i)
        W[i] = weight_value(P, i);
    for (int64_t i = 0; i < nb; ++i)
        b[i] = (double)P->biases[i];
    for (int l = 0; l < P->n_layers; ++l) {
        int e4 = P->precision == OR_FP8;
        in_div[l] = e4 ? (double)P->act_scale[l] : 1.0;
        scale[l] = e4 ? (double)P->act_scale[l] * (double)P->w_scale[l] : 1.0;
    }
    flip_ctx C = {P->n_layers, P->dims, W, b, scale, in_div, P->precision, y_dev, tol, out_half, 0, max_leaves,
                  {0}, {0}};
    int r = flip_run(&C, x, x_err);
    free(W);
    free(b);
    return r;
}

/* Training network (bfloat16 operands when P->bf16): as oracle_mlp_explain, with FP32 outputs. */
int oracle_train_mlp_explain(const oracle_train_mlp *P, const double *x, const double *x_err, const double *y_dev,
                             double tol, long max_leaves)
{
    int64_t nw = 0;
    for (int l = 0; l < P->n_layers; ++l)
        nw += (int64_t)P->dims[l] * P->dims[l + 1];
    double *W = malloc(sizeof(double) * (size_t)nw);
    double one[OR_MAX_LAYERS];
    for (int64_t i = 0; i < nw; ++i)
        W[i] = rnd_t(P, P->W[i]);
    for (int l = 0; l < P->n_layers; ++l)
        one[l] = 1.0;
    flip_ctx C = {P->n_layers, P->dims, W, P->b, one, one, P->bf16 ? OR_BF16 : OR_FP32, y_dev, tol, 0, 0,
                  max_leaves, {0}, {0}};
    int r = flip_run(&C, x, x_err);
    free(W);
    return r;
}

/*
 * Per-element bounds for the device's training gradients (given output
 * gradients grad_out[n][C], as oracle_train_backward_given):
 *   A = the sum over queries and terms of |term| of every gradient element
 *       (the same products as the gradient, each taken in absolute value);
 *   R = the part of the device-minus-oracle difference that operand flips can
 *       cause beyond FP32 rounding (none without bfloat16 operands, whose
 *       rounding is the only one): for a layer input whose rounding the
 *       error windows leave open (as in oracle_mlp_explain, with a window
 *       grown by the flips of the layer inputs before it), |g| times the
 *       flip's size in the weight gradient; for a ReLU unit whose
 *       pre-activation lies within its window of 0, every term that passes
 *       through it, in absolute value.
 * The device gradient then lies within c A + R of the oracle's, c covering
 * the FP32 accumulation over the batch and the two-term bfloat16 split of
 * the output gradient.  A and R have the layout of the gradients and are
 * accumulated into (zero them first).
 */
void oracle_train_backward_bounds(const oracle_train_features *F, const oracle_train_mlp *P, int64_t n,
                                  const float *u, const float *v, const float *s, const double *grad_out,
                                  oracle_train_grads *A, oracle_train_grads *R)
{
    const double ulp24 = ldexp(1.0, -24);
    int nout = P->dims[P->n_layers];
    for (int64_t q = 0; q < n; ++q) {
        tap_list L;
        train_taps(F, u[q], v[q], s[q], &L);
        texel_eval taps[64];
        int nin = 3 * F->n_tex + (F->lod_input ? 1 : 0);
        double x[64], xmag[64];
        memset(x, 0, sizeof x);
        memset(xmag, 0, sizeof xmag);
        for (int k = 0; k < L.n; ++k) {
            int t = L.tex[k];
            const double *p = F->params[t] + L.block[k] * (F->free_texels ? 3 : OR_BLOCK_PARAMS);
            if (F->free_texels)
                texel_free(p, &taps[k]);
            else
                texel_ste_v(p, F->partition[t][L.block[k]], L.texel[k], F->is_signed, F->literal, &taps[k]);
            for (int c = 0; c < 3; ++c) {
                x[3 * t + c] += L.weight[k] * taps[k].value[c];
                xmag[3 * t + c] += fabs(L.weight[k] * taps[k].value[c]);
            }
        }
        if (F->lod_input) {
            double sq = isnan(s[q]) ? 0.0 : (double)s[q];
            x[3 * F->n_tex] = sq > 0.0 ? sq : 0.0;
        }
        /* forward with error windows and flip sizes */
        double act[OR_MAX_LAYERS + 1][64], fr[OR_MAX_LAYERS + 1][64], pre[OR_MAX_LAYERS][64];
        int amb[OR_MAX_LAYERS][64];
        for (int i = 0; i < nin; ++i) {
            double e = 8.0 * ulp24 * xmag[i];
            act[0][i] = rnd_t(P, x[i]);
            double lo = rnd_t(P, x[i] - e), hi = rnd_t(P, x[i] + e);
            fr[0][i] = P->bf16 ? fmax(fabs(hi - act[0][i]), fabs(act[0][i] - lo)) : 0.0;
        }
        int64_t woff = 0, boff = 0, woffs[OR_MAX_LAYERS], boffs[OR_MAX_LAYERS];
        for (int l = 0; l < P->n_layers; ++l) {
            int ni = P->dims[l], no = P->dims[l + 1];
            woffs[l] = woff;
            boffs[l] = boff;
            for (int o = 0; o < no; ++o) {
                double acc = 0.0, mag = 0.0, flip = 0.0;
                for (int i = 0; i < ni; ++i) {
                    double w = rnd_t(P, P->W[woff + (int64_t)o * ni + i]);
                    acc += w * act[l][i];
                    mag += fabs(w * act[l][i]);
                    flip += fabs(w) * fr[l][i];
                }
                double bb = P->b[boff + o];
                pre[l][o] = acc + bb;
                double we = 4.0 * (ni + 2) * ulp24 * (mag + fabs(bb)) + flip;
                amb[l][o] = 0;
                if (l + 1 < P->n_layers) {
                    double h = pre[l][o] > 0.0 ? pre[l][o] : 0.0;
                    double hl = pre[l][o] - we, hh = pre[l][o] + we;
                    act[l + 1][o] = rnd_t(P, h);
                    double lo = rnd_t(P, hl > 0.0 ? hl : 0.0), hi = rnd_t(P, hh > 0.0 ? hh : 0.0);
                    fr[l + 1][o] = P->bf16 ? fmax(fabs(hi - act[l + 1][o]), fabs(act[l + 1][o] - lo)) : 0.0;
                    amb[l][o] = fabs(pre[l][o]) <= we;
                }
            }
            woff += (int64_t)ni * no;
            boff += no;
        }
        /* backward in absolute values: a = all terms, r = the terms the flips leave open */
        double a[64], r[64];
        for (int c = 0; c < nout; ++c) {
            a[c] = fabs(grad_out[q * nout + c]);
            r[c] = 0.0;
        }
        for (int l = P->n_layers - 1; l >= 0; --l) {
            int ni = P->dims[l], no = P->dims[l + 1];
            double ad[64], rd[64];
            for (int i = 0; i < ni; ++i)
                ad[i] = rd[i] = 0.0;
            for (int o = 0; o < no; ++o) {
                double ga = a[o], gr = r[o];
                if (l + 1 < P->n_layers) {
                    if (amb[l][o])
                        gr = ga;
                    else if (!(pre[l][o] > 0.0))
                        ga = gr = 0.0;
                }
                A->b_grad[boffs[l] + o] += ga;
                R->b_grad[boffs[l] + o] += gr;
                for (int i = 0; i < ni; ++i) {
                    double w = fabs(rnd_t(P, P->W[woffs[l] + (int64_t)o * ni + i]));
                    A->W_grad[woffs[l] + (int64_t)o * ni + i] += ga * fabs(act[l][i]);
                    R->W_grad[woffs[l] + (int64_t)o * ni + i] += gr * fabs(act[l][i]) + ga * fr[l][i];
                    ad[i] += ga * w;
                    rd[i] += gr * w;
                }
            }
            for (int i = 0; i < ni; ++i) {
                a[i] = ad[i];
                r[i] = rd[i];
            }
        }
        for (int k = 0; k < L.n; ++k) {
            int t = L.tex[k];
            texel_eval *T = &taps[k];
            if (F->free_texels) {
                double *ga = A->feat_grad[t] + L.block[k] * 3, *gr = R->feat_grad[t] + L.block[k] * 3;
                for (int c = 0; c < 3; ++c) {
                    ga[c] += a[3 * t + c] * L.weight[k] * fabs(T->d_ea[c]);
                    gr[c] += r[3 * t + c] * L.weight[k] * fabs(T->d_ea[c]);
                }
                continue;
            }
            double *ga = A->feat_grad[t] + L.block[k] * OR_BLOCK_PARAMS;
            double *gr = R->feat_grad[t] + L.block[k] * OR_BLOCK_PARAMS;
            for (int c = 0; c < 3; ++c) {
                double da = a[3 * t + c] * L.weight[k], dr = r[3 * t + c] * L.weight[k];
                if (T->e_in_a[c]) {
                    ga[(2 * T->region) * 3 + c] += da * fabs(T->d_ea[c]);
                    gr[(2 * T->region) * 3 + c] += dr * fabs(T->d_ea[c]);
                }
                if (T->e_in_b[c]) {
                    ga[(2 * T->region + 1) * 3 + c] += da * fabs(T->d_eb[c]);
                    gr[(2 * T->region + 1) * 3 + c] += dr * fabs(T->d_eb[c]);
                }
                if (T->x_in) {
                    ga[12 + L.texel[k]] += da * fabs(T->d_x[c]);
                    gr[12 + L.texel[k]] += dr * fabs(T->d_x[c]);
                }
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* BC6H mode-10 block encoder: partition selection and initial block         */
/* parameters from free per-texel features (Sec. 5.1)                         */
/* ------------------------------------------------------------------------- */
/*
 * The paper initialises the block parameters and fixes the partitions by
 * compressing a quickly trained set of unconstrained features with the BC6
 * algorithm, without saying which search that algorithm performs.  This
 * encoder is the plain two-region search, in double precision, per block
 * and for each of the 32 two-region partitions:
 *   1. the 16 target texels are mapped to the integer domain in which the
 *      format interpolates (the binary16 bit pattern of the value, 0 for
 *      values <= 0, 0x7BFF above the half range);
 *   2. a line is fitted to each region there: the region's mean and 3 x 3
 *      covariance, the principal axis by 8 power iterations started from the
 *      covariance column of the largest diagonal entry, and the segment
 *      between the smallest and largest projections onto that axis;
 *   3. both segment ends are quantised to 6-bit endpoints by inverting the
 *      unquantise (1024 e + 512) and finish (x 31/64) steps and rounding;
 *   4. each texel takes the 3-bit index whose decoded value (the format
 *      decoder's) is closest in squared RGB error;
 * and the partition with the smallest total error is kept.  Ties go to the
 * smaller index and the smaller partition number.  The device encoder takes
 * these steps in single precision and then improves the winner (endpoint
 * codes moved by one while the error falls), so the device's error is at
 * most this one's up to single-precision rounding of the error sums.
 */

/* binary16 bit pattern of a non-negative, representable half value */
static uint16_t half_bits_of(double h)
{
    if (h <= 0.0)
        return 0;
    int e = (int)floor(log2(h));
    if (e < -14)
        return (uint16_t)nearbyint(h / ldexp(1.0, -24));
    /* guard the exact powers of two against log2 rounding */
    if (ldexp(1.0, e) > h)
        --e;
    if (ldexp(1.0, e + 1) <= h)
        ++e;
    return (uint16_t)(((e + 15) << 10) | (int)nearbyint((h / ldexp(1.0, e) - 1.0) * 1024.0));
}

/* interpolation-domain coordinate of a target value */
static double enc_coord(float v)
{
    if (!(v > 0.0f))
        return 0.0;
    double h = oracle_round_half((double)v);
    if (!(h <= 65504.0))
        return 31743.0;
    return (double)half_bits_of(h);
}

/* decoded UF16 value of one channel with b-bit endpoints a, b (modes 10 and 11) and weight w */
static double enc_value(int bits, int a, int b, int w)
{
    int ua = bc6h_unquantize(a, bits, 0), ub = bc6h_unquantize(b, bits, 0);
    return oracle_half_to_double(bc6h_finish(floor_div64(ua * (64 - w) + ub * w + 32), 0));
}

/* the endpoint code whose unquantised and finished value is y: (1024 e + 512) 31/64 = y (6 bits) or
 * (64 e + 32) 31/64 = y (10 bits), rounded to the nearest code and clamped */
static int enc_code(int bits, double y)
{
    double e = bits == 6 ? (y * 64.0 / 31.0 - 512.0) / 1024.0 : (y * 64.0 / 31.0 - 32.0) / 64.0;
    double q = nearbyint(e), top = (double)((1 << bits) - 1);
    return q < 0.0 ? 0 : (q > top ? (int)top : (int)q);
}

/* texel t belongs to the fitted set: region r of partition k, or every texel when k < 0 */
static int enc_member(int k, int r, int t) { return k < 0 ? 1 : oracle_bc6h_partition_region(k, t) == r; }

/* Line fit of the member texels of y (region r of partition k; k < 0: all sixteen): segment A .. B between
 * the extreme projections onto the principal axis, in the interpolation domain. */
void oracle_encode_fit_segment(const double y[16][3], int k, int r, double A[3], double B[3])
{
    double m[3] = {0.0, 0.0, 0.0};
    int n = 0;
    for (int t = 0; t < 16; ++t)
        if (enc_member(k, r, t)) {
            for (int c = 0; c < 3; ++c)
                m[c] += y[t][c];
            ++n;
        }
    for (int c = 0; c < 3; ++c)
        m[c] = n ? m[c] / n : 0.0;
    double C[3][3] = {{0.0}};
    for (int t = 0; t < 16; ++t)
        if (enc_member(k, r, t))
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    C[i][j] += (y[t][i] - m[i]) * (y[t][j] - m[j]);
    int jm = 0;
    for (int j = 1; j < 3; ++j)
        if (C[j][j] > C[jm][jm])
            jm = j;
    if (!(C[jm][jm] > 0.0)) {
        for (int c = 0; c < 3; ++c)
            A[c] = B[c] = m[c];
        return;
    }
    double a[3] = {C[0][jm], C[1][jm], C[2][jm]};
    for (int it = 0; it < 8; ++it) {
        double b[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                b[i] += C[i][j] * a[j];
        double len = sqrt(b[0] * b[0] + b[1] * b[1] + b[2] * b[2]);
        if (!(len > 0.0))
            break;
        for (int i = 0; i < 3; ++i)
            a[i] = b[i] / len;
    }
    double aa = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    double lo = INFINITY, hi = -INFINITY;
    for (int t = 0; t < 16; ++t)
        if (enc_member(k, r, t)) {
            double p = 0.0;
            for (int c = 0; c < 3; ++c)
                p += (y[t][c] - m[c]) * a[c];
            p /= aa;
            if (p < lo)
                lo = p;
            if (p > hi)
                hi = p;
        }
    for (int c = 0; c < 3; ++c) {
        A[c] = m[c] + lo * a[c];
        B[c] = m[c] + hi * a[c];
    }
}

/* squared RGB error of target v against index i (weight table of `bits`-bit endpoints: 3 or 4 bit indices) */
static double enc_texel_error(int bits, const int ea[3], const int eb[3], int i, const float *v)
{
    int w = bits == 6 ? k_weights3[i] : k_weights4[i];
    double e = 0.0;
    for (int c = 0; c < 3; ++c) {
        double d = enc_value(bits, ea[c], eb[c], w) - (double)v[c];
        e += d * d;
    }
    return e;
}

/* best index of every member texel for the segment (ea, eb); returns the members' total error */
static double enc_assign(int bits, int k, int r, const int ea[3], const int eb[3], const float *v, int idx[16])
{
    int ni = bits == 6 ? 8 : 16;
    double total = 0.0;
    for (int t = 0; t < 16; ++t) {
        if (!enc_member(k, r, t))
            continue;
        double best = INFINITY;
        int bi = 0;
        for (int i = 0; i < ni; ++i) {
            double e = enc_texel_error(bits, ea, eb, i, v + 3 * t);
            if (e < best) {
                best = e;
                bi = i;
            }
        }
        idx[t] = bi;
        total += best;
    }
    return total;
}

static void enc_targets(const float *v, double y[16][3])
{
    for (int t = 0; t < 16; ++t)
        for (int c = 0; c < 3; ++c)
            y[t][c] = enc_coord(v[3 * t + c]);
}

/* Encode one block: v[3 t + c] = target of texel t (row-major in the block), channel c.  Outputs the block
 * parameters in the training layout (e1, e2 = region-0 segment, e3, e4 = region-1 segment, RGB each, then
 * x_t = index / 7), the partition, its total squared error and that of every partition (errs may be NULL).
 * A NaN target has no closest index: its texel's error and every total are infinite, and partition 0 is kept. */
void oracle_encode_mode10_block(const float *v, double params[28], int *k_out, double *err_out, double errs[32])
{
    double y[16][3];
    enc_targets(v, y);
    int best_k = -1;
    double best = INFINITY;
    for (int k = 0; k < 32; ++k) {
        int e[4][3], idx[16];
        double total = 0.0;
        for (int r = 0; r < 2; ++r) {
            double A[3], B[3];
            oracle_encode_fit_segment((const double(*)[3])y, k, r, A, B);
            for (int c = 0; c < 3; ++c) {
                e[2 * r][c] = enc_code(6, A[c]);
                e[2 * r + 1][c] = enc_code(6, B[c]);
            }
            total += enc_assign(6, k, r, e[2 * r], e[2 * r + 1], v, idx);
        }
        if (errs)
            errs[k] = total;
        if (best_k < 0 || total < best) {
            best = total;
            best_k = k;
            *err_out = total;
            for (int j = 0; j < 12; ++j)
                params[j] = (double)e[j / 3][j % 3];
            for (int t = 0; t < 16; ++t)
                params[12 + t] = idx[t] / 7.0;
        }
    }
    *k_out = best_k;
}

/* Encode one block in mode 11 (one region, 10-bit endpoints, 4-bit indices): the line fit over all sixteen
 * texels, its ends quantised to 10 bits, each texel the index of the smallest squared RGB error.  e[0] / e[1] =
 * segment start / end (RGB), idx[16], the total error in *err_out. */
void oracle_encode_mode11_block(const float *v, int e[2][3], int idx[16], double *err_out)
{
    double y[16][3], A[3], B[3];
    enc_targets(v, y);
    oracle_encode_fit_segment((const double(*)[3])y, -1, 0, A, B);
    for (int c = 0; c < 3; ++c) {
        e[0][c] = enc_code(10, A[c]);
        e[1][c] = enc_code(10, B[c]);
    }
    *err_out = enc_assign(10, -1, 0, e[0], e[1], v, idx);
}

/* A plain two-mode BC6H UF16 compressor of one block: the mode-10 encoding above (written by the mode-10
 * export) against the mode-11 encoding; the smaller total error wins (ties and NaN totals: mode 10).  blk[16],
 * the written block's error and mode (10 or 11). */
void oracle_compress_bc6h_block(const float *v, uint8_t blk[16], double *err_out, int *mode_out)
{
    double params[28], err10, err11;
    int k;
    oracle_encode_mode10_block(v, params, &k, &err10, NULL);
    int e[2][3], idx[16];
    oracle_encode_mode11_block(v, e, idx, &err11);
    if (!(err11 < err10)) {
        oracle_train_export_block_v(params, k, 0, blk);
        *err_out = err10;
        *mode_out = 10;
        return;
    }
    if (idx[0] >= 8) { /* the anchor index must fit 3 bits: swap the endpoints, mirror the indices */
        for (int c = 0; c < 3; ++c) {
            int tmp = e[0][c];
            e[0][c] = e[1][c];
            e[1][c] = tmp;
        }
        for (int t = 0; t < 16; ++t)
            idx[t] = 15 - idx[t];
    }
    int raw[12] = {0};
    for (int c = 0; c < 3; ++c) {
        raw[c] = e[0][c];
        raw[3 + c] = e[1][c];
    }
    oracle_bc6h_encode_fields(11, raw, 0, idx, blk);
    *err_out = err11;
    *mode_out = 11;
}

/* The compressor over a mipmapped texture (layout as oracle_encode_mode10_texture): blocks[blocks][16],
 * err[blocks], modes[blocks]. */
void oracle_compress_bc6h_texture(const float *texels, int res, int levels, uint8_t *blocks, double *err,
                                  uint8_t *modes)
{
    int64_t toff = 0, b = 0;
    for (int l = 0; l < levels; ++l) {
        int W = res >> l, wb = W / 4;
        for (int by = 0; by < wb; ++by)
            for (int bx = 0; bx < wb; ++bx, ++b) {
                float v[48];
                for (int j = 0; j < 4; ++j)
                    for (int i = 0; i < 4; ++i)
                        for (int c = 0; c < 3; ++c)
                            v[3 * (4 * j + i) + c] = texels[toff + ((int64_t)(4 * by + j) * W + (4 * bx + i)) * 3 + c];
                int mode;
                oracle_compress_bc6h_block(v, blocks + 16 * b, err + b, &mode);
                modes[b] = (uint8_t)mode;
            }
        toff += (int64_t)W * W * 3;
    }
}

/* Encode a mipmapped texture: texels[level][W][W][3] (levels concatenated from level 0), blocks in the
 * training order (per level, row-major).  params[blocks][28], part[blocks], err[blocks]. */
void oracle_encode_mode10_texture(const float *texels, int res, int levels, double *params, uint8_t *part, double *err)
{
    int64_t toff = 0, b = 0;
    for (int l = 0; l < levels; ++l) {
        int W = res >> l, wb = W / 4;
        for (int by = 0; by < wb; ++by)
            for (int bx = 0; bx < wb; ++bx, ++b) {
                float v[48];
                for (int j = 0; j < 4; ++j)
                    for (int i = 0; i < 4; ++i)
                        for (int c = 0; c < 3; ++c)
                            v[3 * (4 * j + i) + c] = texels[toff + ((int64_t)(4 * by + j) * W + (4 * bx + i)) * 3 + c];
                int k;
                oracle_encode_mode10_block(v, params + b * 28, &k, err + b, NULL);
                part[b] = (uint8_t)k;
            }
        toff += (int64_t)W * W * 3;
    }
}
