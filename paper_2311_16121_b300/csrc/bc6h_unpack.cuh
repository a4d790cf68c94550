// bc6h_unpack.cuh -- device-side BC6H block decoder (integer, bit-exact).
//
// The block format is the one Sec. 4.1-4.2 of the paper build on and refer
// to the Direct3D BC6H definition for: a 128-bit block with a 2- or 5-bit
// mode field, 1 or 2 regions of two RGB endpoints (delta-coded relative to
// the first endpoint in 12 of the 14 modes), a 5-bit partition id for the
// 32 two-region shapes, and per-texel 3-bit (two regions) or 4-bit (one
// region) indices whose anchor texels omit the top bit.  Decoding unquantises
// the endpoints to 16 bits, interpolates them with 6-bit weights (Eq. 8 is
// the paper's form of this step) and scales by 31/64 (unsigned) or 31/32
// (signed, sign-magnitude) into half-float bit patterns (Eq. 7 folds this
// factor into the unquantisation; Eq. 9 is the reinterpretation of the bits).
//
// Layout strategy for sm_103a: the block lives in two 64-bit registers; each
// mode's fields are pulled out by straight-line shift/mask code whose bit
// position is a compile-time constant, so one mode costs a few dozen integer
// instructions.  All index bits lie in the upper 64-bit word (they start at
// bit 65 or 82), so a texel needs one variable shift.
#pragma once
#include <stdint.h>

namespace bcf {

struct Bc6hBlock {
    uint64_t lo, hi;
};

// Decoded block header: unquantised endpoints of both regions plus the
// facts the texel stage needs.
struct Bc6hHeader {
    int e[4][3];    // unquantised endpoints (region r uses e[2r], e[2r+1]); signed for SF16
    int two;        // 1: two regions (3-bit indices), 0: one region (4-bit)
    int partition;  // 0..31 (two-region modes)
    int valid;      // 0 for the reserved mode values: every texel decodes to 0
};

// Region-1 membership masks of the 32 two-region partitions, bit t = texel t
// (texel t = 4 * row + column).
__device__ __constant__ uint16_t kPartitionMask[32] = {
    0xCCCC, 0x8888, 0xEEEE, 0xECC8, 0xC880, 0xFEEC, 0xFEC8, 0xEC80, 0xC800, 0xFFEC, 0xFE80,
    0xE800, 0xFFE8, 0xFF00, 0xFFF0, 0xF000, 0xF710, 0x008E, 0x7100, 0x08CE, 0x008C, 0x7310,
    0x3100, 0x8CCE, 0x088C, 0x3110, 0x6666, 0x366C, 0x17E8, 0x0FF0, 0x718E, 0x399C};

// Global-memory copy of the masks for lane-divergent lookups (a constant-bank
// read with 32 different addresses serialises; an L1 hit does not).
__device__ const uint16_t kPartitionMaskG[32] = {
    0xCCCC, 0x8888, 0xEEEE, 0xECC8, 0xC880, 0xFEEC, 0xFEC8, 0xEC80, 0xC800, 0xFFEC, 0xFE80,
    0xE800, 0xFFE8, 0xFF00, 0xFFF0, 0xF000, 0xF710, 0x008E, 0x7100, 0x08CE, 0x008C, 0x7310,
    0x3100, 0x8CCE, 0x088C, 0x3110, 0x6666, 0x366C, 0x17E8, 0x0FF0, 0x718E, 0x399C};

__device__ __forceinline__ uint32_t partition_mask(int k) { return __ldg(&kPartitionMaskG[k]); }

// Anchor texel of region 1: 15, 2 or 8, coded in 2 bits per partition
// (0 -> 15, 1 -> 2, 2 -> 8) inside one 64-bit immediate.
__device__ __forceinline__ int anchor2_of(int k)
{
    // partitions 0..16: 15; 17..31: 2 8 2 2 8 8 15 2 8 2 2 8 8 2 2
    const uint64_t code = (1ull << 34) | (2ull << 36) | (1ull << 38) | (1ull << 40) | (2ull << 42) | (2ull << 44) |
                          (0ull << 46) | (1ull << 48) | (2ull << 50) | (1ull << 52) | (1ull << 54) | (2ull << 56) |
                          (2ull << 58) | (1ull << 60) | (1ull << 62);
    int c = (int)((code >> (2 * k)) & 3);
    return c == 0 ? 15 : (c == 1 ? 2 : 8);
}

// Interpolation weights, 7 bits per entry: 3-bit indices {0,9,18,27,37,46,55,64},
// 4-bit indices {0,4,9,13,17,21,26,30 | 34,38,43,47,51,55,60,64}.
__device__ __forceinline__ int weight3(int i)
{
    const uint64_t w = 0ull | (9ull << 7) | (18ull << 14) | (27ull << 21) | (37ull << 28) | (46ull << 35) |
                       (55ull << 42) | (64ull << 49);
    return (int)((w >> (7 * i)) & 127);
}
__device__ __forceinline__ int weight4(int i)
{
    const uint64_t a = 0ull | (4ull << 7) | (9ull << 14) | (13ull << 21) | (17ull << 28) | (21ull << 35) |
                       (26ull << 42) | (30ull << 49);
    const uint64_t b = 34ull | (38ull << 7) | (43ull << 14) | (47ull << 21) | (51ull << 28) | (55ull << 35) |
                       (60ull << 42) | (64ull << 49);
    return (int)(((i < 8 ? a : b) >> (7 * (i & 7))) & 127);
}

// Bits [p, p+n) of the 128-bit block; p and n are compile-time constants at
// every call site below, so exactly one branch survives.
__device__ __forceinline__ int bits_at(const Bc6hBlock &b, int p, int n)
{
    uint64_t v;
    if (p + n <= 64)
        v = b.lo >> p;
    else if (p >= 64)
        v = b.hi >> (p - 64);
    else
        v = (b.lo >> p) | (b.hi << (64 - p));
    return (int)(v & ((1ull << n) - 1));
}

__device__ __forceinline__ int sext(int v, int bits)
{
    int s = 32 - bits;
    return (v << s) >> s;
}

__device__ __forceinline__ int unquantize(int c, int epb, bool sgn)
{
    if (!sgn) {
        if (epb >= 15)
            return c;
        if (c == 0)
            return 0;
        if (c == (1 << epb) - 1)
            return 0xFFFF;
        return ((c << 16) + 0x8000) >> epb;
    }
    if (epb >= 16)
        return c;
    int m = c < 0 ? -c : c;
    int u;
    if (m == 0)
        u = 0;
    else if (m >= (1 << (epb - 1)) - 1)
        u = 0x7FFF;
    else
        u = ((m << 15) + 0x4000) >> (epb - 1);
    return c < 0 ? -u : u;
}

// Mode field -> mode index 0..13 (modes 1..14), or -1 for a reserved value.
__device__ __forceinline__ int mode_index(uint32_t low)
{
    uint32_t m2 = low & 3;
    if (m2 < 2)
        return (int)m2;
    uint32_t code = low & 31;
    // codes 4j+2 -> modes 3..10 (idx 2..9); codes 3, 7, 11, 15 -> modes 11..14; 19, 23, 27, 31 reserved
    if (m2 == 2)
        return 2 + (int)(code >> 2);
    return code < 16 ? 10 + (int)(code >> 2) : -1;
}

#define BCF_TAKE(var, lsb, n)                      \
    {                                              \
        var |= bits_at(blk, p, n) << (lsb);        \
        p += (n);                                  \
    }

// Decode the header of one block: mode, endpoints (with delta transform and
// sign handling) and partition; endpoints are returned unquantised.
__device__ __forceinline__ void bc6h_header(const Bc6hBlock &blk, bool sgn, Bc6hHeader &H)
{
    int r0 = 0, g0 = 0, b0 = 0, r1 = 0, g1 = 0, b1 = 0, r2 = 0, g2 = 0, b2 = 0, r3 = 0, g3 = 0, b3 = 0, d = 0;
    int epb = 0, dr = 0, dg = 0, db = 0, xf = 1, two = 1;
    const int mi = mode_index((uint32_t)blk.lo);
    switch (mi) {
    case 0: { // mode 1: 10-bit base, 5.5.5 deltas
        int p = 2;
        BCF_TAKE(g2, 4, 1) BCF_TAKE(b2, 4, 1) BCF_TAKE(b3, 4, 1) BCF_TAKE(r0, 0, 10) BCF_TAKE(g0, 0, 10)
        BCF_TAKE(b0, 0, 10) BCF_TAKE(r1, 0, 5) BCF_TAKE(g3, 4, 1) BCF_TAKE(g2, 0, 4) BCF_TAKE(g1, 0, 5)
        BCF_TAKE(b3, 0, 1) BCF_TAKE(g3, 0, 4) BCF_TAKE(b1, 0, 5) BCF_TAKE(b3, 1, 1) BCF_TAKE(b2, 0, 4)
        BCF_TAKE(r2, 0, 5) BCF_TAKE(b3, 2, 1) BCF_TAKE(r3, 0, 5) BCF_TAKE(b3, 3, 1) BCF_TAKE(d, 0, 5)
        epb = 10; dr = 5; dg = 5; db = 5;
        break;
    }
    case 1: { // mode 2: 7-bit base, 6.6.6 deltas
        int p = 2;
        BCF_TAKE(g2, 5, 1) BCF_TAKE(g3, 4, 1) BCF_TAKE(g3, 5, 1) BCF_TAKE(r0, 0, 7) BCF_TAKE(b3, 0, 1)
        BCF_TAKE(b3, 1, 1) BCF_TAKE(b2, 4, 1) BCF_TAKE(g0, 0, 7) BCF_TAKE(b2, 5, 1) BCF_TAKE(b3, 2, 1)
        BCF_TAKE(g2, 4, 1) BCF_TAKE(b0, 0, 7) BCF_TAKE(b3, 3, 1) BCF_TAKE(b3, 5, 1) BCF_TAKE(b3, 4, 1)
        BCF_TAKE(r1, 0, 6) BCF_TAKE(g2, 0, 4) BCF_TAKE(g1, 0, 6) BCF_TAKE(g3, 0, 4) BCF_TAKE(b1, 0, 6)
        BCF_TAKE(b2, 0, 4) BCF_TAKE(r2, 0, 6) BCF_TAKE(r3, 0, 6) BCF_TAKE(d, 0, 5)
        epb = 7; dr = 6; dg = 6; db = 6;
        break;
    }
    case 2: { // mode 3: 11-bit base, 5.4.4
        int p = 5;
        BCF_TAKE(r0, 0, 10) BCF_TAKE(g0, 0, 10) BCF_TAKE(b0, 0, 10) BCF_TAKE(r1, 0, 5) BCF_TAKE(r0, 10, 1)
        BCF_TAKE(g2, 0, 4) BCF_TAKE(g1, 0, 4) BCF_TAKE(g0, 10, 1) BCF_TAKE(b3, 0, 1) BCF_TAKE(g3, 0, 4)
        BCF_TAKE(b1, 0, 4) BCF_TAKE(b0, 10, 1) BCF_TAKE(b3, 1, 1) BCF_TAKE(b2, 0, 4) BCF_TAKE(r2, 0, 5)
        BCF_TAKE(b3, 2, 1) BCF_TAKE(r3, 0, 5) BCF_TAKE(b3, 3, 1) BCF_TAKE(d, 0, 5)
        epb = 11; dr = 5; dg = 4; db = 4;
        break;
    }
    case 3: { // mode 4: 11-bit base, 4.5.4
        int p = 5;
        BCF_TAKE(r0, 0, 10) BCF_TAKE(g0, 0, 10) BCF_TAKE(b0, 0, 10) BCF_TAKE(r1, 0, 4) BCF_TAKE(r0, 10, 1)
        BCF_TAKE(g3, 4, 1) BCF_TAKE(g2, 0, 4) BCF_TAKE(g1, 0, 5) BCF_TAKE(g0, 10, 1) BCF_TAKE(g3, 0, 4)
        BCF_TAKE(b1, 0, 4) BCF_TAKE(b0, 10, 1) BCF_TAKE(b3, 1, 1) BCF_TAKE(b2, 0, 4) BCF_TAKE(r2, 0, 4)
        BCF_TAKE(b3, 0, 1) BCF_TAKE(b3, 2, 1) BCF_TAKE(r3, 0, 4) BCF_TAKE(g2, 4, 1) BCF_TAKE(b3, 3, 1)
        BCF_TAKE(d, 0, 5)
        epb = 11; dr = 4; dg = 5; db = 4;
        break;
    }
    case 4: { // mode 5: 11-bit base, 4.4.5
        int p = 5;
        BCF_TAKE(r0, 0, 10) BCF_TAKE(g0, 0, 10) BCF_TAKE(b0, 0, 10) BCF_TAKE(r1, 0, 4) BCF_TAKE(r0, 10, 1)
        BCF_TAKE(b2, 4, 1) BCF_TAKE(g2, 0, 4) BCF_TAKE(g1, 0, 4) BCF_TAKE(g0, 10, 1) BCF_TAKE(b3, 0, 1)
        BCF_TAKE(g3, 0, 4) BCF_TAKE(b1, 0, 5) BCF_TAKE(b0, 10, 1) BCF_TAKE(b2, 0, 4) BCF_TAKE(r2, 0, 4)
        BCF_TAKE(b3, 1, 1) BCF_TAKE(b3, 2, 1) BCF_TAKE(r3, 0, 4) BCF_TAKE(b3, 4, 1) BCF_TAKE(b3, 3, 1)
        BCF_TAKE(d, 0, 5)
        epb = 11; dr = 4; dg = 4; db = 5;
        break;
    }
    case 5: { // mode 6: 9-bit base, 5.5.5
        int p = 5;
        BCF_TAKE(r0, 0, 9) BCF_TAKE(b2, 4, 1) BCF_TAKE(g0, 0, 9) BCF_TAKE(g2, 4, 1) BCF_TAKE(b0, 0, 9)
        BCF_TAKE(b3, 4, 1) BCF_TAKE(r1, 0, 5) BCF_TAKE(g3, 4, 1) BCF_TAKE(g2, 0, 4) BCF_TAKE(g1, 0, 5)
        BCF_TAKE(b3, 0, 1) BCF_TAKE(g3, 0, 4) BCF_TAKE(b1, 0, 5) BCF_TAKE(b3, 1, 1) BCF_TAKE(b2, 0, 4)
        BCF_TAKE(r2, 0, 5) BCF_TAKE(b3, 2, 1) BCF_TAKE(r3, 0, 5) BCF_TAKE(b3, 3, 1) BCF_TAKE(d, 0, 5)
        epb = 9; dr = 5; dg = 5; db = 5;
        break;
    }
    case 6: { // mode 7: 8-bit base, 6.5.5
        int p = 5;
        BCF_TAKE(r0, 0, 8) BCF_TAKE(g3, 4, 1) BCF_TAKE(b2, 4, 1) BCF_TAKE(g0, 0, 8) BCF_TAKE(b3, 2, 1)
        BCF_TAKE(g2, 4, 1) BCF_TAKE(b0, 0, 8) BCF_TAKE(b3, 3, 1) BCF_TAKE(b3, 4, 1) BCF_TAKE(r1, 0, 6)
        BCF_TAKE(g2, 0, 4) BCF_TAKE(g1, 0, 5) BCF_TAKE(b3, 0, 1) BCF_TAKE(g3, 0, 4) BCF_TAKE(b1, 0, 5)
        BCF_TAKE(b3, 1, 1) BCF_TAKE(b2, 0, 4) BCF_TAKE(r2, 0, 6) BCF_TAKE(r3, 0, 6) BCF_TAKE(d, 0, 5)
        epb = 8; dr = 6; dg = 5; db = 5;
        break;
    }
    case 7: { // mode 8: 8-bit base, 5.6.5
        int p = 5;
        BCF_TAKE(r0, 0, 8) BCF_TAKE(b3, 0, 1) BCF_TAKE(b2, 4, 1) BCF_TAKE(g0, 0, 8) BCF_TAKE(g2, 5, 1)
        BCF_TAKE(g2, 4, 1) BCF_TAKE(b0, 0, 8) BCF_TAKE(g3, 5, 1) BCF_TAKE(b3, 4, 1) BCF_TAKE(r1, 0, 5)
        BCF_TAKE(g3, 4, 1) BCF_TAKE(g2, 0, 4) BCF_TAKE(g1, 0, 6) BCF_TAKE(g3, 0, 4) BCF_TAKE(b1, 0, 5)
        BCF_TAKE(b3, 1, 1) BCF_TAKE(b2, 0, 4) BCF_TAKE(r2, 0, 5) BCF_TAKE(b3, 2, 1) BCF_TAKE(r3, 0, 5)
        BCF_TAKE(b3, 3, 1) BCF_TAKE(d, 0, 5)
        epb = 8; dr = 5; dg = 6; db = 5;
        break;
    }
    case 8: { // mode 9: 8-bit base, 5.5.6
        int p = 5;
        BCF_TAKE(r0, 0, 8) BCF_TAKE(b3, 1, 1) BCF_TAKE(b2, 4, 1) BCF_TAKE(g0, 0, 8) BCF_TAKE(b2, 5, 1)
        BCF_TAKE(g2, 4, 1) BCF_TAKE(b0, 0, 8) BCF_TAKE(b3, 5, 1) BCF_TAKE(b3, 4, 1) BCF_TAKE(r1, 0, 5)
        BCF_TAKE(g3, 4, 1) BCF_TAKE(g2, 0, 4) BCF_TAKE(g1, 0, 5) BCF_TAKE(b3, 0, 1) BCF_TAKE(g3, 0, 4)
        BCF_TAKE(b1, 0, 6) BCF_TAKE(b2, 0, 4) BCF_TAKE(r2, 0, 5) BCF_TAKE(b3, 2, 1) BCF_TAKE(r3, 0, 5)
        BCF_TAKE(b3, 3, 1) BCF_TAKE(d, 0, 5)
        epb = 8; dr = 5; dg = 5; db = 6;
        break;
    }
    case 9: { // mode 10: four 6-bit endpoints, no deltas (the mode trained features export to)
        int p = 5;
        BCF_TAKE(r0, 0, 6) BCF_TAKE(g3, 4, 1) BCF_TAKE(b3, 0, 1) BCF_TAKE(b3, 1, 1) BCF_TAKE(b2, 4, 1)
        BCF_TAKE(g0, 0, 6) BCF_TAKE(g2, 5, 1) BCF_TAKE(b2, 5, 1) BCF_TAKE(b3, 2, 1) BCF_TAKE(g2, 4, 1)
        BCF_TAKE(b0, 0, 6) BCF_TAKE(g3, 5, 1) BCF_TAKE(b3, 3, 1) BCF_TAKE(b3, 5, 1) BCF_TAKE(b3, 4, 1)
        BCF_TAKE(r1, 0, 6) BCF_TAKE(g2, 0, 4) BCF_TAKE(g1, 0, 6) BCF_TAKE(g3, 0, 4) BCF_TAKE(b1, 0, 6)
        BCF_TAKE(b2, 0, 4) BCF_TAKE(r2, 0, 6) BCF_TAKE(r3, 0, 6) BCF_TAKE(d, 0, 5)
        epb = 6; dr = 6; dg = 6; db = 6; xf = 0;
        break;
    }
    case 10: { // mode 11: one region, two 10-bit endpoints
        int p = 5;
        BCF_TAKE(r0, 0, 10) BCF_TAKE(g0, 0, 10) BCF_TAKE(b0, 0, 10) BCF_TAKE(r1, 0, 10) BCF_TAKE(g1, 0, 10)
        BCF_TAKE(b1, 0, 10)
        epb = 10; dr = 10; dg = 10; db = 10; xf = 0; two = 0;
        break;
    }
    case 11: { // mode 12: one region, 11-bit base, 9-bit delta
        int p = 5;
        BCF_TAKE(r0, 0, 10) BCF_TAKE(g0, 0, 10) BCF_TAKE(b0, 0, 10) BCF_TAKE(r1, 0, 9) BCF_TAKE(r0, 10, 1)
        BCF_TAKE(g1, 0, 9) BCF_TAKE(g0, 10, 1) BCF_TAKE(b1, 0, 9) BCF_TAKE(b0, 10, 1)
        epb = 11; dr = 9; dg = 9; db = 9; two = 0;
        break;
    }
    case 12: { // mode 13: one region, 12-bit base (bits 10-11 stored high bit first), 8-bit delta
        int p = 5;
        BCF_TAKE(r0, 0, 10) BCF_TAKE(g0, 0, 10) BCF_TAKE(b0, 0, 10) BCF_TAKE(r1, 0, 8) BCF_TAKE(r0, 11, 1)
        BCF_TAKE(r0, 10, 1) BCF_TAKE(g1, 0, 8) BCF_TAKE(g0, 11, 1) BCF_TAKE(g0, 10, 1) BCF_TAKE(b1, 0, 8)
        BCF_TAKE(b0, 11, 1) BCF_TAKE(b0, 10, 1)
        epb = 12; dr = 8; dg = 8; db = 8; two = 0;
        break;
    }
    case 13: { // mode 14: one region, 16-bit base (bits 10-15 stored high bit first), 4-bit delta
        int p = 5;
        BCF_TAKE(r0, 0, 10) BCF_TAKE(g0, 0, 10) BCF_TAKE(b0, 0, 10) BCF_TAKE(r1, 0, 4)
        BCF_TAKE(r0, 15, 1) BCF_TAKE(r0, 14, 1) BCF_TAKE(r0, 13, 1) BCF_TAKE(r0, 12, 1) BCF_TAKE(r0, 11, 1)
        BCF_TAKE(r0, 10, 1) BCF_TAKE(g1, 0, 4) BCF_TAKE(g0, 15, 1) BCF_TAKE(g0, 14, 1) BCF_TAKE(g0, 13, 1)
        BCF_TAKE(g0, 12, 1) BCF_TAKE(g0, 11, 1) BCF_TAKE(g0, 10, 1) BCF_TAKE(b1, 0, 4) BCF_TAKE(b0, 15, 1)
        BCF_TAKE(b0, 14, 1) BCF_TAKE(b0, 13, 1) BCF_TAKE(b0, 12, 1) BCF_TAKE(b0, 11, 1) BCF_TAKE(b0, 10, 1)
        epb = 16; dr = 4; dg = 4; db = 4; two = 0;
        break;
    }
    default:
        H.valid = 0;
        H.two = 0;
        H.partition = 0;
        for (int i = 0; i < 4; ++i)
            H.e[i][0] = H.e[i][1] = H.e[i][2] = 0;
        return;
    }
    H.valid = 1;
    H.two = two;
    H.partition = d;
    int raw[4][3] = {{r0, g0, b0}, {r1, g1, b1}, {r2, g2, b2}, {r3, g3, b3}};
    const int dbits[3] = {dr, dg, db};
    const int mask = (1 << epb) - 1;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        int base = sgn ? sext(raw[0][c], epb) : raw[0][c];
        H.e[0][c] = unquantize(base, epb, sgn);
#pragma unroll
        for (int i = 1; i < 4; ++i) {
            if (i >= 2 && !two) {
                H.e[i][c] = 0;
                continue;
            }
            int v = raw[i][c];
            if (sgn || xf)
                v = sext(v, xf ? dbits[c] : epb);
            if (xf) {
                v = (base + v) & mask;
                if (sgn)
                    v = sext(v, epb);
            }
            H.e[i][c] = unquantize(v, epb, sgn);
        }
    }
}
#undef BCF_TAKE

// Scale to half bits: 31/64 (unsigned); signed: 31/32 of the magnitude, sign
// bit set only when the scaled magnitude is non-zero (no -0).
__device__ __forceinline__ uint32_t finish(int v, bool sgn)
{
    if (!sgn)
        return (uint32_t)((v * 31) >> 6);
    const uint32_t mag = (uint32_t)(((v < 0 ? -v : v) * 31) >> 5);
    return (v < 0 && mag != 0u) ? (0x8000u | mag) : mag;
}

// Texel t (= 4 * row + column) of a decoded block: three half bit patterns.
__device__ __forceinline__ void bc6h_texel(const Bc6hBlock &blk, const Bc6hHeader &H, int t, bool sgn, uint32_t &r,
                                           uint32_t &g, uint32_t &b)
{
    int region, w, pos, nb;
    if (H.two) {
        int a2 = anchor2_of(H.partition);
        region = (int)((partition_mask(H.partition) >> t) & 1);
        pos = 82 + 3 * t - (t > 0) - (t > a2);
        nb = 3 - ((t == 0) | (t == a2));
        w = weight3((int)((blk.hi >> (pos - 64)) & ((1u << nb) - 1)));
    } else {
        region = 0;
        pos = 65 + 4 * t - (t > 0);
        nb = 4 - (t == 0);
        w = weight4((int)((blk.hi >> (pos - 64)) & ((1u << nb) - 1)));
    }
    const int *ea = region ? H.e[2] : H.e[0];
    const int *eb = region ? H.e[3] : H.e[1];
    int vr = (ea[0] * (64 - w) + eb[0] * w + 32) >> 6;
    int vg = (ea[1] * (64 - w) + eb[1] * w + 32) >> 6;
    int vb = (ea[2] * (64 - w) + eb[2] * w + 32) >> 6;
    r = H.valid ? finish(vr, sgn) : 0u;
    g = H.valid ? finish(vg, sgn) : 0u;
    b = H.valid ? finish(vb, sgn) : 0u;
}

__device__ __forceinline__ Bc6hBlock load_block(const uint4 *p)
{
    uint4 v = __ldg(p);
    Bc6hBlock b;
    b.lo = (uint64_t)v.x | ((uint64_t)v.y << 32);
    b.hi = (uint64_t)v.z | ((uint64_t)v.w << 32);
    return b;
}

} // namespace bcf

namespace bcf {

// All 16 texels of a decoded block, written through `store(t, rgb_lo, b)`
// with rgb_lo = R | G << 16 and b = B (half bit patterns).  The partition
// mask, anchor and index stream are read once for the block; indices are
// consumed from a running shift of the upper 64-bit word.
template <class Store>
__device__ __forceinline__ void bc6h_all_texels(const Bc6hBlock &blk, const Bc6hHeader &H, bool sgn, Store store)
{
    uint64_t idx;
    uint32_t pmask = 0;
    int a2 = 16;
    if (H.two) {
        pmask = partition_mask(H.partition);
        a2 = anchor2_of(H.partition);
        idx = blk.hi >> 18; // index bits start at bit 82
    } else {
        idx = blk.hi >> 1;  // index bits start at bit 65
    }
#pragma unroll
    for (int t = 0; t < 16; ++t) {
        int w;
        if (H.two) {
            const int nb = (t == 0 || t == a2) ? 2 : 3;
            w = weight3((int)(idx & ((1u << nb) - 1)));
            idx >>= nb;
        } else {
            const int nb = t == 0 ? 3 : 4;
            w = weight4((int)(idx & ((1u << nb) - 1)));
            idx >>= nb;
        }
        const int region = (int)((pmask >> t) & 1);
        const int *ea = region ? H.e[2] : H.e[0];
        const int *eb = region ? H.e[3] : H.e[1];
        const int vr = (ea[0] * (64 - w) + eb[0] * w + 32) >> 6;
        const int vg = (ea[1] * (64 - w) + eb[1] * w + 32) >> 6;
        const int vb = (ea[2] * (64 - w) + eb[2] * w + 32) >> 6;
        const uint32_t r = H.valid ? finish(vr, sgn) : 0u;
        const uint32_t g = H.valid ? finish(vg, sgn) : 0u;
        const uint32_t b = H.valid ? finish(vb, sgn) : 0u;
        store(t, r | (g << 16), b);
    }
}

} // namespace bcf

namespace bcf {

// Texels [t0, t0 + nt) of a decoded block (t0 + nt <= 16), as
// bc6h_all_texels.  The index stream is entered at texel t0: the indices of
// texels 0 .. t0-1 occupy q t0 bits, minus one for texel 0 and one for the
// second anchor when it lies among them.  Each region's channels are kept as
// (64 a + 32, b - a), so a texel channel is (64 a + 32 + (b - a) w) >> 6 --
// the same integer as (a (64 - w) + b w + 32) >> 6.  Reserved modes have all
// endpoints zero, which decodes to zero texels.
template <class Store>
__device__ __forceinline__ void bc6h_texel_range(const Bc6hBlock &blk, const Bc6hHeader &H, bool sgn, int t0, int nt,
                                                 Store store)
{
    uint64_t idx;
    uint32_t pmask = 0;
    int a2 = 16;
    if (H.two) {
        pmask = partition_mask(H.partition);
        a2 = anchor2_of(H.partition);
        idx = blk.hi >> (18 + 3 * t0 - (t0 > 0) - (a2 < t0));
    } else {
        idx = blk.hi >> (1 + 4 * t0 - (t0 > 0));
    }
    int base0[3], del0[3], base1[3], del1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        base0[c] = 64 * H.e[0][c] + 32;
        del0[c] = H.e[1][c] - H.e[0][c];
        base1[c] = 64 * H.e[2][c] + 32;
        del1[c] = H.e[3][c] - H.e[2][c];
    }
#pragma unroll 1
    for (int t = t0; t < t0 + nt; ++t) {
        int w;
        if (H.two) {
            const int nb = (t == 0 || t == a2) ? 2 : 3;
            w = weight3((int)(idx & ((1u << nb) - 1)));
            idx >>= nb;
        } else {
            const int nb = t == 0 ? 3 : 4;
            w = weight4((int)(idx & ((1u << nb) - 1)));
            idx >>= nb;
        }
        const bool r1 = (pmask >> t) & 1;
        const uint32_t r = finish(((r1 ? base1[0] : base0[0]) + (r1 ? del1[0] : del0[0]) * w) >> 6, sgn);
        const uint32_t g = finish(((r1 ? base1[1] : base0[1]) + (r1 ? del1[1] : del0[1]) * w) >> 6, sgn);
        const uint32_t b = finish(((r1 ? base1[2] : base0[2]) + (r1 ? del1[2] : del0[2]) * w) >> 6, sgn);
        store(t, r | (g << 16), b);
    }
}

} // namespace bcf

namespace bcf {

// Per-block texel stage: the index stream normalised to a fixed field per
// texel (the anchors' implicit zero bit inserted), the region mask, and each
// region's channels as (64 a + 32, b - a).
struct Bc6hTexels {
    uint64_t stream; // index of texel t in bits [q t, q t + q)
    uint32_t pmask;  // region of texel t in bit t
    int q;           // 3 (two regions) or 4 (one region)
    int base[2][3], del[2][3];
};

__device__ __forceinline__ void bc6h_prepare_texels(const Bc6hBlock &blk, const Bc6hHeader &H, Bc6hTexels &X)
{
    if (H.two) {
        const uint64_t raw = blk.hi >> 18;                 // 46 index bits from bit 82
        const uint64_t s1 = ((raw >> 2) << 3) | (raw & 3); // texel 0: 2 stored bits -> a 3-bit field
        const int p = 3 * anchor2_of(H.partition) + 2;     // top bit of the second anchor's field
        X.stream = ((s1 >> p) << (p + 1)) | (s1 & ((1ull << p) - 1));
        X.pmask = partition_mask(H.partition);
        X.q = 3;
    } else {
        const uint64_t raw = blk.hi >> 1;                  // 63 index bits from bit 65
        X.stream = ((raw >> 3) << 4) | (raw & 7);          // texel 0: 3 stored bits -> a 4-bit field
        X.pmask = 0;
        X.q = 4;
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        X.base[0][c] = 64 * H.e[0][c] + 32;
        X.del[0][c] = H.e[1][c] - H.e[0][c];
        X.base[1][c] = 64 * H.e[2][c] + 32;
        X.del[1][c] = H.e[3][c] - H.e[2][c];
    }
}

// Texels t0 .. t0 + N - 1.  Weights: round(64 i / 7) = (146 i + 8) >> 4 for
// 3-bit indices and round(64 i / 15) = (273 i + 32) >> 6 for 4-bit indices
// (exact over the index ranges).  Unsigned scaling by 31/64 as one high
// multiply: (v 31) >> 6 = umulhi(v, 31 << 26) for 0 <= v < 2^16.
template <int N, int Q, bool SGN, class Store>
__device__ __forceinline__ void bc6h_texels_n(const Bc6hTexels &X, int t0, Store store)
{
    const uint64_t s = X.stream >> (Q * t0);
    const uint32_t pm = X.pmask >> t0;
#pragma unroll
    for (int j = 0; j < N; ++j) {
        const int i = (int)(s >> (Q * j)) & ((1 << Q) - 1);
        const int w = Q == 3 ? (146 * i + 8) >> 4 : (273 * i + 32) >> 6;
        const bool r1 = Q == 3 && ((pm >> j) & 1);
        uint32_t ch[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int v = ((r1 ? X.base[1][c] : X.base[0][c]) + (r1 ? X.del[1][c] : X.del[0][c]) * w) >> 6;
            ch[c] = SGN ? finish(v, true) : __umulhi((uint32_t)v, 31u << 26);
        }
        store(t0 + j, ch[0] | (ch[1] << 16), ch[2]);
    }
}

template <int N, class Store>
__device__ __forceinline__ void bc6h_texels(const Bc6hTexels &X, bool sgn, int t0, Store store)
{
    if (sgn) {
        if (X.q == 3)
            bc6h_texels_n<N, 3, true>(X, t0, store);
        else
            bc6h_texels_n<N, 4, true>(X, t0, store);
    } else {
        if (X.q == 3)
            bc6h_texels_n<N, 3, false>(X, t0, store);
        else
            bc6h_texels_n<N, 4, false>(X, t0, store);
    }
}

} // namespace bcf
