// bc6h_pack.cuh -- writers of BC6H UF16 / SF16 blocks in the two modes the library produces: mode 10 (two
// regions, 6-bit endpoints, 3-bit indices; the block features of Sec. 4.2 / Sec. 5.2) and mode 11 (one region,
// 10-bit endpoints, 4-bit indices).  Field order as the format defines it (the decoder in bc6h_unpack.cuh reads
// them back).
#pragma once
#include <stdint.h>

#include "bc6h_unpack.cuh"

namespace bcf {

struct BitWriter {
    uint64_t lo = 0, hi = 0;
    int pos = 0;
    __device__ void put(uint32_t v, int lsb, int n)
    {
        for (int j = 0; j < n; ++j, ++pos) {
            const uint64_t bit = (v >> (lsb + j)) & 1u;
            if (pos < 64)
                lo |= bit << pos;
            else
                hi |= bit << (pos - 64);
        }
    }
    __device__ uint4 block() const
    {
        return make_uint4((uint32_t)lo, (uint32_t)(lo >> 32), (uint32_t)hi, (uint32_t)(hi >> 32));
    }
};

// Mode 10 of partition k from 6-bit endpoint fields q[e][c] (e = 0, 1 region 0; 2, 3 region 1; SF16 codes as
// their low 6 bits) and 3-bit indices.  Where a region's anchor texel would need the top index bit the region's
// endpoints are swapped and its indices mirrored (i -> 7 - i), which keeps every texel value since the 3-bit
// weights satisfy w(7 - i) = 64 - w(i).
__device__ __forceinline__ uint4 bc6h_pack_mode10(int q[4][3], int idx[16], int k)
{
    const uint32_t pm = partition_mask(k);
    const int anchors[2] = {0, anchor2_of(k)};
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        if (idx[anchors[r]] >= 4) {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const int tmp = q[2 * r][c];
                q[2 * r][c] = q[2 * r + 1][c];
                q[2 * r + 1][c] = tmp;
            }
#pragma unroll
            for (int t = 0; t < 16; ++t)
                if ((int)((pm >> t) & 1) == r)
                    idx[t] = 7 - idx[t];
        }
    }
    const uint32_t r0 = q[0][0], g0 = q[0][1], b0 = q[0][2], r1 = q[1][0], g1 = q[1][1], b1 = q[1][2];
    const uint32_t r2 = q[2][0], g2 = q[2][1], b2 = q[2][2], r3 = q[3][0], g3 = q[3][1], b3 = q[3][2];
    BitWriter w;
    w.put(30u, 0, 5); // mode field 11110
    w.put(r0, 0, 6); w.put(g3, 4, 1); w.put(b3, 0, 1); w.put(b3, 1, 1); w.put(b2, 4, 1);
    w.put(g0, 0, 6); w.put(g2, 5, 1); w.put(b2, 5, 1); w.put(b3, 2, 1); w.put(g2, 4, 1);
    w.put(b0, 0, 6); w.put(g3, 5, 1); w.put(b3, 3, 1); w.put(b3, 5, 1); w.put(b3, 4, 1);
    w.put(r1, 0, 6); w.put(g2, 0, 4); w.put(g1, 0, 6); w.put(g3, 0, 4); w.put(b1, 0, 6);
    w.put(b2, 0, 4); w.put(r2, 0, 6); w.put(r3, 0, 6); w.put((uint32_t)k, 0, 5);
#pragma unroll
    for (int t = 0; t < 16; ++t)
        w.put((uint32_t)idx[t], 0, (t == 0 || t == anchors[1]) ? 2 : 3);
    return w.block();
}

// Mode 11 from 10-bit endpoint fields q[e][c] (e = 0, 1) and 4-bit indices; texel 0 is the anchor (its index
// must fit 3 bits: otherwise the endpoints are swapped and the indices mirrored, i -> 15 - i, which keeps every
// texel value since the 4-bit weights satisfy w(15 - i) = 64 - w(i)).
__device__ __forceinline__ uint4 bc6h_pack_mode11(int q[2][3], int idx[16])
{
    if (idx[0] >= 8) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const int tmp = q[0][c];
            q[0][c] = q[1][c];
            q[1][c] = tmp;
        }
#pragma unroll
        for (int t = 0; t < 16; ++t)
            idx[t] = 15 - idx[t];
    }
    BitWriter w;
    w.put(3u, 0, 5); // mode field 00011
#pragma unroll
    for (int e = 0; e < 2; ++e)
#pragma unroll
        for (int c = 0; c < 3; ++c)
            w.put((uint32_t)q[e][c], 0, 10);
#pragma unroll
    for (int t = 0; t < 16; ++t)
        w.put((uint32_t)idx[t], 0, t == 0 ? 3 : 4);
    return w.block();
}

} // namespace bcf
