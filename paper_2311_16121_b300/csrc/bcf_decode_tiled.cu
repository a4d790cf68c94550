// bcf_decode_tiled.cu -- tile-cooperative fused decode (Eq. 3 with Eq. 10 / 11
// filtering over BC6H features).
//
// A CTA takes 256 consecutive queries (one per thread).  Screen queries are
// spatially coherent, so their bilinear footprints share BC6H blocks.  Instead
// of every lane decoding the blocks its own footprint touches, the CTA:
//   1. finds, per texture, the mip levels its queries use and, per level, the
//      box of blocks their footprints touch (warp reductions + shared atomics,
//      block coordinates taken relative to the first query so that boxes
//      straddling the repeat seam stay compact);
//   2. groups the textures into rounds whose boxes fit the shared-memory
//      arena; per round it loads each block once (16-byte loads, kept in
//      registers), counting-sorts the blocks by BC6H mode (warp-aggregated
//      shared atomics) so that a warp decodes blocks of (mostly) one mode, and
//      decodes all 16 texels of every block into the arena (8 bytes per texel,
//      texel slots XOR-swizzled by the block index to spread banks);
//   3. lets every query filter its 2 x 2 footprints trilinearly from the arena
//      in FP32 (exact weights, Eq. 10) and write its quantised feature row
//      straight into its warp's MLP input tile;
//   4. runs the MLP on the tensor cores per warp (register-chained layers for
//      the common 3-layer shapes) and stores the channels coalesced.
// A texture whose boxes alone exceed the arena, or that spans more than three
// levels in the tile, is filtered by the per-lane decode instead.
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "bc6h_unpack.cuh"
#include "bcf_kernels.h"
#include "bcf_mlp.cuh"
#include "bcf_sample.cuh"
#include "bcf_tcmlp.cuh"

namespace bcf {

constexpr int kTileQ = 256;    // queries per CTA tile, one per thread
constexpr int kMaxLv = 3;      // mip levels per texture held per tile
constexpr int kBoxes = BCF_MAX_TEX * kMaxLv;
constexpr int kBins = 15;      // 14 modes + reserved
#ifndef BCF_MAX_SET
#define BCF_MAX_SET 256        // materials per material set
#endif

struct TileMeta {
    float u0, v0;
    int smin_bits, smax_bits;  // tile LOD range (order-preserving integer images of the floats)
    int nrounds;
    int lmin[BCF_MAX_TEX];     // per geometry group: levels [lmin, lmax] hold the tile's footprints
    int lmax[BCF_MAX_TEX];
    int direct[BCF_MAX_TEX];   // per group: 1 = filtered by the per-lane decode
    int gtotal[BCF_MAX_TEX];   // per group: blocks of one texture's boxes
    int bb[kBoxes][4];         // per (group, level slot): min x, max x, min y, max y (relative block coordinates)
    int bw[kBoxes];            // box width in blocks
    int boff[kBoxes];          // offset of the box inside one texture's block set
    int tbase[BCF_MAX_TEX];    // per texture: first arena block of its block set within its round
    int rtex[BCF_MAX_TEX + 1]; // textures [rtex[r], rtex[r+1]) form round r
    int rtotal[BCF_MAX_TEX];   // blocks of round r
    int hist[16];              // blocks per mode bin of the current round
};

// LOD of texture T for query LOD s: level floor(s_t), whether floor(s_t) + 1
// is also sampled, and the lerp fraction (identical arithmetic everywhere).
struct Lod {
    int l0, nlev;
    float lam;
};

__device__ __forceinline__ Lod lod_of(const TexDev &T, float s)
{
    float st = (isnan(s) ? 0.0f : s) + (float)T.lod_bias;
    st = fminf(fmaxf(st, 0.0f), (float)(T.levels - 1));
    const float fl = floorf(st);
    Lod L;
    L.l0 = (int)fl;
    L.lam = st - fl;
    L.nlev = (L.lam > 0.0f && L.l0 + 1 < T.levels) ? 2 : 1;
    return L;
}

// Order-preserving map float -> int (for atomicMin / atomicMax on floats).
__device__ __forceinline__ int f2ord(float f)
{
    const int i = __float_as_int(f);
    return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float ord2f(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

__device__ __forceinline__ int wraprel(int b, int rb, int wb)
{
    const int h = wb >> 1;
    return ((b - rb + h) & (wb - 1)) - h;
}

// Block coordinate (relative to the tile reference for repeat addressing,
// absolute for clamp) of texel column / row i, given the footprint's first
// column i0 and the reference block rb.
__device__ __forceinline__ int rel_block(int i, int i0, int rb, int W, int wrap)
{
    if (wrap)
        return wraprel(i0 >> 2, rb, W >> 2) + ((i >> 2) - (i0 >> 2));
    return min(max(i, 0), W - 1) >> 2;
}

__device__ __forceinline__ int texel_col(int i, int W, int wrap) { return wrap ? (i & 3) : (min(max(i, 0), W - 1) & 3); }

__device__ __forceinline__ int ref_block(float c0, int W) { return ((int)floorf(c0 * (float)W - 0.5f)) >> 2; }

// Arena slot of texel t of arena block b (XOR swizzle spreads the 8-byte
// texels of different blocks over the banks).
__device__ __forceinline__ int arena_slot(int b, int t) { return b * 16 + (t ^ (b & 15)); }


// Shared memory layout of the kernel (host and device agree through this).
struct TiledLayout {
    int w_bytes, b_bytes, meta, sraw, sidx, arena, per_warp, act0, act1, tmp8, ost, total;
};

template <int PREC>
__host__ __device__ inline TiledLayout tiled_layout(const MlpDev &P, int cap, bool generic_mlp)
{
    TiledLayout L;
    const int C = P.dims[P.n_layers];
    int off = 0;
    L.w_bytes = mlp_smem_weight_bytes<PREC>(P);
    off += L.w_bytes;
    L.b_bytes = off;
    off += (mlp_smem_bias_floats(P) * 4 + 15) & ~15;
    L.meta = off;
    off += (int)((2 * sizeof(TileMeta) + 15) & ~15); // double-buffered across tiles
    L.sraw = off;
    off += cap * 16;
    L.sidx = off;
    off += (cap * 2 + 15) & ~15;
    L.arena = off;
    off += cap * 16 * 8;
    // per warp: input tile, (generic MLP: second activation tile), FP8 chaining tile, output staging
    int act = 0;
    for (int l = 0; l < P.n_layers; ++l)
        act = act > 32 * tile_stride_bytes<PREC>(P.kpad[l]) ? act : 32 * tile_stride_bytes<PREC>(P.kpad[l]);
    act = (act + 15) & ~15;
    int maxn = 0;
    for (int l = 0; l < P.n_layers; ++l)
        maxn = maxn > P.npad[l] ? maxn : P.npad[l];
    const int tmp = PREC == BCF_FP8_E4M3 ? ((16 * (maxn + 16) + 15) & ~15) : 0; // one 16-row pass (MlpRows)
    const int ostb = (32 * C * 4 + 15) & ~15;
    L.act0 = 0;
    if (generic_mlp) {
        L.act1 = act;
        L.tmp8 = 2 * act;
        L.ost = L.tmp8 + tmp;
        L.per_warp = L.ost + ostb;
    } else {
        // The register-chained MLP loads the A fragments of all rows of a pass (16 or 32 rows) before it
        // writes that pass's outputs.  The output staging may share the input tile when the outputs of
        // rows 0-15 (16 * C floats) end before input row 16 begins.
        const int in_stride = tile_stride_bytes<PREC>(P.kpad[0]);
        const int in0 = (32 * in_stride + 15) & ~15;
        const bool alias = 16 * C * 4 <= 16 * in_stride;
        const int a0 = alias ? (in0 > ostb ? in0 : ostb) : in0 + ostb;
        L.act1 = 0;
        L.ost = alias ? 0 : in0;
        L.tmp8 = a0;
        L.per_warp = a0 + tmp;
    }
    L.total = off + (kTileQ / 32) * L.per_warp;
    return L;
}

// Shared-memory pointers of one CTA (carved from the dynamic shared memory
// by carve()).
struct TileCtx {
    TileMeta *TM;      // this tile's metadata
    TileMeta *TMnext;  // the other buffer (the next tile's)
    uint4 *sraw;
    uint16_t *sidx;
    uint2 *arena;
    unsigned char *sw;
    float *sb;
    unsigned char *act0, *act1, *tmp8;
    float *ost;
};

template <int PREC>
__device__ __forceinline__ TileCtx carve(unsigned char *smem, const MlpDev &P, int cap, bool generic)
{
    const TiledLayout LY = tiled_layout<PREC>(P, cap, generic);
    TileCtx C;
    C.sw = smem;
    C.sb = (float *)(smem + LY.b_bytes);
    C.TM = (TileMeta *)(smem + LY.meta);
    C.TMnext = C.TM + 1;
    C.sraw = (uint4 *)(smem + LY.sraw);
    C.sidx = (uint16_t *)(smem + LY.sidx);
    C.arena = (uint2 *)(smem + LY.arena);
    const int warp = threadIdx.x >> 5;
    unsigned char *wbase = smem + LY.total - (kTileQ / 32 - warp) * LY.per_warp;
    C.act0 = wbase + LY.act0;
    C.act1 = wbase + LY.act1;
    C.tmp8 = wbase + LY.tmp8;
    C.ost = (float *)(wbase + LY.ost);
    return C;
}

// Reset the fields a tile accumulates into (LOD range, boxes, mode histogram).
__device__ __forceinline__ void reset_tile_meta(TileMeta &T)
{
    if (threadIdx.x == 0) {
        T.smin_bits = INT_MAX;
        T.smax_bits = INT_MIN;
    }
    if (threadIdx.x < 16)
        T.hist[threadIdx.x] = 0;
    for (int i = threadIdx.x; i < kBoxes; i += kTileQ) {
        T.bb[i][0] = T.bb[i][2] = INT_MAX;
        T.bb[i][1] = T.bb[i][3] = INT_MIN;
    }
}

__device__ __forceinline__ void swap_meta(TileCtx &C)
{
    TileMeta *t = C.TM;
    C.TM = C.TMnext;
    C.TMnext = t;
}

// One tile of 256 queries [q_first, q_first + 256) clipped to q_end; this
// thread's query is (u, v, s) (already sanitised; zeros when inactive).
// Every thread of the CTA calls it (it synchronises the CTA).
template <int PREC, int CAP, int K0, int N1, int N2, int NO>
__device__ __forceinline__ void decode_tile(const MaterialDev &M, const TileCtx &C, int64_t q_first, int64_t q_end,
                                            const float u, const float v, const float s, void *__restrict__ out,
                                            int out_fp16)
{
    const MlpDev &P = M.mlp;
    TileMeta &TM = *C.TM;
    uint4 *sraw = C.sraw;
    uint16_t *sidx = C.sidx;
    uint2 *arena = C.arena;
    unsigned char *sw = C.sw;
    float *sb = C.sb;
    unsigned char *act0 = C.act0, *act1 = C.act1, *tmp8 = C.tmp8;
    float *ost = C.ost;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int Cn = P.dims[P.n_layers];
    const int row_stride = tile_stride_bytes<PREC>(P.kpad[0]);
    unsigned char *myrow = act0 + lane * row_stride;
    const float inv0 = PREC == BCF_FP8_E4M3 ? P.inv_act_scale[0] : 1.0f;
    const int nt = M.n_tex;
    const int ng = M.n_groups;
    const int wrap = M.wrap;
    const bool sgn = M.is_signed != 0;
    const unsigned lanes_lt = (1u << lane) - 1u;
    const int64_t q = q_first + threadIdx.x;
    const bool active = q < q_end;
        // ---- this tile's metadata was reset during the previous tile (or before the first); reset the other
        // buffer for the next tile now: its last readers (the previous tile's phases) are behind a barrier
        reset_tile_meta(*C.TMnext);
        if (threadIdx.x == 0) {
            TM.u0 = u;
            TM.v0 = v;
        }

        // ---- 1a. LOD range of the tile (NaN reads as 0, as in lod_of)
        {
            const float sl = isnan(s) ? 0.0f : s;
            const int lo = __reduce_min_sync(0xffffffffu, active ? f2ord(sl) : INT_MAX);
            const int hi = __reduce_max_sync(0xffffffffu, active ? f2ord(sl) : INT_MIN);
            if (lane == 0 && lo != INT_MAX) {
                atomicMin(&TM.smin_bits, lo);
                atomicMax(&TM.smax_bits, hi);
            }
        }
        __syncthreads();
        // ---- 1b. block box per (group, level)
        const float u0 = TM.u0, v0 = TM.v0;
        const float smin = ord2f(TM.smin_bits), smax = ord2f(TM.smax_bits);
        for (int g = 0; g < ng; ++g) {
            const TexDev &T = M.tex[M.group_first[g]];
            // every l0 of the tile lies in [lod(smin).l0, lod(smax).l0]; the upper level adds at most one
            const int lmin = lod_of(T, smin).l0;
            const int lmax = min(lod_of(T, smax).l0 + 1, T.levels - 1);
            if (threadIdx.x == 0) {
                TM.lmin[g] = lmin;
                TM.lmax[g] = lmax;
            }
            if (lmax - lmin + 1 > kMaxLv)
                continue; // this group is filtered per lane
            const Lod L = lod_of(T, s);
            int bx[2][2], by[2][2]; // [side][lo/hi]
            int slot[2] = {-1, -1};
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                bx[side][0] = bx[side][1] = by[side][0] = by[side][1] = 0;
                if (active && side < L.nlev) {
                    const int level = L.l0 + side;
                    const int W = T.res >> level;
                    const int i0 = (int)floorf(u * (float)W - 0.5f), j0 = (int)floorf(v * (float)W - 0.5f);
                    const int rbx = wrap ? ref_block(u0, W) : 0, rby = wrap ? ref_block(v0, W) : 0;
                    bx[side][0] = rel_block(i0, i0, rbx, W, wrap);
                    bx[side][1] = rel_block(i0 + 1, i0, rbx, W, wrap);
                    by[side][0] = rel_block(j0, j0, rby, W, wrap);
                    by[side][1] = rel_block(j0 + 1, j0, rby, W, wrap);
                    slot[side] = level - lmin;
                }
            }
#pragma unroll
            for (int ls = 0; ls < kMaxLv; ++ls) {
                const int sd = slot[0] == ls ? 0 : (slot[1] == ls ? 1 : -1);
                const int mnx = __reduce_min_sync(0xffffffffu, sd >= 0 ? bx[sd][0] : INT_MAX);
                const int mxx = __reduce_max_sync(0xffffffffu, sd >= 0 ? bx[sd][1] : INT_MIN);
                const int mny = __reduce_min_sync(0xffffffffu, sd >= 0 ? by[sd][0] : INT_MAX);
                const int mxy = __reduce_max_sync(0xffffffffu, sd >= 0 ? by[sd][1] : INT_MIN);
                if (lane == 0 && mnx != INT_MAX) {
                    int *bb = TM.bb[g * kMaxLv + ls];
                    atomicMin(&bb[0], mnx);
                    atomicMax(&bb[1], mxx);
                    atomicMin(&bb[2], mny);
                    atomicMax(&bb[3], mxy);
                }
            }
        }
        __syncthreads();
        // ---- 1c. per-group block sets and arena rounds of consecutive textures.  Warp 0: lane k sizes box k,
        // per-group totals and per-texture bases by shuffles; when everything fits the arena (the common case)
        // that is one round; otherwise thread 0 packs the rounds.
        bool fits = false;
        if (warp == 0 && ng * kMaxLv <= 32) {
            const int nbox = ng * kMaxLv;
            int size = 0;
            if (lane < nbox) {
                const int *bb = TM.bb[lane];
                const int bw = bb[0] != INT_MAX ? bb[1] - bb[0] + 1 : 0;
                TM.bw[lane] = bw;
                size = bw ? bw * (bb[3] - bb[2] + 1) : 0;
            }
            // inclusive scan of the box sizes within each group of kMaxLv lanes
            int incl = size;
#pragma unroll
            for (int d = 1; d < kMaxLv; d <<= 1) {
                const int o = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane % kMaxLv >= d)
                    incl += o;
            }
            if (lane < nbox)
                TM.boff[lane] = incl - size;
            const int gt = __shfl_sync(0xffffffffu, incl, lane < ng ? lane * kMaxLv + kMaxLv - 1 : 0);
            int direct = 0;
            if (lane < ng) {
                direct = TM.lmax[lane] - TM.lmin[lane] + 1 > kMaxLv || gt > CAP;
                TM.direct[lane] = direct;
                TM.gtotal[lane] = direct ? 0 : gt;
            }
            __syncwarp();
            // per-texture bases: exclusive scan of the group totals over the textures
            const int tt = lane < nt ? TM.gtotal[M.tex_group[lane]] : 0;
            int ti = tt;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int o = __shfl_up_sync(0xffffffffu, ti, d);
                if (lane >= d)
                    ti += o;
            }
            const int grand = __shfl_sync(0xffffffffu, ti, 31);
            fits = grand <= CAP;
            if (fits) {
                if (lane < nt)
                    TM.tbase[lane] = ti - tt;
                if (lane == 0) {
                    TM.rtex[0] = 0;
                    TM.rtex[1] = nt;
                    TM.rtotal[0] = grand;
                    TM.nrounds = 1;
                }
            }
        }
        if (warp == 0 && lane == 0 && !fits) {
            for (int g = 0; g < ng; ++g) {
                int tt = 0;
                for (int ls = 0; ls < kMaxLv; ++ls) {
                    const int k = g * kMaxLv + ls;
                    const int *bb = TM.bb[k];
                    TM.boff[k] = tt;
                    TM.bw[k] = bb[0] != INT_MAX ? bb[1] - bb[0] + 1 : 0;
                    tt += bb[0] != INT_MAX ? TM.bw[k] * (bb[3] - bb[2] + 1) : 0;
                }
                TM.direct[g] = TM.lmax[g] - TM.lmin[g] + 1 > kMaxLv || tt > CAP;
                TM.gtotal[g] = TM.direct[g] ? 0 : tt;
            }
            int r = 0, acc = 0;
            TM.rtex[0] = 0;
            for (int t = 0; t < nt; ++t) {
                const int tt = TM.gtotal[M.tex_group[t]];
                if (acc + tt > CAP) { // close the current round
                    TM.rtotal[r] = acc;
                    ++r;
                    TM.rtex[r] = t;
                    acc = 0;
                }
                TM.tbase[t] = acc;
                acc += tt;
            }
            TM.rtotal[r] = acc;
            TM.rtex[r + 1] = nt;
            TM.nrounds = r + 1;
        }
        __syncthreads();
        const int nrounds = TM.nrounds;
        for (int r = 0; r < nrounds; ++r) {
            const int t_beg = TM.rtex[r], t_end = TM.rtex[r + 1], total = TM.rtotal[r];
            if (total > 0) {
                // ---- 2. load each block once (two per thread); its rank among the blocks of its mode comes
                // from the (warp-aggregated) histogram atomic
                uint4 blk[2];
                int bin[2], bidx[2], rank[2];
#pragma unroll
                for (int it = 0; it < 2; ++it) {
                    const int b = it * kTileQ + threadIdx.x;
                    const bool valid = b < total;
                    bin[it] = kBins + lane; // unique per lane when invalid: no aggregation
                    bidx[it] = b;
                    blk[it] = make_uint4(0, 0, 0, 0);
                    if (valid) {
                        int t = t_beg;
                        while (b >= TM.tbase[t] + TM.gtotal[M.tex_group[t]])
                            ++t;
                        const int g = M.tex_group[t];
                        const int local0 = b - TM.tbase[t];
                        int k = g * kMaxLv;
                        while (TM.bw[k] == 0 || local0 >= TM.boff[k] + TM.bw[k] * (TM.bb[k][3] - TM.bb[k][2] + 1))
                            ++k;
                        const TexDev &T = M.tex[t];
                        const int level = TM.lmin[g] + (k - g * kMaxLv);
                        const int local = local0 - TM.boff[k];
                        const int bwk = TM.bw[k];
                        const int ry = local / bwk;
                        const int W = T.res >> level, wb = W >> 2;
                        int bxa = TM.bb[k][0] + (local - ry * bwk), bya = TM.bb[k][2] + ry;
                        if (wrap) {
                            bxa = (ref_block(u0, W) + bxa) & (wb - 1);
                            bya = (ref_block(v0, W) + bya) & (wb - 1);
                        }
                        blk[it] = __ldg(T.blocks + level_offset((uint32_t)(T.res >> 2), level) +
                                        (uint32_t)bya * (uint32_t)wb + (uint32_t)bxa);
                        const int mi = mode_index(blk[it].x);
                        bin[it] = mi < 0 ? kBins - 1 : mi;
                    }
                    const unsigned peers = __match_any_sync(0xffffffffu, bin[it]);
                    const int leader = __ffs(peers) - 1;
                    int base = 0;
                    if (valid && lane == leader)
                        base = atomicAdd(&TM.hist[bin[it]], __popc(peers));
                    rank[it] = __shfl_sync(0xffffffffu, base, leader) + __popc(peers & lanes_lt);
                }
                __syncthreads();
                // ---- 3. scatter into mode-sorted order: position = blocks of smaller modes + rank
#pragma unroll
                for (int it = 0; it < 2; ++it) {
                    if (bidx[it] < total) {
                        int pos = rank[it];
                        for (int i = 0; i < bin[it]; ++i)
                            pos += TM.hist[i];
                        sraw[pos] = blk[it];
                        sidx[pos] = (uint16_t)bidx[it];
                    }
                }
                __syncthreads();
                if (threadIdx.x < 16)
                    TM.hist[threadIdx.x] = 0; // for the next round (read again only after the decode barrier)
                // ---- 4. decode the sorted blocks into the texel arena.  The phase's length is one thread's
                // chain (header + its texels), so a block is split over 1, 2 or 4 threads (each decodes the
                // header and 16, 8 or 4 texels), the most that keeps all parts in one pass of the CTA;
                // neighbouring lanes take parts of the same block.
                const int lk = total <= 64 ? 2 : total <= 128 ? 1 : 0;
                for (int i = threadIdx.x; i < (total << lk); i += kTileQ) {
                    const int e = i >> lk, part = i & ((1 << lk) - 1);
                    const uint4 rr = sraw[e];
                    const int bi = sidx[e];
                    Bc6hBlock bk;
                    bk.lo = (uint64_t)rr.x | ((uint64_t)rr.y << 32);
                    bk.hi = (uint64_t)rr.z | ((uint64_t)rr.w << 32);
                    Bc6hHeader H;
                    bc6h_header(bk, sgn, H);
                    Bc6hTexels X;
                    bc6h_prepare_texels(bk, H, X);
                    const auto put = [&](int t, uint32_t rg, uint32_t bb) { arena[arena_slot(bi, t)] = make_uint2(rg, bb); };
                    if (lk == 0)
                        bc6h_texels<16>(X, sgn, 0, put);
                    else if (lk == 1)
                        bc6h_texels<8>(X, sgn, part * 8, put);
                    else
                        bc6h_texels<4>(X, sgn, part * 4, put);
                }
                __syncthreads();
                // ---- 5. filter: per group, the footprint geometry once; per texture, 4 arena texels per level
                for (int g = 0; g < ng; ++g) {
                    if (TM.direct[g])
                        continue;
                    const TexDev &T = M.tex[M.group_first[g]];
                    int ofs[2][4], tex_i[2][4];
                    float wgt[2][4];
                    int nlev = 0;
                    if (active) {
                        const Lod L = lod_of(T, s);
                        nlev = L.nlev;
#pragma unroll
                        for (int side = 0; side < 2; ++side) {
                            const int level = L.l0 + (side < L.nlev ? side : 0);
                            const float scale = L.nlev == 1 ? 1.0f : (side ? L.lam : 1.0f - L.lam);
                            const int W = T.res >> level;
                            const float x = u * (float)W - 0.5f, y = v * (float)W - 0.5f;
                            const float fx0 = floorf(x), fy0 = floorf(y);
                            const float fx = x - fx0, fy = y - fy0;
                            const int i0 = (int)fx0, j0 = (int)fy0;
                            const int k = g * kMaxLv + level - TM.lmin[g];
                            const int rbx = wrap ? ref_block(u0, W) : 0, rby = wrap ? ref_block(v0, W) : 0;
                            const int bwk = TM.bw[k], bhk = TM.bb[k][3] - TM.bb[k][2] + 1;
                            // the box was built from the same integer coordinates, so these are inside it; the
                            // clamps only guarantee in-bounds shared-memory reads
                            const int bxl = min(max(rel_block(i0, i0, rbx, W, wrap) - TM.bb[k][0], 0), bwk - 1);
                            const int bxh = min(max(rel_block(i0 + 1, i0, rbx, W, wrap) - TM.bb[k][0], 0), bwk - 1);
                            const int byl = min(max(rel_block(j0, j0, rby, W, wrap) - TM.bb[k][2], 0), bhk - 1);
                            const int byh = min(max(rel_block(j0 + 1, j0, rby, W, wrap) - TM.bb[k][2], 0), bhk - 1);
                            const int cl = texel_col(i0, W, wrap), ch = texel_col(i0 + 1, W, wrap);
                            const int rl = texel_col(j0, W, wrap) * 4, rh = texel_col(j0 + 1, W, wrap) * 4;
                            const int o = TM.boff[k];
                            ofs[side][0] = o + byl * bwk + bxl;
                            ofs[side][1] = o + byl * bwk + bxh;
                            ofs[side][2] = o + byh * bwk + bxl;
                            ofs[side][3] = o + byh * bwk + bxh;
                            tex_i[side][0] = rl + cl;
                            tex_i[side][1] = rl + ch;
                            tex_i[side][2] = rh + cl;
                            tex_i[side][3] = rh + ch;
                            wgt[side][0] = (1.0f - fx) * (1.0f - fy) * scale;
                            wgt[side][1] = fx * (1.0f - fy) * scale;
                            wgt[side][2] = (1.0f - fx) * fy * scale;
                            wgt[side][3] = fx * fy * scale;
                        }
                    }
                    for (int t = t_beg; t < t_end; ++t) {
                        if (M.tex_group[t] != g)
                            continue;
                        float f0 = 0.0f, f1 = 0.0f, f2 = 0.0f;
                        const int tb = TM.tbase[t];
#pragma unroll
                        for (int side = 0; side < 2; ++side) {
                            if (side < nlev) {
#pragma unroll
                                for (int c = 0; c < 4; ++c) {
                                    const uint2 tx = arena[arena_slot(tb + ofs[side][c], tex_i[side][c])];
                                    const float2 rg = __half22float2(*reinterpret_cast<const __half2 *>(&tx.x));
                                    f0 = fmaf(wgt[side][c], rg.x, f0);
                                    f1 = fmaf(wgt[side][c], rg.y, f1);
                                    f2 = fmaf(wgt[side][c], __half2float(__ushort_as_half((unsigned short)tx.y)), f2);
                                }
                            }
                        }
                        store_feature<PREC>(myrow, 3 * t, f0, inv0);
                        store_feature<PREC>(myrow, 3 * t + 1, f1, inv0);
                        store_feature<PREC>(myrow, 3 * t + 2, f2, inv0);
                    }
                }
            }
            __syncthreads(); // the arena is refilled by the next round / tile
        }
        // ---- 5b. textures of groups that did not fit: per-lane decode
        for (int t = 0; t < nt; ++t) {
            if (!TM.direct[M.tex_group[t]])
                continue;
            float3 f = make_float3(0.f, 0.f, 0.f);
            if (active)
                f = sample_texture(M.tex[t], wrap, sgn, u, v, s);
            store_feature<PREC>(myrow, 3 * t, f.x, inv0);
            store_feature<PREC>(myrow, 3 * t + 1, f.y, inv0);
            store_feature<PREC>(myrow, 3 * t + 2, f.z, inv0);
        }
        {
            int col = 3 * nt;
            if (M.lod_input) {
                store_feature<PREC>(myrow, col, active ? (isnan(s) ? 0.0f : fmaxf(s, 0.0f)) : 0.0f, inv0);
                ++col;
            }
            for (; col < P.kpad[0]; ++col)
                store_feature<PREC>(myrow, col, 0.0f, inv0);
        }
        __syncwarp();
        // ---- 6. MLP on the tensor cores, coalesced store
        if constexpr (K0 == 0)
            warp_mlp<PREC>(P, sw, sb, act0, act1, ost);
        else if constexpr (N2 == 0) // one hidden layer
            warp_mlp2<PREC, K0, N1, NO>(sw, sb, act0, row_stride, ost, Cn);
        else
            warp_mlp3<PREC, K0, N1, N2, NO>(P, sw, sb, act0, row_stride, tmp8,
                                            tile_stride_bytes<BCF_FP8_E4M3>(N1 > N2 ? N1 : N2), ost, Cn);
        __syncwarp();
        const int64_t q0 = q_first + warp * 32;
        if (q0 < q_end) {
            const int rows = (int)min((int64_t)32, q_end - q0);
            const int tot = rows * Cn;
            if (out_fp16) {
                __half *o = (__half *)out + q0 * Cn;
                for (int i = lane; i < tot; i += 32)
                    o[i] = __float2half_rn(ost[i]);
            } else {
                float *o = (float *)out + q0 * Cn;
                for (int i = lane; i < tot; i += 32)
                    o[i] = ost[i];
            }
        }
        __syncwarp();
}

// Single material: the material is a kernel parameter; tiles are assigned
// round-robin to the persistent CTAs, queries are loaded one tile ahead.
template <int PREC, int CAP, int K0, int N1, int N2, int NO>
__global__ void __launch_bounds__(kTileQ, 3) k_decode_tiled(MaterialDev M, const float *__restrict__ qu,
                                                            const float *__restrict__ qv,
                                                            const float *__restrict__ qs, int64_t n,
                                                            void *__restrict__ out, int out_fp16)
{
    static_assert(CAP <= 2 * kTileQ, "blocks are held two per thread while sorting");
    extern __shared__ __align__(16) unsigned char smem[];
    TileCtx C = carve<PREC>(smem, M.mlp, CAP, K0 == 0);
    const int wrap = M.wrap;
    load_mlp_smem<PREC>(M.mlp, C.sw, C.sb);
    reset_tile_meta(*C.TM);
    __syncthreads();
    const int64_t tiles = (n + kTileQ - 1) / kTileQ;
    float nu = 0.0f, nv = 0.0f, ns = 0.0f;
    {
        const int64_t q = (int64_t)blockIdx.x * kTileQ + threadIdx.x;
        if (blockIdx.x < tiles && q < n) {
            nu = qu[q];
            nv = qv[q];
            ns = qs ? qs[q] : 0.0f;
        }
    }
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t q = tile * kTileQ + threadIdx.x;
        const bool active = q < n;
        const float u = active ? sanitize(nu, wrap) : 0.0f;
        const float v = active ? sanitize(nv, wrap) : 0.0f;
        const float s = active ? ns : 0.0f;
        {
            const int64_t qn = (tile + gridDim.x) * kTileQ + threadIdx.x;
            if (tile + gridDim.x < tiles && qn < n) {
                nu = qu[qn];
                nv = qv[qn];
                ns = qs ? qs[qn] : 0.0f;
            }
        }
        decode_tile<PREC, CAP, K0, N1, N2, NO>(M, C, tile * kTileQ, n, u, v, s, out, out_fp16);
        swap_meta(C);
    }
}

// Material set: materials in a device table, material m's queries are
// [offsets[m], offsets[m+1]) of the concatenated arrays.  Tiles are numbered
// material by material; CTAs take `chunk` consecutive tiles at a time from an
// atomic work counter (zeroed before the launch) and reload the material's
// metadata and MLP weights into shared memory when a tile belongs to a new
// material.  Offsets are clipped to [0, n], so malformed ranges cannot
// address outside the query and output arrays; a decreasing pair sets the
// offsets check bit (its range is empty).
template <int PREC, int CAP, int K0, int N1, int N2, int NO>
__global__ void __launch_bounds__(kTileQ, 3) k_decode_set(const MaterialDev *__restrict__ mats, int nmat,
                                                          const int64_t *__restrict__ offsets, const float *__restrict__ qu,
                                                          const float *__restrict__ qv, const float *__restrict__ qs,
                                                          int64_t n, void *__restrict__ out, int out_fp16,
                                                          int *__restrict__ counter, unsigned *__restrict__ check,
                                                          int chunk)
{
    static_assert(CAP <= 2 * kTileQ, "blocks are held two per thread while sorting");
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ MaterialDev Ms;
    __shared__ int64_t tile_first[BCF_MAX_SET + 1];
    __shared__ int grab;
    // every material shares the MLP shape (checked when the set is created), so the layout is that of material 0
    TileCtx C = carve<PREC>(smem, mats[0].mlp, CAP, K0 == 0);
    reset_tile_meta(*C.TM);
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int m = 0; m < nmat; ++m) {
            tile_first[m] = acc;
            const int64_t a = min(max(offsets[m], (int64_t)0), n), b = min(max(offsets[m + 1], (int64_t)0), n);
            acc += b > a ? (b - a + kTileQ - 1) / kTileQ : 0;
            if (blockIdx.x == 0 && offsets[m + 1] < offsets[m] && check)
                atomicOr(check, BCF_CHECK_OFFSETS);
        }
        tile_first[nmat] = acc;
    }
    __syncthreads();
    const int64_t total = tile_first[nmat];
    int cur = -1;
    for (;;) {
        if (threadIdx.x == 0)
            grab = atomicAdd(counter, chunk);
        __syncthreads();
        const int64_t base = grab;
        __syncthreads(); // everyone has read `grab` before thread 0 may overwrite it
        if (base >= total)
            break;
        for (int j = 0; j < chunk && base + j < total; ++j) {
            const int64_t tile = base + j;
            int lo = 0, hi = nmat - 1; // last m with tile_first[m] <= tile
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tile_first[mid] <= tile)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const int m = lo;
            if (m != cur) {
                __syncthreads(); // the previous tile's MLP may still read the weights being replaced
                const int words = (int)(sizeof(MaterialDev) / 4);
                for (int i = threadIdx.x; i < words; i += kTileQ)
                    reinterpret_cast<int *>(&Ms)[i] = reinterpret_cast<const int *>(mats + m)[i];
                __syncthreads();
                load_mlp_smem<PREC>(Ms.mlp, C.sw, C.sb);
                cur = m;
                // (the first __syncthreads of decode_tile orders the loads before their use)
            }
            const int64_t a = min(max(offsets[m], (int64_t)0), n), b = min(max(offsets[m + 1], (int64_t)0), n);
            const int64_t q0 = a + (tile - tile_first[m]) * kTileQ;
            const int64_t q = q0 + threadIdx.x;
            const bool active = q < b;
            const int wrap = Ms.wrap;
            float u = 0.0f, v = 0.0f, s = 0.0f;
            if (active) {
                u = sanitize(qu[q], wrap);
                v = sanitize(qv[q], wrap);
                s = qs ? qs[q] : 0.0f;
            }
            decode_tile<PREC, CAP, K0, N1, N2, NO>(Ms, C, q0, b, u, v, s, out, out_fp16);
            swap_meta(C);
        }
    }
}

// ------------------------------------------------- single-geometry tiles

// Materials whose textures all share one resolution and level count (one geometry group) take a leaner tile
// kernel over tiles of TQ queries (one per thread; 512 or 256, see geo_tq): the footprint geometry is computed
// once per query and kept in registers, the tile's block boxes are
// kept per absolute level (no separate LOD-range pass), every thread sizes the block set itself (no planning
// warp), and a tile costs four CTA barriers:
//   1. per query: LOD, levels and footprint per side; per warp and level the block box by warp reductions,
//      merged into the tile's boxes with shared atomics (block coordinates relative to the tile's first query,
//      so that boxes across the repeat seam stay compact)                                   -- barrier 1
//   2. the textures in rounds that fit the arena; per round every block of every texture of the round is
//      loaded once with a 16-byte load and ranked among the round's blocks of its BC6H mode  -- barrier 2
//   3. scattered into mode order (so that a warp decodes blocks of few modes)               -- barrier 3
//   4. decoded, all 16 texels, into the texel arena                                         -- barrier 4
//   5. filtered per query from the arena (exact FP32, the per-lane decode's operation order) into the warp's
//      MLP input rows; then per warp the register-chained MLP and coalesced stores.
// A tile whose blocks of one texture alone exceed the arena is filtered by the per-lane decode.
#ifndef BCF_GEO_MIN_BLOCKS
#define BCF_GEO_MIN_BLOCKS 4
#endif
constexpr int kGeoMinBlocks = BCF_GEO_MIN_BLOCKS; // resident CTAs per SM the register budget is sized for

struct GeoMeta {
    int box[BCF_MAX_LEVELS][4]; // per level: min x, max x, min y, max y (relative block coordinates)
    unsigned levmask;           // levels holding footprints of the tile
    int hist[16];               // blocks per mode bin of the current round
};

struct GeoLayout {
    int w_bytes, b_bytes, meta, sraw, sidx, arena, per_warp, tmp8, total;
};

template <int PREC, int TQ>
__host__ __device__ inline GeoLayout geo_layout(const MlpDev &P, int cap)
{
    GeoLayout L;
    const int C = P.dims[P.n_layers];
    int off = 0;
    L.w_bytes = mlp_smem_weight_bytes<PREC>(P);
    off += L.w_bytes;
    L.b_bytes = off;
    off += (mlp_smem_bias_floats(P) * 4 + 15) & ~15;
    L.meta = off;
    off += (int)((2 * sizeof(GeoMeta) + 15) & ~15);
    L.sraw = off;
    off += cap * 16;
    L.sidx = off;
    off += (cap * 2 + 15) & ~15;
    L.arena = off;
    off += cap * 16 * 8;
    int maxn = 0;
    for (int l = 0; l < P.n_layers; ++l)
        maxn = maxn > P.npad[l] ? maxn : P.npad[l];
    const int tmp = PREC == BCF_FP8_E4M3 ? ((16 * (maxn + 16) + 15) & ~15) : 0;
    const int ostb = (32 * C * 4 + 15) & ~15;
    const int in_stride = tile_stride_bytes<PREC>(P.kpad[0]);
    const int in0 = (32 * in_stride + 15) & ~15;
    const bool alias = 16 * C * 4 <= 16 * in_stride; // output staging inside the input tile (as tiled_layout)
    const int a0 = alias ? (in0 > ostb ? in0 : ostb) : in0 + ostb;
    L.tmp8 = a0;
    L.per_warp = a0 + tmp;
    L.total = off + (TQ / 32) * L.per_warp;
    return L;
}

// Layout with the MLP on tcgen05 (bcf_tcmlp.cuh): the canonical weight tiles, the A0 / A2 tile (x), the
// mbarrier and the tensor-memory address; the A1 tile and the output staging live in the arena (free once the
// last round's filter is done, which the MLP's first CTA barrier guarantees).
struct GeoTcLayout {
    int w_bytes, b_bytes, meta, sraw, sidx, arena, x, bar, tslot, total;
};

template <int PREC, int K0, int N1, int N2, int NO, int TQ>
__host__ __device__ inline GeoTcLayout geo_tc_layout(const MlpDev &P, int cap)
{
    using T = TcMlp<PREC, TQ / 32, K0, N1, N2, NO>;
    GeoTcLayout L;
    int off = 0;
    L.w_bytes = T::W_BYTES;
    off += (T::W_BYTES + 127) & ~127;
    L.b_bytes = off;
    off += (mlp_smem_bias_floats(P) * 4 + 15) & ~15;
    L.meta = off;
    off += (int)((2 * sizeof(GeoMeta) + 15) & ~15);
    L.sraw = off;
    off += cap * 16;
    L.sidx = off;
    off += (cap * 2 + 127) & ~127;
    L.arena = off;
    const int ostb = TQ * P.dims[P.n_layers] * 4;
    int ab = cap * 16 * 8;
    ab = ab > T::Y_BYTES ? ab : T::Y_BYTES;
    ab = ab > ostb ? ab : ostb;
    off += (ab + 127) & ~127;
    L.x = off;
    off += (T::X_BYTES + 127) & ~127;
    L.bar = off;
    off += 16;
    L.tslot = off;
    off += 16;
    L.total = off;
    return L;
}

__device__ __forceinline__ void reset_geo_meta(GeoMeta &G)
{
    for (int i = threadIdx.x; i < BCF_MAX_LEVELS; i += blockDim.x) {
        G.box[i][0] = G.box[i][2] = INT_MAX;
        G.box[i][1] = G.box[i][3] = INT_MIN;
    }
    if (threadIdx.x < 16)
        G.hist[threadIdx.x] = 0;
    if (threadIdx.x == 0)
        G.levmask = 0u;
}

// Size of the box of level lev (0 if the level holds no footprint).
__device__ __forceinline__ int box_size(const GeoMeta &G, int lev)
{
    const int *b = G.box[lev];
    return b[0] == INT_MAX ? 0 : (b[1] - b[0] + 1) * (b[3] - b[2] + 1);
}

// First block item of level lev's box within one texture's block set (boxes in level order).
__device__ __forceinline__ int box_offset(const GeoMeta &G, unsigned mask, int lev)
{
    int off = 0;
    mask &= (1u << lev) - 1u;
    while (mask) {
        const int l = __ffs(mask) - 1;
        off += box_size(G, l);
        mask &= mask - 1u;
    }
    return off;
}

// The per-lane decode of one texture, out of line: the rare tiles whose blocks exceed the arena take it, and
// keeping its copy of the BC6H decoder out of the tile kernel's body keeps that body's code small.
__device__ __noinline__ float3 sample_texture_ool(const TexDev &T, int wrap, bool sgn, float u, float v, float s)
{
    return sample_texture(T, wrap, sgn, u, v, s);
}

// Arena item tags (shared-memory sort keys of the decode phase): item index in the low kGeoTagBits bits, the
// item's arena swizzle (4 bits) above them.
constexpr int kGeoTagBits = 10;

// Decode arena blocks [first, items) (sorted by mode) with 1 << lk threads per block: each thread decodes the
// header and 16 >> lk texels; sgn is a template parameter so that the unsigned and signed paths are each
// specialised (the caller branches once, uniformly, on the material's format).
template <bool SGN, int TQ>
__device__ __forceinline__ void decode_arena_blocks(const uint4 *sraw, const uint16_t *sidx, uint2 *arena, int items,
                                                    int lk)
{
    for (int i = threadIdx.x; i < (items << lk); i += TQ) {
        const int e = i >> lk, part = i & ((1 << lk) - 1);
        const uint4 rr = sraw[e];
        const int tag = sidx[e];
        uint2 *dst = arena + (tag & ((1 << kGeoTagBits) - 1)) * 16;
        const int swz = tag >> kGeoTagBits;
        Bc6hBlock bk;
        bk.lo = (uint64_t)rr.x | ((uint64_t)rr.y << 32);
        bk.hi = (uint64_t)rr.z | ((uint64_t)rr.w << 32);
        Bc6hHeader H;
        bc6h_header(bk, SGN, H);
        Bc6hTexels X;
        bc6h_prepare_texels(bk, H, X);
        const auto put = [&](int t, uint32_t rg, uint32_t bb) { dst[t ^ swz] = make_uint2(rg, bb); };
        if (lk == 0)
            bc6h_texels<16>(X, SGN, 0, put);
        else
            bc6h_texels<8>(X, SGN, part * 8, put);
    }
}


// With SET, the kernel decodes a material set: M0 is material 0 (the set's MLP shape and shared-memory layout),
// the materials' descriptions are the device table mats, material m's queries are [offsets[m], offsets[m+1]) of
// the concatenated arrays (clipped to [0, n]; a decreasing pair sets BCF_CHECK_OFFSETS and decodes as empty).
// Tiles are numbered material by material (a tile never straddles two materials); persistent CTAs take `chunk`
// consecutive tiles at a time from the work counter (zeroed before the launch) and reload the material's
// description and MLP weights into shared memory when a tile belongs to a new material.  Without SET, M0 is the
// material and tiles go round-robin to the CTAs, each tile's queries loaded one tile ahead.
template <int PREC, int CAP, int K0, int N1, int N2, int NO, bool TC, int TQ, bool SET>
__global__ void __launch_bounds__(TQ, kGeoMinBlocks * 256 / TQ) k_decode_geo(MaterialDev M0, const float *__restrict__ qu,
                                                          const float *__restrict__ qv, const float *__restrict__ qs,
                                                          int64_t n, void *__restrict__ out, int out_fp16,
                                                          unsigned *__restrict__ check,
                                                          const MaterialDev *__restrict__ mats, int nmat,
                                                          const int64_t *__restrict__ offsets,
                                                          int *__restrict__ counter, int chunk)
{
    static_assert(CAP <= TQ && CAP <= (1 << kGeoTagBits), "one block item per thread while loading; item tags");
    constexpr int NW = TQ / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // the MLP shape (and so the layout) is material 0's; every material of a set shares it
    const int Cn = M0.mlp.dims[M0.mlp.n_layers];
    const int row_stride = tile_stride_bytes<PREC>(M0.mlp.kpad[0]);
    int smem_used = 0;
    unsigned char *sw;
    float *sb;
    GeoMeta *meta;
    uint4 *sraw;
    uint16_t *sidx;
    uint2 *arena;
    unsigned char *act0 = nullptr, *tmp8 = nullptr, *xtile = nullptr;
    float *ost;
    uint64_t *bar = nullptr;
    uint32_t *tslot = nullptr;
    if constexpr (TC) {
        const GeoTcLayout LY = geo_tc_layout<PREC, K0, N1, N2, NO, TQ>(M0.mlp, CAP);
        smem_used = LY.total;
        sw = smem;
        sb = (float *)(smem + LY.b_bytes);
        meta = (GeoMeta *)(smem + LY.meta);
        sraw = (uint4 *)(smem + LY.sraw);
        sidx = (uint16_t *)(smem + LY.sidx);
        arena = (uint2 *)(smem + LY.arena);
        xtile = smem + LY.x;
        ost = (float *)(smem + LY.arena); // the output staging: rows [32 warp, 32 warp + 32) of [256][C]
        bar = (uint64_t *)(smem + LY.bar);
        tslot = (uint32_t *)(smem + LY.tslot);
    } else {
        const GeoLayout LY = geo_layout<PREC, TQ>(M0.mlp, CAP);
        smem_used = LY.total;
        sw = smem;
        sb = (float *)(smem + LY.b_bytes);
        meta = (GeoMeta *)(smem + LY.meta);
        sraw = (uint4 *)(smem + LY.sraw);
        sidx = (uint16_t *)(smem + LY.sidx);
        arena = (uint2 *)(smem + LY.arena);
        act0 = smem + LY.total - (NW - warp) * LY.per_warp;
        tmp8 = act0 + LY.tmp8;
        ost = (float *)act0; // output staging aliases the input tile or follows it (geo_layout)
        if (!(16 * Cn * 4 <= 16 * row_stride))
            ost = (float *)(act0 + ((32 * row_stride + 15) & ~15));
    }
    // material sets: the current material's description, the tile table and the work grab, after the layout
    MaterialDev *Ms = nullptr;
    int64_t *tile_first = nullptr;
    int *grab = nullptr;
    if constexpr (SET) {
        unsigned char *x = smem + ((smem_used + 15) & ~15);
        Ms = (MaterialDev *)x;
        x += (sizeof(MaterialDev) + 15) & ~(size_t)15;
        tile_first = (int64_t *)x;
        x += 8 * (BCF_MAX_SET + 1);
        grab = (int *)x;
    }
    const MaterialDev &M = SET ? *Ms : M0; // the current material
    const MlpDev &P = M.mlp;
    const unsigned lanes_lt = (1u << lane) - 1u;

    uint32_t tmem = 0, phase = 0;
    constexpr int kTcCols = TcMlp<PREC, NW, (K0 > 0 ? K0 : 16), (N1 > 0 ? N1 : 16), (N2 > 0 ? N2 : 16),
                                  (NO > 0 ? NO : 16)>::NCOLS;
    if constexpr (TC) {
        if constexpr (!SET)
            tc_load_weights<PREC, NW, K0, N1, N2, NO>(P, sw, sb);
        if (threadIdx.x == 0) {
            mbar_init(bar, 1);
            mbar_init_fence();
        }
        if (warp == 0)
            tc_alloc(tslot, kTcCols);
    } else if constexpr (!SET) {
        load_mlp_smem<PREC>(P, sw, sb);
    }
    if constexpr (SET) {
        if (threadIdx.x == 0) {
            int64_t acc = 0;
            for (int m = 0; m < nmat; ++m) {
                tile_first[m] = acc;
                const int64_t a = min(max(offsets[m], (int64_t)0), n), b = min(max(offsets[m + 1], (int64_t)0), n);
                acc += b > a ? (b - a + TQ - 1) / TQ : 0;
                if (blockIdx.x == 0 && offsets[m + 1] < offsets[m] && check)
                    atomicOr(check, BCF_CHECK_OFFSETS);
            }
            tile_first[nmat] = acc;
        }
    }
    reset_geo_meta(meta[0]);
    reset_geo_meta(meta[1]);
    __syncthreads();
    if constexpr (TC) {
        tc_fence_after();
        tmem = *tslot;
    }

    const int64_t tiles = SET ? 0 : (n + TQ - 1) / TQ;
    float nu = 0.0f, nv = 0.0f, ns = 0.0f, nu_ref = 0.0f, nv_ref = 0.0f;
    if constexpr (!SET) {
        const int64_t q = (int64_t)blockIdx.x * TQ + threadIdx.x;
        if (blockIdx.x < tiles && q < n) {
            nu = qu[q];
            nv = qv[q];
            ns = qs ? qs[q] : 0.0f;
        }
        if (blockIdx.x < tiles) {
            nu_ref = qu[(int64_t)blockIdx.x * TQ];
            nv_ref = qv[(int64_t)blockIdx.x * TQ];
        }
    }
    int parity = 0;
    int64_t tile = blockIdx.x; // without SET: this CTA's next tile
    int64_t gbase = 0;         // SET: the current grab's first tile, and how many of its tiles are taken
    int gtaken = chunk;
    int cur = -1;              // SET: the material whose description and weights are in shared memory
    for (;; parity ^= 1) {
        int64_t q_first, q_end; // this tile's queries: [q_first, min(q_first + TQ, q_end))
        float u, v, s, u_ref, v_ref;
        if constexpr (!SET) {
            if (tile >= tiles)
                break;
            q_first = tile * TQ;
            q_end = n;
            const bool act = q_first + threadIdx.x < n;
            u = act ? sanitize(nu, M.wrap) : 0.0f;
            v = act ? sanitize(nv, M.wrap) : 0.0f;
            s = act ? ns : 0.0f;
            // the tile's first query: the reference of the relative block coordinates
            u_ref = sanitize(nu_ref, M.wrap);
            v_ref = sanitize(nv_ref, M.wrap);
            const int64_t qn = (tile + gridDim.x) * TQ + threadIdx.x;
            if (tile + gridDim.x < tiles && qn < n) {
                nu = qu[qn];
                nv = qv[qn];
                ns = qs ? qs[qn] : 0.0f;
            }
            if (tile + gridDim.x < tiles) {
                nu_ref = qu[(tile + gridDim.x) * TQ];
                nv_ref = qv[(tile + gridDim.x) * TQ];
            }
            tile += gridDim.x;
        } else {
            if (gtaken == chunk) {
                if (threadIdx.x == 0)
                    *grab = atomicAdd(counter, chunk);
                __syncthreads();
                gbase = *grab;
                gtaken = 0;
                __syncthreads(); // everyone has read the grab before thread 0 may overwrite it
            }
            const int64_t t = gbase + gtaken;
            if (t >= tile_first[nmat])
                break; // uniform
            if (++gtaken == chunk || t + 1 >= tile_first[nmat])
                gtaken = chunk;
            int lo = 0, hi = nmat - 1; // the last material m with tile_first[m] <= t
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tile_first[mid] <= t)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const int m = lo;
            if (m != cur) {
                __syncthreads(); // the previous tile's filter and MLP are done with the description and weights
                const int words = (int)(sizeof(MaterialDev) / 4);
                for (int i = threadIdx.x; i < words; i += TQ)
                    reinterpret_cast<int *>(Ms)[i] = reinterpret_cast<const int *>(mats + m)[i];
                __syncthreads();
                if constexpr (TC)
                    tc_load_weights<PREC, NW, K0, N1, N2, NO>(P, sw, sb);
                else
                    load_mlp_smem<PREC>(P, sw, sb);
                cur = m; // (the weights are read after the tile's first barrier)
            }
            const int64_t a = min(max(offsets[m], (int64_t)0), n);
            q_end = min(max(offsets[m + 1], (int64_t)0), n);
            q_first = a + (t - tile_first[m]) * TQ;
            const int64_t q = q_first + threadIdx.x;
            const bool act = q < q_end;
            u = act ? sanitize(qu[q], M.wrap) : 0.0f;
            v = act ? sanitize(qv[q], M.wrap) : 0.0f;
            s = act ? (qs ? qs[q] : 0.0f) : 0.0f;
            u_ref = sanitize(qu[q_first], M.wrap);
            v_ref = sanitize(qv[q_first], M.wrap);
        }
        const float inv0 = PREC == BCF_FP8_E4M3 ? P.inv_act_scale[0] : 1.0f;
        RowWriter<PREC> rw{act0 + lane * row_stride, inv0, 0.0f};
        TcRowWriter<PREC, NW, (K0 > 0 ? K0 : 16), (N1 > 0 ? N1 : 16), (N2 > 0 ? N2 : 16), (NO > 0 ? NO : 16)> tw{
            xtile, (int)threadIdx.x, inv0, 0.0f};
        const auto put = [&](int col, float x) {
            if constexpr (TC)
                tw.put(col, x);
            else
                rw.put(col, x);
        };
        const int nt = M.n_tex;
        const int wrap = M.wrap;
        const bool sgn = M.is_signed != 0;
        const TexDev &T0 = M.tex[0];
        GeoMeta &G = meta[parity];
        const int64_t q = q_first + threadIdx.x;
        const bool active = q < q_end;
        // ---- 1. footprint geometry per side, block boxes per level
        const Lod L = lod_of(T0, s);
        int i0s[2], j0s[2];
        float fxs[2], fys[2];
#pragma unroll
        for (int side = 0; side < 2; ++side) {
            const int level = min(L.l0 + side, T0.levels - 1);
            const int W = T0.res >> level;
            const float x = u * (float)W - 0.5f, y = v * (float)W - 0.5f;
            const float fx0 = floorf(x), fy0 = floorf(y);
            fxs[side] = x - fx0;
            fys[side] = y - fy0;
            i0s[side] = (int)fx0;
            j0s[side] = (int)fy0;
        }
        const bool warp2 = __any_sync(0xffffffffu, active && L.nlev == 2);
        {
            int bxl[2], bxh[2], byl[2], byh[2];
#pragma unroll
            for (int side = 0; side < 2; ++side) {
                if (side == 1 && !warp2) { // warp-uniform
                    bxl[1] = bxh[1] = byl[1] = byh[1] = 0;
                    break;
                }
                const int W = T0.res >> min(L.l0 + side, T0.levels - 1);
                const int rbx = wrap ? ref_block(u_ref, W) : 0, rby = wrap ? ref_block(v_ref, W) : 0;
                bxl[side] = rel_block(i0s[side], i0s[side], rbx, W, wrap);
                bxh[side] = rel_block(i0s[side] + 1, i0s[side], rbx, W, wrap);
                byl[side] = rel_block(j0s[side], j0s[side], rby, W, wrap);
                byh[side] = rel_block(j0s[side] + 1, j0s[side], rby, W, wrap);
            }
            const int lo = __reduce_min_sync(0xffffffffu, active ? L.l0 : INT_MAX);
            const int hi = __reduce_max_sync(0xffffffffu, active ? L.l0 + L.nlev - 1 : INT_MIN);
            for (int lev = lo; lev <= hi; ++lev) { // warp-uniform
                const int side = lev - L.l0;
                const bool use = active && side >= 0 && side < L.nlev;
                const int mnx = __reduce_min_sync(0xffffffffu, use ? (side ? bxl[1] : bxl[0]) : INT_MAX);
                const int mxx = __reduce_max_sync(0xffffffffu, use ? (side ? bxh[1] : bxh[0]) : INT_MIN);
                const int mny = __reduce_min_sync(0xffffffffu, use ? (side ? byl[1] : byl[0]) : INT_MAX);
                const int mxy = __reduce_max_sync(0xffffffffu, use ? (side ? byh[1] : byh[0]) : INT_MIN);
                if (lane == 0 && mnx != INT_MAX) {
                    int *b = G.box[lev];
                    atomicMin(&b[0], mnx);
                    atomicMax(&b[1], mxx);
                    atomicMin(&b[2], mny);
                    atomicMax(&b[3], mxy);
                    atomicOr(&G.levmask, 1u << lev);
                }
            }
        }
        __syncthreads(); // barrier 1
        // the other buffer's last readers (the previous tile) are behind this barrier: reset it for the next tile
        reset_geo_meta(meta[parity ^ 1]);
        const unsigned mask = G.levmask;
        int nb = 0; // blocks of one texture's block set
        {
            unsigned mm = mask;
            while (mm) {
                nb += box_size(G, __ffs(mm) - 1);
                mm &= mm - 1u;
            }
        }
        const int per_round = nb > 0 ? min(nt, CAP / nb) : nt;
        if (per_round == 0) {
            // one texture's blocks exceed the arena: the per-lane decode for this tile
            for (int t = 0; t < nt; ++t) {
                float3 f = make_float3(0.f, 0.f, 0.f);
                if (active)
                    f = sample_texture_ool(M.tex[t], wrap, sgn, u, v, s);
                put(3 * t, f.x);
                put(3 * t + 1, f.y);
                put(3 * t + 2, f.z);
            }
            __syncthreads(); // the next tile's box atomics stay behind this tile's reset of their buffer
        } else {
            const float inv_nb = 1.0f / (float)max(nb, 1);
            for (int t0 = 0; t0 < nt; t0 += per_round) {
                const int rt = min(per_round, nt - t0);
                const int items = nb * rt;
                // ---- 2. load each block of the round once; rank it among the round's blocks of its mode
                const int it = threadIdx.x;
                const bool valid = it < items;
                uint4 blk = make_uint4(0, 0, 0, 0);
                int bin = kBins + lane; // unique per lane when invalid: no aggregation
                int jlow = 0; // item within its texture's block set, low 4 bits: the arena swizzle
                if (valid) {
                    const int tt = (int)(((float)it + 0.5f) * inv_nb);
                    int j = it - tt * nb;
                    jlow = j & 15;
                    unsigned mm = mask;
                    int lev = __ffs(mm) - 1;
                    for (;;) { // the level whose box holds item j
                        const int sz = box_size(G, lev);
                        if (j < sz)
                            break;
                        j -= sz;
                        mm &= mm - 1u;
                        lev = __ffs(mm) - 1;
                    }
                    const int *b = G.box[lev];
                    const int bw = b[1] - b[0] + 1;
                    const int ry = (int)(((float)j + 0.5f) / (float)bw);
                    const TexDev &T = M.tex[t0 + tt];
                    const int W = T.res >> lev, wb = W >> 2;
                    int bxa = b[0] + (j - ry * bw), bya = b[2] + ry;
                    if (wrap) {
                        bxa = (ref_block(u_ref, W) + bxa) & (wb - 1);
                        bya = (ref_block(v_ref, W) + bya) & (wb - 1);
                    }
                    blk = __ldg(T.blocks + T.level_off[lev] + (uint32_t)bya * (uint32_t)wb + (uint32_t)bxa);
                    const int mi = mode_index(blk.x);
                    bin = mi < 0 ? kBins - 1 : mi;
                }
                const unsigned peers = __match_any_sync(0xffffffffu, bin);
                const int leader = __ffs(peers) - 1;
                int base = 0;
                if (valid && lane == leader)
                    base = atomicAdd(&G.hist[bin], __popc(peers));
                const int rank = __shfl_sync(0xffffffffu, base, leader) + __popc(peers & lanes_lt);
                __syncthreads(); // barrier 2
                // ---- 3. scatter into mode order: position = blocks of smaller modes + rank
                {
                    const int h = lane < 16 ? G.hist[lane] : 0;
                    int incl = h;
#pragma unroll
                    for (int d = 1; d < 16; d <<= 1) {
                        const int o = __shfl_up_sync(0xffffffffu, incl, d);
                        if (lane >= d)
                            incl += o;
                    }
                    const int excl = incl - h;
                    const int start = __shfl_sync(0xffffffffu, excl, valid ? bin : 0);
                    if (valid) {
                        sraw[start + rank] = blk;
                        sidx[start + rank] = (uint16_t)(it | (jlow << kGeoTagBits));
                    }
                }
                __syncthreads(); // barrier 3
                if (threadIdx.x < 16)
                    G.hist[threadIdx.x] = 0; // for the next round (read again only after its barrier 2)
                // ---- 4. decode the sorted blocks into the arena: one thread per block, two when that fills the CTA
                const int lk = items * 2 <= TQ ? 1 : 0;
                if (sgn)
                    decode_arena_blocks<true, TQ>(sraw, sidx, arena, items, lk);
                else
                    decode_arena_blocks<false, TQ>(sraw, sidx, arena, items, lk);
                __syncthreads(); // barrier 4
                // ---- 5. filter the round's textures from the arena: per side the corner geometry, shared by
                // every texture (item offsets within one texture's block set), then 4 arena texels per texture
                const bool any2 = warp2;
                int cb[2][4]; // arena texel of each corner within texture 0's block set (swizzled)
                float cw[2][4];
#pragma unroll
                for (int side = 0; side < 2; ++side) {
                    if (side == 1 && !any2)
                        break; // warp-uniform: no lane of the warp samples a second level
                    const int level = min(L.l0 + side, T0.levels - 1);
                    const float scale = L.nlev == 1 ? 1.0f : (side ? L.lam : 1.0f - L.lam);
                    const int W = T0.res >> level;
                    const int *b = G.box[level];
                    const bool in_box = active && side < L.nlev; // the box of this level holds the footprint
                    const int bw = in_box ? b[1] - b[0] + 1 : 1, bh = in_box ? b[3] - b[2] + 1 : 1;
                    const int bx0 = in_box ? b[0] : 0, by0 = in_box ? b[2] : 0;
                    const int o = in_box ? box_offset(G, mask, level) : 0;
                    const int rbx = wrap ? ref_block(u_ref, W) : 0, rby = wrap ? ref_block(v_ref, W) : 0;
                    const int i0 = i0s[side], j0 = j0s[side];
                    // the box was built from the same coordinates, so these lie inside it; the clamps only keep
                    // shared-memory reads in bounds
                    const int xl = min(max(rel_block(i0, i0, rbx, W, wrap) - bx0, 0), bw - 1);
                    const int xh = min(max(rel_block(i0 + 1, i0, rbx, W, wrap) - bx0, 0), bw - 1);
                    const int yl = min(max(rel_block(j0, j0, rby, W, wrap) - by0, 0), bh - 1);
                    const int yh = min(max(rel_block(j0 + 1, j0, rby, W, wrap) - by0, 0), bh - 1);
                    const int cl = texel_col(i0, W, wrap), ch = texel_col(i0 + 1, W, wrap);
                    const int rl = texel_col(j0, W, wrap) * 4, rh = texel_col(j0 + 1, W, wrap) * 4;
                    const int j00 = o + yl * bw + xl, j01 = o + yl * bw + xh, j10 = o + yh * bw + xl,
                              j11 = o + yh * bw + xh;
                    cb[side][0] = j00 * 16 + ((rl + cl) ^ (j00 & 15));
                    cb[side][1] = j01 * 16 + ((rl + ch) ^ (j01 & 15));
                    cb[side][2] = j10 * 16 + ((rh + cl) ^ (j10 & 15));
                    cb[side][3] = j11 * 16 + ((rh + ch) ^ (j11 & 15));
                    const float fx = fxs[side], fy = fys[side];
                    cw[side][0] = (1.0f - fx) * (1.0f - fy) * scale;
                    cw[side][1] = fx * (1.0f - fy) * scale;
                    cw[side][2] = (1.0f - fx) * fy * scale;
                    cw[side][3] = fx * fy * scale;
                }
                for (int tt = 0; tt < rt; ++tt) {
                    float f0 = 0.0f, f1 = 0.0f, f2 = 0.0f;
                    if (active) {
                        const uint2 *at = arena + tt * nb * 16;
#pragma unroll
                        for (int side = 0; side < 2; ++side) {
                            if (side < L.nlev) {
#pragma unroll
                                for (int c = 0; c < 4; ++c) {
                                    const uint2 tx = at[cb[side][c]];
                                    const float2 rg = __half22float2(*reinterpret_cast<const __half2 *>(&tx.x));
                                    f0 = fmaf(cw[side][c], rg.x, f0);
                                    f1 = fmaf(cw[side][c], rg.y, f1);
                                    f2 = fmaf(cw[side][c], __half2float(__ushort_as_half((unsigned short)tx.y)), f2);
                                }
                            }
                        }
                    }
                    const int t = t0 + tt;
                    put(3 * t, f0);
                    put(3 * t + 1, f1);
                    put(3 * t + 2, f2);
                }
            }
        }
        {
            int col = 3 * nt;
            if (M.lod_input) {
                put(col, active ? (isnan(s) ? 0.0f : fmaxf(s, 0.0f)) : 0.0f);
                ++col;
            }
            if constexpr (TC) {
                tw.finish(col); // pads the row to K0
            } else {
                for (; col < P.kpad[0]; ++col)
                    put(col, 0.0f);
                rw.finish(col);
            }
        }
        // ---- 6. MLP on the tensor cores, coalesced store
        if constexpr (TC) {
            // the CTA tile's TQ rows through tcgen05 (its first barrier also ends every warp's filter)
            bool ok = tc_mlp3<PREC, NW, K0, N1, N2, NO>(P, sw, sb, xtile, (unsigned char *)arena, ost, Cn, bar, phase,
                                                       tmem, 1 << 20);
            ok = __syncthreads_and(ok) != 0;
            if (!ok) {
                if (threadIdx.x == 0 && check)
                    atomicOr(check, BCF_CHECK_TIMEOUT);
                break; // uniform: stop taking tiles
            }
            const int64_t q0 = q_first + warp * 32;
            if (q0 < q_end) {
                if constexpr (SET) // a set's tiles start at any query: outputs aligned or not
                    store_rows_any(ost + warp * 32 * Cn, out, q0, (int)min((int64_t)32, q_end - q0), Cn, out_fp16,
                                   lane);
                else
                    store_warp_rows(ost + warp * 32 * Cn, out, q0, (int)min((int64_t)32, q_end - q0), Cn, out_fp16,
                                    lane);
            }
        } else {
            __syncwarp();
            if constexpr (N2 == 0)
                warp_mlp2<PREC, K0, N1, NO>(sw, sb, act0, row_stride, ost, Cn);
            else
                warp_mlp3<PREC, K0, N1, N2, NO>(P, sw, sb, act0, row_stride, tmp8,
                                                tile_stride_bytes<BCF_FP8_E4M3>(N1 > N2 ? N1 : N2), ost, Cn);
            __syncwarp();
            const int64_t q0 = q_first + warp * 32;
            if (q0 < q_end) {
                if constexpr (SET) // a set's tiles start at any query: outputs aligned or not
                    store_rows_any(ost, out, q0, (int)min((int64_t)32, q_end - q0), Cn, out_fp16, lane);
                else
                    store_warp_rows(ost, out, q0, (int)min((int64_t)32, q_end - q0), Cn, out_fp16, lane);
            }
            __syncwarp();
        }
    }
    if constexpr (TC) {
        // every MMA of this CTA has completed (each was waited for, or the bounded wait below gives up): free
        // the tensor memory
        tc_fence_before();
        __syncthreads();
        if (warp == 0) {
            tc_fence_after();
            tc_dealloc(tmem, kTcCols);
        }
    }
}

// ---------------------------------------------------------------- launcher

constexpr int kArenaCap = 320;

static int tiled_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0)
            sms = 148;
    }
    return sms;
}

// Tile size of the single-geometry kernel: 512 queries where the MLP's operand tiles are small (hidden width
// <= 32, or E4M3 operands), which halves the per-query share of the tile's fixed work (the BC6H header paths,
// run once per mode present in a warp, and the barriers) at two resident CTAs of 16 warps per SM; 256 queries
// for the 64-wide 16-bit MLP, whose 512-row operand tiles would leave room for one CTA per SM (measured on the
// 8 x 4096^2 frame: 7.13 ms at 256, 7.43 ms at 512; E4M3 6.88 ms at 256, 5.49 ms at 512).
#ifndef BCF_GEO_TQ_NARROW
#define BCF_GEO_TQ_NARROW 512
#endif
#ifndef BCF_GEO_TQ_WIDE
#define BCF_GEO_TQ_WIDE 256
#endif
template <int PREC, int N1>
constexpr int geo_tq() { return (N1 <= 32 || PREC == BCF_FP8_E4M3) ? BCF_GEO_TQ_NARROW : BCF_GEO_TQ_WIDE; }
// block arena: one block per thread (one round for almost every tile); 224 blocks for 256-query tiles, which
// keeps 4 CTAs per SM
constexpr int geo_cap(int tq) { return tq >= 512 ? 512 : 224; }

template <int PREC, int K0, int N1, int N2, int NO, bool TC>
static cudaError_t launch_geo_engine(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                                     void *out, int out_fp16, cudaStream_t st)
{
    constexpr int TQ = geo_tq<PREC, N1>(), CAP = geo_cap(TQ);
    int64_t smem;
    int max_per_sm = 32;
    if constexpr (TC) {
        smem = geo_tc_layout<PREC, K0, N1, N2, NO, TQ>(M.mlp, CAP).total;
        // every resident CTA holds its tensor-memory columns for its whole life: at most 512 columns per SM
        max_per_sm = 512 / TcMlp<PREC, TQ / 32, K0, N1, N2, NO>::NCOLS;
    } else {
        smem = geo_layout<PREC, TQ>(M.mlp, CAP).total;
    }
    if (smem > 227 * 1024)
        return cudaErrorInvalidConfiguration;
    auto kern = k_decode_geo<PREC, CAP, K0, N1, N2, NO, TC, TQ, false>;
    static int configured = 0;
    if (!configured) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        configured = 1;
    }
    static int per_sm = 0;
    if (!per_sm) {
        // resident CTAs per SM from the kernel's registers and shared memory (the occupancy query reports a
        // single CTA for kernels that use tensor memory)
        cudaFuncAttributes fa{};
        int regs = 64;
        if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess && fa.numRegs > 0)
            regs = fa.numRegs;
        int dev = 0, smem_sm = 228 * 1024;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        const int by_regs = 65536 / (TQ * ((regs + 7) & ~7));
        const int by_smem = smem_sm / (int)(smem + 1024);
        per_sm = max(1, min(min(by_regs, by_smem), max_per_sm));
    }
    const int64_t tiles = (n + TQ - 1) / TQ;
    const int64_t grid = min(tiles, (int64_t)tiled_sms() * per_sm);
    kern<<<(unsigned)grid, TQ, (size_t)smem, st>>>(M, u, v, s, n, out, out_fp16, check_word(), nullptr, 0, nullptr,
                                                   nullptr, 1);
    return cudaGetLastError();
}

// Shared memory of the material-set instance: the single-material layout, then the current material's
// description, the tile table and the work grab.
constexpr int64_t geo_set_extra_bytes()
{
    return 16 + (((int64_t)sizeof(MaterialDev) + 15) & ~15) + 8 * (BCF_MAX_SET + 1) + 16;
}

// Material sets whose materials are single-geometry (every texture of a material at one resolution and level
// count) take the single-geometry kernel with SET: persistent CTAs (cfg.ctas_per_sm per SM, capped by residency)
// grabbing cfg.chunk tiles at a time.
template <int PREC, int K0, int N1, int N2, int NO, bool TC>
static cudaError_t launch_geo_set_engine(const MaterialDev &M0, const MaterialDev *mats, int nmat,
                                         const int64_t *offsets, const float *u, const float *v, const float *s,
                                         int64_t n, void *out, int out_fp16, int *counter, unsigned *check,
                                         const SetConfig &cfg, cudaStream_t st)
{
    constexpr int TQ = geo_tq<PREC, N1>(), CAP = geo_cap(TQ);
    int64_t smem;
    int max_per_sm = 32;
    if constexpr (TC) {
        smem = geo_tc_layout<PREC, K0, N1, N2, NO, TQ>(M0.mlp, CAP).total;
        max_per_sm = 512 / TcMlp<PREC, TQ / 32, K0, N1, N2, NO>::NCOLS;
    } else {
        smem = geo_layout<PREC, TQ>(M0.mlp, CAP).total;
    }
    smem += geo_set_extra_bytes();
    if (smem > 227 * 1024)
        return cudaErrorInvalidConfiguration;
    auto kern = k_decode_geo<PREC, CAP, K0, N1, N2, NO, TC, TQ, true>;
    static int configured = 0;
    if (!configured) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        configured = 1;
    }
    static int per_sm = 0;
    if (!per_sm) {
        cudaFuncAttributes fa{};
        int regs = 64;
        if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess && fa.numRegs > 0)
            regs = fa.numRegs;
        int dev = 0, smem_sm = 228 * 1024;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        const int by_regs = 65536 / (TQ * ((regs + 7) & ~7));
        const int by_smem = smem_sm / (int)(smem + 1024);
        per_sm = max(1, min(min(by_regs, by_smem), max_per_sm));
    }
    const int ctas = max(1, min(per_sm, cfg.ctas_per_sm));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess)
        return e;
    kern<<<(unsigned)(tiled_sms() * ctas), TQ, (size_t)smem, st>>>(M0, u, v, s, n, out, out_fp16, check, mats, nmat,
                                                                    offsets, counter, max(cfg.chunk, 1));
    return cudaGetLastError();
}

template <int PREC, int K0, int N1, int N2, int NO>
static cudaError_t launch_geo_set_shape(const MaterialDev &M0, const MaterialDev *mats, int nmat,
                                        const int64_t *offsets, const float *u, const float *v, const float *s,
                                        int64_t n, void *out, int out_fp16, int *counter, unsigned *check,
                                        const SetConfig &cfg, cudaStream_t st)
{
    if constexpr (N2 != 0)
        if (M0.mlp_engine == 1)
            return launch_geo_set_engine<PREC, K0, N1, N2, NO, true>(M0, mats, nmat, offsets, u, v, s, n, out,
                                                                      out_fp16, counter, check, cfg, st);
    return launch_geo_set_engine<PREC, K0, N1, N2, NO, false>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16,
                                                               counter, check, cfg, st);
}

// 1 when the set's MLP shape has a single-geometry instance (the shapes launch_tiled_prec dispatches to it)
template <int PREC>
static cudaError_t launch_geo_set_prec(const MaterialDev &M0, const MaterialDev *mats, int nmat,
                                       const int64_t *offsets, const float *u, const float *v, const float *s,
                                       int64_t n, void *out, int out_fp16, int *counter, unsigned *check,
                                       const SetConfig &cfg, cudaStream_t st, bool &done)
{
    done = true;
    const MlpDev &P = M0.mlp;
    if (P.n_layers == 3) {
        const int k0 = P.kpad[0], n1 = P.npad[0], n2 = P.npad[1], no = P.npad[2];
        constexpr int kq = PREC == BCF_FP8_E4M3 ? 32 : 16;
        if (k0 == kq && n1 == 32 && n2 == 32 && no == 16)
            return launch_geo_set_shape<PREC, kq, 32, 32, 16>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16,
                                                               counter, check, cfg, st);
        if (k0 == 32 && n1 == 64 && n2 == 64 && no == 16)
            return launch_geo_set_shape<PREC, 32, 64, 64, 16>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16,
                                                               counter, check, cfg, st);
    }
    if constexpr (PREC != BCF_FP8_E4M3)
        if (P.n_layers == 2 && P.kpad[0] == 16 && P.npad[0] == 16 && P.npad[1] == 16)
            return launch_geo_set_shape<PREC, 16, 16, 0, 16>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16,
                                                              counter, check, cfg, st);
    done = false;
    return cudaSuccess;
}

template <int PREC, int K0, int N1, int N2, int NO>
static cudaError_t launch_geo_shape(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                                    void *out, int out_fp16, cudaStream_t st)
{
    if constexpr (N2 != 0)
        if (M.mlp_engine == 1)
            return launch_geo_engine<PREC, K0, N1, N2, NO, true>(M, u, v, s, n, out, out_fp16, st);
    return launch_geo_engine<PREC, K0, N1, N2, NO, false>(M, u, v, s, n, out, out_fp16, st);
}

template <int PREC, int K0, int N1, int N2, int NO>
static cudaError_t launch_tiled_shape(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                                      void *out, int out_fp16, cudaStream_t st)
{
    if constexpr (K0 != 0)
        if (M.n_groups == 1)
            return launch_geo_shape<PREC, K0, N1, N2, NO>(M, u, v, s, n, out, out_fp16, st);
    const int64_t smem = tiled_layout<PREC>(M.mlp, kArenaCap, K0 == 0).total;
    if (smem > 227 * 1024)
        return cudaErrorInvalidConfiguration;
    auto kern = k_decode_tiled<PREC, kArenaCap, K0, N1, N2, NO>;
    static int configured = 0;
    if (!configured) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        configured = 1;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTileQ, (size_t)smem);
    const int64_t tiles = (n + kTileQ - 1) / kTileQ;
    const int64_t grid = min(tiles, (int64_t)tiled_sms() * max(per_sm, 1));
    kern<<<(unsigned)grid, kTileQ, (size_t)smem, st>>>(M, u, v, s, n, out, out_fp16);
    return cudaGetLastError();
}

template <int PREC>
static cudaError_t launch_tiled_prec(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                                     void *out, int out_fp16, cudaStream_t st)
{
    const MlpDev &P = M.mlp;
    if (P.n_layers == 3) {
        const int k0 = P.kpad[0], n1 = P.npad[0], n2 = P.npad[1], no = P.npad[2];
        constexpr int kq = PREC == BCF_FP8_E4M3 ? 32 : 16;
        if (k0 == kq && n1 == 32 && n2 == 32 && no == 16)
            return launch_tiled_shape<PREC, kq, 32, 32, 16>(M, u, v, s, n, out, out_fp16, st);
        if (k0 == 32 && n1 == 64 && n2 == 64 && no == 16)
            return launch_tiled_shape<PREC, 32, 64, 64, 16>(M, u, v, s, n, out, out_fp16, st);
    }
    if constexpr (PREC != BCF_FP8_E4M3)
        if (P.n_layers == 2 && P.kpad[0] == 16 && P.npad[0] == 16 && P.npad[1] == 16)
            return launch_tiled_shape<PREC, 16, 16, 0, 16>(M, u, v, s, n, out, out_fp16, st);
    return launch_tiled_shape<PREC, 0, 0, 0, 0>(M, u, v, s, n, out, out_fp16, st);
}

cudaError_t launch_decode_tiled(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                                void *out, int out_fp16, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    switch (M.mlp.precision) {
    case BCF_FP16: return launch_tiled_prec<BCF_FP16>(M, u, v, s, n, out, out_fp16, st);
    case BCF_BF16: return launch_tiled_prec<BCF_BF16>(M, u, v, s, n, out, out_fp16, st);
    case BCF_FP8_E4M3: return launch_tiled_prec<BCF_FP8_E4M3>(M, u, v, s, n, out, out_fp16, st);
    default: return cudaErrorInvalidValue;
    }
}

// ------------------------------------------------------ material sets

template <int PREC, int CAP, int K0, int N1, int N2, int NO>
static cudaError_t launch_set_shape(const MaterialDev &M0, const MaterialDev *mats, int nmat, const int64_t *offsets,
                                    const float *u, const float *v, const float *s, int64_t n, void *out,
                                    int out_fp16, int *counter, unsigned *check, const SetConfig &cfg, cudaStream_t st)
{
    const int64_t smem = tiled_layout<PREC>(M0.mlp, CAP, K0 == 0).total;
    if (smem > 200 * 1024)
        return cudaErrorInvalidConfiguration;
    auto kern = k_decode_set<PREC, CAP, K0, N1, N2, NO>;
    static int configured = 0;
    if (!configured) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        configured = 1;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTileQ, (size_t)smem);
    per_sm = max(1, min(per_sm, cfg.ctas_per_sm));
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess)
        return e;
    kern<<<(unsigned)(tiled_sms() * per_sm), kTileQ, (size_t)smem, st>>>(mats, nmat, offsets, u, v, s, n, out,
                                                                           out_fp16, counter, check, max(cfg.chunk, 1));
    return cudaGetLastError();
}

template <int PREC, int CAP>
static cudaError_t launch_set_cap(const MaterialDev &M0, const MaterialDev *mats, int nmat, const int64_t *offsets,
                                  const float *u, const float *v, const float *s, int64_t n, void *out, int out_fp16,
                                  int *counter, unsigned *check, const SetConfig &cfg, cudaStream_t st)
{
    const MlpDev &P = M0.mlp;
    if (P.n_layers == 3) {
        const int k0 = P.kpad[0], n1 = P.npad[0], n2 = P.npad[1], no = P.npad[2];
        constexpr int kq = PREC == BCF_FP8_E4M3 ? 32 : 16;
        if (k0 == kq && n1 == 32 && n2 == 32 && no == 16)
            return launch_set_shape<PREC, CAP, kq, 32, 32, 16>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16,
                                                                counter, check, cfg, st);
    }
    return launch_set_shape<PREC, CAP, 0, 0, 0, 0>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16, counter, check,
                                                   cfg, st);
}

template <int PREC>
static cudaError_t launch_set_prec(const MaterialDev &M0, const MaterialDev *mats, int nmat, const int64_t *offsets,
                                   const float *u, const float *v, const float *s, int64_t n, void *out, int out_fp16,
                                   int *counter, unsigned *check, const SetConfig &cfg, cudaStream_t st)
{
    if (cfg.cap == 256)
        return launch_set_cap<PREC, 256>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16, counter, check, cfg, st);
    return launch_set_cap<PREC, 320>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16, counter, check, cfg, st);
}

cudaError_t launch_decode_set(const MaterialDev &M0, const MaterialDev *mats, int nmat, const int64_t *offsets,
                              const float *u, const float *v, const float *s, int64_t n, void *out, int out_fp16,
                              int *counter, unsigned *check, const SetConfig &cfg, bool single_geometry,
                              cudaStream_t st)
{
    if (single_geometry) {
        bool done = false;
        cudaError_t e = cudaSuccess;
        switch (M0.mlp.precision) {
        case BCF_FP16:
            e = launch_geo_set_prec<BCF_FP16>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16, counter, check, cfg,
                                              st, done);
            break;
        case BCF_BF16:
            e = launch_geo_set_prec<BCF_BF16>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16, counter, check, cfg,
                                              st, done);
            break;
        case BCF_FP8_E4M3:
            e = launch_geo_set_prec<BCF_FP8_E4M3>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16, counter, check,
                                                  cfg, st, done);
            break;
        default: break;
        }
        if (done)
            return e;
    }
    switch (M0.mlp.precision) {
    case BCF_FP16:
        return launch_set_prec<BCF_FP16>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16, counter, check, cfg, st);
    case BCF_BF16:
        return launch_set_prec<BCF_BF16>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16, counter, check, cfg, st);
    case BCF_FP8_E4M3:
        return launch_set_prec<BCF_FP8_E4M3>(M0, mats, nmat, offsets, u, v, s, n, out, out_fp16, counter, check, cfg,
                                             st);
    default: return cudaErrorInvalidValue;
    }
}

int64_t decode_tiled_smem_bytes(const MlpDev &P)
{
    switch (P.precision) {
    case BCF_FP16: return tiled_layout<BCF_FP16>(P, kArenaCap, true).total;
    case BCF_BF16: return tiled_layout<BCF_BF16>(P, kArenaCap, true).total;
    case BCF_FP8_E4M3: return tiled_layout<BCF_FP8_E4M3>(P, kArenaCap, true).total;
    default: return 0;
    }
}

} // namespace bcf
