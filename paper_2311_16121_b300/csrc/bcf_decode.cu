// bcf_decode.cu -- decode kernels: whole-image BC6H unpack, feature sampling,
// and the fused query decode (unpack + trilinear filter + MLP, Eq. 3).
#include <cuda_fp16.h>

#include "bc6h_unpack.cuh"
#include "bcf_kernels.h"
#include "bcf_mlp.cuh"
#include "bcf_tcmlp.cuh"
#include "bcf_sample.cuh"

namespace bcf {

// ------------------------------------------------------------ image unpack

// One thread per block; the CTA decodes up to 64 consecutive blocks of one
// block row into shared memory, then the four texel rows of that run are
// written out with coalesced 8-byte stores.
constexpr int kUnpackRun = 64;

template <bool SGN>
__global__ void __launch_bounds__(kUnpackRun) k_unpack_image(const uint4 *__restrict__ blocks, int bw, int bh,
                                                             uint16_t *__restrict__ out)
{
    __shared__ __align__(16) uint16_t tile[4][kUnpackRun * 4 * 3];
    const int runs_per_row = (bw + kUnpackRun - 1) / kUnpackRun;
    const int by = blockIdx.x / runs_per_row;
    const int bx0 = (blockIdx.x % runs_per_row) * kUnpackRun;
    const int nb = min(kUnpackRun, bw - bx0);
    const int tx = threadIdx.x;
    if (tx < nb) {
        const Bc6hBlock blk = load_block(blocks + (size_t)by * bw + bx0 + tx);
        Bc6hHeader H;
        bc6h_header(blk, SGN, H);
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            uint32_t r, g, b;
            bc6h_texel(blk, H, t, SGN, r, g, b);
            uint16_t *d = &tile[t >> 2][(tx * 4 + (t & 3)) * 3];
            d[0] = (uint16_t)r;
            d[1] = (uint16_t)g;
            d[2] = (uint16_t)b;
        }
    }
    __syncthreads();
    // each texel row of the run is 24 * nb bytes = 3 * nb 8-byte words, 8-byte aligned in `out`
    const size_t W = (size_t)bw * 4;
    const int words = 3 * nb;
    for (int rr = 0; rr < 4; ++rr) {
        uint64_t *dst = reinterpret_cast<uint64_t *>(out + ((size_t)(by * 4 + rr) * W + (size_t)bx0 * 4) * 3);
        const uint64_t *src = reinterpret_cast<const uint64_t *>(&tile[rr][0]);
        for (int w = tx; w < words; w += blockDim.x)
            dst[w] = src[w];
    }
}

// ---------------------------------------------------------- feature sample

__global__ void __launch_bounds__(128) k_sample_features(MaterialDev M, const float *__restrict__ u,
                                                         const float *__restrict__ v, const float *__restrict__ s,
                                                         int64_t n, float *__restrict__ feat)
{
    const int nf = 3 * M.n_tex;
    __shared__ float srow[128 * (3 * BCF_MAX_TEX + 1)];
    float *row = srow + threadIdx.x * (nf + 1);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        query_features(M, u[q], v[q], s ? s[q] : 0.0f, row);
        float *o = feat + q * nf;
        for (int i = 0; i < nf; ++i)
            o[i] = row[i];
    }
}

// --------------------------------------------------- fused decode, FP32 SIMT

// The plain evaluation: one thread per query, per-query BC6H unpack of the
// texels it filters, FP32 SIMT MLP with weights broadcast from shared memory.
template <int D0, int D1, int D2, int D3, bool HW = false>
__global__ void __launch_bounds__(128) k_decode_fp32(MaterialDev M, TexUnitObjs T, const float *__restrict__ u,
                                                     const float *__restrict__ v, const float *__restrict__ s,
                                                     int64_t n, void *__restrict__ out, int out_fp16)
{
    __shared__ float sW[D1 * D0 + D2 * D1 + D3 * D2];
    __shared__ float sB[D1 + D2 + D3];
    __shared__ float sX[128 * D0];
    const float *Wg = (const float *)M.mlp.weights;
    for (int i = threadIdx.x; i < D1 * D0 + D2 * D1 + D3 * D2; i += blockDim.x)
        sW[i] = Wg[i];
    for (int i = threadIdx.x; i < D1 + D2 + D3; i += blockDim.x)
        sB[i] = M.mlp.biases[i];
    __syncthreads();
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        float x[D0];
        float *row = sX + threadIdx.x * D0;
        if (HW) // the texture unit's texels, the same exact filter (variant 3)
            query_features_hwpoint(M, T, u[q], v[q], s ? s[q] : 0.0f, row);
        else
            query_features(M, u[q], v[q], s ? s[q] : 0.0f, row);
#pragma unroll
        for (int i = 0; i < D0; ++i)
            x[i] = row[i];
        float h1[D1], h2[D2], y[D3];
        dense_fp32<D0, D1, true>(sW, sB, x, h1);
        dense_fp32<D1, D2, true>(sW + D1 * D0, sB + D1, h1, h2);
        dense_fp32<D2, D3, false>(sW + D1 * D0 + D2 * D1, sB + D1 + D2, h2, y);
        if (out_fp16) {
            __half *o = (__half *)out + q * D3;
#pragma unroll
            for (int c = 0; c < D3; ++c)
                o[c] = __float2half_rn(y[c]);
        } else {
            float *o = (float *)out + q * D3;
#pragma unroll
            for (int c = 0; c < D3; ++c)
                o[c] = y[c];
        }
    }
}

// Generic FP32 path for any layer count / width: activations in local memory.
__global__ void __launch_bounds__(128) k_decode_fp32_generic(MaterialDev M, const float *__restrict__ u,
                                                             const float *__restrict__ v,
                                                             const float *__restrict__ s, int64_t n,
                                                             void *__restrict__ out, int out_fp16)
{
    const MlpDev &P = M.mlp;
    const float *Wg = (const float *)P.weights;
    const int C = P.dims[P.n_layers];
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        float a[BCF_MAX_WIDTH], b[BCF_MAX_WIDTH];
        query_features(M, u[q], v[q], s ? s[q] : 0.0f, a);
        for (int l = 0; l < P.n_layers; ++l) {
            const int ni = P.dims[l], no = P.dims[l + 1];
            for (int o = 0; o < no; ++o) {
                float acc = P.biases[P.b_off[l] + o];
                for (int i = 0; i < ni; ++i)
                    acc = fmaf(Wg[P.w_off[l] + o * ni + i], a[i], acc);
                b[o] = (l + 1 < P.n_layers) ? fmaxf(acc, 0.0f) : acc;
            }
            for (int o = 0; o < no; ++o)
                a[o] = b[o];
        }
        for (int c = 0; c < C; ++c) {
            if (out_fp16)
                ((__half *)out)[q * C + c] = __float2half_rn(a[c]);
            else
                ((float *)out)[q * C + c] = a[c];
        }
    }
}

// ------------------------------------------------ fused decode, tensor cores

// per warp: act0, act1, the output staging [32][C] floats and (generic MLP only) FP32 feature rows
// [32][n_in + 1]; the register-chained MLP's features go straight into act0
__host__ __device__ inline int mma_per_warp_bytes(int act_bytes, int act1_bytes, int C, int n_in, bool rows)
{
    return act_bytes + act1_bytes + ((32 * C + 3) & ~3) * 4 + (rows ? 32 * (n_in + 1) * 4 : 0);
}

// Second activation buffer of a warp: the generic MLP ping-pongs two full tiles; the register-chained one
// (three layers, K0 > 0) needs only FP8's 16-row re-quantisation tile, 16-bit operands none.
template <int PREC, int K0, int N1, int N2>
__host__ __device__ inline int mma_act1_bytes(int act_bytes)
{
    if (K0 == 0)
        return act_bytes;
    return PREC == BCF_FP8_E4M3 ? 16 * tile_stride_bytes<BCF_FP8_E4M3>(N1 > N2 ? N1 : N2) : 0;
}

// One warp per tile of 32 queries: per-lane unpack + filter of its query,
// the quantised feature row goes to the warp's activation tile, the MLP runs
// on the tensor cores, the [32][C] result is staged and stored coalesced.
template <int PREC, int HW, int K0, int N1, int N2, int NO>
__global__ void __launch_bounds__(128) k_decode_mma(MaterialDev M, TexUnitObjs T, const float *__restrict__ u,
                                                    const float *__restrict__ v, const float *__restrict__ s,
                                                    int64_t n, void *__restrict__ out, int out_fp16, int act_bytes)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const MlpDev &P = M.mlp;
    const int wbytes = mlp_smem_weight_bytes<PREC>(P);
    unsigned char *sw = smem;
    float *sb = (float *)(smem + wbytes);
    const int nbias = mlp_smem_bias_floats(P);
    unsigned char *wbase = smem + wbytes + ((nbias * 4 + 15) & ~15);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = P.dims[P.n_layers];
    // per warp: act0, act1 (act_bytes each), output staging [32][C] floats, feature rows [32][n_in + 1]
    const int act1_bytes = mma_act1_bytes<PREC, K0, N1, N2>(act_bytes);
    const int per_warp = mma_per_warp_bytes(act_bytes, act1_bytes, C, M.n_in, K0 == 0);
    unsigned char *act0 = wbase + warp * per_warp;
    unsigned char *act1 = act0 + act_bytes;
    float *ost = (float *)(act1 + act1_bytes);
    float *frow = ost + ((32 * C + 3) & ~3) + lane * (M.n_in + 1);

    load_mlp_smem<PREC>(P, sw, sb);
    __syncthreads();

    const int warps_total = gridDim.x * (blockDim.x >> 5);
    const int64_t tiles = (n + 31) / 32;
    const int row_stride = tile_stride_bytes<PREC>(P.kpad[0]);
    for (int64_t tile = blockIdx.x * (int64_t)(blockDim.x >> 5) + warp; tile < tiles; tile += warps_total) {
        const int64_t q = tile * 32 + lane;
        if constexpr (K0 != 0) {
            // features straight into the lane's operand row, zero-padded to K0
            unsigned char *row = act0 + lane * row_stride;
            const float inv0 = PREC == BCF_FP8_E4M3 ? P.inv_act_scale[0] : 1.0f;
            const bool live = q < n;
            const float sq = live && s ? s[q] : 0.0f;
            const float uu = sanitize(live ? u[q] : 0.0f, M.wrap), vv = sanitize(live ? v[q] : 0.0f, M.wrap);
#pragma unroll 1
            for (int t = 0; t < M.n_tex; ++t) {
                float3 f = make_float3(0.0f, 0.0f, 0.0f);
                if (live) {
                    if (HW == 1)
                        f = texture_trilinear_hw(M.tex[t], T.tex[t], uu, vv, sq);
                    else if (HW == 2)
                        f = sample_texture_hwpoint(M.tex[t], T.texp[t], M.wrap, uu, vv, sq);
                    else
                        f = sample_texture(M.tex[t], M.wrap, M.is_signed != 0, uu, vv, sq);
                }
                store_feature<PREC>(row, 3 * t, f.x, inv0);
                store_feature<PREC>(row, 3 * t + 1, f.y, inv0);
                store_feature<PREC>(row, 3 * t + 2, f.z, inv0);
            }
            int col = 3 * M.n_tex;
            if (M.lod_input)
                store_feature<PREC>(row, col++, live ? (isnan(sq) ? 0.0f : fmaxf(sq, 0.0f)) : 0.0f, inv0);
            for (; col < K0; ++col)
                store_feature<PREC>(row, col, 0.0f, inv0);
        } else {
            if (q < n) {
                if (HW == 1)
                    query_features_hw(M, T, u[q], v[q], s ? s[q] : 0.0f, frow);
                else if (HW == 2)
                    query_features_hwpoint(M, T, u[q], v[q], s ? s[q] : 0.0f, frow);
                else
                    query_features(M, u[q], v[q], s ? s[q] : 0.0f, frow);
            } else {
                for (int i = 0; i < M.n_in; ++i)
                    frow[i] = 0.0f;
            }
            store_input_row<PREC>(P, frow, M.n_in, act0 + lane * row_stride);
        }
        __syncwarp();
        if constexpr (K0 == 0)
            warp_mlp<PREC>(P, sw, sb, act0, act1, ost);
        else if constexpr (N2 == 0) // one hidden layer (the paper's decoder shape)
            warp_mlp2<PREC, K0, N1, NO>(sw, sb, act0, row_stride, ost, C);
        else // the common shapes: layers chained through registers (act1 is the FP8 re-quantisation tile)
            warp_mlp3<PREC, K0, N1, N2, NO>(P, sw, sb, act0, row_stride, act1,
                                            tile_stride_bytes<BCF_FP8_E4M3>(N1 > N2 ? N1 : N2), ost, C);
        __syncwarp();
        // coalesced store of the warp's rows [tile*32, tile*32 + rows)
        const int rows = (int)min((int64_t)32, n - tile * 32);
        const int total = rows * C;
        if (out_fp16) {
            __half *o = (__half *)out + tile * 32 * C;
            for (int i = lane; i < total; i += 32)
                o[i] = __float2half_rn(ost[i]);
        } else {
            float *o = (float *)out + tile * 32 * C;
            for (int i = lane; i < total; i += 32)
                o[i] = ost[i];
        }
        __syncwarp();
    }
}

// The same decode with the MLP on tcgen05 (bcf_set_mlp_engine): persistent CTAs of 4 warps over 128-query tiles;
// each thread computes its query's features (texture-unit texels or trilinear, or the per-lane BC6H decode,
// exactly as k_decode_mma) into the CTA's canonical A0 tile, the tile goes through tc_mlp3 (one thread issues
// 128-row MMAs per layer, accumulators in tensor memory), and every warp stores its 32 rows.
template <int PREC, int HW, int K0, int N1, int N2, int NO>
struct MmaTcLayout {
    using T = TcMlp<PREC, 4, K0, N1, N2, NO>;
    int b_off, x_off, y_off, bar_off, tslot_off, total;
    __host__ __device__ explicit MmaTcLayout(const MlpDev &P)
    {
        const int C = P.dims[P.n_layers];
        b_off = (T::W_BYTES + 127) & ~127;
        x_off = b_off + ((mlp_smem_bias_floats(P) * 4 + 127) & ~127);
        y_off = x_off + ((T::X_BYTES + 127) & ~127);
        const int yb = T::Y_BYTES > 128 * C * 4 ? T::Y_BYTES : 128 * C * 4;
        bar_off = y_off + ((yb + 127) & ~127);
        tslot_off = bar_off + 16;
        total = tslot_off + 16;
    }
};

template <int PREC, int HW, int K0, int N1, int N2, int NO>
__global__ void __launch_bounds__(128) k_decode_mma_tc(MaterialDev M, TexUnitObjs T, const float *__restrict__ u,
                                                       const float *__restrict__ v, const float *__restrict__ s,
                                                       int64_t n, void *__restrict__ out, int out_fp16,
                                                       unsigned *__restrict__ check)
{
    using TM = TcMlp<PREC, 4, K0, N1, N2, NO>;
    extern __shared__ __align__(16) unsigned char smem[];
    const MlpDev &P = M.mlp;
    const MmaTcLayout<PREC, HW, K0, N1, N2, NO> LY(P);
    unsigned char *sw = smem;
    float *sb = (float *)(smem + LY.b_off);
    unsigned char *x = smem + LY.x_off, *y = smem + LY.y_off;
    uint64_t *bar = (uint64_t *)(smem + LY.bar_off);
    uint32_t *tslot = (uint32_t *)(smem + LY.tslot_off);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = P.dims[P.n_layers];
    tc_load_weights<PREC, 4, K0, N1, N2, NO>(P, sw, sb);
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
    }
    if (warp == 0)
        tc_alloc(tslot, TM::NCOLS);
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    uint32_t phase = 0;
    const float inv0 = PREC == BCF_FP8_E4M3 ? P.inv_act_scale[0] : 1.0f;
    const int64_t tiles = (n + 127) / 128;
    for (int64_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int64_t q = tile * 128 + threadIdx.x;
        const bool live = q < n;
        TcRowWriter<PREC, 4, K0, N1, N2, NO> tw{x, (int)threadIdx.x, inv0, 0.0f};
        const float sq = live && s ? s[q] : 0.0f;
        const float uu = sanitize(live ? u[q] : 0.0f, M.wrap), vv = sanitize(live ? v[q] : 0.0f, M.wrap);
#pragma unroll 1
        for (int t = 0; t < M.n_tex; ++t) {
            float3 f = make_float3(0.0f, 0.0f, 0.0f);
            if (live) {
                if (HW == 1)
                    f = texture_trilinear_hw(M.tex[t], T.tex[t], uu, vv, sq);
                else if (HW == 2)
                    f = sample_texture_hwpoint(M.tex[t], T.texp[t], M.wrap, uu, vv, sq);
                else
                    f = sample_texture(M.tex[t], M.wrap, M.is_signed != 0, uu, vv, sq);
            }
            tw.put(3 * t, f.x);
            tw.put(3 * t + 1, f.y);
            tw.put(3 * t + 2, f.z);
        }
        int col = 3 * M.n_tex;
        if (M.lod_input)
            tw.put(col++, live ? (isnan(sq) ? 0.0f : fmaxf(sq, 0.0f)) : 0.0f);
        tw.finish(col); // pads the row to K0
        bool ok = tc_mlp3<PREC, 4, K0, N1, N2, NO>(P, sw, sb, x, y, (float *)y, C, bar, phase, tmem, 1 << 20);
        ok = __syncthreads_and(ok) != 0;
        if (!ok) {
            if (threadIdx.x == 0 && check)
                atomicOr(check, BCF_CHECK_TIMEOUT);
            break; // uniform: stop taking tiles
        }
        const int64_t q0 = tile * 128 + warp * 32;
        if (q0 < n)
            store_warp_rows((const float *)y + warp * 32 * C, out, q0, (int)min((int64_t)32, n - q0), C, out_fp16,
                            lane);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tc_dealloc(tmem, TM::NCOLS);
    }
}

// Material sets through the texture unit: every warp of the persistent CTAs works on its own -- it takes
// `chunk` consecutive 32-query tiles at a time from the work counter (tiles are numbered material by material
// and never straddle two materials), keeps its own copy of its current material's MLP weights in shared memory
// (reloaded by the warp alone when its tile belongs to a new material), reads the material's description and
// texture objects from the device tables, and decodes its 32 queries as variant 3 does (texture-unit texels,
// exact FP32 filter, register-chained tensor-core MLP).  No CTA barrier after the start: the warps run as
// independently as in the single-material kernel.
constexpr int kSetTexWarps = 4;

// Shared bytes of one warp of k_decode_set_tex: its weights, biases and MLP operand rows.
template <int PREC, int K0, int N1, int N2>
__host__ __device__ inline int set_tex_warp_bytes(const MlpDev &P, int act_bytes)
{
    const int w = (mlp_smem_weight_bytes<PREC>(P) + 15) & ~15, bb = (mlp_smem_bias_floats(P) * 4 + 15) & ~15;
    return w + bb + mma_per_warp_bytes(act_bytes, mma_act1_bytes<PREC, K0, N1, N2>(act_bytes), P.dims[P.n_layers], 0,
                                       false);
}

template <int PREC, int K0, int N1, int N2, int NO>
__global__ void __launch_bounds__(32 * kSetTexWarps) k_decode_set_tex(
    const MaterialDev *__restrict__ mats, const TexUnitObjs *__restrict__ texs, int nmat,
    const int64_t *__restrict__ offsets, const float *__restrict__ qu, const float *__restrict__ qv,
    const float *__restrict__ qs, int64_t n, void *__restrict__ out, int out_fp16, int *__restrict__ counter,
    unsigned *__restrict__ check, int act_bytes, int chunk)
{
    constexpr int kTile = 32; // one warp's tile
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int64_t tile_first[BCF_MAX_SET + 1];
    const MlpDev &P0 = mats[0].mlp; // every material shares the MLP shape (checked when the set is created)
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int C = P0.dims[P0.n_layers];
    unsigned char *sw = smem + warp * set_tex_warp_bytes<PREC, K0, N1, N2>(P0, act_bytes);
    float *sb = (float *)(sw + ((mlp_smem_weight_bytes<PREC>(P0) + 15) & ~15));
    unsigned char *act0 = (unsigned char *)sb + ((mlp_smem_bias_floats(P0) * 4 + 15) & ~15);
    const int act1_bytes = mma_act1_bytes<PREC, K0, N1, N2>(act_bytes);
    unsigned char *act1 = act0 + act_bytes;
    float *ost = (float *)(act1 + act1_bytes);
    const int row_stride = tile_stride_bytes<PREC>(K0);
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int m = 0; m < nmat; ++m) {
            tile_first[m] = acc;
            const int64_t a = min(max(offsets[m], (int64_t)0), n), b = min(max(offsets[m + 1], (int64_t)0), n);
            acc += b > a ? (b - a + kTile - 1) / kTile : 0;
            if (blockIdx.x == 0 && offsets[m + 1] < offsets[m] && check)
                atomicOr(check, BCF_CHECK_OFFSETS);
        }
        tile_first[nmat] = acc;
    }
    __syncthreads();
    const int64_t total = tile_first[nmat];
    int cur = -1;
    for (;;) {
        int64_t base = 0;
        if (lane == 0)
            base = atomicAdd(counter, chunk);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= total)
            break; // warp-uniform
        for (int64_t tile = base; tile < base + chunk && tile < total; ++tile) {
            int lo = 0, hi = nmat - 1; // last m with tile_first[m] <= tile
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (tile_first[mid] <= tile)
                    lo = mid;
                else
                    hi = mid - 1;
            }
            const int m = lo;
            const MaterialDev &M = mats[m];
            if (m != cur) {
                __syncwarp(); // the warp's previous MLP is done with the weights being replaced
                load_mlp_smem<PREC>(M.mlp, sw, sb, lane, 32);
                __syncwarp();
                cur = m;
            }
            const int64_t a = min(max(offsets[m], (int64_t)0), n), b = min(max(offsets[m + 1], (int64_t)0), n);
            const int64_t q0w = a + (tile - tile_first[m]) * kTile;
            const int64_t q = q0w + lane;
            const bool live = q < b;
            const float inv0 = PREC == BCF_FP8_E4M3 ? M.mlp.inv_act_scale[0] : 1.0f;
            const int wrap = M.wrap, nt = M.n_tex;
            RowWriter<PREC> rw{act0 + lane * row_stride, inv0, 0.0f};
            const float sq = live && qs ? qs[q] : 0.0f;
            const float uu = sanitize(live ? qu[q] : 0.0f, wrap), vv = sanitize(live ? qv[q] : 0.0f, wrap);
#pragma unroll 1
            for (int t = 0; t < nt; ++t) {
                float3 f = make_float3(0.0f, 0.0f, 0.0f);
                if (live)
                    f = sample_texture_hwpoint(M.tex[t], texs[m].texp[t], wrap, uu, vv, sq);
                rw.put(3 * t, f.x);
                rw.put(3 * t + 1, f.y);
                rw.put(3 * t + 2, f.z);
            }
            int col = 3 * nt;
            if (M.lod_input)
                rw.put(col++, live ? (isnan(sq) ? 0.0f : fmaxf(sq, 0.0f)) : 0.0f);
            for (; col < K0; ++col)
                rw.put(col, 0.0f);
            rw.finish(col);
            __syncwarp();
            if constexpr (N2 == 0)
                warp_mlp2<PREC, K0, N1, NO>(sw, sb, act0, row_stride, ost, C);
            else
                warp_mlp3<PREC, K0, N1, N2, NO>(M.mlp, sw, sb, act0, row_stride, act1,
                                                tile_stride_bytes<BCF_FP8_E4M3>(N1 > N2 ? N1 : N2), ost, C);
            __syncwarp();
            store_rows_any(ost, out, q0w, (int)min((int64_t)32, b - q0w), C, out_fp16, lane);
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------- launchers

static int sm_count()
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

cudaError_t launch_unpack_image(const void *blocks, int bw, int bh, int is_signed, uint16_t *out, cudaStream_t st)
{
    const int runs = (bw + kUnpackRun - 1) / kUnpackRun;
    const int64_t grid = (int64_t)runs * bh;
    if (grid == 0)
        return cudaSuccess;
    if (is_signed)
        k_unpack_image<true><<<(unsigned)grid, kUnpackRun, 0, st>>>((const uint4 *)blocks, bw, bh, out);
    else
        k_unpack_image<false><<<(unsigned)grid, kUnpackRun, 0, st>>>((const uint4 *)blocks, bw, bh, out);
    return cudaGetLastError();
}

static unsigned grid_for(int64_t items, int threads, int per_sm)
{
    int64_t need = (items + threads - 1) / threads;
    int64_t cap = (int64_t)sm_count() * per_sm;
    return (unsigned)max((int64_t)1, min(need, cap));
}

cudaError_t launch_sample_features(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                                   float *feat, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    const unsigned grid = grid_for(n, 128, 8);
    k_sample_features<<<grid, 128, 0, st>>>(M, u, v, s, n, feat);
    return cudaGetLastError();
}

#define BCF_FP32_CASE(D0, D1, D2, D3)                                                                              \
    if (P.n_layers == 3 && P.dims[0] == D0 && P.dims[1] == D1 && P.dims[2] == D2 && P.dims[3] == D3) {             \
        const TexUnitObjs none = {};                                                                               \
        k_decode_fp32<D0, D1, D2, D3><<<grid, 128, 0, st>>>(M, none, u, v, s, n, out, out_fp16);                   \
        return cudaGetLastError();                                                                                 \
    }

cudaError_t launch_decode_fp32(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                               void *out, int out_fp16, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    const MlpDev &P = M.mlp;
    const unsigned grid = grid_for(n, 128, 16);
    BCF_FP32_CASE(6, 16, 16, 8)
    BCF_FP32_CASE(13, 32, 32, 9)
    BCF_FP32_CASE(12, 16, 16, 9)
    BCF_FP32_CASE(25, 64, 64, 9)
    k_decode_fp32_generic<<<grid, 128, 0, st>>>(M, u, v, s, n, out, out_fp16);
    return cudaGetLastError();
}

// FP32 materials on variant 3: the texture unit's texels and the same exact filter, then the plain FP32 MLP
// (the common three-layer shapes; others keep the software texels)
#define BCF_FP32_HW_CASE(D0, D1, D2, D3)                                                                           \
    if (P.n_layers == 3 && P.dims[0] == D0 && P.dims[1] == D1 && P.dims[2] == D2 && P.dims[3] == D3) {             \
        k_decode_fp32<D0, D1, D2, D3, true><<<grid, 128, 0, st>>>(M, T, u, v, s, n, out, out_fp16);                 \
        return cudaGetLastError();                                                                                 \
    }

cudaError_t launch_decode_fp32_texunit(const MaterialDev &M, const TexUnitObjs &T, const float *u, const float *v,
                                       const float *s, int64_t n, void *out, int out_fp16, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    const MlpDev &P = M.mlp;
    const unsigned grid = grid_for(n, 128, 16);
    BCF_FP32_HW_CASE(6, 16, 16, 8)
    BCF_FP32_HW_CASE(13, 32, 32, 9)
    BCF_FP32_HW_CASE(12, 16, 16, 9)
    BCF_FP32_HW_CASE(25, 64, 64, 9)
    return launch_decode_fp32(M, u, v, s, n, out, out_fp16, st);
}

template <int PREC>
static int mma_act_bytes(const MlpDev &P)
{
    int mx = 0;
    for (int l = 0; l < P.n_layers; ++l)
        mx = max(mx, 32 * tile_stride_bytes<PREC>(P.kpad[l]));
    return (mx + 15) & ~15;
}

template <int PREC, int K0 = 0, int N1 = 0, int N2 = 0>
int64_t mma_smem_bytes(const MlpDev &P, int warps)
{
    const int C = P.dims[P.n_layers];
    const int act = mma_act_bytes<PREC>(P);
    const int per_warp = mma_per_warp_bytes(act, mma_act1_bytes<PREC, K0, N1, N2>(act), C, P.dims[0], K0 == 0);
    return (int64_t)mlp_smem_weight_bytes<PREC>(P) + ((mlp_smem_bias_floats(P) * 4 + 15) & ~15) +
           (int64_t)warps * per_warp;
}

template <int PREC, int HW, int K0, int N1, int N2, int NO>
static cudaError_t launch_mma_tc_shape(const MaterialDev &M, const TexUnitObjs &T, const float *u, const float *v,
                                       const float *s, int64_t n, void *out, int out_fp16, cudaStream_t st)
{
    using TM = TcMlp<PREC, 4, K0, N1, N2, NO>;
    const int64_t smem = MmaTcLayout<PREC, HW, K0, N1, N2, NO>(M.mlp).total;
    if (smem > 200 * 1024)
        return cudaErrorInvalidConfiguration;
    auto kern = k_decode_mma_tc<PREC, HW, K0, N1, N2, NO>;
    static int per_sm = 0;
    if (!per_sm) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        // resident CTAs per SM from registers, shared memory and tensor-memory columns (512 per SM; every
        // CTA holds its columns for its whole life)
        cudaFuncAttributes fa{};
        int regs = 64;
        if (cudaFuncGetAttributes(&fa, kern) == cudaSuccess && fa.numRegs > 0)
            regs = fa.numRegs;
        int dev = 0, smem_sm = 228 * 1024;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        const int by_regs = 65536 / (128 * ((regs + 7) & ~7));
        const int by_smem = smem_sm / (int)(smem + 1024);
        per_sm = max(1, min(min(by_regs, by_smem), min(512 / TM::NCOLS, 16)));
    }
    const int64_t tiles = (n + 127) / 128;
    const int64_t grid = min(tiles, (int64_t)sm_count() * per_sm);
    kern<<<(unsigned)grid, 128, (size_t)smem, st>>>(M, T, u, v, s, n, out, out_fp16, check_word());
    return cudaGetLastError();
}

template <int PREC, int HW, int K0, int N1, int N2, int NO>
static cudaError_t launch_mma_shape(const MaterialDev &M, const TexUnitObjs &T, const float *u, const float *v,
                                    const float *s, int64_t n, void *out, int out_fp16, cudaStream_t st)
{
    if constexpr (K0 != 0 && N2 != 0)
        if (M.mlp_engine == BCF_MLP_TCGEN05)
            return launch_mma_tc_shape<PREC, HW, K0, N1, N2, NO>(M, T, u, v, s, n, out, out_fp16, st);
    const int threads = 128;
    const int64_t smem = mma_smem_bytes<PREC, K0, N1, N2>(M.mlp, threads / 32);
    if (smem > 200 * 1024)
        return cudaErrorInvalidConfiguration;
    auto kern = k_decode_mma<PREC, HW, K0, N1, N2, NO>;
    static int configured = 0;
    if (!configured) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        configured = 1;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, (size_t)smem);
    const unsigned grid = grid_for((n + 31) / 32, threads / 32, max(per_sm, 1));
    kern<<<grid, threads, (size_t)smem, st>>>(M, T, u, v, s, n, out, out_fp16, mma_act_bytes<PREC>(M.mlp));
    return cudaGetLastError();
}

template <int PREC, int HW>
static cudaError_t launch_mma(const MaterialDev &M, const TexUnitObjs &T, const float *u, const float *v,
                              const float *s, int64_t n, void *out, int out_fp16, cudaStream_t st)
{
    const MlpDev &P = M.mlp;
    if (P.n_layers == 3) {
        const int k0 = P.kpad[0], n1 = P.npad[0], n2 = P.npad[1], no = P.npad[2];
        constexpr int kq = PREC == BCF_FP8_E4M3 ? 32 : 16;
        if (k0 == kq && n1 == 32 && n2 == 32 && no == 16)
            return launch_mma_shape<PREC, HW, kq, 32, 32, 16>(M, T, u, v, s, n, out, out_fp16, st);
        if (k0 == 32 && n1 == 64 && n2 == 64 && no == 16)
            return launch_mma_shape<PREC, HW, 32, 64, 64, 16>(M, T, u, v, s, n, out, out_fp16, st);
    }
    if constexpr (PREC != BCF_FP8_E4M3)
        if (P.n_layers == 2 && P.kpad[0] == 16 && P.npad[0] == 16 && P.npad[1] == 16)
            return launch_mma_shape<PREC, HW, 16, 16, 0, 16>(M, T, u, v, s, n, out, out_fp16, st);
    return launch_mma_shape<PREC, HW, 0, 0, 0, 0>(M, T, u, v, s, n, out, out_fp16, st);
}

cudaError_t launch_decode_mma(const MaterialDev &M, const float *u, const float *v, const float *s, int64_t n,
                              void *out, int out_fp16, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    const TexUnitObjs none = {};
    switch (M.mlp.precision) {
    case BCF_FP16: return launch_mma<BCF_FP16, 0>(M, none, u, v, s, n, out, out_fp16, st);
    case BCF_BF16: return launch_mma<BCF_BF16, 0>(M, none, u, v, s, n, out, out_fp16, st);
    case BCF_FP8_E4M3: return launch_mma<BCF_FP8_E4M3, 0>(M, none, u, v, s, n, out, out_fp16, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_decode_texunit(const MaterialDev &M, const TexUnitObjs &T, int exact_filter, const float *u,
                                  const float *v, const float *s, int64_t n, void *out, int out_fp16, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    switch (M.mlp.precision * 2 + (exact_filter ? 1 : 0)) {
    case BCF_FP16 * 2: return launch_mma<BCF_FP16, 1>(M, T, u, v, s, n, out, out_fp16, st);
    case BCF_FP16 * 2 + 1: return launch_mma<BCF_FP16, 2>(M, T, u, v, s, n, out, out_fp16, st);
    case BCF_BF16 * 2: return launch_mma<BCF_BF16, 1>(M, T, u, v, s, n, out, out_fp16, st);
    case BCF_BF16 * 2 + 1: return launch_mma<BCF_BF16, 2>(M, T, u, v, s, n, out, out_fp16, st);
    case BCF_FP8_E4M3 * 2: return launch_mma<BCF_FP8_E4M3, 1>(M, T, u, v, s, n, out, out_fp16, st);
    case BCF_FP8_E4M3 * 2 + 1: return launch_mma<BCF_FP8_E4M3, 2>(M, T, u, v, s, n, out, out_fp16, st);
    default: return cudaErrorInvalidValue;
    }
}

int64_t decode_mma_smem_bytes(const MlpDev &P)
{
    switch (P.precision) {
    case BCF_FP16: return mma_smem_bytes<BCF_FP16>(P, 4);
    case BCF_BF16: return mma_smem_bytes<BCF_BF16>(P, 4);
    case BCF_FP8_E4M3: return mma_smem_bytes<BCF_FP8_E4M3>(P, 4);
    default: return 0;
    }
}


template <int PREC, int K0, int N1, int N2, int NO>
static cudaError_t launch_set_tex_shape(const MaterialDev &M0, const MaterialDev *mats, const TexUnitObjs *texs,
                                        int nmat, const int64_t *offsets, const float *u, const float *v,
                                        const float *s, int64_t n, void *out, int out_fp16, int *counter,
                                        unsigned *check, const SetConfig &cfg, cudaStream_t st)
{
    const MlpDev &P = M0.mlp;
    const int act = mma_act_bytes<PREC>(P);
    const int64_t smem = (int64_t)kSetTexWarps * set_tex_warp_bytes<PREC, K0, N1, N2>(P, act);
    if (smem > 160 * 1024)
        return cudaErrorInvalidConfiguration;
    auto kern = k_decode_set_tex<PREC, K0, N1, N2, NO>;
    static int configured = 0;
    if (!configured) {
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 * 1024);
        configured = 1;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kSetTexWarps, (size_t)smem);
    if (cfg.ctas_per_sm > 0)
        per_sm = min(per_sm, cfg.ctas_per_sm);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess)
        return e;
    kern<<<(unsigned)(sm_count() * max(per_sm, 1)), 32 * kSetTexWarps, (size_t)smem, st>>>(
        mats, texs, nmat, offsets, u, v, s, n, out, out_fp16, counter, check, act, max(cfg.chunk, 1));
    return cudaGetLastError();
}

static bool set_tex_two_layer(const MlpDev &P);

bool set_tex_supported(const MaterialDev &M0)
{
    const MlpDev &P = M0.mlp;
    if (P.precision == BCF_FP32)
        return false;
    if (set_tex_two_layer(P))
        return true;
    if (P.n_layers != 3)
        return false;
    const int kq = P.precision == BCF_FP8_E4M3 ? 32 : 16;
    return (P.kpad[0] == kq && P.npad[0] == 32 && P.npad[1] == 32 && P.npad[2] == 16) ||
           (P.kpad[0] == 32 && P.npad[0] == 64 && P.npad[1] == 64 && P.npad[2] == 16);
}

static bool set_tex_two_layer(const MlpDev &P)
{
    return P.n_layers == 2 && P.precision != BCF_FP8_E4M3 && P.kpad[0] == 16 && P.npad[0] == 16 && P.npad[1] == 16;
}

cudaError_t launch_decode_set_tex(const MaterialDev &M0, const MaterialDev *mats, const TexUnitObjs *texs, int nmat,
                                  const int64_t *offsets, const float *u, const float *v, const float *s, int64_t n,
                                  void *out, int out_fp16, int *counter, unsigned *check, const SetConfig &cfg,
                                  cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    const MlpDev &P = M0.mlp;
    const bool wide = P.kpad[0] == 32 && P.npad[0] == 64;
    if (set_tex_two_layer(P)) {
        if (P.precision == BCF_BF16)
            return launch_set_tex_shape<BCF_BF16, 16, 16, 0, 16>(M0, mats, texs, nmat, offsets, u, v, s, n, out,
                                                                  out_fp16, counter, check, cfg, st);
        return launch_set_tex_shape<BCF_FP16, 16, 16, 0, 16>(M0, mats, texs, nmat, offsets, u, v, s, n, out,
                                                              out_fp16, counter, check, cfg, st);
    }
#define BCF_SET_TEX(PR, KQ)                                                                                          \
    return wide ? launch_set_tex_shape<PR, 32, 64, 64, 16>(M0, mats, texs, nmat, offsets, u, v, s, n, out, out_fp16, \
                                                           counter, check, cfg, st)                                         \
                : launch_set_tex_shape<PR, KQ, 32, 32, 16>(M0, mats, texs, nmat, offsets, u, v, s, n, out, out_fp16, \
                                                           counter, check, cfg, st)
    switch (P.precision) {
    case BCF_FP16: BCF_SET_TEX(BCF_FP16, 16);
    case BCF_BF16: BCF_SET_TEX(BCF_BF16, 16);
    case BCF_FP8_E4M3: BCF_SET_TEX(BCF_FP8_E4M3, 32);
    default: return cudaErrorInvalidValue;
    }
#undef BCF_SET_TEX
}

} // namespace bcf
