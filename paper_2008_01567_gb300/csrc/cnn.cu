// 2.5D CNN denoising agents H_xy,t, H_yz,t, H_zx,t (Sec. IV, Eq. (14)).
//
// Network (depth, width and BatchNorm as fixed for this library, the paper's
// figure being unavailable): conv 5->64 + ReLU, 8 x (conv 64->64 + BN + ReLU),
// conv 64->1, output = centre frame - network output (the residual through the
// selection of the centre channel).  Input channels are the 5 time-points
// t-2..t+2 of the same slice, clamped at the ends of the time axis.
//
// Inference data path, per chunk of whole time-points:
//   pack5     FP32 4D volume -> BF16 [img][H][W][64]: for every pixel the 5x3x3
//             neighbourhood (45 values, zero padded to 64) in the order
//             k = frame*9 + ky*3 + kx, so layer 1 becomes a K = 64 GEMM.
//   conv_tc   tcgen05 implicit GEMM, M = 128 pixels (a 16 x 8 block of one
//             image), N = 64 (or 16 for the last layer), K = 9 taps x 64
//             channels.  TMA brings, per tile, the three column-shifted
//             18 x 8 x 64 halo blocks; tap (dy, dx) is the dx block offset by
//             dy * 8 rows = dy * 1024 bytes, so all nine taps read the same
//             three swizzled buffers.  FP32 accumulators live in TMEM (two
//             buffers, so the epilogue of one tile overlaps the MMAs of the next).
//   epilogue  bias + ReLU + BF16 through a swizzled staging tile and a TMA
//             store; the last layer writes centre - R straight into the FP32
//             4D output volume.
// BatchNorm is folded into the weights and biases (fold_kernel).
#include <cuda.h>
#include <cuda_bf16.h>
#include <math.h>

#include <vector>

#include "common.cuh"
#include "tc.cuh"

namespace msf {
namespace cnn {

constexpr int LAYERS = 10;
constexpr int CH = 64;
constexpr int FRAMES = 5;
constexpr int KPACK = 64;           // packed layer-1 K (45 used)
constexpr float BN_EPS = 1e-5f;
constexpr int THREADS = 192;        // warp 0 TMA, warp 1 MMA, warps 2-5 epilogue
constexpr int TILE_A = 16, TILE_B = 8;
constexpr int HALO_BYTES = (TILE_A + 2) * TILE_B * 128;   // 18432
constexpr int TILE_BYTES = TILE_A * TILE_B * 128;         // 16384
constexpr int TMEM_COLS = 128;

enum Epi { EPI_RELU = 0, EPI_RESID = 1 };

// Flat FP32 parameter layout (see msf.h): W_l, b_l for l = 0..9, then gamma,
// beta, running mean, running var for the 8 BatchNorm layers.
struct Offsets {
    size_t w[LAYERS], b[LAYERS], gamma[LAYERS], beta[LAYERS], mean[LAYERS], var[LAYERS];
    size_t total;
};

static int cin_of(int l) { return l == 0 ? FRAMES : CH; }
static int cout_of(int l) { return l == LAYERS - 1 ? 1 : CH; }

static Offsets offsets() {
    Offsets o{};
    size_t p = 0;
    for (int l = 0; l < LAYERS; ++l) {
        o.w[l] = p;
        p += (size_t)cout_of(l) * cin_of(l) * 9;
        o.b[l] = p;
        p += cout_of(l);
    }
    for (int l = 0; l < LAYERS; ++l) o.gamma[l] = o.beta[l] = o.mean[l] = o.var[l] = (size_t)-1;
    for (int l = 1; l < LAYERS - 1; ++l) {
        o.gamma[l] = p; p += CH;
        o.beta[l] = p; p += CH;
        o.mean[l] = p; p += CH;
        o.var[l] = p; p += CH;
    }
    o.total = p;
    return o;
}

// Packed weights of layer l: [taps][rows][64] BF16, rows = N of the GEMM.
static int taps_of(int l) { return l == 0 ? 1 : 9; }
static int rows_of(int l) { return l == LAYERS - 1 ? 16 : CH; }

struct FoldArgs {
    int layer, taps, rows, cin, cout;
    long long w, b, gamma, beta, mean, var;   // offsets into params (-1: none)
};

// BatchNorm folding and BF16 packing of one layer:
//   w' = w * g/sqrt(var+eps),  b' = (b - mean) g/sqrt(var+eps) + beta.
// Layer 1 is packed as a single K = 64 slice in the pack5 order; the last
// layer's 1 output channel is padded to 16 rows.
__global__ void fold_kernel(const float* __restrict__ params, __nv_bfloat16* __restrict__ wpack,
                            float* __restrict__ bias, FoldArgs f) {
    const int n_el = f.taps * f.rows * KPACK;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_el; e += gridDim.x * blockDim.x) {
        const int tap = e / (f.rows * KPACK);
        const int n = (e / KPACK) % f.rows;
        const int k = e % KPACK;
        float val = 0.0f;
        if (n < f.cout) {
            float s = 1.0f;
            if (f.gamma >= 0) s = params[f.gamma + n] / sqrtf(params[f.var + n] + BN_EPS);
            if (f.layer == 0) {
                if (k < FRAMES * 9) val = params[f.w + (size_t)n * f.cin * 9 + k];   // [n][c][ky][kx], k = c*9+ky*3+kx
            } else {
                val = params[f.w + ((size_t)n * f.cin + k) * 9 + tap] * s;
            }
        }
        wpack[e] = __float2bfloat16_rn(val);
    }
    for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < f.rows; n += gridDim.x * blockDim.x) {
        float bv = 0.0f;
        if (n < f.cout) {
            bv = params[f.b + n];
            if (f.gamma >= 0) {
                const float s = params[f.gamma + n] / sqrtf(params[f.var + n] + BN_EPS);
                bv = (bv - params[f.mean + n]) * s + params[f.beta + n];
            }
        }
        bias[n] = bv;
    }
}

// ---------------------------------------------------------------- geometry

struct SliceGeom {
    int orient;          // 0 xy-t, 1 yz-t, 2 zx-t
    int nx, ny, nz, nt;
    int S, H, W;         // slices per frame, image rows, image cols
    int t0, nframes;     // frames of this chunk
};

// 4D index of image pixel (a, b) of slice s at time-point t.
__device__ __forceinline__ size_t vol_index(const SliceGeom& g, int t, int s, int a, int b) {
    if (g.orient == 0) return (((size_t)t * g.nz + s) * g.ny + a) * g.nx + b;        // s=z, a=y, b=x
    if (g.orient == 1) return (((size_t)t * g.nz + a) * g.ny + b) * g.nx + s;        // s=x, a=z, b=y
    return (((size_t)t * g.nz + b) * g.ny + s) * g.nx + a;                          // s=y, a=x, b=z
}

// One thread per pixel of the chunk; the thread-to-pixel order follows the
// volume's contiguous axis (x) so that the 45 gathers coalesce.
__global__ void pack5_kernel(const float* __restrict__ vol, uint4* __restrict__ out, SliceGeom g) {
    const size_t per_frame = (size_t)g.S * g.H * g.W;
    const size_t total = per_frame * g.nframes;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int tl = (int)(p / per_frame);
        size_t r = p % per_frame;
        int s, a, b;
        if (g.orient == 0) {          // b (= x) fastest
            b = (int)(r % g.W); r /= g.W; a = (int)(r % g.H); s = (int)(r / g.H);
        } else if (g.orient == 1) {   // s (= x) fastest
            s = (int)(r % g.S); r /= g.S; b = (int)(r % g.W); a = (int)(r / g.W);
        } else {                      // a (= x) fastest
            a = (int)(r % g.H); r /= g.H; b = (int)(r % g.W); s = (int)(r / g.W);
        }
        const int t = g.t0 + tl;
        float v[FRAMES * 9];
#pragma unroll
        for (int c = 0; c < FRAMES; ++c) {
            const int tc = min(max(t + c - 2, 0), g.nt - 1);
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int aa = a + ky - 1, bb = b + kx - 1;
                    v[c * 9 + ky * 3 + kx] =
                        (aa >= 0 && aa < g.H && bb >= 0 && bb < g.W) ? __ldg(vol + vol_index(g, tc, s, aa, bb)) : 0.0f;
                }
            }
        }
        uint32_t w[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const float lo = 2 * i < FRAMES * 9 ? v[2 * i] : 0.0f;
            const float hi = 2 * i + 1 < FRAMES * 9 ? v[2 * i + 1] : 0.0f;
            __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
            w[i] = *reinterpret_cast<uint32_t*>(&h);
        }
        const size_t img = (size_t)tl * g.S + s;
        uint4* dst = out + ((img * g.H + a) * g.W + b) * 8;
#pragma unroll
        for (int c = 0; c < 8; ++c) dst[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
    }
}

// ---------------------------------------------------------------- tcgen05 conv

struct TileGeom {
    int H, W, imgs;          // images of this launch (img index 0..imgs-1)
    int tiles_a, tiles_b, total;
};

__device__ __forceinline__ void decode_tile(const TileGeom& tg, int tile, int& img, int& a0, int& b0) {
    const int per = tg.tiles_a * tg.tiles_b;
    img = tile / per;
    const int r = tile - img * per;
    a0 = (r / tg.tiles_b) * TILE_A;
    b0 = (r % tg.tiles_b) * TILE_B;
}

template <int TAPS, int N, int NS, int EPI>
struct ConvCfg {
    static constexpr int A_BYTES = TAPS == 9 ? 3 * HALO_BYTES : TILE_BYTES;
    static constexpr int W_BYTES = TAPS * N * 128;
    static constexpr int O_BYTES = EPI == EPI_RELU ? 2 * TILE_BYTES : 0;
    static constexpr int BAR_BYTES = 256;
    static constexpr int SMEM = 1024 + NS * A_BYTES + W_BYTES + O_BYTES + BAR_BYTES;
};

// Persistent warp-specialised implicit-GEMM 3x3 (TAPS = 9) or 1x1 (TAPS = 1)
// convolution over BF16 NHWC activations.  Tile t of the static round-robin
// sequence blockIdx.x, blockIdx.x + gridDim.x, ... is a 16 x 8 pixel block.
template <int TAPS, int N, int NS, int EPI>
__global__ void __launch_bounds__(THREADS, 1)
conv_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_w,
               const __grid_constant__ CUtensorMap map_out, const float* __restrict__ bias, TileGeom tg,
               SliceGeom sg, const float* __restrict__ centre, float* __restrict__ outv, int* __restrict__ err) {
    using C = ConvCfg<TAPS, N, NS, EPI>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sW = sA + NS * C::A_BYTES;
    uint8_t* sO = sW + C::W_BYTES;
    uint64_t* bars = (uint64_t*)(sO + C::O_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + NS;
    uint64_t* tfull = bars + 2 * NS;
    uint64_t* tempty = tfull + 2;
    uint64_t* wbar = tempty + 2;
    uint32_t* tmem_slot = (uint32_t*)(wbar + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&tfull[b], 1);
            tc::mbar_init(&tempty[b], 128);
        }
        tc::mbar_init(wbar, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem_base = *tmem_slot;

    auto give_up = [&](int code) {
        *abort_flag = 1;
        atomicExch(err, code);
    };

    if (warp == 0) {
        if (lane == 0) {
            // ---------------- producer: weights once, then the A tiles
            int issued[NS];
            for (int s = 0; s < NS; ++s) issued[s] = 0;
            tc::mbar_expect_tx(wbar, C::W_BYTES);
            for (int tap = 0; tap < TAPS; ++tap) tc::tma_load_2d(sW + tap * N * 128, &map_w, wbar, 0, tap * N);
            int it = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < tg.total; tile += gridDim.x, ++it) {
                const int s = it % NS, u = it / NS;
                if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                int img, a0, b0;
                decode_tile(tg, tile, img, a0, b0);
                uint8_t* dst = sA + s * C::A_BYTES;
                tc::mbar_expect_tx(&full[s], C::A_BYTES);
                if (TAPS == 9) {
#pragma unroll
                    for (int dx = 0; dx < 3; ++dx)
                        tc::tma_load_4d(dst + dx * HALO_BYTES, &map_a, &full[s], 0, b0 + dx - 1, a0 - 1, img);
                } else {
                    tc::tma_load_4d(dst, &map_a, &full[s], 0, b0, a0, img);
                }
                issued[s] = u + 1;
            }
            if (!ok) {
                give_up(MSF_ERR_TIMEOUT);
                // let the copies already issued land before the CTA exits
                for (int s = 0; s < NS; ++s)
                    if (issued[s] > 0) tc::mbar_wait(&full[s], (issued[s] - 1) & 1, nullptr, 100000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            constexpr uint32_t idesc = tc::idesc_bf16<128, N>();
            bool ok = tc::mbar_wait(wbar, 0, abort_flag);
            tc::fence_after_sync();
            int it = 0;
            for (int tile = blockIdx.x; ok && tile < tg.total; tile += gridDim.x, ++it) {
                const int s = it % NS, u = it / NS, ab = it & 1, ua = it >> 1;
                if (!tc::mbar_wait(&full[s], u & 1, abort_flag)) { ok = false; break; }
                if (ua > 0 && !tc::mbar_wait(&tempty[ab], (ua - 1) & 1, abort_flag)) { ok = false; break; }
                tc::fence_after_sync();
                const uint32_t d_tmem = tmem_base + ab * N;
                const uint32_t a_base = tc::smem_u32(sA + s * C::A_BYTES);
                const uint32_t w_base = tc::smem_u32(sW);
#pragma unroll
                for (int tap = 0; tap < TAPS; ++tap) {
                    const uint32_t a_off = TAPS == 9 ? (tap % 3) * HALO_BYTES + (tap / 3) * 1024 : 0;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        const uint64_t ad = tc::desc_sw128(a_base + a_off + kk * 32);
                        const uint64_t bd = tc::desc_sw128(w_base + tap * N * 128 + kk * 32);
                        tc::mma_bf16(d_tmem, ad, bd, idesc, (tap | kk) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&empty[s]);
                tc::mma_commit(&tfull[ab]);
            }
            if (!ok) give_up(MSF_ERR_TIMEOUT);
        }
    } else {
        // ---------------- epilogue: 4 warps, TMEM lane quarter = warp % 4
        const int q = warp & 3;
        const int row = q * 32 + lane;           // accumulator row = pixel of the tile
        int it = 0;
        for (int tile = blockIdx.x; tile < tg.total; tile += gridDim.x, ++it) {
            const int ab = it & 1, ua = it >> 1;
            if (!tc::mbar_wait(&tfull[ab], ua & 1, abort_flag)) {
                give_up(MSF_ERR_TIMEOUT);
                break;
            }
            tc::fence_after_sync();
            uint32_t r[N];
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + ab * N;
#pragma unroll
            for (int c = 0; c < N / 16; ++c) tc::tmem_ld16(taddr + c * 16, r + c * 16);
            tc::tmem_ld_wait();
            tc::fence_before_sync();
            tc::mbar_arrive(&tempty[ab]);
            int img, a0, b0;
            decode_tile(tg, tile, img, a0, b0);
            if (EPI == EPI_RELU) {
                uint32_t w[N / 2];
#pragma unroll
                for (int j = 0; j < N / 2; ++j) {
                    const float lo = fmaxf(__uint_as_float(r[2 * j]) + __ldg(bias + 2 * j), 0.0f);
                    const float hi = fmaxf(__uint_as_float(r[2 * j + 1]) + __ldg(bias + 2 * j + 1), 0.0f);
                    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
                    w[j] = *reinterpret_cast<uint32_t*>(&h);
                }
                // per-warp staging: this warp's 32 rows are 4 image rows of
                // the tile; lane 0 stores them with its own bulk group, so no
                // barrier spans more than one warp
                uint8_t* stage = sO + ((it & 1) * 4 + q) * (TILE_BYTES / 4);
                if (lane == 0) tc::tma_store_wait_read<1>();
                __syncwarp();
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    *reinterpret_cast<uint4*>(stage + lane * 128 + ((c ^ (lane & 7)) << 4)) =
                        make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    // a block wholly below the image has nothing to store
                    if (a0 + q * (TILE_A / 4) < tg.H) tc::tma_store_4d(&map_out, stage, 0, b0, a0 + q * (TILE_A / 4), img);
                    tc::tma_store_commit();
                }
            } else {
                const float R = __uint_as_float(r[0]) + __ldg(bias);
                const int a = a0 + row / TILE_B, b = b0 + row % TILE_B;
                if (a < tg.H && b < tg.W) {
                    const int t = sg.t0 + img / sg.S, s = img % sg.S;
                    const size_t idx = vol_index(sg, t, s, a, b);
                    outv[idx] = centre[idx] - R;
                }
            }
        }
        if (EPI == EPI_RELU && lane == 0) tc::tma_store_wait_all();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ---------------------------------------------------------------- host helpers

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 4D BF16 activation tensor [imgs][H][W][64] with a box of 64 x 8 x rows x 1.
static msf_status make_act_map(CUtensorMap* m, void* base, int imgs, int H, int W, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[4] = {(cuuint64_t)CH, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)imgs};
    cuuint64_t strides[3] = {(cuuint64_t)CH * 2, (cuuint64_t)W * CH * 2, (cuuint64_t)H * W * CH * 2};
    cuuint32_t box[4] = {(cuuint32_t)CH, (cuuint32_t)TILE_B, (cuuint32_t)box_rows, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled (activations) failed: %d", (int)r);
    return MSF_OK;
}

// 2D BF16 weights [rows_total][64] with a box of 64 x rows.
static msf_status make_w_map(CUtensorMap* m, void* base, int rows_total, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)KPACK, (cuuint64_t)rows_total};
    cuuint64_t strides[1] = {(cuuint64_t)KPACK * 2};
    cuuint32_t box[2] = {(cuuint32_t)KPACK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled (weights) failed: %d", (int)r);
    return MSF_OK;
}

static int g_num_sms = 0;

template <int TAPS, int N, int NS, int EPI>
static msf_status launch_conv(const CUtensorMap& ma, const CUtensorMap& mw, const CUtensorMap& mo, const float* bias,
                              const TileGeom& tg, const SliceGeom& sg, const float* centre, float* outv, int* err,
                              cudaStream_t st) {
    using C = ConvCfg<TAPS, N, NS, EPI>;
    auto kern = conv_tc_kernel<TAPS, N, NS, EPI>;
    static bool attr = false;
    if (!attr) {
        MSF_TRY_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM));
        attr = true;
    }
    if (g_num_sms == 0) {
        int dev = 0;
        MSF_TRY_CUDA(cudaGetDevice(&dev));
        MSF_TRY_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    const int grid = tg.total < g_num_sms ? tg.total : g_num_sms;
    if (grid <= 0) return MSF_OK;
    MSF_PROF(TAPS == 1 ? "conv1_tc" : (EPI == EPI_RESID ? "conv10_tc" : "conv3x3_tc"), st);
    kern<<<grid, THREADS, C::SMEM, st>>>(ma, mw, mo, bias, tg, sg, centre, outv, err);
    MSF_LAUNCH_CHECK();
    return MSF_OK;
}

}  // namespace cnn
}  // namespace msf

// ====================================================================== handle

using namespace msf;
using namespace msf::cnn;

struct msf_cnn {
    int64_t max_pixels = 0;
    Offsets off;
    float* d_params = nullptr;      // FP32 master parameters
    float* d_grad = nullptr;
    float* d_m = nullptr;           // Adam moments
    float* d_v = nullptr;
    __nv_bfloat16* d_wpack = nullptr;
    float* d_bias = nullptr;        // [10][64]
    size_t wpack_off[LAYERS];
    __nv_bfloat16* d_act[2] = {nullptr, nullptr};
    int* d_err = nullptr;
    bool folded = false;
    int64_t adam_t = 0;
    // training workspace (allocated on first use by msf_train_step)
    void* train_ws = nullptr;
    size_t train_ws_bytes = 0;
};

static msf_status fold_all(msf_cnn* c, cudaStream_t st) {
    for (int l = 0; l < LAYERS; ++l) {
        FoldArgs f;
        f.layer = l;
        f.taps = taps_of(l);
        f.rows = rows_of(l);
        f.cin = cin_of(l);
        f.cout = cout_of(l);
        f.w = (long long)c->off.w[l];
        f.b = (long long)c->off.b[l];
        const bool bn = l > 0 && l < LAYERS - 1;
        f.gamma = bn ? (long long)c->off.gamma[l] : -1;
        f.beta = bn ? (long long)c->off.beta[l] : -1;
        f.mean = bn ? (long long)c->off.mean[l] : -1;
        f.var = bn ? (long long)c->off.var[l] : -1;
        MSF_PROF("fold", st);
        fold_kernel<<<64, 256, 0, st>>>(c->d_params, c->d_wpack + c->wpack_off[l], c->d_bias + l * CH, f);
        MSF_LAUNCH_CHECK();
    }
    c->folded = true;
    return MSF_OK;
}

extern "C" size_t msf_cnn_param_count(void) { return offsets().total; }

extern "C" msf_status msf_cnn_create(int64_t max_pixels, msf_cnn** out) {
    MSF_REQUIRE(out, "msf_cnn_create: NULL argument");
    *out = nullptr;
    MSF_REQUIRE(max_pixels >= 128, "msf_cnn_create: max_pixels must be >= 128");
    MSF_TRY(check_device());
    msf_cnn* c = new msf_cnn();
    c->max_pixels = max_pixels;
    c->off = offsets();
    size_t wp = 0;
    for (int l = 0; l < LAYERS; ++l) {
        c->wpack_off[l] = wp;
        wp += (size_t)taps_of(l) * rows_of(l) * KPACK;
    }
    const size_t P = c->off.total;
    const size_t act = (size_t)max_pixels * CH * sizeof(__nv_bfloat16);
    bool ok = cudaMalloc(&c->d_params, P * 4) == cudaSuccess && cudaMalloc(&c->d_grad, P * 4) == cudaSuccess &&
              cudaMalloc(&c->d_m, P * 4) == cudaSuccess && cudaMalloc(&c->d_v, P * 4) == cudaSuccess &&
              cudaMalloc(&c->d_wpack, wp * 2) == cudaSuccess && cudaMalloc(&c->d_bias, LAYERS * CH * 4) == cudaSuccess &&
              cudaMalloc(&c->d_act[0], act) == cudaSuccess && cudaMalloc(&c->d_act[1], act) == cudaSuccess &&
              cudaMalloc(&c->d_err, sizeof(int)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        msf_cnn_destroy(c);
        return fail(MSF_ERR_NOMEM, "msf_cnn_create: out of device memory");
    }
    cudaMemset(c->d_params, 0, P * 4);
    cudaMemset(c->d_m, 0, P * 4);
    cudaMemset(c->d_v, 0, P * 4);
    cudaMemset(c->d_err, 0, sizeof(int));
    *out = c;
    return MSF_OK;
}

extern "C" void msf_cnn_destroy(msf_cnn* c) {
    if (!c) return;
    cudaFree(c->d_params); cudaFree(c->d_grad); cudaFree(c->d_m); cudaFree(c->d_v);
    cudaFree(c->d_wpack); cudaFree(c->d_bias);
    cudaFree(c->d_act[0]); cudaFree(c->d_act[1]);
    cudaFree(c->d_err);
    cudaFree(c->train_ws);
    delete c;
}

extern "C" msf_status msf_cnn_set_params(msf_cnn* c, const float* h_params, size_t n) {
    MSF_REQUIRE(c && h_params, "msf_cnn_set_params: NULL argument");
    MSF_REQUIRE(n == c->off.total, "msf_cnn_set_params: expected %zu parameters, got %zu", c->off.total, n);
    MSF_TRY_CUDA(cudaMemcpy(c->d_params, h_params, n * 4, cudaMemcpyHostToDevice));
    MSF_TRY_CUDA(cudaMemset(c->d_m, 0, n * 4));
    MSF_TRY_CUDA(cudaMemset(c->d_v, 0, n * 4));
    c->adam_t = 0;
    MSF_TRY(fold_all(c, nullptr));
    MSF_TRY_CUDA(cudaDeviceSynchronize());
    return MSF_OK;
}

extern "C" msf_status msf_cnn_get_params(msf_cnn* c, float* h_params, size_t n) {
    MSF_REQUIRE(c && h_params, "msf_cnn_get_params: NULL argument");
    MSF_REQUIRE(n == c->off.total, "msf_cnn_get_params: expected %zu parameters, got %zu", c->off.total, n);
    MSF_TRY_CUDA(cudaDeviceSynchronize());
    MSF_TRY_CUDA(cudaMemcpy(h_params, c->d_params, n * 4, cudaMemcpyDeviceToHost));
    return MSF_OK;
}

extern "C" msf_status msf_denoise(msf_cnn* c, msf_orient orient, const msf_vol* vol, const float* d_in,
                                  float* d_out, void* stream) {
    MSF_REQUIRE(c && vol && d_in && d_out, "msf_denoise: NULL argument");
    MSF_REQUIRE(orient >= MSF_XY_T && orient <= MSF_ZX_T, "msf_denoise: bad orientation %d", (int)orient);
    MSF_REQUIRE(vol->nx > 0 && vol->ny > 0 && vol->nz > 0 && vol->nt > 0, "msf_denoise: bad volume");
    MSF_REQUIRE(d_in != d_out, "msf_denoise: input and output must differ");
    cudaStream_t st = as_stream(stream);
    SliceGeom sg;
    sg.orient = (int)orient;
    sg.nx = vol->nx; sg.ny = vol->ny; sg.nz = vol->nz; sg.nt = vol->nt;
    if (orient == MSF_XY_T) { sg.S = vol->nz; sg.H = vol->ny; sg.W = vol->nx; }
    else if (orient == MSF_YZ_T) { sg.S = vol->nx; sg.H = vol->nz; sg.W = vol->ny; }
    else { sg.S = vol->ny; sg.H = vol->nx; sg.W = vol->nz; }
    const int64_t per_frame = (int64_t)sg.S * sg.H * sg.W;
    MSF_REQUIRE(per_frame <= c->max_pixels,
                "msf_denoise: one time-point has %lld pixels but the handle holds %lld (max_pixels)",
                (long long)per_frame, (long long)c->max_pixels);
    MSF_REQUIRE(per_frame * 128 < ((int64_t)1 << 40), "msf_denoise: frame too large");
    if (!c->folded) MSF_TRY(fold_all(c, st));
    const int fchunk = (int)(c->max_pixels / per_frame);
    const int imgs_cap = fchunk * sg.S;
    CUtensorMap m16[2], m18[2], m4[2], mw[LAYERS];
    for (int b = 0; b < 2; ++b) {
        MSF_TRY(make_act_map(&m16[b], c->d_act[b], imgs_cap, sg.H, sg.W, TILE_A));
        MSF_TRY(make_act_map(&m18[b], c->d_act[b], imgs_cap, sg.H, sg.W, TILE_A + 2));
        MSF_TRY(make_act_map(&m4[b], c->d_act[b], imgs_cap, sg.H, sg.W, TILE_A / 4));
    }
    for (int l = 0; l < LAYERS; ++l)
        MSF_TRY(make_w_map(&mw[l], c->d_wpack + c->wpack_off[l], taps_of(l) * rows_of(l), rows_of(l)));
    for (int t0 = 0; t0 < vol->nt; t0 += fchunk) {
        sg.t0 = t0;
        sg.nframes = fchunk < vol->nt - t0 ? fchunk : vol->nt - t0;
        {
            MSF_PROF("pack5", st);
            pack5_kernel<<<152 * 16, 256, 0, st>>>(d_in, reinterpret_cast<uint4*>(c->d_act[0]), sg);
            MSF_LAUNCH_CHECK();
        }
        TileGeom tg;
        tg.H = sg.H; tg.W = sg.W; tg.imgs = sg.nframes * sg.S;
        tg.tiles_a = (sg.H + TILE_A - 1) / TILE_A;
        tg.tiles_b = (sg.W + TILE_B - 1) / TILE_B;
        tg.total = tg.imgs * tg.tiles_a * tg.tiles_b;
        int cur = 0;
        MSF_TRY((launch_conv<1, 64, 4, EPI_RELU>(m16[0], mw[0], m4[1], c->d_bias, tg, sg, nullptr, nullptr,
                                                c->d_err, st)));
        cur = 1;
        for (int l = 1; l < LAYERS - 1; ++l) {
            MSF_TRY((launch_conv<9, 64, 2, EPI_RELU>(m18[cur], mw[l], m4[cur ^ 1], c->d_bias + l * CH, tg, sg,
                                                    nullptr, nullptr, c->d_err, st)));
            cur ^= 1;
        }
        MSF_TRY((launch_conv<9, 16, 2, EPI_RESID>(m18[cur], mw[LAYERS - 1], m4[cur ^ 1],
                                                 c->d_bias + (LAYERS - 1) * CH, tg, sg, d_in, d_out, c->d_err, st)));
    }
    return MSF_OK;
}

extern "C" msf_status msf_train_step(msf_cnn*, const float*, const float*, int, int, int, float, float*, void*) {
    return msf::fail(MSF_ERR_UNSUPPORTED, "msf_train_step: not built yet");
}
