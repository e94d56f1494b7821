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

#include <string.h>

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

// EPI_RELU:  relu(acc + bias) -> BF16 activations (TMA store)
// EPI_RAW:   acc + bias -> BF16 (TMA store): pre-BatchNorm outputs and input gradients
// EPI_RESID: last layer, centre - (acc + bias) -> FP32 4D output volume
// EPI_F32:   last layer, acc + bias -> FP32 [img][H][W] (training)
// EPI_PART:  last 64 -> 64 layer fused with the output layer (row-pair kernel):
//            per-tap output-layer sums -> FP32 planes [9][img][H][W]
// EPI_RAW32: acc + bias -> FP32 [img][H][W][64] (training: pre-BatchNorm outputs,
//            kept in FP32 because normalising subtracts their batch mean),
//            stored by TMA through map_out (make_f32_out_map); the kernel also
//            writes per-warp partial sums of the outputs and their squares
//            (the BatchNorm moments) to moments[CTA * 4 + warp][2][64]
enum Epi { EPI_RELU = 0, EPI_RESID = 1, EPI_RAW = 2, EPI_F32 = 3, EPI_RAW32 = 4, EPI_PART = 5 };

__host__ __device__ constexpr bool epi_stores_bf16(int e) { return e == EPI_RELU || e == EPI_RAW; }

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
    long long ss, sa, sb;    // element strides of slice, row and column in a frame
};

// Strides of (slice, row, col) inside one [nz][ny][nx] frame for an orientation.
static void set_strides(SliceGeom& g) {
    const long long sx = 1, sy = g.nx, sz = (long long)g.nx * g.ny;
    if (g.orient == 0) { g.ss = sz; g.sa = sy; g.sb = sx; }        // s=z, a=y, b=x
    else if (g.orient == 1) { g.ss = sx; g.sa = sz; g.sb = sy; }   // s=x, a=z, b=y
    else { g.ss = sy; g.sa = sx; g.sb = sz; }                      // s=y, a=x, b=z
}

// 4D index of image pixel (a, b) of slice s at time-point t.
__device__ __forceinline__ size_t vol_index(const SliceGeom& g, int t, int s, int a, int b) {
    if (g.orient == 0) return (((size_t)t * g.nz + s) * g.ny + a) * g.nx + b;        // s=z, a=y, b=x
    if (g.orient == 1) return (((size_t)t * g.nz + a) * g.ny + b) * g.nx + s;        // s=x, a=z, b=y
    return (((size_t)t * g.nz + b) * g.ny + s) * g.nx + a;                          // s=y, a=x, b=z
}

// Frame [nz][ny][nx] -> the agent's [S][H][W] order, as a 2D transpose of
// [rows][cols] -> [cols][rows] through 32 x 33 shared tiles: yz-t moves x to the
// front (rows = nz*ny, cols = nx), zx-t moves z to the back (rows = nz, cols = ny*nx).
__global__ void orient_transpose_kernel(const float* __restrict__ in, float* __restrict__ out, long long rows,
                                        long long cols) {
    __shared__ float tile[32][33];
    const long long r0 = (long long)blockIdx.y * 32, c0 = (long long)blockIdx.x * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const long long r = r0 + k, c = c0 + threadIdx.x;
        if (r < rows && c < cols) tile[k][threadIdx.x] = in[r * cols + c];
    }
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) {
        const long long c = c0 + k, r = r0 + threadIdx.x;
        if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][k];
    }
}

// The time-points a chunk of the first layer reads, each already in the
// agent's [S][H][W] order; f[k] is time-point first + k.
struct PackFrames {
    const float* f[20];     // frame pointers for time-points first .. first+count-1
    int first, count;
};

// ---------------------------------------------------------------- tcgen05 conv

// One arrival per warp on a barrier that counts warps: every lane has fenced
// its own accesses before this call; the warp converges, then lane 0 arrives
// (32 lanes arriving on one barrier word would serialise in shared memory).
__device__ __forceinline__ void warp_arrive(uint64_t* bar) {
    __syncwarp();
    if ((threadIdx.x & 31) == 0) tc::mbar_arrive(bar);
}

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

// Stage counts of the A-operand ring (one slot = all boxes of one tile), as
// measured fastest on GB300 for 384 x 384 slices: deeper rings or per-box slots
// were slower for every variant.
constexpr int NS_3X3 = 2, NS_LAST = 2, NS_1X1 = 4;

template <int TAPS, int N, int NS, int EPI>
struct ConvCfg {
    // A operand ring: NS slots of GROUP TMA boxes each.  A 3x3 tile takes
    // three boxes (the 18-row halo shifted by dx = -1, 0, +1), a 1x1 tile one
    // 16-row box; a slot holds a whole tile.
    static constexpr int BOXES = TAPS == 9 ? 3 : 1;
    static constexpr int GROUP = BOXES;
    static constexpr int SLOTS_PER_TILE = BOXES / GROUP;
    static constexpr int BOX_BYTES = TAPS == 9 ? HALO_BYTES : TILE_BYTES;
    static constexpr int SLOT_BYTES = GROUP * BOX_BYTES;
    static constexpr int W_BYTES = TAPS * N * 128;
    static constexpr int O_BYTES = epi_stores_bf16(EPI) ? TILE_BYTES : 0;
    // EPI_RAW32: per epilogue warp, its 32 pixels x 64 FP32 outputs of a tile
    // (the transpose behind the BatchNorm moments)
    static constexpr int M_BYTES = EPI == EPI_RAW32 ? 4 * 32 * 256 : 0;
    static constexpr int BAR_BYTES = 512;   // barriers, TMEM slot, abort flag (256 B), bias (256 B)
    static constexpr int SMEM = 1024 + NS * SLOT_BYTES + W_BYTES + O_BYTES + M_BYTES + BAR_BYTES;
    static_assert(BOXES % GROUP == 0, "a slot group must divide the boxes of a tile");
    static_assert((2 * NS + 5) * 8 + 8 <= 256, "barrier block overflows into the bias");
    static_assert(SMEM <= 232448, "more dynamic shared memory than a CTA may have");
};

// Persistent warp-specialised implicit-GEMM 3x3 (TAPS = 9) or 1x1 (TAPS = 1)
// convolution over BF16 NHWC activations.  Tile t of the static round-robin
// sequence blockIdx.x, blockIdx.x + gridDim.x, ... is a 16 x 8 pixel block.
// The producer streams A boxes through an NS-slot ring; the MMA issuer frees a
// slot once the taps that read it are issued.
template <int TAPS, int N, int NS, int EPI>
__global__ void __launch_bounds__(THREADS, 1)
conv_tc_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_w,
               const __grid_constant__ CUtensorMap map_out, const float* __restrict__ bias, TileGeom tg,
               SliceGeom sg, const float* __restrict__ centre, float* __restrict__ outv, double* __restrict__ moments,
               int* __restrict__ err) {
    using C = ConvCfg<TAPS, N, NS, EPI>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sW = sA + NS * C::SLOT_BYTES;
    uint8_t* sO = sW + C::W_BYTES;
    uint8_t* sM = sO + C::O_BYTES;
    uint64_t* bars = (uint64_t*)(sM + C::M_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + NS;
    uint64_t* tfull = bars + 2 * NS;
    uint64_t* tempty = tfull + 2;
    uint64_t* wbar = tempty + 2;
    uint32_t* tmem_slot = (uint32_t*)(wbar + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    float* sbias = (float*)((uint8_t*)bars + 256);
    if (threadIdx.x < N) sbias[threadIdx.x] = bias[threadIdx.x];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&tfull[b], 1);
            tc::mbar_init(&tempty[b], 4);     // one arrival per epilogue warp
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
            int j = 0;   // box sequence number
            bool ok = true;
            for (int tile = blockIdx.x; ok && tile < tg.total; tile += gridDim.x) {
                int img, a0, b0;
                decode_tile(tg, tile, img, a0, b0);
#pragma unroll
                for (int g = 0; g < C::SLOTS_PER_TILE; ++g, ++j) {
                    const int s = j % NS, u = j / NS;
                    if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    uint8_t* dst = sA + s * C::SLOT_BYTES;
                    tc::mbar_expect_tx(&full[s], C::SLOT_BYTES);
#pragma unroll
                    for (int k = 0; k < C::GROUP; ++k) {
                        const int bx = g * C::GROUP + k;
                        if (TAPS == 9)
                            tc::tma_load_4d(dst + k * C::BOX_BYTES, &map_a, &full[s], 0, b0 + bx - 1, a0 - 1, img);
                        else
                            tc::tma_load_4d(dst, &map_a, &full[s], 0, b0, a0, img);
                    }
                    issued[s] = u + 1;
                }
                // the CTA's next tile into L2 while this one computes (the outer dx
                // boxes of a 3x3 tile cover the middle one)
                if (ok && tile + (int)gridDim.x < tg.total) {
                    int nimg, na0, nb0;
                    decode_tile(tg, tile + (int)gridDim.x, nimg, na0, nb0);
                    if (TAPS == 9) {
                        tc::tma_prefetch_4d(&map_a, 0, nb0 - 1, na0 - 1, nimg);
                        tc::tma_prefetch_4d(&map_a, 0, nb0 + 1, na0 - 1, nimg);
                    } else {
                        tc::tma_prefetch_4d(&map_a, 0, nb0, na0, nimg);
                    }
                }
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
            const uint32_t w_base = tc::smem_u32(sW);
            int it = 0, j = 0;
            for (int tile = blockIdx.x; ok && tile < tg.total; tile += gridDim.x, ++it) {
                const int ab = it & 1, ua = it >> 1;
                if (ua > 0 && !tc::mbar_wait(&tempty[ab], (ua - 1) & 1, abort_flag)) { ok = false; break; }
                tc::fence_after_sync();
                const uint32_t d_tmem = tmem_base + ab * N;
                // box bx holds the halo shifted by dx = bx - 1; its three dy
                // taps start 0, 1 and 2 image rows (1024 B each) into it
#pragma unroll
                for (int g = 0; g < C::SLOTS_PER_TILE; ++g, ++j) {
                    const int s = j % NS, u = j / NS;
                    if (!tc::mbar_wait(&full[s], u & 1, abort_flag)) { ok = false; break; }
                    tc::fence_after_sync();
#pragma unroll
                    for (int k = 0; k < C::GROUP; ++k) {
                        const int bx = g * C::GROUP + k;
                        const uint32_t a_base = tc::smem_u32(sA + s * C::SLOT_BYTES + k * C::BOX_BYTES);
#pragma unroll
                        for (int dy = 0; dy < (TAPS == 9 ? 3 : 1); ++dy) {
                            const int tap = TAPS == 9 ? dy * 3 + bx : 0;
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk) {
                                const uint64_t ad = tc::desc_sw128(a_base + dy * 1024 + kk * 32);
                                const uint64_t bd = tc::desc_sw128(w_base + tap * N * 128 + kk * 32);
                                tc::mma_bf16(d_tmem, ad, bd, idesc, (bx | dy | kk) ? 1u : 0u);
                            }
                        }
                    }
                    tc::mma_commit(&empty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&tfull[ab]);
            }
            if (!ok) give_up(MSF_ERR_TIMEOUT);
        }
    } else {
        // ---------------- epilogue: 4 warps, TMEM lane quarter = warp % 4
        const int q = warp & 3;
        const int row = q * 32 + lane;           // accumulator row = pixel of the tile
        // EPI_RAW32: this warp's BatchNorm moments of channels 2 lane, 2 lane + 1
        double msum[2] = {0.0, 0.0}, msq[2] = {0.0, 0.0};
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
            warp_arrive(&tempty[ab]);
            int img, a0, b0;
            decode_tile(tg, tile, img, a0, b0);
            if (epi_stores_bf16(EPI)) {
                uint32_t w[N / 2];
#pragma unroll
                for (int j = 0; j < N / 2; ++j) {
                    float lo = __uint_as_float(r[2 * j]) + sbias[2 * j];
                    float hi = __uint_as_float(r[2 * j + 1]) + sbias[2 * j + 1];
                    if (EPI == EPI_RELU) {
                        lo = fmaxf(lo, 0.0f);
                        hi = fmaxf(hi, 0.0f);
                    }
                    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
                    w[j] = *reinterpret_cast<uint32_t*>(&h);
                }
                // per-warp staging: this warp's 32 rows are 4 image rows of
                // the tile; lane 0 stores them with its own bulk group, so no
                // barrier spans more than one warp.  The previous tile's store
                // from this stage must have left shared memory first.
                uint8_t* stage = sO + q * (TILE_BYTES / 4);
                if (lane == 0) tc::tma_store_wait_read<0>();
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
            } else if (EPI == EPI_RAW32) {
                static_assert(EPI != EPI_RAW32 || N == CH, "moments are summed for 64 channels");
                const int a = a0 + row / TILE_B, b = b0 + row % TILE_B;
                const bool in = a < tg.H && b < tg.W;
                float v[N];
#pragma unroll
                for (int j = 0; j < N; ++j) v[j] = in ? __uint_as_float(r[j]) + sbias[j] : 0.0f;
                // the warp's 4 x 8 pixels are staged in its own 8 KB as two
                // boxes of 32 channels (pixel = 128-byte row, 16-byte chunks in
                // the 128-byte swizzle) and leave by two TMA stores; the staged
                // copy also gives the BatchNorm moments: lane l sums channels
                // 2l, 2l + 1 over the 32 pixels in FP32 and adds the tile's sums
                // into its FP64 moments.  The previous tile's stores must have
                // read the buffer first.
                uint8_t* tr = sM + q * (32 * 256);
                if (lane == 0) tc::tma_store_wait_read<0>();
                __syncwarp();
#pragma unroll
                for (int c = 0; c < N / 4; ++c)
                    *reinterpret_cast<float4*>(tr + (c >> 3) * 4096 + lane * 128 + (((c & 7) ^ (lane & 7)) << 4)) =
                        make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
                tc::fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) {
                    if (a0 + q * (TILE_A / 4) < tg.H) {
                        tc::tma_store_4d(&map_out, tr, 0, b0, a0 + q * (TILE_A / 4), img);
                        tc::tma_store_4d(&map_out, tr + 4096, 32, b0, a0 + q * (TILE_A / 4), img);
                    }
                    tc::tma_store_commit();
                }
                float s0 = 0.0f, s1 = 0.0f, q0 = 0.0f, q1 = 0.0f;
                const uint8_t* col = tr + (lane >> 4) * 4096 + (lane & 1) * 8;
                const int chunk = (lane & 15) >> 1;
#pragma unroll 8
                for (int rr = 0; rr < 32; ++rr) {
                    const float2 x = *reinterpret_cast<const float2*>(col + rr * 128 + ((chunk ^ (rr & 7)) << 4));
                    s0 += x.x;
                    s1 += x.y;
                    q0 = fmaf(x.x, x.x, q0);
                    q1 = fmaf(x.y, x.y, q1);
                }
                msum[0] += (double)s0;
                msum[1] += (double)s1;
                msq[0] += (double)q0;
                msq[1] += (double)q1;
            } else {
                const float R = __uint_as_float(r[0]) + sbias[0];
                const int a = a0 + row / TILE_B, b = b0 + row % TILE_B;
                if (a < tg.H && b < tg.W) {
                    if (EPI == EPI_RESID) {
                        const int t = sg.t0 + img / sg.S, s = img % sg.S;
                        const size_t idx = vol_index(sg, t, s, a, b);
                        outv[idx] = centre[idx] - R;
                    } else {
                        outv[((size_t)img * tg.H + a) * tg.W + b] = R;
                    }
                }
            }
        }
        if ((epi_stores_bf16(EPI) || EPI == EPI_RAW32) && lane == 0) tc::tma_store_wait_all();
        if (EPI == EPI_RAW32) {
            // partials [blockIdx.x * 4 + q][2][64]: sum z, sum z^2
            double* dst = moments + (size_t)(blockIdx.x * 4 + q) * 2 * CH;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                dst[2 * lane + k] = msum[k];
                dst[CH + 2 * lane + k] = msq[k];
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ---------------------------------------------------------------- fused first layer

// First layer (3x3 over the 5 frames, Eq. (14)'s 2.5D input) as one persistent
// kernel.  TMA brings each tile's five FP32 frame patches (rows a0 - 1 ..
// a0 + 4, columns b0 - 4 .. b0 + 35, zero outside the image) into a ring;
// producer warps build each pixel's 45 inputs (5 frames x 3 x 3, padded to
// K = 64, k = frame * 9 + ky * 3 + kx) as a 128-byte BF16 row in shared
// memory; one MMA warp multiplies a 128-pixel tile by the packed 64 x 64
// weights (four K16 steps); epilogue warps store relu(acc + bias) as BF16
// activations.  A tile is 4 image rows x 32 columns; tile row q is accumulator
// lanes 32q .. 32q + 31.  With four MMAs per tile the epilogue of a tile (TMEM
// load, conversion, staging, store) is a long chain, so two groups of four
// epilogue warps take alternate tiles; a warp of its own issues the patch
// copies, so that no producer waits for the others before its next tile.
constexpr int C1_ROWS = 4, C1_COLS = 32;
constexpr int C1_EPI_GROUPS = 2;
constexpr int C1_LOADER_WARP = 5;
constexpr int C1_THREADS = 32 * (2 + 4 + 4 * C1_EPI_GROUPS);   // warp 0 MMA, 1-4 producers, 5 loader, then the epilogue

constexpr int C1_PCOLS = C1_COLS + 8, C1_PROWS = C1_ROWS + 2;   // frame patch: 40 x 6 FP32

struct C1Cfg {
    static constexpr int NS = 4;                              // A-operand stages
    static constexpr int NF = 4;                              // frame-patch stages
    static constexpr int NB = 2 * C1_EPI_GROUPS;              // TMEM accumulators, 64 columns each
    static constexpr int TMEM_ALLOC = 256;
    static constexpr int STAGE_BYTES = TILE_BYTES;            // 128 rows x 128 B
    static constexpr int PATCH_BYTES = C1_PCOLS * C1_PROWS * 4;   // 960 B copied per patch
    static constexpr int PATCH_STRIDE = 1024;                 // patches 128-byte aligned in shared memory
    static constexpr int F_BYTES = FRAMES * PATCH_STRIDE;     // one tile's five patches
    static constexpr int W_BYTES = CH * 128;
    static constexpr int O_BYTES = C1_EPI_GROUPS * TILE_BYTES;   // one staging tile per epilogue group
    static constexpr int BAR_BYTES = 512;
    static constexpr int SMEM = 1024 + NS * STAGE_BYTES + W_BYTES + O_BYTES + NF * F_BYTES + BAR_BYTES;
    static_assert((2 * NS + 2 * NF + 2 * NB + 1) * 8 + 8 <= 256, "barrier block overflows into the bias");
    static_assert(F_BYTES % 128 == 0, "frame stages must stay 128-byte aligned");
    static_assert(NB * CH <= TMEM_ALLOC, "accumulators exceed the TMEM allocation");
};

__device__ __forceinline__ void decode_c1_tile(const TileGeom& tg, int tile, int& img, int& a0, int& b0) {
    const int per = tg.tiles_a * tg.tiles_b;
    img = tile / per;
    const int r = tile - img * per;
    a0 = (r / tg.tiles_b) * C1_ROWS;
    b0 = (r % tg.tiles_b) * C1_COLS;
}

// PATCH = false (image width not a multiple of 4, which the frame tensor map
// cannot stride) reads the frames with plain loads instead of the patch ring.
template <bool PATCH>
__global__ void __launch_bounds__(C1_THREADS, 1)
conv1_fused_kernel(const __grid_constant__ CUtensorMap map_w, const __grid_constant__ CUtensorMap map_out,
                   const __grid_constant__ CUtensorMap map_f, const float* __restrict__ bias, PackFrames pf,
                   SliceGeom g, TileGeom tg, int* __restrict__ err) {
    using C = C1Cfg;
    constexpr int NS = C::NS, NF = C::NF;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sW = sA + NS * C::STAGE_BYTES;
    uint8_t* sO = sW + C::W_BYTES;
    uint8_t* sF = sO + C::O_BYTES;
    uint64_t* bars = (uint64_t*)(sF + NF * C::F_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = bars + NS;
    uint64_t* ffull = bars + 2 * NS;
    uint64_t* fempty = ffull + NF;   // all four producer warps have read a patch stage
    uint64_t* tfull = fempty + NF;
    uint64_t* tempty = tfull + C::NB;
    uint64_t* wbar = tempty + C::NB;
    uint32_t* tmem_slot = (uint32_t*)(wbar + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    float* sbias = (float*)((uint8_t*)bars + 256);
    if (threadIdx.x < CH) sbias[threadIdx.x] = bias[threadIdx.x];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        // full, fempty: one arrival per producer warp; tempty: per epilogue warp
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full[s], 4);
            tc::mbar_init(&empty[s], 1);
        }
        for (int f = 0; f < NF; ++f) {
            tc::mbar_init(&ffull[f], 1);
            tc::mbar_init(&fempty[f], 4);
        }
        for (int b = 0; b < C::NB; ++b) {
            tc::mbar_init(&tfull[b], 1);
            tc::mbar_init(&tempty[b], 4);
        }
        tc::mbar_init(wbar, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tmem_slot, C::TMEM_ALLOC);
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
            // ---------------- weights, then the MMA issuer
            constexpr uint32_t idesc = tc::idesc_bf16<128, CH>();
            tc::mbar_expect_tx(wbar, C::W_BYTES);
            tc::tma_load_2d(sW, &map_w, wbar, 0, 0);
            bool ok = tc::mbar_wait(wbar, 0, abort_flag);
            tc::fence_after_sync();
            const uint32_t w_base = tc::smem_u32(sW);
            int it = 0;
            for (int tile = blockIdx.x; ok && tile < tg.total; tile += gridDim.x, ++it) {
                const int s = it % NS, u = it / NS, ab = it % C::NB, ua = it / C::NB;
                if (ua > 0 && !tc::mbar_wait(&tempty[ab], (ua - 1) & 1, abort_flag)) { ok = false; break; }
                if (!tc::mbar_wait(&full[s], u & 1, abort_flag)) { ok = false; break; }
                tc::fence_after_sync();
                const uint32_t a_base = tc::smem_u32(sA + s * C::STAGE_BYTES);
#pragma unroll
                for (int kk = 0; kk < 4; ++kk)
                    tc::mma_bf16(tmem_base + ab * CH, tc::desc_sw128(a_base + kk * 32), tc::desc_sw128(w_base + kk * 32),
                                 idesc, kk ? 1u : 0u);
                tc::mma_commit(&empty[s]);
                tc::mma_commit(&tfull[ab]);
            }
            if (!ok) give_up(MSF_ERR_TIMEOUT);
        }
    } else if (warp == C1_LOADER_WARP) {
        // ---------------- frame-patch copies: tile it into patch stage it % NF,
        // once all four producer warps are done with that stage's previous tile
        if (PATCH && lane == 0) {
            int issued[NF];
            for (int f = 0; f < NF; ++f) issued[f] = 0;
            bool ok = true;
            int it = 0;
            for (int tile = blockIdx.x; tile < tg.total; tile += gridDim.x, ++it) {
                const int fs = it % NF, fu = it / NF;
                if (fu > 0 && !tc::mbar_wait(&fempty[fs], (fu - 1) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                int img, a0, b0;
                decode_c1_tile(tg, tile, img, a0, b0);
                const int t = g.t0 + img / g.S, sl = img % g.S;
                tc::fence_proxy_async_smem();
                tc::mbar_expect_tx(&ffull[fs], FRAMES * C::PATCH_BYTES);
#pragma unroll
                for (int c = 0; c < FRAMES; ++c) {
                    const int tc_ = min(max(t + c - 2, 0), g.nt - 1);
                    tc::tma_load_4d(sF + fs * C::F_BYTES + c * C::PATCH_STRIDE, &map_f, &ffull[fs], b0 - 4, a0 - 1,
                                    sl, tc_ - pf.first);
                }
                issued[fs] = fu + 1;
            }
            if (!ok) {
                give_up(MSF_ERR_TIMEOUT);
                // let the copies already issued land before the CTA exits
                for (int f = 0; f < NF; ++f)
                    if (issued[f] > 0) tc::mbar_wait(&ffull[f], (issued[f] - 1) & 1, nullptr, 100000000ull);
            }
        }
    } else if (warp <= 4) {
        // ---------------- producers: warp 1 + r builds tile row r
        const int r = warp - 1;
        int it = 0;
        for (int tile = blockIdx.x; tile < tg.total; tile += gridDim.x, ++it) {
            const int s = it % NS, u = it / NS, fs = it % NF, fu = it / NF;
            if ((PATCH && !tc::mbar_wait(&ffull[fs], fu & 1, abort_flag)) ||
                (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1, abort_flag))) {
                give_up(MSF_ERR_TIMEOUT);
                break;
            }
            uint32_t w[32];
            if (PATCH) {
                // pixel (a0 + r, b0 + lane): patch row r + ky, column lane + kx + 3
                const float* patch = reinterpret_cast<const float*>(sF + fs * C::F_BYTES) + r * C1_PCOLS + lane + 3;
                auto tap = [&](int k) {
                    return k < FRAMES * 9
                               ? patch[(k / 9) * (C::PATCH_STRIDE / 4) + ((k % 9) / 3) * C1_PCOLS + (k % 3)]
                               : 0.0f;
                };
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    __nv_bfloat162 hv = __floats2bfloat162_rn(tap(2 * i), tap(2 * i + 1));
                    w[i] = *reinterpret_cast<uint32_t*>(&hv);
                }
            } else {
                float v[FRAMES * 9];
                int img, a0, b0;
                decode_c1_tile(tg, tile, img, a0, b0);
                const int a = a0 + r, b = b0 + lane;
#pragma unroll
                for (int k = 0; k < FRAMES * 9; ++k) v[k] = 0.0f;
                if (a < g.H && b < g.W) {
                    const int t = g.t0 + img / g.S, sl = img % g.S;
                    const size_t off = ((size_t)sl * g.H + a) * g.W + b;
#pragma unroll
                    for (int c = 0; c < FRAMES; ++c) {
                        const int tc_ = min(max(t + c - 2, 0), g.nt - 1);
                        const float* f = pf.f[tc_ - pf.first] + off;
#pragma unroll
                        for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                            for (int kx = 0; kx < 3; ++kx)
                                if (a + ky - 1 >= 0 && a + ky - 1 < g.H && b + kx - 1 >= 0 && b + kx - 1 < g.W)
                                    v[c * 9 + ky * 3 + kx] = __ldg(f + (ky - 1) * g.W + (kx - 1));
                    }
                }
#pragma unroll
                for (int i = 0; i < 32; ++i) {
                    const float lo = 2 * i < FRAMES * 9 ? v[2 * i] : 0.0f;
                    const float hi = 2 * i + 1 < FRAMES * 9 ? v[2 * i + 1] : 0.0f;
                    __nv_bfloat162 hv = __floats2bfloat162_rn(lo, hi);
                    w[i] = *reinterpret_cast<uint32_t*>(&hv);
                }
            }
            const int m = r * 32 + lane;     // accumulator row of this pixel
            uint8_t* row = sA + s * C::STAGE_BYTES + m * 128;
#pragma unroll
            for (int c = 0; c < 8; ++c)
                *reinterpret_cast<uint4*>(row + ((c ^ (m & 7)) << 4)) =
                    make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                tc::mbar_arrive(&full[s]);
                if (PATCH) tc::mbar_arrive(&fempty[fs]);   // this producer warp is done with patch stage fs
            }
        }
    } else {
        // ---------------- epilogue: group e = (warp - 6) / 4 takes tiles
        // it = e, e + C1_EPI_GROUPS, ...; TMEM lane quarter q = warp % 4 = tile row q
        const int q = warp & 3, grp = (warp - C1_LOADER_WARP - 1) / 4;
        int it = grp;
        for (int tile = blockIdx.x + grp * gridDim.x; tile < tg.total;
             tile += C1_EPI_GROUPS * gridDim.x, it += C1_EPI_GROUPS) {
            const int ab = it % C::NB, ua = it / C::NB;
            if (!tc::mbar_wait(&tfull[ab], ua & 1, abort_flag)) {
                give_up(MSF_ERR_TIMEOUT);
                break;
            }
            tc::fence_after_sync();
            uint32_t r[CH];
            const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + ab * CH;
#pragma unroll
            for (int c = 0; c < CH / 16; ++c) tc::tmem_ld16(taddr + c * 16, r + c * 16);
            tc::tmem_ld_wait();
            tc::fence_before_sync();
            warp_arrive(&tempty[ab]);
            int img, a0, b0;
            decode_c1_tile(tg, tile, img, a0, b0);
            uint32_t w[CH / 2];
#pragma unroll
            for (int k = 0; k < CH / 4; ++k) {
                const float4 bv = reinterpret_cast<const float4*>(sbias)[k];
                const float v0 = fmaxf(__uint_as_float(r[4 * k]) + bv.x, 0.0f);
                const float v1 = fmaxf(__uint_as_float(r[4 * k + 1]) + bv.y, 0.0f);
                const float v2 = fmaxf(__uint_as_float(r[4 * k + 2]) + bv.z, 0.0f);
                const float v3 = fmaxf(__uint_as_float(r[4 * k + 3]) + bv.w, 0.0f);
                __nv_bfloat162 h0 = __floats2bfloat162_rn(v0, v1), h1 = __floats2bfloat162_rn(v2, v3);
                w[2 * k] = *reinterpret_cast<uint32_t*>(&h0);
                w[2 * k + 1] = *reinterpret_cast<uint32_t*>(&h1);
            }
            uint8_t* stage = sO + grp * TILE_BYTES + q * (TILE_BYTES / 4);
            if (lane == 0) tc::tma_store_wait_read<0>();
            __syncwarp();
#pragma unroll
            for (int c = 0; c < 8; ++c)
                *reinterpret_cast<uint4*>(stage + lane * 128 + ((c ^ (lane & 7)) << 4)) =
                    make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
            tc::fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) {
                if (a0 + q < tg.H) tc::tma_store_4d(&map_out, stage, 0, b0, a0 + q, img);
                tc::tma_store_commit();
            }
        }
        if (lane == 0) tc::tma_store_wait_all();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base, C::TMEM_ALLOC);
    }
}

// ---------------------------------------------------------------- row-pair 3x3 conv

// A 3x3 64 -> 64 layer whose tile puts 16 row PAIRS x 8 columns (256 output
// pixels) on the 128 accumulator rows: row m = 8 i + j holds pixel
// (a0 + 2i, b0 + j) in accumulator columns 0-63 (group 0) and pixel
// (a0 + 2i + 1, b0 + j) in columns 64-127 (group 1).  Input row a0 + 2i + s,
// s = -1 .. 2, reaches group 0 through kernel row dy = s and group 1 through
// dy = s - 1, so one A slice feeds both groups with B = [W(dy = s); W(dy = s-1)]
// (N = 128; N = 64 at s = -1 and s = 2 where one group has no tap).  The
// tensor math is the same as in the 16 x 8 tile, issued as 12 A slices x 4
// K-steps per 256 pixels instead of 18 x 4: fewer MMAs and A-slice reads.
// Rows of one parity come from one TMA box: the activation maps view the
// image rows as (H / 2 pairs) x (2 parities), which needs an even H.
constexpr int PAIR_ROWS = 16;                                 // row pairs per tile
constexpr int PBOX_BYTES = (PAIR_ROWS + 1) * TILE_B * 128;    // 17408: 17 pair rows of one parity

struct PairCfg {
    // stages; one stage = one parity x 3 dx boxes.  Six one-box stages (the
    // same shared memory, loads up to five boxes ahead) measured 25% slower on
    // GB300 at 384 x 384 (4.04 against 3.24 ms per 384^3 layer).
    static constexpr int NS = 2;
    static constexpr int STAGE_BYTES = 3 * PBOX_BYTES;
    static constexpr int W_BYTES = 9 * CH * 128;
    static constexpr int W10_BYTES = 16 * 128;                // output layer: 16 rows (9 taps) x 64 channels
    static constexpr int O_BYTES = 2 * TILE_BYTES;            // staging of group 0 and group 1
    static constexpr int BAR_BYTES = 512;                     // barriers, TMEM slot, abort flag (256 B), bias (256 B)
    static constexpr int SMEM = 1024 + NS * STAGE_BYTES + W_BYTES + W10_BYTES + O_BYTES + BAR_BYTES;
    static constexpr int NACC = 3;                            // TMEM accumulators (tiles in flight)
    static_assert((2 * NS + 2 * NACC + 3) * 8 + 8 <= 256, "barrier block overflows into the bias");
    static_assert(SMEM <= 232448, "more dynamic shared memory than a CTA may have");
};

__device__ __forceinline__ void decode_pair_tile(const TileGeom& tg, int tile, int& img, int& a0, int& b0) {
    const int per = tg.tiles_a * tg.tiles_b;
    img = tile / per;
    const int r = tile - img * per;
    a0 = (r / tg.tiles_b) * (2 * PAIR_ROWS);
    b0 = (r % tg.tiles_b) * TILE_B;
}

// EPI_RELU stores relu(acc + bias) as BF16 activations.  EPI_PART is the
// network's last 64 -> 64 layer fused with the 64 -> 1 output layer: the BF16
// activations are staged in shared memory only, where eight M128 N16 K16 MMAs
// per tile multiply them by the output layer's weights arranged as one tap per
// row (map_w10: [9 taps][64], rows 9-15 zero-filled).  Column t of that product
// is P_t(p) = sum_c w10[t][c] act(p, c), written to part[t * plane + p];
// resid_stencil_kernel then forms R(p) = bias + sum_t P_t(p + offset_t).
template <int EPI, class Src>
__device__ __forceinline__ void conv_pair_body(const Src& src, const CUtensorMap* map_w, const CUtensorMap* map_w10,
                                               const float* __restrict__ bias, int* __restrict__ err) {
    static_assert(EPI == EPI_RELU || EPI == EPI_PART, "row-pair conv: ReLU layers only");
    constexpr bool FUSED = EPI == EPI_PART;
    using C = PairCfg;
    constexpr int NS = C::NS;
    constexpr uint32_t WBLK = CH * 128;   // one tap's 64 x 64 BF16 weights
    // NACC accumulators of 128 columns (the MMA warp runs up to NACC - 1 tiles
    // ahead of the epilogue), then, for EPI_PART, the per-tap sums (2 x 16)
    constexpr int NACC = C::NACC;
    constexpr int TMEM_PAIR = 4 * TMEM_COLS;
    constexpr uint32_t P_COL = NACC * 2 * CH;
    static_assert(P_COL + 2 * 16 <= TMEM_PAIR, "TMEM columns");
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sW = sA + NS * C::STAGE_BYTES;
    uint8_t* sW10 = sW + C::W_BYTES;
    uint8_t* sO = sW10 + C::W10_BYTES;
    uint64_t* bars = (uint64_t*)(sO + C::O_BYTES);
    uint64_t* full = bars;
    uint64_t* empty = full + NS;
    uint64_t* tfull = empty + NS;
    uint64_t* tempty = tfull + NACC;
    uint64_t* wbar = tempty + NACC;
    uint64_t* staged = wbar + 1;     // EPI_PART: activations of a tile staged (one arrival per epilogue warp)
    uint64_t* pfull = staged + 1;    // EPI_PART: per-tap sums of a tile in TMEM
    uint32_t* tmem_slot = (uint32_t*)(pfull + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
    float* sbias = (float*)((uint8_t*)bars + 256);
    if (threadIdx.x < CH) sbias[threadIdx.x] = bias[threadIdx.x];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < NS; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < NACC; ++b) {
            tc::mbar_init(&tfull[b], 1);
            tc::mbar_init(&tempty[b], 4);     // one arrival per epilogue warp
        }
        tc::mbar_init(wbar, 1);
        tc::mbar_init(staged, 4);
        tc::mbar_init(pfull, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, TMEM_PAIR);
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
            // ---------------- producer: weights once, then two parity stages per tile
            int issued[NS];
            for (int s = 0; s < NS; ++s) issued[s] = 0;
            // per dx, the blocks W(dy = +1), W(0), W(-1) back to back, so that
            // [W(s); W(s - 1)] is one contiguous 128-row B operand
            tc::mbar_expect_tx(wbar, C::W_BYTES + (FUSED ? C::W10_BYTES : 0));
            for (int dx = 0; dx < 3; ++dx)
                for (int d = 0; d < 3; ++d)
                    tc::tma_load_2d(sW + (dx * 3 + d) * WBLK, map_w, wbar, 0, ((2 - d) * 3 + dx) * CH);
            if (FUSED) tc::tma_load_2d(sW10, map_w10, wbar, 0, 0);
            int j = 0;
            bool ok = true;
            typename Src::Cursor cur;
            for (int tile = blockIdx.x; ok && tile < src.total(); tile += gridDim.x) {
                int img, a0, b0;
                const int job = src.locate(tile, cur);
                decode_pair_tile(src.geom(job), cur.local, img, a0, b0);
#pragma unroll
                for (int p = 0; p < 2; ++p, ++j) {
                    const int s = j % NS, u = j / NS;
                    if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1, abort_flag)) {
                        ok = false;
                        break;
                    }
                    uint8_t* dst = sA + s * C::STAGE_BYTES;
                    tc::mbar_expect_tx(&full[s], C::STAGE_BYTES);
                    // parity p: box entry k is image row a0 - p + 2k (zero-filled outside the image)
#pragma unroll
                    for (int bx = 0; bx < 3; ++bx)
                        tc::tma_load_5d(dst + bx * PBOX_BYTES, src.map_a(job), &full[s], 0, b0 + bx - 1, p, a0 / 2 - p, img);
                    issued[s] = u + 1;
                }
                // the next tile of this CTA into L2 while this one computes, so that its
                // loads, issued once a stage frees, do not wait for DRAM (the outer dx
                // boxes cover the middle one)
                const int nxt = tile + (int)gridDim.x;
                if (ok && nxt < src.total()) {
                    typename Src::Cursor pc = cur;
                    const int pjob = src.locate(nxt, pc);
                    int pimg, pa0, pb0;
                    decode_pair_tile(src.geom(pjob), pc.local, pimg, pa0, pb0);
#pragma unroll
                    for (int p = 0; p < 2; ++p)
#pragma unroll
                        for (int bx = 0; bx < 3; bx += 2)
                            tc::tma_prefetch_5d(src.map_a(pjob), 0, pb0 + bx - 1, p, pa0 / 2 - p, pimg);
                }
            }
            if (!ok) {
                give_up(MSF_ERR_TIMEOUT);
                for (int s = 0; s < NS; ++s)
                    if (issued[s] > 0) tc::mbar_wait(&full[s], (issued[s] - 1) & 1, nullptr, 100000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer
            constexpr uint32_t id128 = tc::idesc_bf16<128, 128>();
            constexpr uint32_t id64 = tc::idesc_bf16<128, 64>();
            constexpr uint32_t id16 = tc::idesc_bf16<128, 16>();
            bool ok = tc::mbar_wait(wbar, 0, abort_flag);
            tc::fence_after_sync();
            const uint32_t w_base = tc::smem_u32(sW);
            // EPI_PART: the per-tap sums of tile k, once its activations are staged
            auto part_mmas = [&](int k) {
                if (!tc::mbar_wait(staged, k & 1, abort_flag)) return false;
                tc::fence_after_sync();
#pragma unroll
                for (int g = 0; g < 2; ++g)
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk)
                        tc::mma_bf16(tmem_base + P_COL + g * 16, tc::desc_sw128(tc::smem_u32(sO + g * TILE_BYTES) + kk * 32),
                                     tc::desc_sw128(tc::smem_u32(sW10) + kk * 32), id16, kk ? 1u : 0u);
                tc::mma_commit(pfull);
                return true;
            };
            int it = 0, j = 0;
            for (int tile = blockIdx.x; ok && tile < src.total(); tile += gridDim.x, ++it) {
                const int ab = it % NACC, ua = it / NACC;
                if (ua > 0 && !tc::mbar_wait(&tempty[ab], (ua - 1) & 1, abort_flag)) { ok = false; break; }
                tc::fence_after_sync();
                const uint32_t d = tmem_base + ab * 2 * CH;
#pragma unroll
                for (int p = 0; p < 2; ++p, ++j) {
                    const int s = j % NS, u = j / NS;
                    if (!tc::mbar_wait(&full[s], u & 1, abort_flag)) { ok = false; break; }
                    tc::fence_after_sync();
#pragma unroll
                    for (int bx = 0; bx < 3; ++bx) {
                        const uint32_t a = tc::smem_u32(sA + s * C::STAGE_BYTES + bx * PBOX_BYTES);
                        const uint32_t wb = w_base + bx * 3 * WBLK;   // W(+1, dx) of this dx
                        if (p == 0) {
                            // s = 0: group 0 by dy 0, group 1 by dy -1; the first
                            // of these MMAs initialises all 128 columns
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                tc::mma_bf16(d, tc::desc_sw128(a + kk * 32), tc::desc_sw128(wb + WBLK + kk * 32), id128,
                                             (bx | kk) ? 1u : 0u);
                            // s = 2: group 1 by dy +1
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                tc::mma_bf16(d + CH, tc::desc_sw128(a + 1024 + kk * 32), tc::desc_sw128(wb + kk * 32),
                                             id64, 1u);
                        } else {
                            // s = -1: group 0 by dy -1
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                tc::mma_bf16(d, tc::desc_sw128(a + kk * 32), tc::desc_sw128(wb + 2 * WBLK + kk * 32),
                                             id64, 1u);
                            // s = +1: group 0 by dy +1, group 1 by dy 0
#pragma unroll
                            for (int kk = 0; kk < 4; ++kk)
                                tc::mma_bf16(d, tc::desc_sw128(a + 1024 + kk * 32), tc::desc_sw128(wb + kk * 32), id128,
                                             1u);
                        }
                    }
                    tc::mma_commit(&empty[s]);
                }
                if (!ok) break;
                tc::mma_commit(&tfull[ab]);
                // the previous tile's per-tap sums queue behind this tile's MMAs
                if (FUSED && it > 0 && !part_mmas(it - 1)) { ok = false; break; }
            }
            if (FUSED && ok && it > 0 && !part_mmas(it - 1)) ok = false;
            if (!ok) give_up(MSF_ERR_TIMEOUT);
        }
    } else {
        // ---------------- epilogue: 4 warps, TMEM lane quarter q = warp % 4
        // holds row pairs 4q .. 4q + 3 of the tile
        const int q = warp & 3;
        int it = 0;
        typename Src::Cursor cur;
        for (int tile = blockIdx.x; tile < src.total(); tile += gridDim.x, ++it) {
            const int ab = it % NACC, ua = it / NACC;
            if (!tc::mbar_wait(&tfull[ab], ua & 1, abort_flag)) {
                give_up(MSF_ERR_TIMEOUT);
                break;
            }
            tc::fence_after_sync();
            int img, a0, b0;
            const int job = src.locate(tile, cur);
            const TileGeom& tg = src.geom(job);
            decode_pair_tile(tg, cur.local, img, a0, b0);
#pragma unroll
            for (int g = 0; g < 2; ++g) {
                uint32_t r[CH];
                const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + ab * 2 * CH + g * CH;
#pragma unroll
                for (int c = 0; c < CH / 16; ++c) tc::tmem_ld16(taddr + c * 16, r + c * 16);
                tc::tmem_ld_wait();
                if (g == 1) {
                    tc::fence_before_sync();
                    warp_arrive(&tempty[ab]);
                }
                uint32_t w[CH / 2];
#pragma unroll
                for (int k = 0; k < CH / 4; ++k) {
                    const float4 bv = reinterpret_cast<const float4*>(sbias)[k];
                    const float v0 = fmaxf(__uint_as_float(r[4 * k]) + bv.x, 0.0f);
                    const float v1 = fmaxf(__uint_as_float(r[4 * k + 1]) + bv.y, 0.0f);
                    const float v2 = fmaxf(__uint_as_float(r[4 * k + 2]) + bv.z, 0.0f);
                    const float v3 = fmaxf(__uint_as_float(r[4 * k + 3]) + bv.w, 0.0f);
                    __nv_bfloat162 h0 = __floats2bfloat162_rn(v0, v1), h1 = __floats2bfloat162_rn(v2, v3);
                    w[2 * k] = *reinterpret_cast<uint32_t*>(&h0);
                    w[2 * k + 1] = *reinterpret_cast<uint32_t*>(&h1);
                }
                // group g occupies 128 consecutive 128-byte rows (warp q: rows
                // 32q .. 32q + 31), in the 128-byte swizzle shared by the TMA
                // store and the MMA operand descriptor
                uint8_t* stage = sO + g * TILE_BYTES + q * (TILE_BYTES / 4);
                if (!FUSED) {
                    // the previous tile's store from this buffer must have left it
                    if (lane == 0) tc::tma_store_wait_read<1>();
                    __syncwarp();
                }
#pragma unroll
                for (int c = 0; c < 8; ++c)
                    *reinterpret_cast<uint4*>(stage + lane * 128 + ((c ^ (lane & 7)) << 4)) =
                        make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
                tc::fence_proxy_async_smem();
                if (!FUSED) {
                    __syncwarp();
                    if (lane == 0) {
                        // group g of this warp: 4 pair rows x 8 pixels, one bulk store
                        const int pr = a0 / 2 + 4 * q;
                        if (pr < tg.H / 2) tc::tma_store_5d(src.map_out(job), stage, 0, b0, g, pr, img);
                        tc::tma_store_commit();
                    }
                }
            }
            if (FUSED) {
                // hand the staged activations to the MMA warp, then write the
                // per-tap sums it returns; the staging is free again once they are
                tc::fence_before_sync();
                warp_arrive(staged);
                if (!tc::mbar_wait(pfull, it & 1, abort_flag)) {
                    give_up(MSF_ERR_TIMEOUT);
                    break;
                }
                tc::fence_after_sync();
                uint32_t pv[2][16];
#pragma unroll
                for (int g = 0; g < 2; ++g)
                    tc::tmem_ld16(tmem_base + ((uint32_t)(q * 32) << 16) + P_COL + g * 16, pv[g]);
                tc::tmem_ld_wait();
#pragma unroll
                for (int g = 0; g < 2; ++g) {
                    const int a = a0 + 2 * (4 * q + (lane >> 3)) + g, b = b0 + (lane & 7);
                    if (a < tg.H && b < tg.W) {
                        float* dst = src.part(job) + ((size_t)img * tg.H + a) * tg.W + b;
                        const long long plane = src.plane(job);
#pragma unroll
                        for (int t = 0; t < 9; ++t) dst[(size_t)t * plane] = __uint_as_float(pv[g][t]);
                    }
                }
            }
        }
        if (!FUSED && lane == 0) tc::tma_store_wait_all();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base, TMEM_PAIR);
    }
}

// Tile sources of the row-pair layer.  One problem: the launch's own maps and
// geometry.  Several problems (one persistent launch over a batch): a work list
// of jobs, each with its activation maps (kernel parameters, so TMA reads them
// from the parameter space), its tile geometry and the first global tile index;
// a CTA walks the global tiles blockIdx.x, blockIdx.x + gridDim.x, ... and finds
// each tile's job by advancing a cursor (its tiles increase monotonically).
struct PairSingle {
    const CUtensorMap* a;
    const CUtensorMap* out;
    TileGeom tg;
    float* part_;
    long long plane_;
    struct Cursor { int local = 0; };
    __device__ __forceinline__ int total() const { return tg.total; }
    __device__ __forceinline__ int locate(int tile, Cursor& c) const { c.local = tile; return 0; }
    __device__ __forceinline__ const TileGeom& geom(int) const { return tg; }
    __device__ __forceinline__ const CUtensorMap* map_a(int) const { return a; }
    __device__ __forceinline__ const CUtensorMap* map_out(int) const { return out; }
    __device__ __forceinline__ float* part(int) const { return part_; }
    __device__ __forceinline__ long long plane(int) const { return plane_; }
};

constexpr int PAIR_MAX_JOBS = 16;

struct PairJob {
    CUtensorMap a;       // activations in, (pairs x parity) view with the 17-pair box
    CUtensorMap out;     // activations out, 4-pair box (EPI_RELU)
    TileGeom tg;         // row-pair tiles of this problem's images
    int tile0;           // first global tile of this job
    float* part;         // EPI_PART: per-tap planes of this problem
    long long plane;
};

struct PairJobs {
    PairJob job[PAIR_MAX_JOBS];
    int n, total;
};

struct PairMulti {
    const PairJobs* J;
    struct Cursor { int job = 0, local = 0; };
    __device__ __forceinline__ int total() const { return J->total; }
    __device__ __forceinline__ int locate(int tile, Cursor& c) const {
        while (c.job + 1 < J->n && tile >= J->job[c.job + 1].tile0) ++c.job;
        c.local = tile - J->job[c.job].tile0;
        return c.job;
    }
    __device__ __forceinline__ const TileGeom& geom(int j) const { return J->job[j].tg; }
    __device__ __forceinline__ const CUtensorMap* map_a(int j) const { return &J->job[j].a; }
    __device__ __forceinline__ const CUtensorMap* map_out(int j) const { return &J->job[j].out; }
    __device__ __forceinline__ float* part(int j) const { return J->job[j].part; }
    __device__ __forceinline__ long long plane(int j) const { return J->job[j].plane; }
};

template <int EPI>
__global__ void __launch_bounds__(THREADS, 1)
conv_pair_kernel(const __grid_constant__ CUtensorMap map_a, const __grid_constant__ CUtensorMap map_w,
                 const __grid_constant__ CUtensorMap map_out, const __grid_constant__ CUtensorMap map_w10,
                 const float* __restrict__ bias, TileGeom tg, int* __restrict__ err, float* __restrict__ part,
                 long long plane) {
    PairSingle src{&map_a, &map_out, tg, part, plane};
    conv_pair_body<EPI>(src, &map_w, &map_w10, bias, err);
}

// The same layer over a batch of problems in one persistent launch (shared
// weights and bias).
template <int EPI>
__global__ void __launch_bounds__(THREADS, 1)
conv_pair_multi_kernel(const __grid_constant__ PairJobs jobs, const __grid_constant__ CUtensorMap map_w,
                       const __grid_constant__ CUtensorMap map_w10, const float* __restrict__ bias,
                       int* __restrict__ err) {
    PairMulti src{&jobs};
    conv_pair_body<EPI>(src, &map_w, &map_w10, bias, err);
}

// Output layer from the per-tap planes of EPI_PART:
// R(a, b) = bias + sum_{dy,dx} P_{(dy+1)*3+dx+1}(a + dy, b + dx) over taps inside
// the image (the layer's zero padding), written as centre - R in volume order.
// A block covers 32 (u) x 32 (b) outputs of one frame: u is the image row a
// (xy-t, zx-t) or the slice s (yz-t), and `w` the remaining index.  The planes
// are read along b; the volume is contiguous along b for xy-t, along s for
// yz-t and along a for zx-t, so the last two write through a shared-memory
// transpose.
template <int ORIENT>
__global__ void __launch_bounds__(256) resid_stencil_kernel(const float* __restrict__ part, long long plane,
                                                            const float* __restrict__ bias, SliceGeom sg,
                                                            const float* __restrict__ centre, float* __restrict__ outv) {
    __shared__ float tile[32][33];
    const int H = sg.H, W = sg.W, S = sg.S;
    const int U = ORIENT == 1 ? S : H, NW = ORIENT == 1 ? H : S;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int b0 = blockIdx.x * 32, u0 = blockIdx.y * 32;
    const float b10 = bias[0];
    for (int z = blockIdx.z; z < sg.nframes * NW; z += gridDim.z) {
        const int f = z / NW, w = z % NW;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int u = u0 + ty + 8 * k, b = b0 + tx;
            if (u >= U || b >= W) continue;
            const int a = ORIENT == 1 ? w : u, s = ORIENT == 1 ? u : w;
            const long long p = ((long long)(f * S + s) * H + a) * W + b;
            float R = 0.0f;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy) {
                if (a + dy < 0 || a + dy >= H) continue;
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if (b + dx < 0 || b + dx >= W) continue;
                    R += __ldg(part + (size_t)((dy + 1) * 3 + dx + 1) * plane + p + (long long)dy * W + dx);
                }
            }
            R += b10;
            if (ORIENT == 0) {
                const size_t idx = vol_index(sg, sg.t0 + f, s, a, b);
                outv[idx] = centre[idx] - R;
            } else {
                tile[ty + 8 * k][tx] = R;
            }
        }
        if (ORIENT != 0) {
            __syncthreads();
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int u = u0 + tx, b = b0 + ty + 8 * k;
                if (u >= U || b >= W) continue;
                const int a = ORIENT == 1 ? w : u, s = ORIENT == 1 ? u : w;
                const size_t idx = vol_index(sg, sg.t0 + f, s, a, b);
                outv[idx] = centre[idx] - tile[tx][ty + 8 * k];
            }
            __syncthreads();
        }
    }
}

template <int ORIENT>
static void launch_stencil(const float* part, long long plane, const float* bias, const SliceGeom& sg,
                           const float* centre, float* outv, cudaStream_t st) {
    const int U = ORIENT == 1 ? sg.S : sg.H, NW = ORIENT == 1 ? sg.H : sg.S;
    const int nz = sg.nframes * NW;
    const dim3 grid((unsigned)((sg.W + 31) / 32), (unsigned)((U + 31) / 32), (unsigned)(nz < 65535 ? nz : 65535));
    resid_stencil_kernel<ORIENT><<<grid, dim3(32, 8), 0, st>>>(part, plane, bias, sg, centre, outv);
}

// ---------------------------------------------------------------- tcgen05 weight gradients (training)

// Weight gradients of a 64 -> 64 3x3 layer on the tensor cores:
//   dW[tap][co][ci] = sum_p dz[p][co] act[p + off(tap)][ci]
// as D[(tap, ci)][co] += A[(tap, ci)][p] B[p][co] over pixel K-steps of 16.
// Both operands are MN-major: the 128-byte rows of the TMA boxes are pixels
// (K) holding 64 channels (M or N), exactly as the forward convolution loads
// them.  A tile is 16 x 8 pixels; its act halo comes in three boxes (columns
// shifted by dx = -1, 0, +1, 18 rows each) and tap (dy, dx)'s window of K-step
// k (tile rows 2k, 2k+1) starts (2k + dy + 1) * 1024 bytes into box dx + 1.
// Two taps share one M = 128 MMA (the second 64 rows of A start the address
// difference of their windows further: the descriptor's leading byte offset),
// so each K-step is five MMAs of 128 x 64 x 16; the ninth tap is paired with
// tap 7 again and that half of the result is dropped.  Every CTA accumulates
// its tiles (a fixed round-robin sequence) in TMEM and writes one partial
// dW[9][64][64]; the partials are summed over CTAs in a fixed order.
constexpr int WG_STAGES = 2;
constexpr int WG_STAGE_BYTES = 3 * HALO_BYTES + TILE_BYTES;   // act boxes dx = -1, 0, +1, then dz
constexpr int WG_SLACK = 40960;      // unused tail: keeps every descriptor reach inside the CTA's allocation
constexpr int WG_SMEM = 1024 + WG_STAGES * WG_STAGE_BYTES + WG_SLACK + 256;
constexpr int WG_TMEM_COLS = 512;    // five 64-column accumulators
constexpr int WG_MAX_CTAS = 256;
static_assert(WG_SMEM <= 232448, "more dynamic shared memory than a CTA may have");

__host__ __device__ constexpr int wg_lo(int g) { return g == 0 ? 0 : g == 1 ? 3 : g == 2 ? 4 : g == 3 ? 6 : 7; }
__host__ __device__ constexpr int wg_hi(int g) { return g == 0 ? 1 : g == 1 ? 2 : g == 2 ? 5 : g == 3 ? 7 : 8; }
// byte offset of tap t's window (K-step 0) inside a stage: box dx + 1, row dy + 1
__host__ __device__ constexpr int wg_win(int t) { return (t % 3) * HALO_BYTES + (t / 3) * 1024; }
static_assert(wg_win(wg_hi(0)) > wg_win(wg_lo(0)) && wg_win(wg_hi(1)) > wg_win(wg_lo(1)) &&
                  wg_win(wg_hi(2)) > wg_win(wg_lo(2)) && wg_win(wg_hi(3)) > wg_win(wg_lo(3)) &&
                  wg_win(wg_hi(4)) > wg_win(wg_lo(4)),
              "the second tap of an MMA pair must lie above the first (positive leading byte offset)");

// TAPS = 1 is the first layer on its packed 5 x 3 x 3 neighbourhoods (no halo):
// one act box and the dz box per tile, and one MMA per K-step whose second 64
// rows of A are the dz box (dropped), so D[k][co] comes out in rows 0-63.
template <int TAPS>
__global__ void __launch_bounds__(THREADS, 1)
wgrad_tc_kernel(const __grid_constant__ CUtensorMap map_act, const __grid_constant__ CUtensorMap map_dz,
                float* __restrict__ part, TileGeom tg, int* __restrict__ err) {
    static_assert(TAPS == 9 || TAPS == 1, "3x3 hidden layers or the packed first layer");
    constexpr int SB = TAPS == 9 ? WG_STAGE_BYTES : 2 * TILE_BYTES;     // stage bytes
    constexpr int DZ_OFF = TAPS == 9 ? 3 * HALO_BYTES : TILE_BYTES;      // the dz box inside a stage
    constexpr int NG = TAPS == 9 ? 5 : 1;                                // MMAs per K-step
    extern __shared__ uint8_t smem_raw[];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sS = smem;
    uint64_t* bars = (uint64_t*)(sS + WG_STAGES * SB + WG_SLACK);
    uint64_t* full = bars;
    uint64_t* empty = bars + WG_STAGES;
    uint64_t* done = bars + 2 * WG_STAGES;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < WG_STAGES; ++s) {
            tc::mbar_init(&full[s], 1);
            tc::mbar_init(&empty[s], 1);
        }
        tc::mbar_init(done, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 1) {
        tc::tmem_alloc(tmem_slot, WG_TMEM_COLS);
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
            // ---------------- producer: three act halo boxes and the dz box per tile
            int issued[WG_STAGES] = {0, 0};
            bool ok = true;
            int j = 0;
            for (int tile = blockIdx.x; tile < tg.total; tile += gridDim.x, ++j) {
                const int s = j % WG_STAGES, u = j / WG_STAGES;
                if (u > 0 && !tc::mbar_wait(&empty[s], (u - 1) & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                int img, a0, b0;
                decode_tile(tg, tile, img, a0, b0);
                uint8_t* dst = sS + s * SB;
                tc::mbar_expect_tx(&full[s], SB);
                if (TAPS == 9) {
#pragma unroll
                    for (int bx = 0; bx < 3; ++bx)
                        tc::tma_load_4d(dst + bx * HALO_BYTES, &map_act, &full[s], 0, b0 + bx - 1, a0 - 1, img);
                } else {
                    tc::tma_load_4d(dst, &map_act, &full[s], 0, b0, a0, img);
                }
                tc::tma_load_4d(dst + DZ_OFF, &map_dz, &full[s], 0, b0, a0, img);
                issued[s] = u + 1;
            }
            if (!ok) {
                give_up(MSF_ERR_TIMEOUT);
                for (int s = 0; s < WG_STAGES; ++s)
                    if (issued[s] > 0) tc::mbar_wait(&full[s], (issued[s] - 1) & 1, nullptr, 100000000ull);
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // ---------------- MMA issuer: 8 K-steps x 5 tap pairs per tile, all into TMEM
            constexpr uint32_t idesc = tc::idesc_bf16_mn<128, 64>();
            bool ok = true;
            int j = 0;
            for (int tile = blockIdx.x; tile < tg.total; tile += gridDim.x, ++j) {
                const int s = j % WG_STAGES, u = j / WG_STAGES;
                if (!tc::mbar_wait(&full[s], u & 1, abort_flag)) {
                    ok = false;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t st_base = tc::smem_u32(sS + s * SB);
#pragma unroll
                for (int k = 0; k < TILE_A / 2; ++k) {
                    const uint64_t bd = tc::desc_sw128_mn(st_base + DZ_OFF + k * 2048, 1024);
                    if (TAPS == 9) {
#pragma unroll
                        for (int g = 0; g < NG; ++g) {
                            const uint32_t lo = st_base + wg_win(wg_lo(g)) + k * 2048;
                            const uint64_t ad =
                                tc::desc_sw128_mn(lo, (uint32_t)(wg_win(wg_hi(g)) - wg_win(wg_lo(g))));
                            tc::mma_bf16(tmem_base + g * 64, ad, bd, idesc, (j | k) ? 1u : 0u);
                        }
                    } else {
                        const uint64_t ad = tc::desc_sw128_mn(st_base + k * 2048, (uint32_t)DZ_OFF);
                        tc::mma_bf16(tmem_base, ad, bd, idesc, (j | k) ? 1u : 0u);
                    }
                }
                tc::mma_commit(&empty[s]);
            }
            if (ok) tc::mma_commit(done);
            else give_up(MSF_ERR_TIMEOUT);
        }
    } else {
        // ---------------- epilogue: TMEM lane quarter q = warp % 4 holds rows 32q..32q+31
        const int q = warp & 3;
        const int m = q * 32 + lane;          // accumulator row: (tap half, ci)
        if (tc::mbar_wait(done, 0, abort_flag)) {
            tc::fence_after_sync();
            float* out = part + (size_t)blockIdx.x * 9 * CH * CH;
#pragma unroll 1
            for (int g = 0; g < NG; ++g) {
                // the dropped halves (warp-uniform): tap 7 again, or the first
                // layer's dz rows
                if ((TAPS == 9 && g == 4 && q < 2) || (TAPS == 1 && q >= 2)) continue;
                uint32_t r[64];
                const uint32_t taddr = tmem_base + ((uint32_t)(q * 32) << 16) + g * 64;
#pragma unroll
                for (int c = 0; c < 4; ++c) tc::tmem_ld16(taddr + c * 16, r + c * 16);
                tc::tmem_ld_wait();
                const int tap = TAPS == 1 ? 0 : (m < 64 ? wg_lo(g) : wg_hi(g)), ci = m & 63;
                float* o = out + (size_t)tap * CH * CH + ci;
#pragma unroll
                for (int co = 0; co < CH; ++co) o[co * CH] = __uint_as_float(r[co]);
            }
        } else {
            give_up(MSF_ERR_TIMEOUT);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) {
        tc::fence_after_sync();
        tc::tmem_dealloc(tmem_base, WG_TMEM_COLS);
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
static msf_status make_act_map(CUtensorMap* m, void* base, int imgs, int H, int W, int box_rows,
                               int box_cols = TILE_B) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[4] = {(cuuint64_t)CH, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)imgs};
    cuuint64_t strides[3] = {(cuuint64_t)CH * 2, (cuuint64_t)W * CH * 2, (cuuint64_t)H * W * CH * 2};
    cuuint32_t box[4] = {(cuuint32_t)CH, (cuuint32_t)box_cols, (cuuint32_t)box_rows, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled (activations) failed: %d", (int)r);
    return MSF_OK;
}

// 4D FP32 tensor [imgs][H][W][64] (pre-BatchNorm outputs) for TMA stores of
// one epilogue warp's 4 x 8 pixels, in two boxes of 32 channels (128 bytes,
// the widest inner box the 128-byte swizzle takes).
static msf_status make_f32_out_map(CUtensorMap* m, void* base, int imgs, int H, int W) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[4] = {(cuuint64_t)CH, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)imgs};
    cuuint64_t strides[3] = {(cuuint64_t)CH * 4, (cuuint64_t)W * CH * 4, (cuuint64_t)H * W * CH * 4};
    cuuint32_t box[4] = {32, (cuuint32_t)TILE_B, (cuuint32_t)(TILE_A / 4), 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled (FP32 outputs) failed: %d", (int)r);
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

// 5D view of a BF16 activation tensor [imgs][H][W][64], H even: dims
// (64, W, parity, H / 2, imgs), so that one box holds rows of one parity.
static msf_status make_pair_map(CUtensorMap* m, void* base, int imgs, int H, int W, int box_pairs) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    if (H % 2) return fail(MSF_ERR_ARG, "row-pair activation map needs an even height, got %d", H);
    const cuuint64_t row = (cuuint64_t)W * CH * 2;
    cuuint64_t dims[5] = {(cuuint64_t)CH, (cuuint64_t)W, 2, (cuuint64_t)(H / 2), (cuuint64_t)imgs};
    cuuint64_t strides[4] = {(cuuint64_t)CH * 2, row, 2 * row, (cuuint64_t)H * row};
    cuuint32_t box[5] = {(cuuint32_t)CH, (cuuint32_t)TILE_B, 1, (cuuint32_t)box_pairs, 1};
    cuuint32_t es[5] = {1, 1, 1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled (row pairs) failed: %d", (int)r);
    return MSF_OK;
}

// The output layer's packed weights [9 taps][16 rows][64] viewed as one row per
// tap (row 0 of each tap), box 64 x 16: rows 9-15 lie outside and read as zero.
static msf_status make_w10_map(CUtensorMap* m, void* base) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)KPACK, 9};
    cuuint64_t strides[1] = {(cuuint64_t)16 * KPACK * 2};
    cuuint32_t box[2] = {(cuuint32_t)KPACK, 16};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled (output-layer taps) failed: %d", (int)r);
    return MSF_OK;
}

// FP32 frames [count][S][H][W], consecutive in memory, with a box of one patch
// of the first layer (C1_PCOLS x C1_PROWS of one slice of one frame).
static msf_status make_frame_map(CUtensorMap* m, const float* base, int S, int H, int W, int count) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    if ((W * 4) % 16) return fail(MSF_ERR_ARG, "first-layer frame map needs W a multiple of 4, got %d", W);
    cuuint64_t dims[4] = {(cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)S, (cuuint64_t)count};
    cuuint64_t strides[3] = {(cuuint64_t)W * 4, (cuuint64_t)H * W * 4, (cuuint64_t)S * H * W * 4};
    cuuint32_t box[4] = {(cuuint32_t)C1_PCOLS, (cuuint32_t)C1_PROWS, 1, 1};
    cuuint32_t es[4] = {1, 1, 1, 1};
    CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(MSF_ERR_CUDA, "cuTensorMapEncodeTiled (frames) failed: %d", (int)r);
    return MSF_OK;
}

static int g_num_sms = 0;

template <int TAPS, int N, int NS, int EPI>
static cudaError_t set_smem_attr() {
    return cudaFuncSetAttribute(conv_tc_kernel<TAPS, N, NS, EPI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                ConvCfg<TAPS, N, NS, EPI>::SMEM);
}

// One-time, out-of-stream set-up of every conv variant (shared-memory limits)
// and of the SM count; done before any launch so that no such call ever lands
// inside a stream capture.
static msf_status ensure_kernel_attrs() {
    static bool done = false;
    if (done) return MSF_OK;
    int dev = 0;
    MSF_TRY_CUDA(cudaGetDevice(&dev));
    MSF_TRY_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
    MSF_TRY_CUDA((set_smem_attr<1, 64, NS_1X1, EPI_RELU>()));
    MSF_TRY_CUDA((set_smem_attr<9, 64, NS_3X3, EPI_RELU>()));
    MSF_TRY_CUDA((set_smem_attr<9, 64, NS_3X3, EPI_RAW>()));
    MSF_TRY_CUDA((set_smem_attr<9, 64, NS_3X3, EPI_RAW32>()));
    MSF_TRY_CUDA((set_smem_attr<9, 16, NS_LAST, EPI_RESID>()));
    MSF_TRY_CUDA((set_smem_attr<9, 16, NS_LAST, EPI_F32>()));
    MSF_TRY_CUDA(cudaFuncSetAttribute(conv_pair_kernel<EPI_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      PairCfg::SMEM));
    MSF_TRY_CUDA(cudaFuncSetAttribute(conv1_fused_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      C1Cfg::SMEM));
    MSF_TRY_CUDA(cudaFuncSetAttribute(conv1_fused_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      C1Cfg::SMEM));
    MSF_TRY_CUDA(cudaFuncSetAttribute(conv_pair_kernel<EPI_PART>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      PairCfg::SMEM));
    MSF_TRY_CUDA(cudaFuncSetAttribute(wgrad_tc_kernel<9>, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM));
    MSF_TRY_CUDA(cudaFuncSetAttribute(wgrad_tc_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, WG_SMEM));
    MSF_TRY_CUDA(cudaFuncSetAttribute(conv_pair_multi_kernel<EPI_RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      PairCfg::SMEM));
    MSF_TRY_CUDA(cudaFuncSetAttribute(conv_pair_multi_kernel<EPI_PART>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      PairCfg::SMEM));
    done = true;
    return MSF_OK;
}

template <int TAPS, int N, int NS, int EPI>
static msf_status launch_conv(const CUtensorMap& ma, const CUtensorMap& mw, const CUtensorMap& mo, const float* bias,
                              const TileGeom& tg, const SliceGeom& sg, const float* centre, float* outv, int* err,
                              cudaStream_t st, double* moments = nullptr) {
    using C = ConvCfg<TAPS, N, NS, EPI>;
    auto kern = conv_tc_kernel<TAPS, N, NS, EPI>;
    MSF_TRY(ensure_kernel_attrs());
    const int grid = tg.total < g_num_sms ? tg.total : g_num_sms;
    if (grid <= 0) return MSF_OK;
    MSF_PROF(TAPS == 1 ? "conv1_tc"
                       : (N == 16 ? "conv10_tc"
                                  : (EPI == EPI_RAW ? "conv3x3_dgrad_tc" : (EPI == EPI_RAW32 ? "conv3x3_fp32_tc" : "conv3x3_tc"))),
             st);
    if (EPI == EPI_RAW32 && !moments) return fail(MSF_ERR_ARG, "launch_conv: FP32 outputs need a moments buffer");
    kern<<<grid, THREADS, C::SMEM, st>>>(ma, mw, mo, bias, tg, sg, centre, outv, moments, err);
    MSF_LAUNCH_CHECK();
    return MSF_OK;
}

// Row-pair 3x3 layer over images of even height (tg in row-pair tiles).
template <int EPI>
static msf_status launch_pair(const CUtensorMap& ma, const CUtensorMap& mw, const CUtensorMap& mo,
                              const CUtensorMap& mw10, const float* bias, const TileGeom& tg, int* err, cudaStream_t st,
                              float* part = nullptr, long long plane = 0) {
    MSF_TRY(ensure_kernel_attrs());
    const int grid = tg.total < g_num_sms ? tg.total : g_num_sms;
    if (grid <= 0) return MSF_OK;
    MSF_PROF(EPI == EPI_PART ? "conv3x3_out_tc" : "conv3x3_tc", st);
    conv_pair_kernel<EPI><<<grid, THREADS, PairCfg::SMEM, st>>>(ma, mw, mo, mw10, bias, tg, err, part, plane);
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
    uint8_t* d_frozen = nullptr;    // 1 for parameters Adam leaves alone (running statistics)
    __nv_bfloat16* d_wpack = nullptr;
    float* d_bias = nullptr;        // [10][64]
    size_t wpack_off[LAYERS];
    __nv_bfloat16* d_act[2] = {nullptr, nullptr};
    float* d_frames = nullptr;      // up to 5 * max_pixels floats: frames in the agent's [S][H][W] order
    int* d_err = nullptr;
    bool folded = false;
    int64_t adam_t = 0;
    uint64_t gen = 1;               // bumped whenever the parameters change
    // training workspace (msf_cnn_train_reserve)
    int64_t train_cap = 0;
    void* train_ws = nullptr;
    size_t train_ws_bytes = 0;
    // optional record of the inter-layer gradients of the last step
    // (msf_cnn_train_trace): dz of layers 0..8 and da of layers 1..9, BF16 [P][64]
    bool trace_on = false;
    __nv_bfloat16* trace = nullptr;
    int64_t trace_cap = 0;
    int64_t last_P = 0;
    // launch choices of msf_denoise per orientation, for one slice shape
    // (msf_cnn_autotune / msf_cnn_set_tuning); tile 0 = by height parity
    struct Tune {
        int S = 0, H = 0, W = 0;   // the slice shape the choice is for (0: none)
        int tile = 0;              // MSF_TILE_AUTO, MSF_TILE_16x8 or MSF_TILE_PAIR
        int chunk = 0;             // time-points per chunk (0: as many as fit, at most 16)
    } tune[3];
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
    MSF_TRY(ensure_kernel_attrs());
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
              cudaMalloc(&c->d_frames, (size_t)max_pixels * 5 * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&c->d_err, sizeof(int)) == cudaSuccess && cudaMalloc(&c->d_frozen, P) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        msf_cnn_destroy(c);
        return fail(MSF_ERR_NOMEM, "msf_cnn_create: out of device memory");
    }
    cudaMemset(c->d_params, 0, P * 4);
    cudaMemset(c->d_m, 0, P * 4);
    cudaMemset(c->d_v, 0, P * 4);
    cudaMemset(c->d_err, 0, sizeof(int));
    {
        std::vector<uint8_t> frozen(P, 0);
        for (int l = 1; l < LAYERS - 1; ++l)
            for (int k = 0; k < CH; ++k) frozen[c->off.mean[l] + k] = frozen[c->off.var[l] + k] = 1;
        cudaMemcpy(c->d_frozen, frozen.data(), P, cudaMemcpyHostToDevice);
        cudaMemset(c->d_grad, 0, P * 4);
    }
    *out = c;
    return MSF_OK;
}

extern "C" void msf_cnn_destroy(msf_cnn* c) {
    if (!c) return;
    cudaFree(c->d_params); cudaFree(c->d_grad); cudaFree(c->d_m); cudaFree(c->d_v);
    cudaFree(c->d_wpack); cudaFree(c->d_bias);
    cudaFree(c->d_act[0]); cudaFree(c->d_act[1]);
    cudaFree(c->d_frames);
    cudaFree(c->d_err);
    cudaFree(c->d_frozen);
    cudaFree(c->train_ws);
    cudaFree(c->trace);
    delete c;
}

extern "C" msf_status msf_cnn_set_params(msf_cnn* c, const float* h_params, size_t n) {
    MSF_REQUIRE(c && h_params, "msf_cnn_set_params: NULL argument");
    MSF_REQUIRE(n == c->off.total, "msf_cnn_set_params: expected %zu parameters, got %zu", c->off.total, n);
    MSF_TRY_CUDA(cudaMemcpy(c->d_params, h_params, n * 4, cudaMemcpyHostToDevice));
    MSF_TRY_CUDA(cudaMemset(c->d_m, 0, n * 4));
    MSF_TRY_CUDA(cudaMemset(c->d_v, 0, n * 4));
    c->adam_t = 0;
    c->gen += 1;
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

// Layer 1 of one chunk (time-points sg.t0 .. sg.t0 + sg.nframes - 1): the
// frames the chunk reads are brought into the agent's [S][H][W] order, then the
// fused first layer writes the 64-channel activations into c->d_act[1].
static msf_status first_layer(msf_cnn* c, const SliceGeom& sg, const msf_vol* vol, msf_orient orient,
                              const float* d_in, const CUtensorMap& mw0, const CUtensorMap& m1o, int64_t per_frame,
                              cudaStream_t st) {
    const int t0 = sg.t0;
    // the time-points this chunk reads, in the agent's [S][H][W] order
    PackFrames pf;
    pf.first = t0 - 2 > 0 ? t0 - 2 : 0;
    const int last = t0 + sg.nframes + 1 < vol->nt - 1 ? t0 + sg.nframes + 1 : vol->nt - 1;
    pf.count = last - pf.first + 1;
    MSF_REQUIRE(pf.count <= 20 && (int64_t)pf.count * per_frame <= 5 * c->max_pixels,
                "msf_denoise: internal frame window too large");
    for (int k = 0; k < pf.count; ++k) {
        const float* src = d_in + (size_t)(pf.first + k) * per_frame;
        if (orient == MSF_XY_T) {
            pf.f[k] = src;
        } else {
            float* dst = c->d_frames + (size_t)k * per_frame;
            const long long rows = orient == MSF_YZ_T ? (long long)vol->nz * vol->ny : vol->nz;
            const long long cols = orient == MSF_YZ_T ? vol->nx : (long long)vol->ny * vol->nx;
            MSF_PROF("orient_transpose", st);
            orient_transpose_kernel<<<dim3((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32)),
                                      dim3(32, 8), 0, st>>>(src, dst, rows, cols);
            MSF_LAUNCH_CHECK();
            pf.f[k] = dst;
        }
    }
    // first layer straight from the frames
    TileGeom t1;
    t1.H = sg.H; t1.W = sg.W; t1.imgs = sg.nframes * sg.S;
    t1.tiles_a = (sg.H + C1_ROWS - 1) / C1_ROWS;
    t1.tiles_b = (sg.W + C1_COLS - 1) / C1_COLS;
    t1.total = t1.imgs * t1.tiles_a * t1.tiles_b;
    MSF_TRY(ensure_kernel_attrs());
    MSF_PROF("conv1_tc", st);
    // the patch ring needs the frames consecutive (they are: the input
    // volume or the transposed copies) and rows of a multiple of 16 bytes
    const int grid1 = t1.total < g_num_sms ? t1.total : g_num_sms;
    if (sg.W % 4 == 0) {
        CUtensorMap mf;
        MSF_TRY(make_frame_map(&mf, pf.f[0], sg.S, sg.H, sg.W, pf.count));
        conv1_fused_kernel<true><<<grid1, C1_THREADS, C1Cfg::SMEM, st>>>(mw0, m1o, mf, c->d_bias, pf, sg, t1,
                                                                           c->d_err);
    } else {
        conv1_fused_kernel<false><<<grid1, C1_THREADS, C1Cfg::SMEM, st>>>(mw0, m1o, m1o, c->d_bias, pf, sg,
                                                                            t1, c->d_err);
    }
    MSF_LAUNCH_CHECK();
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
    set_strides(sg);
    const int64_t per_frame = (int64_t)sg.S * sg.H * sg.W;
    MSF_REQUIRE(per_frame <= c->max_pixels,
                "msf_denoise: one time-point has %lld pixels but the handle holds %lld (max_pixels)",
                (long long)per_frame, (long long)c->max_pixels);
    MSF_REQUIRE(per_frame * 128 < ((int64_t)1 << 40), "msf_denoise: frame too large");
    if (!c->folded) MSF_TRY(fold_all(c, st));
    const msf_cnn::Tune& tu = c->tune[(int)orient];
    const bool tuned = tu.S == sg.S && tu.H == sg.H && tu.W == sg.W;
    int fchunk = (int)(c->max_pixels / per_frame < 16 ? c->max_pixels / per_frame : 16);
    if (tuned && tu.chunk > 0 && tu.chunk < fchunk) fchunk = tu.chunk;
    const int imgs_cap = fchunk * sg.S;
    CUtensorMap m18[2], m4[2], mw[LAYERS];
    for (int b = 0; b < 2; ++b) {
        MSF_TRY(make_act_map(&m18[b], c->d_act[b], imgs_cap, sg.H, sg.W, TILE_A + 2));
        MSF_TRY(make_act_map(&m4[b], c->d_act[b], imgs_cap, sg.H, sg.W, TILE_A / 4));
    }
    CUtensorMap m1o;   // first-layer output: one row of 32 pixels per store
    MSF_TRY(make_act_map(&m1o, c->d_act[1], imgs_cap, sg.H, sg.W, 1, C1_COLS));
    for (int l = 0; l < LAYERS; ++l)
        MSF_TRY(make_w_map(&mw[l], c->d_wpack + c->wpack_off[l], taps_of(l) * rows_of(l), rows_of(l)));
    // images of even height take the row-pair kernel for the 64 -> 64 layers,
    // the last of them fused with the output layer
    const bool pairs = sg.H % 2 == 0 && !(tuned && tu.tile == MSF_TILE_16x8);
    CUtensorMap p17[2], p4[2], mw10;
    if (pairs) {
        for (int b = 0; b < 2; ++b) {
            MSF_TRY(make_pair_map(&p17[b], c->d_act[b], imgs_cap, sg.H, sg.W, PAIR_ROWS + 1));
            MSF_TRY(make_pair_map(&p4[b], c->d_act[b], imgs_cap, sg.H, sg.W, 4));
        }
        MSF_TRY(make_w10_map(&mw10, c->d_wpack + c->wpack_off[LAYERS - 1]));
    }
    for (int t0 = 0; t0 < vol->nt; t0 += fchunk) {
        sg.t0 = t0;
        sg.nframes = fchunk < vol->nt - t0 ? fchunk : vol->nt - t0;
        MSF_TRY(first_layer(c, sg, vol, orient, d_in, mw[0], m1o, per_frame, st));
        TileGeom tg;
        tg.H = sg.H; tg.W = sg.W; tg.imgs = sg.nframes * sg.S;
        tg.tiles_a = (sg.H + TILE_A - 1) / TILE_A;
        tg.tiles_b = (sg.W + TILE_B - 1) / TILE_B;
        tg.total = tg.imgs * tg.tiles_a * tg.tiles_b;
        int cur = 1;
        TileGeom tp = tg;
        tp.tiles_a = (sg.H + 2 * PAIR_ROWS - 1) / (2 * PAIR_ROWS);
        tp.total = tp.imgs * tp.tiles_a * tp.tiles_b;
        const long long plane = (long long)tg.imgs * sg.H * sg.W;
        for (int l = 1; l < LAYERS - 1; ++l) {
            if (pairs && l == LAYERS - 2)
                // per-tap planes of the output layer instead of activations
                MSF_TRY((launch_pair<EPI_PART>(p17[cur], mw[l], p4[cur ^ 1], mw10, c->d_bias + l * CH, tp, c->d_err,
                                               st, reinterpret_cast<float*>(c->d_act[cur ^ 1]), plane)));
            else if (pairs)
                MSF_TRY((launch_pair<EPI_RELU>(p17[cur], mw[l], p4[cur ^ 1], p4[cur ^ 1], c->d_bias + l * CH, tp,
                                               c->d_err, st)));
            else
                MSF_TRY((launch_conv<9, 64, NS_3X3, EPI_RELU>(m18[cur], mw[l], m4[cur ^ 1], c->d_bias + l * CH, tg,
                                                              sg, nullptr, nullptr, c->d_err, st)));
            cur ^= 1;
        }
        if (pairs) {
            MSF_PROF("resid_stencil", st);
            const float* part = reinterpret_cast<const float*>(c->d_act[cur]);
            const float* b10 = c->d_bias + (LAYERS - 1) * CH;
            if (orient == MSF_XY_T) launch_stencil<0>(part, plane, b10, sg, d_in, d_out, st);
            else if (orient == MSF_YZ_T) launch_stencil<1>(part, plane, b10, sg, d_in, d_out, st);
            else launch_stencil<2>(part, plane, b10, sg, d_in, d_out, st);
            MSF_LAUNCH_CHECK();
        } else {
            MSF_TRY((launch_conv<9, 16, NS_LAST, EPI_RESID>(m18[cur], mw[LAYERS - 1], m4[cur ^ 1],
                                                            c->d_bias + (LAYERS - 1) * CH, tg, sg, d_in, d_out,
                                                            c->d_err, st)));
        }
    }
    return MSF_OK;
}

// The slices of `vol` in orientation `orient`.
static SliceGeom slice_geom(msf_orient orient, const msf_vol* vol) {
    SliceGeom sg;
    sg.orient = (int)orient;
    sg.nx = vol->nx; sg.ny = vol->ny; sg.nz = vol->nz; sg.nt = vol->nt;
    if (orient == MSF_XY_T) { sg.S = vol->nz; sg.H = vol->ny; sg.W = vol->nx; }
    else if (orient == MSF_YZ_T) { sg.S = vol->nx; sg.H = vol->nz; sg.W = vol->ny; }
    else { sg.S = vol->ny; sg.H = vol->nx; sg.W = vol->nz; }
    set_strides(sg);
    sg.t0 = 0;
    sg.nframes = vol->nt;
    return sg;
}

extern "C" msf_status msf_denoise_batch(msf_cnn* const* cnns, int n, msf_orient orient, const msf_vol* vols,
                                        const float* const* d_in, float* const* d_out, void* stream) {
    MSF_REQUIRE(cnns && vols && d_in && d_out && n > 0, "msf_denoise_batch: NULL argument or empty batch");
    MSF_REQUIRE(n <= PAIR_MAX_JOBS, "msf_denoise_batch: at most %d problems", PAIR_MAX_JOBS);
    MSF_REQUIRE(orient >= MSF_XY_T && orient <= MSF_ZX_T, "msf_denoise_batch: bad orientation %d", (int)orient);
    for (int p = 0; p < n; ++p) {
        MSF_REQUIRE(cnns[p] && d_in[p] && d_out[p] && d_in[p] != d_out[p], "msf_denoise_batch: problem %d: bad pointers", p);
        for (int q = 0; q < p; ++q)
            MSF_REQUIRE(cnns[q] != cnns[p], "msf_denoise_batch: problems %d and %d share a handle (its workspace)", q, p);
    }
    cudaStream_t st = as_stream(stream);
    MSF_TRY(ensure_kernel_attrs());
    struct Prob {
        msf_cnn* c;
        int idx;
        SliceGeom sg;
        int64_t per_frame;
        CUtensorMap p17[2], p4[2], mw0, m1o;
        TileGeom tp;
        long long plane;
    };
    std::vector<Prob> batch;
    for (int p = 0; p < n; ++p) {
        msf_cnn* c = cnns[p];
        const msf_vol* vol = &vols[p];
        MSF_REQUIRE(vol->nx > 0 && vol->ny > 0 && vol->nz > 0 && vol->nt > 0, "msf_denoise_batch: bad volume %d", p);
        const SliceGeom sg = slice_geom(orient, vol);
        const int64_t per_frame = (int64_t)sg.S * sg.H * sg.W;
        const msf_cnn::Tune& tu = c->tune[(int)orient];
        const bool tuned = tu.S == sg.S && tu.H == sg.H && tu.W == sg.W;
        int64_t fchunk = c->max_pixels / per_frame < 16 ? c->max_pixels / per_frame : 16;
        if (tuned && tu.chunk > 0 && tu.chunk < fchunk) fchunk = tu.chunk;
        const bool pairs = sg.H % 2 == 0 && !(tuned && tu.tile == MSF_TILE_16x8);
        if (!pairs || fchunk < vol->nt || per_frame * 128 >= ((int64_t)1 << 40)) {
            // not in one row-pair chunk: this problem runs on its own
            MSF_TRY(msf_denoise(c, orient, vol, d_in[p], d_out[p], stream));
            continue;
        }
        if (!c->folded) MSF_TRY(fold_all(c, st));
        Prob b;
        b.c = c;
        b.idx = p;
        b.sg = sg;
        b.per_frame = per_frame;
        const int imgs = vol->nt * sg.S;
        for (int k = 0; k < 2; ++k) {
            MSF_TRY(make_pair_map(&b.p17[k], c->d_act[k], imgs, sg.H, sg.W, PAIR_ROWS + 1));
            MSF_TRY(make_pair_map(&b.p4[k], c->d_act[k], imgs, sg.H, sg.W, 4));
        }
        MSF_TRY(make_w_map(&b.mw0, c->d_wpack + c->wpack_off[0], taps_of(0) * rows_of(0), rows_of(0)));
        MSF_TRY(make_act_map(&b.m1o, c->d_act[1], imgs, sg.H, sg.W, 1, C1_COLS));
        b.tp.H = sg.H; b.tp.W = sg.W; b.tp.imgs = imgs;
        b.tp.tiles_a = (sg.H + 2 * PAIR_ROWS - 1) / (2 * PAIR_ROWS);
        b.tp.tiles_b = (sg.W + TILE_B - 1) / TILE_B;
        b.tp.total = imgs * b.tp.tiles_a * b.tp.tiles_b;
        b.plane = (long long)imgs * sg.H * sg.W;
        batch.push_back(b);
    }
    if (batch.empty()) return MSF_OK;
    // the 64 -> 64 layers' weights and biases: the first batched handle's
    // (every handle of a batch holds the same parameters)
    msf_cnn* c0 = batch[0].c;
    CUtensorMap mw[LAYERS], mw10;
    for (int l = 1; l < LAYERS - 1; ++l)
        MSF_TRY(make_w_map(&mw[l], c0->d_wpack + c0->wpack_off[l], taps_of(l) * rows_of(l), rows_of(l)));
    MSF_TRY(make_w10_map(&mw10, c0->d_wpack + c0->wpack_off[LAYERS - 1]));
    for (Prob& b : batch)
        MSF_TRY(first_layer(b.c, b.sg, &vols[b.idx], orient, d_in[b.idx], b.mw0, b.m1o, b.per_frame, st));
    PairJobs J;
    memset(&J, 0, sizeof(J));
    J.n = (int)batch.size();
    J.total = 0;
    for (int i = 0; i < J.n; ++i) {
        J.job[i].tg = batch[i].tp;
        J.job[i].tile0 = J.total;
        J.job[i].plane = batch[i].plane;
        J.total += batch[i].tp.total;
    }
    const int grid = J.total < g_num_sms ? J.total : g_num_sms;
    int cur = 1;
    for (int l = 1; l < LAYERS - 1; ++l) {
        const bool last = l == LAYERS - 2;
        for (int i = 0; i < J.n; ++i) {
            J.job[i].a = batch[i].p17[cur];
            J.job[i].out = batch[i].p4[cur ^ 1];
            J.job[i].part = last ? reinterpret_cast<float*>(batch[i].c->d_act[cur ^ 1]) : nullptr;
        }
        MSF_PROF(last ? "conv3x3_out_tc" : "conv3x3_tc", st);
        if (last)
            conv_pair_multi_kernel<EPI_PART><<<grid, THREADS, PairCfg::SMEM, st>>>(J, mw[l], mw10, c0->d_bias + l * CH,
                                                                                  c0->d_err);
        else
            conv_pair_multi_kernel<EPI_RELU><<<grid, THREADS, PairCfg::SMEM, st>>>(J, mw[l], mw10, c0->d_bias + l * CH,
                                                                                  c0->d_err);
        MSF_LAUNCH_CHECK();
        cur ^= 1;
    }
    for (Prob& b : batch) {
        MSF_PROF("resid_stencil", st);
        const float* part = reinterpret_cast<const float*>(b.c->d_act[cur]);
        const float* b10 = b.c->d_bias + (LAYERS - 1) * CH;
        if (orient == MSF_XY_T) launch_stencil<0>(part, b.plane, b10, b.sg, d_in[b.idx], d_out[b.idx], st);
        else if (orient == MSF_YZ_T) launch_stencil<1>(part, b.plane, b10, b.sg, d_in[b.idx], d_out[b.idx], st);
        else launch_stencil<2>(part, b.plane, b10, b.sg, d_in[b.idx], d_out[b.idx], st);
        MSF_LAUNCH_CHECK();
    }
    return MSF_OK;
}

extern "C" msf_status msf_cnn_set_tuning(msf_cnn* c, msf_orient orient, const msf_vol* vol, int tile, int chunk) {
    MSF_REQUIRE(c && vol, "msf_cnn_set_tuning: NULL argument");
    MSF_REQUIRE(orient >= MSF_XY_T && orient <= MSF_ZX_T, "msf_cnn_set_tuning: bad orientation %d", (int)orient);
    MSF_REQUIRE(tile == MSF_TILE_AUTO || tile == MSF_TILE_16x8 || tile == MSF_TILE_PAIR,
                "msf_cnn_set_tuning: unknown tile shape %d", tile);
    MSF_REQUIRE(chunk >= 0 && chunk <= 16, "msf_cnn_set_tuning: chunk must lie in 0..16");
    int S, H, W;
    if (orient == MSF_XY_T) { S = vol->nz; H = vol->ny; W = vol->nx; }
    else if (orient == MSF_YZ_T) { S = vol->nx; H = vol->nz; W = vol->ny; }
    else { S = vol->ny; H = vol->nx; W = vol->nz; }
    MSF_REQUIRE(tile != MSF_TILE_PAIR || H % 2 == 0, "msf_cnn_set_tuning: row-pair tiles need an even slice height");
    msf_cnn::Tune& t = c->tune[(int)orient];
    t.S = S; t.H = H; t.W = W; t.tile = tile; t.chunk = chunk;
    c->gen += 1;   // a captured MACE iteration must be captured again
    return MSF_OK;
}

extern "C" msf_status msf_cnn_autotune(msf_cnn* c, const msf_vol* vol, const float* d_in, float* d_out, void* stream,
                                       int* h_choice) {
    MSF_REQUIRE(c && vol && d_in && d_out, "msf_cnn_autotune: NULL argument");
    MSF_REQUIRE(d_in != d_out, "msf_cnn_autotune: input and output must differ");
    cudaStream_t st = as_stream(stream);
    cudaEvent_t e0, e1;
    MSF_TRY_CUDA(cudaEventCreate(&e0));
    MSF_TRY_CUDA(cudaEventCreate(&e1));
    msf_status rc = MSF_OK;
    for (int o = 0; o < 3 && rc == MSF_OK; ++o) {
        const msf_orient orient = (msf_orient)o;
        const int H = o == MSF_XY_T ? vol->ny : (o == MSF_YZ_T ? vol->nz : vol->nx);
        const int tiles[2] = {MSF_TILE_PAIR, MSF_TILE_16x8};
        const int chunks[3] = {16, 8, 4};
        float best = 1e30f;
        int bt = MSF_TILE_AUTO, bc = 0;
        for (int ti = 0; ti < 2 && rc == MSF_OK; ++ti) {
            if (tiles[ti] == MSF_TILE_PAIR && H % 2 != 0) continue;
            for (int ci = 0; ci < 3 && rc == MSF_OK; ++ci) {
                if (ci > 0 && chunks[ci] >= vol->nt) continue;   // the same launches as a larger chunk
                rc = msf_cnn_set_tuning(c, orient, vol, tiles[ti], chunks[ci]);
                if (rc == MSF_OK) rc = msf_denoise(c, orient, vol, d_in, d_out, stream);   // warm
                if (rc != MSF_OK) break;
                cudaEventRecord(e0, st);
                for (int r = 0; r < 2 && rc == MSF_OK; ++r) rc = msf_denoise(c, orient, vol, d_in, d_out, stream);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = fail(MSF_ERR_CUDA, "msf_cnn_autotune: timing failed");
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (rc == MSF_OK && ms < best) { best = ms; bt = tiles[ti]; bc = chunks[ci]; }
            }
        }
        if (rc == MSF_OK) rc = msf_cnn_set_tuning(c, orient, vol, bt, bc);
        if (h_choice && rc == MSF_OK) {
            h_choice[2 * o] = bt;
            h_choice[2 * o + 1] = bc;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

// ====================================================================== training (Sec. V)
//
// One step on a batch of B noisy 5-frame patches [B][5][H][W] and clean centre
// slices [B][H][W]: forward with BatchNorm batch statistics, loss
// mean((centre - R - clean)^2), backward, Adam on the FP32 master parameters.
// Activations and gradients between layers are BF16 [P][64] (P = B*H*W);
// reductions (BatchNorm statistics, loss, weight gradients) are FP32/FP64.
//   forward convs: tcgen05 (layer 1 on the packed 45-value neighbourhoods,
//                  hidden layers with EPI_RAW, last layer with EPI_F32)
//   input grads:   tcgen05 with the transposed, flipped kernels
//                  W'[tap'][ci][co] = W[co][ci][2-ky][2-kx]
//   weight grads:  tcgen05 (wgrad_tc_kernel: MN-major operands, per-CTA TMEM
//                  accumulation, CTA partials summed in a fixed order); the
//                  64 -> 1 output layer's in FP32 SIMT

namespace msf {
namespace cnn {

constexpr float BN_MOMENTUM = 0.1f;
constexpr int WG_CHUNK = 4096;      // pixels per weight-gradient block
// Blocks of the elementwise training launches.  Their grid-stride loops step
// by EW_BLOCKS * 256 elements of 8 channels, a multiple of 8, so a thread keeps
// the same channel octet (i & 7) for all its elements.
constexpr int EW_BLOCKS = 152 * 8;


// Workspace carved from one allocation.
struct TrainWS {
    __nv_bfloat16* act[LAYERS];     // act[0] packed input, act[l] output of layer l-1 (l = 1..9)
    float* z[LAYERS];               // z[l], l = 1..8: pre-BatchNorm conv outputs (FP32)
    __nv_bfloat16* g[2];            // gradient ping-pong
    float* R;                       // last-layer output
    float* dR;
    double* part;                   // reduction partials
    double* sums;                   // [8][4][64]: sum z, sum z^2, sum dy, sum dy*xhat
    float* bnp;                     // [8][2][64]: mean, istd of the batch
    float* wpart;                   // weight-gradient partials
    __nv_bfloat16* wf;              // packed forward weights (no BatchNorm folding)
    __nv_bfloat16* wb;              // packed input-gradient weights, layers 1..8
    float* bf;                      // [10][64] forward biases
    float* zeros;                   // [64]
    double* loss;                   // [1]
    int nchunks, nred;
};

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static size_t train_layout(int64_t P, TrainWS* w, uint8_t* base) {
    size_t o = 0;
    auto take = [&](size_t bytes) {
        uint8_t* p = base ? base + o : nullptr;
        o += align256(bytes);
        return p;
    };
    const size_t act = (size_t)P * CH * 2;
    TrainWS t{};
    for (int l = 0; l < LAYERS; ++l) t.act[l] = (__nv_bfloat16*)take(act);
    for (int l = 1; l < LAYERS - 1; ++l) t.z[l] = (float*)take(act * 2);
    t.g[0] = (__nv_bfloat16*)take(act);
    t.g[1] = (__nv_bfloat16*)take(act);
    t.R = (float*)take((size_t)P * 4);
    t.dR = (float*)take((size_t)P * 4);
    t.nchunks = (int)((P + WG_CHUNK - 1) / WG_CHUNK);
    t.nred = 2 * 152;
    t.part = (double*)take((size_t)(t.nred > EW_BLOCKS ? t.nred : EW_BLOCKS) * 2 * CH * 8);
    t.sums = (double*)take((size_t)8 * 4 * CH * 8);
    t.bnp = (float*)take((size_t)8 * 2 * CH * 4);
    t.wpart = (float*)take((size_t)(t.nchunks > WG_MAX_CTAS ? t.nchunks : WG_MAX_CTAS) * 9 * CH * CH * 4);
    size_t wp = 0;
    for (int l = 0; l < LAYERS; ++l) wp += (size_t)taps_of(l) * rows_of(l) * KPACK;
    t.wf = (__nv_bfloat16*)take(wp * 2);
    t.wb = (__nv_bfloat16*)take((size_t)8 * 9 * CH * CH * 2);
    t.bf = (float*)take(LAYERS * CH * 4);
    t.zeros = (float*)take(CH * 4);
    t.loss = (double*)take(8);
    if (w) *w = t;
    return o;
}

// [B][5][H][W] FP32 -> packed BF16 [B][H][W][64] (k = frame*9 + ky*3 + kx).
__global__ void pack_batch_kernel(const float* __restrict__ x, uint4* __restrict__ out, int B, int H, int W) {
    const size_t total = (size_t)B * H * W;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < total; p += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(p % W), a = (int)((p / W) % H), img = (int)(p / ((size_t)H * W));
        float v[FRAMES * 9];
#pragma unroll
        for (int c = 0; c < FRAMES; ++c)
#pragma unroll
            for (int ky = 0; ky < 3; ++ky)
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int aa = a + ky - 1, bb = b + kx - 1;
                    v[c * 9 + ky * 3 + kx] = (aa >= 0 && aa < H && bb >= 0 && bb < W)
                                                 ? x[(((size_t)img * FRAMES + c) * H + aa) * W + bb] : 0.0f;
                }
        uint32_t w[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            __nv_bfloat162 h = __floats2bfloat162_rn(2 * i < 45 ? v[2 * i] : 0.0f, 2 * i + 1 < 45 ? v[2 * i + 1] : 0.0f);
            w[i] = *reinterpret_cast<uint32_t*>(&h);
        }
        uint4* dst = out + p * 8;
#pragma unroll
        for (int c = 0; c < 8; ++c) dst[c] = make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
    }
}

// Input-gradient kernels of the hidden layers: W'[tap'][ci][co] = W[co][ci][2-ky][2-kx].
__global__ void pack_dgrad_kernel(const float* __restrict__ params, __nv_bfloat16* __restrict__ wb, Offsets o) {
    const int n = 8 * 9 * CH * CH;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int l = 1 + e / (9 * CH * CH);
        const int r = e % (9 * CH * CH);
        const int tap = r / (CH * CH), ci = (r / CH) % CH, co = r % CH;
        const int ky = 2 - tap / 3, kx = 2 - tap % 3;
        wb[e] = __float2bfloat16_rn(params[o.w[l] + ((size_t)co * CH + ci) * 9 + ky * 3 + kx]);
    }
}

__device__ __forceinline__ void bf16x8_to_f32(uint4 u, float* f) {
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        f[2 * i] = __uint_as_float(w[i] << 16);
        f[2 * i + 1] = __uint_as_float(w[i] & 0xFFFF0000u);
    }
}

__device__ __forceinline__ uint4 f32_to_bf16x8(const float* f) {
    uint32_t w[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat162 h = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
        w[i] = *reinterpret_cast<uint32_t*>(&h);
    }
    return make_uint4(w[0], w[1], w[2], w[3]);
}

__device__ __forceinline__ void f32x8_load(const float* p, float* f) {
    const float4 a = *reinterpret_cast<const float4*>(p), b = *reinterpret_cast<const float4*>(p + 4);
    f[0] = a.x; f[1] = a.y; f[2] = a.z; f[3] = a.w; f[4] = b.x; f[5] = b.y; f[6] = b.z; f[7] = b.w;
}

// The two channel sums of the BatchNorm backward over P pixels: sum dy and
// sum dy*xhat with dy = g * [gamma xhat + beta > 0], xhat = (z - mean) istd
// (g: BF16 [P][64], z: FP32 [P][64]).  256 threads = 8 lanes of 8 channels x
// 32 pixel rows; writes FP64 partials [block][2][64].
__global__ void __launch_bounds__(256, 2) bn_bwd_reduce_kernel(const uint4* __restrict__ g, const float* __restrict__ z,
                                                               const float* __restrict__ bnp,
                                                               const float* __restrict__ gamma,
                                                               const float* __restrict__ beta, size_t P,
                                                               double* __restrict__ part) {
    // sh[k][row][c]: this thread's FP64 sums (its 8 channels of pixel row `row`)
    __shared__ double sh[2][32][65];
    const int lane8 = threadIdx.x & 7, row = threadIdx.x >> 3;
#pragma unroll
    for (int i = 0; i < 8; ++i) sh[0][row][lane8 * 8 + i] = sh[1][row][lane8 * 8 + i] = 0.0;
    float mean[8], istd[8], ga[8], be[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        mean[i] = bnp[lane8 * 8 + i];
        istd[i] = bnp[CH + lane8 * 8 + i];
        ga[i] = gamma[lane8 * 8 + i];
        be[i] = beta[lane8 * 8 + i];
    }
    // Each thread sums runs of RED_RUN of its pixels in FP32 and adds each run
    // into its FP64 sums (FP64 arithmetic is a small fraction of the FP32 rate
    // on this GPU); the order of every addition is fixed.  The loads of a run
    // are issued BATCH at a time before any of them is added (pixels past P
    // read as g = 0, which leaves the sums unchanged), so that each thread
    // keeps several loads in flight.
    constexpr int RED_RUN = 32, BATCH = 4;
    const size_t stride = (size_t)gridDim.x * 32;
    for (size_t p = blockIdx.x * (size_t)32 + row; p < P; p += RED_RUN * stride) {
        float r0[8], r1[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) r0[i] = r1[i] = 0.0f;
#pragma unroll
        for (int k0 = 0; k0 < RED_RUN; k0 += BATCH) {
            if (p + (size_t)k0 * stride >= P) break;
            uint4 hv[BATCH];
            float4 zv[BATCH][2];
#pragma unroll
            for (int b = 0; b < BATCH; ++b) {
                const size_t q = p + (size_t)(k0 + b) * stride;
                const bool in = q < P;
                hv[b] = in ? g[q * 8 + lane8] : make_uint4(0u, 0u, 0u, 0u);
                const float4* src = reinterpret_cast<const float4*>(z + q * CH + lane8 * 8);
                zv[b][0] = in ? src[0] : make_float4(mean[0], mean[1], mean[2], mean[3]);
                zv[b][1] = in ? src[1] : make_float4(mean[4], mean[5], mean[6], mean[7]);
            }
#pragma unroll
            for (int b = 0; b < BATCH; ++b) {
                float a[8];
                bf16x8_to_f32(hv[b], a);
                const float zz[8] = {zv[b][0].x, zv[b][0].y, zv[b][0].z, zv[b][0].w,
                                     zv[b][1].x, zv[b][1].y, zv[b][1].z, zv[b][1].w};
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const float xh = (zz[i] - mean[i]) * istd[i];
                    const float dy = (ga[i] * xh + be[i] > 0.0f) ? a[i] : 0.0f;
                    r0[i] += dy;
                    r1[i] = fmaf(dy, xh, r1[i]);
                }
            }
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            sh[0][row][lane8 * 8 + i] += (double)r0[i];
            sh[1][row][lane8 * 8 + i] += (double)r1[i];
        }
    }
    __syncthreads();
    if (threadIdx.x < 2 * CH) {
        const int k = threadIdx.x >> 6, c = threadIdx.x & 63;
        double s = 0.0;
        for (int r = 0; r < 32; ++r) s += sh[k][r][c];
        part[((size_t)blockIdx.x * 2 + k) * CH + c] = s;
    }
}

// Sum over the nblk per-block partials [nblk][2][64] of entry (k, c), by one
// warp: lane l adds blocks l, l+32, ... in order, then a fixed shuffle tree
// (the same order on every run); the result is in lane 0.
__device__ __forceinline__ double warp_partial_sum(const double* __restrict__ part, int nblk, int k, int c, int ln) {
    double s = 0.0;
    for (int b = ln; b < nblk; b += 32) s += part[((size_t)b * 2 + k) * CH + c];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(0xffffffffu, s, off);
    return s;
}

// Sums per-block channel partials [nblk][2][64] into out[nout], one warp per
// output (launched as nout / 8 blocks of 256 threads).  Optionally also as
// FP32 into lo32[c] (outputs 0..63) and hi32[c] (outputs 64..127), the
// gradient entries they are.
__global__ void __launch_bounds__(256) channel_finalize_kernel(const double* __restrict__ part, int nblk,
                                                               double* __restrict__ out, int nout,
                                                               float* __restrict__ lo32, float* __restrict__ hi32) {
    const int o = blockIdx.x * 8 + (threadIdx.x >> 5), ln = threadIdx.x & 31;
    if (o >= nout) return;
    const double s = warp_partial_sum(part, nblk, o >> 6, o & 63, ln);
    if (ln == 0) {
        out[o] = s;
        float* d32 = o < CH ? lo32 : hi32;
        if (d32) d32[o & 63] = (float)s;
    }
}

// The BatchNorm moments of one layer from the conv's per-warp partials: sums
// (sum z, sum z^2) into sums[2][64], then the batch statistics (biased
// variance) into bnp = (mean, 1/std) and the running statistics (momentum 0.1,
// unbiased variance).  One warp per channel, 8 blocks of 256 threads.
__global__ void __launch_bounds__(256) bn_moments_kernel(const double* __restrict__ part, int nblk,
                                                         double* __restrict__ sums, float* __restrict__ bnp,
                                                         float* __restrict__ rmean, float* __restrict__ rvar, double P) {
    const int c = blockIdx.x * 8 + (threadIdx.x >> 5), ln = threadIdx.x & 31;
    if (c >= CH) return;
    const double s = warp_partial_sum(part, nblk, 0, c, ln);
    const double s2 = warp_partial_sum(part, nblk, 1, c, ln);
    if (ln == 0) {
        sums[c] = s;
        sums[CH + c] = s2;
        const double mean = s / P;
        const double var = fmax(s2 / P - mean * mean, 0.0);
        bnp[c] = (float)mean;
        bnp[CH + c] = (float)(1.0 / sqrt(var + (double)BN_EPS));
        rmean[c] = (1.0f - BN_MOMENTUM) * rmean[c] + BN_MOMENTUM * (float)mean;
        rvar[c] = (1.0f - BN_MOMENTUM) * rvar[c] + BN_MOMENTUM * (float)(var * P / (P > 1 ? P - 1 : 1));
    }
}



// a = relu(gamma (z - mean) istd + beta)
// (launched with EW_BLOCKS blocks of 256 threads: a thread keeps one channel
// octet, whose parameters it loads once)
__global__ void __launch_bounds__(256) bn_apply_relu_kernel(const float* __restrict__ z, uint4* __restrict__ a,
                                                            const float* __restrict__ bnp,
                                                            const float* __restrict__ gamma,
                                                            const float* __restrict__ beta, size_t n8) {
    const size_t i0 = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    const int c0 = (int)(i0 & 7) * 8;
    float ga[8], mu[8], is[8], be[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        ga[k] = gamma[c0 + k];
        mu[k] = bnp[c0 + k];
        is[k] = bnp[CH + c0 + k];
        be[k] = beta[c0 + k];
    }
    for (size_t i = i0; i < n8; i += (size_t)gridDim.x * blockDim.x) {
        float v[8];
        f32x8_load(z + i * 8, v);
#pragma unroll
        for (int k = 0; k < 8; ++k) v[k] = fmaxf(ga[k] * (v[k] - mu[k]) * is[k] + be[k], 0.0f);
        a[i] = f32_to_bf16x8(v);
    }
}

// Per-channel sums of the BF16 values a thread stores (its channel octet):
// runs of up to 32 elements in FP32, each run added into the thread's FP64
// sums (kept in shared memory, sh[thread / 8][octet * 8 + k]); then the
// block's 32 threads of each octet are summed in thread order into
// part[block][0][64] (part[block][1][*] = 0), the layout channel_finalize_kernel
// reads.
struct OctetSums {
    double (*sh)[CH + 1];
    float run[8];
    int n;
    __device__ __forceinline__ void init(double (*shared)[CH + 1]) {
        sh = shared;
#pragma unroll
        for (int k = 0; k < 8; ++k) run[k] = 0.0f, sh[threadIdx.x >> 3][(threadIdx.x & 7) * 8 + k] = 0.0;
        n = 0;
    }
    __device__ __forceinline__ void add(uint4 v) {
        float f[8];
        bf16x8_to_f32(v, f);
#pragma unroll
        for (int k = 0; k < 8; ++k) run[k] += f[k];
        if (++n == 32) flush();
    }
    __device__ __forceinline__ void flush() {
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            sh[threadIdx.x >> 3][(threadIdx.x & 7) * 8 + k] += (double)run[k];
            run[k] = 0.0f;
        }
        n = 0;
    }
    __device__ __forceinline__ void store(double* __restrict__ part) {
        flush();
        __syncthreads();
        if (threadIdx.x < CH) {
            double t = 0.0;
            for (int r = 0; r < 32; ++r) t += sh[r][threadIdx.x];
            part[(size_t)blockIdx.x * 2 * CH + threadIdx.x] = t;
            part[(size_t)blockIdx.x * 2 * CH + CH + threadIdx.x] = 0.0;
        }
    }
};

// dz = gamma istd (dy - sum(dy)/P - xhat sum(dy xhat)/P), dy = g [y > 0].
// The per-channel factors are formed once per block (the two FP64 means
// rounded to FP32, as the element loop used them); the element loop is FP32.
// Also writes the per-block sums of the stored dz (the conv bias gradient) to
// part (OctetSums; launched with EW_BLOCKS blocks of 256 threads).
__global__ void __launch_bounds__(256) bn_bwd_apply_kernel(const uint4* __restrict__ g, const float* __restrict__ z,
                                                           uint4* __restrict__ dz, const float* __restrict__ bnp,
                                                           const float* __restrict__ gamma,
                                                           const float* __restrict__ beta,
                                                           const double* __restrict__ sums, double P, size_t n8,
                                                           double* __restrict__ part) {
    __shared__ __align__(16) float s_mean[CH], s_istd[CH], s_g[CH], s_b[CH], s_m1[CH], s_m2[CH];
    if (threadIdx.x < CH) {
        const int c = threadIdx.x;
        s_mean[c] = bnp[c];
        s_istd[c] = bnp[CH + c];
        s_g[c] = gamma[c];
        s_b[c] = beta[c];
        s_m1[c] = (float)(sums[c] / P);
        s_m2[c] = (float)(sums[CH + c] / P);
    }
    __shared__ double bsum[32][CH + 1];
    OctetSums bias;
    bias.init(bsum);
    __syncthreads();
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n8; i += (size_t)gridDim.x * blockDim.x) {
        const int c0 = (int)(i & 7) * 8;
        float gv[8], zv[8], o[8], mu[8], is[8], ga[8], be[8], m1[8], m2[8];
        bf16x8_to_f32(g[i], gv);
        f32x8_load(z + i * 8, zv);
        f32x8_load(s_mean + c0, mu);
        f32x8_load(s_istd + c0, is);
        f32x8_load(s_g + c0, ga);
        f32x8_load(s_b + c0, be);
        f32x8_load(s_m1 + c0, m1);
        f32x8_load(s_m2 + c0, m2);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            const float xh = (zv[k] - mu[k]) * is[k];
            const float dy = (ga[k] * xh + be[k] > 0.0f) ? gv[k] : 0.0f;
            o[k] = ga[k] * is[k] * (dy - m1[k] - xh * m2[k]);
        }
        const uint4 v = f32_to_bf16x8(o);
        dz[i] = v;
        bias.add(v);
    }
    bias.store(part);
}

// dz = g * [a > 0] (layer 1: ReLU without BatchNorm); per-block sums of dz
// (the conv bias gradient) to part as in bn_bwd_apply_kernel.
__global__ void __launch_bounds__(256) relu_bwd_kernel(const uint4* __restrict__ g, const uint4* __restrict__ a,
                                                       uint4* __restrict__ dz, size_t n8, double* __restrict__ part) {
    __shared__ double bsum[32][CH + 1];
    OctetSums bias;
    bias.init(bsum);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n8; i += (size_t)gridDim.x * blockDim.x) {
        float gv[8], av[8];
        bf16x8_to_f32(g[i], gv);
        bf16x8_to_f32(a[i], av);
#pragma unroll
        for (int k = 0; k < 8; ++k) gv[k] = av[k] > 0.0f ? gv[k] : 0.0f;
        const uint4 v = f32_to_bf16x8(gv);
        dz[i] = v;
        bias.add(v);
    }
    bias.store(part);
}

// out = centre - R; loss partials of (out - clean)^2; dR = -2 (out - clean)/P.
__global__ void __launch_bounds__(256) loss_kernel(const float* __restrict__ x, const float* __restrict__ clean,
                                                   const float* __restrict__ R, float* __restrict__ dR, int B, int H,
                                                   int W, double* __restrict__ part) {
    const size_t P = (size_t)B * H * W, HW = (size_t)H * W;
    const float scale = (float)(2.0 / (double)P);
    double s = 0.0;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const size_t img = p / HW, r = p % HW;
        const float centre = x[(img * FRAMES + 2) * HW + r];
        const float d = centre - R[p] - clean[p];
        dR[p] = -scale * d;
        s += (double)d * d;
    }
    s = block_sum_f64(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void loss_finalize_kernel(const double* __restrict__ part, int n, double P, double* __restrict__ loss) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_sum_f64(s);
    if (threadIdx.x == 0) *loss = s / P;
}

// Input gradient of the last layer (64 -> 1): da[p][ci] = sum_tap W[ci][tap] dR[p - off(tap)].
__global__ void last_dgrad_kernel(const float* __restrict__ dR, const float* __restrict__ params, size_t w_off,
                                  uint4* __restrict__ da, int B, int H, int W) {
    __shared__ float w[CH * 9];
    for (int i = threadIdx.x; i < CH * 9; i += blockDim.x) w[i] = params[w_off + i];   // [0][ci][ky][kx]
    __syncthreads();
    const size_t P = (size_t)B * H * W;
    for (size_t p = blockIdx.x * (size_t)blockDim.x + threadIdx.x; p < P; p += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(p % W), a = (int)((p / W) % H);
        const size_t base = p - (size_t)a * W - b;
        float d[9];
#pragma unroll
        for (int tap = 0; tap < 9; ++tap) {
            const int aa = a - (tap / 3 - 1), bb = b - (tap % 3 - 1);
            d[tap] = (aa >= 0 && aa < H && bb >= 0 && bb < W) ? dR[base + (size_t)aa * W + bb] : 0.0f;
        }
#pragma unroll
        for (int c8 = 0; c8 < 8; ++c8) {
            float o[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                float s = 0.0f;
#pragma unroll
                for (int tap = 0; tap < 9; ++tap) s += w[(c8 * 8 + k) * 9 + tap] * d[tap];
                o[k] = s;
            }
            da[p * 8 + c8] = f32_to_bf16x8(o);
        }
    }
}

// Sums weight-gradient partials over chunks into the flat gradient layout.
// layer 0: grad[w0 + co*45 + k] for k < 45; hidden: grad[w + (co*64 + ci)*9 + tap].
__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int nchunks, int taps, int layer0,
                                    float* __restrict__ grad) {
    const int n = taps * CH * CH;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        const int tap = e / (CH * CH), co = (e / CH) % CH, ci = e % CH;
        float s = 0.0f;
        for (int c = 0; c < nchunks; ++c) s += part[((size_t)c * 9 + tap) * CH * CH + co * CH + ci];
        if (layer0) {
            if (ci < FRAMES * 9) grad[co * FRAMES * 9 + ci] = s;
        } else {
            grad[((size_t)co * CH + ci) * 9 + tap] = s;
        }
    }
}

// Last layer weight gradient: part[chunk][tap][ci] = sum_p dR[p] act[p + off(tap)][ci].
__global__ void __launch_bounds__(256) wgrad_last_kernel(const float* __restrict__ dR, const uint4* __restrict__ act,
                                                         float* __restrict__ part, int B, int H, int W) {
    const int tap = blockIdx.x, chunk = blockIdx.y;
    const int dy = tap / 3 - 1, dx = tap % 3 - 1;
    const size_t P = (size_t)B * H * W;
    const size_t p_lo = (size_t)chunk * WG_CHUNK;
    const size_t p_hi = p_lo + WG_CHUNK < P ? p_lo + WG_CHUNK : P;
    const int lane8 = threadIdx.x & 7, row = threadIdx.x >> 3;    // 32 pixel rows x 8 channel groups
    float acc[8] = {};
    for (size_t p = p_lo + row; p < p_hi; p += 32) {
        const int b = (int)(p % W), a = (int)((p / W) % H);
        const int aa = a + dy, bb = b + dx;
        if (aa < 0 || aa >= H || bb < 0 || bb >= W) continue;
        float u[8];
        bf16x8_to_f32(act[(p + (ptrdiff_t)dy * W + dx) * 8 + lane8], u);
        const float d = dR[p];
#pragma unroll
        for (int k = 0; k < 8; ++k) acc[k] = fmaf(d, u[k], acc[k]);
    }
    // reduce the 32 rows through shared memory
    __shared__ float red[32][CH + 1];
#pragma unroll
    for (int k = 0; k < 8; ++k) red[row][lane8 * 8 + k] = acc[k];
    __syncthreads();
    if (threadIdx.x < CH) {
        float s = 0.0f;
        for (int r = 0; r < 32; ++r) s += red[r][threadIdx.x];
        part[((size_t)chunk * 9 + tap) * CH + threadIdx.x] = s;
    }
}

__global__ void wgrad_last_reduce_kernel(const float* __restrict__ part, int nchunks, float* __restrict__ grad) {
    const int e = threadIdx.x + blockIdx.x * blockDim.x;   // tap*64 + ci
    if (e >= 9 * CH) return;
    const int tap = e / CH, ci = e % CH;
    float s = 0.0f;
    for (int c = 0; c < nchunks; ++c) s += part[((size_t)c * 9 + tap) * CH + ci];
    grad[ci * 9 + tap] = s;
}

__global__ void sum_f32_kernel(const float* __restrict__ x, size_t n, double* __restrict__ part) {
    double s = 0.0;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) s += x[i];
    s = block_sum_f64(s);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void store_sum_kernel(const double* __restrict__ part, int n, float* __restrict__ out) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += part[i];
    s = block_sum_f64(s);
    if (threadIdx.x == 0) *out = (float)s;
}

// Adam (Kingma & Ba 2015) with bias correction: c1 = 1/(1-b1^t), c2 = 1/(1-b2^t).
__global__ void adam_kernel(float* __restrict__ theta, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, size_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2, const uint8_t* __restrict__ frozen) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        if (frozen[i]) continue;
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

// ---------------------------------------------------------------- training pairs

__device__ __forceinline__ uint64_t mix64(uint64_t z) {   // SplitMix64 finaliser (Steele et al. 2014)
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float u01(uint64_t h) { return ((h >> 40) + 0.5f) * (1.0f / 16777216.0f); }

// Patch p of the batch: a random frame of the phantom stack, a random slicing
// axis (the 5 channels are 5 adjacent slices along it, standing in for time),
// a random slice, a random 2D position, a random flip / transpose, and a noise
// level sigma ~ U[lo, hi].  Noisy channels get independent N(0, sigma^2) noise
// (Box-Muller on counter-based hashes); the target is the clean centre slice.
__global__ void training_batch_kernel(const float* __restrict__ vol, int nx, int ny, int nz, int nframes, int B,
                                      int Hp, int Wp, float s_lo, float s_hi, uint64_t seed, float* __restrict__ noisy,
                                      float* __restrict__ clean) {
    const size_t per = (size_t)FRAMES * Hp * Wp;
    const size_t total = per * B;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
        const int bi = (int)(e / per);
        const int c = (int)((e / ((size_t)Hp * Wp)) % FRAMES);
        const int i = (int)((e / Wp) % Hp), j = (int)(e % Wp);
        const uint64_t h0 = mix64(seed ^ (0x1234567ull + (uint64_t)bi * 0x9E3779B97F4A7C15ull));
        const uint64_t h1 = mix64(h0), h2 = mix64(h1), h3 = mix64(h2), h4 = mix64(h3), h5 = mix64(h4);
        const int frame = (int)(u01(h0) * nframes) % nframes;
        const int axis = (int)(u01(h1) * 3) % 3;           // 0: slices along z, 1: along x, 2: along y
        const int flips = (int)(h2 & 7);
        const float sigma = s_lo + (s_hi - s_lo) * u01(h5);
        int S, A, Bd;                                       // slices, rows, cols of the chosen plane
        if (axis == 0) { S = nz; A = ny; Bd = nx; } else if (axis == 1) { S = nx; A = nz; Bd = ny; } else { S = ny; A = nx; Bd = nz; }
        const int s = (int)(u01(h3) * S) % S;
        const int a0 = (int)(u01(h4) * (A - Hp + 1)) % (A - Hp + 1);
        const int b0 = (int)(u01(mix64(h5)) * (Bd - Wp + 1)) % (Bd - Wp + 1);
        int ii = i, jj = j;
        if (flips & 1) ii = Hp - 1 - ii;
        if (flips & 2) jj = Wp - 1 - jj;
        if ((flips & 4) && Hp == Wp) { const int tt = ii; ii = jj; jj = tt; }
        const int sc = min(max(s + c - 2, 0), S - 1);
        const int a = a0 + ii, b = b0 + jj;
        size_t idx;
        if (axis == 0) idx = ((size_t)sc * ny + a) * nx + b;
        else if (axis == 1) idx = ((size_t)a * ny + b) * nx + sc;
        else idx = ((size_t)b * ny + sc) * nx + a;
        const float v = vol[(size_t)frame * nx * ny * nz + idx];
        const uint64_t hn = mix64(seed + 0xD1B54A32D192ED03ull * (e + 1));
        const float u1 = u01(hn), u2 = u01(mix64(hn));
        const float gauss = sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
        noisy[e] = v + sigma * gauss;
        if (c == 2) clean[((size_t)bi * Hp + i) * Wp + j] = v;
    }
}

}  // namespace cnn
}  // namespace msf

static msf_status trace_alloc(msf_cnn* c);


extern "C" msf_status msf_cnn_train_reserve(msf_cnn* c, int64_t max_train_pixels) {
    MSF_REQUIRE(c, "msf_cnn_train_reserve: NULL handle");
    MSF_REQUIRE(max_train_pixels >= 128 && max_train_pixels <= ((int64_t)1 << 28),
                "msf_cnn_train_reserve: need 128 to 2^28 pixels, got %lld", (long long)max_train_pixels);
    if (max_train_pixels <= c->train_cap) return MSF_OK;
    cudaFree(c->train_ws);
    c->train_ws = nullptr;
    c->train_cap = 0;
    const size_t bytes = train_layout(max_train_pixels, nullptr, nullptr);
    if (cudaMalloc(&c->train_ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(MSF_ERR_NOMEM, "msf_cnn_train_reserve: cannot allocate %zu bytes", bytes);
    }
    c->train_ws_bytes = bytes;
    c->train_cap = max_train_pixels;
    return trace_alloc(c);
}

extern "C" msf_status msf_cnn_get_grads(msf_cnn* c, float* h_grads, size_t n) {
    MSF_REQUIRE(c && h_grads, "msf_cnn_get_grads: NULL argument");
    MSF_REQUIRE(n == c->off.total, "msf_cnn_get_grads: expected %zu values, got %zu", c->off.total, n);
    MSF_TRY_CUDA(cudaDeviceSynchronize());
    MSF_TRY_CUDA(cudaMemcpy(h_grads, c->d_grad, n * 4, cudaMemcpyDeviceToHost));
    return MSF_OK;
}

extern "C" msf_status msf_training_batch(const float* d_vol, const msf_vol* vol, int B, int H, int W, double sigma_lo,
                                         double sigma_hi, uint64_t seed, float* d_noisy, float* d_clean, void* stream) {
    MSF_REQUIRE(d_vol && vol && d_noisy && d_clean, "msf_training_batch: NULL argument");
    MSF_REQUIRE(B > 0 && H > 0 && W > 0, "msf_training_batch: empty batch");
    MSF_REQUIRE(H <= vol->nx && H <= vol->ny && H <= vol->nz && W <= vol->nx && W <= vol->ny && W <= vol->nz,
                "msf_training_batch: patch larger than the volume");
    MSF_REQUIRE(sigma_lo >= 0 && sigma_hi >= sigma_lo, "msf_training_batch: need 0 <= sigma_lo <= sigma_hi");
    cudaStream_t st = as_stream(stream);
    MSF_PROF("training_batch", st);
    training_batch_kernel<<<EW_BLOCKS, 256, 0, st>>>(d_vol, vol->nx, vol->ny, vol->nz, vol->nt, B, H, W, (float)sigma_lo,
                                                   (float)sigma_hi, seed, d_noisy, d_clean);
    MSF_LAUNCH_CHECK();
    return MSF_OK;
}

enum TraceKind { TRACE_DZ = 0, TRACE_DA = 1 };

// Slot of the trace buffer: dz of layer l (0..8) in slots 0..8, da of layer l
// (1..9) in slots 9..17; each slot holds trace_cap pixels x 64 BF16.
static __nv_bfloat16* trace_slot(msf_cnn* c, int kind, int l) {
    const int slot = kind == TRACE_DZ ? l : 8 + l;
    return c->trace + (size_t)slot * c->trace_cap * CH;
}

static msf_status trace_record(msf_cnn* c, int kind, int l, const __nv_bfloat16* src, int64_t P, cudaStream_t st) {
    if (!c->trace_on || !c->trace) return MSF_OK;
    MSF_TRY_CUDA(cudaMemcpyAsync(trace_slot(c, kind, l), src, (size_t)P * CH * 2, cudaMemcpyDeviceToDevice, st));
    return MSF_OK;
}

static msf_status trace_alloc(msf_cnn* c) {
    cudaFree(c->trace);
    c->trace = nullptr;
    c->trace_cap = 0;
    if (!c->trace_on || c->train_cap == 0) return MSF_OK;
    if (cudaMalloc(&c->trace, (size_t)18 * c->train_cap * CH * 2) != cudaSuccess) {
        cudaGetLastError();
        c->trace_on = false;
        return fail(MSF_ERR_NOMEM, "msf_cnn_train_trace: cannot allocate the trace");
    }
    c->trace_cap = c->train_cap;
    return MSF_OK;
}

extern "C" msf_status msf_cnn_train_trace(msf_cnn* c, int on) {
    MSF_REQUIRE(c, "msf_cnn_train_trace: NULL handle");
    MSF_REQUIRE(!on || c->train_cap > 0, "msf_cnn_train_trace: call msf_cnn_train_reserve first");
    c->trace_on = on != 0;
    return trace_alloc(c);
}

extern "C" msf_status msf_cnn_train_tensor(msf_cnn* c, int kind, int layer, void* h_dst, size_t bytes) {
    MSF_REQUIRE(c && h_dst, "msf_cnn_train_tensor: NULL argument");
    MSF_REQUIRE(c->last_P > 0 && c->train_ws, "msf_cnn_train_tensor: no training step has run");
    TrainWS w;
    train_layout(c->train_cap, &w, (uint8_t*)c->train_ws);
    const size_t P = (size_t)c->last_P;
    const void* src = nullptr;
    size_t need = 0;
    switch (kind) {
        case MSF_TT_ACT:
            MSF_REQUIRE(layer >= 1 && layer <= 9, "msf_cnn_train_tensor: activation layer %d not in 1..9", layer);
            src = w.act[layer]; need = P * CH * 2; break;
        case MSF_TT_Z:
            MSF_REQUIRE(layer >= 1 && layer <= 8, "msf_cnn_train_tensor: pre-BatchNorm layer %d not in 1..8", layer);
            src = w.z[layer]; need = P * CH * 4; break;
        case MSF_TT_DZ:
        case MSF_TT_DA:
            MSF_REQUIRE(c->trace_on && c->trace, "msf_cnn_train_tensor: gradients need msf_cnn_train_trace(c, 1) "
                                                 "before the step");
            MSF_REQUIRE(kind == MSF_TT_DZ ? (layer >= 0 && layer <= 8) : (layer >= 1 && layer <= 9),
                        "msf_cnn_train_tensor: gradient layer %d out of range", layer);
            src = trace_slot(c, kind == MSF_TT_DZ ? TRACE_DZ : TRACE_DA, layer); need = P * CH * 2; break;
        case MSF_TT_R: src = w.R; need = P * 4; break;
        case MSF_TT_DR: src = w.dR; need = P * 4; break;
        case MSF_TT_BN:
            MSF_REQUIRE(layer >= 1 && layer <= 8, "msf_cnn_train_tensor: BatchNorm layer %d not in 1..8", layer);
            src = w.bnp + (size_t)(layer - 1) * 2 * CH; need = 2 * CH * 4; break;
        default:
            return fail(MSF_ERR_ARG, "msf_cnn_train_tensor: unknown kind %d", kind);
    }
    MSF_REQUIRE(bytes == need, "msf_cnn_train_tensor: expected %zu bytes, got %zu", need, bytes);
    MSF_TRY_CUDA(cudaDeviceSynchronize());
    MSF_TRY_CUDA(cudaMemcpy(h_dst, src, need, cudaMemcpyDeviceToHost));
    return MSF_OK;
}

extern "C" msf_status msf_train_step(msf_cnn* c, const float* d_noisy, const float* d_clean, int B, int H, int W,
                                     float lr, float* h_loss, void* stream) {
    MSF_REQUIRE(c && d_noisy && d_clean, "msf_train_step: NULL argument");
    MSF_REQUIRE(B > 0 && H > 0 && W > 0, "msf_train_step: empty batch");
    const int64_t P = (int64_t)B * H * W;
    MSF_REQUIRE(P <= c->train_cap,
                "msf_train_step: batch of %lld pixels exceeds the reserved training workspace (%lld); "
                "call msf_cnn_train_reserve first", (long long)P, (long long)c->train_cap);
    MSF_REQUIRE(lr > 0, "msf_train_step: lr must be positive");
    cudaStream_t st = as_stream(stream);
    TrainWS w;
    train_layout(c->train_cap, &w, (uint8_t*)c->train_ws);
    const Offsets& o = c->off;
    const size_t n8 = (size_t)P * 8;
    const int nchunks = (int)((P + WG_CHUNK - 1) / WG_CHUNK);

    // weights of this step: forward (no folding) and input-gradient kernels
    size_t wf_off[LAYERS], wp = 0;
    for (int l = 0; l < LAYERS; ++l) { wf_off[l] = wp; wp += (size_t)taps_of(l) * rows_of(l) * KPACK; }
    {
        MSF_PROF("train_pack_weights", st);
        for (int l = 0; l < LAYERS; ++l) {
            FoldArgs f;
            f.layer = l; f.taps = taps_of(l); f.rows = rows_of(l); f.cin = cin_of(l); f.cout = cout_of(l);
            f.w = (long long)o.w[l]; f.b = (long long)o.b[l];
            f.gamma = f.beta = f.mean = f.var = -1;
            fold_kernel<<<64, 256, 0, st>>>(c->d_params, w.wf + wf_off[l], w.bf + l * CH, f);
        }
        pack_dgrad_kernel<<<256, 256, 0, st>>>(c->d_params, w.wb, o);
        MSF_LAUNCH_CHECK();
        MSF_TRY_CUDA(cudaMemsetAsync(w.zeros, 0, CH * 4, st));
    }
    CUtensorMap m16[LAYERS], m18[LAYERS], m4[LAYERS], g16[2], g18[2], g4[2], mw[LAYERS], mb[8], f4[LAYERS - 1];
    for (int l = 1; l < LAYERS - 1; ++l) MSF_TRY(make_f32_out_map(&f4[l], w.z[l], B, H, W));
    for (int l = 0; l < LAYERS; ++l) {
        MSF_TRY(make_act_map(&m16[l], w.act[l], B, H, W, TILE_A));
        MSF_TRY(make_act_map(&m18[l], w.act[l], B, H, W, TILE_A + 2));
        MSF_TRY(make_act_map(&m4[l], w.act[l], B, H, W, TILE_A / 4));
        MSF_TRY(make_w_map(&mw[l], w.wf + wf_off[l], taps_of(l) * rows_of(l), rows_of(l)));
    }
    for (int k = 0; k < 2; ++k) {
        MSF_TRY(make_act_map(&g16[k], w.g[k], B, H, W, TILE_A));
        MSF_TRY(make_act_map(&g18[k], w.g[k], B, H, W, TILE_A + 2));
        MSF_TRY(make_act_map(&g4[k], w.g[k], B, H, W, TILE_A / 4));
    }
    for (int l = 0; l < 8; ++l) MSF_TRY(make_w_map(&mb[l], w.wb + (size_t)l * 9 * CH * CH, 9 * CH, CH));
    TileGeom tg;
    tg.H = H; tg.W = W; tg.imgs = B;
    tg.tiles_a = (H + TILE_A - 1) / TILE_A;
    tg.tiles_b = (W + TILE_B - 1) / TILE_B;
    tg.total = B * tg.tiles_a * tg.tiles_b;
    SliceGeom sg{};
    MSF_TRY(ensure_kernel_attrs());
    // weight-gradient CTAs: one per SM (at most WG_MAX_CTAS), none without a tile
    int wg_ctas = g_num_sms < WG_MAX_CTAS ? g_num_sms : WG_MAX_CTAS;
    if (wg_ctas > tg.total) wg_ctas = tg.total;
    const int nred = w.nred;
    // CTAs of the persistent 16 x 8 convs (as launch_conv sizes them)
    const int conv_grid = tg.total < g_num_sms ? tg.total : g_num_sms;
    // the BatchNorm backward's two channel sums of layer l into out[2][64]
    auto bn_bwd_sums = [&](const __nv_bfloat16* g, const float* z, const float* bnp, const float* ga, const float* be,
                           double* out, float* lo32, float* hi32) -> msf_status {
        {
            MSF_PROF("train_reduce", st);
            bn_bwd_reduce_kernel<<<nred, 256, 0, st>>>((const uint4*)g, z, bnp, ga, be, P, w.part);
            MSF_LAUNCH_CHECK();
        }
        MSF_PROF("train_reduce_finalize", st);
        channel_finalize_kernel<<<2 * CH / 8, 256, 0, st>>>(w.part, nred, out, 2 * CH, lo32, hi32);
        MSF_LAUNCH_CHECK();
        return MSF_OK;
    };

    // ---------------- forward
    {
        MSF_PROF("train_pack_input", st);
        pack_batch_kernel<<<EW_BLOCKS, 256, 0, st>>>(d_noisy, (uint4*)w.act[0], B, H, W);
        MSF_LAUNCH_CHECK();
    }
    MSF_TRY((launch_conv<1, 64, NS_1X1, EPI_RELU>(m16[0], mw[0], m4[1], w.bf, tg, sg, nullptr, nullptr, c->d_err, st)));
    for (int l = 1; l <= 8; ++l) {
        // the conv also sums the BatchNorm moments of its outputs, per epilogue warp
        MSF_TRY((launch_conv<9, 64, NS_3X3, EPI_RAW32>(m18[l], mw[l], f4[l], w.bf + l * CH, tg, sg, nullptr, w.z[l],
                                                      c->d_err, st, w.part)));
        double* sums = w.sums + (size_t)(l - 1) * 4 * CH;
        float* bnp = w.bnp + (size_t)(l - 1) * 2 * CH;
        {
            MSF_PROF("train_bn_stats", st);
            bn_moments_kernel<<<CH / 8, 256, 0, st>>>(w.part, 4 * conv_grid, sums, bnp, c->d_params + o.mean[l],
                                                      c->d_params + o.var[l], (double)P);
            MSF_LAUNCH_CHECK();
        }
        {
            MSF_PROF("train_bn_apply", st);
            bn_apply_relu_kernel<<<EW_BLOCKS, 256, 0, st>>>(w.z[l], (uint4*)w.act[l + 1], bnp,
                                                          c->d_params + o.gamma[l], c->d_params + o.beta[l], n8);
            MSF_LAUNCH_CHECK();
        }
    }
    MSF_TRY((launch_conv<9, 16, NS_LAST, EPI_F32>(m18[9], mw[9], m4[9], w.bf + 9 * CH, tg, sg, nullptr, w.R, c->d_err, st)));
    {
        MSF_PROF("train_loss", st);
        loss_kernel<<<nred, 256, 0, st>>>(d_noisy, d_clean, w.R, w.dR, B, H, W, w.part);
        loss_finalize_kernel<<<1, 256, 0, st>>>(w.part, nred, (double)P, w.loss);
        MSF_LAUNCH_CHECK();
    }
    // ---------------- backward
    {
        MSF_PROF("train_last_bwd", st);
        last_dgrad_kernel<<<EW_BLOCKS, 256, 0, st>>>(w.dR, c->d_params, o.w[9], (uint4*)w.g[0], B, H, W);
        MSF_TRY(trace_record(c, TRACE_DA, 9, w.g[0], P, st));
        wgrad_last_kernel<<<dim3(9, nchunks), 256, 0, st>>>(w.dR, (const uint4*)w.act[9], w.wpart, B, H, W);
        wgrad_last_reduce_kernel<<<(9 * CH + 255) / 256, 256, 0, st>>>(w.wpart, nchunks, c->d_grad + o.w[9]);
        sum_f32_kernel<<<nred, 256, 0, st>>>(w.dR, (size_t)P, w.part);
        store_sum_kernel<<<1, 256, 0, st>>>(w.part, nred, c->d_grad + o.b[9]);
        MSF_LAUNCH_CHECK();
    }
    int cur = 0;   // w.g[cur] holds the gradient w.r.t. act[l + 1]
    for (int l = 8; l >= 1; --l) {
        double* sums = w.sums + (size_t)(l - 1) * 4 * CH;
        float* bnp = w.bnp + (size_t)(l - 1) * 2 * CH;
        const float* ga = c->d_params + o.gamma[l];
        const float* be = c->d_params + o.beta[l];
        // d beta = sum dy, d gamma = sum dy xhat
        MSF_TRY(bn_bwd_sums(w.g[cur], w.z[l], bnp, ga, be, sums + 2 * CH, c->d_grad + o.beta[l], c->d_grad + o.gamma[l]));
        {
            MSF_PROF("train_bn_bwd", st);
            bn_bwd_apply_kernel<<<EW_BLOCKS, 256, 0, st>>>((const uint4*)w.g[cur], w.z[l], (uint4*)w.g[cur ^ 1], bnp,
                                                           ga, be, sums + 2 * CH, (double)P, n8, w.part);
            MSF_LAUNCH_CHECK();
        }
        MSF_TRY(trace_record(c, TRACE_DZ, l, w.g[cur ^ 1], P, st));
        // dz in g[cur ^ 1]: conv bias grad (its block sums came with dz), weight grad, input grad
        {
            MSF_PROF("train_reduce_finalize", st);
            channel_finalize_kernel<<<CH / 8, 256, 0, st>>>(w.part, EW_BLOCKS, sums, CH, c->d_grad + o.b[l], nullptr);
            MSF_LAUNCH_CHECK();
        }
        {
            MSF_PROF("wgrad_tc", st);
            wgrad_tc_kernel<9><<<wg_ctas, THREADS, WG_SMEM, st>>>(m18[l], g16[cur ^ 1], w.wpart, tg, c->d_err);
            MSF_LAUNCH_CHECK();
        }
        {
            MSF_PROF("wgrad_reduce", st);
            wgrad_reduce_kernel<<<144, 256, 0, st>>>(w.wpart, wg_ctas, 9, 0, c->d_grad + o.w[l]);
            MSF_LAUNCH_CHECK();
        }
        MSF_TRY((launch_conv<9, 64, NS_3X3, EPI_RAW>(g18[cur ^ 1], mb[l - 1], g4[cur], w.zeros, tg, sg, nullptr, nullptr,
                                               c->d_err, st)));
        // g[cur] now holds the gradient w.r.t. act[l]
        MSF_TRY(trace_record(c, TRACE_DA, l, w.g[cur], P, st));
    }
    {
        MSF_PROF("train_first_bwd", st);
        relu_bwd_kernel<<<EW_BLOCKS, 256, 0, st>>>((const uint4*)w.g[cur], (const uint4*)w.act[1], (uint4*)w.g[cur ^ 1],
                                                   n8, w.part);
        MSF_LAUNCH_CHECK();
    }
    MSF_TRY(trace_record(c, TRACE_DZ, 0, w.g[cur ^ 1], P, st));
    {
        MSF_PROF("train_reduce_finalize", st);
        channel_finalize_kernel<<<CH / 8, 256, 0, st>>>(w.part, EW_BLOCKS, w.sums, CH, c->d_grad + o.b[0], nullptr);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("wgrad_tc", st);
        wgrad_tc_kernel<1><<<wg_ctas, THREADS, WG_SMEM, st>>>(m16[0], g16[cur ^ 1], w.wpart, tg, c->d_err);
        MSF_LAUNCH_CHECK();
    }
    {
        MSF_PROF("wgrad_reduce", st);
        wgrad_reduce_kernel<<<16, 256, 0, st>>>(w.wpart, wg_ctas, 1, 1, c->d_grad + o.w[0]);
        MSF_LAUNCH_CHECK();
    }
    // ---------------- Adam on everything except the running statistics
    c->adam_t += 1;
    const double c1 = 1.0 / (1.0 - pow(0.9, (double)c->adam_t));
    const double c2 = 1.0 / (1.0 - pow(0.999, (double)c->adam_t));
    {
        MSF_PROF("train_adam", st);
        adam_kernel<<<152 * 4, 256, 0, st>>>(c->d_params, c->d_grad, c->d_m, c->d_v, o.total, lr, 0.9f, 0.999f, 1e-8f,
                                             (float)c1, (float)c2, c->d_frozen);
        MSF_LAUNCH_CHECK();
    }
    c->folded = false;
    c->gen += 1;
    c->last_P = P;
    if (h_loss) {
        double l = 0.0;
        MSF_TRY_CUDA(cudaMemcpyAsync(&l, w.loss, 8, cudaMemcpyDeviceToHost, st));
        MSF_TRY_CUDA(cudaStreamSynchronize(st));
        int herr = 0;
        MSF_TRY_CUDA(cudaMemcpy(&herr, c->d_err, sizeof(int), cudaMemcpyDeviceToHost));
        if (herr) return fail((msf_status)herr, "msf_train_step: a device-side wait timed out");
        if (!isfinite(l)) return fail(MSF_ERR_NUMERIC, "msf_train_step: non-finite loss");
        *h_loss = (float)l;
    }
    return MSF_OK;
}

// ====================================================================== hooks for the MACE orchestration

uint64_t msf::cnn_generation(const msf_cnn* c) { return c ? c->gen : 0; }

// Everything msf_denoise does outside stream order, done ahead of a graph
// capture: kernel attributes, the SM count, and the folding of the weights.
msf_status msf::cnn_prepare(msf_cnn* c, cudaStream_t st) {
    if (!c) return MSF_OK;
    MSF_TRY(ensure_kernel_attrs());
    if (!c->folded) MSF_TRY(fold_all(c, st));
    return MSF_OK;
}

// ====================================================================== failure detection self-test

namespace msf {
namespace cnn {
// Waits on an mbarrier that nothing ever completes, with the same bounded wait
// the conv kernels use; must give up after limit_ns and report a timeout.
__global__ void wait_selftest_kernel(uint64_t limit_ns, int* status) {
    __shared__ uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        abort_flag = 0;
        tc::fence_mbar_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool ok = tc::mbar_wait(&bar, 0, &abort_flag, limit_ns);
        *status = ok ? (int)MSF_OK : (int)MSF_ERR_TIMEOUT;
    }
}
}  // namespace cnn
}  // namespace msf

extern "C" msf_status msf_selftest_wait(uint64_t limit_ns, void* stream) {
    MSF_REQUIRE(limit_ns > 0 && limit_ns <= 2000000000ull, "msf_selftest_wait: limit must be in (0, 2 s]");
    MSF_TRY(check_device());
    cudaStream_t st = as_stream(stream);
    int* d_status = nullptr;
    int h = -1;
    MSF_TRY_CUDA(cudaMalloc(&d_status, sizeof(int)));
    cudaError_t e = cudaMemsetAsync(d_status, 0xff, sizeof(int), st);
    if (e == cudaSuccess) {
        wait_selftest_kernel<<<1, 32, 0, st>>>(limit_ns, d_status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_status);
    if (e != cudaSuccess) return fail(MSF_ERR_CUDA, "msf_selftest_wait: %s", cudaGetErrorString(e));
    if (h == (int)MSF_ERR_TIMEOUT) return fail(MSF_ERR_TIMEOUT, "msf_selftest_wait: the bounded wait gave up as designed");
    return (msf_status)h;
}
