// Kernels of the learned connectivity estimator: an MLP in -> 256 -> 256 -> 1
// (ReLU hidden layers, sigmoid output, binary cross-entropy), BF16 tensor-core
// GEMMs (tcgen05, FP32 accumulation in tensor memory), FP32 master weights, AdamW.
//
// Precision (mirrored by the FP64 oracle): inputs, weight copies, the first hidden
// activation and the backward activations dH2, dH1 are BF16; every accumulation is
// FP32; the second hidden activation, the output layer and all reductions are FP32.
// Every reduction runs in a fixed order (per-CTA partials summed in CTA order), so
// a result does not depend on scheduling.
//
// One training step is four launches:
//   k_tile   per 128-row tile of the batch: the forward pass (X W1, H1 W2 on the
//            tensor cores), the output layer and loss, dH2 and dH1 = dH2 W2^T, with
//            the per-tile column sums of the bias and output-layer gradients; it
//            writes the batch-major (transposed) operands of the weight gradients
//            in the shared-memory image the next kernel copies in one piece;
//   k_wgrad  dW2 = H1^T dH2 and dW1^T = dH1^T X split over the batch (fixed-order
//            partials), operands brought in by bulk asynchronous copies;
//   k_update the partials summed in order, AdamW on the FP32 masters, and the BF16
//            weight images the tile kernel streams;
//   k_epoch_tail (replayed epochs) the loss of the step and the batch cursor.
//
// Shared-memory operand layout (tcgen05 K-major, no swizzle): a matrix of R rows x 64
// K-elements is a chunk of core matrices of 8 rows x 16 bytes; element (r, c) sits at
// byte (r / 8) 1024 + (c / 8) 128 + (r % 8) 16 + (c % 8) 2 (LBO 128 B along K, SBO
// 1024 B along rows).  Weights and the transposed activations are kept in global
// memory in exactly this image, so one 1D bulk copy lands a chunk.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "ptx.cuh"

namespace gn {
namespace {

constexpr int kH = kMlpHidden;   // 256
constexpr int kKP = kMlpInPad;   // 64
constexpr int kBM = 128;         // batch rows per tile
constexpr uint32_t kWChunk = 256u * 64u * 2u;  // one weight chunk: 256 rows x 64 K, BF16 (32 KB)

__host__ __device__ constexpr uint32_t img_off(uint32_t r, uint32_t c)
{
    return (r >> 3) * 1024u + (c >> 3) * 128u + (r & 7u) * 16u + (c & 7u) * 2u;
}

__device__ __forceinline__ int64_t batch_row(const int64_t *idx, const int64_t *cursor, int B, int64_t r)
{
    if (!idx) return r;
    return idx[(cursor ? *cursor * B : 0) + r];
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b)
{
    const __nv_bfloat162 pr = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&pr);
}

// 32 columns (c0 .. c0 + 31) of this thread's row as BF16 into a K-major operand of
// 128 rows held as chunks of 64 K-elements (16 KB apart).
__device__ __forceinline__ void put_row32(uint8_t *op, int row, int c0, const float (&v)[32])
{
    uint8_t *base = op + (c0 >> 6) * 16384 + (row >> 3) * 1024 + (row & 7) * 16 + ((c0 & 63) >> 3) * 128;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 u = make_uint4(pack_bf16(v[8 * q], v[8 * q + 1]), pack_bf16(v[8 * q + 2], v[8 * q + 3]),
                                   pack_bf16(v[8 * q + 4], v[8 * q + 5]), pack_bf16(v[8 * q + 6], v[8 * q + 7]));
        *reinterpret_cast<uint4 *>(base + q * 128) = u;
    }
}

// The warp's 32 rows x 32 features (f0 .. f0 + 31) as BF16 into the batch-major image
// of a weight-gradient operand: rows = features, K = the 64 batch rows of a chunk.
// `chunk` points at the 64-row chunk's image (feature f, batch row m at img_off(f, m));
// mrow0 = the first of the warp's rows within that chunk (0 or 32).  Through a
// per-warp staging tile so each lane stores 16 contiguous bytes (8 rows of one
// feature) and 8 lanes cover 128 contiguous bytes.
__device__ __forceinline__ void put_cols32(uint8_t *chunk, int f0, int mrow0, const float (&v)[32], uint16_t *stage,
                                           int lane)
{
    constexpr int kPitch = 40;  // uint16 per staging row: 32 rows + 8 pad (80 B, 16-byte aligned)
#pragma unroll
    for (int j = 0; j < 32; ++j)
        stage[j * kPitch + lane] = __bfloat16_as_ushort(__float2bfloat16_rn(v[j]));
    __syncwarp();
#pragma unroll
    for (int it = 0; it < 4; ++it) {
        const int f = 8 * it + (lane & 7), g = lane >> 3;  // feature, group of 8 rows
        const uint4 u = *reinterpret_cast<const uint4 *>(stage + f * kPitch + 8 * g);
        *reinterpret_cast<uint4 *>(chunk + img_off(f0 + f, mrow0 + 8 * g)) = u;
    }
    __syncwarp();
}

// Column sums of 32 values over the warp's 32 rows (reduce-scatter: lane l ends with
// column l), a fixed order.
__device__ __forceinline__ float col_sum32(float (&v)[32], int lane)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
        const bool upper = (lane & o) != 0;
#pragma unroll
        for (int i = 0; i < o; ++i) {
            const float send = upper ? v[i] : v[i + o];
            const float keep = upper ? v[i + o] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

struct TileArgs {
    const float *X;          // [.][in_dim] FP32 features
    const int64_t *idx;      // row b of the batch is X[idx[cursor B + b]] (null: X[b])
    const int64_t *cursor;   // device batch cursor of a replayed epoch, or null
    const float *y;          // labels (null: inference only)
    int B, Bp, in_dim;
    const uint8_t *wimg;     // 9 weight chunks: W1t, W2t (4 K-chunks), W2b (4 K-chunks)
    const float *params;     // FP32 masters: b1, b2, w3, b3 read here
    int64_t off_b1, off_b2, off_w3, off_b3;
    float *p_out;            // [B] probabilities
    uint8_t *xt_img, *h1t_img, *dh2t_img, *dh1t_img;  // batch-major operand images, per 64-row chunk
    float *part_head;        // [tiles][2 kH + 2]: dw3, db2, db3, loss of each tile
    float *part_b1;          // [tiles][kH]
    unsigned int *status;
};

// Shared memory of k_tile (dynamic): weight ring 2 x 32 KB | X 16 KB | H1 64 KB | dH2 64 KB
// | staging 4 x 2560 B.  The column sums (2 x 4 warps x 256 floats) reuse the X operand,
// which is dead once layer 1's MMAs are complete.
constexpr int kOffRing = 0;
constexpr int kOffX = kOffRing + 2 * static_cast<int>(kWChunk);
constexpr int kOffH1 = kOffX + 16384;
constexpr int kOffD2 = kOffH1 + 65536;
constexpr int kOffStage = kOffD2 + 65536;
constexpr int kOffCols = kOffX;
constexpr int kTileSmem = kOffStage + 4 * 2560;
static_assert(2 * 4 * kH * 4 <= 16384, "column sums fit the X operand");

template <bool kTrain>
__global__ void __launch_bounds__(128, 1) k_tile(const TileArgs g)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_full[2], s_empty[2], s_mma;
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ float s_red[4][2];
    uint8_t *ring = smem + kOffRing;
    uint8_t *sX = smem + kOffX;
    uint8_t *sH1 = smem + kOffH1;
    uint8_t *sD2 = smem + kOffD2;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    uint16_t *stage = reinterpret_cast<uint16_t *>(smem + kOffStage + warp * 2560);
    float *cols = reinterpret_cast<float *>(smem + kOffCols);  // [2][4 warps][kH]
    const int tile = blockIdx.x;
    const int64_t row = static_cast<int64_t>(tile) * kBM + t;  // this thread's batch row
    const bool valid = row < g.B;
    constexpr uint32_t kIdesc = idesc_bf16_f32(128, 256);
    const int n_chunks = kTrain ? 9 : 5;  // W1t, W2t x 4, (W2b x 4)

    if (warp == 0) {
        tmem_alloc(&s_tmem, 512);
        tmem_relinquish();
    }
    if (t == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&s_full[i], 1);
            mbar_init(&s_empty[i], 1);
        }
        mbar_init(&s_mma, 1);
        fence_barrier_init();
        s_fail = 0;
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = s_tmem;
    bool ok = true;
    auto load = [&](int c) {  // weight chunk c into stage c & 1
        mbar_arrive_expect_tx(&s_full[c & 1], kWChunk);
        bulk_g2s(ring + (c & 1) * kWChunk, g.wimg + static_cast<size_t>(c) * kWChunk, kWChunk, &s_full[c & 1]);
    };
    int loaded = 0;  // chunks whose copies were issued (thread 0)
    if (t == 0) {
        load(0);
        load(1);
        loaded = 2;
    }
    // refill: chunk c's MMAs are complete -> its stage takes chunk c + 2
    auto refill = [&](int c) {
        if (!mbar_wait_bounded(&s_empty[c & 1], (c >> 1) & 1, kDefaultWaitLimit)) ok = false;
        if (ok && c + 2 < n_chunks) {
            load(c + 2);
            loaded = c + 3;
        }
    };
    // four M=128 N=256 K=16 MMAs of chunk c (A: a K-chunk of an operand in shared memory)
    auto mma = [&](int c, const uint8_t *a, uint32_t d, bool first) {
        if (!mbar_wait_bounded(&s_full[c & 1], (c >> 1) & 1, kDefaultWaitLimit)) ok = false;
        if (!ok) return;
        tc_fence_after_sync();
        const uint8_t *b = ring + (c & 1) * kWChunk;
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
            tc_mma_bf16(d, smem_desc_kmajor(a + ks * 256, 128, 1024), smem_desc_kmajor(b + ks * 256, 128, 1024),
                        kIdesc, (!first || ks) ? 1u : 0u);
        tc_commit(&s_empty[c & 1]);
    };
    // every thread waits for the MMAs committed to s_mma (phase `ph`); the barrier
    // after it makes s_fail the same for every thread
    int mma_commits = 0;  // thread 0
    auto wait_mma = [&](int ph) {
        if (!mbar_wait_bounded(&s_mma, ph, kDefaultWaitLimit)) {
            s_fail = 1;
            atomicOr(g.status, kStatusTimeout);
        }
        tc_fence_after_sync();
        __syncthreads();
    };

    // ---- X rows: FP32 -> BF16 into the layer-1 operand (and its batch-major image)
    {
        float xv[64];
        const int64_t src = valid ? batch_row(g.idx, g.cursor, g.B, row) : 0;
#pragma unroll
        for (int c = 0; c < 64; ++c) xv[c] = (valid && c < g.in_dim) ? g.X[src * g.in_dim + c] : 0.0f;
        put_row32(sX, t, 0, *reinterpret_cast<float(*)[32]>(&xv[0]));
        put_row32(sX, t, 32, *reinterpret_cast<float(*)[32]>(&xv[32]));
        if constexpr (kTrain) {
            uint8_t *chunk = g.xt_img + (static_cast<size_t>(tile) * 2 + (t >> 6)) * (64 * 64 * 2);
            put_cols32(chunk, 0, (t & 63) & ~31, *reinterpret_cast<float(*)[32]>(&xv[0]), stage, lane);
            put_cols32(chunk, 32, (t & 63) & ~31, *reinterpret_cast<float(*)[32]>(&xv[32]), stage, lane);
        }
    }
    fence_async_shared();
    __syncthreads();

    // ---- layer 1: C1 = X W1 (tensor memory columns 0 .. 255)
    if (t == 0) {
        mma(0, sX, tmem, true);
        if (ok) {
            tc_commit(&s_mma);
            ++mma_commits;
        }
        refill(0);
    }
    wait_mma(0);
    // epilogue 1: H1 = relu(C1 + b1), BF16 into the layer-2 operand (+ its batch-major image)
    const uint32_t lane_base = static_cast<uint32_t>(32 * warp) << 16;
    if (!s_fail) {
#pragma unroll 1
        for (int c0 = 0; c0 < kH; c0 += 32) {
            uint32_t raw[32];
            tmem_ld32(tmem + lane_base + c0, raw);
            tmem_ld_wait();
            float v[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) v[j] = fmaxf(__uint_as_float(raw[j]) + __ldg(g.params + g.off_b1 + c0 + j), 0.0f);
            put_row32(sH1, t, c0, v);
            if constexpr (kTrain) {
                uint8_t *chunk = g.h1t_img + (static_cast<size_t>(tile) * 2 + (t >> 6)) * (kH * 64 * 2);
                put_cols32(chunk, c0, (t & 63) & ~31, v, stage, lane);
            }
        }
    }
    fence_async_shared();
    tc_fence_before_sync();
    __syncthreads();

    // ---- layer 2: C2 = H1 W2 (columns 256 .. 511), W2t in four K-chunks
    if (t == 0 && !s_fail) {
        tc_fence_after_sync();
        mma(1, sH1, tmem + 256, true);
        mma(2, sH1 + 16384, tmem + 256, false);
        refill(1);
        mma(3, sH1 + 2 * 16384, tmem + 256, false);
        refill(2);
        mma(4, sH1 + 3 * 16384, tmem + 256, false);
        if (ok) {
            tc_commit(&s_mma);
            ++mma_commits;
        }
        refill(3);
    }
    wait_mma(1);

    // ---- output layer: z = relu(C2 + b2) . w3 + b3, p = sigmoid(z)
    float z = 0.0f;
    if (!s_fail) {
#pragma unroll 1
        for (int c0 = 0; c0 < kH; c0 += 32) {
            uint32_t raw[32];
            tmem_ld32(tmem + lane_base + 256 + c0, raw);
            tmem_ld_wait();
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float h = fmaxf(__uint_as_float(raw[j]) + __ldg(g.params + g.off_b2 + c0 + j), 0.0f);
                z = fmaf(h, __ldg(g.params + g.off_w3 + c0 + j), z);
            }
        }
    }
    z += __ldg(g.params + g.off_b3);
    const float p = 1.0f / (1.0f + expf(-z));
    if (valid) g.p_out[row] = p;

    if constexpr (kTrain) {
        // ---- first backward step: dz = (p - y) / B; dH2 = dz w3 [h2 > 0] (BF16); column
        // sums of dz h2 (dw3) and of dH2 (db2) over the tile's rows; loss and db3
        const float yy = valid ? g.y[batch_row(g.idx, g.cursor, g.B, row)] : 0.0f;
        const float dz = valid ? (p - yy) * (1.0f / static_cast<float>(g.B)) : 0.0f;
        float loss = 0.0f;
        if (valid) {
            const float eps = 1e-12f;
            loss = -(yy * logf(p + eps) + (1.0f - yy) * logf(1.0f - p + eps));
        }
        if (!s_fail) {
#pragma unroll 1
            for (int c0 = 0; c0 < kH; c0 += 32) {
                uint32_t raw[32];
                tmem_ld32(tmem + lane_base + 256 + c0, raw);
                tmem_ld_wait();
                float d[32], hw[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float h = fmaxf(__uint_as_float(raw[j]) + __ldg(g.params + g.off_b2 + c0 + j), 0.0f);
                    d[j] = h > 0.0f ? dz * __ldg(g.params + g.off_w3 + c0 + j) : 0.0f;
                    hw[j] = dz * h;
                }
                put_row32(sD2, t, c0, d);
                uint8_t *chunk = g.dh2t_img + (static_cast<size_t>(tile) * 2 + (t >> 6)) * (kH * 64 * 2);
                put_cols32(chunk, c0, (t & 63) & ~31, d, stage, lane);
                cols[(0 * 4 + warp) * kH + c0 + lane] = col_sum32(hw, lane);  // dw3
                cols[(1 * 4 + warp) * kH + c0 + lane] = col_sum32(d, lane);   // db2
            }
        }
        float rs[2] = {dz, loss};
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) rs[k] += __shfl_xor_sync(0xffffffffu, rs[k], o);
        if (lane == 0) {
            s_red[warp][0] = rs[0];
            s_red[warp][1] = rs[1];
        }
        fence_async_shared();
        tc_fence_before_sync();
        __syncthreads();
        // per-tile partials of dw3, db2 (warps in order), db3 and the loss
        float *ph = g.part_head + static_cast<int64_t>(tile) * (2 * kH + 2);
        for (int i = t; i < 2 * kH; i += 128) {
            const int which = i / kH, c = i % kH;
            const float *q = cols + which * 4 * kH + c;
            ph[i] = ((q[0] + q[kH]) + q[2 * kH]) + q[3 * kH];
        }
        if (t == 0) {
            ph[2 * kH] = ((s_red[0][0] + s_red[1][0]) + s_red[2][0]) + s_red[3][0];
            ph[2 * kH + 1] = ((s_red[0][1] + s_red[1][1]) + s_red[2][1]) + s_red[3][1];
        }
        __syncthreads();  // the column sums are read before epilogue 3 rewrites them

        // ---- dH1 = dH2 W2^T (columns 0 .. 255 again), W2b in four K-chunks
        if (t == 0 && !s_fail) {
            tc_fence_after_sync();
            refill(4);
            mma(5, sD2, tmem, true);
            mma(6, sD2 + 16384, tmem, false);
            refill(5);
            mma(7, sD2 + 2 * 16384, tmem, false);
            refill(6);
            mma(8, sD2 + 3 * 16384, tmem, false);
            if (ok) {
                tc_commit(&s_mma);
                ++mma_commits;
            }
        }
        wait_mma(0);
        // epilogue 3: dH1 = C3 [h1 > 0] (BF16 batch-major image) and its column sums (db1)
        if (!s_fail) {
#pragma unroll 1
            for (int c0 = 0; c0 < kH; c0 += 32) {
                uint32_t raw[32];
                tmem_ld32(tmem + lane_base + c0, raw);
                tmem_ld_wait();
                // this row's 32 stored H1 values (the mask), 16 bytes at a time
                const uint8_t *hb = sH1 + (c0 >> 6) * 16384 + (t >> 3) * 1024 + (t & 7) * 16 + ((c0 & 63) >> 3) * 128;
                float d[32];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const uint4 u = *reinterpret_cast<const uint4 *>(hb + q * 128);
                    const uint32_t w4[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
                    for (int h = 0; h < 8; ++h) {
                        const uint16_t bits = static_cast<uint16_t>((h & 1) ? (w4[h >> 1] >> 16) : (w4[h >> 1] & 0xFFFFu));
                        const float hv = __bfloat162float(__ushort_as_bfloat16(bits));
                        d[8 * q + h] = hv > 0.0f ? __uint_as_float(raw[8 * q + h]) : 0.0f;
                    }
                }
                uint8_t *chunk = g.dh1t_img + (static_cast<size_t>(tile) * 2 + (t >> 6)) * (kH * 64 * 2);
                put_cols32(chunk, c0, (t & 63) & ~31, d, stage, lane);
                cols[warp * kH + c0 + lane] = col_sum32(d, lane);  // db1
            }
        }
        __syncthreads();
        float *pb = g.part_b1 + static_cast<int64_t>(tile) * kH;
        for (int c = t; c < kH; c += 128) {
            const float *q = cols + c;
            pb[c] = ((q[0] + q[kH]) + q[2 * kH]) + q[3 * kH];
        }
    }

    // leave: on a time-out wait (bounded) for the copies and MMAs in flight first
    if (t == 0 && !ok) {
        atomicOr(g.status, kStatusTimeout);
        s_fail = 1;
        for (int c = 0; c < loaded; ++c) mbar_wait_bounded(&s_full[c & 1], (c >> 1) & 1, kDefaultWaitLimit);
        tc_commit(&s_mma);  // completes once every MMA this thread issued is done
        mbar_wait_bounded(&s_mma, mma_commits & 1, kDefaultWaitLimit);
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, 512);
    }
}

// ---------------------------------------------------------------------------
// Weight gradients over the batch, split into `splits` ranges of 64-row chunks:
//   problem 0 (CTA x = 0, 1):  dW2[k][n]  = sum_m H1T[k][m] dH2T[n][m], k-tile x
//   problem 1 (CTA x = 2, 3):  dW1T[n][k] = sum_m dH1T[n][m] XT[k][m], n-tile x - 2
// Each CTA copies its A (128 rows x 64, 16 KB) and B (256 or 64 rows x 64) chunk images
// with bulk copies through a 3-stage ring, one thread issues the MMAs, and the FP32
// tile of its split goes to part_w2[split] ([256][256]) or part_w1[split] ([256][64]).
struct WgradArgs {
    const uint8_t *h1t_img, *dh2t_img, *dh1t_img, *xt_img;
    int n_mchunks, chunks_per_split;
    float *part_w2, *part_w1;
    unsigned int *status;
};

constexpr int kWgStages = 3;
constexpr uint32_t kWgA = 16384, kWgB = 32768;
constexpr int kWgradSmem = kWgStages * static_cast<int>(kWgA + kWgB);

__global__ void __launch_bounds__(128, 1) k_wgrad(const WgradArgs g)
{
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t s_full[kWgStages], s_empty[kWgStages];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int prob = blockIdx.x >> 1, mt = blockIdx.x & 1;
    const int split = blockIdx.y;
    const int N = prob == 0 ? 256 : 64;
    const uint32_t bbytes = prob == 0 ? kWgB : 8192u;
    const int c_begin = split * g.chunks_per_split;
    const int c_end = min(g.n_mchunks, c_begin + g.chunks_per_split);
    const int nk = max(0, c_end - c_begin);
    const uint8_t *A = prob == 0 ? g.h1t_img : g.dh1t_img;
    const uint8_t *Bm = prob == 0 ? g.dh2t_img : g.xt_img;
    const size_t a_stride = kH * 64 * 2;                      // one chunk of a 256-feature image
    const size_t b_stride = prob == 0 ? kH * 64 * 2 : 64 * 64 * 2;

    if (warp == 0) {
        tmem_alloc(&s_tmem, 256);
        tmem_relinquish();
    }
    if (t == 0) {
        for (int i = 0; i < kWgStages; ++i) {
            mbar_init(&s_full[i], 1);
            mbar_init(&s_empty[i], 1);
        }
        fence_barrier_init();
        s_fail = 0;
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t idesc = prob == 0 ? idesc_bf16_f32(128, 256) : idesc_bf16_f32(128, 64);

    if (t == 0) {
        bool ok = true;
        auto load = [&](int i) {
            const int s = i % kWgStages;
            uint8_t *sa = smem + s * (kWgA + kWgB);
            mbar_arrive_expect_tx(&s_full[s], kWgA + bbytes);
            const size_t mc = static_cast<size_t>(c_begin + i);
            bulk_g2s(sa, A + mc * a_stride + mt * kWgA, kWgA, &s_full[s]);
            bulk_g2s(sa + kWgA, Bm + mc * b_stride, bbytes, &s_full[s]);
        };
        int issued = 0;
        for (; issued < min(nk, kWgStages); ++issued) load(issued);
        for (int i = 0; i < nk && ok; ++i) {
            const int s = i % kWgStages;
            if (!mbar_wait_bounded(&s_full[s], (i / kWgStages) & 1, kDefaultWaitLimit)) {
                ok = false;
                break;
            }
            tc_fence_after_sync();
            const uint8_t *sa = smem + s * (kWgA + kWgB);
#pragma unroll
            for (int ks = 0; ks < 4; ++ks)
                tc_mma_bf16(tmem, smem_desc_kmajor(sa + ks * 256, 128, 1024),
                            smem_desc_kmajor(sa + kWgA + ks * 256, 128, 1024), idesc, (i | ks) ? 1u : 0u);
            tc_commit(&s_empty[s]);
            if (issued < nk) {
                // the stage of chunk i is refilled once its MMAs are done
                if (!mbar_wait_bounded(&s_empty[s], (i / kWgStages) & 1, kDefaultWaitLimit)) {
                    ok = false;
                    break;
                }
                load(issued++);
            }
        }
        if (ok && nk > 0) {
            // the last chunk's commit covers every MMA before it
            const int last = nk - 1;
            if (!mbar_wait_bounded(&s_empty[last % kWgStages], (last / kWgStages) & 1, kDefaultWaitLimit)) ok = false;
        }
        if (!ok) {
            s_fail = 1;
            atomicOr(g.status, kStatusTimeout);
            for (int i = 0; i < issued; ++i) mbar_wait_bounded(&s_full[i % kWgStages], (i / kWgStages) & 1, kDefaultWaitLimit);
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();

    if (!s_fail) {
        const int r = mt * 128 + 32 * warp + lane;  // output row (k of dW2, n of dW1T)
        float *out = prob == 0 ? g.part_w2 + static_cast<size_t>(split) * kH * kH + static_cast<size_t>(r) * kH
                               : g.part_w1 + static_cast<size_t>(split) * kH * kKP + static_cast<size_t>(r) * kKP;
#pragma unroll 1
        for (int c0 = 0; c0 < N; c0 += 32) {
            uint32_t raw[32];
            if (nk > 0) {
                tmem_ld32(tmem + (static_cast<uint32_t>(32 * warp) << 16) + c0, raw);
                tmem_ld_wait();
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) raw[j] = 0u;
            }
            float4 *o = reinterpret_cast<float4 *>(out + c0);
#pragma unroll
            for (int q = 0; q < 8; ++q)
                o[q] = make_float4(__uint_as_float(raw[4 * q]), __uint_as_float(raw[4 * q + 1]),
                                   __uint_as_float(raw[4 * q + 2]), __uint_as_float(raw[4 * q + 3]));
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, 256);
    }
}

// ---------------------------------------------------------------------------
// Gradients from the partials (each summed in split / tile order), then optionally
// AdamW on the FP32 masters and the BF16 weight images.  One thread per parameter of
// the packed layout [W1 (in x 256) | b1 | W2 (256 x 256) | b2 | w3 | b3]; thread
// n_params writes the loss sum.
struct UpdateArgs {
    const float *part_w2, *part_w1, *part_head, *part_b1;
    int n_splits, n_tiles, in_dim;
    int64_t n_params, off_b1, off_W2, off_b2, off_w3, off_b3;
    float *grads, *loss_sum;
    // AdamW (null w: gradients only)
    float *w, *m, *v;
    float lr, beta1, beta2, eps, wd, bc1, bc2;
    const float *bc_table;   // replayed epochs: bias corrections [2 cursor + {0, 1}]
    const int64_t *cursor;
    uint8_t *wimg;           // the BF16 images of W1t, W2t, W2b
};

__device__ __forceinline__ void put_img(uint8_t *wimg, int chunk, int r, int c, float x)
{
    *reinterpret_cast<__nv_bfloat16 *>(wimg + static_cast<size_t>(chunk) * kWChunk + img_off(r, c)) =
        __float2bfloat16_rn(x);
}

// BF16 copies of one weight into the images: W1[k][n] -> W1t (row n, col k); W2[k][n] ->
// W2t chunk k / 64 (row n, col k % 64) and W2b chunk n / 64 (row k, col n % 64).
__device__ __forceinline__ void put_weight(uint8_t *wimg, bool is_w2, int k, int n, float x)
{
    if (!is_w2) {
        put_img(wimg, 0, n, k, x);
    } else {
        put_img(wimg, 1 + (k >> 6), n, k & 63, x);
        put_img(wimg, 5 + (n >> 6), k, n & 63, x);
    }
}

__global__ void k_update(const UpdateArgs g)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i > g.n_params) return;
    if (i == g.n_params) {
        float s = 0.0f;
        for (int tl = 0; tl < g.n_tiles; ++tl) s += g.part_head[static_cast<int64_t>(tl) * (2 * kH + 2) + 2 * kH + 1];
        *g.loss_sum = s;
        return;
    }
    float gr = 0.0f;
    bool is_w = false, is_w2 = false;
    int wk = 0, wn = 0;
    if (i < g.off_b1) {  // W1[k][n]: partials hold dW1^T [n][k]
        wk = static_cast<int>(i / kH);
        wn = static_cast<int>(i % kH);
        for (int z = 0; z < g.n_splits; ++z) gr += g.part_w1[static_cast<int64_t>(z) * kH * kKP + wn * kKP + wk];
        is_w = true;
    } else if (i < g.off_W2) {  // b1
        const int c = static_cast<int>(i - g.off_b1);
        for (int tl = 0; tl < g.n_tiles; ++tl) gr += g.part_b1[static_cast<int64_t>(tl) * kH + c];
    } else if (i < g.off_b2) {  // W2[k][n]
        const int64_t j = i - g.off_W2;
        wk = static_cast<int>(j / kH);
        wn = static_cast<int>(j % kH);
        for (int z = 0; z < g.n_splits; ++z) gr += g.part_w2[static_cast<int64_t>(z) * kH * kH + j];
        is_w = is_w2 = true;
    } else {  // b2, w3, b3 from the tile partials [dw3 | db2 | db3 | loss]
        int col;
        if (i < g.off_w3) col = kH + static_cast<int>(i - g.off_b2);
        else if (i < g.off_b3) col = static_cast<int>(i - g.off_w3);
        else col = 2 * kH;
        for (int tl = 0; tl < g.n_tiles; ++tl) gr += g.part_head[static_cast<int64_t>(tl) * (2 * kH + 2) + col];
    }
    g.grads[i] = gr;
    if (!g.w) return;
    float bc1 = g.bc1, bc2 = g.bc2;
    if (g.bc_table) {
        bc1 = g.bc_table[2 * *g.cursor];
        bc2 = g.bc_table[2 * *g.cursor + 1];
    }
    const float mi = g.beta1 * g.m[i] + (1.0f - g.beta1) * gr;
    const float vi = g.beta2 * g.v[i] + (1.0f - g.beta2) * gr * gr;
    g.m[i] = mi;
    g.v[i] = vi;
    const float mhat = mi / bc1, vhat = vi / bc2;
    const float wv = g.w[i] * (1.0f - g.lr * g.wd) - g.lr * mhat / (sqrtf(vhat) + g.eps);
    g.w[i] = wv;
    if (is_w) put_weight(g.wimg, is_w2, wk, wn, wv);
}

// All BF16 weight images from the FP32 masters, padding (W1 columns k >= in_dim) zero.
__global__ void k_refresh(const float *__restrict__ W1, int in_dim, const float *__restrict__ W2, uint8_t *wimg)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kH * kKP) {
        const int k = i / kH, n = i % kH;
        put_weight(wimg, false, k, n, k < in_dim ? W1[k * kH + n] : 0.0f);
    }
    if (i < kH * kH) put_weight(wimg, true, i / kH, i % kH, W2[i]);
}

// End of a replayed training step: its mean loss to losses[cursor], then the
// cursor moves to the next batch.
__global__ void k_epoch_tail(const float *__restrict__ loss_sum, int B, int64_t *cursor, float *__restrict__ losses)
{
    losses[*cursor] = *loss_sum / static_cast<float>(B);
    *cursor += 1;
}

}  // namespace

// ---------------------------------------------------------------------------
size_t mlp_wimg_bytes() { return 9 * static_cast<size_t>(kWChunk); }
size_t mlp_xt_bytes(int Bp) { return static_cast<size_t>(Bp / 64) * 64 * 64 * 2; }
size_t mlp_ht_bytes(int Bp) { return static_cast<size_t>(Bp / 64) * kH * 64 * 2; }
int mlp_wgrad_splits(int Bp, int *chunks_per_split)
{
    const int n = Bp / 64;
    const int cps = (n + 31) / 32;
    *chunks_per_split = cps;
    return (n + cps - 1) / cps;
}

cudaError_t mlp_prepare()
{
    cudaError_t e = cudaFuncSetAttribute(k_tile<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_tile<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTileSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgradSmem);
    return e;
}

cudaError_t mlp_launch_tile(const MlpBuffers &b, const float *X, const int64_t *idx, const int64_t *cursor,
                            const float *y, int B, int Bp, float *p_out, cudaStream_t s)
{
    if (Bp % kBM != 0 || B < 1 || B > Bp) return cudaErrorInvalidValue;
    TileArgs g{};
    g.X = X;
    g.idx = idx;
    g.cursor = cursor;
    g.y = y;
    g.B = B;
    g.Bp = Bp;
    g.in_dim = b.in_dim;
    g.wimg = static_cast<const uint8_t *>(b.wimg);
    g.params = b.params;
    g.off_b1 = b.off_b1;
    g.off_b2 = b.off_b2;
    g.off_w3 = b.off_w3;
    g.off_b3 = b.off_b3;
    g.p_out = p_out;
    g.xt_img = static_cast<uint8_t *>(b.xt_img);
    g.h1t_img = static_cast<uint8_t *>(b.h1t_img);
    g.dh2t_img = static_cast<uint8_t *>(b.dh2t_img);
    g.dh1t_img = static_cast<uint8_t *>(b.dh1t_img);
    g.part_head = b.part_head;
    g.part_b1 = b.part_b1;
    g.status = b.status;
    if (y)
        k_tile<true><<<Bp / kBM, 128, kTileSmem, s>>>(g);
    else
        k_tile<false><<<Bp / kBM, 128, kTileSmem, s>>>(g);
    return cudaGetLastError();
}

cudaError_t mlp_launch_wgrad(const MlpBuffers &b, int Bp, cudaStream_t s)
{
    WgradArgs g{};
    g.h1t_img = static_cast<const uint8_t *>(b.h1t_img);
    g.dh2t_img = static_cast<const uint8_t *>(b.dh2t_img);
    g.dh1t_img = static_cast<const uint8_t *>(b.dh1t_img);
    g.xt_img = static_cast<const uint8_t *>(b.xt_img);
    g.n_mchunks = Bp / 64;
    const int splits = mlp_wgrad_splits(Bp, &g.chunks_per_split);
    g.part_w2 = b.part_w2;
    g.part_w1 = b.part_w1;
    g.status = b.status;
    k_wgrad<<<dim3(4, splits), 128, kWgradSmem, s>>>(g);
    return cudaGetLastError();
}

cudaError_t mlp_launch_update(const MlpBuffers &b, int Bp, bool adamw, float lr, float wd, float bc1, float bc2,
                              const float *bc_table, const int64_t *cursor, cudaStream_t s)
{
    UpdateArgs g{};
    g.part_w2 = b.part_w2;
    g.part_w1 = b.part_w1;
    g.part_head = b.part_head;
    g.part_b1 = b.part_b1;
    int cps = 0;
    g.n_splits = mlp_wgrad_splits(Bp, &cps);
    g.n_tiles = Bp / kBM;
    g.in_dim = b.in_dim;
    g.n_params = b.n_params;
    g.off_b1 = b.off_b1;
    g.off_W2 = b.off_W2;
    g.off_b2 = b.off_b2;
    g.off_w3 = b.off_w3;
    g.off_b3 = b.off_b3;
    g.grads = b.grads;
    g.loss_sum = b.loss_sum;
    if (adamw) {
        g.w = b.params;
        g.m = b.m;
        g.v = b.v;
    }
    g.lr = lr;
    g.beta1 = 0.9f;
    g.beta2 = 0.999f;
    g.eps = 1e-8f;
    g.wd = wd;
    g.bc1 = bc1;
    g.bc2 = bc2;
    g.bc_table = bc_table;
    g.cursor = cursor;
    g.wimg = static_cast<uint8_t *>(b.wimg);
    const int64_t n = b.n_params + 1;
    k_update<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(g);
    return cudaGetLastError();
}

cudaError_t mlp_launch_refresh(const MlpBuffers &b, cudaStream_t s)
{
    k_refresh<<<(kH * kH + 255) / 256, 256, 0, s>>>(b.params + b.off_W1, b.in_dim, b.params + b.off_W2,
                                                     static_cast<uint8_t *>(b.wimg));
    return cudaGetLastError();
}

cudaError_t mlp_launch_epoch_tail(const float *loss_sum, int B, int64_t *cursor, float *losses, cudaStream_t s)
{
    k_epoch_tail<<<1, 1, 0, s>>>(loss_sum, B, cursor, losses);
    return cudaGetLastError();
}

}  // namespace gn
