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
//            weight images the tile kernel streams; in a replayed epoch its last
//            CTA also records the step's loss and moves the batch cursor on.
//
// Shared-memory operand layout (tcgen05 K-major, 128-byte swizzle): a matrix of R rows x
// 64 K-elements is a chunk of 128-byte rows; element (r, c) sits at byte r 128 +
// ((c / 8) xor (r % 8)) 16 + (c % 8) 2 (8-row groups 1024 bytes apart), so the tensor
// core's operand fetches spread over the shared-memory banks.  Weights and the transposed
// activations are kept in global memory in exactly this image, so one 1D bulk copy lands a
// chunk.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "ptx.cuh"

namespace gn {
namespace {

constexpr int kH = kMlpHidden;   // 256
constexpr int kKP = kMlpInPad;   // 64
constexpr int kBM = 128;         // batch rows per tile
constexpr uint32_t kWChunk = 256u * 64u * 2u;  // one weight chunk: 256 rows x 64 K, BF16 (32 KB)
constexpr int kWChunks = 9;                     // W1, W2 x 4, W2^T x 4
constexpr int kWStages = 2;                     // ring slots of the tile kernel's weight chunks
constexpr size_t kWImage = static_cast<size_t>(kWChunks) * kWChunk;

// byte of element (r, c) in a K-major chunk of 64 K-elements per row with the 128-byte
// swizzle (rows 128 bytes apart, 16-byte unit j of row r at position j ^ (r % 8))
__host__ __device__ constexpr uint32_t img_off(uint32_t r, uint32_t c)
{
    return r * 128u + ((((c >> 3) ^ r) & 7u) << 4) + (c & 7u) * 2u;
}

// Programmatic dependent launch: the kernels of a step are launched with the PDL
// attribute, each lets the next one start at once (its prologue -- tensor-memory
// allocation, barrier set-up -- overlaps this kernel) and waits for the previous grid
// (griddepcontrol.wait: complete, its writes visible) before it reads that grid's output.
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

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

// The 16-byte unit holding columns c .. c + 7 (c % 8 == 0) of `row` in a K-major operand
// of 128 rows held as swizzled chunks of 64 K-elements (16 KB apart).
__device__ __forceinline__ uint8_t *op_unit(uint8_t *op, int row, int c)
{
    return op + (c >> 6) * 16384 + row * 128 + ((((c & 63) >> 3) ^ row) & 7) * 16;
}

// 32 columns (c0 .. c0 + 31) of this thread's row as BF16 into such an operand.
__device__ __forceinline__ void put_row32(uint8_t *op, int row, int c0, const float (&v)[32])
{
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint4 u = make_uint4(pack_bf16(v[8 * q], v[8 * q + 1]), pack_bf16(v[8 * q + 2], v[8 * q + 3]),
                                   pack_bf16(v[8 * q + 4], v[8 * q + 5]), pack_bf16(v[8 * q + 6], v[8 * q + 7]));
        *reinterpret_cast<uint4 *>(op_unit(op, row, c0 + 8 * q)) = u;
    }
}

// Transpose of an 8 x 8 block of 16-bit values held by 8 consecutive lanes (lane i: row
// i as four words of two values); afterwards lane i holds column i (rows in order).
// Three exchange stages: 4 x 4 blocks (xor 4), 2 x 2 blocks of words (xor 2), halves
// of words (xor 1).
__device__ __forceinline__ void transpose8(uint32_t (&w)[4], int i)
{
    {
        const bool top = (i & 4) == 0;
        const uint32_t r0 = __shfl_xor_sync(0xffffffffu, top ? w[2] : w[0], 4);
        const uint32_t r1 = __shfl_xor_sync(0xffffffffu, top ? w[3] : w[1], 4);
        if (top) {
            w[2] = r0;
            w[3] = r1;
        } else {
            w[0] = r0;
            w[1] = r1;
        }
    }
    {
        const bool hi = (i & 2) != 0;
        const uint32_t r0 = __shfl_xor_sync(0xffffffffu, hi ? w[0] : w[1], 2);
        const uint32_t r1 = __shfl_xor_sync(0xffffffffu, hi ? w[2] : w[3], 2);
        if (!hi) {
            w[1] = r0;
            w[3] = r1;
        } else {
            w[0] = r0;
            w[2] = r1;
        }
    }
    const bool odd = (i & 1) != 0;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const uint32_t r = __shfl_xor_sync(0xffffffffu, odd ? (w[p] & 0xFFFFu) : (w[p] >> 16), 1);
        w[p] = odd ? ((w[p] & 0xFFFF0000u) | r) : ((w[p] & 0xFFFFu) | (r << 16));
    }
}

// 32 features (f0 .. f0 + 31) of the warp's 32 rows (this thread: row `mrow` of the
// 64-row chunk, a multiple-of-8 group per 8 lanes) as BF16 into the batch-major image of
// a weight-gradient operand (rows = features, K = the chunk's 64 batch rows).  Blocks of
// 8 rows x 8 features are transposed across 8 lanes, so each lane stores 16 bytes (8 rows
// of one feature) and the four lanes of a feature fill 64 contiguous bytes.
__device__ __forceinline__ void put_col32(uint8_t *chunk, int f0, int mrow, const float (&v)[32], int lane)
{
    const int mg = mrow >> 3, i = lane & 7;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        uint32_t w[4];
#pragma unroll
        for (int p = 0; p < 4; ++p) w[p] = pack_bf16(v[8 * b + 2 * p], v[8 * b + 2 * p + 1]);
        transpose8(w, i);
        const int f = f0 + 8 * b + i;
        *reinterpret_cast<uint4 *>(chunk + f * 128 + (((mg ^ f) & 7) << 4)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
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

// Shared memory of k_tile (dynamic, from a 1024-byte aligned base): weight ring 2 x 32 KB |
// X 16 KB | H1 64 KB | dH2 64 KB.  Weight chunks also land in buffers that are dead at
// the time: W2t K-chunks 2 and 3 in the dH2 operand (written only after layer 2), W2^T
// K-chunks 2 and 3 in the H1 operand once layer 2 is done with it (the ReLU mask of H1
// is kept apart as bits), so every chunk of a GEMM is in flight before the GEMM starts.
// The column sums (2 x 4 lane groups x 256 floats) reuse the X operand, which is dead
// once layer 1's MMAs are complete.
constexpr int kOffRing = 0;
constexpr int kOffX = kOffRing + kWStages * static_cast<int>(kWChunk);
constexpr int kOffH1 = kOffX + 16384;
constexpr int kOffD2 = kOffH1 + 65536;
constexpr int kOffCols = kOffX;
constexpr int kTileSmem = kOffD2 + 65536 + 1024;  // + the alignment of the base
static_assert(2 * 4 * kH * 4 <= 16384, "column sums fit the X operand");
constexpr int kTileThreads = 512;

// 16 warps: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 (its lane group: rows of
// the tile) and owns columns 64 (w / 4) .. + 63 (its column quarter) of every 256-wide
// layer, so each epilogue pass is two 32-column loads per warp.
template <bool kTrain>
__global__ void __launch_bounds__(kTileThreads, 1) k_tile(const TileArgs g)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);  // swizzle atoms: 1 KB aligned
    __shared__ __align__(8) uint64_t s_full[kWChunks], s_empty[2], s_mma;
    __shared__ uint32_t s_mask[kBM][kH / 32];  // H1 > 0 (as stored, BF16), bit per column
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ float s_b1[kH], s_b2[kH], s_w3[kH];
    __shared__ float s_zp[4][kBM];  // partial output-layer sums per column quarter
    __shared__ float s_dz[kBM];
    __shared__ float s_red[4][2];
    uint8_t *ring = smem + kOffRing;
    uint8_t *sX = smem + kOffX;
    uint8_t *sH1 = smem + kOffH1;
    uint8_t *sD2 = smem + kOffD2;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int lg = warp & 3, cq = warp >> 2;
    const int rl = 32 * lg + lane;                              // this thread's row in the tile
    float *cols = reinterpret_cast<float *>(smem + kOffCols);   // [2][4 lane groups][kH]
    const int tile = blockIdx.x;
    const int64_t row = static_cast<int64_t>(tile) * kBM + rl;
    const bool valid = row < g.B;
    const size_t img_chunk = static_cast<size_t>(tile) * 2 + (rl >> 6);  // this row's 64-row chunk
    const int mrow = rl & 63;
    const uint32_t lane_base = static_cast<uint32_t>(32 * lg) << 16;
    constexpr uint32_t kIdesc = idesc_bf16_f32(128, 256);
    const int n_chunks = kTrain ? kWChunks : 5;  // W1t, W2t x 4, (W2b x 4)
    const uint8_t *wimg = g.wimg;

    pdl_trigger();
    if (warp == 0) {
        tmem_alloc(&s_tmem, 512);
        tmem_relinquish();
    }
    if (t == 0) {
        for (int i = 0; i < kWChunks; ++i) mbar_init(&s_full[i], 1);
        for (int i = 0; i < 2; ++i) mbar_init(&s_empty[i], 1);
        mbar_init(&s_mma, 1);
        fence_barrier_init();
        s_fail = 0;
    }
    pdl_wait();  // the previous step's parameters, weight images and batch cursor
    for (int i = t; i < kH; i += kTileThreads) {
        s_b1[i] = g.params[g.off_b1 + i];
        s_b2[i] = g.params[g.off_b2 + i];
        s_w3[i] = g.params[g.off_w3 + i];
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = s_tmem;
    bool ok = true;
    // the buffer each weight chunk lands in: W1t and W2t K-chunks 0, 1 in the ring, W2t
    // K-chunks 2, 3 in the dH2 operand, W2^T K-chunks 0, 1 back in the ring, 2, 3 in the H1
    // operand; each chunk completes on its own mbarrier (one phase each)
    auto wbuf = [&](int c) -> uint8_t * {
        constexpr int kRingOf[kWChunks] = {0, 1, 0, -1, -2, 1, 0, -3, -4};
        const int r = kRingOf[c];
        return r >= 0 ? ring + r * kWChunk : r >= -2 ? sD2 + (-1 - r) * kWChunk : sH1 + (-3 - r) * kWChunk;
    };
    unsigned loaded = 0;  // bit c: chunk c's copy was issued (thread 0)
    auto load = [&](int c) {
        if (c >= n_chunks) return;
        mbar_arrive_expect_tx(&s_full[c], kWChunk);
        bulk_g2s(wbuf(c), wimg + static_cast<size_t>(c) * kWChunk, kWChunk, &s_full[c]);
        loaded |= 1u << c;
    };
    if (t == 0) {
        load(0);
        load(1);
        load(3);
        load(4);
    }
    // four M=128 N=256 K=16 MMAs of chunk c; A: the matching 64-element K-chunk of an
    // operand in shared memory (both operands 128-byte swizzled); completion of the ring
    // chunks 0, 1, 2 is committed to the ring slot's mbarrier
    auto mma = [&](int c, const uint8_t *a, uint32_t d, bool first) {
        if (!mbar_wait_bounded(&s_full[c], 0, kDefaultWaitLimit)) ok = false;
        if (!ok) return;
        tc_fence_after_sync();
        const uint8_t *b = wbuf(c);
#pragma unroll
        for (int ks = 0; ks < 4; ++ks)
            tc_mma_bf16(d, smem_desc_sw128(a + ks * 32), smem_desc_sw128(b + ks * 32), kIdesc,
                        (!first || ks) ? 1u : 0u);
        if (c <= 2) tc_commit(&s_empty[c & 1]);
    };
    // the ring slot of chunk c (0, 1 or 2) is free again once its MMAs are complete
    auto slot_free = [&](int c) {
        if (!mbar_wait_bounded(&s_empty[c & 1], c >> 1, kDefaultWaitLimit)) ok = false;
    };
    int mma_commits = 0;  // thread 0
    auto commit_mma = [&]() {
        if (ok) {
            tc_commit(&s_mma);
            ++mma_commits;
        }
    };
    // every thread waits for the MMAs committed to s_mma (phase `ph`); the barrier
    // after it makes s_fail the same for every thread
    auto wait_mma = [&](int ph) {
        if (!mbar_wait_bounded(&s_mma, ph, kDefaultWaitLimit)) {
            s_fail = 1;
            atomicOr(g.status, kStatusTimeout);
        }
        tc_fence_after_sync();
        __syncthreads();
    };
    // 32 accumulator columns (c0 ..) of this thread's row
    auto acc32 = [&](uint32_t col, float (&v)[32]) {
        uint32_t raw[32];
        tmem_ld32(tmem + lane_base + col, raw);
        tmem_ld_wait();
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(raw[j]);
    };

    // ---- X rows: FP32 -> BF16 into the layer-1 operand (and its batch-major image);
    // column quarters 0 and 1 take input columns 0 .. 31 and 32 .. 63
    if (cq < 2) {
        float xv[32];
        const int64_t src = valid ? batch_row(g.idx, g.cursor, g.B, row) : 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const int c = 32 * cq + j;
            xv[j] = (valid && c < g.in_dim) ? g.X[src * g.in_dim + c] : 0.0f;
        }
        put_row32(sX, rl, 32 * cq, xv);
        if constexpr (kTrain) put_col32(g.xt_img + img_chunk * (64 * 64 * 2), 32 * cq, mrow, xv, lane);
    }
    fence_async_shared();
    __syncthreads();

    // ---- layer 1: C1 = X W1 (tensor memory columns 0 .. 255)
    if (t == 0) {
        mma(0, sX, tmem, true);
        commit_mma();
        slot_free(0);
        if (ok) load(2);
    }
    wait_mma(0);
    // epilogue 1: H1 = relu(C1 + b1), BF16 into the layer-2 operand (+ its batch-major image)
    if (!s_fail) {
#pragma unroll 1
        for (int c0 = 64 * cq; c0 < 64 * cq + 64; c0 += 32) {
            float v[32];
            acc32(c0, v);
#pragma unroll
            uint32_t m = 0;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                v[j] = fmaxf(v[j] + s_b1[c0 + j], 0.0f);
                m |= (__bfloat162float(__float2bfloat16_rn(v[j])) > 0.0f ? 1u : 0u) << j;
            }
            s_mask[rl][c0 >> 5] = m;
            put_row32(sH1, rl, c0, v);
            if constexpr (kTrain) put_col32(g.h1t_img + img_chunk * (kH * 64 * 2), c0, mrow, v, lane);
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
        slot_free(1);
        if (ok) load(5);
        mma(3, sH1 + 2 * 16384, tmem + 256, false);
        mma(4, sH1 + 3 * 16384, tmem + 256, false);
        commit_mma();
        slot_free(2);
        if (ok) load(6);
        // layer 2 is done with H1 (and with the W2t chunks in the dH2 operand): W2^T
        // K-chunks 2, 3 go to the H1 operand
        if (kTrain && ok) {
            if (!mbar_wait_bounded(&s_mma, 1, kDefaultWaitLimit)) ok = false;
            if (ok) {
                load(7);
                load(8);
            }
        }
    }
    wait_mma(1);

    // ---- output layer: z = relu(C2 + b2) . w3 + b3 (each quarter's columns in order,
    // then the quarters in order), p = sigmoid(z)
    {
        float zq = 0.0f;
        if (!s_fail) {
#pragma unroll 1
            for (int c0 = 64 * cq; c0 < 64 * cq + 64; c0 += 32) {
                float v[32];
                acc32(256 + c0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) zq = fmaf(fmaxf(v[j] + s_b2[c0 + j], 0.0f), s_w3[c0 + j], zq);
            }
        }
        s_zp[cq][rl] = zq;
    }
    __syncthreads();
    if (cq == 0) {
        const float z = (((s_zp[0][rl] + s_zp[1][rl]) + s_zp[2][rl]) + s_zp[3][rl]) + g.params[g.off_b3];
        const float p = 1.0f / (1.0f + expf(-z));
        if (valid) g.p_out[row] = p;
        if constexpr (kTrain) {
            const float yy = valid ? g.y[batch_row(g.idx, g.cursor, g.B, row)] : 0.0f;
            const float dz = valid ? (p - yy) * (1.0f / static_cast<float>(g.B)) : 0.0f;
            float loss = 0.0f;
            if (valid) {
                const float eps = 1e-12f;
                loss = -(yy * logf(p + eps) + (1.0f - yy) * logf(1.0f - p + eps));
            }
            s_dz[rl] = dz;
            float rs[2] = {dz, loss};
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) rs[k] += __shfl_xor_sync(0xffffffffu, rs[k], o);
            if (lane == 0) {
                s_red[lg][0] = rs[0];
                s_red[lg][1] = rs[1];
            }
        }
    }

    if constexpr (kTrain) {
        __syncthreads();
        // ---- first backward step: dH2 = dz w3 [h2 > 0] (BF16); column sums of dz h2 (dw3)
        // and of dH2 (db2) over each lane group's rows
        const float dz = s_dz[rl];
        if (!s_fail) {
#pragma unroll 1
            for (int c0 = 64 * cq; c0 < 64 * cq + 64; c0 += 32) {
                float v[32], d[32];
                acc32(256 + c0, v);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const float h = fmaxf(v[j] + s_b2[c0 + j], 0.0f);
                    d[j] = h > 0.0f ? dz * s_w3[c0 + j] : 0.0f;
                    v[j] = dz * h;
                }
                put_row32(sD2, rl, c0, d);
                put_col32(g.dh2t_img + img_chunk * (kH * 64 * 2), c0, mrow, d, lane);
                cols[(0 * 4 + lg) * kH + c0 + lane] = col_sum32(v, lane);  // dw3
                cols[(1 * 4 + lg) * kH + c0 + lane] = col_sum32(d, lane);  // db2
            }
        }
        fence_async_shared();
        tc_fence_before_sync();
        __syncthreads();
        // per-tile partials of dw3, db2 (lane groups in order), db3 and the loss
        float *ph = g.part_head + static_cast<int64_t>(tile) * (2 * kH + 2);
        for (int i = t; i < 2 * kH; i += kTileThreads) {
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
            for (int c = 5; c < kWChunks; ++c) mma(c, sD2 + (c - 5) * 16384, tmem, c == 5);
            commit_mma();
        }
        wait_mma(0);
        // epilogue 3: dH1 = C3 [h1 > 0] (BF16 batch-major image) and its column sums (db1)
        if (!s_fail) {
#pragma unroll 1
            for (int c0 = 64 * cq; c0 < 64 * cq + 64; c0 += 32) {
                float d[32];
                acc32(c0, d);
                // the ReLU mask of this row's stored H1 values
                const uint32_t m = s_mask[rl][c0 >> 5];
#pragma unroll
                for (int j = 0; j < 32; ++j)
                    if (!((m >> j) & 1u)) d[j] = 0.0f;
                put_col32(g.dh1t_img + img_chunk * (kH * 64 * 2), c0, mrow, d, lane);
                cols[lg * kH + c0 + lane] = col_sum32(d, lane);  // db1
            }
        }
        __syncthreads();
        float *pb = g.part_b1 + static_cast<int64_t>(tile) * kH;
        for (int c = t; c < kH; c += kTileThreads) {
            const float *q = cols + c;
            pb[c] = ((q[0] + q[kH]) + q[2 * kH]) + q[3 * kH];
        }
    }

    // leave: on a time-out wait (bounded) for the copies and MMAs in flight first
    if (t == 0 && !ok) {
        atomicOr(g.status, kStatusTimeout);
        s_fail = 1;
        for (int c = 0; c < kWChunks; ++c)
            if (loaded & (1u << c)) mbar_wait_bounded(&s_full[c], 0, kDefaultWaitLimit);
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
// with bulk copies through a 3-stage ring, one thread issues the MMAs, and 8 warps (a
// lane group and a column half each) write the FP32 tile of its split to
// part_w2[split] ([k][n], 256 x 256) or part_w1[split] (dW1 itself, [k][n], 64 x 256).
struct WgradArgs {
    const uint8_t *h1t_img, *dh2t_img, *dh1t_img, *xt_img;
    int n_mchunks, chunks_per_split;
    float *part_w2, *part_w1;
    unsigned int *status;
};

constexpr int kWgStages = 4;  // a split's chunks (4 at a batch of 8192) all in flight at once
constexpr uint32_t kWgA = 16384, kWgB = 32768;
constexpr int kWgradSmem = kWgStages * static_cast<int>(kWgA + kWgB) + 1024;  // + the alignment of the base

constexpr int kWgradThreads = 256;

__global__ void __launch_bounds__(kWgradThreads, 1) k_wgrad(const WgradArgs g)
{
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);  // swizzle atoms: 1 KB aligned
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

    pdl_trigger();
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
    pdl_wait();  // the tile kernel's operand images

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
                tc_mma_bf16(tmem, smem_desc_sw128(sa + ks * 32), smem_desc_sw128(sa + kWgA + ks * 32), idesc,
                            (i | ks) ? 1u : 0u);
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
        const int lg = warp & 3, half = warp >> 2;
        const int r = mt * 128 + 32 * lg + lane;  // output row (k of dW2, n of dW1T)
#pragma unroll 1
        for (int c0 = half * (N / 2); c0 < (half + 1) * (N / 2); c0 += 32) {
            uint32_t raw[32];
            if (nk > 0) {
                tmem_ld32(tmem + (static_cast<uint32_t>(32 * lg) << 16) + c0, raw);
                tmem_ld_wait();
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) raw[j] = 0u;
            }
            if (prob == 0) {
                float4 *o = reinterpret_cast<float4 *>(g.part_w2 + static_cast<size_t>(split) * kH * kH +
                                                       static_cast<size_t>(r) * kH + c0);
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    o[q] = make_float4(__uint_as_float(raw[4 * q]), __uint_as_float(raw[4 * q + 1]),
                                       __uint_as_float(raw[4 * q + 2]), __uint_as_float(raw[4 * q + 3]));
            } else {
                // dW1[k][n]: the warp's lanes (consecutive n) write 128 contiguous bytes per k
                float *o = g.part_w1 + static_cast<size_t>(split) * kKP * kH + r;
#pragma unroll
                for (int j = 0; j < 32; ++j) o[static_cast<size_t>(c0 + j) * kH] = __uint_as_float(raw[j]);
            }
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
    int64_t *cursor;
    float *losses;           // replayed epochs: the step's mean loss to losses[cursor] (null: single steps)
    unsigned int *ticket;    // ... counted CTAs (zero between steps)
    int B;
    uint8_t *wimg;           // the BF16 images of W1t, W2t, W2b
};

__device__ __forceinline__ void put_img(uint8_t *wimg, int chunk, int r, int c, float x)
{
    *reinterpret_cast<__nv_bfloat16 *>(wimg + static_cast<size_t>(chunk) * kWChunk + img_off(r, c)) =
        __float2bfloat16_rn(x);
}

// BF16 copies of one weight into the images (chunks of 64 K-elements): W1[k][n] -> W1t
// (row n, col k); W2[k][n] -> W2t chunk 1 + k / 64 (row n, col k % 64) and W2b chunk
// 5 + n / 64 (row k, col n % 64).
__device__ __forceinline__ void put_weight(uint8_t *wimg, bool is_w2, int k, int n, float x)
{
    if (!is_w2) {
        put_img(wimg, 0, n, k, x);
    } else {
        put_img(wimg, 1 + (k >> 6), n, k & 63, x);
        put_img(wimg, 5 + (n >> 6), k, n & 63, x);
    }
}

// sum_{z < n} p[z * stride] in order z = 0, 1, ...: the loads of 32 partials are
// issued together, then added one after another (the order a plain loop has)
__device__ __forceinline__ float sum_partials(const float *p, int n, int64_t stride)
{
    float s = 0.0f;
    int z0 = 0;
    for (; z0 + 32 <= n; z0 += 32) {
        float x[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) x[j] = __ldg(p + static_cast<int64_t>(z0 + j) * stride);
#pragma unroll
        for (int j = 0; j < 32; ++j) s += x[j];
    }
    for (; z0 < n; ++z0) s += __ldg(p + static_cast<int64_t>(z0) * stride);
    return s;
}

// Parameter i's gradient from the partials (and its AdamW step); `cur` is the batch
// cursor of a replayed epoch.
__device__ __forceinline__ void update_param(const UpdateArgs &g, int64_t i, int64_t cur)
{
    float gr = 0.0f;
    bool is_w = false, is_w2 = false;
    int wk = 0, wn = 0;
    if (i < g.off_b1) {  // W1[k][n]
        wk = static_cast<int>(i / kH);
        wn = static_cast<int>(i % kH);
        gr = sum_partials(g.part_w1 + i, g.n_splits, static_cast<int64_t>(kH) * kKP);
        is_w = true;
    } else if (i < g.off_W2) {  // b1
        const int c = static_cast<int>(i - g.off_b1);
        gr = sum_partials(g.part_b1 + c, g.n_tiles, kH);
    } else if (i < g.off_b2) {  // W2[k][n]
        const int64_t j = i - g.off_W2;
        wk = static_cast<int>(j / kH);
        wn = static_cast<int>(j % kH);
        gr = sum_partials(g.part_w2 + j, g.n_splits, static_cast<int64_t>(kH) * kH);
        is_w = is_w2 = true;
    } else {  // b2, w3, b3 from the tile partials [dw3 | db2 | db3 | loss]
        int col;
        if (i < g.off_w3) col = kH + static_cast<int>(i - g.off_b2);
        else if (i < g.off_b3) col = static_cast<int>(i - g.off_w3);
        else col = 2 * kH;
        gr = sum_partials(g.part_head + col, g.n_tiles, 2 * kH + 2);
    }
    g.grads[i] = gr;
    if (!g.w) return;
    float bc1 = g.bc1, bc2 = g.bc2;
    if (g.bc_table) {
        bc1 = g.bc_table[2 * cur];
        bc2 = g.bc_table[2 * cur + 1];
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

// One thread per parameter; the loss sum by thread n_params, or, in a replayed epoch,
// by the CTA that finishes last (a ticket counter): it writes the step's mean loss to
// losses[cursor] and advances the cursor once every CTA has read it.
__global__ void k_update(const UpdateArgs g)
{
    __shared__ int64_t s_cur;
    __shared__ int s_last;
    pdl_trigger();
    pdl_wait();  // the partials of the tile and weight-gradient kernels
    const bool epoch = g.losses != nullptr;
    if (epoch) {
        if (threadIdx.x == 0) s_cur = *g.cursor;
        __syncthreads();
    }
    const int64_t cur = epoch ? s_cur : (g.cursor ? *g.cursor : 0);
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i < g.n_params) update_param(g, i, cur);
    else if (i == g.n_params && !epoch) *g.loss_sum = sum_partials(g.part_head + 2 * kH + 1, g.n_tiles, 2 * kH + 2);
    if (!epoch) return;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(g.ticket, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (s_last && threadIdx.x == 0) {
        __threadfence();
        const float loss = sum_partials(g.part_head + 2 * kH + 1, g.n_tiles, 2 * kH + 2);
        *g.loss_sum = loss;
        g.losses[cur] = loss / static_cast<float>(g.B);
        *g.cursor = cur + 1;
        *g.ticket = 0;
    }
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

}  // namespace

// ---------------------------------------------------------------------------
template <class... KArgs, class... Args>
cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

size_t mlp_wimg_bytes() { return kWImage; }
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
    if (y) return launch_pdl(k_tile<true>, dim3(Bp / kBM), dim3(kTileThreads), kTileSmem, s, g);
    return launch_pdl(k_tile<false>, dim3(Bp / kBM), dim3(kTileThreads), kTileSmem, s, g);
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
    return launch_pdl(k_wgrad, dim3(4, splits), dim3(kWgradThreads), kWgradSmem, s, g);
}

cudaError_t mlp_launch_update(const MlpBuffers &b, int Bp, bool adamw, float lr, float wd, float bc1, float bc2,
                              const float *bc_table, int64_t *cursor, float *losses, unsigned int *ticket, int B,
                              cudaStream_t s)
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
    g.losses = losses;
    g.ticket = ticket;
    g.B = B;
    g.wimg = static_cast<uint8_t *>(b.wimg);
    const int64_t n = b.n_params + 1;
    return launch_pdl(k_update, dim3(static_cast<unsigned>((n + 255) / 256)), dim3(256), 0, s, g);
}

cudaError_t mlp_launch_refresh(const MlpBuffers &b, cudaStream_t s)
{
    k_refresh<<<(kH * kH + 255) / 256, 256, 0, s>>>(b.params + b.off_W1, b.in_dim, b.params + b.off_W2,
                                                     static_cast<uint8_t *>(b.wimg));
    return cudaGetLastError();
}


}  // namespace gn
