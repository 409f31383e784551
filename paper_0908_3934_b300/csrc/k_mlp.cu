// Kernels of the learned connectivity estimator: an MLP in -> 256 -> 256 -> 1
// (ReLU hidden layers, sigmoid output, binary cross-entropy), BF16 tensor-core
// GEMMs with FP32 accumulation, FP32 master weights and AdamW.
//
// Precision (mirrored by the FP64 oracle): inputs, weight copies, the first hidden
// activation and the backward activations are BF16; every accumulation is FP32;
// the second hidden activation, the output layer and all reductions are FP32.
// Every reduction is done in a fixed order (per-CTA partials, then a reduction
// kernel), so results do not depend on scheduling.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "ptx.cuh"

namespace gn {
namespace {

constexpr int kH = 256;    // hidden width
constexpr int kKP = 64;    // padded input width

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// ---------------------------------------------------------------------------
// Row b of the batch is X[idx[o + b]] (or X[b] without idx), FP32 -> Xb [Bp][64]
// BF16, zero padded (columns >= in, rows >= B).  o = (*cursor) B with a device batch
// cursor (a replayed training epoch), else 0.
__device__ __forceinline__ int64_t batch_row(const int64_t *idx, const int64_t *cursor, int B, int64_t r)
{
    if (!idx) return r;
    return idx[(cursor ? *cursor * B : 0) + r];
}

__global__ void k_cast_x(const float *__restrict__ X, const int64_t *__restrict__ idx, const int64_t *__restrict__ cursor,
                         int B, int in_dim, int Bp, __nv_bfloat16 *__restrict__ Xb)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= static_cast<int64_t>(Bp) * kKP) return;
    const int r = static_cast<int>(i / kKP), c = static_cast<int>(i % kKP);
    float v = 0.0f;
    if (r < B && c < in_dim) {
        v = X[batch_row(idx, cursor, B, r) * in_dim + c];
    }
    Xb[i] = __float2bfloat16_rn(v);
}

// ---------------------------------------------------------------------------
// Layer GEMM C[m][n] = sum_k A[m][k] Bt[n][k] (A row-major [M][K] BF16, Bt row-major
// [256][K] BF16, FP32 accumulation, K a multiple of 64) with a fused epilogue:
// kReluBf16: BF16 relu(C + bias); kReluF32: FP32 relu(C + bias); kMaskBf16: BF16
// C where mask > 0 (else 0), plus per-64-row column sums of that output.
enum Epi { kReluBf16 = 0, kReluF32 = 1, kMaskBf16 = 2 };

// ---------------------------------------------------------------------------
// Every GEMM of the MLP on tcgen05: C[m][n] = sum_k A[m][k] B[n][k] (both operands
// K-contiguous BF16, FP32 accumulation in tensor memory).  One CTA of 128 threads
// computes a 128 x BN tile over `kc` chunks of 64 along K (CTA z of a split-K grid
// starts at chunk z * kc).  Chunks are double-buffered: the 128 threads copy A and B
// rows with 16-byte cp.async into the K-major core-matrix layout (8 rows x 16 bytes
// per core matrix, 128 bytes apart along K, 1024 bytes apart along rows -- thread c
// writes bytes [16c, 16c + 16) of a buffer), one thread issues four 128 x BN x 16
// MMAs per chunk and commits them to the chunk's mbarrier.  Epilogue: warp w reads
// TMEM lanes 32w .. 32w + 31 (its rows) with tcgen05.ld, 32 columns at a time:
//   kReluBf16   BF16 relu(C + bias) (+ a transposed copy [col][row])
//   kReluF32    FP32 relu(C + bias)
//   kMaskBf16   BF16 C where mask > 0, else 0 (+ transposed copy), and per-64-row
//               column sums of it to col_partial[row / 64][col] in a fixed order
//               (reduce-scatter over a warp's 32 rows, then the two warps of a group)
//   kPartF32    FP32 C tile of split z to partial[z][row][col]
//   kPartF32T   the same transposed, partial[z][col][row]
// Every wait is bounded: on a time-out the CTA sets *status, waits once more for its
// MMAs, frees its tensor memory and leaves.
enum GemmEpi { kPartF32 = 3, kPartF32T = 4 };

struct GemmArgs {
    const __nv_bfloat16 *A;  // [.][lda], rows m0 ..
    int64_t lda;
    const __nv_bfloat16 *B;  // [.][ldb], rows n0 ..
    int64_t ldb;
    int kc;                  // chunks of 64 along K per CTA
    const float *bias;
    const __nv_bfloat16 *mask;
    void *out;               // row-major, kH columns
    __nv_bfloat16 *out_t;    // transposed BF16 copy [kH][ldt], or null
    int64_t ldt;
    float *col_partial;
    float *partial;          // split-K tiles
    int64_t partial_stride;  // floats between the tiles of consecutive splits
    unsigned int *status;
};

template <int EPI, int BN>
__global__ void __launch_bounds__(128) k_gemm_tc(const GemmArgs g)
{
    constexpr int BM = 128, BK = 64;
    constexpr int kStageA = BM * BK * 2, kStageB = BN * BK * 2;  // bytes of one buffer
    constexpr uint32_t kIdesc = idesc_bf16_f32(BM, BN);
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *sA = smem_raw;                  // [2][kStageA]
    uint8_t *sB = smem_raw + 2 * kStageA;    // [2][kStageB]
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t s_tmem;
    __shared__ int s_fail;
    __shared__ float s_cs[4][BN];

    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int64_t m0 = static_cast<int64_t>(blockIdx.x) * BM;
    const int n0 = blockIdx.y * BN;
    const int64_t kbase = static_cast<int64_t>(blockIdx.z) * g.kc * BK;
    if (warp == 0) {
        tmem_alloc(&s_tmem, BN);
        tmem_relinquish();
    }
    if (t == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        fence_barrier_init();
        s_fail = 0;
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();
    const uint32_t tmem = s_tmem;

    auto load = [&](int stage, int64_t k0) {
        uint8_t *a = sA + stage * kStageA;
        uint8_t *b = sB + stage * kStageB;
#pragma unroll
        for (int i = 0; i < BM * 8 / 128; ++i) {
            const int c = t + 128 * i;  // 16-byte piece: row (c & 7) + 8 (c >> 6), K piece (c >> 3) & 7
            const int r = (c & 7) + 8 * (c >> 6), kp = (c >> 3) & 7;
            cp_async16(a + 16 * c, g.A + (m0 + r) * g.lda + k0 + kp * 8);
            if (c < BN * 8) cp_async16(b + 16 * c, g.B + static_cast<int64_t>(n0 + r) * g.ldb + k0 + kp * 8);
        }
        cp_async_commit();
    };

    const int nk = g.kc;
    bool ok = true;
    load(0, kbase);
    for (int kc = 0; kc < nk; ++kc) {
        if (kc + 1 < nk) {
            // buffer (kc + 1) & 1 was last read by the MMAs of chunk kc - 1
            if (kc >= 1 && !mbar_wait_bounded(&s_bar[(kc - 1) & 1], ((kc - 1) >> 1) & 1, kDefaultWaitLimit)) ok = false;
            load((kc + 1) & 1, kbase + static_cast<int64_t>(kc + 1) * BK);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        fence_async_shared();
        __syncthreads();
        if (t == 0) {
            tc_fence_after_sync();
            const uint8_t *a = sA + (kc & 1) * kStageA;
            const uint8_t *b = sB + (kc & 1) * kStageB;
#pragma unroll
            for (int ks = 0; ks < BK / 16; ++ks)
                tc_mma_bf16(tmem, smem_desc_kmajor(a + ks * 256, 128, 1024), smem_desc_kmajor(b + ks * 256, 128, 1024),
                            kIdesc, (kc | ks) != 0);
            tc_commit(&s_bar[kc & 1]);
        }
    }
    // the last chunk's commit covers every MMA of the tile
    if (!mbar_wait_bounded(&s_bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1, kDefaultWaitLimit)) ok = false;
    if (!ok) {
        s_fail = 1;
        atomicOr(g.status, kStatusTimeout);
        mbar_wait_bounded(&s_bar[(nk - 1) & 1], ((nk - 1) >> 1) & 1, kDefaultWaitLimit);
    }
    tc_fence_before_sync();
    __syncthreads();
    tc_fence_after_sync();

    if (!s_fail) {
        const int64_t row = m0 + 32 * warp + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 32) {
            uint32_t raw[32];
            tmem_ld32(tmem + (static_cast<uint32_t>(32 * warp) << 16) + c0, raw);
            tmem_ld_wait();
            float v[32];
            const int col0 = n0 + c0;
            uint4 mk[4];  // the row's 32 mask values, 16 bytes at a time
            if constexpr (EPI == kMaskBf16) {
                const uint4 *mp = reinterpret_cast<const uint4 *>(g.mask + row * kH + col0);
#pragma unroll
                for (int q = 0; q < 4; ++q) mk[q] = mp[q];
            }
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const float acc = __uint_as_float(raw[j]);
                if constexpr (EPI == kMaskBf16) {
                    const uint32_t w = (&mk[j >> 3].x)[(j & 7) >> 1];
                    const uint16_t h = static_cast<uint16_t>((j & 1) ? (w >> 16) : (w & 0xFFFFu));
                    v[j] = __bfloat162float(__ushort_as_bfloat16(h)) > 0.0f ? acc : 0.0f;
                } else if constexpr (EPI == kReluBf16 || EPI == kReluF32)
                    v[j] = fmaxf(acc + g.bias[col0 + j], 0.0f);
                else
                    v[j] = acc;
            }
            if constexpr (EPI == kReluF32 || EPI == kPartF32) {
                float *base = EPI == kReluF32 ? static_cast<float *>(g.out) + row * kH + col0
                                              : g.partial + blockIdx.z * g.partial_stride + row * kH + col0;
                float4 *o = reinterpret_cast<float4 *>(base);
#pragma unroll
                for (int q = 0; q < 8; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
            } else if constexpr (EPI == kPartF32T) {
                // [col][row]: the warp's lanes write 32 consecutive rows of each column
                float *base = g.partial + blockIdx.z * g.partial_stride;
#pragma unroll
                for (int j = 0; j < 32; ++j) base[static_cast<int64_t>(col0 + j) * kH + row] = v[j];
            } else {
                uint4 *o = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(g.out) + row * kH + col0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    uint32_t w[4];
#pragma unroll
                    for (int h = 0; h < 4; ++h) {
                        const __nv_bfloat162 pr = __floats2bfloat162_rn(v[8 * q + 2 * h], v[8 * q + 2 * h + 1]);
                        w[h] = *reinterpret_cast<const uint32_t *>(&pr);
                    }
                    o[q] = make_uint4(w[0], w[1], w[2], w[3]);
                }
                if (g.out_t) {
#pragma unroll
                    for (int j = 0; j < 32; ++j)
                        g.out_t[static_cast<int64_t>(col0 + j) * g.ldt + row] = __float2bfloat16_rn(v[j]);
                }
            }
            if constexpr (EPI == kMaskBf16) {
                // reduce-scatter over the warp's rows: lane l ends with column c0 + l
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
                s_cs[warp][c0 + lane] = v[0];
            }
        }
        if constexpr (EPI == kMaskBf16) {
            __syncthreads();
            // t = column: rows 0..63 are warps 0, 1; rows 64..127 warps 2, 3
            const int64_t grp = static_cast<int64_t>(blockIdx.x) * 2;
            if (t < BN) {
                g.col_partial[grp * kH + n0 + t] = s_cs[0][t] + s_cs[1][t];
                g.col_partial[(grp + 1) * kH + n0 + t] = s_cs[2][t] + s_cs[3][t];
            }
        }
    }
    tc_fence_before_sync();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after_sync();
        tmem_dealloc(tmem, BN);
    }
}

// BF16 transpose in[R][C] -> out[C][R] through 32 x 32 shared-memory tiles.
__global__ void k_transpose_bf16(const __nv_bfloat16 *__restrict__ in, int R, int C, __nv_bfloat16 *__restrict__ out)
{
    __shared__ __nv_bfloat16 tile[32][34];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    for (int i = ty; i < 32; i += 8)
        if (r0 + i < R && c0 + tx < C) tile[i][tx] = in[static_cast<int64_t>(r0 + i) * C + c0 + tx];
    __syncthreads();
    for (int i = ty; i < 32; i += 8)
        if (c0 + i < C && r0 + tx < R) out[static_cast<int64_t>(c0 + i) * R + r0 + tx] = tile[tx][i];
}

// ---------------------------------------------------------------------------
// Output layer and loss: z = h2 . w3 + b3, p = sigmoid(z).  With labels, also the
// first backward step: dz = (p - y) / B, dh2 = dz w3 [h2 > 0] (BF16 for the
// GEMMs), and per-CTA partial sums (fixed order) of dw3 = sum dz h2,
// db2 = sum dh2, db3 = sum dz and the BCE loss.  One warp per row, 8 warps per CTA,
// `rows_per_cta` rows per CTA.
__global__ void __launch_bounds__(256) k_head(const float *__restrict__ H2, const float *__restrict__ w3,
                                              const float *__restrict__ b3p, const float *__restrict__ y,
                                              const int64_t *__restrict__ idx, const int64_t *__restrict__ cursor,
                                              int B, int rows_per_cta,
                                              float *__restrict__ p_out, __nv_bfloat16 *__restrict__ dH2,
                                              float *__restrict__ partial)
{
    __shared__ float s_w3[kH];
    __shared__ float s_acc[8][2 * kH + 2];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    s_w3[t] = w3[t];
    for (int i = t; i < 8 * (2 * kH + 2); i += 256) (&s_acc[0][0])[i] = 0.0f;
    __syncthreads();
    const int64_t r0 = static_cast<int64_t>(blockIdx.x) * rows_per_cta;
    const float b3 = *b3p;
    const bool train = y != nullptr;
    const float inv_b = 1.0f / static_cast<float>(B);
    for (int rr = warp; rr < rows_per_cta; rr += 8) {
        const int64_t r = r0 + rr;
        float h[8];
        float z = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            h[q] = H2[r * kH + q * 32 + lane];
            z = fmaf(h[q], s_w3[q * 32 + lane], z);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) z += __shfl_xor_sync(0xffffffffu, z, o);
        z += b3;
        const float p = 1.0f / (1.0f + expf(-z));
        if (lane == 0 && r < B) p_out[r] = p;
        if (!train) continue;
        const bool valid = r < B;
        const float yy = valid ? y[batch_row(idx, cursor, B, r)] : 0.0f;
        const float dz = valid ? (p - yy) * inv_b : 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int k = q * 32 + lane;
            const float d = h[q] > 0.0f ? dz * s_w3[k] : 0.0f;
            dH2[r * kH + k] = __float2bfloat16_rn(d);
            s_acc[warp][k] += dz * h[q];      // dw3
            s_acc[warp][kH + k] += d;         // db2
        }
        if (lane == 0 && valid) {
            s_acc[warp][2 * kH] += dz;
            const float eps = 1e-12f;
            s_acc[warp][2 * kH + 1] += -(yy * logf(p + eps) + (1.0f - yy) * logf(1.0f - p + eps));
        }
    }
    if (!train) return;
    __syncthreads();
    for (int i = t; i < 2 * kH + 2; i += 256) {
        float s = 0.0f;
        for (int w = 0; w < 8; ++w) s += s_acc[w][i];
        partial[static_cast<int64_t>(blockIdx.x) * (2 * kH + 2) + i] = s;
    }
}

// Sum n partial vectors of length len in order: out[i] = sum_j part[j][i].
__global__ void k_sum_partials(const float *__restrict__ part, int n, int64_t len, float *__restrict__ out)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= len) return;
    float s = 0.0f;
    for (int j = 0; j < n; ++j) s += part[static_cast<int64_t>(j) * len + i];
    out[i] = s;
}

// The same for short vectors with many partials: a warp per element, lane l adds
// partials l, l + 32, ... in order, then the warp's butterfly (a fixed order too).
__global__ void k_sum_partials_warp(const float *__restrict__ part, int n, int64_t len, float *__restrict__ out)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x / 32) + threadIdx.x / 32;
    const int lane = threadIdx.x & 31;
    if (i >= len) return;
    float s = 0.0f;
    for (int j = lane; j < n; j += 32) s += part[static_cast<int64_t>(j) * len + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[i] = s;
}

// End of a replayed training step: its mean loss to losses[cursor], then the
// cursor moves to the next batch.
__global__ void k_epoch_tail(const float *__restrict__ loss_sum, int B, int64_t *cursor, float *__restrict__ losses)
{
    losses[*cursor] = *loss_sum / static_cast<float>(B);
    *cursor += 1;
}

// AdamW on FP32 masters (decoupled weight decay), then the BF16 copies:
// W1t[n][k] (k < 64), W2t[n][k] and W2b[k][n] = W2[k][n].
// With a batch cursor the bias corrections come from bc_table[2 cursor + {0, 1}]
// (filled by the host with the same arithmetic as the scalar path).
__global__ void k_adamw(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                        int64_t n, float lr, float beta1, float beta2, float eps, float wd, float bc1, float bc2,
                        const float *__restrict__ bc_table, const int64_t *__restrict__ cursor)
{
    const int64_t i = blockIdx.x * static_cast<int64_t>(blockDim.x) + threadIdx.x;
    if (i >= n) return;
    if (bc_table) {
        bc1 = bc_table[2 * *cursor];
        bc2 = bc_table[2 * *cursor + 1];
    }
    const float gi = g[i];
    const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
    const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float mhat = mi / bc1, vhat = vi / bc2;
    w[i] = w[i] * (1.0f - lr * wd) - lr * mhat / (sqrtf(vhat) + eps);
}

__global__ void k_refresh_bf16(const float *__restrict__ W1, int in_dim, const float *__restrict__ W2,
                               __nv_bfloat16 *__restrict__ W1t, __nv_bfloat16 *__restrict__ W2t,
                               __nv_bfloat16 *__restrict__ W2b)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < kH * kKP) {
        const int n = i / kKP, k = i % kKP;
        W1t[i] = __float2bfloat16_rn(k < in_dim ? W1[k * kH + n] : 0.0f);
    }
    if (i < kH * kH) {
        const int n = i / kH, k = i % kH;
        W2t[i] = __float2bfloat16_rn(W2[k * kH + n]);
        W2b[i] = __float2bfloat16_rn(W2[i]);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
cudaError_t mlp_launch_cast(const float *X, const int64_t *idx, const int64_t *cursor, int B, int in_dim, int Bp,
                            void *Xb, cudaStream_t s)
{
    const int64_t n = static_cast<int64_t>(Bp) * kKP;
    k_cast_x<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(X, idx, cursor, B, in_dim, Bp,
                                                                   static_cast<__nv_bfloat16 *>(Xb));
    return cudaGetLastError();
}

template <int BN>
constexpr int gemm_smem() { return 2 * 128 * 64 * 2 + 2 * BN * 64 * 2; }  // two buffers each of A and B chunks

template <int EPI, int BN>
cudaError_t gemm_attr()
{
    return cudaFuncSetAttribute(k_gemm_tc<EPI, BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, gemm_smem<BN>());
}

cudaError_t mlp_prepare()
{
    cudaError_t e = gemm_attr<kReluBf16, 128>();
    if (e == cudaSuccess) e = gemm_attr<kReluF32, 128>();
    if (e == cudaSuccess) e = gemm_attr<kMaskBf16, 128>();
    if (e == cudaSuccess) e = gemm_attr<kPartF32, 128>();
    if (e == cudaSuccess) e = gemm_attr<kPartF32T, 64>();
    return e;
}

cudaError_t mlp_launch_layer(int epi, const void *A, int Bp, int K, const void *Bt, const float *bias, const void *mask,
                             void *out, void *out_t, float *col_partial, unsigned int *status, cudaStream_t s)
{
    if (Bp % 128 != 0 || K % 64 != 0) return cudaErrorInvalidValue;
    GemmArgs g{};
    g.A = static_cast<const __nv_bfloat16 *>(A);
    g.lda = K;
    g.B = static_cast<const __nv_bfloat16 *>(Bt);
    g.ldb = K;
    g.kc = K / 64;
    g.bias = bias;
    g.mask = static_cast<const __nv_bfloat16 *>(mask);
    g.out = out;
    g.out_t = static_cast<__nv_bfloat16 *>(out_t);
    g.ldt = Bp;
    g.col_partial = col_partial;
    g.status = status;
    const dim3 grid(Bp / 128, kH / 128);
    switch (epi) {
        case kReluBf16: k_gemm_tc<kReluBf16, 128><<<grid, 128, gemm_smem<128>(), s>>>(g); break;
        case kReluF32: k_gemm_tc<kReluF32, 128><<<grid, 128, gemm_smem<128>(), s>>>(g); break;
        case kMaskBf16: k_gemm_tc<kMaskBf16, 128><<<grid, 128, gemm_smem<128>(), s>>>(g); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t mlp_launch_wgrad(const void *AT, int M, const void *BT, int N, int Bp, int chunk, bool transposed,
                             float *partial, unsigned int *status, cudaStream_t s)
{
    if (M % 128 != 0 || Bp % chunk != 0 || chunk % 64 != 0 || (N != 256 && N != 64) || (N == 64) != transposed)
        return cudaErrorInvalidValue;
    GemmArgs g{};
    g.A = static_cast<const __nv_bfloat16 *>(AT);
    g.lda = Bp;
    g.B = static_cast<const __nv_bfloat16 *>(BT);
    g.ldb = Bp;
    g.kc = chunk / 64;
    g.partial = partial;
    g.partial_stride = static_cast<int64_t>(M) * N;
    g.status = status;
    if (transposed) {
        k_gemm_tc<kPartF32T, 64><<<dim3(M / 128, 1, Bp / chunk), 128, gemm_smem<64>(), s>>>(g);
    } else {
        k_gemm_tc<kPartF32, 128><<<dim3(M / 128, N / 128, Bp / chunk), 128, gemm_smem<128>(), s>>>(g);
    }
    return cudaGetLastError();
}

cudaError_t mlp_launch_transpose(const void *in, int R, int C, void *out, cudaStream_t s)
{
    const dim3 grid((C + 31) / 32, (R + 31) / 32);
    k_transpose_bf16<<<grid, dim3(32, 8), 0, s>>>(static_cast<const __nv_bfloat16 *>(in), R, C,
                                                  static_cast<__nv_bfloat16 *>(out));
    return cudaGetLastError();
}

cudaError_t mlp_launch_head(const float *H2, const float *w3, const float *b3, const float *y, const int64_t *idx,
                            const int64_t *cursor, int B, int Bp, int rows_per_cta, float *p, void *dH2, float *partial,
                            cudaStream_t s)
{
    k_head<<<Bp / rows_per_cta, 256, 0, s>>>(H2, w3, b3, y, idx, cursor, B, rows_per_cta, p,
                                              static_cast<__nv_bfloat16 *>(dH2), partial);
    return cudaGetLastError();
}

cudaError_t mlp_launch_sum(const float *part, int n, int64_t len, float *out, cudaStream_t s)
{
    if (len <= 4096 && n > 32)
        k_sum_partials_warp<<<static_cast<unsigned>((len + 7) / 8), 256, 0, s>>>(part, n, len, out);
    else
        k_sum_partials<<<static_cast<unsigned>((len + 255) / 256), 256, 0, s>>>(part, n, len, out);
    return cudaGetLastError();
}

cudaError_t mlp_launch_adamw(float *w, const float *g, float *m, float *v, int64_t n, float lr, float beta1, float beta2,
                             float eps, float wd, float bc1, float bc2, const float *bc_table, const int64_t *cursor,
                             cudaStream_t s)
{
    k_adamw<<<static_cast<unsigned>((n + 255) / 256), 256, 0, s>>>(w, g, m, v, n, lr, beta1, beta2, eps, wd, bc1, bc2,
                                                                   bc_table, cursor);
    return cudaGetLastError();
}

cudaError_t mlp_launch_epoch_tail(const float *loss_sum, int B, int64_t *cursor, float *losses, cudaStream_t s)
{
    k_epoch_tail<<<1, 1, 0, s>>>(loss_sum, B, cursor, losses);
    return cudaGetLastError();
}

cudaError_t mlp_launch_refresh(const float *W1, int in_dim, const float *W2, void *W1t, void *W2t, void *W2b,
                               cudaStream_t s)
{
    k_refresh_bf16<<<(kH * kH + 255) / 256, 256, 0, s>>>(W1, in_dim, W2, static_cast<__nv_bfloat16 *>(W1t),
                                                          static_cast<__nv_bfloat16 *>(W2t),
                                                          static_cast<__nv_bfloat16 *>(W2b));
    return cudaGetLastError();
}

}  // namespace gn
