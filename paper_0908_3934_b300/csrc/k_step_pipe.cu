// Persistent, bulk-copy pipelined step kernel: one launch advances the whole
// network by one step, as k_step does, but each CTA walks a strided list of row
// blocks and keeps S row blocks in flight.
//
// Per row block b (rows [r0, r1), edges [e0, e1) of the by-target list):
//   thread 0 (producer) issues 1D bulk asynchronous copies (TMA) of
//     - the packed edge keys and weights of [e0, e1)   (16-byte aligned superset)
//     - row_ptr[r0 .. r1], the current state v~(n) of rows [r0, r1) (ring slot n)
//       and their (w~, c~)
//   into stage (i mod S) of shared memory, S - 1 blocks ahead of the block being
//   processed, completing on that stage's mbarrier;
//   every thread then waits on the mbarrier, gathers the delayed values
//   ring[(n - D) & (R - 1)][src] of its edges (the only global reads left on the
//   critical path; they hit the live history slots in L2), parks w * v~ in shared
//   memory, the rows are summed and the fused node update writes step n + 1.
// The edge stream thus flows from HBM while earlier blocks wait on their gathers.
// Rows longer than one block's capacity read their edges directly from global.
//
// Every mbarrier wait is bounded; a wait that gives up sets kStatusTimeout in the
// status word, the CTA stops taking blocks, waits (bounded) for its own copies in
// flight and exits; the host reports GN_ETIMEOUT.
#include "step_common.cuh"

namespace gn {
namespace {

using namespace step;

constexpr uint32_t kWaitLimit = 1u << 22;

template <int T, int EPT, int KEYB>
struct PipeLayout {
    static constexpr int CAP = T * EPT;
    static constexpr int MAXR = T;
    static constexpr int align(int x) { return (x + 127) & ~127; }
    static constexpr int KEYS = 0;
    static constexpr int W = KEYS + align(CAP * KEYB);
    static constexpr int RP = W + align(CAP * 4);
    static constexpr int V = RP + align((MAXR + 8) * 4);
    static constexpr int WC = V + align((MAXR + 8) * 4);
    static constexpr int STAGE = WC + align((MAXR + 4) * 8);
};

template <int T, int EPT, int S, int KEYB>
constexpr int pipe_smem()
{
    using L = PipeLayout<T, EPT, KEYB>;
    return S * L::STAGE + L::CAP * 4 + T * 4 + 128;
}

template <int T, int EPT, int S, int KEYB, bool kStream>
__device__ __forceinline__ void issue_block(const StepArgs &a, int b, uint8_t *stage, uint64_t *bar, int64_t slot_n,
                                            uint64_t pol_edges)
{
    using L = PipeLayout<T, EPT, KEYB>;
    const int4 d = a.bdesc[b];  // r0, r1, e0, e1
    const bool lng = (d.y - d.x == 1) && (d.w - d.z > L::CAP - 3);
    const int ea = d.z & ~3;
    const int ee = lng ? ea : ((d.w + 3) & ~3);
    const int ra = d.x & ~3, re = (d.y + 4) & ~3;  // row_ptr needs r0..r1 inclusive
    const int wa = d.x & ~1, we = (d.y + 1) & ~1;
    const uint32_t bk = static_cast<uint32_t>(ee - ea) * KEYB;
    const uint32_t bw = static_cast<uint32_t>(ee - ea) * 4;
    const uint32_t br = static_cast<uint32_t>(re - ra) * 4;
    const uint32_t bwc = static_cast<uint32_t>(we - wa) * 8;
    mbar_arrive_expect_tx(bar, bk + bw + 2 * br + bwc);
    if (bk) {
        const uint8_t *ks = static_cast<const uint8_t *>(a.ekey) + static_cast<int64_t>(ea) * KEYB;
        if constexpr (kStream) {
            bulk_g2s_hint(stage + L::KEYS, ks, bk, bar, pol_edges);
            bulk_g2s_hint(stage + L::W, a.ew + ea, bw, bar, pol_edges);
        } else {
            bulk_g2s(stage + L::KEYS, ks, bk, bar);
            bulk_g2s(stage + L::W, a.ew + ea, bw, bar);
        }
    }
    bulk_g2s(stage + L::RP, a.row_ptr + ra, br, bar);
    bulk_g2s(stage + L::V, a.ring + slot_n * a.ring_stride + ra, br, bar);
    bulk_g2s(stage + L::WC, a.wc + wa, bwc, bar);
}

template <int kM, int T, int EPT, int S, int KEYB, bool kStream>
__global__ void __launch_bounds__(T) k_step_pipe(const StepArgs a, const int k)
{
    using L = PipeLayout<T, EPT, KEYB>;
    constexpr int CAP = L::CAP;
    constexpr bool kPacked = KEYB == 4;
    extern __shared__ __align__(128) uint8_t smem[];
    uint8_t *stages = smem;
    float *s_prod = reinterpret_cast<float *>(smem + S * L::STAGE);
    float *s_long = s_prod + CAP;
    uint64_t *bars = reinterpret_cast<uint64_t *>(s_long + T);
    int *s_abort = reinterpret_cast<int *>(bars + S);

    const int t = threadIdx.x;
    const int64_t n = *a.d_step + k;
    const int64_t slot_n = n & a.ring_mask;
    const int nb = a.n_blocks;
    const uint64_t pol_edges = l2_evict_first();
    const uint64_t pol_ring = l2_evict_last();

    if (t == 0) {
        for (int s = 0; s < S; ++s) mbar_init(&bars[s], 1);
        *s_abort = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (t == 0)
        for (int s = 0; s < S - 1; ++s) {
            const int b = blockIdx.x + s * gridDim.x;
            if (b < nb) issue_block<T, EPT, S, KEYB, kStream>(a, b, stages + s * L::STAGE, &bars[s], slot_n, pol_edges);
        }

    int i = 0;
    for (;; ++i) {
        const int b = blockIdx.x + i * gridDim.x;
        if (b >= nb) break;
        if (t == 0) {
            const int bn = blockIdx.x + (i + S - 1) * gridDim.x;
            const int sn = (i + S - 1) % S;
            if (bn < nb)
                issue_block<T, EPT, S, KEYB, kStream>(a, bn, stages + sn * L::STAGE, &bars[sn], slot_n, pol_edges);
        }
        const int st = i % S;
        uint8_t *sb = stages + st * L::STAGE;
        // the descriptor comes from global memory (valid even if the wait gives up)
        const int4 d = __ldg(a.bdesc + b);
        const bool ok = mbar_wait_bounded(&bars[st], (i / S) & 1, kWaitLimit);
        if (!ok) *s_abort = 1;

        const int r0 = d.x, r1 = d.y, e0 = d.z, e1 = d.w;
        const int nr = r1 - r0;
        const int ra = r0 & ~3, wa = r0 & ~1;
        const int *s_rp = reinterpret_cast<const int *>(sb + L::RP) + (r0 - ra);
        const float *s_v = reinterpret_cast<const float *>(sb + L::V) + (r0 - ra);
        const float2 *s_wc = reinterpret_cast<const float2 *>(sb + L::WC) + (r0 - wa);
        const bool lng = (nr == 1) && (e1 - e0 > CAP - 3);

        if (lng) {
            float p = 0.0f;
            if (ok)
                for (int base = e0 & ~3; base < e1; base += CAP) {
#pragma unroll
                    for (int q = 0; q < EPT / 4; ++q) {
                        const int eb = base + 4 * (t + T * q);
                        const EdgeQuad<kPacked> qd = load_quad<kPacked, kStream>(a, eb);
                        const float4 wv = ld_weight4<kStream>(a.ew + eb);
                        const float wq[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                        for (int j = 0; j < 4; ++j)
                            if (eb + j >= e0 && eb + j < e1)
                                p = fmaf(wq[j], gather_hint(a, n, qd.src[j], qd.d[j], pol_ring), p);
                    }
                }
            p = warp_sum(p);
            if ((t & 31) == 0) s_long[t >> 5] = p;
            __syncthreads();
            if (*s_abort) break;
            if (t == 0) {
                float S_in = 0.0f;
                for (int w = 0; w < T / 32; ++w) S_in += s_long[w];
                node_update<kM>(a, r0, n, s_v[0], s_wc[0], S_in);
            }
            __syncthreads();
            continue;
        }

        // gathers of the block's edges (keys and weights already in shared memory)
        if (ok) {
            const int ea = e0 & ~3;
#pragma unroll
            for (int q = 0; q < EPT / 4; ++q) {
                const int off = 4 * (t + T * q);
                if (ea + off >= e1) break;
                uint32_t src[4], dd[4];
                if constexpr (kPacked) {
                    const uint4 kv = *reinterpret_cast<const uint4 *>(sb + L::KEYS + off * 4);
                    const uint32_t kk[4] = {kv.x, kv.y, kv.z, kv.w};
                    const uint32_t m = (1u << a.dbits) - 1u;
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        src[j] = kk[j] >> a.dbits;
                        dd[j] = kk[j] & m;
                    }
                } else {
                    const uint4 k0 = *reinterpret_cast<const uint4 *>(sb + L::KEYS + off * 8);
                    const uint4 k1 = *reinterpret_cast<const uint4 *>(sb + L::KEYS + off * 8 + 16);
                    src[0] = k0.x; dd[0] = k0.y; src[1] = k0.z; dd[1] = k0.w;
                    src[2] = k1.x; dd[2] = k1.y; src[3] = k1.z; dd[3] = k1.w;
                }
                const float4 wv = *reinterpret_cast<const float4 *>(sb + L::W + off * 4);
                const float wq[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int e = ea + off + j;
                    if (e >= e0 && e < e1) s_prod[e - e0] = wq[j] * gather_hint(a, n, src[j], dd[j], pol_ring);
                }
            }
        }
        __syncthreads();
        if (*s_abort) break;

        // row sums: short rows by their own thread, long rows by a warp
        float S_in = 0.0f;
        bool warp_row = false;
        if (t < nr) {
            const int a0 = s_rp[t] - e0, a1 = s_rp[t + 1] - e0;
            warp_row = (a1 - a0) > kWarpRow;
            if (!warp_row)
                for (int q = a0; q < a1; ++q) S_in += s_prod[q];
        }
        {
            const int lane = t & 31;
            for (int rr = t >> 5; rr < nr; rr += T / 32) {
                const int a0 = s_rp[rr] - e0, a1 = s_rp[rr + 1] - e0;
                if (a1 - a0 > kWarpRow) {
                    float p = 0.0f;
                    for (int q = a0 + lane; q < a1; q += 32) p += s_prod[q];
                    p = warp_sum(p);
                    if (lane == 0) s_long[rr] = p;
                }
            }
        }
        __syncthreads();
        if (warp_row) S_in = s_long[t];
        if (t < nr) node_update<kM>(a, r0 + t, n, s_v[t], s_wc[t], S_in);
        __syncthreads();  // stage st and s_prod are free again
    }

    if (*s_abort) {
        if (t == 0) {
            atomicOr(a.status, kStatusTimeout);
            // let the copies this CTA still has in flight land before it exits
            for (int j = i; j < i + S; ++j) {
                const int bj = blockIdx.x + j * gridDim.x;
                if (bj < nb) mbar_wait_bounded(&bars[j % S], (j / S) & 1, kWaitLimit);
            }
        }
    }
}

template <int kM, int T, int EPT, int S, int KEYB, bool kStream>
cudaError_t launch_variant(const StepArgs &a, int grid, int k, cudaStream_t s)
{
    constexpr int smem = pipe_smem<T, EPT, S, KEYB>();
    k_step_pipe<kM, T, EPT, S, KEYB, kStream><<<grid, T, smem, s>>>(a, k);
    return cudaGetLastError();
}

template <int kM, int T, int EPT, int S, int KEYB, bool kStream>
cudaError_t prepare_variant(int *ctas)
{
    constexpr int smem = pipe_smem<T, EPT, S, KEYB>();
    cudaError_t e = cudaFuncSetAttribute(k_step_pipe<kM, T, EPT, S, KEYB, kStream>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, k_step_pipe<kM, T, EPT, S, KEYB, kStream>, T, smem);
}

constexpr int kT = 256, kEPT = 8, kS = 3;  // shape 0 of kStepShapes

}  // namespace

int step_pipe_smem_bytes(bool packed)
{
    return packed ? pipe_smem<kT, kEPT, kS, 4>() : pipe_smem<kT, kEPT, kS, 8>();
}

cudaError_t step_pipe_prepare(int model, bool packed, bool stream_edges, int *ctas_per_sm)
{
    return with_model(model, [&](auto m) {
        constexpr int M = decltype(m)::value;
        if (packed)
            return stream_edges ? prepare_variant<M, kT, kEPT, kS, 4, true>(ctas_per_sm)
                                : prepare_variant<M, kT, kEPT, kS, 4, false>(ctas_per_sm);
        return stream_edges ? prepare_variant<M, kT, kEPT, kS, 8, true>(ctas_per_sm)
                            : prepare_variant<M, kT, kEPT, kS, 8, false>(ctas_per_sm);
    });
}

cudaError_t launch_step_pipe(const StepArgs &a, int grid, int k, bool packed, bool stream_edges, cudaStream_t s)
{
    if (grid <= 0 || a.n_blocks <= 0) return cudaSuccess;
    return with_model(a.model, [&](auto m) {
        constexpr int M = decltype(m)::value;
        if (packed)
            return stream_edges ? launch_variant<M, kT, kEPT, kS, 4, true>(a, grid, k, s)
                                : launch_variant<M, kT, kEPT, kS, 4, false>(a, grid, k, s);
        return stream_edges ? launch_variant<M, kT, kEPT, kS, 8, true>(a, grid, k, s)
                            : launch_variant<M, kT, kEPT, kS, 8, false>(a, grid, k, s);
    });
}

}  // namespace gn
