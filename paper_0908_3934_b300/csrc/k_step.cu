// The fused step kernel: one launch advances every node of a network by dt.
//
// One CTA owns a row block -- consecutive target nodes (rows of the by-target
// edge list) holding at most kStepCap - 3 edges, or one longer row on its own.
//   1. Each thread prefetches the state of "its" row (v~(n) from the ring, w~, c~).
//   2. The CTA streams its edge chunk with 16-byte loads (coalesced: a warp reads
//      512 contiguous bytes per load), gathers the delayed value of each edge,
//      S_j(n) = sum_e w_e v~_src(n - D_e)      (Eq. Yjset, Sec. 2)
//      read from ring slot (n - D_e) & (R - 1), and parks w_e * v~ in shared memory.
//   3. Row sums: short rows by their own thread, long rows by a whole warp with a
//      shuffle reduction.
//   4. Per node: stimulus U (pulses, Philox background), the FHN Euler update about
//      the rest point (Sec. 3.1, Eq. fnstate), the history write, the low-pass
//      readout and, on sample steps, the noisy observation (Sec. 3.3), events
//      and first arrivals.
// The kernel boundary is the step barrier: every read is of step n (or older),
// every write is of step n + 1, and slot (n + 1) & (R - 1) is never read in step n
// because every delay is at most R - 2.
#include "step_common.cuh"

namespace gn {
namespace {

using namespace step;

template <int T, int EPT, bool kPacked, bool kStream>
__global__ void __launch_bounds__(T) k_step(const StepArgs a, const int k)
{
    constexpr int CAP = T * EPT;
    constexpr int kWarpRow = 48;  // rows longer than this are summed by a warp
    __shared__ float s_prod[CAP];
    __shared__ float s_long[T];
    __shared__ int s_rp[T + 1];

    const int64_t n = *a.d_step + k;
    const int t = threadIdx.x;
    const int r0 = a.blk[blockIdx.x], r1 = a.blk[blockIdx.x + 1];
    const int nr = r1 - r0;
    const int e0 = a.row_ptr[r0], e1 = a.row_ptr[r1];
    const int r = r0 + t;

    float v = 0.0f;
    float2 wc = make_float2(0.0f, 0.0f);
    if (t < nr) {
        v = a.ring[(n & a.ring_mask) * a.ring_stride + r];
        wc = a.wc[r];
        s_rp[t] = a.row_ptr[r];
    }
    if (t == 0) s_rp[nr] = e1;

    if (nr == 1 && e1 - e0 > CAP - 3) {
        // one long row: the whole CTA loops over chunks of its edges
        float p = 0.0f;
        for (int base = e0 & ~3; base < e1; base += CAP) {
#pragma unroll
            for (int i = 0; i < EPT / 4; ++i) {
                const int eb = base + 4 * (t + T * i);
                const EdgeQuad<kPacked> q = load_quad<kPacked, kStream>(a, eb);
                const float4 wv = ld_weight4<kStream>(a.ew + eb);
                const float wq[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (eb + j >= e0 && eb + j < e1) p = fmaf(wq[j], gather(a, n, q.src[j], q.d[j]), p);
            }
        }
        p = warp_sum(p);
        if ((t & 31) == 0) s_long[t >> 5] = p;
        __syncthreads();
        if (t == 0) {
            float S = 0.0f;
            for (int i = 0; i < T / 32; ++i) S += s_long[i];
            node_update(a, r0, n, v, wc, S);
        }
        return;
    }

    // 2. stream the chunk [e0, e1) and park the delayed products in shared memory
    const int ebase = e0 & ~3;
#pragma unroll
    for (int i = 0; i < EPT / 4; ++i) {
        const int eb = ebase + 4 * (t + T * i);
        if (eb >= e1) break;
        const EdgeQuad<kPacked> q = load_quad<kPacked, kStream>(a, eb);
        const float4 wv = ld_weight4<kStream>(a.ew + eb);
        const float wq[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = eb + j;
            if (e >= e0 && e < e1) s_prod[e - e0] = wq[j] * gather(a, n, q.src[j], q.d[j]);
        }
    }
    __syncthreads();

    // 3. row sums
    float S = 0.0f;
    bool warp_row = false;
    if (t < nr) {
        const int a0 = s_rp[t] - e0, a1 = s_rp[t + 1] - e0;
        warp_row = (a1 - a0) > kWarpRow;
        if (!warp_row)
            for (int i = a0; i < a1; ++i) S += s_prod[i];
    }
    {
        const int lane = t & 31;
        for (int rr = t >> 5; rr < nr; rr += T / 32) {
            const int a0 = s_rp[rr] - e0, a1 = s_rp[rr + 1] - e0;
            if (a1 - a0 > kWarpRow) {
                float p = 0.0f;
                for (int i = a0 + lane; i < a1; i += 32) p += s_prod[i];
                p = warp_sum(p);
                if (lane == 0) s_long[rr] = p;
            }
        }
    }
    __syncthreads();
    if (warp_row) S = s_long[t];

    // 4. node update
    if (t < nr) node_update(a, r, n, v, wc, S);
}

__global__ void k_advance(int64_t *d_step, int64_t by)
{
    *d_step += by;
}

}  // namespace

cudaError_t launch_step(const StepArgs &a, int n_blocks, int k, bool packed, bool stream_edges,
                        cudaStream_t s)
{
    constexpr int T = kStepThreads, EPT = kStepEPT;
    if (n_blocks <= 0) return cudaSuccess;
    if (packed) {
        if (stream_edges)
            k_step<T, EPT, true, true><<<n_blocks, T, 0, s>>>(a, k);
        else
            k_step<T, EPT, true, false><<<n_blocks, T, 0, s>>>(a, k);
    } else {
        if (stream_edges)
            k_step<T, EPT, false, true><<<n_blocks, T, 0, s>>>(a, k);
        else
            k_step<T, EPT, false, false><<<n_blocks, T, 0, s>>>(a, k);
    }
    return cudaGetLastError();
}

cudaError_t launch_advance(int64_t *d_step, int64_t by, cudaStream_t s)
{
    k_advance<<<1, 1, 0, s>>>(d_step, by);
    return cudaGetLastError();
}

}  // namespace gn
