// Batched form: thousands of independent networks of uneven size advanced by
// one persistent launch.
//
// Each CTA pops network ids from an atomic work queue whose order is largest
// first (longest-processing-time order, so the big networks start early and the
// small ones fill the tail), copies that network's step arguments into shared
// memory and runs all of its n steps: per step it walks the network's row blocks
// -- gather the delayed values of a block's edges (Eq. Yjset), park w * v~ in
// shared memory, sum the rows, apply the fused node update (Sec. 3.1 FHN
// transition, Sec. 3.3 readout) -- and a CTA barrier separates the steps.  The
// networks are independent, so no grid-wide synchronisation is needed.
//
// The history ring is written and read inside the same launch, so every read of
// step data is a coherent load (never the read-only path); the barrier between
// steps makes the CTA's writes of step n visible to its reads of step n + 1.
#include <mutex>

#include "step_common.cuh"

namespace gn {
namespace {

using namespace step;

// Coherent (L1-allocating, non read-only) loads for data written in this launch.
__device__ __forceinline__ float gather_coherent(const StepArgs &a, int64_t n, uint32_t src, uint32_t d)
{
    const int64_t slot = (n - static_cast<int64_t>(d)) & a.ring_mask;
    return a.ring[slot * a.ring_stride + src];
}

template <int T, int EPT, bool kPacked>
__device__ __forceinline__ void batch_block(const StepArgs &a, int64_t n, int b, float *s_prod, float *s_long,
                                            int *s_rp)
{
    constexpr int CAP = T * EPT;
    constexpr int NQ = EPT / 4;
    const int t = threadIdx.x;
    const int4 d = __ldg(a.bdesc + b);
    const int r0 = d.x, r1 = d.y, e0 = d.z, e1 = d.w;
    const int nr = r1 - r0;
    const int r = r0 + t;
    float v = 0.0f;
    float2 wc = make_float2(0.0f, 0.0f);
    if (t < nr) {
        s_rp[t] = __ldg(a.row_ptr + r);
        v = a.ring[(n & a.ring_mask) * a.ring_stride + r];
        wc = a.wc[r];
    }
    if (t == 0) s_rp[nr] = e1;
    const bool lng = (nr == 1) && (e1 - e0 > CAP - 3);
    const int ebase = e0 & ~3;
    if (lng) {
        float p = 0.0f;
        for (int base = ebase; base < e1; base += CAP) {
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                const int eb = base + 4 * (t + T * i);
                const EdgeQuad<kPacked> qq = load_quad<kPacked, false>(a, eb);
                const float4 ww = ld_weight4<false>(a.ew + eb);
                const float wq[4] = {ww.x, ww.y, ww.z, ww.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (eb + j >= e0 && eb + j < e1) p = fmaf(wq[j], gather_coherent(a, n, qq.src[j], qq.d[j]), p);
            }
        }
        p = warp_sum(p);
        if ((t & 31) == 0) s_long[t >> 5] = p;
        __syncthreads();
        if (t == 0) {
            float S = 0.0f;
            for (int i = 0; i < T / 32; ++i) S += s_long[i];
            node_update<0>(a, r0, n, v, wc, S);
        }
        __syncthreads();
        return;
    }
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        const int eb = ebase + 4 * (t + T * i);
        if (eb >= e1) break;
        const RawQuad<kPacked> q = load_raw<kPacked, false>(a, eb);
        const float4 wv = ld_weight4<false>(a.ew + eb);
        const float wq[4] = {wv.x, wv.y, wv.z, wv.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = eb + j;
            if (e >= e0 && e < e1) {
                uint32_t src, dd;
                decode<kPacked>(a, q, j, src, dd);
                s_prod[e - e0] = wq[j] * gather_coherent(a, n, src, dd);
            }
        }
    }
    __syncthreads();
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
    if (t < nr) node_update<0>(a, r, n, v, wc, S);
    __syncthreads();  // s_prod, s_rp and s_long are reused by the next block
}

template <int T, int EPT>
__global__ void __launch_bounds__(T) k_batch(const StepArgs *__restrict__ nets, const int *__restrict__ order,
                                             int n_nets, int *queue, const int64_t *d_step, int n_steps)
{
    constexpr int CAP = T * EPT;
    __shared__ StepArgs sa;
    __shared__ float s_prod[CAP];
    __shared__ float s_long[T];
    __shared__ int s_rp[T + 1];
    __shared__ int s_q;
    const int t = threadIdx.x;
    const int64_t n0 = *d_step;
    for (;;) {
        if (t == 0) s_q = atomicAdd(queue, 1);
        __syncthreads();
        const int qi = s_q;
        if (qi >= n_nets) break;
        {
            const int id = __ldg(order + qi);
            const int *src = reinterpret_cast<const int *>(nets + id);
            int *dst = reinterpret_cast<int *>(&sa);
            for (int i = t; i < static_cast<int>(sizeof(StepArgs) / 4); i += T) dst[i] = __ldg(src + i);
        }
        __syncthreads();
        const bool packed = sa.packed != 0;
        for (int64_t n = n0; n < n0 + n_steps; ++n) {
            if (packed) {
                for (int b = 0; b < sa.n_blocks; ++b) batch_block<T, EPT, true>(sa, n, b, s_prod, s_long, s_rp);
            } else {
                for (int b = 0; b < sa.n_blocks; ++b) batch_block<T, EPT, false>(sa, n, b, s_prod, s_long, s_rp);
            }
        }
        __syncthreads();  // sa and s_q are rewritten for the next network
    }
}

}  // namespace

const int kBatchThreads[kNumBatchShapes] = {128, 256, 512};

int batch_block_cap(int shape) { return kBatchThreads[shape] * 8; }

cudaError_t launch_batch(const StepArgs *nets, const int *order, int n_nets, int *queue, const int64_t *d_step,
                         int n_steps, int shape, int grid, cudaStream_t s)
{
    if (n_nets <= 0 || n_steps <= 0) return cudaSuccess;
    switch (shape) {
        case 0: k_batch<128, 8><<<grid, 128, 0, s>>>(nets, order, n_nets, queue, d_step, n_steps); break;
        case 1: k_batch<256, 8><<<grid, 256, 0, s>>>(nets, order, n_nets, queue, d_step, n_steps); break;
        case 2: k_batch<512, 8><<<grid, 512, 0, s>>>(nets, order, n_nets, queue, d_step, n_steps); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t batch_occupancy(int shape, int *ctas_per_sm)
{
    switch (shape) {
        case 0: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_batch<128, 8>, 128, 0);
        case 1: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_batch<256, 8>, 256, 0);
        case 2: return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, k_batch<512, 8>, 512, 0);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace gn

// ---------------------------------------------------------------------------
// Allocation-free stepping of a batch (gn_batch_step_static).
//
// The work queue of one launch -- the counter CTAs take networks from and the
// largest-first schedule -- lives in this file-scope device array instead of in
// memory the batch allocated.  It holds at most kStaticQueueNets networks; all
// calls share it, and it keeps the last call's contents (the counter is cleared
// and the schedule rewritten before every launch).  Two calls that overlap on the
// GPU (on different streams, or on different batches at once) race on it.
namespace gn {
namespace {

struct StaticQueue {
    int counter;
    int pad[63];  // keep the schedule 256-byte aligned
    int order[kStaticQueueNets];
};

static __device__ __align__(256) StaticQueue g_static_queue;

constexpr int kMaxDevices = 64;
// the array's device address on each device, looked up once per device (under the
// lock, so host threads making their first calls at once do not race on the cache)
StaticQueue *g_queue_addr[kMaxDevices] = {};
std::mutex g_queue_lock;

cudaError_t static_queue_address(int device, StaticQueue **out)
{
    std::lock_guard<std::mutex> lock(g_queue_lock);
    if (!g_queue_addr[device]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_queue);  // the caller made `device` current
        if (e != cudaSuccess) return e;
        g_queue_addr[device] = static_cast<StaticQueue *>(p);
    }
    *out = g_queue_addr[device];
    return cudaSuccess;
}
}  // namespace

cudaError_t launch_batch_static(const StepArgs *nets, const int *d_order, int n_nets, const int64_t *d_step,
                                int n_steps, int shape, int grid, int device, cudaStream_t s)
{
    if (n_nets <= 0 || n_steps <= 0) return cudaSuccess;
    if (n_nets > kStaticQueueNets || device < 0 || device >= kMaxDevices) return cudaErrorInvalidValue;
    StaticQueue *q = nullptr;
    cudaError_t e = static_queue_address(device, &q);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(&q->counter, 0, sizeof(int), s);
    if (e != cudaSuccess) return e;
    // the schedule comes from the batch's device copy: a device-to-device copy in
    // stream order, with no host buffer to wait on
    e = cudaMemcpyAsync(q->order, d_order, static_cast<size_t>(n_nets) * sizeof(int), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    switch (shape) {
        case 0: k_batch<128, 8><<<grid, 128, 0, s>>>(nets, q->order, n_nets, &q->counter, d_step, n_steps); break;
        case 1: k_batch<256, 8><<<grid, 256, 0, s>>>(nets, q->order, n_nets, &q->counter, d_step, n_steps); break;
        case 2: k_batch<512, 8><<<grid, 512, 0, s>>>(nets, q->order, n_nets, &q->counter, d_step, n_steps); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gn
