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
#include "internal.cuh"
#include "philox.cuh"

namespace gn {
namespace {

template <bool kStream>
__device__ __forceinline__ uint4 ld_edge4(const void *p)
{
    if constexpr (kStream)
        return __ldcs(reinterpret_cast<const uint4 *>(p));
    else
        return __ldg(reinterpret_cast<const uint4 *>(p));
}

template <bool kStream>
__device__ __forceinline__ float4 ld_weight4(const float *p)
{
    if constexpr (kStream)
        return __ldcs(reinterpret_cast<const float4 *>(p));
    else
        return __ldg(reinterpret_cast<const float4 *>(p));
}

__device__ __forceinline__ float warp_sum(float x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
}

// Edge e's source and delay from its packed or wide key.
template <bool kPacked>
struct EdgeQuad {
    uint32_t src[4], d[4];
};

template <bool kPacked, bool kStream>
__device__ __forceinline__ EdgeQuad<kPacked> load_quad(const StepArgs &a, int64_t eb)
{
    EdgeQuad<kPacked> q;
    if constexpr (kPacked) {
        const uint4 k = ld_edge4<kStream>(static_cast<const uint32_t *>(a.ekey) + eb);
        const uint32_t m = (1u << a.dbits) - 1u;
        const uint32_t kk[4] = {k.x, k.y, k.z, k.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            q.src[i] = kk[i] >> a.dbits;
            q.d[i] = kk[i] & m;
        }
    } else {
        const uint2 *base = static_cast<const uint2 *>(a.ekey) + eb;
        const uint4 k0 = ld_edge4<kStream>(base);
        const uint4 k1 = ld_edge4<kStream>(base + 2);
        q.src[0] = k0.x; q.d[0] = k0.y; q.src[1] = k0.z; q.d[1] = k0.w;
        q.src[2] = k1.x; q.d[2] = k1.y; q.src[3] = k1.z; q.d[3] = k1.w;
    }
    return q;
}

__device__ __forceinline__ float gather(const StepArgs &a, int64_t n, uint32_t src, uint32_t d)
{
    const int64_t slot = (n - static_cast<int64_t>(d)) & a.ring_mask;
    return __ldg(a.ring + slot * a.N + src);
}

// Stimulus, FHN Euler step, history write, readout, noise, events, arrival.
__device__ __forceinline__ void node_update(const StepArgs &a, int r, int64_t n, float v, float2 wc, float S)
{
    float U = 0.0f;
    const int n_pulses = *a.n_pulses;
    if (n_pulses > 0) {
        int lo = 0, hi = n_pulses;  // first pulse with p_node >= r
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (a.p_node[mid] < r) lo = mid + 1; else hi = mid;
        }
        for (int p = lo; p < n_pulses && a.p_node[p] == r; ++p)
            if (a.p_on[p] <= n && n < a.p_off[p]) U += a.p_amp[p];
    }
    int32_t orig = -1;
    if (a.bg_thr) {
        orig = __ldg(a.perm + r);
        const int32_t c0 = a.bgc[r];
        int32_t cnt = c0;
        if (draw(a.bg_seed, static_cast<uint32_t>(orig), n, kStreamBackground).x < a.bg_thr) cnt = a.bg_width;
        if (cnt > 0) {
            U += a.bg_amp;
            cnt -= 1;
        }
        if (cnt != c0) a.bgc[r] = cnt;
    }
    if (a.bias) S += __ldg(a.bias + r);

    const float w = wc.x, c = wc.y;
    const float dv = fmaf(v, fmaf(v, fmaf(a.q3, v, a.q2), a.k1), -a.cw * w) + S + U;
    const float v1 = fmaf(a.dt, dv, v);
    const float w1 = fmaf(a.dte, fmaf(-a.g, w, v), w);
    const float c1 = fmaf(a.alpha, v1 - c, c);

    a.ring[((n + 1) & a.ring_mask) * a.N + r] = v1;
    a.wc[r] = make_float2(w1, c1);

    if (v < a.theta_s && v1 >= a.theta_s) {
        const unsigned long long i = atomicAdd(a.ev_count, 1ull);
        if (i < static_cast<unsigned long long>(a.ev_cap)) {
            a.ev_node[i] = r;
            a.ev_step[i] = n + 1;
        }
    }
    if (v1 != 0.0f && v == 0.0f && a.first[r] < 0) a.first[r] = n + 1;

    if (((n + 1) % a.sample_every) == 0) {
        const int64_t k = (n + 1) / a.sample_every - 1;
        if (orig < 0) orig = __ldg(a.perm + r);
        const float xi = gauss_from(draw(a.obs_seed, static_cast<uint32_t>(orig), k, kStreamObservation));
        const float y = fmaf(a.gain, a.vrest + c1, a.offset) + a.sigma * xi;
        a.obs[(k % a.obs_cap) * a.N + orig] = y;  // rows are written in the caller's node order
    }
}

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
        v = a.ring[(n & a.ring_mask) * a.N + r];
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
