// The fused step kernel: one launch advances every node of a network by dt.
//
// One CTA owns a row block -- consecutive target nodes (rows of the by-target
// edge list) holding at most T * EPT - 3 edges and T rows, or one longer row on
// its own.  Launches are chained with programmatic dependent launch:
//   0. the CTA lets the next step's grid start as soon as SMs free up
//      (griddepcontrol.launch_dependents);
//   1. it loads everything that does not change between steps -- its block
//      descriptor, row pointers, caller ids and its packed edge records
//      (16-byte loads, a warp reads 512 contiguous bytes) -- while the previous
//      step may still be finishing;
//   2. griddepcontrol.wait: from here on the previous step's writes are visible;
//      it reads the state of its rows (v~(n) from the ring, w~, c~, background
//      counters) and gathers, for every edge,
//        S_j(n) = sum_e w_e v~_src(n - D_e)      (Eq. Yjset, Sec. 2)
//      from ring slot (n - D_e) & (R - 1), parking w_e * v~ in shared memory;
//   3. row sums: short rows by their own thread, long rows by a warp (shuffle);
//   4. per node: stimulus, the FHN Euler update about the rest point (Sec. 3.1,
//      Eq. fnstate), the history write, the low-pass readout and, on sample
//      steps, the noisy observation (Sec. 3.3), events and first arrivals.
// Every read of step data is of step n (or older) and every write is of step n+1;
// slot (n + 1) & (R - 1) is never read in step n because every delay is <= R - 2.
#include "step_common.cuh"

namespace gn {
namespace {

using namespace step;

__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <int kM, int T, int EPT, int MINB, bool kPacked, bool kStream>
__global__ void __launch_bounds__(T, MINB) k_step(const StepArgs a, const int k)
{
    constexpr int CAP = T * EPT;
    constexpr int NQ = EPT / 4;  // edge quads per thread
    __shared__ float s_prod[CAP];
    __shared__ float s_long[T];
    __shared__ int s_rp[T + 1];

    pdl_launch_dependents();
    const int t = threadIdx.x;
    const int4 d = __ldg(a.bdesc + blockIdx.x);
    const int r0 = d.x, r1 = d.y, e0 = d.z, e1 = d.w;
    const int nr = r1 - r0;
    const int r = r0 + t;

    // 1. step-invariant inputs
    int32_t orig = kLoad;
    if (t < nr) {
        s_rp[t] = __ldg(a.row_ptr + r);
        orig = __ldg(a.perm + r);
    }
    if (t == 0) s_rp[nr] = e1;
    const bool lng = (nr == 1) && (e1 - e0 > CAP - 3);
    const int ebase = e0 & ~3;
    RawQuad<kPacked> q[NQ];
    float4 wv[NQ];
    if (!lng) {
#pragma unroll
        for (int i = 0; i < NQ; ++i) {
            const int eb = ebase + 4 * (t + T * i);
            if (eb < e1) {
                q[i] = load_raw<kPacked, kStream>(a, eb);
                wv[i] = ld_weight4<kStream>(a.ew + eb);
            }
        }
    }

    // 2. step data of the previous launch
    pdl_wait();
    const int64_t n = *a.d_step + k;
    float v = 0.0f;
    float2 wc = make_float2(0.0f, 0.0f);
    int32_t cnt0 = kLoad;
    if (t < nr) {
        if constexpr (kM == 0) v = a.ring[(n & a.ring_mask) * a.ring_stride + r];  // spiking models keep V apart
        wc = a.wc[r];
        if (a.bg_thr) cnt0 = a.bgc[r];
    }

    if (lng) {
        // one long row: the whole CTA loops over chunks of its edges
        float p = 0.0f;
        for (int base = ebase; base < e1; base += CAP) {
#pragma unroll
            for (int i = 0; i < NQ; ++i) {
                const int eb = base + 4 * (t + T * i);
                const EdgeQuad<kPacked> qq = load_quad<kPacked, kStream>(a, eb);
                const float4 ww = ld_weight4<kStream>(a.ew + eb);
                const float wq[4] = {ww.x, ww.y, ww.z, ww.w};
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (eb + j >= e0 && eb + j < e1) p = fmaf(wq[j], gather(a, n, qq.src[j], qq.d[j]), p);
            }
        }
        p = warp_sum(p);
        if ((t & 31) == 0) s_long[t >> 5] = p;
        __syncthreads();
        if (t == 0) {
            float S = 0.0f;
            for (int i = 0; i < T / 32; ++i) S += s_long[i];
            node_update<kM>(a, r0, n, v, wc, S, orig, cnt0);
        }
        return;
    }

    // gathers: every edge of the block, products parked in shared memory
#pragma unroll
    for (int i = 0; i < NQ; ++i) {
        const int eb = ebase + 4 * (t + T * i);
        if (eb >= e1) break;
        const float wq[4] = {wv[i].x, wv[i].y, wv[i].z, wv[i].w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int e = eb + j;
            if (e >= e0 && e < e1) {
                uint32_t src, dd;
                decode<kPacked>(a, q[i], j, src, dd);
                s_prod[e - e0] = wq[j] * gather(a, n, src, dd);
            }
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
    if (t < nr) node_update<kM>(a, r, n, v, wc, S, orig, cnt0);
}

__global__ void k_advance(int64_t *d_step, int64_t by)
{
    *d_step += by;
}

template <int kM, int T, int EPT, int MINB, bool kPacked, bool kStream>
cudaError_t launch_pdl(const StepArgs &a, int n_blocks, int k, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(n_blocks));
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step<kM, T, EPT, MINB, kPacked, kStream>, a, k);
}

template <int kM, int T, int EPT, int MINB>
cudaError_t launch_shape(const StepArgs &a, int n_blocks, int k, bool packed, bool stream_edges, cudaStream_t s)
{
    if (packed)
        return stream_edges ? launch_pdl<kM, T, EPT, MINB, true, true>(a, n_blocks, k, s)
                            : launch_pdl<kM, T, EPT, MINB, true, false>(a, n_blocks, k, s);
    return stream_edges ? launch_pdl<kM, T, EPT, MINB, false, true>(a, n_blocks, k, s)
                        : launch_pdl<kM, T, EPT, MINB, false, false>(a, n_blocks, k, s);
}

}  // namespace

// {threads, edges per thread, CTAs per SM the register allocation must allow}
const StepShape kStepShapes[kNumStepShapes] = {{256, 8, 1}, {256, 8, 8}, {128, 16, 1}, {128, 8, 16}, {512, 8, 1}};

cudaError_t launch_step(const StepArgs &a, int n_blocks, int k, int shape, bool packed, bool stream_edges,
                        cudaStream_t s)
{
    if (n_blocks <= 0) return cudaSuccess;
    return with_model(a.model, [&](auto m) {
        constexpr int M = decltype(m)::value;
        switch (shape) {
            case 0: return launch_shape<M, 256, 8, 1>(a, n_blocks, k, packed, stream_edges, s);
            case 1: return launch_shape<M, 256, 8, 8>(a, n_blocks, k, packed, stream_edges, s);
            case 2: return launch_shape<M, 128, 16, 1>(a, n_blocks, k, packed, stream_edges, s);
            case 3: return launch_shape<M, 128, 8, 16>(a, n_blocks, k, packed, stream_edges, s);
            case 4: return launch_shape<M, 512, 8, 1>(a, n_blocks, k, packed, stream_edges, s);
            default: return cudaErrorInvalidValue;
        }
    });
}

cudaError_t launch_advance(int64_t *d_step, int64_t by, cudaStream_t s)
{
    k_advance<<<1, 1, 0, s>>>(d_step, by);
    return cudaGetLastError();
}

}  // namespace gn
