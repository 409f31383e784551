// Resident step kernel for small networks: one CTA holds the whole network in
// shared memory -- its by-target edge list, the history ring and the node state --
// and advances it many steps per launch, a CTA barrier between the phases of a
// step.  A small network on the grid kernels spends its step in launch latency
// (a few microseconds per launch); here a step costs its arithmetic.
//
// Step n -> n + 1 (Sec. 2 Eq. Yjset, Sec. 3.1 - 3.3), as in every step kernel:
//   1. S_j(n) = sum_e w_e v~_src(n - D_e): a row of at most kWarpRow edges by one
//      thread in row order, a longer row by a warp (lane l: edges l, l + 32, ...,
//      then the butterfly), each term rounded to FP32 before it is added -- the
//      summation order of every step kernel, so the results are bit-identical;
//   2. barrier; the node update (step_common.cuh, the same code the grid kernels
//      run) of every node, its state read and written in shared memory through a
//      copy of the step arguments whose state pointers point there; barrier.
// FitzHugh-Nagumo keeps the FP32 history ring (the ring is the state); the spiking
// models keep spd(V) as one bit per node and slot, packed by warp ballot, so a
// Hodgkin-Huxley ring of hundreds of slots fits.  Slot n + 1 is written in step n
// and read by no gather of step n (every delay is <= R - 2).  Observations,
// events, first arrivals and every read-only table (caller ids, pulses, cell
// parameters, RAW bias) stay in global memory.  At the end of the launch the ring
// and the state are written back, so any kernel can take the next step.
#include "step_common.cuh"

namespace gn {
namespace {

using namespace step;

template <int kM, int T>
__global__ void __launch_bounds__(T, 1) k_resident(const StepArgs g, const ResidentLayout L, const int n_steps)
{
    extern __shared__ __align__(16) uint8_t sm[];
    __shared__ StepArgs sa;
    __shared__ int s_nlong;
    __shared__ unsigned long long s_evc, s_evbase;
    __shared__ int32_t s_npulses;
    constexpr bool kSpk = (kM & 3) != 0;
    constexpr int W = T / 32;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int N = L.N, R = L.R;
    const int64_t E = L.E;
    uint32_t *key = reinterpret_cast<uint32_t *>(sm + L.off_key);
    float *w = reinterpret_cast<float *>(sm + L.off_w);
    int32_t *rp = reinterpret_cast<int32_t *>(sm + L.off_rp);
    float *S = reinterpret_cast<float *>(sm + L.off_S);  // [2][N]: step n writes half n & 1
    int32_t *lng = reinterpret_cast<int32_t *>(sm + L.off_long);
    float *ring_f = reinterpret_cast<float *>(sm + L.off_ring);      // FitzHugh-Nagumo: [R][stride]
    uint32_t *bits = reinterpret_cast<uint32_t *>(sm + L.off_ring);  // spiking: [R][words]
    float2 *wc = reinterpret_cast<float2 *>(sm + L.off_wc);
    float *iz_v = reinterpret_cast<float *>(sm + L.off_v);
    float2 *rpq = reinterpret_cast<float2 *>(sm + L.off_rpq);
    float4 *hh = reinterpret_cast<float4 *>(sm + L.off_hh);
    int32_t *bgc = reinterpret_cast<int32_t *>(sm + L.off_bgc);
    float *acc = reinterpret_cast<float *>(sm + L.off_acc);
    int32_t *perm = reinterpret_cast<int32_t *>(sm + L.off_perm);
    int64_t *first = reinterpret_cast<int64_t *>(sm + L.off_first);
    int32_t *ev_node = reinterpret_cast<int32_t *>(sm + L.off_evn);
    int64_t *ev_step = reinterpret_cast<int64_t *>(sm + L.off_evs);
    int32_t *p_node = reinterpret_cast<int32_t *>(sm + L.off_pnode);
    int64_t *p_on = reinterpret_cast<int64_t *>(sm + L.off_pon);
    int64_t *p_off = reinterpret_cast<int64_t *>(sm + L.off_poff);
    float *p_amp = reinterpret_cast<float *>(sm + L.off_pamp);
    const int n_pulses = *g.n_pulses;
    const bool local_pulses = n_pulses <= L.pulse_cap;

    if (t == 0) {
        sa = g;
        sa.ring = kSpk ? nullptr : ring_f;
        sa.ring_stride = L.stride;
        sa.wc = wc;
        sa.bgc = bgc;  // background counters always have a place (a background may be set later)
        sa.obs_acc = g.frame_avg ? acc : nullptr;
        sa.first = first;
        // events gather in shared memory and go to the network's buffer in batches
        sa.ev_node = ev_node;
        sa.ev_step = ev_step;
        sa.ev_count = &s_evc;
        sa.ev_cap = L.ev_cap;
        if (local_pulses) {
            sa.n_pulses = &s_npulses;
            sa.p_node = p_node;
            sa.p_on = p_on;
            sa.p_off = p_off;
            sa.p_amp = p_amp;
            s_npulses = n_pulses;
        }
        if constexpr (kSpk) {
            sa.iz_v = iz_v;
            sa.rp = rpq;
            sa.hh_g = (kM & 3) == 2 ? hh : nullptr;
        }
        s_nlong = 0;
        s_evc = 0;
    }
    // everything into shared memory
    const uint32_t *gkey = static_cast<const uint32_t *>(g.ekey);
    for (int64_t e = t; e < E; e += T) {
        key[e] = __ldg(gkey + e);
        w[e] = __ldg(g.ew + e);
    }
    for (int i = t; i <= N; i += T) rp[i] = __ldg(g.row_ptr + i);
    if constexpr (kSpk) {
        for (int i = t; i < R * L.words; i += T) {
            const int slot = i / L.words, wd = i % L.words;
            const float *src = g.ring + static_cast<int64_t>(slot) * g.ring_stride + 32 * wd;
            uint32_t b = 0;
            for (int k = 0; k < 32 && 32 * wd + k < N; ++k) b |= (src[k] != 0.0f ? 1u : 0u) << k;
            bits[i] = b;
        }
    } else {
        for (int i = t; i < R * N; i += T) {
            const int slot = i / N, j = i % N;
            ring_f[slot * L.stride + j] = g.ring[static_cast<int64_t>(slot) * g.ring_stride + j];
        }
    }
    for (int j = t; j < N; j += T) {
        wc[j] = g.wc[j];
        if constexpr (kSpk) {
            iz_v[j] = g.iz_v[j];
            rpq[j] = g.rp[j];
            if constexpr ((kM & 3) == 2) hh[j] = g.hh_g[j];
        }
        bgc[j] = g.bgc[j];
        if (g.frame_avg) acc[j] = g.obs_acc[j];
        perm[j] = __ldg(g.perm + j);
        first[j] = g.first[j];
    }
    if (local_pulses)
        for (int i = t; i < n_pulses; i += T) {
            p_node[i] = g.p_node[i];
            p_on[i] = g.p_on[i];
            p_off[i] = g.p_off[i];
            p_amp[i] = g.p_amp[i];
        }
    __syncthreads();
    for (int r = t; r < N; r += T)
        if (rp[r + 1] - rp[r] > kWarpRow) lng[atomicAdd(&s_nlong, 1)] = r;
    __syncthreads();
    const int n_long = s_nlong;
    const int dbits = g.dbits;
    const uint32_t dmask = (1u << dbits) - 1u;
    const uint32_t rmask = static_cast<uint32_t>(g.ring_mask);
    const int64_t n0 = *g.d_step;
    // each thread's own copy of the step arguments: the node update reads its fields from
    // registers instead of shared memory
    const StepArgs la = sa;
    // the observation bookkeeping as counters: step n samples when (n + 1) % sample_every
    // == 0, its sample number is (n + 1) / sample_every - 1 and its row that modulo obs_cap
    const int se = la.sample_every;
    int ph = static_cast<int>((n0 + 1) % se);
    int64_t kk = (n0 + 1) / se;
    int64_t cidx = kk >= 1 ? (kk - 1) % la.obs_cap : la.obs_cap - 1;

    // the buffered events to the network's event list (every thread; after a barrier)
    auto flush = [&]() {
        if (t == 0) {
            s_evbase = atomicAdd(g.ev_count, s_evc);
        }
        __syncthreads();
        const unsigned long long cnt = s_evc, base = s_evbase;
        for (unsigned long long i = t; i < cnt; i += T)
            if (base + i < static_cast<unsigned long long>(g.ev_cap)) {
                g.ev_node[base + i] = ev_node[i];
                g.ev_step[base + i] = ev_step[i];
            }
        __syncthreads();
        if (t == 0) s_evc = 0;
        __syncthreads();
    };

    for (int s = 0; s < n_steps; ++s) {
        const int64_t n = n0 + s;
        const uint32_t n32 = static_cast<uint32_t>(n);
        StepClock ck;
        ck.sample = ph == 0;
        ck.k = kk - 1;
        ck.row = cidx * N;
        float *Sn = S + (s & 1) * N;
        // the delayed input value of a packed edge key
        auto val = [&](uint32_t k) -> float {
            const uint32_t src = k >> dbits;
            const uint32_t slot = (n32 - (k & dmask)) & rmask;
            if constexpr (kSpk)
                return ((bits[slot * L.words + (src >> 5)] >> (src & 31u)) & 1u) ? 1.0f : 0.0f;
            else
                return ring_f[slot * L.stride + src];
        };
        // 1. input sums (reads ring slots n - D <= n - 1, written a step or more ago)
        for (int r = t; r < N; r += T) {
            const int a0 = rp[r], a1 = rp[r + 1];
            if (a1 - a0 <= kWarpRow) {
                float sum = 0.0f;
                int e = a0;
                for (; e + 8 <= a1; e += 8) {  // loads of 8 terms in flight, added in row order
                    uint32_t k8[8];
                    float w8[8], x8[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        k8[j] = key[e + j];
                        w8[j] = w[e + j];
                    }
#pragma unroll
                    for (int j = 0; j < 8; ++j) x8[j] = val(k8[j]);
#pragma unroll
                    for (int j = 0; j < 8; ++j) sum = __fadd_rn(sum, __fmul_rn(w8[j], x8[j]));
                }
                for (; e < a1; ++e) sum = __fadd_rn(sum, __fmul_rn(w[e], val(key[e])));
                Sn[r] = sum;
            }
        }
        // long rows: four rows per warp at a time, each lane's partial in row order
        for (int i = warp; i < n_long; i += 4 * W) {
            int a0[4], a1[4];
            float p[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int ii = i + q * W;
                const int r = ii < n_long ? lng[ii] : 0;
                a0[q] = ii < n_long ? rp[r] : 0;
                a1[q] = ii < n_long ? rp[r + 1] : 0;
                p[q] = 0.0f;
            }
            const int len = max(max(a1[0] - a0[0], a1[1] - a0[1]), max(a1[2] - a0[2], a1[3] - a0[3]));
            for (int o = lane; o < len; o += 32) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (a0[q] + o < a1[q]) p[q] = __fadd_rn(p[q], __fmul_rn(w[a0[q] + o], val(key[a0[q] + o])));
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const float x = warp_sum(p[q]);
                const int ii = i + q * W;
                if (lane == 0 && ii < n_long) Sn[lng[ii]] = x;
            }
        }
        // barrier; flush the buffered events if this step could overflow the buffer (at
        // most one event per node and step).  Each thread reads the count after its own
        // updates of the previous step; the last of them sees every event of that step
        // (the others wait at this barrier), so the largest reading is the exact count and
        // every thread takes the same decision.
        const unsigned long long seen = *static_cast<volatile unsigned long long *>(&s_evc);
        if (__syncthreads_or(seen > static_cast<unsigned long long>(L.ev_cap - N))) flush();
        // 2. node updates: node r by thread r % T (its own state, its own ring entries);
        // slot n + 1 is read by no gather of step n + 1 (every delay is at least one step)
        for (int base = 0; base < N; base += T) {
            const int r = base + t;
            if constexpr (kSpk) {
                bool spike = false;
                if (r < N) {
                    node_update<kM | kNoRing>(la, r, n, ck, 0.0f, wc[r], Sn[r], perm[r]);
                    const float vpeak = (kM & 3) == 1 ? izh_par(la, r).vpeak : hh_par(la, r).vpeak;
                    spike = iz_v[r] >= vpeak;
                }
                const uint32_t b = __ballot_sync(0xffffffffu, spike);
                if (lane == 0 && base + 32 * warp < N) bits[((n32 + 1u) & rmask) * L.words + (base + 32 * warp) / 32] = b;
            } else {
                if (r < N) node_update<kM>(la, r, n, ck, ring_f[(n32 & rmask) * L.stride + r], wc[r], Sn[r], perm[r]);
            }
        }
        if (++ph == se) {
            ph = 0;
            ++kk;
            cidx = cidx + 1 == la.obs_cap ? 0 : cidx + 1;
        }
    }
    __syncthreads();
    flush();

    // write the ring and the state back
    if constexpr (kSpk) {
        for (int i = t; i < R * N; i += T) {
            const int slot = i / N, j = i % N;
            g.ring[static_cast<int64_t>(slot) * g.ring_stride + j] =
                ((bits[slot * L.words + (j >> 5)] >> (j & 31)) & 1u) ? 1.0f : 0.0f;
        }
    } else {
        for (int i = t; i < R * N; i += T) {
            const int slot = i / N, j = i % N;
            g.ring[static_cast<int64_t>(slot) * g.ring_stride + j] = ring_f[slot * L.stride + j];
        }
    }
    for (int j = t; j < N; j += T) {
        g.wc[j] = wc[j];
        if constexpr (kSpk) {
            g.iz_v[j] = iz_v[j];
            g.rp[j] = rpq[j];
            if constexpr ((kM & 3) == 2) g.hh_g[j] = hh[j];
        }
        g.bgc[j] = bgc[j];
        if (g.frame_avg) g.obs_acc[j] = acc[j];
        g.first[j] = first[j];
    }
}

template <int kM, int T>
cudaError_t launch_res(const StepArgs &a, const ResidentLayout &L, int n_steps, cudaStream_t s)
{
    static_assert(T % 32 == 0, "whole warps");
    k_resident<kM, T><<<1, T, L.bytes, s>>>(a, L, n_steps);
    return cudaGetLastError();
}

template <int kM, int T>
cudaError_t prepare_res(size_t bytes, size_t *max_bytes)
{
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, k_resident<kM, T>);
    if (e != cudaSuccess) return e;
    int dev = 0, optin = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    *max_bytes = static_cast<size_t>(optin) > fa.sharedSizeBytes ? optin - fa.sharedSizeBytes : 0;
    if (bytes > *max_bytes) return cudaSuccess;  // the caller sees it does not fit
    return cudaFuncSetAttribute(k_resident<kM, T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                static_cast<int>(bytes));
}

}  // namespace

const int kResidentThreads[kNumResidentShapes] = {256, 512, 1024};

ResidentLayout resident_layout(int N, int64_t E, int R, int model, bool frame_avg, int ev_factor)
{
    ResidentLayout L{};
    L.N = N;
    L.E = E;
    L.R = R;
    L.words = (N + 31) / 32;
    L.stride = N;
    L.ev_cap = ev_factor * N;
    L.pulse_cap = kResidentPulses;
    const bool spk = model != 0;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t at = off;
        off = (off + bytes + 15) & ~static_cast<size_t>(15);
        return static_cast<uint32_t>(at);
    };
    const size_t n = static_cast<size_t>(N);
    L.off_key = take(4 * static_cast<size_t>(E));
    L.off_w = take(4 * static_cast<size_t>(E));
    L.off_rp = take(4 * (n + 1));
    L.off_S = take(8 * n);
    L.off_long = take(4 * n);
    L.off_ring = take(spk ? 4 * static_cast<size_t>(R) * L.words : 4 * static_cast<size_t>(R) * n);
    L.off_wc = take(8 * n);
    L.off_v = take(spk ? 4 * n : 0);
    L.off_rpq = take(spk ? 8 * n : 0);
    L.off_hh = take(model == 2 ? 16 * n : 0);
    L.off_bgc = take(4 * n);
    L.off_acc = take(frame_avg ? 4 * n : 0);
    L.off_perm = take(4 * n);
    L.off_first = take(8 * n);
    L.off_evn = take(4 * static_cast<size_t>(L.ev_cap));
    L.off_evs = take(8 * static_cast<size_t>(L.ev_cap));
    L.off_pnode = take(4 * static_cast<size_t>(L.pulse_cap));
    L.off_pon = take(8 * static_cast<size_t>(L.pulse_cap));
    L.off_poff = take(8 * static_cast<size_t>(L.pulse_cap));
    L.off_pamp = take(4 * static_cast<size_t>(L.pulse_cap));
    L.bytes = off;
    return L;
}

cudaError_t resident_prepare(int model, int shape, size_t bytes, size_t *max_bytes)
{
    return with_model(model, [&](auto m) {
        constexpr int M = decltype(m)::value;
        switch (shape) {
            case 0: return prepare_res<M, 256>(bytes, max_bytes);
            case 1: return prepare_res<M, 512>(bytes, max_bytes);
            case 2: return prepare_res<M, 1024>(bytes, max_bytes);
            default: return cudaErrorInvalidValue;
        }
    });
}

cudaError_t launch_resident(const StepArgs &a, const ResidentLayout &L, int n_steps, int shape, cudaStream_t s)
{
    if (n_steps <= 0) return cudaSuccess;
    return with_model(a.model, [&](auto m) {
        constexpr int M = decltype(m)::value;
        switch (shape) {
            case 0: return launch_res<M, 256>(a, L, n_steps, s);
            case 1: return launch_res<M, 512>(a, L, n_steps, s);
            case 2: return launch_res<M, 1024>(a, L, n_steps, s);
            default: return cudaErrorInvalidValue;
        }
    });
}

}  // namespace gn
