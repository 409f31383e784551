// Device functions shared by the step kernels (k_step.cu, k_step_pipe.cu):
// edge-record decoding, the delayed gather and the fused per-node update.
#pragma once
#include "internal.cuh"
#include "philox.cuh"
#include "ptx.cuh"

#include <climits>

namespace gn {
namespace step {

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

// Raw edge records of four consecutive edges, held in registers until they are
// decoded: one 16-byte word (packed keys) or two (wide keys).
template <bool kPacked>
struct RawQuad {
    uint4 k0;
};
template <>
struct RawQuad<false> {
    uint4 k0, k1;
};

template <bool kPacked, bool kStream>
__device__ __forceinline__ RawQuad<kPacked> load_raw(const StepArgs &a, int64_t eb)
{
    RawQuad<kPacked> r;
    if constexpr (kPacked) {
        r.k0 = ld_edge4<kStream>(static_cast<const uint32_t *>(a.ekey) + eb);
    } else {
        const uint2 *base = static_cast<const uint2 *>(a.ekey) + eb;
        r.k0 = ld_edge4<kStream>(base);
        r.k1 = ld_edge4<kStream>(base + 2);
    }
    return r;
}

template <bool kPacked>
__device__ __forceinline__ void decode(const StepArgs &a, const RawQuad<kPacked> &r, int j, uint32_t &src,
                                       uint32_t &d)
{
    if constexpr (kPacked) {
        const uint32_t k = j == 0 ? r.k0.x : j == 1 ? r.k0.y : j == 2 ? r.k0.z : r.k0.w;
        src = k >> a.dbits;
        d = k & ((1u << a.dbits) - 1u);
    } else {
        const uint4 &h = j < 2 ? r.k0 : r.k1;
        src = (j & 1) ? h.z : h.x;
        d = (j & 1) ? h.w : h.y;
    }
}

__device__ __forceinline__ float gather(const StepArgs &a, int64_t n, uint32_t src, uint32_t d)
{
    const int64_t slot = (n - static_cast<int64_t>(d)) & a.ring_mask;
    return __ldg(a.ring + slot * a.ring_stride + src);
}

// The same with an L2 priority hint (keeps the live history slots resident
// while the edge stream passes through L2).
__device__ __forceinline__ float gather_hint(const StepArgs &a, int64_t n, uint32_t src, uint32_t d, uint64_t pol)
{
    const int64_t slot = (n - static_cast<int64_t>(d)) & a.ring_mask;
    return ldg_hint(a.ring + slot * a.ring_stride + src, pol);
}

constexpr int32_t kLoad = INT32_MIN;  // "not prefetched" marker for node_update

__device__ __forceinline__ void record_event(const StepArgs &a, int r, int64_t step)
{
    const unsigned long long i = atomicAdd(a.ev_count, 1ull);
    if (i < static_cast<unsigned long long>(a.ev_cap)) {
        a.ev_node[i] = r;
        a.ev_step[i] = step;
    }
}

// The observation bookkeeping of step n -> n + 1: whether it takes a sample (every
// sample_every steps), the sample's number k and the offset of its row in the
// observation ring.  Kernels compute it per node (step_clock); the resident kernel
// keeps it as counters across its steps.
struct StepClock {
    bool sample;
    int64_t k;    // sample number (when sample)
    int64_t row;  // (k % obs_cap) * N (when sample)
};

__device__ __forceinline__ StepClock step_clock(const StepArgs &a, int64_t n)
{
    StepClock c{};
    c.sample = ((n + 1) % a.sample_every) == 0;
    if (c.sample) {
        c.k = (n + 1) / a.sample_every - 1;
        c.row = (c.k % a.obs_cap) * a.N;
    }
    return c;
}

// The readout state a sample reads: c1, or with camera frame averaging the mean of
// c over the sample_every steps of the frame (summed in step order, then divided).
__device__ __forceinline__ float frame_value(const StepArgs &a, int r, float c1, bool sample)
{
    if (!a.frame_avg) return c1;
    const float acc = __fadd_rn(a.obs_acc[r], c1);
    a.obs_acc[r] = sample ? 0.0f : acc;
    return sample ? __fdiv_rn(acc, static_cast<float>(a.sample_every)) : c1;
}

// Spiking-node outputs of step n -> n + 1: spike ring (spd(V1)), events, first
// spike, and the calcium readout every sample_every steps.  A plastic net's ring
// word also carries s in whole steps: s_j' = (1 - spd(V_j)) (s_j + dt), from the
// word of step n.
// (kRing false: the caller keeps its own spike ring and writes it; the resident
// kernel packs spd into bits by warp ballot)
template <bool kPl, bool kRing = true>
__device__ __forceinline__ void spiking_outputs(const StepArgs &a, int r, int64_t n, const StepClock &ck, bool above,
                                                bool above1, float c1, int32_t orig, uint32_t word_now)
{
    const int64_t at = ((n + 1) & a.ring_mask) * a.ring_stride + r;
    if constexpr (!kRing) {
    } else if constexpr (kPl) {
        const uint32_t k1 = (word_now & 1u) ? 0u : min((word_now >> 1) + 1u, kSpikeStepsMax);
        reinterpret_cast<uint32_t *>(a.ring)[at] = (k1 << 1) | (above1 ? 1u : 0u);
    } else {
        a.ring[at] = above1 ? 1.0f : 0.0f;
    }
    if (above1 && !above) {
        record_event(a, r, n + 1);
        if (a.first[r] < 0) a.first[r] = n + 1;
    }
    const float cs = frame_value(a, r, c1, ck.sample);
    if (ck.sample) {
        if (orig == kLoad) orig = __ldg(a.perm + r);
        const float xi = gauss_from(draw(a.obs_seed, static_cast<uint32_t>(orig), ck.k, kStreamObservation));
        a.obs[ck.row + orig] = __fmaf_rn(a.sigma, xi, __fmaf_rn(a.gain, cs, a.offset));
    }
}

// Parameters of a spiking node: the network's scalars, or its cell type's row.
struct IzhPar {
    float dtc, k, vr, vt, vpeak, vreset, dta, b, d, iext, a2, two_a, caq;
};
struct HhPar {
    float dtc, gna, gk, gl, ena, ek, el, vpeak, iext, a2, two_a, caq;
};

__device__ __forceinline__ IzhPar izh_par(const StepArgs &a, int r)
{
    if (a.cell_type) {
        const float *q = a.type_par + kTypeStride * __ldg(a.cell_type + r);
        return {__ldg(q),     __ldg(q + 1), __ldg(q + 2),           __ldg(q + 3),           __ldg(q + 4),
                __ldg(q + 5), __ldg(q + 6), __ldg(q + 7),           __ldg(q + 8),           __ldg(q + 9),
                __ldg(q + kTypeA2), __ldg(q + kTypeA2 + 1), __ldg(q + kTypeA2 + 2)};
    }
    return {a.iz_dtc, a.iz_k, a.iz_vr, a.iz_vt, a.iz_vpeak, a.iz_vreset, a.iz_dta, a.iz_b, a.iz_d, a.iz_iext,
            a.ps_a2, a.ps_2a, a.ca_q};
}

__device__ __forceinline__ HhPar hh_par(const StepArgs &a, int r)
{
    if (a.cell_type) {
        const float *q = a.type_par + kTypeStride * __ldg(a.cell_type + r);
        return {__ldg(q),     __ldg(q + 1), __ldg(q + 2),       __ldg(q + 3),           __ldg(q + 4),
                __ldg(q + 5), __ldg(q + 6), __ldg(q + 7),       __ldg(q + 8),           __ldg(q + kTypeA2),
                __ldg(q + kTypeA2 + 1), __ldg(q + kTypeA2 + 2)};
    }
    return {a.iz_dtc, a.hh_gna, a.hh_gk, a.hh_gl, a.hh_ena, a.hh_ek, a.hh_el, a.iz_vpeak, a.iz_iext,
            a.ps_a2, a.ps_2a, a.ca_q};
}

// c' = c + dt (-c / tau_c + spd), every operation rounded as written (the spiking
// updates spell out their FP32 operations, so that every kernel that inlines them
// rounds the same way whatever the compiler would contract)
__device__ __forceinline__ float calcium_step(const StepArgs &a, float c, float caq, bool spd)
{
    const float q = __fmul_rn(c, caq);
    return __fmaf_rn(a.dt, spd ? __fsub_rn(1.0f, q) : -q, c);
}

// Izhikevich simple model with an alpha-function PSC and the calcium readout
// (Sec. 3.1 Eq. izsimple / izpsc, Sec. 3.2.1 Eq. alphapsc and spd, Sec. 3.3 Eq.
// casimple), forward Euler from step n to n + 1; the state is absolute.  Everything
// but p, the one variable that reads S = sum_e w_e spd(V_src(n - D_e)), is updated
// here (the ring holds spd); returns (r, p) at step n for psc_finish.  A spike
// resets V, so every step with V >= V_peak is a new spike.
template <bool kPl, bool kRing = true>
__device__ __forceinline__ float2 izh_begin(const StepArgs &a, int r, int64_t n, const StepClock &ck, float2 wc, float U,
                                         int32_t orig, uint32_t word_now)
{
    const IzhPar z = izh_par(a, r);
    const float V = a.iz_v[r];
    const float W = wc.x, c = wc.y;
    const float2 rp = a.rp[r];
    const bool spike = V >= z.vpeak;
    float V1, W1;
    if (!spike) {
        const float dv = __fsub_rn(V, z.vr);
        const float quad = __fmul_rn(__fmul_rn(z.k, dv), __fsub_rn(V, z.vt));
        V1 = __fmaf_rn(z.dtc, __fadd_rn(__fadd_rn(__fadd_rn(__fsub_rn(quad, W), rp.x), U), z.iext), V);
        W1 = __fmaf_rn(z.dta, __fsub_rn(__fmul_rn(z.b, dv), W), W);
    } else {
        V1 = z.vreset;
        W1 = __fadd_rn(W, z.d);
    }
    const float c1 = calcium_step(a, c, z.caq, spike);
    a.iz_v[r] = V1;
    a.wc[r] = make_float2(W1, c1);
    spiking_outputs<kPl, kRing>(a, r, n, ck, false, V1 >= z.vpeak, c1, orig, word_now);
    return rp;
}

// x / (1 - e^(-x / y)) with its limit y at x = 0 (the removable 0/0 of alpha_m, alpha_n)
__device__ __forceinline__ float hh_trap(float x, float y)
{
    return x == 0.0f ? y : __fdiv_rn(x, -expm1f(__fdiv_rn(-x, y)));
}

// Hodgkin-Huxley + alpha-PSC + calcium node (model 2): classic squid-axon rates
// (mV, ms), forward Euler of V and the gates m, n, h from step-n values, the PSC and
// calcium as in izh_begin (p is left to psc_finish); no reset, events are upward
// crossings of V_peak.
template <bool kPl, bool kRing = true>
__device__ __forceinline__ float2 hh_begin(const StepArgs &a, int r, int64_t n, const StepClock &ck, float2 wc, float U,
                                        int32_t orig, uint32_t word_now)
{
    const HhPar z = hh_par(a, r);
    const float V = a.iz_v[r];
    const float4 g = a.hh_g[r];
    const float2 rp = a.rp[r];
    const float c = wc.y;
    const float e65 = __fadd_rn(V, 65.0f);
    const float am = __fmul_rn(0.1f, hh_trap(__fadd_rn(V, 40.0f), 10.0f));
    const float bm = __fmul_rn(4.0f, expf(__fdiv_rn(-e65, 18.0f)));
    const float ah = __fmul_rn(0.07f, expf(__fdiv_rn(-e65, 20.0f)));
    const float bh = __fdiv_rn(1.0f, __fadd_rn(1.0f, expf(__fdiv_rn(-__fadd_rn(V, 35.0f), 10.0f))));
    const float an = __fmul_rn(0.01f, hh_trap(__fadd_rn(V, 55.0f), 10.0f));
    const float bn = __fmul_rn(0.125f, expf(__fdiv_rn(-e65, 80.0f)));
    const float m3h = __fmul_rn(__fmul_rn(__fmul_rn(g.x, g.x), g.x), g.z);
    const float n2 = __fmul_rn(g.y, g.y);
    const float i_na = __fmul_rn(__fmul_rn(z.gna, m3h), __fsub_rn(V, z.ena));
    const float i_k = __fmul_rn(__fmul_rn(z.gk, __fmul_rn(n2, n2)), __fsub_rn(V, z.ek));
    const float i_l = __fmul_rn(z.gl, __fsub_rn(V, z.el));
    const float i_ion = __fadd_rn(__fadd_rn(i_na, i_k), i_l);
    const float V1 = __fmaf_rn(z.dtc, __fadd_rn(__fadd_rn(__fsub_rn(rp.x, i_ion), U), z.iext), V);
    // x' = x + dt (alpha (1 - x) - beta x)
    auto gate = [&](float x, float al, float be) {
        return __fmaf_rn(a.dt, __fsub_rn(__fmul_rn(al, __fsub_rn(1.0f, x)), __fmul_rn(be, x)), x);
    };
    const float m1 = gate(g.x, am, bm), n1 = gate(g.y, an, bn), h1 = gate(g.z, ah, bh);
    const bool above = V >= z.vpeak;
    const float c1 = calcium_step(a, c, z.caq, above);
    a.iz_v[r] = V1;
    a.hh_g[r] = make_float4(m1, n1, h1, 0.0f);
    a.wc[r] = make_float2(0.0f, c1);
    spiking_outputs<kPl, kRing>(a, r, n, ck, above, V1 >= z.vpeak, c1, orig, word_now);
    return rp;
}

// The alpha-function PSC of either spiking model from its step-n values (r, p):
// r' = r + dt p, p' = p + dt (-a^2 r - 2 a p + S).
// (the node's PSC constants are looked up again here rather than kept live across
// the gathers and piece sums between the two halves of the update)
__device__ __forceinline__ void psc_finish(const StepArgs &a, int r, float2 rp, float S)
{
    float a2 = a.ps_a2, two_a = a.ps_2a;
    if (a.cell_type) {
        const float *q = a.type_par + kTypeStride * __ldg(a.cell_type + r);
        a2 = __ldg(q + kTypeA2);
        two_a = __ldg(q + kTypeA2 + 1);
    }
    const float r1 = __fmaf_rn(a.dt, rp.y, rp.x);
    const float p1 = __fmaf_rn(a.dt, __fadd_rn(__fsub_rn(__fmul_rn(-a2, rp.x), __fmul_rn(two_a, rp.y)), S), rp.y);
    a.rp[r] = make_float2(r1, p1);
}

// Control input U_j(n): explicit pulses and background pulses.  `orig` (caller id)
// and `cnt0` (background counter) may be prefetched by the caller; kLoad makes it
// read them (orig is returned loaded if it was needed).
__device__ __forceinline__ float stimulus(const StepArgs &a, int r, int64_t n, int32_t &orig, int32_t cnt0)
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
    if (a.bg_thr) {
        if (orig == kLoad) orig = __ldg(a.perm + r);
        const int32_t c0 = cnt0 == kLoad ? a.bgc[r] : cnt0;
        int32_t cnt = c0;
        if (draw(a.bg_seed, static_cast<uint32_t>(orig), n, kStreamBackground).x < a.bg_thr) cnt = a.bg_width;
        if (cnt > 0) {
            U += a.bg_amp;
            cnt -= 1;
        }
        if (cnt != c0) a.bgc[r] = cnt;
    }
    return U;
}

// The S-independent part of a spiking node's step (model kM & 3 = 1 or 2, kM &
// kPlastic with plastic weights, where word_now is the node's ring word of step n;
// kM & kNoRing: the spike ring is left to the caller): stimulus and everything but
// p; returns (r, p) at step n for psc_finish.
template <int kM>
__device__ __forceinline__ float2 spiking_begin(const StepArgs &a, int r, int64_t n, const StepClock &ck, float2 wc,
                                                int32_t orig, int32_t cnt0, uint32_t word_now = 0)
{
    constexpr bool kPl = (kM & kPlastic) != 0;
    constexpr bool kRing = (kM & kNoRing) == 0;
    const float U = stimulus(a, r, n, orig, cnt0);
    if constexpr ((kM & 3) == 1)
        return izh_begin<kPl, kRing>(a, r, n, ck, wc, U, orig, word_now);
    else
        return hh_begin<kPl, kRing>(a, r, n, ck, wc, U, orig, word_now);
}

template <int kM>
__device__ __forceinline__ float2 spiking_begin(const StepArgs &a, int r, int64_t n, float2 wc, int32_t orig,
                                                int32_t cnt0, uint32_t word_now = 0)
{
    return spiking_begin<kM>(a, r, n, step_clock(a, n), wc, orig, cnt0, word_now);
}

// Stimulus, node model kM's Euler step (0 FitzHugh-Nagumo, 1 Izhikevich, 2
// Hodgkin-Huxley), history write, readout, noise, events, arrival.  `orig` (caller
// id) and `cnt0` (background counter) may be prefetched by the caller; kLoad makes
// node_update read them itself.  `ck`: the step's observation bookkeeping.
template <int kM>
__device__ __forceinline__ void node_update(const StepArgs &a, int r, int64_t n, const StepClock &ck, float v,
                                            float2 wc, float S, int32_t orig = kLoad, int32_t cnt0 = kLoad)
{
    if constexpr (kM != 0) {
        psc_finish(a, r, spiking_begin<kM>(a, r, n, ck, wc, orig, cnt0), S);
        return;
    }
    const float U = stimulus(a, r, n, orig, cnt0);
    if (a.bias) S += __ldg(a.bias + r);

    const float w = wc.x, c = wc.y;
    const float dv = fmaf(v, fmaf(v, fmaf(a.q3, v, a.q2), a.k1), -a.cw * w) + S + U;
    const float v1 = fmaf(a.dt, dv, v);
    const float w1 = fmaf(a.dte, fmaf(-a.g, w, v), w);
    const float c1 = fmaf(a.alpha, v1 - c, c);

    a.ring[((n + 1) & a.ring_mask) * a.ring_stride + r] = v1;
    a.wc[r] = make_float2(w1, c1);

    if (v < a.theta_s && v1 >= a.theta_s) record_event(a, r, n + 1);
    if (v1 != 0.0f && v == 0.0f && a.first[r] < 0) a.first[r] = n + 1;

    const float cs = frame_value(a, r, c1, ck.sample);
    if (ck.sample) {
        if (orig == kLoad) orig = __ldg(a.perm + r);
        const float xi = gauss_from(draw(a.obs_seed, static_cast<uint32_t>(orig), ck.k, kStreamObservation));
        const float y = __fmaf_rn(a.sigma, xi, __fmaf_rn(a.gain, __fadd_rn(a.vrest, cs), a.offset));
        a.obs[ck.row + orig] = y;  // rows are written in the caller's node order
    }
}

template <int kM>
__device__ __forceinline__ void node_update(const StepArgs &a, int r, int64_t n, float v, float2 wc, float S,
                                            int32_t orig = kLoad, int32_t cnt0 = kLoad)
{
    node_update<kM>(a, r, n, step_clock(a, n), v, wc, S, orig, cnt0);
}

}  // namespace step
}  // namespace gn
