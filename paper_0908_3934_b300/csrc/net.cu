// Host runtime of libgeonet.so: the C ABI of include/geonet.h for one network.
//
// gn_net_create validates and copies the caller's network, quantises the delays
// on the GPU in FP64, renumbers nodes along a Morton curve (so the sources of
// neighbouring targets sit close in memory and their gathers share sectors),
// builds the by-target edge list with each row sorted by source, packs each edge
// as (src << log2 R) | D next to its FP32 weight, cuts the rows into blocks of at
// most kStepCap - 3 edges for the step kernel, and captures a CUDA graph of
// kGraphSteps step launches.  Everything is held in device memory; the host keeps
// only the permutations and the delay table for output in the caller's order.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/geonet.h"
#include "internal.cuh"

namespace {

thread_local std::string g_last_error;

struct Fail {
    gn_status st;
};

[[noreturn]] void fail(gn_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    throw Fail{st};
}

void cuda_check(cudaError_t e, const char *what)
{
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) fail(GN_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    fail(GN_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cuda_check(cudaSetDevice(dev), "cudaSetDevice");
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Rest point of the isolated FHN vertex: W = (V + f)/g on the W-nullcline and
// a V - b V^3 - c (V + f)/g + I = 0, strictly decreasing when a < c/g.
bool rest_point(const gn_fhn_params &p, double *v_out, double *w_out)
{
    if (!(p.g > 0.0) || !(p.b > 0.0) || !(p.a < p.c / p.g)) return false;
    auto F = [&](double v) { return p.a * v - p.b * v * v * v - p.c * (v + p.f) / p.g + p.i_ext; };
    double lo = -1.0, hi = 1.0;
    for (int i = 0; i < 2000 && F(lo) < 0.0; ++i) lo *= 2.0;
    for (int i = 0; i < 2000 && F(hi) > 0.0; ++i) hi *= 2.0;
    if (!(F(lo) >= 0.0) || !(F(hi) <= 0.0)) return false;
    for (int i = 0; i < 200; ++i) {
        const double m = 0.5 * (lo + hi);
        (F(m) > 0.0 ? lo : hi) = m;
    }
    double v = 0.5 * (lo + hi);
    for (int i = 0; i < 3; ++i) v -= F(v) / (p.a - 3.0 * p.b * v * v - p.c / p.g);
    *v_out = v;
    *w_out = (v + p.f) / p.g;
    return true;
}

// Interleave the low `bits` bits of each coordinate (Morton / Z-order key).
uint64_t spread(uint64_t x, int dims)
{
    uint64_t r = 0;
    for (int b = 0; b < 64 / dims; ++b) r |= ((x >> b) & 1ull) << (b * dims);
    return r;
}

template <class T>
struct DevArray {
    T *p = nullptr;
    size_t n = 0;
    void alloc(size_t count, size_t *total)
    {
        n = count;
        if (count == 0) return;
        cuda_check(cudaMalloc(reinterpret_cast<void **>(&p), count * sizeof(T)), "cudaMalloc");
        *total += count * sizeof(T);
    }
    void release()
    {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
};

constexpr int kGraphSteps = 64;

}  // namespace

struct gn_net {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int32_t N = 0, dim = 0;
    int64_t E = 0;
    int32_t R = 0, dbits = 0, dmax = 0, dmin = 0;
    int64_t n_clamped = 0;
    bool packed = true;
    bool stream_edges = true;
    int n_blocks = 0;
    int step_kernel = 0;       // 0 persistent pipelined, 1 row block per CTA
    int grid = 0;              // CTAs per launch
    int32_t stride = 0;        // ring slot stride (floats)
    double v_rest = 0.0, w_rest = 0.0, dt = 0.0;
    int32_t sample_every = 1;
    int64_t obs_cap = 0, ev_cap = 0;
    int64_t step = 0, read_cursor = 0;
    std::vector<int32_t> perm;        // internal -> caller
    std::vector<int32_t> inv;         // caller -> internal
    std::vector<int32_t> delay;       // caller edge order
    size_t bytes = 0;
    DevArray<float> ring, ew, bias, obs, p_amp;
    DevArray<float2> wc;
    DevArray<uint8_t> ekey;
    DevArray<int32_t> row_ptr, blk, bgc, d_perm, p_node, ev_node, d_npulses;
    int64_t pulse_cap = 0;
    DevArray<int64_t> first, p_on, p_off, ev_step, d_step;
    DevArray<unsigned long long> ev_count;
    DevArray<int4> bdesc;
    DevArray<unsigned int> status;
    gn::StepArgs args{};
    std::vector<uint8_t> stage_pulses;
    cudaGraphExec_t graph = nullptr;
    bool graph_stale = true;

    ~gn_net()
    {
        if (graph) cudaGraphExecDestroy(graph);
        for (auto *a : {&ring, &ew, &bias, &obs, &p_amp}) a->release();
        wc.release();
        ekey.release();
        for (auto *a : {&row_ptr, &blk, &bgc, &d_perm, &p_node, &ev_node, &d_npulses}) a->release();
        for (auto *a : {&first, &p_on, &p_off, &ev_step, &d_step}) a->release();
        ev_count.release();
        bdesc.release();
        status.release();
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

void sync(gn_net *net)
{
    cuda_check(cudaStreamSynchronize(net->stream), "kernel execution");
    unsigned int st = 0;
    cuda_check(cudaMemcpy(&st, net->status.p, 4, cudaMemcpyDeviceToHost), "D2H status");
    if (st) {
        cudaMemset(net->status.p, 0, 4);
        if (st & gn::kStatusTimeout) fail(GN_ETIMEOUT, "a bounded device-side wait gave up (status %u)", st);
        fail(GN_EINTERNAL, "device status word %u", st);
    }
}

cudaError_t launch_one(const gn_net *net, int k, cudaStream_t s)
{
    if (net->step_kernel == 0) return gn::launch_step_pipe(net->args, net->grid, k, net->packed, net->stream_edges, s);
    return gn::launch_step(net->args, net->n_blocks, k, net->packed, net->stream_edges, s);
}

template <class F>
gn_status guarded(F &&f)
{
    try {
        f();
        return GN_OK;
    } catch (const Fail &e) {
        return e.st;
    } catch (const std::bad_alloc &) {
        g_last_error = "host allocation failed";
        return GN_ENOMEM;
    } catch (...) {
        g_last_error = "unexpected exception";
        return GN_EINTERNAL;
    }
}

void build_graph(gn_net *net)
{
    if (net->graph) {
        cudaGraphExecDestroy(net->graph);
        net->graph = nullptr;
    }
    cudaStream_t cs;
    cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int k = 0; k < kGraphSteps && e == cudaSuccess; ++k) e = launch_one(net, k, cs);
        if (e == cudaSuccess) e = gn::launch_advance(net->d_step.p, kGraphSteps, cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&net->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cuda_check(e, "graph capture of the step chunk");
    net->graph_stale = false;
}

void validate_desc(const gn_net_desc *d)
{
    if (!d) fail(GN_EINVAL, "descriptor is NULL");
    if (d->n_nodes <= 0) fail(GN_EINVAL, "n_nodes must be positive");
    if (d->dim < 1 || d->dim > 3) fail(GN_EINVAL, "dim must be 1, 2 or 3");
    if (!d->pos) fail(GN_EINVAL, "pos is NULL");
    if (d->n_edges < 0) fail(GN_EINVAL, "n_edges < 0");
    if (d->n_edges > 2147483647LL - 4 * gn::kEdgePad) fail(GN_ERANGE, "too many edges (limit 2^31 - 16384)");
    if (d->n_edges > 0 && (!d->src || !d->dst || !d->weight)) fail(GN_EINVAL, "edge arrays are NULL");
    if (!(d->dt_ms > 0.0) || !std::isfinite(d->dt_ms)) fail(GN_EINVAL, "dt_ms must be positive");
    if (!(d->obs.tau_ms > 0.0)) fail(GN_EINVAL, "obs.tau_ms must be positive");
    if (d->obs.sample_every <= 0) fail(GN_EINVAL, "obs.sample_every must be positive");
    if (d->coupling != GN_COUPLE_REST && d->coupling != GN_COUPLE_RAW) fail(GN_EINVAL, "unknown coupling");
    if (d->ring_depth < 0 || (d->ring_depth & (d->ring_depth - 1))) fail(GN_EINVAL, "ring_depth must be a power of two");
    if (d->edge_format != 0 && d->edge_format != 1) fail(GN_EINVAL, "edge_format must be 0 or 1");
    if (d->step_kernel != 0 && d->step_kernel != 1) fail(GN_EINVAL, "step_kernel must be 0 or 1");
    const int64_t np = static_cast<int64_t>(d->n_nodes) * d->dim;
    for (int64_t i = 0; i < np; ++i)
        if (!std::isfinite(d->pos[i])) fail(GN_EINVAL, "position %lld is not finite", (long long)i);
    for (int64_t e = 0; e < d->n_edges; ++e) {
        const int32_t i = d->src[e], j = d->dst[e];
        if (i < 0 || i >= d->n_nodes || j < 0 || j >= d->n_nodes)
            fail(GN_EINVAL, "edge %lld: node id out of range", (long long)e);
        if (i == j) fail(GN_EINVAL, "edge %lld: self-loop (the input set excludes i = j)", (long long)e);
        if (!std::isfinite(d->weight[e])) fail(GN_EINVAL, "edge %lld: weight not finite", (long long)e);
        if (d->delay_steps) {
            if (d->delay_steps[e] < 1) fail(GN_EINVAL, "edge %lld: explicit delay < 1 step", (long long)e);
        } else {
            const double s = d->speed ? d->speed[e] : d->speed_scalar;
            if (!(s > 0.0) || !std::isfinite(s)) fail(GN_EINVAL, "edge %lld: speed must be positive", (long long)e);
        }
    }
}

void compute_delays(gn_net *net, const gn_net_desc *d)
{
    const int64_t E = d->n_edges;
    net->delay.assign(E, 1);
    net->n_clamped = 0;
    if (E == 0) return;
    if (d->delay_steps) {
        std::copy(d->delay_steps, d->delay_steps + E, net->delay.begin());
        return;
    }
    size_t tmp = 0;
    DevArray<double> pos, speed;
    DevArray<int32_t> src, dst, dl;
    DevArray<uint8_t> cl;
    try {
        pos.alloc(static_cast<size_t>(d->n_nodes) * d->dim, &tmp);
        src.alloc(E, &tmp);
        dst.alloc(E, &tmp);
        dl.alloc(E, &tmp);
        cl.alloc(E, &tmp);
        if (d->speed) speed.alloc(E, &tmp);
        cuda_check(cudaMemcpyAsync(pos.p, d->pos, pos.n * sizeof(double), cudaMemcpyHostToDevice, net->stream), "H2D pos");
        cuda_check(cudaMemcpyAsync(src.p, d->src, E * 4, cudaMemcpyHostToDevice, net->stream), "H2D src");
        cuda_check(cudaMemcpyAsync(dst.p, d->dst, E * 4, cudaMemcpyHostToDevice, net->stream), "H2D dst");
        if (d->speed)
            cuda_check(cudaMemcpyAsync(speed.p, d->speed, E * 8, cudaMemcpyHostToDevice, net->stream), "H2D speed");
        cuda_check(gn::launch_delay(E, d->dim, pos.p, src.p, dst.p, speed.p, d->speed_scalar, d->dt_ms, dl.p, cl.p,
                                    net->stream),
                   "delay kernel");
        std::vector<uint8_t> hcl(E);
        cuda_check(cudaMemcpyAsync(net->delay.data(), dl.p, E * 4, cudaMemcpyDeviceToHost, net->stream), "D2H delay");
        cuda_check(cudaMemcpyAsync(hcl.data(), cl.p, E, cudaMemcpyDeviceToHost, net->stream), "D2H clamp");
        sync(net);
        for (int64_t e = 0; e < E; ++e) net->n_clamped += hcl[e];
    } catch (...) {
        pos.release(); speed.release(); src.release(); dst.release(); dl.release(); cl.release();
        throw;
    }
    pos.release(); speed.release(); src.release(); dst.release(); dl.release(); cl.release();
}

void renumber(gn_net *net, const gn_net_desc *d)
{
    const int32_t N = d->n_nodes;
    net->perm.resize(N);
    std::iota(net->perm.begin(), net->perm.end(), 0);
    if (d->renumber >= 0 && N > 1) {
        const int dims = d->dim;
        const int bits = 21;  // 21 bits per axis: a 63-bit key in 3D
        std::vector<double> lo(dims, INFINITY), hi(dims, -INFINITY);
        for (int32_t i = 0; i < N; ++i)
            for (int k = 0; k < dims; ++k) {
                lo[k] = std::min(lo[k], d->pos[(int64_t)i * dims + k]);
                hi[k] = std::max(hi[k], d->pos[(int64_t)i * dims + k]);
            }
        double ext = 0.0;
        for (int k = 0; k < dims; ++k) ext = std::max(ext, hi[k] - lo[k]);
        const double scale = ext > 0.0 ? (std::ldexp(1.0, bits) - 1.0) / ext : 0.0;
        std::vector<uint64_t> key(N);
        for (int32_t i = 0; i < N; ++i) {
            uint64_t code = 0;
            for (int k = 0; k < dims; ++k) {
                const uint64_t q = static_cast<uint64_t>((d->pos[(int64_t)i * dims + k] - lo[k]) * scale);
                code |= spread(q, dims) << k;
            }
            key[i] = code;
        }
        std::stable_sort(net->perm.begin(), net->perm.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    }
    net->inv.resize(N);
    for (int32_t r = 0; r < N; ++r) net->inv[net->perm[r]] = r;
}

// By-target edge list with rows sorted by source (two stable counting sorts),
// packed keys and weights, row pointers and row blocks; uploaded to the device.
void build_csr(gn_net *net, const gn_net_desc *d)
{
    const int32_t N = d->n_nodes;
    const int64_t E = d->n_edges;
    std::vector<int32_t> order(E), tmp(E);
    std::vector<int64_t> cnt(static_cast<size_t>(N) + 1, 0);
    for (int64_t e = 0; e < E; ++e) cnt[net->inv[d->src[e]] + 1]++;
    for (int32_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
    for (int64_t e = 0; e < E; ++e) tmp[cnt[net->inv[d->src[e]]]++] = static_cast<int32_t>(e);
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int64_t e = 0; e < E; ++e) cnt[net->inv[d->dst[e]] + 1]++;
    for (int32_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
    std::vector<int32_t> row_ptr(static_cast<size_t>(N) + 1);
    for (int32_t i = 0; i <= N; ++i) row_ptr[i] = static_cast<int32_t>(cnt[i]);
    for (int64_t k = 0; k < E; ++k) {
        const int32_t e = tmp[k];
        order[cnt[net->inv[d->dst[e]]]++] = e;
    }
    tmp.clear();
    tmp.shrink_to_fit();

    const size_t Ep = static_cast<size_t>(E) + gn::kEdgePad;
    std::vector<float> w(Ep, 0.0f);
    std::vector<float> bias;
    if (d->coupling == GN_COUPLE_RAW) bias.assign(N, 0.0f);
    if (net->packed) {
        std::vector<uint32_t> key(Ep, 0u);
        for (int64_t p = 0; p < E; ++p) {
            const int32_t e = order[p];
            key[p] = (static_cast<uint32_t>(net->inv[d->src[e]]) << net->dbits) | static_cast<uint32_t>(net->delay[e]);
            w[p] = d->weight[e];
        }
        net->ekey.alloc(Ep * 4, &net->bytes);
        cuda_check(cudaMemcpy(net->ekey.p, key.data(), Ep * 4, cudaMemcpyHostToDevice), "H2D keys");
    } else {
        std::vector<uint32_t> key(2 * Ep, 0u);
        for (int64_t p = 0; p < E; ++p) {
            const int32_t e = order[p];
            key[2 * p] = static_cast<uint32_t>(net->inv[d->src[e]]);
            key[2 * p + 1] = static_cast<uint32_t>(net->delay[e]);
            w[p] = d->weight[e];
        }
        net->ekey.alloc(Ep * 8, &net->bytes);
        cuda_check(cudaMemcpy(net->ekey.p, key.data(), Ep * 8, cudaMemcpyHostToDevice), "H2D keys");
    }
    if (!bias.empty()) {
        for (int32_t r = 0; r < N; ++r) {
            double s = 0.0;
            for (int32_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) s += static_cast<double>(w[p]);
            bias[r] = static_cast<float>(net->v_rest * s);
        }
        net->bias.alloc(N, &net->bytes);
        cuda_check(cudaMemcpy(net->bias.p, bias.data(), N * 4, cudaMemcpyHostToDevice), "H2D bias");
    }
    net->ew.alloc(Ep, &net->bytes);
    cuda_check(cudaMemcpy(net->ew.p, w.data(), Ep * 4, cudaMemcpyHostToDevice), "H2D weights");
    // padded so 16-byte bulk copies of row_ptr[r0 & ~3 .. (r1 + 4) & ~3) stay inside
    row_ptr.resize(static_cast<size_t>(N) + 1 + 8, row_ptr[N]);
    net->row_ptr.alloc(row_ptr.size(), &net->bytes);
    cuda_check(cudaMemcpy(net->row_ptr.p, row_ptr.data(), row_ptr.size() * 4, cudaMemcpyHostToDevice), "H2D row_ptr");

    // row blocks: consecutive rows with at most kStepCap - 3 edges and kStepMaxRows rows;
    // a longer row gets a block of its own
    std::vector<int32_t> blk{0};
    const int cap = gn::kStepCap - 3;
    int32_t r = 0;
    while (r < N) {
        const int deg0 = row_ptr[r + 1] - row_ptr[r];
        if (deg0 > cap) {
            blk.push_back(++r);
            continue;
        }
        int edges = 0, rows = 0;
        while (r < N && rows < gn::kStepMaxRows) {
            const int deg = row_ptr[r + 1] - row_ptr[r];
            if (deg > cap || edges + deg > cap) break;
            edges += deg;
            ++rows;
            ++r;
        }
        blk.push_back(r);
    }
    net->n_blocks = static_cast<int>(blk.size()) - 1;
    net->blk.alloc(blk.size(), &net->bytes);
    cuda_check(cudaMemcpy(net->blk.p, blk.data(), blk.size() * 4, cudaMemcpyHostToDevice), "H2D blocks");
    std::vector<int4> desc(net->n_blocks);
    for (int b = 0; b < net->n_blocks; ++b) desc[b] = make_int4(blk[b], blk[b + 1], row_ptr[blk[b]], row_ptr[blk[b + 1]]);
    net->bdesc.alloc(desc.size(), &net->bytes);
    if (!desc.empty())
        cuda_check(cudaMemcpy(net->bdesc.p, desc.data(), desc.size() * sizeof(int4), cudaMemcpyHostToDevice), "H2D desc");
}

// Replace the pulse table: validated and sorted by internal node on the host, then
// copied in stream order (steps already queued keep the old table).  The arrays
// only grow; a growth re-points the kernel arguments, so the step graph is rebuilt.
void upload_pulses(gn_net *net, const gn_pulse *pulses, int32_t n)
{
    struct P {
        int32_t node;
        int64_t on, off;
        float amp;
    };
    std::vector<P> ps;
    ps.reserve(n);
    for (int32_t i = 0; i < n; ++i) {
        const gn_pulse &p = pulses[i];
        if (p.node < 0 || p.node >= net->N) fail(GN_EINVAL, "pulse %d: node out of range", i);
        if (!std::isfinite(p.t_on_ms) || !std::isfinite(p.t_off_ms) || !std::isfinite(p.amp))
            fail(GN_EINVAL, "pulse %d: not finite", i);
        const long long on = llround(p.t_on_ms / net->dt), off = llround(p.t_off_ms / net->dt);
        if (off <= on) continue;
        ps.push_back(P{net->inv[p.node], on, off, p.amp});
    }
    std::stable_sort(ps.begin(), ps.end(), [](const P &a, const P &b) { return a.node < b.node; });
    const int64_t m = static_cast<int64_t>(ps.size());
    if (m > net->pulse_cap) {
        sync(net);
        net->p_node.release();
        net->p_on.release();
        net->p_off.release();
        net->p_amp.release();
        const int64_t cap = std::max<int64_t>(m, 2 * net->pulse_cap);
        net->p_node.alloc(cap, &net->bytes);
        net->p_on.alloc(cap, &net->bytes);
        net->p_off.alloc(cap, &net->bytes);
        net->p_amp.alloc(cap, &net->bytes);
        net->pulse_cap = cap;
        net->args.p_node = net->p_node.p;
        net->args.p_on = net->p_on.p;
        net->args.p_off = net->p_off.p;
        net->args.p_amp = net->p_amp.p;
        net->graph_stale = true;
    }
    net->stage_pulses.resize(static_cast<size_t>(m) * 24 + 4);
    auto *nd = reinterpret_cast<int32_t *>(net->stage_pulses.data());
    auto *on = reinterpret_cast<int64_t *>(nd + m + (m & 1));
    auto *off = on + m;
    auto *amp = reinterpret_cast<float *>(off + m);
    for (int64_t i = 0; i < m; ++i) {
        nd[i] = ps[i].node;
        on[i] = ps[i].on;
        off[i] = ps[i].off;
        amp[i] = ps[i].amp;
    }
    if (m) {
        cuda_check(cudaMemcpyAsync(net->p_node.p, nd, m * 4, cudaMemcpyHostToDevice, net->stream), "H2D pulses");
        cuda_check(cudaMemcpyAsync(net->p_on.p, on, m * 8, cudaMemcpyHostToDevice, net->stream), "H2D pulses");
        cuda_check(cudaMemcpyAsync(net->p_off.p, off, m * 8, cudaMemcpyHostToDevice, net->stream), "H2D pulses");
        cuda_check(cudaMemcpyAsync(net->p_amp.p, amp, m * 4, cudaMemcpyHostToDevice, net->stream), "H2D pulses");
    }
    int32_t mm = static_cast<int32_t>(m);
    // a copy from pageable memory is staged before cudaMemcpyAsync returns, so the
    // host table may change right after; the device sees it in stream order
    cuda_check(cudaMemcpyAsync(net->d_npulses.p, &mm, 4, cudaMemcpyHostToDevice, net->stream), "H2D pulse count");
}

template <class T>
void permute_rows_to_caller(const gn_net *net, const T *internal, T *out, int64_t rows)
{
    const int32_t N = net->N;
    for (int64_t k = 0; k < rows; ++k)
        for (int32_t r = 0; r < N; ++r) out[k * N + net->perm[r]] = internal[k * N + r];
}

void check_net(const gn_net *net)
{
    if (!net) fail(GN_EINVAL, "handle is NULL");
}

}  // namespace

extern "C" {

const char *gn_last_error(void) { return g_last_error.c_str(); }

gn_status gn_net_create(const gn_net_desc *desc, gn_net **out)
{
    if (!out) {
        g_last_error = "out is NULL";
        return GN_EINVAL;
    }
    *out = nullptr;
    gn_net *net = nullptr;
    gn_status st = guarded([&] {
        validate_desc(desc);
        double vr, wr;
        if (!rest_point(desc->fhn, &vr, &wr)) fail(GN_EINVAL, "FHN parameters have no unique rest point (need g > 0, b > 0, a < c/g)");
        net = new gn_net();
        net->device = desc->device;
        DeviceGuard dg(desc->device);
        net->N = desc->n_nodes;
        net->dim = desc->dim;
        net->E = desc->n_edges;
        net->v_rest = vr;
        net->w_rest = wr;
        net->dt = desc->dt_ms;
        net->sample_every = desc->obs.sample_every;
        if (desc->cuda_stream) {
            net->stream = static_cast<cudaStream_t>(desc->cuda_stream);
        } else {
            cuda_check(cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking), "cudaStreamCreate");
            net->own_stream = true;
        }
        compute_delays(net, desc);
        int32_t dmax = 1, dmin = net->E ? INT32_MAX : 1;
        for (int32_t D : net->delay) {
            dmax = std::max(dmax, D);
            dmin = std::min(dmin, D);
        }
        net->dmax = dmax;
        net->dmin = dmin;
        if (dmax > (1 << 30)) fail(GN_ERANGE, "delay of %d steps is out of range", dmax);
        int32_t R = 2;
        while (R < dmax + 2) R <<= 1;
        if (desc->ring_depth) {
            if (desc->ring_depth < dmax + 2)
                fail(GN_ERANGE, "ring_depth %d cannot hold the largest delay %d (needs >= D_max + 2)", desc->ring_depth, dmax);
            R = desc->ring_depth;
        }
        net->R = R;
        net->dbits = 0;
        while ((1 << net->dbits) < R) ++net->dbits;
        net->packed = desc->edge_format == 0 && (static_cast<int64_t>(net->N) << net->dbits) <= (1ll << 32);
        if (static_cast<double>(R) * net->N * 4.0 > 200e9) fail(GN_ERANGE, "history ring of %d x %d floats is too large", R, net->N);
        renumber(net, desc);
        build_csr(net, desc);
        // edges are streamed past L2 unless they fit comfortably in it
        const double edge_bytes = static_cast<double>(net->E) * (net->packed ? 8.0 : 12.0);
        net->stream_edges = edge_bytes > 48e6;

        const int32_t N = net->N;
        net->stride = ((N + 4) + 31) / 32 * 32;
        net->ring.alloc(static_cast<size_t>(R) * net->stride, &net->bytes);
        net->wc.alloc(static_cast<size_t>(N) + 2, &net->bytes);
        net->status.alloc(1, &net->bytes);
        cuda_check(cudaMemset(net->status.p, 0, 4), "memset");
        net->bgc.alloc(N, &net->bytes);
        net->first.alloc(N, &net->bytes);
        net->d_perm.alloc(N, &net->bytes);
        net->obs_cap = desc->obs_capacity > 0 ? desc->obs_capacity : 1024;
        net->obs.alloc(static_cast<size_t>(net->obs_cap) * N, &net->bytes);
        net->ev_cap = desc->event_capacity > 0 ? desc->event_capacity : (1 << 20);
        net->ev_node.alloc(net->ev_cap, &net->bytes);
        net->ev_step.alloc(net->ev_cap, &net->bytes);
        net->ev_count.alloc(1, &net->bytes);
        net->d_step.alloc(1, &net->bytes);
        net->d_npulses.alloc(1, &net->bytes);
        cuda_check(cudaMemset(net->d_npulses.p, 0, 4), "memset");
        cuda_check(cudaMemset(net->ring.p, 0, net->ring.n * 4), "memset");
        cuda_check(cudaMemset(net->wc.p, 0, net->wc.n * 8), "memset");
        cuda_check(cudaMemset(net->bgc.p, 0, net->bgc.n * 4), "memset");
        cuda_check(cudaMemset(net->first.p, 0xff, net->first.n * 8), "memset");
        cuda_check(cudaMemset(net->obs.p, 0, net->obs.n * 4), "memset");
        cuda_check(cudaMemset(net->ev_count.p, 0, 8), "memset");
        cuda_check(cudaMemset(net->d_step.p, 0, 8), "memset");
        cuda_check(cudaMemcpy(net->d_perm.p, net->perm.data(), N * 4, cudaMemcpyHostToDevice), "H2D perm");

        gn::StepArgs &a = net->args;
        a.N = N;
        a.ring_stride = net->stride;
        a.ring_mask = R - 1;
        a.bdesc = net->bdesc.p;
        a.n_blocks = net->n_blocks;
        a.status = net->status.p;
        a.dbits = net->dbits;
        a.ekey = net->ekey.p;
        a.ew = net->ew.p;
        a.row_ptr = net->row_ptr.p;
        a.blk = net->blk.p;
        a.ring = net->ring.p;
        a.wc = net->wc.p;
        a.bgc = net->bgc.p;
        a.bias = net->bias.p;
        a.first = net->first.p;
        a.perm = net->d_perm.p;
        a.n_pulses = net->d_npulses.p;
        const gn_fhn_params &f = desc->fhn;
        a.dt = static_cast<float>(desc->dt_ms);
        a.k1 = static_cast<float>(f.a - 3.0 * f.b * vr * vr);
        a.q2 = static_cast<float>(-3.0 * f.b * vr);
        a.q3 = static_cast<float>(-f.b);
        a.cw = static_cast<float>(f.c);
        a.dte = static_cast<float>(desc->dt_ms * f.e);
        a.g = static_cast<float>(f.g);
        a.alpha = static_cast<float>(desc->dt_ms / desc->obs.tau_ms);
        a.theta_s = static_cast<float>(desc->theta - vr);
        a.gain = desc->obs.gain;
        a.offset = desc->obs.offset;
        a.sigma = desc->obs.sigma;
        a.vrest = static_cast<float>(vr);
        a.sample_every = desc->obs.sample_every;
        a.obs_seed = desc->obs.seed;
        a.bg_thr = 0;
        a.obs = net->obs.p;
        a.obs_cap = net->obs_cap;
        a.ev_node = net->ev_node.p;
        a.ev_step = net->ev_step.p;
        a.ev_count = net->ev_count.p;
        a.ev_cap = net->ev_cap;
        a.d_step = net->d_step.p;
        net->step_kernel = desc->step_kernel;
        if (net->step_kernel == 0) {
            int per_sm = 0, sms = 0;
            cuda_check(gn::step_pipe_prepare(net->packed, net->stream_edges, &per_sm), "step kernel setup");
            cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, desc->device), "device query");
            if (per_sm < 1) fail(GN_ECUDA, "the pipelined step kernel does not fit on an SM");
            net->grid = std::min(net->n_blocks, per_sm * sms);
        } else {
            net->grid = net->n_blocks;
        }
        cuda_check(cudaDeviceSynchronize(), "create");
    });
    if (st != GN_OK) {
        delete net;
        return st;
    }
    *out = net;
    return GN_OK;
}

gn_status gn_net_destroy(gn_net *net)
{
    if (!net) return GN_OK;
    return guarded([&] {
        DeviceGuard dg(net->device);
        cudaStreamSynchronize(net->stream);
        delete net;
    });
}

gn_status gn_net_get_info(const gn_net *net, gn_net_info *info)
{
    return guarded([&] {
        check_net(net);
        if (!info) fail(GN_EINVAL, "info is NULL");
        info->n_nodes = net->N;
        info->n_edges = net->E;
        info->dim = net->dim;
        info->ring_depth = net->R;
        info->max_delay = net->dmax;
        info->min_delay = net->dmin;
        info->n_clamped = net->n_clamped;
        info->edge_format = net->packed ? 0 : 1;
        info->n_blocks = net->n_blocks;
        info->step_kernel = net->step_kernel;
        info->grid = net->grid;
        info->step = net->step;
        info->samples = net->step / net->sample_every;
        info->v_rest = net->v_rest;
        info->w_rest = net->w_rest;
        info->device_bytes = net->bytes;
    });
}

gn_status gn_get_delays(const gn_net *net, int32_t *out)
{
    return guarded([&] {
        check_net(net);
        if (!out && net->E) fail(GN_EINVAL, "out is NULL");
        std::copy(net->delay.begin(), net->delay.end(), out);
    });
}

gn_status gn_get_rest(const gn_net *net, double *v_rest, double *w_rest)
{
    return guarded([&] {
        check_net(net);
        if (v_rest) *v_rest = net->v_rest;
        if (w_rest) *w_rest = net->w_rest;
    });
}

gn_status gn_set_stimulus(gn_net *net, const gn_pulse *pulses, int32_t n_pulses)
{
    return guarded([&] {
        check_net(net);
        if (n_pulses < 0 || (n_pulses > 0 && !pulses)) fail(GN_EINVAL, "bad pulse array");
        DeviceGuard dg(net->device);
        upload_pulses(net, pulses, n_pulses);
    });
}

gn_status gn_set_background(gn_net *net, double rate_hz, float amp, double dur_ms, uint64_t seed)
{
    return guarded([&] {
        check_net(net);
        if (!(rate_hz >= 0.0) || !std::isfinite(rate_hz) || !std::isfinite(amp) || !(dur_ms >= 0.0))
            fail(GN_EINVAL, "bad background parameters");
        DeviceGuard dg(net->device);
        sync(net);
        const double p = (rate_hz * net->dt) / 1000.0;
        uint32_t thr = 0;
        if (p > 0.0) {
            const double t = std::floor(std::ldexp(p, 32));
            thr = t >= 4294967295.0 ? 4294967295u : static_cast<uint32_t>(t);
        }
        net->args.bg_thr = thr;
        net->args.bg_amp = amp;
        net->args.bg_width = static_cast<int32_t>(llround(dur_ms / net->dt));
        net->args.bg_seed = seed;
        net->graph_stale = true;
    });
}

gn_status gn_step(gn_net *net, int64_t n_steps)
{
    return guarded([&] {
        check_net(net);
        if (n_steps < 0) fail(GN_EINVAL, "n_steps < 0");
        if (n_steps == 0) return;
        DeviceGuard dg(net->device);
        if (net->graph_stale) build_graph(net);
        int64_t left = n_steps;
        while (left >= kGraphSteps) {
            cuda_check(cudaGraphLaunch(net->graph, net->stream), "cudaGraphLaunch");
            left -= kGraphSteps;
        }
        for (int64_t k = 0; k < left; ++k)
            cuda_check(launch_one(net, static_cast<int>(k), net->stream), "step launch");
        if (left) cuda_check(gn::launch_advance(net->d_step.p, left, net->stream), "advance launch");
        net->step += n_steps;
    });
}

gn_status gn_synchronize(gn_net *net)
{
    return guarded([&] {
        check_net(net);
        DeviceGuard dg(net->device);
        sync(net);
        cuda_check(cudaGetLastError(), "device");
    });
}

gn_status gn_observe(gn_net *net, float *out, int64_t max_samples, int64_t *first_sample, int64_t *written)
{
    return guarded([&] {
        check_net(net);
        if (max_samples < 0) fail(GN_EINVAL, "max_samples < 0");
        DeviceGuard dg(net->device);
        const int64_t produced = net->step / net->sample_every;
        bool lost = false;
        if (produced - net->read_cursor > net->obs_cap) {
            net->read_cursor = produced - net->obs_cap;
            lost = true;
        }
        const int64_t m = std::min(max_samples, produced - net->read_cursor);
        if (first_sample) *first_sample = net->read_cursor;
        if (written) *written = m;
        const size_t row = static_cast<size_t>(net->N) * 4;
        // rows are already in caller order; at most two copies (the ring may wrap)
        int64_t done = out ? 0 : m;  // out == NULL: discard
        while (done < m) {
            const int64_t k = (net->read_cursor + done) % net->obs_cap;
            const int64_t len = std::min(m - done, net->obs_cap - k);
            cuda_check(cudaMemcpyAsync(out + done * net->N, net->obs.p + k * net->N, len * row, cudaMemcpyDeviceToHost,
                                       net->stream),
                       "D2H observations");
            done += len;
        }
        sync(net);
        net->read_cursor += m;
        if (lost) fail(GN_EOVERFLOW, "observation buffer overflowed: older samples were lost");
    });
}

gn_status gn_get_state(gn_net *net, float *v, float *w, float *c, int32_t *bg_count, int64_t *step)
{
    return guarded([&] {
        check_net(net);
        DeviceGuard dg(net->device);
        sync(net);
        const int32_t N = net->N;
        std::vector<float> tmp(N);
        if (v) {
            cuda_check(cudaMemcpy(tmp.data(), net->ring.p + (net->step & (net->R - 1)) * net->stride, N * 4,
                                  cudaMemcpyDeviceToHost),
                       "D2H v");
            permute_rows_to_caller(net, tmp.data(), v, 1);
        }
        if (w || c) {
            std::vector<float2> t2(N);
            cuda_check(cudaMemcpy(t2.data(), net->wc.p, N * 8, cudaMemcpyDeviceToHost), "D2H wc");
            for (int32_t r = 0; r < N; ++r) {
                if (w) w[net->perm[r]] = t2[r].x;
                if (c) c[net->perm[r]] = t2[r].y;
            }
        }
        if (bg_count) {
            std::vector<int32_t> t(N);
            cuda_check(cudaMemcpy(t.data(), net->bgc.p, N * 4, cudaMemcpyDeviceToHost), "D2H bg");
            permute_rows_to_caller(net, t.data(), bg_count, 1);
        }
        if (step) *step = net->step;
    });
}

gn_status gn_set_state(gn_net *net, const float *hist, int32_t depth, const float *w, const float *c,
                       const int32_t *bg_count, int64_t step)
{
    return guarded([&] {
        check_net(net);
        if (depth < 1 || depth > net->R || !hist) fail(GN_EINVAL, "hist must hold 1..ring_depth rows");
        if (step < 0) fail(GN_EINVAL, "step < 0");
        DeviceGuard dg(net->device);
        sync(net);
        const int32_t N = net->N;
        const size_t R = net->R;
        const size_t stride = net->stride;
        std::vector<float> ring(R * stride, 0.0f);
        for (int32_t k = 0; k < depth; ++k) {
            const int64_t slot = (step - k) & (net->R - 1);
            for (int32_t j = 0; j < N; ++j) ring[slot * stride + net->inv[j]] = hist[static_cast<int64_t>(k) * N + j];
        }
        std::vector<float2> wc(N, make_float2(0.0f, 0.0f));
        std::vector<int32_t> bg(N, 0);
        for (int32_t j = 0; j < N; ++j) {
            const int32_t r = net->inv[j];
            wc[r] = make_float2(w ? w[j] : 0.0f, c ? c[j] : 0.0f);
            if (bg_count) bg[r] = bg_count[j];
        }
        cuda_check(cudaMemcpy(net->ring.p, ring.data(), R * stride * 4, cudaMemcpyHostToDevice), "H2D ring");
        cuda_check(cudaMemcpy(net->wc.p, wc.data(), N * 8ull, cudaMemcpyHostToDevice), "H2D wc");
        cuda_check(cudaMemcpy(net->bgc.p, bg.data(), N * 4ull, cudaMemcpyHostToDevice), "H2D bg");
        cuda_check(cudaMemset(net->first.p, 0xff, N * 8ull), "memset");
        cuda_check(cudaMemset(net->ev_count.p, 0, 8), "memset");
        cuda_check(cudaMemcpy(net->d_step.p, &step, 8, cudaMemcpyHostToDevice), "H2D step");
        net->step = step;
        net->read_cursor = step / net->sample_every;
    });
}

gn_status gn_get_history(gn_net *net, float *out, int32_t depth)
{
    return guarded([&] {
        check_net(net);
        if (depth < 1 || depth > net->R) fail(GN_EINVAL, "depth must be in [1, ring_depth]");
        if (!out) fail(GN_EINVAL, "out is NULL");
        DeviceGuard dg(net->device);
        sync(net);
        const int32_t N = net->N;
        std::vector<float> tmp(N);
        for (int32_t k = 0; k < depth; ++k) {
            const int64_t slot = (net->step - k) & (net->R - 1);
            cuda_check(cudaMemcpy(tmp.data(), net->ring.p + slot * net->stride, N * 4, cudaMemcpyDeviceToHost),
                       "D2H history");
            permute_rows_to_caller(net, tmp.data(), out + static_cast<int64_t>(k) * N, 1);
        }
    });
}

gn_status gn_get_arrivals(gn_net *net, int64_t *first_arrival)
{
    return guarded([&] {
        check_net(net);
        if (!first_arrival) fail(GN_EINVAL, "out is NULL");
        DeviceGuard dg(net->device);
        sync(net);
        std::vector<int64_t> t(net->N);
        cuda_check(cudaMemcpy(t.data(), net->first.p, net->N * 8, cudaMemcpyDeviceToHost), "D2H arrivals");
        permute_rows_to_caller(net, t.data(), first_arrival, 1);
    });
}

gn_status gn_get_events(gn_net *net, int32_t *node, int64_t *step, int64_t cap, int64_t *n_total)
{
    return guarded([&] {
        check_net(net);
        if (cap < 0 || (cap > 0 && (!node || !step))) fail(GN_EINVAL, "bad output buffers");
        DeviceGuard dg(net->device);
        sync(net);
        unsigned long long cnt = 0;
        cuda_check(cudaMemcpy(&cnt, net->ev_count.p, 8, cudaMemcpyDeviceToHost), "D2H event count");
        const int64_t kept = std::min<int64_t>(static_cast<int64_t>(cnt), net->ev_cap);
        std::vector<int32_t> nd(kept);
        std::vector<int64_t> st(kept);
        if (kept) {
            cuda_check(cudaMemcpy(nd.data(), net->ev_node.p, kept * 4, cudaMemcpyDeviceToHost), "D2H events");
            cuda_check(cudaMemcpy(st.data(), net->ev_step.p, kept * 8, cudaMemcpyDeviceToHost), "D2H events");
        }
        std::vector<std::pair<int64_t, int32_t>> ev(kept);
        for (int64_t i = 0; i < kept; ++i) ev[i] = {st[i], net->perm[nd[i]]};
        std::sort(ev.begin(), ev.end());
        const int64_t m = std::min(cap, kept);
        for (int64_t i = 0; i < m; ++i) {
            step[i] = ev[i].first;
            node[i] = ev[i].second;
        }
        if (n_total) *n_total = kept;
        if (static_cast<int64_t>(cnt) > net->ev_cap) fail(GN_EOVERFLOW, "event buffer overflowed (%llu events)", cnt);
    });
}

namespace {
struct CkptHeader {
    uint64_t magic;
    int64_t N, R, step;
};
constexpr uint64_t kCkptMagic = 0x67656f6e65743031ull;  // "geonet01"
}  // namespace

gn_status gn_save_state(gn_net *net, void *buf, size_t cap, size_t *used)
{
    return guarded([&] {
        check_net(net);
        const size_t N = net->N, RS = net->ring.n;
        const size_t need = sizeof(CkptHeader) + RS * 4 + N * 8 + N * 4 + N * 8;
        if (used) *used = need;
        if (!buf) return;
        if (cap < need) fail(GN_ERANGE, "checkpoint buffer too small (%zu < %zu)", cap, need);
        DeviceGuard dg(net->device);
        sync(net);
        auto *p = static_cast<uint8_t *>(buf);
        CkptHeader h{kCkptMagic, net->N, net->R, net->step};
        std::memcpy(p, &h, sizeof h);
        p += sizeof h;
        cuda_check(cudaMemcpy(p, net->ring.p, RS * 4, cudaMemcpyDeviceToHost), "D2H ring");
        p += RS * 4;
        cuda_check(cudaMemcpy(p, net->wc.p, N * 8, cudaMemcpyDeviceToHost), "D2H wc");
        p += N * 8;
        cuda_check(cudaMemcpy(p, net->bgc.p, N * 4, cudaMemcpyDeviceToHost), "D2H bg");
        p += N * 4;
        cuda_check(cudaMemcpy(p, net->first.p, N * 8, cudaMemcpyDeviceToHost), "D2H first");
    });
}

gn_status gn_load_state(gn_net *net, const void *buf, size_t size)
{
    return guarded([&] {
        check_net(net);
        if (!buf) fail(GN_EINVAL, "buf is NULL");
        const size_t N = net->N, RS = net->ring.n;
        const size_t need = sizeof(CkptHeader) + RS * 4 + N * 8 + N * 4 + N * 8;
        if (size < need) fail(GN_EINVAL, "checkpoint is truncated");
        CkptHeader h;
        std::memcpy(&h, buf, sizeof h);
        if (h.magic != kCkptMagic || h.N != net->N || h.R != net->R) fail(GN_EINVAL, "checkpoint does not match this network");
        DeviceGuard dg(net->device);
        sync(net);
        const auto *p = static_cast<const uint8_t *>(buf) + sizeof h;
        cuda_check(cudaMemcpy(net->ring.p, p, RS * 4, cudaMemcpyHostToDevice), "H2D ring");
        p += RS * 4;
        cuda_check(cudaMemcpy(net->wc.p, p, N * 8, cudaMemcpyHostToDevice), "H2D wc");
        p += N * 8;
        cuda_check(cudaMemcpy(net->bgc.p, p, N * 4, cudaMemcpyHostToDevice), "H2D bg");
        p += N * 4;
        cuda_check(cudaMemcpy(net->first.p, p, N * 8, cudaMemcpyHostToDevice), "H2D first");
        net->step = h.step;
        net->read_cursor = h.step / net->sample_every;
        cuda_check(cudaMemcpy(net->d_step.p, &h.step, 8, cudaMemcpyHostToDevice), "H2D step");
        cuda_check(cudaMemset(net->ev_count.p, 0, 8), "memset");
    });
}

}  // extern "C"
