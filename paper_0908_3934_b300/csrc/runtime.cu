// Internal host runtime of libgeonet.so (see runtime.h).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <numeric>

#include "runtime.h"

namespace gnrt {

namespace {
thread_local std::string g_last_error;
}

void set_error(const std::string &msg) { g_last_error = msg; }
const char *last_error() { return g_last_error.c_str(); }

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

DeviceGuard::DeviceGuard(int dev)
{
    cudaGetDevice(&prev);
    if (prev != dev) cuda_check(cudaSetDevice(dev), "cudaSetDevice");
}

DeviceGuard::~DeviceGuard()
{
    int cur = -1;
    cudaGetDevice(&cur);
    if (prev >= 0 && cur != prev) cudaSetDevice(prev);
}

gn_status guarded_call(void (*fn)(void *), void *ctx)
{
    try {
        fn(ctx);
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
    if (d->step_kernel < 0 || d->step_kernel > 5) fail(GN_EINVAL, "step_kernel must be 0 to 5");
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
    if (d->model != GN_MODEL_FHN && d->model != GN_MODEL_IZH && d->model != GN_MODEL_HH)
        fail(GN_EINVAL, "unknown node model");
    if (d->stdp.enable) {
        if (d->model == GN_MODEL_FHN) fail(GN_EINVAL, "plasticity needs a spiking node model");
        if (!std::isfinite(d->stdp.alpha) || !std::isfinite(d->stdp.beta) || d->stdp.beta < 0.0)
            fail(GN_EINVAL, "plasticity needs a finite alpha and a finite beta >= 0");
        if (d->step_kernel == 1 || d->step_kernel == 2 || d->step_kernel == 4 || d->step_kernel == 5)
            fail(GN_EINVAL, "plastic networks run the staged step kernel (step_kernel 0 or 3)");
    }
    auto check_hh = [](const gn_hh_params &z) {
        for (double x : {z.C, z.g_na, z.g_k, z.g_l, z.e_na, z.e_k, z.e_l, z.v_peak, z.i_ext, z.psc_a, z.tau_c})
            if (!std::isfinite(x)) fail(GN_EINVAL, "Hodgkin-Huxley parameters must be finite");
        if (!(z.C > 0.0) || !(z.tau_c > 0.0) || z.psc_a < 0.0)
            fail(GN_EINVAL, "Hodgkin-Huxley parameters need C > 0, tau_c > 0, psc_a >= 0");
    };
    auto check_izh = [](const gn_izh_params &z) {
        for (double x : {z.C, z.k, z.v_r, z.v_t, z.v_peak, z.v_reset, z.a, z.b, z.d, z.i_ext, z.psc_a, z.tau_c})
            if (!std::isfinite(x)) fail(GN_EINVAL, "Izhikevich parameters must be finite");
        if (!(z.C > 0.0) || !(z.tau_c > 0.0) || z.psc_a < 0.0)
            fail(GN_EINVAL, "Izhikevich parameters need C > 0, tau_c > 0, psc_a >= 0");
    };
    if (d->n_cell_types < 0 || d->n_cell_types > gn::kMaxCellTypes)
        fail(GN_EINVAL, "n_cell_types must be in [0, %d]", gn::kMaxCellTypes);
    if (d->n_cell_types > 0) {
        if (d->model == GN_MODEL_FHN) fail(GN_EINVAL, "cell types need a spiking node model");
        if (!d->cell_type || (d->model == GN_MODEL_IZH ? !d->izh_types : !d->hh_types))
            fail(GN_EINVAL, "cell types need the parameter sets and each node's set");
        for (int t = 0; t < d->n_cell_types; ++t) {
            if (d->model == GN_MODEL_IZH) check_izh(d->izh_types[t]);
            else check_hh(d->hh_types[t]);
        }
        for (int32_t j = 0; j < d->n_nodes; ++j)
            if (d->cell_type[j] >= d->n_cell_types) fail(GN_EINVAL, "node %d: cell type out of range", j);
    }
    if (d->model == GN_MODEL_HH) {
        check_hh(d->hh);
        return;
    }
    if (d->model == GN_MODEL_IZH) {
        check_izh(d->izh);
        return;
    }
    double vr, wr;
    if (!rest_point(d->fhn, &vr, &wr))
        fail(GN_EINVAL, "FHN parameters have no unique rest point (need g > 0, b > 0, a < c/g)");
}

void quantise_delays(const gn_net_desc *descs, int n_nets, cudaStream_t s, std::vector<std::vector<int32_t>> &delay,
                     std::vector<int64_t> &n_clamped)
{
    delay.assign(n_nets, {});
    n_clamped.assign(n_nets, 0);
    // concatenate the geometric networks: positions with node offsets, edges with
    // global node ids, per-edge speeds; one FP64 launch for all of them
    std::vector<double> pos, speed;
    std::vector<int32_t> src, dst;
    std::vector<int> geo;
    std::vector<int64_t> eoff;
    int dim = -1;
    bool mixed_dim = false;
    for (int i = 0; i < n_nets; ++i) {
        const gn_net_desc &d = descs[i];
        if (d.delay_steps) {
            delay[i].assign(d.delay_steps, d.delay_steps + d.n_edges);
            continue;
        }
        if (dim < 0) dim = d.dim;
        if (d.dim != dim) mixed_dim = true;
    }
    for (int pass = 0; pass < (mixed_dim ? 3 : 1); ++pass) {
        const int want_dim = mixed_dim ? pass + 1 : dim;
        pos.clear(); speed.clear(); src.clear(); dst.clear(); geo.clear(); eoff.clear();
        int64_t noff = 0;
        for (int i = 0; i < n_nets; ++i) {
            const gn_net_desc &d = descs[i];
            if (d.delay_steps || d.dim != want_dim) continue;
            geo.push_back(i);
            eoff.push_back(static_cast<int64_t>(src.size()));
            if (noff + d.n_nodes > 2147483647LL) fail(GN_ERANGE, "too many nodes in one batch");
            pos.insert(pos.end(), d.pos, d.pos + static_cast<int64_t>(d.n_nodes) * d.dim);
            for (int64_t e = 0; e < d.n_edges; ++e) {
                src.push_back(static_cast<int32_t>(d.src[e] + noff));
                dst.push_back(static_cast<int32_t>(d.dst[e] + noff));
                speed.push_back(d.speed ? d.speed[e] : d.speed_scalar);
            }
            noff += d.n_nodes;
        }
        if (geo.empty()) continue;
        eoff.push_back(static_cast<int64_t>(src.size()));
        const int64_t E = static_cast<int64_t>(src.size());
        std::vector<int32_t> dl(E);
        std::vector<uint8_t> cl(E);
        if (E > 0) {
            size_t tmp = 0;
            DevArray<double> d_pos, d_speed;
            DevArray<int32_t> d_src, d_dst, d_dl;
            DevArray<uint8_t> d_cl;
            auto release = [&] {
                d_pos.release(); d_speed.release(); d_src.release(); d_dst.release(); d_dl.release(); d_cl.release();
            };
            try {
                d_pos.upload(pos, &tmp);
                d_speed.upload(speed, &tmp);
                d_src.upload(src, &tmp);
                d_dst.upload(dst, &tmp);
                d_dl.alloc(E, &tmp);
                d_cl.alloc(E, &tmp);
                // every network of this pass shares dt only if all dts match; else one launch per network
                bool same_dt = true;
                for (int i : geo) same_dt = same_dt && descs[i].dt_ms == descs[geo[0]].dt_ms;
                if (same_dt) {
                    cuda_check(gn::launch_delay(E, want_dim, d_pos.p, d_src.p, d_dst.p, d_speed.p, 0.0,
                                                descs[geo[0]].dt_ms, d_dl.p, d_cl.p, s),
                               "delay kernel");
                } else {
                    for (size_t g = 0; g < geo.size(); ++g) {
                        const int64_t a = eoff[g], b = eoff[g + 1];
                        cuda_check(gn::launch_delay(b - a, want_dim, d_pos.p, d_src.p + a, d_dst.p + a, d_speed.p + a,
                                                    0.0, descs[geo[g]].dt_ms, d_dl.p + a, d_cl.p + a, s),
                                   "delay kernel");
                    }
                }
                cuda_check(cudaMemcpyAsync(dl.data(), d_dl.p, E * 4, cudaMemcpyDeviceToHost, s), "D2H delay");
                cuda_check(cudaMemcpyAsync(cl.data(), d_cl.p, E, cudaMemcpyDeviceToHost, s), "D2H clamp");
                cuda_check(cudaStreamSynchronize(s), "delay kernel");
            } catch (...) {
                release();
                throw;
            }
            release();
        }
        for (size_t g = 0; g < geo.size(); ++g) {
            const int i = geo[g];
            delay[i].assign(dl.begin() + eoff[g], dl.begin() + eoff[g + 1]);
            int64_t c = 0;
            for (int64_t e = eoff[g]; e < eoff[g + 1]; ++e) c += cl[e];
            n_clamped[i] = c;
        }
    }
}

namespace {

// Interleave the low bits of each coordinate (Morton / Z-order key).
uint64_t spread(uint64_t x, int dims)
{
    uint64_t r = 0;
    for (int b = 0; b < 64 / dims; ++b) r |= ((x >> b) & 1ull) << (b * dims);
    return r;
}

void renumber(const gn_net_desc *d, HostNet &h)
{
    const int32_t N = d->n_nodes;
    h.perm.resize(N);
    std::iota(h.perm.begin(), h.perm.end(), 0);
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
        std::stable_sort(h.perm.begin(), h.perm.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    }
    h.inv.resize(N);
    for (int32_t r = 0; r < N; ++r) h.inv[h.perm[r]] = r;
}

}  // namespace

void host_build(const gn_net_desc *d, std::vector<int32_t> delay, int64_t n_clamped, int block_cap, int block_rows,
                HostNet &h)
{
    h.N = d->n_nodes;
    h.dim = d->dim;
    h.E = d->n_edges;
    h.delay = std::move(delay);
    h.n_clamped = n_clamped;
    h.model = d->model;
    if (d->model == GN_MODEL_IZH) {
        h.v_rest = d->izh.v_r;  // the state without input: V = v_r, W = 0
        h.w_rest = 0.0;
    } else if (d->model == GN_MODEL_HH) {
        h.v_rest = -65.0;  // the starting state (the gates at their values there)
        h.w_rest = 0.0;
    } else {
        rest_point(d->fhn, &h.v_rest, &h.w_rest);
    }
    const int32_t N = h.N;
    const int64_t E = h.E;
    if (d->n_cell_types > 0) h.type_par = cell_type_rows(d);
    int32_t dmax = 1, dmin = E ? INT32_MAX : 1;
    for (int32_t D : h.delay) {
        dmax = std::max(dmax, D);
        dmin = std::min(dmin, D);
    }
    h.dmax = dmax;
    h.dmin = dmin;
    if (dmax > (1 << 30)) fail(GN_ERANGE, "delay of %d steps is out of range", dmax);
    int32_t R = 2;
    while (R < dmax + 2) R <<= 1;
    if (d->ring_depth) {
        if (d->ring_depth < dmax + 2)
            fail(GN_ERANGE, "ring_depth %d cannot hold the largest delay %d (needs >= D_max + 2)", d->ring_depth, dmax);
        R = d->ring_depth;
    }
    h.R = R;
    h.dbits = 0;
    while ((1 << h.dbits) < R) ++h.dbits;
    h.packed = d->edge_format == 0 && (static_cast<int64_t>(N) << h.dbits) <= (1ll << 32);
    h.stride = ((N + 4) + 31) / 32 * 32;
    if (static_cast<double>(R) * h.stride * 4.0 > 200e9)
        fail(GN_ERANGE, "history ring of %d x %d floats is too large", R, N);
    renumber(d, h);
    if (d->model != GN_MODEL_FHN) {
        h.v0.assign(N, static_cast<float>(h.v_rest));
        if (d->n_cell_types > 0) {
            h.cell.assign(N, 0);
            for (int32_t j = 0; j < N; ++j) {
                const uint8_t t = d->cell_type[j];
                h.cell[h.inv[j]] = t;
                if (d->model == GN_MODEL_IZH) h.v0[h.inv[j]] = static_cast<float>(d->izh_types[t].v_r);
            }
        }
    }

    // by-target rows sorted by source: stable counting sort by source, then by target
    std::vector<int32_t> order(E), tmp(E);
    std::vector<int64_t> cnt(static_cast<size_t>(N) + 1, 0);
    for (int64_t e = 0; e < E; ++e) cnt[h.inv[d->src[e]] + 1]++;
    for (int32_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
    for (int64_t e = 0; e < E; ++e) tmp[cnt[h.inv[d->src[e]]]++] = static_cast<int32_t>(e);
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int64_t e = 0; e < E; ++e) cnt[h.inv[d->dst[e]] + 1]++;
    for (int32_t i = 0; i < N; ++i) cnt[i + 1] += cnt[i];
    h.row_ptr.assign(static_cast<size_t>(N) + 1 + 8, 0);
    for (int32_t i = 0; i <= N; ++i) h.row_ptr[i] = static_cast<int32_t>(cnt[i]);
    for (int i = N + 1; i < N + 9; ++i) h.row_ptr[i] = h.row_ptr[N];
    for (int64_t k = 0; k < E; ++k) {
        const int32_t e = tmp[k];
        order[cnt[h.inv[d->dst[e]]]++] = e;
    }
    tmp.clear();
    tmp.shrink_to_fit();

    const size_t Ep = static_cast<size_t>(E) + gn::kEdgePad;
    h.w.assign(Ep, 0.0f);
    h.key.assign(h.packed ? Ep : 2 * Ep, 0u);
    for (int64_t p = 0; p < E; ++p) {
        const int32_t e = order[p];
        const uint32_t s = static_cast<uint32_t>(h.inv[d->src[e]]);
        if (h.packed) {
            h.key[p] = (s << h.dbits) | static_cast<uint32_t>(h.delay[e]);
        } else {
            h.key[2 * p] = s;
            h.key[2 * p + 1] = static_cast<uint32_t>(h.delay[e]);
        }
        h.w[p] = d->weight[e];
    }
    if (d->stdp.enable) h.eorig = std::move(order);
    if (d->coupling == GN_COUPLE_RAW && d->model == GN_MODEL_FHN) {
        h.bias.assign(N, 0.0f);
        for (int32_t r = 0; r < N; ++r) {
            double sum = 0.0;
            for (int32_t p = h.row_ptr[r]; p < h.row_ptr[r + 1]; ++p) sum += static_cast<double>(h.w[p]);
            h.bias[r] = static_cast<float>(h.v_rest * sum);
        }
    }

    make_blocks(h.row_ptr, N, block_cap, block_rows, h.blk, h.desc);
}

void make_blocks(const std::vector<int32_t> &row_ptr, int32_t N, int cap_edges, int max_rows, std::vector<int32_t> &blk,
                 std::vector<int4> &desc)
{
    blk.assign(1, 0);
    const int cap = cap_edges - 3;
    int32_t r = 0;
    while (r < N) {
        const int deg0 = row_ptr[r + 1] - row_ptr[r];
        if (deg0 > cap) {
            blk.push_back(++r);
            continue;
        }
        int edges = 0, rows = 0;
        while (r < N && rows < max_rows) {
            const int deg = row_ptr[r + 1] - row_ptr[r];
            if (deg > cap || edges + deg > cap) break;
            edges += deg;
            ++rows;
            ++r;
        }
        blk.push_back(r);
    }
    const int nb = static_cast<int>(blk.size()) - 1;
    desc.resize(nb);
    for (int b = 0; b < nb; ++b) desc[b] = make_int4(blk[b], blk[b + 1], row_ptr[blk[b]], row_ptr[blk[b + 1]]);
}

void fill_step_params(const gn_net_desc *d, const HostNet &h, gn::StepArgs &a)
{
    const double vr = h.v_rest;
    const gn_fhn_params &f = d->fhn;
    a.N = h.N;
    a.ring_stride = h.stride;
    a.ring_mask = h.R - 1;
    // GN_TEST_WAIT_LIMIT=k makes the staged kernel's first copy wait give up after k
    // polls: a test of the timeout path that needs no fault (the kernel still waits
    // the full bound for its copies before it leaves)
    a.wait_limit = gn::kDefaultWaitLimit;
    if (const char *e = getenv("GN_TEST_WAIT_LIMIT"); e && *e) a.wait_limit = static_cast<uint32_t>(strtoul(e, nullptr, 10));
    a.dbits = h.dbits;
    a.packed = h.packed ? 1 : 0;
    a.n_blocks = h.n_blocks();
    a.dt = static_cast<float>(d->dt_ms);
    a.k1 = static_cast<float>(f.a - 3.0 * f.b * vr * vr);
    a.q2 = static_cast<float>(-3.0 * f.b * vr);
    a.q3 = static_cast<float>(-f.b);
    a.cw = static_cast<float>(f.c);
    a.dte = static_cast<float>(d->dt_ms * f.e);
    a.g = static_cast<float>(f.g);
    a.alpha = static_cast<float>(d->dt_ms / d->obs.tau_ms);
    a.theta_s = static_cast<float>(d->theta - vr);
    a.gain = d->obs.gain;
    a.offset = d->obs.offset;
    a.sigma = d->obs.sigma;
    a.vrest = static_cast<float>(vr);
    a.sample_every = d->obs.sample_every;
    a.frame_avg = d->obs.frame_average ? 1 : 0;
    a.obs_seed = d->obs.seed;
    a.bg_thr = 0;
    a.bg_amp = 0.0f;
    a.bg_width = 0;
    a.bg_seed = 0;
    a.model = d->model;
    if (d->model == GN_MODEL_IZH) {
        const gn_izh_params &z = d->izh;
        a.iz_dtc = static_cast<float>(d->dt_ms / z.C);
        a.iz_k = static_cast<float>(z.k);
        a.iz_vr = static_cast<float>(z.v_r);
        a.iz_vt = static_cast<float>(z.v_t);
        a.iz_vpeak = static_cast<float>(z.v_peak);
        a.iz_vreset = static_cast<float>(z.v_reset);
        a.iz_dta = static_cast<float>(d->dt_ms * z.a);
        a.iz_b = static_cast<float>(z.b);
        a.iz_d = static_cast<float>(z.d);
        a.iz_iext = static_cast<float>(z.i_ext);
        a.ps_a2 = static_cast<float>(z.psc_a * z.psc_a);
        a.ps_2a = static_cast<float>(2.0 * z.psc_a);
        a.ca_q = static_cast<float>(1.0 / z.tau_c);
        a.vrest = 0.0f;  // the readout is gain c + offset
    }
    a.stdp = d->stdp.enable ? 1 : 0;
    a.stdp_dta = static_cast<float>(d->dt_ms * d->stdp.alpha);
    a.stdp_beta = static_cast<float>(d->stdp.beta);
    if (d->model == GN_MODEL_HH) {
        const gn_hh_params &z = d->hh;
        a.iz_dtc = static_cast<float>(d->dt_ms / z.C);
        a.iz_vpeak = static_cast<float>(z.v_peak);
        a.iz_iext = static_cast<float>(z.i_ext);
        a.hh_gna = static_cast<float>(z.g_na);
        a.hh_gk = static_cast<float>(z.g_k);
        a.hh_gl = static_cast<float>(z.g_l);
        a.hh_ena = static_cast<float>(z.e_na);
        a.hh_ek = static_cast<float>(z.e_k);
        a.hh_el = static_cast<float>(z.e_l);
        a.ps_a2 = static_cast<float>(z.psc_a * z.psc_a);
        a.ps_2a = static_cast<float>(2.0 * z.psc_a);
        a.ca_q = static_cast<float>(1.0 / z.tau_c);
        a.vrest = 0.0f;
    }
}

std::vector<float> cell_type_rows(const gn_net_desc *d)
{
    std::vector<float> rows(static_cast<size_t>(d->n_cell_types) * gn::kTypeStride, 0.0f);
    const double dt = d->dt_ms;
    for (int t = 0; t < d->n_cell_types; ++t) {
        float *q = rows.data() + static_cast<size_t>(t) * gn::kTypeStride;
        if (d->model == GN_MODEL_IZH) {
            const gn_izh_params &z = d->izh_types[t];
            const double v[10] = {dt / z.C, z.k, z.v_r, z.v_t, z.v_peak, z.v_reset, dt * z.a, z.b, z.d, z.i_ext};
            for (int i = 0; i < 10; ++i) q[i] = static_cast<float>(v[i]);
        } else {
            const gn_hh_params &z = d->hh_types[t];
            const double v[9] = {dt / z.C, z.g_na, z.g_k, z.g_l, z.e_na, z.e_k, z.e_l, z.v_peak, z.i_ext};
            for (int i = 0; i < 9; ++i) q[i] = static_cast<float>(v[i]);
        }
        const double psc_a = d->model == GN_MODEL_IZH ? d->izh_types[t].psc_a : d->hh_types[t].psc_a;
        const double tau_c = d->model == GN_MODEL_IZH ? d->izh_types[t].tau_c : d->hh_types[t].tau_c;
        q[gn::kTypeA2] = static_cast<float>(psc_a * psc_a);
        q[gn::kTypeA2 + 1] = static_cast<float>(2.0 * psc_a);
        q[gn::kTypeA2 + 2] = static_cast<float>(1.0 / tau_c);
    }
    return rows;
}

void hh_rest_gates(double *m, double *n, double *h)
{
    // at V = -65 mV: alpha_m = 0.1 (-25) / (1 - e^2.5), beta_m = 4,
    // alpha_h = 0.07, beta_h = 1 / (1 + e^3), alpha_n = 0.01 (-10) / (1 - e^1), beta_n = 0.125
    const double am = 2.5 / std::expm1(2.5), bm = 4.0;
    const double ah = 0.07, bh = 1.0 / (1.0 + std::exp(3.0));
    const double an = 0.1 / std::expm1(1.0), bn = 0.125;
    *m = am / (am + bm);
    *n = an / (an + bn);
    *h = ah / (ah + bh);
}

PulseTable make_pulses(const gn_pulse *pulses, int32_t n, int32_t n_nodes, double dt, const std::vector<int32_t> &inv)
{
    struct P {
        int32_t node;
        int64_t on, off;
        float amp;
    };
    if (n < 0 || (n > 0 && !pulses)) fail(GN_EINVAL, "bad pulse array");
    std::vector<P> ps;
    ps.reserve(n);
    for (int32_t i = 0; i < n; ++i) {
        const gn_pulse &p = pulses[i];
        if (p.node < 0 || p.node >= n_nodes) fail(GN_EINVAL, "pulse %d: node out of range", i);
        if (!std::isfinite(p.t_on_ms) || !std::isfinite(p.t_off_ms) || !std::isfinite(p.amp))
            fail(GN_EINVAL, "pulse %d: not finite", i);
        const long long on = llround(p.t_on_ms / dt), off = llround(p.t_off_ms / dt);
        if (off <= on) continue;
        ps.push_back(P{inv[p.node], on, off, p.amp});
    }
    std::stable_sort(ps.begin(), ps.end(), [](const P &a, const P &b) { return a.node < b.node; });
    PulseTable t;
    for (const P &p : ps) {
        t.node.push_back(p.node);
        t.on.push_back(p.on);
        t.off.push_back(p.off);
        t.amp.push_back(p.amp);
    }
    return t;
}

uint32_t background_threshold(double rate_hz, double dt_ms)
{
    const double p = (rate_hz * dt_ms) / 1000.0;
    if (!(p > 0.0)) return 0u;
    const double t = std::floor(std::ldexp(p, 32));
    return t >= 4294967295.0 ? 4294967295u : static_cast<uint32_t>(t);
}

}  // namespace gnrt
