// Host runtime of libgeonet.so: the single-network part of the C ABI
// (include/geonet.h).
//
// gn_net_create validates and copies the caller's network, quantises the delays
// on the GPU in FP64, renumbers nodes along a Morton curve (so the sources of
// neighbouring targets sit close in memory and their gathers share sectors),
// builds the by-target edge list with each row sorted by source, packs each edge
// as (src << log2 R) | D next to its FP32 weight, cuts the rows into blocks of at
// most T * EPT - 3 edges for the step kernels (the CTA shape is picked by timing
// the candidates on the first gn_step unless the caller fixes the kernel), and
// captures a CUDA graph of kGraphSteps step launches.  Everything is held in device memory; the host keeps
// only the permutations and the delay table for output in the caller's order.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <string>
#include <vector>

#include "runtime.h"

using gnrt::cuda_check;
using gnrt::DevArray;
using gnrt::DeviceGuard;
using gnrt::fail;
using gnrt::guarded;

namespace {
constexpr int kGraphSteps = 64;
}  // namespace

struct gn_net {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t copy_stream = nullptr;  // observation copies queued by gn_observe_async
    cudaEvent_t copy_ready = nullptr;    // recorded on `stream` before each such copy
    int32_t N = 0, dim = 0;
    int64_t E = 0;
    int32_t R = 0, dbits = 0, dmax = 0, dmin = 0;
    int64_t n_clamped = 0;
    bool packed = true;
    bool stream_edges = true;
    int n_blocks = 0;
    int step_kernel = 0;       // 0 not chosen yet (autotune), 1 row block per CTA, 2 persistent pipelined,
                               // 3 staged tiles, 4 resident (the whole network in one CTA's shared memory)
    int shape = 0;             // index into gn::kStepShapes (kernel 2 uses shape 0; kernel 3: gn::kStagedShapes)
    int grid = 0;              // CTAs per launch
    std::vector<int32_t> h_row_ptr;  // host copy, to cut row blocks for another shape
    gn::ResidentLayout res{};  // kernel 4: shared-memory layout of the network
    int32_t stride = 0;        // ring slot stride (floats)
    double v_rest = 0.0, w_rest = 0.0, dt = 0.0;
    int32_t sample_every = 1;
    int64_t obs_cap = 0, ev_cap = 0;
    int64_t step = 0, read_cursor = 0;
    std::vector<int32_t> perm;        // internal -> caller
    std::vector<int32_t> inv;         // caller -> internal
    std::vector<int32_t> delay;       // caller edge order
    size_t bytes = 0;
    DevArray<float> ring, ew, bias, obs, p_amp, iz_v;
    DevArray<float> obs_acc;         // frame sums of the readout state (frame averaging)
    DevArray<float2> wc, rp;
    DevArray<float4> hh_g;           // Hodgkin-Huxley gates (m, n, h, 0)
    DevArray<uint8_t> cell;          // heterogeneous cells: each node's parameter set
    DevArray<float> type_par;        // ... and the sets' parameter rows
    int32_t model = GN_MODEL_FHN;
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
    // staged layout (kernel 3), built from the host edge list, which is kept until
    // the kernel is final
    int st_shape = -1;
    int n_tiles = 0;
    size_t st_smem = 0;
    int64_t st_gathers = 0, st_entries = 0, st_slots = 0;
    int st_max_u = 0, st_max_x = 0, st_max_p = 0;
    int st_early = 0;  // gather order of the staged kernel (mode of launch_step_staged)
    size_t ps_smem = 0;                   // kind 5 (persistent staged tiles): shared memory per CTA
    bool ps_cluster = false;              // ... the grid is one thread-block cluster (at most 16 tiles)
    DevArray<unsigned int> ps_counts;     // ... and its step barrier (64 words)
    DevArray<int4> st_tile, st_tile2;
    DevArray<uint32_t> st_ukey;
    DevArray<int2> st_slice;
    DevArray<float> st_w;
    DevArray<uint16_t> st_u, st_plist;
    DevArray<int32_t> st_rq;
    std::unique_ptr<gnrt::HostNet> host;
    // plastic weights: the entries' caller edges (host) and the lane slots' piece info
    bool stdp = false;
    std::vector<int32_t> st_eidx;
    DevArray<uint32_t> st_pinfo;

    void release_staged()
    {
        st_tile.release();
        st_tile2.release();
        st_ukey.release();
        st_slice.release();
        st_w.release();
        st_u.release();
        st_plist.release();
        st_rq.release();
        st_pinfo.release();
        st_eidx.clear();
        st_shape = -1;
        n_tiles = 0;
    }

    ~gn_net()
    {
        if (graph) cudaGraphExecDestroy(graph);
        for (auto *a : {&ring, &ew, &bias, &obs, &p_amp, &iz_v, &obs_acc}) a->release();
        wc.release();
        rp.release();
        hh_g.release();
        cell.release();
        type_par.release();
        ekey.release();
        for (auto *a : {&row_ptr, &blk, &bgc, &d_perm, &p_node, &ev_node, &d_npulses}) a->release();
        for (auto *a : {&first, &p_on, &p_off, &ev_step, &d_step}) a->release();
        ev_count.release();
        bdesc.release();
        status.release();
        release_staged();
        ps_counts.release();
        if (copy_stream) {
            cudaStreamSynchronize(copy_stream);
            cudaStreamDestroy(copy_stream);
        }
        if (copy_ready) cudaEventDestroy(copy_ready);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

void sync(gn_net *net)
{
    cuda_check(cudaStreamSynchronize(net->stream), "kernel execution");
    if (net->copy_stream) cuda_check(cudaStreamSynchronize(net->copy_stream), "observation copies");
    unsigned int st = 0;
    if (!net->status.p) return;
    cuda_check(cudaMemcpy(&st, net->status.p, 4, cudaMemcpyDeviceToHost), "D2H status");
    if (st) {
        cudaMemset(net->status.p, 0, 4);
        if (st & gn::kStatusTimeout) fail(GN_ETIMEOUT, "a bounded device-side wait gave up (status %u)", st);
        fail(GN_EINTERNAL, "device status word %u", st);
    }
}

// One step launch of the configured kernel with arguments `a` (the network's own,
// or a scratch copy while autotuning).
cudaError_t launch_kind(const gn::StepArgs &a, const gn_net *net, int k, cudaStream_t s)
{
    switch (net->step_kernel) {
        case 4: return k == 0 ? gn::launch_resident(a, net->res, 1, net->shape, s) : cudaErrorInvalidValue;
        case 2: return gn::launch_step_pipe(a, net->grid, k, net->packed, net->stream_edges, s);
        case 3:
            return gn::launch_step_staged(a, net->grid, k, gn::kStagedShapes[net->shape], net->packed,
                                          net->stream_edges, net->st_smem, net->st_early, s);
        default: return gn::launch_step(a, a.n_blocks, k, net->shape, net->packed, net->stream_edges, s);
    }
}

cudaError_t launch_one(const gn_net *net, int k, cudaStream_t s) { return launch_kind(net->args, net, k, s); }

bool same_tiles(const gn::StagedShape &a, const gn::StagedShape &b)
{
    return a.threads == b.threads && a.ucap == b.ucap && a.ecap == b.ecap && a.pcap == b.pcap;
}

// Build and upload the staged layout for a shape (shapes that cut the same tiles
// share it); false if it cannot hold the network (a tile needs more shared memory
// than a CTA may have).
bool set_staged(gn_net *net, int shape)
{
    if (net->st_shape == shape) return true;
    const gn::StagedShape sh = gn::kStagedShapes[shape];
    if (net->st_shape < 0 || !same_tiles(gn::kStagedShapes[net->st_shape], sh)) {
        if (!net->host) return false;
        gnrt::StagedLayout L;
        if (!gnrt::build_staged(*net->host, sh.threads, sh.ucap, sh.ecap, sh.pcap, L)) return false;
        net->release_staged();
        net->st_tile.upload(L.tile, &net->bytes);
        net->st_tile2.upload(L.tile2, &net->bytes);
        net->st_ukey.upload(L.ukey, &net->bytes);
        net->st_slice.upload(L.slice, &net->bytes);
        net->st_w.upload(L.w, &net->bytes);
        net->st_u.upload(L.u, &net->bytes);
        net->st_plist.upload(L.plist, &net->bytes);
        net->st_rq.upload(L.rq, &net->bytes);
        if (net->stdp) {
            net->st_pinfo.upload(L.pinfo, &net->bytes);
            net->st_eidx = std::move(L.eidx);
        }
        gn::StepArgs &a = net->args;
        a.st_tile = net->st_tile.p;
        a.st_tile2 = net->st_tile2.p;
        a.st_ukey = net->st_ukey.p;
        a.st_slice = net->st_slice.p;
        a.st_w = net->st_w.p;
        a.st_u = net->st_u.p;
        a.st_rq = net->st_rq.p;
        a.st_plist = net->st_plist.p;
        a.st_pinfo = net->st_pinfo.p;
        a.st_ucap = L.max_u;
        a.st_xcap = L.max_x;
        net->st_max_u = L.max_u;
        net->st_max_x = L.max_x;
        net->st_max_p = L.max_p;
        net->n_tiles = static_cast<int>(L.tile.size());
        net->st_gathers = static_cast<int64_t>(L.ukey.size()) / (net->packed ? 1 : 2);
        net->st_entries = static_cast<int64_t>(L.w.size());
        net->st_slots = 32 * static_cast<int64_t>(L.slice.size());
        if (net->E == 0) net->st_gathers = net->st_entries = net->st_slots = 0;  // an empty layout's placeholders
        else {
            int64_t g = 0;  // gathers without the alignment padding of each tile's key block
            for (const int4 &t : L.tile) g += t.w;
            net->st_gathers = g;
        }
    }
    int max_smem = 0;
    cuda_check(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, net->device), "device query");
    const size_t smem = 16 + static_cast<size_t>(net->st_max_u) * (net->packed ? 4 : 12) +
                        (sh.stage_entries ? static_cast<size_t>(net->st_max_x) * 6 : 0) +
                        static_cast<size_t>(net->st_max_p) * 4;
    if (smem > static_cast<size_t>(max_smem)) return false;
    if (net->stdp && sh.stage_entries) return false;  // plastic weights are written back to global memory
    int per_sm = 0, sms = 0;
    cuda_check(gn::step_staged_prepare(sh, net->model, net->stdp, net->packed, net->stream_edges, smem, &per_sm),
               "staged kernel setup");
    cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, net->device), "device query");
    // early gathers (static weights): a grid that outnumbers the CTAs the device holds at
    // once lets the next grid start first thing (mode 1); a smaller one lets it start
    // after each CTA's wait (mode 2: on the test set's 300- and 1000-node nets 3.3 against
    // 4.5 us and 3.4 against 5.9 us per step).  GN_STAGED_EARLY=0 waits first (mode 0).
    const bool big = per_sm > 0 && static_cast<int64_t>(net->n_tiles) > static_cast<int64_t>(per_sm) * sms;
    net->st_early = net->stdp ? 0 : big ? 1 : 2;
    if (const char *e = getenv("GN_STAGED_EARLY"); e && *e == '0') net->st_early = 0;
    net->st_smem = smem;
    net->st_shape = shape;
    return true;
}

// The persistent staged kernel (kind 5) on the staged layout of `shape`: its tiles'
// keys, entries, gathered values and piece sums in one CTA's shared memory each, and
// every tile's CTA resident at once; false if the network does not fit.
bool set_persist(gn_net *net, int shape)
{
    if (net->stdp || !set_staged(net, shape) || net->n_tiles < 1) return false;
    const gn::StagedShape sh = gn::kStagedShapes[shape];
    const size_t smem = 16 + static_cast<size_t>(net->st_max_u) * (net->packed ? 8 : 12) +
                        static_cast<size_t>(net->st_max_x) * 6 + static_cast<size_t>(net->st_max_p) * 4;
    int max_smem = 0, per_sm = 0, sms = 0;
    cuda_check(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, net->device), "device query");
    if (smem > static_cast<size_t>(max_smem)) return false;
    // a net of at most kMaxClusterTiles tiles runs as one cluster (GN_PERSIST_CLUSTER=0 turns that off)
    net->ps_cluster = false;
    const char *ce = getenv("GN_PERSIST_CLUSTER");
    if (net->n_tiles <= gn::kMaxClusterTiles && !(ce && *ce == '0')) {
        int clusters = 0;
        const cudaError_t e =
            gn::step_persist_prepare(sh, net->model, net->packed, true, net->n_tiles, smem, &clusters);
        if (e == cudaSuccess && clusters >= 1) net->ps_cluster = true;
        else cudaGetLastError();
        if (const char *log = getenv("GN_PERSIST_LOG"))
            if (FILE *f = fopen(log, "a")) {
                fprintf(f, "persistent shape %d tiles %d smem %zu: cluster query %s, %d clusters\n", shape,
                        net->n_tiles, smem, cudaGetErrorString(e), clusters);
                fclose(f);
            }
    }
    if (!net->ps_cluster) {
        cuda_check(gn::step_persist_prepare(sh, net->model, net->packed, false, net->n_tiles, smem, &per_sm),
                   "persistent kernel setup");
        cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, net->device), "device query");
        if (static_cast<int64_t>(net->n_tiles) > static_cast<int64_t>(per_sm) * sms) return false;
    }
    if (!net->ps_counts.p) net->ps_counts.alloc(64, &net->bytes);
    net->ps_smem = smem;
    return true;
}

// Cut the row blocks for a CTA shape and point the kernel arguments at them.
void set_blocks(gn_net *net, int shape)
{
    std::vector<int32_t> blk;
    std::vector<int4> desc;
    const gn::StepShape sh = gn::kStepShapes[shape];
    gnrt::make_blocks(net->h_row_ptr, net->N, sh.threads * sh.ept, sh.threads, blk, desc);
    net->blk.release();
    net->bdesc.release();
    net->blk.upload(blk, &net->bytes);
    net->bdesc.upload(desc, &net->bytes);
    net->n_blocks = static_cast<int>(desc.size());
    net->args.blk = net->blk.p;
    net->args.bdesc = net->bdesc.p;
    net->args.n_blocks = net->n_blocks;
    net->shape = shape;
}

// Whether the resident kernel in CTA shape `shape` holds the network; on success
// its layout is set and the kernel's shared-memory limit raised.
bool set_resident(gn_net *net, int shape)
{
    if (net->stdp || !net->packed || net->N < 1) return false;
    int longest = 0;
    for (int32_t j = 0; j < net->N; ++j) longest = std::max(longest, net->h_row_ptr[j + 1] - net->h_row_ptr[j]);
    if (longest > gn::kResidentMaxRow) return false;
    for (int ev_factor : {2, 1}) {  // a buffer of two events per node where it fits
        const gn::ResidentLayout L =
            gn::resident_layout(net->N, net->E, net->R, net->model, net->args.frame_avg != 0, ev_factor);
        size_t max_bytes = 0;
        cuda_check(gn::resident_prepare(net->model, shape, L.bytes, &max_bytes), "resident kernel setup");
        if (L.bytes <= max_bytes) {
            net->res = L;
            return true;
        }
    }
    return false;
}

void configure(gn_net *net, int kind, int shape)
{
    if (kind == 5) {
        if (!set_persist(net, shape))
            fail(GN_EINVAL, "the persistent staged kernel cannot hold this network (every tile's CTA must be "
                            "resident at once, with its keys and entries in shared memory; static weights)");
        net->step_kernel = 5;
        net->shape = shape;
        net->grid = net->n_tiles;
        net->graph_stale = true;
        return;
    }
    if (kind == 4) {
        if (!set_resident(net, shape))
            fail(GN_EINVAL, "the resident step kernel cannot hold this network (it must fit one CTA's shared "
                            "memory, with packed edge keys, rows of at most %d edges and static weights)",
                 gn::kResidentMaxRow);
        net->step_kernel = 4;
        net->shape = shape;
        net->grid = 1;
        net->graph_stale = true;
        return;
    }
    if (kind == 3) {
        if (!set_staged(net, shape))
            fail(GN_EINVAL, "the staged step kernel cannot hold this network (a tile needs more shared memory "
                            "than a CTA may have)");
        net->step_kernel = 3;
        net->shape = shape;
        net->grid = net->n_tiles;
        net->graph_stale = true;
        return;
    }
    if (kind == 2) shape = 0;
    set_blocks(net, shape);
    net->step_kernel = kind;
    if (kind == 2) {
        int per_sm = 0, sms = 0;
        cuda_check(gn::step_pipe_prepare(net->model, net->packed, net->stream_edges, &per_sm), "step kernel setup");
        cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, net->device), "device query");
        if (per_sm < 1) fail(GN_ECUDA, "the pipelined step kernel does not fit on an SM");
        net->grid = std::min(net->n_blocks, per_sm * sms);
    } else {
        net->grid = net->n_blocks;
    }
    net->graph_stale = true;
}

// Key of a tuning result: device, sizes and the options that change the kernel.
std::string tune_key(const gn_net *net)
{
    cudaDeviceProp prop{};
    cudaGetDeviceProperties(&prop, net->device);
    std::string name(prop.name);
    for (char &ch : name)
        if (ch == ' ') ch = '_';
    char buf[256];
    snprintf(buf, sizeof buf, "%s|sm%d|N%d|E%lld|R%d|p%d|s%d|bg%d|m%d", name.c_str(), prop.multiProcessorCount, net->N,
             static_cast<long long>(net->E), net->R, net->packed ? 1 : 0, net->stream_edges ? 1 : 0,
             net->args.bg_thr ? 1 : 0, net->model);
    return buf;
}

// Autotune cache: the file named by GN_AUTOTUNE_CACHE holds lines "key kind shape".
bool tune_cache_lookup(const std::string &key, int *kind, int *shape)
{
    const char *path = getenv("GN_AUTOTUNE_CACHE");
    if (!path || !*path) return false;
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char k[256];
    int a = 0, b = 0;
    bool found = false;
    while (fscanf(f, "%255s %d %d", k, &a, &b) == 3)
        if (key == k && b >= 0 &&
            (((a == 1 || a == 2) && b < gn::kNumStepShapes) || ((a == 3 || a == 5) && b < gn::kNumStagedShapes) ||
             (a == 4 && b < gn::kNumResidentShapes))) {
            *kind = a;
            *shape = b;
            found = true;
        }
    fclose(f);
    return found;
}

void tune_cache_store(const std::string &key, int kind, int shape)
{
    const char *path = getenv("GN_AUTOTUNE_CACHE");
    if (!path || !*path) return;
    FILE *f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d\n", key.c_str(), kind, shape);
    fclose(f);
}

// Autotuner: time every candidate (row-block kernel in each CTA shape, the
// persistent pipelined kernel and the staged kernel in each of its shapes) for a few steps on a scratch copy of the dynamic
// state -- the network's own state is not touched -- and keep the fastest.  With
// GN_AUTOTUNE_CACHE set, a cached choice for the same device and network sizes is
// reused and new choices are appended; with GN_AUTOTUNE_LOG set, every candidate's
// time is appended to that file.
void autotune(gn_net *net)
{
    const std::string key = tune_key(net);
    int cached_kind = 0, cached_shape = 0;
    if (tune_cache_lookup(key, &cached_kind, &cached_shape) && (cached_kind != 3 || set_staged(net, cached_shape)) &&
        (cached_kind != 4 || set_resident(net, cached_shape)) && (cached_kind != 5 || set_persist(net, cached_shape))) {
        configure(net, cached_kind, cached_shape);
        return;
    }
    const int32_t N = net->N;
    size_t scratch_bytes = 0;
    DevArray<float> ring, obs, iz_v, obs_acc;
    DevArray<float2> wc, rp;
    DevArray<float4> hh_g;
    DevArray<int32_t> bgc, evn;
    DevArray<int64_t> first, evs, dstep;
    DevArray<unsigned long long> evc;
    DevArray<unsigned int> status;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    auto cleanup = [&] {
        ring.release(); obs.release(); wc.release(); bgc.release(); evn.release(); first.release();
        evs.release(); dstep.release(); evc.release(); status.release(); iz_v.release(); rp.release();
        hh_g.release(); obs_acc.release();
        if (t0) cudaEventDestroy(t0);
        if (t1) cudaEventDestroy(t1);
    };
    int best_kind = 1, best_shape = 0;
    try {
        ring.alloc(net->ring.n, &scratch_bytes);
        wc.alloc(net->wc.n, &scratch_bytes);
        bgc.alloc(N, &scratch_bytes);
        first.alloc(N, &scratch_bytes);
        obs.alloc(N, &scratch_bytes);
        evn.alloc(1024, &scratch_bytes);
        evs.alloc(1024, &scratch_bytes);
        evc.alloc(1, &scratch_bytes);
        dstep.alloc(1, &scratch_bytes);
        status.alloc(1, &scratch_bytes);
        if (net->model != GN_MODEL_FHN) {  // the spiking models' state too, from the net's own values
            iz_v.alloc(N, &scratch_bytes);
            rp.alloc(N, &scratch_bytes);
            cuda_check(cudaMemcpyAsync(iz_v.p, net->iz_v.p, N * 4ull, cudaMemcpyDeviceToDevice, net->stream), "D2D");
            cuda_check(cudaMemcpyAsync(rp.p, net->rp.p, N * 8ull, cudaMemcpyDeviceToDevice, net->stream), "D2D");
        }
        if (net->args.frame_avg) {
            obs_acc.alloc(N, &scratch_bytes);
            cuda_check(cudaMemsetAsync(obs_acc.p, 0, N * 4ull, net->stream), "memset");
        }
        if (net->model == GN_MODEL_HH) {
            hh_g.alloc(N, &scratch_bytes);
            cuda_check(cudaMemcpyAsync(hh_g.p, net->hh_g.p, N * 16ull, cudaMemcpyDeviceToDevice, net->stream), "D2D");
        }
        cuda_check(cudaMemsetAsync(ring.p, 0, ring.n * 4, net->stream), "memset");
        cuda_check(cudaMemsetAsync(wc.p, 0, wc.n * 8, net->stream), "memset");
        cuda_check(cudaMemsetAsync(bgc.p, 0, bgc.n * 4, net->stream), "memset");
        cuda_check(cudaMemsetAsync(first.p, 0xff, first.n * 8, net->stream), "memset");
        cuda_check(cudaMemsetAsync(evc.p, 0, 8, net->stream), "memset");
        cuda_check(cudaMemsetAsync(status.p, 0, 4, net->stream), "memset");
        cuda_check(cudaMemcpyAsync(dstep.p, &net->step, 8, cudaMemcpyHostToDevice, net->stream), "H2D");
        cuda_check(cudaEventCreate(&t0), "event");
        cuda_check(cudaEventCreate(&t1), "event");
        float best = 1e30f;
        struct Cand {
            int kind, shape;
        };
        std::vector<Cand> cands;
        for (int sh = 0; sh < gn::kNumStepShapes; ++sh) cands.push_back({1, sh});
        cands.push_back({2, 0});
        for (int sh = 0; sh < gn::kNumStagedShapes; ++sh) cands.push_back({3, sh});
        for (int sh = 0; sh < gn::kNumResidentShapes; ++sh) cands.push_back({4, sh});
        for (int sh = 0; sh < gn::kNumStagedShapes; ++sh) cands.push_back({5, sh});
        for (const Cand &c : cands) {
            if (c.kind == 3 && !set_staged(net, c.shape)) continue;
            if (c.kind == 4 && !set_resident(net, c.shape)) continue;
            if (c.kind == 5 && !set_persist(net, c.shape)) continue;
            configure(net, c.kind, c.shape);
            gn::StepArgs a = net->args;
            a.ring = ring.p;
            a.wc = wc.p;
            a.bgc = bgc.p;
            a.first = first.p;
            a.obs = obs.p;
            a.obs_cap = 1;
            a.ev_node = evn.p;
            a.ev_step = evs.p;
            a.ev_count = evc.p;
            a.ev_cap = 1024;
            a.d_step = dstep.p;
            a.status = status.p;
            a.iz_v = iz_v.p;
            a.rp = rp.p;
            a.hh_g = hh_g.p;
            a.obs_acc = obs_acc.p;
            // each candidate is timed as gn_step runs it: kernels 1 to 3 as a captured graph
            // of kGraphSteps step launches (replayed once untimed, then timed), the resident
            // kernel as one launch of kResidentSteps x kGraphSteps steps, the persistent
            // kernel as one launch of kGraphSteps steps (each after an untimed launch)
            const int timed = kGraphSteps;
            constexpr int kResidentSteps = 8;
            cudaGraphExec_t ge = nullptr;
            if (c.kind == 4) {
                cuda_check(gn::launch_resident(a, net->res, kResidentSteps, c.shape, net->stream), "autotune launch");
            } else if (c.kind == 5) {
                cuda_check(gn::launch_step_persist(a, net->n_tiles, 3, gn::kStagedShapes[c.shape], net->packed,
                                                   net->ps_cluster, net->ps_counts.p, net->ps_smem, net->stream),
                           "autotune launch");
            } else {
                cudaStream_t cs = nullptr;
                cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
                cudaGraph_t g = nullptr;
                cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
                for (int k = 0; k < timed && e == cudaSuccess; ++k) e = launch_kind(a, net, k, cs);
                const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
                if (e == cudaSuccess) e = e2;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
                if (g) cudaGraphDestroy(g);
                cudaStreamDestroy(cs);
                cuda_check(e, "autotune graph capture");
                e = cudaGraphLaunch(ge, net->stream);  // untimed
                if (e != cudaSuccess) cudaGraphExecDestroy(ge);
                cuda_check(e, "autotune launch");
            }
            cudaError_t te = cudaEventRecord(t0, net->stream);
            if (te == cudaSuccess) {
                if (c.kind == 4)
                    te = gn::launch_resident(a, net->res, kResidentSteps * timed, c.shape, net->stream);
                else if (c.kind == 5)
                    te = gn::launch_step_persist(a, net->n_tiles, timed, gn::kStagedShapes[c.shape], net->packed,
                                                 net->ps_cluster, net->ps_counts.p, net->ps_smem, net->stream);
                else
                    te = cudaGraphLaunch(ge, net->stream);
            }
            if (te == cudaSuccess) te = cudaEventRecord(t1, net->stream);
            if (te == cudaSuccess) te = cudaEventSynchronize(t1);
            if (ge) cudaGraphExecDestroy(ge);
            cuda_check(te, "autotune");
            float ms = 0.0f;
            cuda_check(cudaEventElapsedTime(&ms, t0, t1), "event");
            if (c.kind == 4) ms /= kResidentSteps;
            if (const char *log = getenv("GN_AUTOTUNE_LOG")) {
                if (FILE *f = fopen(log, "a")) {
                    fprintf(f, "%s kind %d shape %d ms_per_step %.5f\n", key.c_str(), c.kind, c.shape, ms / timed);
                    fclose(f);
                }
            }
            if (ms < best) {
                best = ms;
                best_kind = c.kind;
                best_shape = c.shape;
            }
        }
        unsigned int st = 0;
        cuda_check(cudaMemcpy(&st, status.p, 4, cudaMemcpyDeviceToHost), "D2H status");
        if (st) fail(GN_ETIMEOUT, "a bounded device-side wait gave up while autotuning");
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
    configure(net, best_kind, best_shape);
    tune_cache_store(key, best_kind, best_shape);
}

// The kernel is final: drop the host edge list and any staged layout it does not use.
void finalize_kernel(gn_net *net)
{
    if (net->step_kernel != 3 && net->step_kernel != 5) net->release_staged();
    net->host.reset();
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

// Replace the pulse table: validated and sorted by internal node on the host, then
// copied in stream order (steps already queued keep the old table).  The arrays
// only grow; a growth re-points the kernel arguments, so the step graph is rebuilt.
void upload_pulses(gn_net *net, const gn_pulse *pulses, int32_t n)
{
    gnrt::PulseTable t = gnrt::make_pulses(pulses, n, net->N, net->dt, net->inv);
    const int64_t m = static_cast<int64_t>(t.node.size());
    if (m > net->pulse_cap) {
        cuda_check(cudaStreamSynchronize(net->stream), "pulse upload");
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
    // a copy from pageable memory is staged before cudaMemcpyAsync returns, so the
    // host table may change right after; the device sees it in stream order
    if (m) {
        cuda_check(cudaMemcpyAsync(net->p_node.p, t.node.data(), m * 4, cudaMemcpyHostToDevice, net->stream), "H2D pulses");
        cuda_check(cudaMemcpyAsync(net->p_on.p, t.on.data(), m * 8, cudaMemcpyHostToDevice, net->stream), "H2D pulses");
        cuda_check(cudaMemcpyAsync(net->p_off.p, t.off.data(), m * 8, cudaMemcpyHostToDevice, net->stream), "H2D pulses");
        cuda_check(cudaMemcpyAsync(net->p_amp.p, t.amp.data(), m * 4, cudaMemcpyHostToDevice, net->stream), "H2D pulses");
    }
    const int32_t mm = static_cast<int32_t>(m);
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

const char *gn_last_error(void) { return gnrt::last_error(); }

gn_status gn_net_create(const gn_net_desc *desc, gn_net **out)
{
    if (!out) {
        gnrt::set_error("out is NULL");
        return GN_EINVAL;
    }
    *out = nullptr;
    gn_net *net = nullptr;
    gn_status st = guarded([&] {
        gnrt::validate_desc(desc);
        net = new gn_net();
        net->device = desc->device;
        DeviceGuard dg(desc->device);
        if (desc->cuda_stream) {
            net->stream = static_cast<cudaStream_t>(desc->cuda_stream);
        } else {
            cuda_check(cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking), "cudaStreamCreate");
            net->own_stream = true;
        }
        std::vector<std::vector<int32_t>> delays;
        std::vector<int64_t> clamped;
        gnrt::quantise_delays(desc, 1, net->stream, delays, clamped);
        gnrt::HostNet h;
        const gn::StepShape sh0 = gn::kStepShapes[0];
        gnrt::host_build(desc, std::move(delays[0]), clamped[0], sh0.threads * sh0.ept, sh0.threads, h);

        net->N = h.N;
        net->dim = h.dim;
        net->E = h.E;
        net->R = h.R;
        net->dbits = h.dbits;
        net->dmax = h.dmax;
        net->dmin = h.dmin;
        net->n_clamped = h.n_clamped;
        net->packed = h.packed;
        net->stride = h.stride;
        net->n_blocks = h.n_blocks();
        net->v_rest = h.v_rest;
        net->w_rest = h.w_rest;
        net->dt = desc->dt_ms;
        net->sample_every = desc->obs.sample_every;
        net->perm = h.perm;
        net->inv = h.inv;
        net->delay = h.delay;
        net->h_row_ptr = h.row_ptr;
        // edges are streamed past L2 unless they fit comfortably in it (GN_STREAM_EDGES=0 or 1
        // in the environment overrides the rule)
        net->stream_edges = static_cast<double>(net->E) * (net->packed ? 8.0 : 12.0) > 48e6;
        if (const char *e = getenv("GN_STREAM_EDGES"); e && (*e == '0' || *e == '1')) net->stream_edges = *e == '1';

        const int32_t N = net->N;
        net->ekey.alloc(h.key.size() * 4, &net->bytes);
        cuda_check(cudaMemcpy(net->ekey.p, h.key.data(), h.key.size() * 4, cudaMemcpyHostToDevice), "H2D keys");
        net->ew.upload(h.w, &net->bytes);
        net->bias.upload(h.bias, &net->bytes);
        net->row_ptr.upload(h.row_ptr, &net->bytes);
        net->d_perm.upload(h.perm, &net->bytes);
        net->ring.alloc(static_cast<size_t>(net->R) * net->stride, &net->bytes);
        net->wc.alloc(static_cast<size_t>(N) + 2, &net->bytes);
        net->status.alloc(1, &net->bytes);
        net->bgc.alloc(N, &net->bytes);
        net->first.alloc(N, &net->bytes);
        net->obs_cap = desc->obs_capacity > 0 ? desc->obs_capacity : 1024;
        net->obs.alloc(static_cast<size_t>(net->obs_cap) * N, &net->bytes);
        net->ev_cap = desc->event_capacity > 0 ? desc->event_capacity : (1 << 20);
        net->ev_node.alloc(net->ev_cap, &net->bytes);
        net->ev_step.alloc(net->ev_cap, &net->bytes);
        net->ev_count.alloc(1, &net->bytes);
        net->d_step.alloc(1, &net->bytes);
        net->d_npulses.alloc(1, &net->bytes);
        cuda_check(cudaMemset(net->ring.p, 0, net->ring.n * 4), "memset");
        cuda_check(cudaMemset(net->wc.p, 0, net->wc.n * 8), "memset");
        cuda_check(cudaMemset(net->status.p, 0, 4), "memset");
        cuda_check(cudaMemset(net->bgc.p, 0, net->bgc.n * 4), "memset");
        cuda_check(cudaMemset(net->first.p, 0xff, net->first.n * 8), "memset");
        cuda_check(cudaMemset(net->obs.p, 0, net->obs.n * 4), "memset");
        cuda_check(cudaMemset(net->ev_count.p, 0, 8), "memset");
        cuda_check(cudaMemset(net->d_step.p, 0, 8), "memset");
        cuda_check(cudaMemset(net->d_npulses.p, 0, 4), "memset");
        net->model = desc->model;
        if (net->model != GN_MODEL_FHN) {
            net->iz_v.upload(h.v0, &net->bytes);
            net->rp.alloc(N, &net->bytes);
            cuda_check(cudaMemset(net->rp.p, 0, net->rp.n * 8), "memset");
        }
        if (net->model == GN_MODEL_HH) {
            double m, n, hg;
            gnrt::hh_rest_gates(&m, &n, &hg);
            net->hh_g.upload(std::vector<float4>(N, make_float4(static_cast<float>(m), static_cast<float>(n),
                                                                static_cast<float>(hg), 0.0f)),
                             &net->bytes);
        }

        gn::StepArgs &a = net->args;
        gnrt::fill_step_params(desc, h, a);
        if (a.frame_avg) {
            net->obs_acc.alloc(N, &net->bytes);
            cuda_check(cudaMemset(net->obs_acc.p, 0, N * 4ull), "memset");
        }
        a.obs_acc = net->obs_acc.p;
        if (!h.cell.empty()) {
            net->cell.upload(h.cell, &net->bytes);
            net->type_par.upload(h.type_par, &net->bytes);
        }
        a.cell_type = net->cell.p;
        a.type_par = net->type_par.p;
        a.ekey = net->ekey.p;
        a.ew = net->ew.p;
        a.row_ptr = net->row_ptr.p;
        a.ring = net->ring.p;
        a.wc = net->wc.p;
        a.bgc = net->bgc.p;
        a.bias = net->bias.p;
        a.first = net->first.p;
        a.perm = net->d_perm.p;
        a.n_pulses = net->d_npulses.p;
        a.obs = net->obs.p;
        a.obs_cap = net->obs_cap;
        a.ev_node = net->ev_node.p;
        a.ev_step = net->ev_step.p;
        a.ev_count = net->ev_count.p;
        a.ev_cap = net->ev_cap;
        a.d_step = net->d_step.p;
        a.status = net->status.p;
        a.iz_v = net->iz_v.p;
        a.rp = net->rp.p;
        a.hh_g = net->hh_g.p;

        // the kernel is fixed now or timed on the first gn_step (kind 0)
        // a plastic net runs the staged kernel, fixed now: the weights live in its layout
        net->stdp = desc->stdp.enable != 0;
        const int kind = net->stdp ? 3 : desc->step_kernel;
        if (kind == 0 || kind == 3 || kind == 5) net->host = std::make_unique<gnrt::HostNet>(std::move(h));
        // GN_STEP_SHAPE=i picks the CTA shape of an explicitly chosen kernel 1, 3, 4 or 5
        // (plastic default: the 12288-edge tiles, measured best on the 1M-node net --
        // 0.139 ms per step against 0.149 and 0.167 for 8192 and 16384 edges)
        int shape = net->stdp ? 4 : kind == 4 ? 1 : 0;
        if (const char *e = getenv("GN_STEP_SHAPE"); e && *e && kind >= 1 && kind != 2) {
            shape = atoi(e);
            const int n_shapes = kind == 1                ? gn::kNumStepShapes
                                 : kind == 3 || kind == 5 ? gn::kNumStagedShapes
                                                          : gn::kNumResidentShapes;
            if (shape < 0 || shape >= n_shapes) fail(GN_EINVAL, "GN_STEP_SHAPE=%s is not a shape of kernel %d", e,
                                                       kind);
            if (net->stdp && gn::kStagedShapes[shape].stage_entries)
                fail(GN_EINVAL, "GN_STEP_SHAPE=%s stages the edge entries, which plastic weights cannot use", e);
        }
        configure(net, kind == 2 ? 2 : 1, kind == 1 ? shape : 0);
        if (kind >= 3) configure(net, kind, shape);
        if (kind == 0)
            net->step_kernel = 0;
        else
            finalize_kernel(net);
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
        const bool staged = net->step_kernel == 3 || net->step_kernel == 5, resident = net->step_kernel == 4;
        info->n_blocks = staged ? net->n_tiles : resident ? 1 : net->n_blocks;
        info->step_kernel = net->step_kernel;
        info->step_threads = staged     ? gn::kStagedShapes[net->shape].threads
                             : resident ? gn::kResidentThreads[net->shape]
                                        : gn::kStepShapes[net->shape].threads;
        info->step_edges_per_thread = (staged || resident) ? gn::kWarpRow : gn::kStepShapes[net->shape].ept;
        info->grid = net->grid;
        info->step = net->step;
        info->samples = net->step / net->sample_every;
        info->v_rest = net->v_rest;
        info->w_rest = net->w_rest;
        info->device_bytes = net->bytes;
        info->step_gathers = staged ? net->st_gathers : net->E;
        info->step_entries = staged ? net->st_entries : net->E;
        info->step_lane_slots = staged ? net->st_slots : 0;
        info->step_cluster = net->step_kernel == 5 && net->ps_cluster ? 1 : 0;
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
        const uint32_t thr = gnrt::background_threshold(rate_hz, net->dt);
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
        if (net->step_kernel == 0) {
            autotune(net);
            finalize_kernel(net);
        }
        if (net->step_kernel == 5) {
            // the persistent staged kernel: a launch runs up to kPersistChunk steps
            constexpr int64_t kPersistChunk = 1 << 16;
            for (int64_t left = n_steps; left > 0; left -= kPersistChunk) {
                const int chunk = static_cast<int>(std::min(left, kPersistChunk));
                cuda_check(gn::launch_step_persist(net->args, net->n_tiles, chunk, gn::kStagedShapes[net->shape],
                                                   net->packed, net->ps_cluster, net->ps_counts.p, net->ps_smem,
                                                   net->stream),
                           "persistent launch");
                cuda_check(gn::launch_advance(net->d_step.p, chunk, net->stream), "advance launch");
            }
            net->step += n_steps;
            return;
        }
        if (net->step_kernel == 4) {
            // the resident kernel: a launch runs up to kResidentChunk steps
            constexpr int64_t kResidentChunk = 1 << 16;
            for (int64_t left = n_steps; left > 0; left -= kResidentChunk) {
                const int chunk = static_cast<int>(std::min(left, kResidentChunk));
                cuda_check(gn::launch_resident(net->args, net->res, chunk, net->shape, net->stream), "resident launch");
                cuda_check(gn::launch_advance(net->d_step.p, chunk, net->stream), "advance launch");
            }
            net->step += n_steps;
            return;
        }
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

namespace {

// The unread rows (at most max_samples) copied into out on stream s (at most two
// copies: the ring may wrap); advances the read cursor; true if rows were lost.
bool copy_observations(gn_net *net, float *out, int64_t max_samples, int64_t *first_sample, int64_t *written,
                       cudaStream_t s)
{
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
    int64_t done = out ? 0 : m;  // out == NULL: discard
    while (done < m) {
        const int64_t k = (net->read_cursor + done) % net->obs_cap;
        const int64_t len = std::min(m - done, net->obs_cap - k);
        cuda_check(cudaMemcpyAsync(out + done * net->N, net->obs.p + k * net->N, len * row, cudaMemcpyDeviceToHost, s),
                   "D2H observations");
        done += len;
    }
    net->read_cursor += m;
    return lost;
}

}  // namespace

gn_status gn_observe_async(gn_net *net, float *out, int64_t max_samples, int64_t *first_sample, int64_t *written)
{
    return guarded([&] {
        check_net(net);
        if (max_samples < 0) fail(GN_EINVAL, "max_samples < 0");
        DeviceGuard dg(net->device);
        if (!net->copy_stream) {
            cuda_check(cudaStreamCreateWithFlags(&net->copy_stream, cudaStreamNonBlocking), "cudaStreamCreate");
            cuda_check(cudaEventCreateWithFlags(&net->copy_ready, cudaEventDisableTiming), "cudaEventCreate");
        }
        cuda_check(cudaEventRecord(net->copy_ready, net->stream), "event");
        cuda_check(cudaStreamWaitEvent(net->copy_stream, net->copy_ready, 0), "stream wait");
        if (copy_observations(net, out, max_samples, first_sample, written, net->copy_stream))
            fail(GN_EOVERFLOW, "observation buffer overflowed: older samples were lost");
    });
}

gn_status gn_observe_wait(gn_net *net)
{
    return guarded([&] {
        check_net(net);
        DeviceGuard dg(net->device);
        if (net->copy_stream) cuda_check(cudaStreamSynchronize(net->copy_stream), "observation copies");
    });
}

gn_status gn_observe(gn_net *net, float *out, int64_t max_samples, int64_t *first_sample, int64_t *written)
{
    return guarded([&] {
        check_net(net);
        if (max_samples < 0) fail(GN_EINVAL, "max_samples < 0");
        DeviceGuard dg(net->device);
        // rows are already in caller order
        const bool lost = copy_observations(net, out, max_samples, first_sample, written, net->stream);
        sync(net);
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
            const float *src = net->model != GN_MODEL_FHN ? net->iz_v.p
                                                          : net->ring.p + (net->step & (net->R - 1)) * net->stride;
            cuda_check(cudaMemcpy(tmp.data(), src, N * 4, cudaMemcpyDeviceToHost), "D2H v");
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
            for (int32_t j = 0; j < N; ++j) {
                const float x = hist[static_cast<int64_t>(k) * N + j];
                if (net->stdp) {  // the spike bit, s = 0 (gn_set_stdp_history sets s)
                    const uint32_t word = x != 0.0f ? 1u : 0u;
                    std::memcpy(&ring[slot * stride + net->inv[j]], &word, 4);
                } else {
                    ring[slot * stride + net->inv[j]] = x;
                }
            }
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
        if (net->obs_acc.p) cuda_check(cudaMemset(net->obs_acc.p, 0, N * 4ull), "memset");  // a new frame
        cuda_check(cudaMemcpy(net->d_step.p, &step, 8, cudaMemcpyHostToDevice), "H2D step");
        net->step = step;
        net->read_cursor = step / net->sample_every;
    });
}

gn_status gn_get_izh_state(gn_net *net, float *V, float *r, float *p)
{
    return guarded([&] {
        check_net(net);
        if (net->model == GN_MODEL_FHN) fail(GN_EINVAL, "the network does not use a spiking node model");
        DeviceGuard dg(net->device);
        sync(net);
        const int32_t N = net->N;
        if (V) {
            std::vector<float> t(N);
            cuda_check(cudaMemcpy(t.data(), net->iz_v.p, N * 4ull, cudaMemcpyDeviceToHost), "D2H V");
            permute_rows_to_caller(net, t.data(), V, 1);
        }
        if (r || p) {
            std::vector<float2> t(N);
            cuda_check(cudaMemcpy(t.data(), net->rp.p, N * 8ull, cudaMemcpyDeviceToHost), "D2H rp");
            for (int32_t i = 0; i < N; ++i) {
                if (r) r[net->perm[i]] = t[i].x;
                if (p) p[net->perm[i]] = t[i].y;
            }
        }
    });
}

gn_status gn_set_izh_state(gn_net *net, const float *V, const float *r, const float *p)
{
    return guarded([&] {
        check_net(net);
        if (net->model == GN_MODEL_FHN) fail(GN_EINVAL, "the network does not use a spiking node model");
        DeviceGuard dg(net->device);
        sync(net);
        const int32_t N = net->N;
        if (V) {
            std::vector<float> t(N);
            for (int32_t j = 0; j < N; ++j) t[net->inv[j]] = V[j];
            cuda_check(cudaMemcpy(net->iz_v.p, t.data(), N * 4ull, cudaMemcpyHostToDevice), "H2D V");
        }
        if (r || p) {
            std::vector<float2> t(N);
            cuda_check(cudaMemcpy(t.data(), net->rp.p, N * 8ull, cudaMemcpyDeviceToHost), "D2H rp");
            for (int32_t j = 0; j < N; ++j) {
                if (r) t[net->inv[j]].x = r[j];
                if (p) t[net->inv[j]].y = p[j];
            }
            cuda_check(cudaMemcpy(net->rp.p, t.data(), N * 8ull, cudaMemcpyHostToDevice), "H2D rp");
        }
    });
}

gn_status gn_get_hh_gates(gn_net *net, float *m, float *n, float *h)
{
    return guarded([&] {
        check_net(net);
        if (net->model != GN_MODEL_HH) fail(GN_EINVAL, "the network does not use the Hodgkin-Huxley model");
        DeviceGuard dg(net->device);
        sync(net);
        const int32_t N = net->N;
        std::vector<float4> t(N);
        cuda_check(cudaMemcpy(t.data(), net->hh_g.p, N * 16ull, cudaMemcpyDeviceToHost), "D2H gates");
        for (int32_t i = 0; i < N; ++i) {
            if (m) m[net->perm[i]] = t[i].x;
            if (n) n[net->perm[i]] = t[i].y;
            if (h) h[net->perm[i]] = t[i].z;
        }
    });
}

gn_status gn_set_hh_gates(gn_net *net, const float *m, const float *n, const float *h)
{
    return guarded([&] {
        check_net(net);
        if (net->model != GN_MODEL_HH) fail(GN_EINVAL, "the network does not use the Hodgkin-Huxley model");
        DeviceGuard dg(net->device);
        sync(net);
        const int32_t N = net->N;
        std::vector<float4> t(N);
        cuda_check(cudaMemcpy(t.data(), net->hh_g.p, N * 16ull, cudaMemcpyDeviceToHost), "D2H gates");
        for (int32_t j = 0; j < N; ++j) {
            float4 &g = t[net->inv[j]];
            if (m) g.x = m[j];
            if (n) g.y = n[j];
            if (h) g.z = h[j];
        }
        cuda_check(cudaMemcpy(net->hh_g.p, t.data(), N * 16ull, cudaMemcpyHostToDevice), "H2D gates");
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
            if (net->stdp)  // the spike bit of a plastic net's ring word
                for (float &x : tmp) {
                    uint32_t word;
                    std::memcpy(&word, &x, 4);
                    x = (word & 1u) ? 1.0f : 0.0f;
                }
            permute_rows_to_caller(net, tmp.data(), out + static_cast<int64_t>(k) * N, 1);
        }
    });
}

namespace {

void check_plastic(const gn_net *net)
{
    if (!net->stdp) fail(GN_EINVAL, "the network does not have plastic weights");
}

}  // namespace

gn_status gn_get_weights(gn_net *net, float *w)
{
    return guarded([&] {
        check_net(net);
        check_plastic(net);
        if (!w) fail(GN_EINVAL, "w is NULL");
        DeviceGuard dg(net->device);
        sync(net);
        std::vector<float> t(net->st_w.n);
        cuda_check(cudaMemcpy(t.data(), net->st_w.p, t.size() * 4, cudaMemcpyDeviceToHost), "D2H weights");
        for (size_t x = 0; x < t.size(); ++x)
            if (net->st_eidx[x] >= 0) w[net->st_eidx[x]] = t[x];
    });
}

gn_status gn_set_weights(gn_net *net, const float *w)
{
    return guarded([&] {
        check_net(net);
        check_plastic(net);
        if (!w) fail(GN_EINVAL, "w is NULL");
        for (int64_t e = 0; e < net->E; ++e)
            if (!std::isfinite(w[e])) fail(GN_EINVAL, "edge %lld: weight not finite", static_cast<long long>(e));
        DeviceGuard dg(net->device);
        sync(net);
        std::vector<float> t(net->st_w.n, 0.0f);
        for (size_t x = 0; x < t.size(); ++x)
            if (net->st_eidx[x] >= 0) t[x] = w[net->st_eidx[x]];
        cuda_check(cudaMemcpy(net->st_w.p, t.data(), t.size() * 4, cudaMemcpyHostToDevice), "H2D weights");
    });
}

gn_status gn_get_stdp_history(gn_net *net, float *s_hist, int32_t depth)
{
    return guarded([&] {
        check_net(net);
        check_plastic(net);
        if (depth < 1 || depth > net->R) fail(GN_EINVAL, "depth must be in [1, ring_depth]");
        if (!s_hist) fail(GN_EINVAL, "s_hist is NULL");
        DeviceGuard dg(net->device);
        sync(net);
        const int32_t N = net->N;
        std::vector<uint32_t> t(N);
        for (int32_t k = 0; k < depth; ++k) {
            const int64_t slot = (net->step - k) & (net->R - 1);
            cuda_check(cudaMemcpy(t.data(), net->ring.p + slot * net->stride, N * 4ull, cudaMemcpyDeviceToHost),
                       "D2H history");
            for (int32_t i = 0; i < N; ++i)
                s_hist[static_cast<int64_t>(k) * N + net->perm[i]] =
                    static_cast<float>(static_cast<double>(t[i] >> 1) * net->dt);
        }
    });
}

gn_status gn_set_stdp_history(gn_net *net, const float *s_hist, int32_t depth)
{
    return guarded([&] {
        check_net(net);
        check_plastic(net);
        if (depth < 1 || depth > net->R) fail(GN_EINVAL, "depth must be in [1, ring_depth]");
        if (!s_hist) fail(GN_EINVAL, "s_hist is NULL");
        const int32_t N = net->N;
        for (int64_t x = 0; x < static_cast<int64_t>(depth) * N; ++x)
            if (!(s_hist[x] >= 0.0f) || !std::isfinite(s_hist[x])) fail(GN_EINVAL, "s must be finite and >= 0");
        DeviceGuard dg(net->device);
        sync(net);
        std::vector<uint32_t> t(N);
        for (int32_t k = 0; k < depth; ++k) {
            const int64_t slot = (net->step - k) & (net->R - 1);
            uint32_t *dev = reinterpret_cast<uint32_t *>(net->ring.p + slot * net->stride);
            cuda_check(cudaMemcpy(t.data(), dev, N * 4ull, cudaMemcpyDeviceToHost), "D2H history");
            for (int32_t j = 0; j < N; ++j) {
                const double steps = std::nearbyint(static_cast<double>(s_hist[static_cast<int64_t>(k) * N + j]) / net->dt);
                const uint32_t kq = static_cast<uint32_t>(std::min(steps, static_cast<double>(gn::kSpikeStepsMax)));
                uint32_t &word = t[net->inv[j]];
                word = (kq << 1) | (word & 1u);
            }
            cuda_check(cudaMemcpy(dev, t.data(), N * 4ull, cudaMemcpyHostToDevice), "H2D history");
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
        // spiking models: V, (r, p); Hodgkin-Huxley also (m, n, h, 0)
        const size_t extra = (net->model != GN_MODEL_FHN ? N * 12 : 0) + (net->model == GN_MODEL_HH ? N * 16 : 0) +
                             (net->stdp ? net->st_w.n * 4 : 0);
        const size_t need = sizeof(CkptHeader) + RS * 4 + N * 8 + N * 4 + N * 8 + extra;
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
        p += N * 8;
        if (extra) {
            cuda_check(cudaMemcpy(p, net->iz_v.p, N * 4, cudaMemcpyDeviceToHost), "D2H V");
            p += N * 4;
            cuda_check(cudaMemcpy(p, net->rp.p, N * 8, cudaMemcpyDeviceToHost), "D2H rp");
            p += N * 8;
            if (net->model == GN_MODEL_HH) {
                cuda_check(cudaMemcpy(p, net->hh_g.p, N * 16, cudaMemcpyDeviceToHost), "D2H gates");
                p += N * 16;
            }
            if (net->stdp) cuda_check(cudaMemcpy(p, net->st_w.p, net->st_w.n * 4, cudaMemcpyDeviceToHost), "D2H weights");
        }
    });
}

gn_status gn_load_state(gn_net *net, const void *buf, size_t size)
{
    return guarded([&] {
        check_net(net);
        if (!buf) fail(GN_EINVAL, "buf is NULL");
        const size_t N = net->N, RS = net->ring.n;
        const size_t extra = (net->model != GN_MODEL_FHN ? N * 12 : 0) + (net->model == GN_MODEL_HH ? N * 16 : 0) +
                             (net->stdp ? net->st_w.n * 4 : 0);
        const size_t need = sizeof(CkptHeader) + RS * 4 + N * 8 + N * 4 + N * 8 + extra;
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
        p += N * 8;
        if (extra) {
            cuda_check(cudaMemcpy(net->iz_v.p, p, N * 4, cudaMemcpyHostToDevice), "H2D V");
            p += N * 4;
            cuda_check(cudaMemcpy(net->rp.p, p, N * 8, cudaMemcpyHostToDevice), "H2D rp");
            p += N * 8;
            if (net->model == GN_MODEL_HH) {
                cuda_check(cudaMemcpy(net->hh_g.p, p, N * 16, cudaMemcpyHostToDevice), "H2D gates");
                p += N * 16;
            }
            if (net->stdp) cuda_check(cudaMemcpy(net->st_w.p, p, net->st_w.n * 4, cudaMemcpyHostToDevice), "H2D weights");
        }
        net->step = h.step;
        net->read_cursor = h.step / net->sample_every;
        cuda_check(cudaMemcpy(net->d_step.p, &h.step, 8, cudaMemcpyHostToDevice), "H2D step");
        if (net->obs_acc.p) cuda_check(cudaMemset(net->obs_acc.p, 0, N * 4), "memset");  // a new frame
        cuda_check(cudaMemset(net->ev_count.p, 0, 8), "memset");
    });
}

}  // extern "C"
