// Host runtime of the batched form (gn_batch_* in include/geonet.h): many
// independent networks in pooled device arrays, advanced together from captured
// graphs by the persistent k_batch or by the staged tile kernel.
//
// gn_batch_create builds every network exactly as gn_net_create does (one FP64
// delay launch for the whole batch, Morton renumbering and the by-target edge list
// per network), then concatenates their arrays into pools; each network's step
// arguments point into the pools.  The work queue is ordered largest first.
//
// Two kernels step a batch: the persistent k_batch (CTAs take whole networks off
// the queue and run every step of them) and the staged form (each member's staged
// layout -- see build_staged -- pooled, one launch per step over every member's
// tiles, steps chained with programmatic dependent launch and replayed from a
// graph).  Both sum a node's inputs in the order every step kernel uses, so the
// choice never changes a result.  The first gn_batch_step picks the kernel (and
// k_batch's CTA size) by timing the candidates on a scratch copy of the dynamic
// state; GN_BATCH_KERNEL=1 or 3 restricts the choice to k_batch or the staged form
// (4: the staged form with L2 blocking, below).
//
// L2 blocking of the staged form.  When the members' per-step working set (edge
// entries, gather keys, live history slots, node state) outgrows L2, every step
// re-reads it from DRAM.  The members are then cut into contiguous groups, and a
// graph chunk runs each group's steps back to back: members are independent, so a
// group may run ahead of the others within the chunk, and after the chunk's first
// step a group's steps read its data from L2.  A group smaller than a wave of CTAs
// leaves SMs idle between its steps, so 1, 2 or 4 groups run at once (lanes), each
// lane a chain of launches on its own stream; the groups in flight share the L2
// budget.  The launches are the same kernel over a group's tiles (its members'
// tile pointers start at the group's first tile), so grouping never changes a
// result either; the first gn_batch_step times the schedules with the other
// candidates.  The lanes schedule runs the same groups in one cooperative launch
// per chunk (k_batch_lanes): lanes of CTAs instead of launch chains, a counting
// barrier in global memory instead of each launch boundary.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "runtime.h"

using gnrt::cuda_check;
using gnrt::DevArray;
using gnrt::DeviceGuard;
using gnrt::fail;
using gnrt::guarded;

namespace {

constexpr int kGraphSteps = 64;             // staged form: steps per captured graph
constexpr int kStaged = gn::kNumBatchShapes;  // shape index of the staged form
constexpr int kLanes = kStaged + 1;            // ... and of its persistent lanes schedule (k_batch_lanes)
// per-step working set of a member beyond its edge structure, per node: the live
// history slots (max delay + 2, 4 bytes each) come on top of these node-state bytes
// (w and readout 8, background counter 4, arrival step 8, caller id 4, sample 4)
constexpr double kNodeStateBytes = 28.0;
constexpr double kDefaultGroupBytes = 80e6;  // L2 budget of the groups stepped at once (L2 is 126 MB)

// One group of the staged form's L2 blocking: tiles [t0, t0 + nt) of the pool.
struct StGroup {
    int t0 = 0, nt = 0;
    bool first = false;  // its grid outnumbers the resident CTAs: launch the next grid first
};

// Host view of one member network.
struct Member {
    int32_t N = 0;
    int64_t E = 0;
    int32_t R = 0, stride = 0, dmax = 0, dmin = 0;
    int64_t n_clamped = 0;
    bool packed = true;
    double v_rest = 0.0, w_rest = 0.0, dt = 0.0;
    int32_t sample_every = 1;
    int64_t node_off = 0, ring_off = 0, edge_off = 0, keyw_off = 0, rp_off = 0, obs_off = 0, ev_off = 0;
    int64_t ev_cap = 0, pulse_off = 0, pulse_cap = 0, read_cursor = 0;
    int64_t desc_off[gn::kNumBatchShapes] = {};
    int32_t st_t0 = 0, st_nt = 0;  // staged form: the member's tiles in the pool
    double st_bytes = 0.0;         // ... and the bytes of its entries and gather keys
    int32_t n_blocks[gn::kNumBatchShapes] = {};
    std::vector<int32_t> perm, inv, delay;
};

}  // namespace

struct gn_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int32_t n_nets = 0;
    int64_t obs_cap = 0;
    int64_t step = 0;
    int shape = -1;  // -1: autotune on the first step
    int grid = 0;
    size_t bytes = 0;
    std::vector<Member> m;
    std::vector<gn::StepArgs> args;  // host copy, shape-independent fields
    std::vector<int32_t> order;      // largest first
    DevArray<uint8_t> ekey;
    DevArray<float> ew, ring, bias, obs, p_amp;
    DevArray<float2> wc;
    DevArray<int32_t> row_ptr, bgc, perm, ev_node, p_node, npulses, d_order, queue;
    DevArray<int64_t> first, ev_step, p_on, p_off, d_step;
    DevArray<unsigned long long> ev_count;
    DevArray<unsigned int> status;
    DevArray<int4> bdesc[gn::kNumBatchShapes];
    DevArray<gn::StepArgs> d_args;
    cudaGraphExec_t graph = nullptr;
    int64_t graph_steps = 0;
    // staged form: pooled layouts of every member (tile_net: member of each tile)
    bool staged_ok = false, st_packed = true, st_stream = false;
    bool st_big = false;      // the ungrouped structure outgrows L2: stream it with evict-first loads
    std::vector<StGroup> st_groups;  // chosen schedule: one group of every tile, or L2-sized groups
    int st_lanes = 1;                // groups stepped concurrently, one chain of launches per lane
    std::vector<cudaStream_t> lane_stream;  // lanes 1, 2, ... (lane 0 runs on the batch's stream)
    std::vector<cudaEvent_t> lane_event;    // fork, then one join per extra lane
    DevArray<int2> st_gtab;                 // lanes schedule: {first tile, tiles} of each group
    DevArray<unsigned int> lane_count;      // ... and the lanes' barrier counters (32 words each)
    int n_tiles = 0;
    size_t st_smem = 0;
    DevArray<int4> st_tile, st_tile2;
    DevArray<uint32_t> st_ukey;
    DevArray<int2> st_slice;
    DevArray<float> st_w;
    DevArray<uint16_t> st_u, st_plist;
    DevArray<int32_t> st_rq, st_tile_net;
    // node model shared by every member; spiking members' V, (r, p), gates
    int32_t model = GN_MODEL_FHN;
    std::vector<uint8_t> hetero;  // members with cell types
    DevArray<float> iz_v;
    DevArray<float2> rp;
    DevArray<float4> hh_g;
    DevArray<float> obs_acc;  // frame sums of the readout state (members with frame averaging)
    DevArray<uint8_t> cell;   // heterogeneous members: each node's parameter set
    DevArray<float> type_par; // ... and each member's rows (kMaxCellTypes rows per member)

    ~gn_batch()
    {
        if (graph) cudaGraphExecDestroy(graph);
        ekey.release();
        for (auto *a : {&ew, &ring, &bias, &obs, &p_amp}) a->release();
        wc.release();
        for (auto *a : {&row_ptr, &bgc, &perm, &ev_node, &p_node, &npulses, &d_order, &queue}) a->release();
        for (auto *a : {&first, &ev_step, &p_on, &p_off, &d_step}) a->release();
        ev_count.release();
        status.release();
        for (auto &a : bdesc) a.release();
        d_args.release();
        st_tile.release();
        st_tile2.release();
        st_ukey.release();
        st_slice.release();
        st_w.release();
        st_u.release();
        st_plist.release();
        st_rq.release();
        st_tile_net.release();
        st_gtab.release();
        lane_count.release();
        iz_v.release();
        rp.release();
        hh_g.release();
        obs_acc.release();
        cell.release();
        type_par.release();
        for (cudaStream_t x : lane_stream) cudaStreamDestroy(x);
        for (cudaEvent_t x : lane_event) cudaEventDestroy(x);
        if (own_stream && stream) cudaStreamDestroy(stream);
    }
};

namespace {

void check_batch(const gn_batch *b, int32_t net = 0)
{
    if (!b) fail(GN_EINVAL, "batch handle is NULL");
    if (net < 0 || net >= b->n_nets) fail(GN_EINVAL, "network index %d out of range", net);
}

void sync(gn_batch *b)
{
    cuda_check(cudaStreamSynchronize(b->stream), "kernel execution");
    unsigned int st = 0;
    cuda_check(cudaMemcpy(&st, b->status.p, 4, cudaMemcpyDeviceToHost), "D2H status");
    if (st) {
        cudaMemset(b->status.p, 0, 4);
        fail(st & gn::kStatusTimeout ? GN_ETIMEOUT : GN_EINTERNAL, "device status word %u", st);
    }
}

// The block-descriptor shape of the step arguments: the persistent kernel's chosen
// CTA size, else the first (the staged form reads no block descriptors).
int desc_shape(const gn_batch *b) { return b->shape >= 0 && b->shape < gn::kNumBatchShapes ? b->shape : 0; }

// Step arguments for a CTA shape (block descriptors differ per shape) and a staged
// schedule: a member's tile pointers start at its group's first tile, the tile its
// group's launches number 0.
std::vector<gn::StepArgs> args_for(const gn_batch *b, int shape, const std::vector<StGroup> &groups)
{
    std::vector<gn::StepArgs> out = b->args;
    size_t g = 0;
    for (int i = 0; i < b->n_nets; ++i) {
        out[i].bdesc = b->bdesc[shape].p + b->m[i].desc_off[shape];
        out[i].n_blocks = b->m[i].n_blocks[shape];
        if (!b->staged_ok) continue;
        while (g + 1 < groups.size() && b->m[i].st_t0 >= groups[g + 1].t0) ++g;
        const int t0 = groups.empty() ? 0 : groups[g].t0;
        out[i].st_tile = b->st_tile.p + t0;
        out[i].st_tile2 = b->st_tile2.p + t0;
    }
    return out;
}

void upload_args(gn_batch *b)
{
    const std::vector<gn::StepArgs> a = args_for(b, desc_shape(b), b->st_groups);
    cuda_check(cudaMemcpy(b->d_args.p, a.data(), a.size() * sizeof(gn::StepArgs), cudaMemcpyHostToDevice), "H2D args");
}

// L2 budget in bytes of the groups stepped at once (each of `lanes` groups takes
// an equal share): GN_BATCH_GROUP_KB in the environment (0 turns the L2 blocking
// off), else kDefaultGroupBytes.
double group_budget()
{
    const char *e = getenv("GN_BATCH_GROUP_KB");
    if (e && *e) return std::max(0.0, atof(e)) * 1024.0;
    return kDefaultGroupBytes;
}

// Lanes fixed by GN_BATCH_LANES in the environment (1 to 8), else 0.
int lanes_env()
{
    const char *e = getenv("GN_BATCH_LANES");
    if (!e || !*e) return 0;
    const int l = atoi(e);
    if (l < 1 || l > 8) fail(GN_EINVAL, "GN_BATCH_LANES must be 1 to 8");
    return l;
}

// Contiguous groups of members whose per-step working sets fit `budget` bytes
// (a member larger than the budget is a group of its own); one group of every tile
// when budget <= 0.
std::vector<StGroup> make_groups(const gn_batch *b, double budget)
{
    std::vector<StGroup> g;
    double acc = 0.0;
    int t0 = 0;
    for (const Member &mm : b->m) {
        const double live = std::min(mm.R, mm.dmax + 2);
        const double ws = mm.st_bytes + static_cast<double>(mm.N) * (4.0 * live + kNodeStateBytes);
        if (budget > 0.0 && acc > 0.0 && acc + ws > budget && mm.st_t0 > t0) {
            g.push_back({t0, mm.st_t0 - t0, false});
            t0 = mm.st_t0;
            acc = 0.0;
        }
        acc += ws;
    }
    if (b->n_tiles > t0) g.push_back({t0, b->n_tiles - t0, false});
    return g;
}

// Prepare the staged kernel for the batch's format and stream setting and mark the
// groups whose grid outnumbers the CTAs the device holds at once (those launch the
// next grid first; GN_STAGED_EARLY=0 turns that off).
void prepare_staged(gn_batch *b, std::vector<StGroup> &groups)
{
    int per_sm = 0, sms = 0;
    cuda_check(gn::batch_staged_prepare(b->model, b->st_packed, b->st_stream, b->st_smem, &per_sm),
               "staged kernel setup");
    cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device), "device query");
    const char *e = getenv("GN_STAGED_EARLY");
    const bool off = e && *e == '0';
    for (StGroup &g : groups)
        g.first = !off && per_sm > 0 && static_cast<int64_t>(g.nt) > static_cast<int64_t>(per_sm) * sms;
}

void drop_graph(gn_batch *b)
{
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
}

// Streams and events of `lanes` concurrent chains (created once, kept until the
// batch is destroyed).
void ensure_lanes(gn_batch *b, int lanes)
{
    while (static_cast<int>(b->lane_stream.size()) < lanes - 1) {
        cudaStream_t x = nullptr;
        cuda_check(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking), "cudaStreamCreate");
        b->lane_stream.push_back(x);
    }
    while (static_cast<int>(b->lane_event.size()) < lanes) {
        cudaEvent_t x = nullptr;
        cuda_check(cudaEventCreateWithFlags(&x, cudaEventDisableTiming), "cudaEventCreate");
        b->lane_event.push_back(x);
    }
}

// The lanes schedule: its kernel prepared for the batch's format; returns its
// cooperative grid (every CTA the device holds at once).
// GN_BATCH_LANE_CTAS=k in the environment holds it to k CTAs per SM.
int lanes_grid(gn_batch *b)
{
    int per_sm = 0, sms = 0;
    cuda_check(gn::batch_lanes_prepare(b->model, b->st_packed, b->st_smem, &per_sm), "lanes kernel setup");
    cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device), "device query");
    if (const char *e = getenv("GN_BATCH_LANE_CTAS"); e && *e) per_sm = std::min(per_sm, std::max(1, atoi(e)));
    if (per_sm < 1) fail(GN_ECUDA, "the lanes kernel does not fit on an SM");
    if (!b->lane_count.p) b->lane_count.alloc(gn::kLaneWords * gn::kMaxBatchLanes, &b->bytes);
    return per_sm * sms;
}

void upload_groups(const std::vector<StGroup> &groups, DevArray<int2> &out, size_t *bytes)
{
    std::vector<int2> t;
    for (const StGroup &g : groups) t.push_back(make_int2(g.t0, g.nt));
    out.release();
    out.upload(t, bytes);
}

// Steps 0 .. n - 1 of the lanes schedule over `gtab` (n_groups groups): the barrier
// counters cleared, then one cooperative launch in min(lanes, n_groups) lanes.
cudaError_t launch_lanes(const gn_batch *b, const gn::StepArgs *args, const int2 *gtab, int n_groups, int lanes,
                         int grid, int n, cudaStream_t s)
{
    lanes = std::max(1, std::min(lanes, n_groups));
    cudaError_t e = cudaMemsetAsync(b->lane_count.p, 0, b->lane_count.n * sizeof(unsigned int), s);
    if (e == cudaSuccess)
        e = gn::launch_batch_lanes(b->model, args, b->st_tile_net.p, gtab, n_groups, lanes, n, b->lane_count.p,
                                   b->status.p, b->args[0].wait_limit, b->st_packed, grid, b->st_smem, s);
    return e;
}

void set_shape(gn_batch *b, int shape, bool grouped, int lanes)
{
    if (shape == kLanes) {
        b->st_stream = false;
        b->st_groups = make_groups(b, group_budget() / lanes);
        b->st_lanes = lanes;
        b->grid = lanes_grid(b);
        upload_groups(b->st_groups, b->st_gtab, &b->bytes);
        b->shape = kLanes;
        upload_args(b);
        drop_graph(b);
        return;
    }
    if (shape == kStaged) {
        // grouped members keep their structure in L2 across the chunk; otherwise a
        // structure larger than L2 is streamed past the history
        b->st_stream = grouped ? false : b->st_big;
        b->st_groups = make_groups(b, grouped ? group_budget() / lanes : 0.0);
        b->st_lanes = grouped ? lanes : 1;
        ensure_lanes(b, b->st_lanes);
        prepare_staged(b, b->st_groups);
        b->shape = kStaged;
        b->grid = b->n_tiles;
        upload_args(b);
        drop_graph(b);
        return;
    }
    int per_sm = 0, sms = 0;
    cuda_check(gn::batch_occupancy(shape, &per_sm), "occupancy");
    cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device), "device query");
    if (per_sm < 1) fail(GN_ECUDA, "the batch kernel does not fit on an SM");
    b->shape = shape;
    b->grid = std::max(1, std::min(b->n_nets, per_sm * sms));
    b->st_groups.clear();
    b->st_lanes = 1;
    upload_args(b);
    drop_graph(b);
}

// Steps k0 .. k0 + n - 1 of the staged form.  Group g runs in lane g % lanes; a
// lane steps its groups one after another, each through all n steps, as one chain
// of launches on its own stream (lane 0 on s, the others forked from s and joined
// back into it).  Lanes touch disjoint members, so they need no ordering.
cudaError_t launch_staged(const gn_batch *b, const gn::StepArgs *args, const std::vector<StGroup> &groups, int lanes,
                          int k0, int n, cudaStream_t s)
{
    lanes = std::max(1, std::min(lanes, static_cast<int>(groups.size())));
    cudaError_t e = cudaSuccess;
    if (lanes > 1) {
        e = cudaEventRecord(b->lane_event[0], s);
        for (int l = 1; l < lanes && e == cudaSuccess; ++l) e = cudaStreamWaitEvent(b->lane_stream[l - 1], b->lane_event[0], 0);
    }
    for (int l = 0; l < lanes && e == cudaSuccess; ++l) {
        cudaStream_t ls = l == 0 ? s : b->lane_stream[l - 1];
        for (size_t gi = l; gi < groups.size() && e == cudaSuccess; gi += lanes) {
            const StGroup &g = groups[gi];
            for (int k = k0; k < k0 + n && e == cudaSuccess; ++k)
                e = gn::launch_batch_staged(b->model, args, b->st_tile_net.p + g.t0, g.nt, k, b->st_packed,
                                            b->st_stream, b->st_smem, g.first, ls);
        }
    }
    for (int l = 1; l < lanes && e == cudaSuccess; ++l) {
        e = cudaEventRecord(b->lane_event[l], b->lane_stream[l - 1]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->lane_event[l], 0);
    }
    return e;
}

void launch_steps(gn_batch *b, const gn::StepArgs *args, int64_t *d_step, int n_steps, int shape, int grid,
                  const std::vector<StGroup> &groups, int lanes, cudaStream_t s, const int2 *gtab = nullptr)
{
    if (shape == kStaged) {
        cuda_check(launch_staged(b, args, groups, lanes, 0, n_steps, s), "staged batch launch");
        return;
    }
    if (shape == kLanes) {
        cuda_check(launch_lanes(b, args, gtab, static_cast<int>(groups.size()), lanes, grid, n_steps, s),
                   "lanes batch launch");
        return;
    }
    cuda_check(cudaMemsetAsync(b->queue.p, 0, 4, s), "queue reset");
    cuda_check(gn::launch_batch(args, b->d_order.p, b->n_nets, b->queue.p, d_step, n_steps, shape, grid, s),
               "batch launch");
}

// An executable graph of the launches `body` issues on a capturing stream.
template <class F>
cudaGraphExec_t capture_graph(F &&body)
{
    cudaStream_t cs;
    cuda_check(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking), "cudaStreamCreate");
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        e = body(cs);
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cuda_check(e, "graph capture of the batch step");
    return ge;
}

// Time each candidate (k_batch in each CTA shape, the staged form with and without
// L2 blocking, the lanes schedule in 1 to 8 lanes) per step on a scratch copy of
// the dynamic state: k_batch over 16 steps in one launch, the staged form over one
// graph chunk replayed from a graph as gn_batch_step runs it (a chunk of many
// small groups issues thousands of launches, which direct launches would time as
// host work).  A single candidate is taken untimed.  A lanes candidate that cannot
// be launched (a cooperative launch refused) is left out.
void autotune(gn_batch *b, bool persistent, bool staged, bool lanes_ok)
{
    struct Cand {
        int shape;
        bool grouped;
        int lanes;
    };
    std::vector<Cand> cands;
    if (persistent)
        for (int shape = 0; shape < gn::kNumBatchShapes; ++shape) cands.push_back({shape, false, 1});
    if (staged && b->staged_ok) {
        cands.push_back({kStaged, false, 1});
        const int fixed = lanes_env();
        for (int lanes : {1, 2, 4})
            if ((!fixed || lanes == fixed) && make_groups(b, group_budget() / lanes).size() > 1)
                cands.push_back({kStaged, true, lanes});
        if (lanes_ok)
            for (int lanes : {1, 2, 4, 8})
                if ((!fixed || lanes == fixed) &&
                    (lanes == 1 || static_cast<int>(make_groups(b, group_budget() / lanes).size()) >= lanes))
                    cands.push_back({kLanes, true, lanes});
    }
    if (cands.empty()) fail(GN_EINVAL, "no batch kernel can step this batch");
    if (cands.size() == 1) {
        set_shape(b, cands[0].shape, cands[0].grouped, cands[0].lanes);
        return;
    }
    size_t tmp = 0;
    DevArray<float> ring, obs, facc, izv;
    DevArray<float2> wc, rpv;
    DevArray<float4> hhg;
    DevArray<int32_t> bgc, evn;
    DevArray<int64_t> first, evs, dstep;
    DevArray<unsigned long long> evc;
    DevArray<gn::StepArgs> dargs;
    DevArray<int2> gtab;
    cudaEvent_t t0 = nullptr, t1 = nullptr;
    auto cleanup = [&] {
        gtab.release();
        ring.release(); obs.release(); wc.release(); bgc.release(); evn.release(); first.release();
        evs.release(); dstep.release(); evc.release(); dargs.release(); facc.release();
        izv.release(); rpv.release(); hhg.release();
        if (t0) cudaEventDestroy(t0);
        if (t1) cudaEventDestroy(t1);
    };
    Cand best = cands[0];
    try {
        int64_t total_nodes = 0;
        for (const Member &mm : b->m) total_nodes += mm.N;
        ring.alloc(b->ring.n, &tmp);
        wc.alloc(b->wc.n, &tmp);
        bgc.alloc(total_nodes, &tmp);
        first.alloc(total_nodes, &tmp);
        obs.alloc(total_nodes, &tmp);
        evn.alloc(b->n_nets, &tmp);
        evs.alloc(b->n_nets, &tmp);
        evc.alloc(b->n_nets, &tmp);
        dstep.alloc(1, &tmp);
        dargs.alloc(b->n_nets, &tmp);
        if (b->obs_acc.p) {
            facc.alloc(total_nodes, &tmp);
            cuda_check(cudaMemset(facc.p, 0, facc.n * 4), "memset");
        }
        cuda_check(cudaMemset(ring.p, 0, ring.n * 4), "memset");
        cuda_check(cudaMemset(wc.p, 0, wc.n * 8), "memset");
        cuda_check(cudaMemset(bgc.p, 0, bgc.n * 4), "memset");
        cuda_check(cudaMemset(first.p, 0xff, first.n * 8), "memset");
        cuda_check(cudaMemset(evc.p, 0, evc.n * 8), "memset");
        if (b->model != GN_MODEL_FHN) {  // spiking state, copied so the candidates step a live network
            izv.alloc(b->iz_v.n, &tmp);
            rpv.alloc(b->rp.n, &tmp);
            cuda_check(cudaMemcpy(izv.p, b->iz_v.p, izv.n * 4, cudaMemcpyDeviceToDevice), "D2D");
            cuda_check(cudaMemcpy(rpv.p, b->rp.p, rpv.n * 8, cudaMemcpyDeviceToDevice), "D2D");
            if (b->hh_g.p) {
                hhg.alloc(b->hh_g.n, &tmp);
                cuda_check(cudaMemcpy(hhg.p, b->hh_g.p, hhg.n * 16, cudaMemcpyDeviceToDevice), "D2D");
            }
        }
        cuda_check(cudaMemcpy(dstep.p, &b->step, 8, cudaMemcpyHostToDevice), "H2D");
        cuda_check(cudaEventCreate(&t0), "event");
        cuda_check(cudaEventCreate(&t1), "event");
        float best_ms = 1e30f;
        for (const Cand &c : cands) {
            std::vector<StGroup> groups;
            int grid = b->n_tiles, steps = 16;
            if (c.shape == kStaged) {
                b->st_stream = c.grouped ? false : b->st_big;
                groups = make_groups(b, c.grouped ? group_budget() / c.lanes : 0.0);
                prepare_staged(b, groups);
                ensure_lanes(b, c.lanes);
                steps = kGraphSteps;
            } else if (c.shape == kLanes) {
                b->st_stream = false;
                groups = make_groups(b, group_budget() / c.lanes);
                grid = lanes_grid(b);
                upload_groups(groups, gtab, &tmp);
                steps = kGraphSteps;
            } else {
                int per_sm = 0, sms = 0;
                cuda_check(gn::batch_occupancy(c.shape, &per_sm), "occupancy");
                cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device), "device query");
                grid = std::max(1, std::min(b->n_nets, per_sm * sms));
            }
            std::vector<gn::StepArgs> a = args_for(b, c.shape >= kStaged ? 0 : c.shape, groups);
            for (int i = 0; i < b->n_nets; ++i) {
                const Member &mm = b->m[i];
                a[i].ring = ring.p + mm.ring_off;
                a[i].wc = wc.p + mm.node_off + 2 * i;
                a[i].bgc = bgc.p + mm.node_off;
                a[i].first = first.p + mm.node_off;
                a[i].obs = obs.p + mm.node_off;
                a[i].obs_cap = 1;
                a[i].ev_node = evn.p + i;
                a[i].ev_step = evs.p + i;
                a[i].ev_count = evc.p + i;
                a[i].ev_cap = 1;
                if (a[i].obs_acc) a[i].obs_acc = facc.p + mm.node_off;
                if (izv.p) {
                    a[i].iz_v = izv.p + mm.node_off;
                    a[i].rp = rpv.p + mm.node_off;
                    if (hhg.p) a[i].hh_g = hhg.p + mm.node_off;
                }
            }
            cuda_check(cudaMemcpy(dargs.p, a.data(), a.size() * sizeof(gn::StepArgs), cudaMemcpyHostToDevice), "H2D");
            cudaGraphExec_t ge = nullptr;
            if (c.shape == kLanes) {
                // direct launches, as gn_batch_step issues them (one per chunk)
                const cudaError_t e =
                    launch_lanes(b, dargs.p, gtab.p, static_cast<int>(groups.size()), c.lanes, grid, steps, b->stream);
                if (e != cudaSuccess) {  // a cooperative launch the device refuses
                    cudaGetLastError();
                    continue;
                }
            } else if (c.shape == kStaged) {
                ge = capture_graph([&](cudaStream_t cs) {
                    return launch_staged(b, dargs.p, groups, c.lanes, 0, steps, cs);
                });
                const cudaError_t e = cudaGraphLaunch(ge, b->stream);  // warm-up
                if (e != cudaSuccess) cudaGraphExecDestroy(ge);
                cuda_check(e, "cudaGraphLaunch");
            } else {
                launch_steps(b, dargs.p, dstep.p, 2, c.shape, grid, groups, c.lanes, b->stream);
            }
            cudaError_t e = cudaEventRecord(t0, b->stream);
            if (e == cudaSuccess) {
                if (ge)
                    e = cudaGraphLaunch(ge, b->stream);
                else if (c.shape == kLanes)
                    e = launch_lanes(b, dargs.p, gtab.p, static_cast<int>(groups.size()), c.lanes, grid, steps,
                                     b->stream);
                else
                    launch_steps(b, dargs.p, dstep.p, steps, c.shape, grid, groups, c.lanes, b->stream);
            }
            if (e == cudaSuccess) e = cudaEventRecord(t1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            if (ge) cudaGraphExecDestroy(ge);
            cuda_check(e, "autotune");
            float ms = 0.0f;
            cuda_check(cudaEventElapsedTime(&ms, t0, t1), "event");
            if (ms / steps < best_ms) {
                best_ms = ms / steps;
                best = c;
            }
        }
    } catch (...) {
        cleanup();
        throw;
    }
    cleanup();
    set_shape(b, best.shape, best.grouped, best.lanes);
}

void build_graph(gn_batch *b, int64_t n_steps)
{
    drop_graph(b);
    b->graph = capture_graph([&](cudaStream_t cs) {
        cudaError_t e;
        if (b->shape == kStaged) {
            e = launch_staged(b, b->d_args.p, b->st_groups, b->st_lanes, 0, static_cast<int>(n_steps), cs);
        } else {
            e = cudaMemsetAsync(b->queue.p, 0, 4, cs);
            if (e == cudaSuccess)
                e = gn::launch_batch(b->d_args.p, b->d_order.p, b->n_nets, b->queue.p, b->d_step.p,
                                     static_cast<int>(n_steps), b->shape, b->grid, cs);
        }
        if (e == cudaSuccess) e = gn::launch_advance(b->d_step.p, n_steps, cs);
        return e;
    });
    b->graph_steps = n_steps;
}

// Staged layouts of every member, pooled: tile descriptors point into the pools,
// each member's row piece lists keep member-local rows (its args point at its part
// of st_rq).  Sets b->staged_ok (false if a member's layout does not fit or the
// members mix edge formats) and returns each member's offset into st_rq.
std::vector<int64_t> build_staged_pool(gn_batch *b, const std::vector<gnrt::HostNet> &hs)
{
    const int n = static_cast<int>(hs.size());
    std::vector<int64_t> rq_off(n, 0);
    b->staged_ok = true;
    b->st_packed = hs[0].packed;
    for (const gnrt::HostNet &h : hs) b->staged_ok = b->staged_ok && h.packed == b->st_packed;
    if (!b->staged_ok) return rq_off;
    const gn::StagedShape sh = gn::kBatchStagedShape;
    const int kw = b->st_packed ? 1 : 2;
    std::vector<int4> tile, tile2;
    std::vector<uint32_t> ukey;
    std::vector<int2> slice;
    std::vector<float> w;
    std::vector<uint16_t> u, plist;
    std::vector<int32_t> rq, tile_net;
    int max_u = 0, max_x = 0, max_p = 0;
    for (int i = 0; i < n; ++i) {
        gnrt::StagedLayout L;
        if (!gnrt::build_staged(hs[i], sh.threads, sh.ucap, sh.ecap, sh.pcap, L)) {
            b->staged_ok = false;
            return rq_off;
        }
        while (w.size() % 32) {  // tile entry blocks stay 128-byte aligned
            w.push_back(0.0f);
            u.push_back(0);
        }
        const int64_t u_off = static_cast<int64_t>(ukey.size()) / kw, s_off = static_cast<int64_t>(slice.size());
        const int64_t x_off = static_cast<int64_t>(w.size()), q_off = static_cast<int64_t>(plist.size());
        if (x_off + static_cast<int64_t>(L.w.size()) >= (1ll << 31) || u_off + static_cast<int64_t>(L.ukey.size()) >= (1ll << 31)) {
            b->staged_ok = false;
            return rq_off;
        }
        b->m[i].st_t0 = static_cast<int32_t>(tile.size());
        b->m[i].st_nt = static_cast<int32_t>(L.tile.size());
        b->m[i].st_bytes = static_cast<double>(L.w.size()) * 6.0 + static_cast<double>(L.ukey.size()) * 4.0;
        for (size_t t = 0; t < L.tile.size(); ++t) {
            int4 a = L.tile[t], c = L.tile2[t];
            a.z += static_cast<int>(u_off);
            c.x += static_cast<int>(s_off);
            c.z += static_cast<int>(x_off);
            tile.push_back(a);
            tile2.push_back(c);
            tile_net.push_back(i);
        }
        ukey.insert(ukey.end(), L.ukey.begin(), L.ukey.end());
        slice.insert(slice.end(), L.slice.begin(), L.slice.end());
        w.insert(w.end(), L.w.begin(), L.w.end());
        u.insert(u.end(), L.u.begin(), L.u.end());
        plist.insert(plist.end(), L.plist.begin(), L.plist.end());
        rq_off[i] = static_cast<int64_t>(rq.size());
        for (int32_t q : L.rq) rq.push_back(static_cast<int32_t>(q + q_off));
        max_u = std::max(max_u, L.max_u);
        max_x = std::max(max_x, L.max_x);
        max_p = std::max(max_p, L.max_p);
    }
    int max_smem = 0;
    cuda_check(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, b->device), "device query");
    b->st_smem = 16 + static_cast<size_t>(max_u) * (b->st_packed ? 4 : 12) + static_cast<size_t>(max_p) * 4;
    if (b->st_smem > static_cast<size_t>(max_smem)) {
        b->staged_ok = false;
        return rq_off;
    }
    b->st_big = static_cast<double>(w.size()) * 6.0 + static_cast<double>(ukey.size()) * 4.0 > 48e6;
    b->st_stream = b->st_big;
    b->n_tiles = static_cast<int>(tile.size());
    b->st_tile.upload(tile, &b->bytes);
    b->st_tile2.upload(tile2, &b->bytes);
    b->st_ukey.upload(ukey, &b->bytes);
    b->st_slice.upload(slice, &b->bytes);
    b->st_w.upload(w, &b->bytes);
    b->st_u.upload(u, &b->bytes);
    b->st_plist.upload(plist, &b->bytes);
    b->st_rq.upload(rq, &b->bytes);
    b->st_tile_net.upload(tile_net, &b->bytes);
    for (int i = 0; i < n; ++i) {
        b->args[i].st_ucap = max_u;
        b->args[i].st_xcap = max_x;
    }
    return rq_off;
}

template <class T>
void to_caller(const Member &mm, const T *internal, T *out)
{
    for (int32_t r = 0; r < mm.N; ++r) out[mm.perm[r]] = internal[r];
}

}  // namespace

extern "C" {

gn_status gn_batch_create(const gn_net_desc *descs, int32_t n_nets, gn_batch **out)
{
    if (!out) {
        gnrt::set_error("out is NULL");
        return GN_EINVAL;
    }
    *out = nullptr;
    gn_batch *b = nullptr;
    gn_status st = guarded([&] {
        if (!descs || n_nets <= 0) fail(GN_EINVAL, "need at least one network");
        for (int i = 0; i < n_nets; ++i) {
            gnrt::validate_desc(descs + i);
            if (descs[i].device != descs[0].device) fail(GN_EINVAL, "all networks of a batch share one device");
            if (descs[i].model != descs[0].model) fail(GN_EINVAL, "every network of a batch uses one node model");
            if (descs[i].stdp.enable) fail(GN_EINVAL, "the batched form does not take plastic weights");
        }
        b = new gn_batch();
        b->device = descs[0].device;
        b->n_nets = n_nets;
        b->model = descs[0].model;
        DeviceGuard dg(b->device);
        if (descs[0].cuda_stream) {
            b->stream = static_cast<cudaStream_t>(descs[0].cuda_stream);
        } else {
            cuda_check(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking), "cudaStreamCreate");
            b->own_stream = true;
        }
        std::vector<std::vector<int32_t>> delays;
        std::vector<int64_t> clamped;
        gnrt::quantise_delays(descs, n_nets, b->stream, delays, clamped);

        // host build of every member, then pooled layout
        b->m.resize(n_nets);
        b->args.resize(n_nets);
        std::vector<gnrt::HostNet> hs(n_nets);
        int64_t nodes = 0, ring = 0, keyw = 0, edges = 0, rp = 0, obs = 0, ev = 0;
        int64_t descs_n[gn::kNumBatchShapes] = {};
        b->obs_cap = descs[0].obs_capacity > 0 ? descs[0].obs_capacity : 256;
        std::vector<std::vector<int4>> shape_desc(gn::kNumBatchShapes);
        for (int i = 0; i < n_nets; ++i) {
            gnrt::HostNet &h = hs[i];
            const int cap0 = gn::batch_block_cap(0);
            gnrt::host_build(descs + i, std::move(delays[i]), clamped[i], cap0, gn::kBatchThreads[0], h);
            Member &mm = b->m[i];
            mm.N = h.N;
            mm.E = h.E;
            mm.R = h.R;
            mm.stride = h.stride;
            mm.dmax = h.dmax;
            mm.dmin = h.dmin;
            mm.n_clamped = h.n_clamped;
            mm.packed = h.packed;
            mm.v_rest = h.v_rest;
            mm.w_rest = h.w_rest;
            mm.dt = descs[i].dt_ms;
            mm.sample_every = descs[i].obs.sample_every;
            mm.perm = h.perm;
            mm.inv = h.inv;
            mm.delay = h.delay;
            mm.node_off = nodes;
            mm.ring_off = ring;
            mm.keyw_off = keyw;
            mm.edge_off = edges;
            mm.rp_off = rp;
            mm.obs_off = obs;
            mm.ev_off = ev;
            mm.ev_cap = std::max<int64_t>(1024, 8 * static_cast<int64_t>(h.N));
            for (int s = 0; s < gn::kNumBatchShapes; ++s) {
                std::vector<int32_t> blk;
                std::vector<int4> d;
                gnrt::make_blocks(h.row_ptr, h.N, gn::batch_block_cap(s), gn::kBatchThreads[s], blk, d);
                mm.desc_off[s] = descs_n[s];
                mm.n_blocks[s] = static_cast<int32_t>(d.size());
                descs_n[s] += static_cast<int64_t>(d.size());
                shape_desc[s].insert(shape_desc[s].end(), d.begin(), d.end());
            }
            nodes += h.N;
            ring += static_cast<int64_t>(h.R) * h.stride;
            // every network's key bytes and weights start on a 256-byte boundary
            // (the kernel reads them with 16-byte vector loads)
            keyw += (static_cast<int64_t>(h.key.size()) * 4 + 255) / 256 * 256;
            edges += (static_cast<int64_t>(h.w.size()) + 63) / 64 * 64;
            rp += static_cast<int64_t>(h.row_ptr.size());
            obs += b->obs_cap * h.N;
            ev += mm.ev_cap;
            gnrt::fill_step_params(descs + i, h, b->args[i]);
        }
        // pools
        b->ekey.alloc(keyw, &b->bytes);
        b->ew.alloc(edges, &b->bytes);
        b->row_ptr.alloc(rp, &b->bytes);
        b->perm.alloc(nodes, &b->bytes);
        for (int i = 0; i < n_nets; ++i) {
            const gnrt::HostNet &h = hs[i];
            const Member &mm = b->m[i];
            cuda_check(cudaMemcpy(b->ekey.p + mm.keyw_off, h.key.data(), h.key.size() * 4, cudaMemcpyHostToDevice), "H2D");
            cuda_check(cudaMemcpy(b->ew.p + mm.edge_off, h.w.data(), h.w.size() * 4, cudaMemcpyHostToDevice), "H2D");
            cuda_check(cudaMemcpy(b->row_ptr.p + mm.rp_off, h.row_ptr.data(), h.row_ptr.size() * 4, cudaMemcpyHostToDevice),
                       "H2D");
            cuda_check(cudaMemcpy(b->perm.p + mm.node_off, h.perm.data(), h.perm.size() * 4, cudaMemcpyHostToDevice), "H2D");
        }
        bool any_raw = false;
        for (int i = 0; i < n_nets; ++i) any_raw = any_raw || !hs[i].bias.empty();
        if (any_raw) {
            b->bias.alloc(nodes, &b->bytes);
            for (int i = 0; i < n_nets; ++i)
                if (!hs[i].bias.empty())
                    cuda_check(cudaMemcpy(b->bias.p + b->m[i].node_off, hs[i].bias.data(), hs[i].bias.size() * 4,
                                          cudaMemcpyHostToDevice),
                               "H2D");
        }
        for (int s = 0; s < gn::kNumBatchShapes; ++s) b->bdesc[s].upload(shape_desc[s], &b->bytes);
        std::vector<int64_t> rq_off = build_staged_pool(b, hs);
        if (b->model != GN_MODEL_FHN) {
            // spiking members run the staged form only; they start at their rest state
            if (!b->staged_ok) fail(GN_EINVAL, "the staged batch kernel cannot hold this batch of spiking networks");
            std::vector<float> v0(nodes);
            bool hetero = false;
            for (int i = 0; i < n_nets; ++i) {
                std::copy(hs[i].v0.begin(), hs[i].v0.end(), v0.begin() + b->m[i].node_off);
                hetero = hetero || !hs[i].cell.empty();
            }
            b->iz_v.upload(v0, &b->bytes);
            if (hetero) {  // every member gets a row block; homogeneous members keep null pointers
                std::vector<uint8_t> cell(nodes, 0);
                std::vector<float> rows(static_cast<size_t>(n_nets) * gn::kMaxCellTypes * gn::kTypeStride, 0.0f);
                for (int i = 0; i < n_nets; ++i) {
                    if (hs[i].cell.empty()) continue;
                    std::copy(hs[i].cell.begin(), hs[i].cell.end(), cell.begin() + b->m[i].node_off);
                    std::copy(hs[i].type_par.begin(), hs[i].type_par.end(),
                              rows.begin() + static_cast<size_t>(i) * gn::kMaxCellTypes * gn::kTypeStride);
                }
                b->cell.upload(cell, &b->bytes);
                b->type_par.upload(rows, &b->bytes);
            }
            b->hetero.assign(n_nets, 0);
            for (int i = 0; i < n_nets; ++i) b->hetero[i] = hs[i].cell.empty() ? 0 : 1;
            b->rp.alloc(nodes, &b->bytes);
            cuda_check(cudaMemset(b->rp.p, 0, b->rp.n * 8), "memset");
            if (b->model == GN_MODEL_HH) {
                double gm, gn_, gh;
                gnrt::hh_rest_gates(&gm, &gn_, &gh);
                b->hh_g.upload(std::vector<float4>(nodes, make_float4(static_cast<float>(gm), static_cast<float>(gn_),
                                                                      static_cast<float>(gh), 0.0f)),
                               &b->bytes);
            }
        }
        hs.clear();
        bool any_frames = false;
        for (int i = 0; i < n_nets; ++i) any_frames = any_frames || descs[i].obs.frame_average;
        if (any_frames) {
            b->obs_acc.alloc(nodes, &b->bytes);
            cuda_check(cudaMemset(b->obs_acc.p, 0, b->obs_acc.n * 4), "memset");
        }
        b->ring.alloc(ring, &b->bytes);
        b->wc.alloc(nodes + 2 * static_cast<int64_t>(n_nets), &b->bytes);
        b->bgc.alloc(nodes, &b->bytes);
        b->first.alloc(nodes, &b->bytes);
        b->obs.alloc(obs, &b->bytes);
        b->ev_node.alloc(ev, &b->bytes);
        b->ev_step.alloc(ev, &b->bytes);
        b->ev_count.alloc(n_nets, &b->bytes);
        b->npulses.alloc(n_nets, &b->bytes);
        b->status.alloc(1, &b->bytes);
        b->d_step.alloc(1, &b->bytes);
        b->queue.alloc(1, &b->bytes);
        b->d_args.alloc(n_nets, &b->bytes);
        cuda_check(cudaMemset(b->ring.p, 0, b->ring.n * 4), "memset");
        cuda_check(cudaMemset(b->wc.p, 0, b->wc.n * 8), "memset");
        cuda_check(cudaMemset(b->bgc.p, 0, b->bgc.n * 4), "memset");
        cuda_check(cudaMemset(b->first.p, 0xff, b->first.n * 8), "memset");
        cuda_check(cudaMemset(b->obs.p, 0, b->obs.n * 4), "memset");
        cuda_check(cudaMemset(b->ev_count.p, 0, b->ev_count.n * 8), "memset");
        cuda_check(cudaMemset(b->npulses.p, 0, b->npulses.n * 4), "memset");
        cuda_check(cudaMemset(b->status.p, 0, 4), "memset");
        cuda_check(cudaMemset(b->d_step.p, 0, 8), "memset");
        for (int i = 0; i < n_nets; ++i) {
            const Member &mm = b->m[i];
            gn::StepArgs &a = b->args[i];
            a.ekey = b->ekey.p + mm.keyw_off;
            a.ew = b->ew.p + mm.edge_off;
            a.row_ptr = b->row_ptr.p + mm.rp_off;
            a.blk = nullptr;
            a.ring = b->ring.p + mm.ring_off;
            a.wc = b->wc.p + mm.node_off + 2 * i;
            a.bgc = b->bgc.p + mm.node_off;
            a.bias = (b->bias.p && descs[i].coupling == GN_COUPLE_RAW) ? b->bias.p + mm.node_off : nullptr;
            a.first = b->first.p + mm.node_off;
            a.perm = b->perm.p + mm.node_off;
            a.n_pulses = b->npulses.p + i;
            a.p_node = nullptr;
            a.p_on = nullptr;
            a.p_off = nullptr;
            a.p_amp = nullptr;
            a.obs = b->obs.p + mm.obs_off;
            a.obs_cap = b->obs_cap;
            a.ev_node = b->ev_node.p + mm.ev_off;
            a.ev_step = b->ev_step.p + mm.ev_off;
            a.ev_count = b->ev_count.p + i;
            a.ev_cap = mm.ev_cap;
            a.d_step = b->d_step.p;
            a.status = b->status.p;
            a.obs_acc = a.frame_avg ? b->obs_acc.p + mm.node_off : nullptr;
            if (b->model != GN_MODEL_FHN) {
                a.iz_v = b->iz_v.p + mm.node_off;
                a.rp = b->rp.p + mm.node_off;
                a.hh_g = b->model == GN_MODEL_HH ? b->hh_g.p + mm.node_off : nullptr;
                if (b->hetero[i]) {
                    a.cell_type = b->cell.p + mm.node_off;
                    a.type_par = b->type_par.p + static_cast<size_t>(i) * gn::kMaxCellTypes * gn::kTypeStride;
                }
            }
            if (b->staged_ok) {
                a.st_tile = b->st_tile.p;
                a.st_tile2 = b->st_tile2.p;
                a.st_ukey = b->st_ukey.p;
                a.st_slice = b->st_slice.p;
                a.st_w = b->st_w.p;
                a.st_u = b->st_u.p;
                a.st_plist = b->st_plist.p;
                a.st_rq = b->st_rq.p + rq_off[i];
            }
        }
        // largest networks first
        b->order.resize(n_nets);
        std::iota(b->order.begin(), b->order.end(), 0);
        std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) {
            return b->m[x].E + b->m[x].N > b->m[y].E + b->m[y].N;
        });
        b->d_order.upload(b->order, &b->bytes);
        b->shape = -1;
        upload_args(b);
        cuda_check(cudaDeviceSynchronize(), "create");
    });
    if (st != GN_OK) {
        delete b;
        return st;
    }
    *out = b;
    return GN_OK;
}

gn_status gn_batch_destroy(gn_batch *b)
{
    if (!b) return GN_OK;
    return guarded([&] {
        DeviceGuard dg(b->device);
        cudaStreamSynchronize(b->stream);
        delete b;
    });
}

gn_status gn_batch_get_info(const gn_batch *b, gn_batch_info *info)
{
    return guarded([&] {
        check_batch(b);
        if (!info) fail(GN_EINVAL, "info is NULL");
        info->n_nets = b->n_nets;
        info->n_nodes = 0;
        info->n_edges = 0;
        for (const Member &mm : b->m) {
            info->n_nodes += mm.N;
            info->n_edges += mm.E;
        }
        info->step = b->step;
        info->cta_threads = b->shape >= kStaged ? gn::kBatchStagedShape.threads
                            : b->shape >= 0       ? gn::kBatchThreads[b->shape]
                                                  : 0;
        info->grid = b->grid;
        info->device_bytes = b->bytes;
        info->step_kernel = b->shape == kLanes ? 5 : b->shape == kStaged ? 3 : b->shape >= 0 ? 1 : 0;
        info->step_groups = b->shape >= kStaged ? static_cast<int32_t>(b->st_groups.size()) : 0;
        info->step_lanes = b->shape >= kStaged ? std::min(b->st_lanes, std::max(1, info->step_groups)) : 0;
    });
}

gn_status gn_batch_get_net_info(const gn_batch *b, int32_t net, gn_net_info *info)
{
    return guarded([&] {
        check_batch(b, net);
        if (!info) fail(GN_EINVAL, "info is NULL");
        const Member &mm = b->m[net];
        std::memset(info, 0, sizeof *info);
        info->n_nodes = mm.N;
        info->n_edges = mm.E;
        info->ring_depth = mm.R;
        info->max_delay = mm.dmax;
        info->min_delay = mm.dmin;
        info->n_clamped = mm.n_clamped;
        info->edge_format = mm.packed ? 0 : 1;
        // tiles when the staged form steps the batch, else row blocks of k_batch's CTA size
        info->n_blocks = b->shape >= kStaged ? mm.st_nt : mm.n_blocks[desc_shape(b)];
        info->step = b->step;
        info->samples = b->step / mm.sample_every;
        info->v_rest = mm.v_rest;
        info->w_rest = mm.w_rest;
    });
}

gn_status gn_batch_get_delays(const gn_batch *b, int32_t net, int32_t *out)
{
    return guarded([&] {
        check_batch(b, net);
        if (!out && b->m[net].E) fail(GN_EINVAL, "out is NULL");
        std::copy(b->m[net].delay.begin(), b->m[net].delay.end(), out);
    });
}

gn_status gn_batch_set_stimulus_all(gn_batch *b, const gn_pulse *pulses, const int32_t *counts)
{
    return guarded([&] {
        check_batch(b);
        if (!counts) fail(GN_EINVAL, "counts is NULL");
        DeviceGuard dg(b->device);
        sync(b);
        std::vector<int32_t> nd;
        std::vector<int64_t> on, off;
        std::vector<float> amp;
        std::vector<int32_t> cnt(b->n_nets);
        int64_t k = 0;
        for (int i = 0; i < b->n_nets; ++i) {
            if (counts[i] < 0) fail(GN_EINVAL, "negative pulse count");
            gnrt::PulseTable t = gnrt::make_pulses(pulses ? pulses + k : nullptr, counts[i], b->m[i].N, b->m[i].dt,
                                                   b->m[i].inv);
            k += counts[i];
            b->m[i].pulse_off = static_cast<int64_t>(nd.size());
            cnt[i] = static_cast<int32_t>(t.node.size());
            nd.insert(nd.end(), t.node.begin(), t.node.end());
            on.insert(on.end(), t.on.begin(), t.on.end());
            off.insert(off.end(), t.off.begin(), t.off.end());
            amp.insert(amp.end(), t.amp.begin(), t.amp.end());
        }
        b->p_node.release();
        b->p_on.release();
        b->p_off.release();
        b->p_amp.release();
        b->p_node.upload(nd, &b->bytes);
        b->p_on.upload(on, &b->bytes);
        b->p_off.upload(off, &b->bytes);
        b->p_amp.upload(amp, &b->bytes);
        cuda_check(cudaMemcpy(b->npulses.p, cnt.data(), cnt.size() * 4, cudaMemcpyHostToDevice), "H2D");
        for (int i = 0; i < b->n_nets; ++i) {
            gn::StepArgs &a = b->args[i];
            const bool has = cnt[i] > 0;
            a.p_node = has ? b->p_node.p + b->m[i].pulse_off : nullptr;
            a.p_on = has ? b->p_on.p + b->m[i].pulse_off : nullptr;
            a.p_off = has ? b->p_off.p + b->m[i].pulse_off : nullptr;
            a.p_amp = has ? b->p_amp.p + b->m[i].pulse_off : nullptr;
        }
        upload_args(b);
    });
}

gn_status gn_batch_set_background(gn_batch *b, int32_t net, double rate_hz, float amp, double dur_ms, uint64_t seed)
{
    return guarded([&] {
        check_batch(b, net);
        if (!(rate_hz >= 0.0) || !std::isfinite(rate_hz) || !std::isfinite(amp) || !(dur_ms >= 0.0))
            fail(GN_EINVAL, "bad background parameters");
        DeviceGuard dg(b->device);
        sync(b);
        gn::StepArgs &a = b->args[net];
        a.bg_thr = gnrt::background_threshold(rate_hz, b->m[net].dt);
        a.bg_amp = amp;
        a.bg_width = static_cast<int32_t>(llround(dur_ms / b->m[net].dt));
        a.bg_seed = seed;
        upload_args(b);
    });
}

gn_status gn_batch_step(gn_batch *b, int64_t n_steps)
{
    return guarded([&] {
        check_batch(b);
        if (n_steps < 0 || n_steps > 2147483647LL) fail(GN_EINVAL, "n_steps out of range");
        if (n_steps == 0) return;
        DeviceGuard dg(b->device);
        if (b->shape < 0) {
            const char *e = getenv("GN_BATCH_KERNEL");
            const int only = e && *e ? atoi(e) : 0;
            if (only != 0 && only != 1 && only != 3 && only != 4 && only != 5)
                fail(GN_EINVAL, "GN_BATCH_KERNEL must be 1, 3, 4 or 5");
            if (only >= 3 && !b->staged_ok) fail(GN_EINVAL, "the staged batch kernel cannot hold this batch");
            if (b->model != GN_MODEL_FHN && only == 1) fail(GN_EINVAL, "spiking batches run the staged batch kernel");
            if (only == 4)
                set_shape(b, kStaged, true, std::max(1, lanes_env()));  // the staged form with L2 blocking, untimed
            else if (only == 5)
                set_shape(b, kLanes, true, std::max(1, lanes_env()));   // its persistent lanes schedule, untimed
            else
                autotune(b, b->model == GN_MODEL_FHN && only != 3, only != 1, only == 0);
        }
        if (b->shape == kLanes) {  // one cooperative launch per chunk, no graph
            for (int64_t left = n_steps; left > 0;) {
                const int n = static_cast<int>(std::min<int64_t>(left, kGraphSteps));
                launch_steps(b, b->d_args.p, b->d_step.p, n, kLanes, b->grid, b->st_groups, b->st_lanes, b->stream,
                             b->st_gtab.p);
                cuda_check(gn::launch_advance(b->d_step.p, n, b->stream), "advance launch");
                left -= n;
            }
        } else if (b->shape == kStaged) {
            if (!b->graph) build_graph(b, kGraphSteps);
            int64_t left = n_steps;
            for (; left >= kGraphSteps; left -= kGraphSteps)
                cuda_check(cudaGraphLaunch(b->graph, b->stream), "cudaGraphLaunch");
            if (left) {
                launch_steps(b, b->d_args.p, b->d_step.p, static_cast<int>(left), kStaged, b->grid, b->st_groups,
                             b->st_lanes, b->stream);
                cuda_check(gn::launch_advance(b->d_step.p, left, b->stream), "advance launch");
            }
        } else {
            if (!b->graph || b->graph_steps != n_steps) build_graph(b, n_steps);
            cuda_check(cudaGraphLaunch(b->graph, b->stream), "cudaGraphLaunch");
        }
        b->step += n_steps;
    });
}

gn_status gn_batch_step_static(gn_batch *b, int64_t n_steps)
{
    return guarded([&] {
        check_batch(b);
        if (n_steps < 0 || n_steps > 2147483647LL) fail(GN_EINVAL, "n_steps out of range");
        if (b->model != GN_MODEL_FHN)
            fail(GN_EINVAL, "the allocation-free step takes FitzHugh-Nagumo batches (the persistent kernel)");
        if (b->n_nets > gn::kStaticQueueNets)
            fail(GN_ERANGE, "a batch of %d networks exceeds the %d networks the static work queue holds", b->n_nets,
                 gn::kStaticQueueNets);
        if (n_steps == 0) return;
        DeviceGuard dg(b->device);
        // the CTA size chosen by an earlier gn_batch_step, else the default one
        // (choosing it here would time candidates on newly allocated scratch state)
        int shape = b->shape, grid = b->grid;
        if (shape < 0 || shape >= kStaged) {
            int per_sm = 0, sms = 0;
            shape = 0;
            cuda_check(gn::batch_occupancy(shape, &per_sm), "occupancy");
            cuda_check(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device), "device query");
            grid = std::max(1, std::min(b->n_nets, std::max(1, per_sm) * sms));
        }
        cuda_check(gn::launch_batch_static(b->d_args.p, b->d_order.p, b->n_nets, b->d_step.p,
                                           static_cast<int>(n_steps), shape, grid, b->device, b->stream),
                   "batch launch with the static work queue");
        cuda_check(gn::launch_advance(b->d_step.p, n_steps, b->stream), "advance launch");
        b->step += n_steps;
    });
}

gn_status gn_batch_export_traces(gn_batch *b, int64_t first_sample, int32_t n_samples, float *out)
{
    return guarded([&] {
        check_batch(b);
        if (n_samples < 1 || first_sample < 0 || !out) fail(GN_EINVAL, "bad trace window or output");
        DeviceGuard dg(b->device);
        int max_nodes = 0;
        std::vector<gn::ExportNet> nets(b->n_nets);
        int64_t node_off = 0;
        for (int i = 0; i < b->n_nets; ++i) {
            const Member &mm = b->m[i];
            const int64_t produced = b->step / mm.sample_every;
            if (first_sample + n_samples > produced) fail(GN_ERANGE, "network %d has only %lld samples", i, (long long)produced);
            if (produced - first_sample > b->obs_cap)
                fail(GN_ERANGE, "network %d no longer holds sample %lld (observation capacity %lld)", i,
                     (long long)first_sample, (long long)b->obs_cap);
            nets[i] = gn::ExportNet{mm.obs_off, node_off, mm.N, 0};
            node_off += mm.N;
            max_nodes = std::max(max_nodes, mm.N);
        }
        gn::ExportNet *d_nets = nullptr;
        cuda_check(cudaMallocAsync(reinterpret_cast<void **>(&d_nets), nets.size() * sizeof(gn::ExportNet), b->stream),
                   "cudaMallocAsync");
        cudaError_t e = cudaMemcpyAsync(d_nets, nets.data(), nets.size() * sizeof(gn::ExportNet), cudaMemcpyHostToDevice,
                                        b->stream);
        if (e == cudaSuccess)
            e = gn::launch_export_traces(b->obs.p, d_nets, b->n_nets, max_nodes, first_sample, n_samples, b->obs_cap,
                                         out, b->stream);
        cudaFreeAsync(d_nets, b->stream);
        cuda_check(e, "trace export");
        sync(b);
    });
}

gn_status gn_batch_synchronize(gn_batch *b)
{
    return guarded([&] {
        check_batch(b);
        DeviceGuard dg(b->device);
        sync(b);
    });
}

gn_status gn_batch_observe(gn_batch *b, int32_t net, float *out, int64_t max_samples, int64_t *first_sample,
                           int64_t *written)
{
    return guarded([&] {
        check_batch(b, net);
        if (max_samples < 0) fail(GN_EINVAL, "max_samples < 0");
        DeviceGuard dg(b->device);
        sync(b);
        Member &mm = b->m[net];
        const int64_t produced = b->step / mm.sample_every;
        bool lost = false;
        if (produced - mm.read_cursor > b->obs_cap) {
            mm.read_cursor = produced - b->obs_cap;
            lost = true;
        }
        const int64_t m = std::min(max_samples, produced - mm.read_cursor);
        if (first_sample) *first_sample = mm.read_cursor;
        if (written) *written = m;
        const float *base = b->obs.p + mm.obs_off;
        int64_t done = out ? 0 : m;
        while (done < m) {
            const int64_t k = (mm.read_cursor + done) % b->obs_cap;
            const int64_t len = std::min(m - done, b->obs_cap - k);
            cuda_check(cudaMemcpy(out + done * mm.N, base + k * mm.N, len * mm.N * 4, cudaMemcpyDeviceToHost),
                       "D2H observations");
            done += len;
        }
        mm.read_cursor += m;
        if (lost) fail(GN_EOVERFLOW, "observation buffer overflowed: older samples were lost");
    });
}

gn_status gn_batch_get_state(gn_batch *b, int32_t net, float *v, float *w, float *c, int32_t *bg_count,
                             int64_t *step)
{
    return guarded([&] {
        check_batch(b, net);
        DeviceGuard dg(b->device);
        sync(b);
        const Member &mm = b->m[net];
        std::vector<float> t(mm.N);
        if (v) {
            const float *src = b->model != GN_MODEL_FHN ? b->iz_v.p + mm.node_off
                                                        : b->ring.p + mm.ring_off + (b->step & (mm.R - 1)) * mm.stride;
            cuda_check(cudaMemcpy(t.data(), src, mm.N * 4, cudaMemcpyDeviceToHost), "D2H v");
            to_caller(mm, t.data(), v);
        }
        if (w || c) {
            std::vector<float2> t2(mm.N);
            cuda_check(cudaMemcpy(t2.data(), b->wc.p + mm.node_off + 2 * net, mm.N * 8, cudaMemcpyDeviceToHost), "D2H wc");
            for (int32_t r = 0; r < mm.N; ++r) {
                if (w) w[mm.perm[r]] = t2[r].x;
                if (c) c[mm.perm[r]] = t2[r].y;
            }
        }
        if (bg_count) {
            std::vector<int32_t> t3(mm.N);
            cuda_check(cudaMemcpy(t3.data(), b->bgc.p + mm.node_off, mm.N * 4, cudaMemcpyDeviceToHost), "D2H bg");
            to_caller(mm, t3.data(), bg_count);
        }
        if (step) *step = b->step;
    });
}

gn_status gn_batch_get_izh_state(gn_batch *b, int32_t net, float *V, float *r, float *p)
{
    return guarded([&] {
        check_batch(b, net);
        if (b->model == GN_MODEL_FHN) fail(GN_EINVAL, "the batch does not use a spiking node model");
        DeviceGuard dg(b->device);
        sync(b);
        const Member &mm = b->m[net];
        if (V) {
            std::vector<float> t(mm.N);
            cuda_check(cudaMemcpy(t.data(), b->iz_v.p + mm.node_off, mm.N * 4, cudaMemcpyDeviceToHost), "D2H V");
            to_caller(mm, t.data(), V);
        }
        if (r || p) {
            std::vector<float2> t(mm.N);
            cuda_check(cudaMemcpy(t.data(), b->rp.p + mm.node_off, mm.N * 8, cudaMemcpyDeviceToHost), "D2H rp");
            for (int32_t i = 0; i < mm.N; ++i) {
                if (r) r[mm.perm[i]] = t[i].x;
                if (p) p[mm.perm[i]] = t[i].y;
            }
        }
    });
}

gn_status gn_batch_get_hh_gates(gn_batch *b, int32_t net, float *m, float *n, float *h)
{
    return guarded([&] {
        check_batch(b, net);
        if (b->model != GN_MODEL_HH) fail(GN_EINVAL, "the batch does not use the Hodgkin-Huxley model");
        DeviceGuard dg(b->device);
        sync(b);
        const Member &mm = b->m[net];
        std::vector<float4> t(mm.N);
        cuda_check(cudaMemcpy(t.data(), b->hh_g.p + mm.node_off, mm.N * 16ull, cudaMemcpyDeviceToHost), "D2H gates");
        for (int32_t i = 0; i < mm.N; ++i) {
            if (m) m[mm.perm[i]] = t[i].x;
            if (n) n[mm.perm[i]] = t[i].y;
            if (h) h[mm.perm[i]] = t[i].z;
        }
    });
}

gn_status gn_batch_set_step(gn_batch *b, int64_t step)
{
    return guarded([&] {
        check_batch(b);
        if (step < 0) fail(GN_EINVAL, "step < 0");
        DeviceGuard dg(b->device);
        sync(b);
        cuda_check(cudaMemcpy(b->d_step.p, &step, 8, cudaMemcpyHostToDevice), "H2D step");
        cuda_check(cudaMemset(b->ev_count.p, 0, b->ev_count.n * 8), "memset");
        b->step = step;
        for (Member &mm : b->m) mm.read_cursor = step / mm.sample_every;
    });
}

gn_status gn_batch_set_state(gn_batch *b, int32_t net, const float *hist, int32_t depth, const float *w,
                             const float *c, const int32_t *bg_count)
{
    return guarded([&] {
        check_batch(b, net);
        const Member &mm = b->m[net];
        if (depth < 1 || depth > mm.R || !hist) fail(GN_EINVAL, "hist must hold 1..ring_depth rows");
        DeviceGuard dg(b->device);
        sync(b);
        const int32_t N = mm.N;
        std::vector<float> ring(static_cast<size_t>(mm.R) * mm.stride, 0.0f);
        for (int32_t k = 0; k < depth; ++k) {
            const int64_t slot = (b->step - k) & (mm.R - 1);
            for (int32_t j = 0; j < N; ++j) ring[slot * mm.stride + mm.inv[j]] = hist[static_cast<int64_t>(k) * N + j];
        }
        std::vector<float2> wc(N);
        std::vector<int32_t> bg(N, 0);
        for (int32_t j = 0; j < N; ++j) {
            wc[mm.inv[j]] = make_float2(w ? w[j] : 0.0f, c ? c[j] : 0.0f);
            if (bg_count) bg[mm.inv[j]] = bg_count[j];
        }
        cuda_check(cudaMemcpy(b->ring.p + mm.ring_off, ring.data(), ring.size() * 4, cudaMemcpyHostToDevice), "H2D");
        cuda_check(cudaMemcpy(b->wc.p + mm.node_off + 2 * net, wc.data(), N * 8ull, cudaMemcpyHostToDevice), "H2D");
        cuda_check(cudaMemcpy(b->bgc.p + mm.node_off, bg.data(), N * 4ull, cudaMemcpyHostToDevice), "H2D");
        cuda_check(cudaMemset(b->first.p + mm.node_off, 0xff, N * 8ull), "memset");
        cuda_check(cudaMemset(b->ev_count.p + net, 0, 8), "memset");
        if (b->args[net].obs_acc) cuda_check(cudaMemset(b->args[net].obs_acc, 0, N * 4ull), "memset");  // a new frame
    });
}

gn_status gn_batch_get_history(gn_batch *b, int32_t net, float *out, int32_t depth)
{
    return guarded([&] {
        check_batch(b, net);
        const Member &mm = b->m[net];
        if (depth < 1 || depth > mm.R || !out) fail(GN_EINVAL, "depth must be in [1, ring_depth]");
        DeviceGuard dg(b->device);
        sync(b);
        std::vector<float> t(mm.N);
        for (int32_t k = 0; k < depth; ++k) {
            const int64_t slot = (b->step - k) & (mm.R - 1);
            cuda_check(cudaMemcpy(t.data(), b->ring.p + mm.ring_off + slot * mm.stride, mm.N * 4, cudaMemcpyDeviceToHost),
                       "D2H");
            to_caller(mm, t.data(), out + static_cast<int64_t>(k) * mm.N);
        }
    });
}

gn_status gn_batch_get_arrivals(gn_batch *b, int32_t net, int64_t *first_arrival)
{
    return guarded([&] {
        check_batch(b, net);
        if (!first_arrival) fail(GN_EINVAL, "out is NULL");
        DeviceGuard dg(b->device);
        sync(b);
        const Member &mm = b->m[net];
        std::vector<int64_t> t(mm.N);
        cuda_check(cudaMemcpy(t.data(), b->first.p + mm.node_off, mm.N * 8, cudaMemcpyDeviceToHost), "D2H");
        to_caller(mm, t.data(), first_arrival);
    });
}

gn_status gn_batch_get_events(gn_batch *b, int32_t net, int32_t *node, int64_t *step, int64_t cap, int64_t *n_total)
{
    return guarded([&] {
        check_batch(b, net);
        if (cap < 0 || (cap > 0 && (!node || !step))) fail(GN_EINVAL, "bad output buffers");
        DeviceGuard dg(b->device);
        sync(b);
        const Member &mm = b->m[net];
        unsigned long long cnt = 0;
        cuda_check(cudaMemcpy(&cnt, b->ev_count.p + net, 8, cudaMemcpyDeviceToHost), "D2H");
        const int64_t kept = std::min<int64_t>(static_cast<int64_t>(cnt), mm.ev_cap);
        std::vector<int32_t> nd(kept);
        std::vector<int64_t> st(kept);
        if (kept) {
            cuda_check(cudaMemcpy(nd.data(), b->ev_node.p + mm.ev_off, kept * 4, cudaMemcpyDeviceToHost), "D2H");
            cuda_check(cudaMemcpy(st.data(), b->ev_step.p + mm.ev_off, kept * 8, cudaMemcpyDeviceToHost), "D2H");
        }
        std::vector<std::pair<int64_t, int32_t>> ev(kept);
        for (int64_t i = 0; i < kept; ++i) ev[i] = {st[i], mm.perm[nd[i]]};
        std::sort(ev.begin(), ev.end());
        const int64_t m = std::min(cap, kept);
        for (int64_t i = 0; i < m; ++i) {
            step[i] = ev[i].first;
            node[i] = ev[i].second;
        }
        if (n_total) *n_total = kept;
        if (static_cast<int64_t>(cnt) > mm.ev_cap) fail(GN_EOVERFLOW, "event buffer overflowed (%llu events)", cnt);
    });
}

}  // extern "C"
