// Internal layout of one network on the device, shared by the kernels and the
// host runtime of libgeonet.so (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <type_traits>

namespace gn {

// Device arrays and constants of one network, in internal (Morton) node order.
//
// HBM layout:
//   ring   float [R][ring_stride]  slot-major history: slot s holds v~ at the latest step
//                        t == s (mod R) that is <= the current step; the current
//                        state v~(n) is slot n & (R-1) (the ring *is* the state).
//   wc     float2 [N]    (w~, c~)
//   ekey   per edge, CSR by target, rows sorted by source:
//            packed:  uint32 (src << dbits) | D, dbits = log2 R
//            wide:    uint2  {src, D}
//   ew     float [E]     weights, same order
//   Edge arrays are padded by kEdgePad entries so 16-byte vector loads that
//   start inside [0, E) never leave the allocation.
struct StepArgs {
    int32_t N;
    int32_t ring_stride;     // floats per ring slot: N rounded up (N + 4 -> multiple of 32)
    int32_t ring_mask;       // R - 1
    int32_t dbits;           // packed keys: bits of D
    int32_t packed;          // 1: 32-bit packed keys, 0: 64-bit {src, D}
    const void *ekey;
    const float *ew;
    const int32_t *row_ptr;  // [N + 1]
    const int32_t *blk;      // [n_blocks + 1] first row of each row block
    float *ring;
    float2 *wc;
    int32_t *bgc;            // [N] background pulse counters, or null
    const float *bias;       // [N] RAW coupling: V* * sum of in-weights, or null
    int64_t *first;          // [N] first step with v~ != 0, -1 = none
    const int32_t *perm;     // [N] internal -> caller node id (RNG counters use caller ids)
    // pulses sorted by internal node id; the count lives in device memory so a new
    // pulse set can be copied in stream order without re-capturing the step graph
    const int32_t *n_pulses;
    const int32_t *p_node;
    const int64_t *p_on;
    const int64_t *p_off;
    const float *p_amp;
    // FHN about the rest point: dv = v (k1 + v (q2 + q3 v)) - cw w + S + U, dw = e (v - g w)
    float dt, k1, q2, q3, cw, dte, g;
    float alpha;             // dt / tau of the readout
    float theta_s;           // event threshold relative to rest, theta - V*
    float gain, offset, sigma, vrest;
    int32_t sample_every;
    int32_t frame_avg;       // camera frame averaging: a sample reads the frame mean of c
    float *obs_acc;          // [N] frame sums of c (frame averaging only)
    uint64_t obs_seed;
    uint32_t bg_thr;         // 0 = no background
    float bg_amp;
    int32_t bg_width;
    uint64_t bg_seed;
    float *obs;              // [obs_cap][N], rows in caller node order
    int64_t obs_cap;
    int32_t *ev_node;
    int64_t *ev_step;
    unsigned long long *ev_count;
    int64_t ev_cap;
    const int64_t *d_step;   // step counter: a launch with offset k runs step *d_step + k
    // persistent pipelined kernel
    const int4 *bdesc;       // [n_blocks] {first row, end row, first edge, end edge}
    int32_t n_blocks;
    unsigned int *status;    // device error word (kStatus* bits), read by the host after a sync
    // staged kernel (k_step_staged.cu): tiles of rows with their distinct gathers
    const int4 *st_tile;     // [tiles] {first row, rows, first gather, gathers}
    const int4 *st_tile2;    // [tiles] {first slice, slices, pieces, 0}
    const void *st_ukey;     // per gather: packed key, or {src, D} when wide
    const int2 *st_slice;    // {first entry, length}
    float *st_w;             // entry weights, column-major in slices of 32 pieces (plastic nets write them)
    const uint16_t *st_u;    // entry gather index within its tile
    const int32_t *st_rq;    // [N + 1] first piece-list entry of each row
    const uint16_t *st_plist;  // lane slot of each piece
    int32_t st_ucap;         // gather slots of a CTA's shared memory (largest padded gather count)
    int32_t st_xcap;         // entry slots of a CTA's shared memory (largest entry count)
    uint32_t wait_limit;     // polls of a bounded mbarrier wait before it reports kStatusTimeout
    // node model: 0 FitzHugh-Nagumo (fields above), 1 Izhikevich + alpha PSC + calcium,
    // 2 Hodgkin-Huxley + alpha PSC + calcium.  The spiking models' ring holds spd(V)
    // and their state is iz_v (V), wc (W, calcium), rp (r, p), plus hh_g (m, n, h, 0)
    // for model 2; iz_dtc (dt / C), iz_vpeak and iz_iext serve both.
    int32_t model;
    float iz_dtc, iz_k, iz_vr, iz_vt, iz_vpeak, iz_vreset, iz_dta, iz_b, iz_d, iz_iext;
    float ps_a2, ps_2a, ca_q;  // PSC a^2, 2a; calcium 1 / tau_c
    float hh_gna, hh_gk, hh_gl, hh_ena, hh_ek, hh_el;
    float *iz_v;
    float2 *rp;
    float4 *hh_g;
    // plasticity (spiking models, staged kernel): the ring word of a node is
    // (s / dt) << 1 | spd(V), s the time since its last spike; dw = stdp_dta sign(q) e^(-beta |q|)
    int32_t stdp;
    float stdp_dta, stdp_beta;   // dt alpha, beta
    const uint32_t *st_pinfo;    // per lane slot: piece length | local row << 16
    // heterogeneous cells (spiking models): each node's parameter set, rows of
    // kTypeStride floats in the order of the scalar fields above (null: homogeneous)
    const uint8_t *cell_type;
    const float *type_par;
};

constexpr int kMaxCellTypes = 8;
constexpr int kTypeStride = 16;
constexpr int kTypeA2 = 13;  // row offset of a_s^2, then 2 a_s and 1 / tau_c (both spiking models)

// A plastic model's kernel code: the node model | kPlastic.
constexpr int kPlastic = 4;
// A spiking model's code | kNoRing: the node update leaves the spike ring to its
// caller (the resident kernel keeps spd as bits).
constexpr int kNoRing = 8;
constexpr uint32_t kSpikeStepsMax = 1u << 30;  // s saturates at this many steps

// Calls f(std::integral_constant<int, m>) for node model m: every step kernel is
// instantiated once per model, so no model's code sits in another model's kernel
// (a branch to the Hodgkin-Huxley update alone cost the FitzHugh-Nagumo kernel 3 %).
template <class F>
inline cudaError_t with_model(int model, F &&f)
{
    switch (model) {
        case 1: return f(std::integral_constant<int, 1>{});
        case 2: return f(std::integral_constant<int, 2>{});
        default: return f(std::integral_constant<int, 0>{});
    }
}

// The same for the staged kernel, which also runs the plastic spiking models
// (codes 1 | kPlastic, 2 | kPlastic).
template <class F>
inline cudaError_t with_model_plastic(int model, bool plastic, F &&f)
{
    if (!plastic) return with_model(model, static_cast<F &&>(f));
    switch (model) {
        case 1: return f(std::integral_constant<int, 1 | kPlastic>{});
        case 2: return f(std::integral_constant<int, 2 | kPlastic>{});
        default: return cudaErrorInvalidValue;
    }
}

constexpr uint32_t kDefaultWaitLimit = 1u << 22;

constexpr unsigned int kStatusTimeout = 1u;  // a bounded mbarrier wait gave up

constexpr int kEdgePad = 4096;

// Summation order of a node's input S_j, the same in every step kernel and in the
// batched kernel, so the kernel the autotuner picks never changes a result: a row
// of at most kWarpRow edges is summed in row order by one thread; a longer row is
// split over 32 lanes (lane l takes edges l, l + 32, ... in order) whose partial
// sums are combined by the butterfly x_l += x_(l xor o), o = 16, 8, 4, 2, 1.  Each
// term w_e * v~ is rounded to FP32 before it is added (no fused multiply-add).
// (Rows longer than one row block's capacity are summed in a shape-dependent order
// by kernels 1, 2 and the batched kernel.)
constexpr int kWarpRow = 48;

// CTA shapes of the row-block step kernel: T threads, EPT edges per thread; its
// row blocks hold at most T * EPT - 3 edges and T rows.  The persistent pipelined
// kernel uses shape 0.
struct StepShape {
    int threads, ept, min_ctas_per_sm;
};
constexpr int kNumStepShapes = 5;
extern const StepShape kStepShapes[kNumStepShapes];

// Kernel launchers (k_step.cu, k_step_pipe.cu, k_delay.cu)
cudaError_t launch_step(const StepArgs &a, int n_blocks, int k, int shape, bool packed, bool stream_edges,
                        cudaStream_t s);
cudaError_t launch_advance(int64_t *d_step, int64_t by, cudaStream_t s);
// staged kernel (k_step_staged.cu): one CTA of `threads` per tile, smem_bytes of
// dynamic shared memory; prepare raises the kernel's shared-memory limit
// stage_entries: 1 copies a tile's edge entries into shared memory with its gather
// keys; 0 keeps only the keys there and prefetches the entries into L2 (less
// shared memory per CTA, more CTAs per SM)
constexpr int kNumStagedShapes = 8;
struct StagedShape {
    int threads, ucap, ecap, pcap, stage_entries;
};
extern const StagedShape kStagedShapes[kNumStagedShapes];
// early: 0 gather after the grid wait; 1 gather before it and let the next grid start
// at once (a grid larger than the CTAs the device holds at once); 2 gather before it
// and let the next grid start after the CTA's own wait (any grid) -- see staged_tile;
// static weights only for 1 and 2
cudaError_t launch_step_staged(const StepArgs &a, int n_tiles, int k, const StagedShape &shape, bool packed,
                               bool stream_edges, size_t smem_bytes, int early, cudaStream_t s);
cudaError_t step_staged_prepare(const StagedShape &shape, int model, bool plastic, bool packed, bool stream_edges,
                                size_t smem_bytes, int *ctas_per_sm);
// persistent staged step of one network (kind 5): one cooperative launch of one CTA
// per tile (all resident at once) runs n_steps steps with each tile's gather keys and
// entries held in shared memory; counts: 64 words (the launch zeroes them first);
// smem_bytes: 16 + max_u (4 or 8 key bytes + 4 value bytes) + max_x 6 + max_p 4
// cluster: the grid (at most kMaxClusterTiles tiles) is one thread-block cluster and the
// step barrier the cluster's; prepare reports CTAs per SM, or (cluster) how many such
// clusters the device holds at once
constexpr int kMaxClusterTiles = 16;
cudaError_t launch_step_persist(const StepArgs &a, int n_tiles, int n_steps, const StagedShape &shape, bool packed,
                                bool cluster, unsigned int *counts, size_t smem_bytes, cudaStream_t s);
cudaError_t step_persist_prepare(const StagedShape &shape, int model, bool packed, bool cluster, int n_tiles,
                                 size_t smem_bytes, int *fits);
// batched form with the staged layout: one launch per step over every member's
// tiles (tile_net[t] = the member of tile t), tiles cut with kBatchStagedShape
constexpr StagedShape kBatchStagedShape = {128, 3072, 4096, 256, 0};
// (every member of node model `model`)
// (launch_first: the grid outnumbers the CTAs the device holds at once)
cudaError_t launch_batch_staged(int model, const StepArgs *nets, const int *tile_net, int n_tiles, int k, bool packed,
                                bool stream_edges, size_t smem_bytes, bool launch_first, cudaStream_t s);
cudaError_t batch_staged_prepare(int model, bool packed, bool stream_edges, size_t smem_bytes, int *ctas_per_sm);
// ... persistent, for L2-blocked groups: one cooperative launch of `grid` CTAs (all
// resident at once) in `lanes` lanes steps each group {first tile, tiles} of
// `groups` n_steps times (group g in lane g % lanes); counts: kLaneWords words per
// lane, zero at launch (the lanes' barrier words); status: the batch's status word
constexpr int kMaxBatchLanes = 8;
constexpr int kLaneWords = 64;  // per lane: the arrival count at word 0 (lanes 256 bytes apart)
cudaError_t launch_batch_lanes(int model, const StepArgs *nets, const int *tile_net, const int2 *groups, int n_groups,
                               int lanes, int n_steps, unsigned int *counts, unsigned int *status, uint32_t limit,
                               bool packed, int grid, size_t smem_bytes, cudaStream_t s);
cudaError_t batch_lanes_prepare(int model, bool packed, size_t smem_bytes, int *ctas_per_sm);
// resident kernel (k_resident.cu): one CTA holds a small network -- edges, row
// pointers, history ring (FitzHugh-Nagumo FP32, spiking models one bit per node) and
// node state -- in shared memory and runs n_steps steps per launch.  Byte offsets of
// each array in the CTA's dynamic shared memory:
struct ResidentLayout {
    int32_t N, R, words, stride;  // nodes, ring slots, 32-bit words per spike-ring slot, floats per FHN slot
    int64_t E;
    int32_t ev_cap;               // events buffered in shared memory (a multiple of N)
    int32_t pulse_cap;            // pulses kept in shared memory (more stay in global memory)
    uint32_t off_key, off_w, off_rp, off_S, off_long, off_ring, off_wc, off_v, off_rpq, off_hh, off_bgc, off_acc;
    uint32_t off_perm, off_first, off_evn, off_evs, off_pnode, off_pon, off_poff, off_pamp;
    size_t bytes;
};
constexpr int kResidentPulses = 256;
constexpr int kNumResidentShapes = 3;
extern const int kResidentThreads[kNumResidentShapes];
// the longest row the resident kernel takes: every kernel sums rows up to this length in
// the same order
constexpr int kResidentMaxRow = 1021;
// ev_factor: events buffered per node (1 or 2; with 1 the buffer is flushed after every
// step that had an event)
ResidentLayout resident_layout(int N, int64_t E, int R, int model, bool frame_avg, int ev_factor);
// raises the kernel's shared-memory limit to `bytes` of dynamic shared memory; returns
// the largest dynamic size a CTA can have in *max_bytes
cudaError_t resident_prepare(int model, int shape, size_t bytes, size_t *max_bytes);
cudaError_t launch_resident(const StepArgs &a, const ResidentLayout &L, int n_steps, int shape, cudaStream_t s);
// persistent bulk-copy pipelined variant (k_step_pipe.cu); grid = CTAs to launch
cudaError_t launch_step_pipe(const StepArgs &a, int grid, int k, bool packed, bool stream_edges, cudaStream_t s);
int step_pipe_smem_bytes(bool packed);
cudaError_t step_pipe_prepare(int model, bool packed, bool stream_edges, int *ctas_per_sm);
// batched form (k_batch.cu): one persistent launch over many networks
constexpr int kNumBatchShapes = 3;
extern const int kBatchThreads[kNumBatchShapes];
int batch_block_cap(int shape);
cudaError_t launch_batch(const StepArgs *nets, const int *order, int n_nets, int *queue, const int64_t *d_step,
                         int n_steps, int shape, int grid, cudaStream_t s);
cudaError_t batch_occupancy(int shape, int *ctas_per_sm);
// the same launch with its work queue in a file-scope device array (no allocation);
// d_order is the batch's own device copy of the schedule, copied device to device
// into the array in stream order
constexpr int kStaticQueueNets = 65536;
cudaError_t launch_batch_static(const StepArgs *nets, const int *d_order, int n_nets, const int64_t *d_step,
                                int n_steps, int shape, int grid, int device, cudaStream_t s);

// estimator (k_est.cu)
struct ExportNet {
    int64_t obs_off;   // first float of the network's observation ring in the pool
    int64_t node_off;  // first row of the network in the node-major output
    int32_t n_nodes;
    int32_t pad;
};
cudaError_t launch_export_traces(const float *obs_pool, const ExportNet *nets, int n_nets, int max_nodes,
                                 int64_t first, int T, int64_t cap, float *out, cudaStream_t s);
// scratch: ncc_scratch_floats(M, T) floats (centred traces and their prefix sums)
cudaError_t launch_ncc(const float *X, int64_t M, int T, float *scratch, const double *pos, int dim, int64_t P,
                       const int *src, const int *dst, const double *radius, double v_max, double sample_ms,
                       float *feat, float *score, cudaStream_t s);
int64_t ncc_scratch_floats(int64_t M, int T);

// MLP of the learned estimator (k_mlp.cu); hidden width 256, inputs padded to 64
constexpr int kMlpHidden = 256;
constexpr int kMlpInPad = 64;
// Device buffers of one MLP (owned by the host runtime, mlp.cu).  Parameters, their
// gradients and Adam moments are packed FP32 [W1 (in x 256) | b1 | W2 | b2 | w3 | b3];
// wimg holds the BF16 weight images the tile kernel streams (9 chunks of 32 KB: W1t, W2t
// in four K-chunks, W2b in four K-chunks); the *_img buffers the batch-major
// operands of the weight gradients, one image per 64 rows of the batch.
struct MlpBuffers {
    int in_dim;
    int64_t n_params, off_W1, off_b1, off_W2, off_b2, off_w3, off_b3;
    float *params, *grads, *m, *v;
    void *wimg, *xt_img, *h1t_img, *dh2t_img, *dh1t_img;
    float *part_w2;    // [splits][256][256]
    float *part_w1;    // [splits][64][256] (dW1, rows k >= in_dim zero)
    float *part_head;  // [tiles][2 * 256 + 2]
    float *part_b1;    // [tiles][256]
    float *loss_sum;   // [1]
    unsigned int *status;
};
cudaError_t mlp_prepare();
size_t mlp_wimg_bytes();
size_t mlp_xt_bytes(int Bp);
size_t mlp_ht_bytes(int Bp);
// splits of the weight-gradient reduction over the batch and the 64-row chunks of each
int mlp_wgrad_splits(int Bp, int *chunks_per_split);
// Forward (+ backward with labels y) of B rows, Bp = B rounded up to 128; row b of the
// batch is X[idx[cursor * B + b]] (idx, cursor may be null).  Every kernel sets
// *status to kStatusTimeout if a bounded wait gave up.
cudaError_t mlp_launch_tile(const MlpBuffers &b, const float *X, const int64_t *idx, const int64_t *cursor,
                            const float *y, int B, int Bp, float *p_out, cudaStream_t s);
cudaError_t mlp_launch_wgrad(const MlpBuffers &b, int Bp, cudaStream_t s);
// gradients into b.grads and the loss sum into b.loss_sum; with adamw also the AdamW
// step (bias corrections bc1, bc2, or bc_table[2 cursor + {0, 1}]) and the weight
// images; with `losses` (a replayed epoch) also the step's mean loss over B rows to
// losses[cursor] and the cursor moved on (`ticket`: a zeroed counter of the launch)
cudaError_t mlp_launch_update(const MlpBuffers &b, int Bp, bool adamw, float lr, float wd, float bc1, float bc2,
                              const float *bc_table, int64_t *cursor, float *losses, unsigned int *ticket, int B,
                              cudaStream_t s);
cudaError_t mlp_launch_refresh(const MlpBuffers &b, cudaStream_t s);

cudaError_t launch_delay(int64_t n_edges, int32_t dim, const double *pos, const int32_t *src,
                         const int32_t *dst, const double *speed, double speed_scalar, double dt_ms,
                         int32_t *delay, uint8_t *clamped, cudaStream_t s);

}  // namespace gn
