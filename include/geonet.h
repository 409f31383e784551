/*
 * geonet.h -- C ABI of libgeonet.so, a B300 (sm_103a) simulator of delayed,
 * weighted signalling on geometric networks after Buibas & Silva, "A framework
 * for simulating and estimating the state and functional topology of complex
 * dynamic geometric networks" (arXiv:0908.3934).
 *
 * The model (all citations are to that paper):
 *   - vertices j with a static position x_j and state y_j = {V_j, W_j}       (Sec. 2, Eq. yjstate)
 *   - directed edges i -> j with weight omega_ij and delay tau_ij             (Sec. 2, Eq. Yjset)
 *   - geodesic delays tau_ij = |x_i - x_j| / s_ij, quantised to whole steps   (Sec. 3.2.1, Eq. delaydist;
 *                                                                              Sec. 2, Eq. gendelay)
 *   - the delayed input S_j(t) = sum_{i->j} omega_ij v_i(t - tau_ij)           (Sec. 2, Eq. Yjset)
 *   - FitzHugh-Nagumo vertex dynamics, forward Euler in steps of dt:          (Sec. 3.1, FHN pair and
 *       V' = V + dt (aV - bV^3 - cW + S + U + I_ext),  W' = W + dt e (V + f - gW)   Eq. fnstate)
 *   - a control input U_j(t) (pulses, background pulses)                      (Sec. 2, u_j in Eq. Htrans)
 *   - the readout: a first-order low-pass c of V and a noisy observation      (Sec. 3.3, calcium model
 *       y = gain (V* + c~) + offset + sigma N(0,1)                              and I = n c + b + N(0, g^2))
 *
 * Conventions shared by every call:
 *   - Status codes, never exceptions.  gn_last_error() gives a message for the
 *     last failing call on the calling thread.
 *   - Every input array is copied during the call; the caller may free it on return.
 *   - Host buffers are caller-owned and in the CALLER's node and edge order: the
 *     library renumbers nodes internally (spatial order) and undoes it on output.
 *   - State is reported relative to the isolated rest point (V*, W*):
 *     v~ = V - V*, w~ = W - W*, c~ = c - V*.  gn_get_rest() gives (V*, W*).
 *   - gn_step() is asynchronous on the net's stream; every call that returns data
 *     to the host synchronises that stream first.
 *   - A handle is not thread-safe: calls on one handle must not overlap.
 */
#ifndef GEONET_H
#define GEONET_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GN_API __attribute__((visibility("default")))
#else
#define GN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GN_OK = 0,
    GN_EINVAL = -1,      /* invalid argument or descriptor */
    GN_ENOMEM = -2,      /* device or host allocation failed */
    GN_ERANGE = -3,      /* a value does not fit: delay > ring_depth - 2, too many nodes/edges */
    GN_ECUDA = -4,       /* a CUDA runtime call failed */
    GN_ESTATE = -5,      /* call not valid in the handle's state */
    GN_ETIMEOUT = -6,    /* a bounded device-side wait gave up */
    GN_EINTERNAL = -7,   /* a device-side consistency check failed */
    GN_EOVERFLOW = -8    /* a device buffer overflowed; the data returned is what was kept */
} gn_status;

enum { GN_COUPLE_REST = 0, GN_COUPLE_RAW = 1 };

/* FitzHugh-Nagumo parameters in the paper's notation (Sec. 3.1):
 *   dV/dt = aV - bV^3 - cW + S + U + i_ext,   dW/dt = e (V + f - gW).
 * The classic (a, b, eps) = (0.7, 0.8, 0.08) model is a = 1, b = 1/3, c = 1,
 * e = 0.08, f = 0.7, g = 0.8.  A unique rest point needs g > 0, b > 0, a < c/g
 * (GN_EINVAL otherwise). */
typedef struct {
    double a, b, c, e, f, g, i_ext;
} gn_fhn_params;

/* Node models (Sec. 3.1): FitzHugh-Nagumo (the parameters above), or the
 * Izhikevich simple model with an alpha-function post-synaptic current and the
 * calcium readout (Eq. izsimple, izpsc, alphapsc, spd, casimple; Sec. 3.1-3.3),
 * forward Euler:
 *   V' = V + dt/C [k (V - v_r)(V - v_t) - W + r + U + i_ext]   if V < v_peak, else v_reset
 *   W' = W + dt a (b (V - v_r) - W)                            if V < v_peak, else W + d
 *   r' = r + dt p,   p' = p + dt (-psc_a^2 r - 2 psc_a p + S),
 *   S_j = sum_{i -> j} w_ij spd(V_i(t - tau_ij)),  spd(V) = 1 if V >= v_peak else 0
 *   c' = c + dt (-c / tau_c + spd(V)),   y = gain c' + offset + sigma xi.
 * Units are the caller's (the usual: pF, nS/mV, mV, 1/ms, nS, pA, ms).  The state
 * starts at V = v_r, W = r = p = c = 0 with no spike before t = 0; the history ring
 * holds spd(V); events are spikes (V >= v_peak) and a node's arrival is its first
 * spike.  The coupling field is ignored; the batched form does not take this model
 * (GN_EINVAL).
 *
 * Third model: Hodgkin-Huxley nodes (Sec. 3.1 and 3.4 name the model and its state
 * {v, m, n, h}; the rates are the classic squid-axon ones, modern convention, rest
 * near -65 mV) with the same alpha-function PSC, spike indicator and calcium, Euler:
 *   V' = V + dt/C [-g_na m^3 h (V - e_na) - g_k n^4 (V - e_k) - g_l (V - e_l) + r + U + i_ext]
 *   x' = x + dt (alpha_x(V) (1 - x) - beta_x(V) x),  x in {m, n, h}, with
 *   alpha_m = 0.1 (V + 40) / (1 - e^-(V+40)/10), beta_m = 4 e^-(V+65)/18,
 *   alpha_h = 0.07 e^-(V+65)/20,                 beta_h = 1 / (1 + e^-(V+35)/10),
 *   alpha_n = 0.01 (V + 55) / (1 - e^-(V+55)/10), beta_n = 0.125 e^-(V+65)/80
 *   (mV, ms; the 0/0 at -40 and -55 mV takes its limit).  r, p, c and y as above with
 *   spd(V) = 1 while V >= v_peak; no reset, and events are the upward crossings of
 *   v_peak.  The state starts at V = -65 mV with each gate at alpha / (alpha + beta)
 *   there, r = p = c = 0; W is unused (0).  The batched form does not take it. */
enum { GN_MODEL_FHN = 0, GN_MODEL_IZH = 1, GN_MODEL_HH = 2 };
typedef struct {
    double C, k, v_r, v_t, v_peak, v_reset, a, b, d, i_ext, psc_a, tau_c;
} gn_izh_params;
typedef struct {
    double C, g_na, g_k, g_l, e_na, e_k, e_l, v_peak, i_ext, psc_a, tau_c;
} gn_hh_params;

/* Spike-time-dependent plasticity (Sec. 3.2, the plasticity transition G_ij of
 * Eq. omegatrans; spiking models only).  Each node carries the time since its last
 * spike, s_j' = (1 - spd(V_j)) (s_j + dt) from s_j = 0, and every weight evolves from
 * step-n values after w_ij(n) has fed S_j(n):
 *   q_ij  = (s_i(t - tau_ij) - s_j(t)) max(spd(V_i(t - tau_ij)), spd(V_j(t)))
 *   w_ij' = w_ij + dt alpha sign(q_ij) exp(-beta |q_ij|)
 * with s and spd before t = 0 taken as 0.  alpha (weight units per ms) and beta
 * (1/ms, >= 0) are one pair for the whole network.  s is kept as a whole number of
 * steps (exact), saturating at 2^30 steps.  A plastic network runs the staged step
 * kernel (step_kernel 0 or 3; 1 and 2 fail with GN_EINVAL) in a CTA shape that reads
 * its edge entries from global memory (GN_STEP_SHAPE, default 4), chosen at create
 * time; the batched form does not take it. */
typedef struct {
    int32_t enable;
    double alpha, beta;
} gn_stdp_params;

/* Readout (Sec. 3.3): c~' = c~ + (dt/tau_ms)(v~' - c~) every step; every
 * sample_every steps y = gain (V* + c~) + offset + sigma xi, xi ~ N(0, 1) drawn
 * from Philox4x32-10 keyed by `seed` with counter (node, sample, 2).  With
 * frame_average != 0 a camera slower than the step is modelled: a sample reads the
 * mean of c~ over the sample_every steps of its frame (the values after each step)
 * instead of the last one; gn_set_state and gn_load_state start a new frame. */
typedef struct {
    double tau_ms;
    int32_t sample_every;
    float gain, offset, sigma;
    uint64_t seed;
    int32_t frame_average;
} gn_obs_params;

/* A network.  pos [n_nodes*dim] (mm, row-major); edges src[e] -> dst[e] with
 * weight[e]; delays from geometry with speed[e] (m/s = mm/ms; NULL: speed_scalar
 * for all edges), or given explicitly in whole steps by delay_steps[e] (>= 1),
 * which bypasses geometry.  Self-loops are rejected (Eq. Yjset sums over i != j);
 * repeated (i, j) pairs are separate terms. */
typedef struct {
    int32_t n_nodes;
    int32_t dim;                 /* 1, 2 or 3 */
    const double *pos;
    int64_t n_edges;
    const int32_t *src;
    const int32_t *dst;
    const float *weight;
    const double *speed;
    double speed_scalar;
    const int32_t *delay_steps;
    double dt_ms;
    gn_fhn_params fhn;
    gn_obs_params obs;
    int32_t coupling;            /* GN_COUPLE_REST: S uses V - V*; GN_COUPLE_RAW: S uses V */
    double theta;                /* event threshold on V (events: V(n) < theta <= V(n+1)) */
    int32_t ring_depth;          /* history slots, a power of two >= D_max + 2; 0 = smallest such */
    int64_t obs_capacity;        /* samples kept on the device; 0 = 1024 */
    int64_t event_capacity;      /* events kept on the device; 0 = 1 << 20 */
    int32_t renumber;            /* 0: renumber nodes in spatial (Morton) order; -1: keep the caller's order */
    int32_t edge_format;         /* 0: packed 32-bit keys when N * ring_depth <= 2^32, else 64-bit; 1: always 64-bit */
    int32_t step_kernel;         /* 0: chosen by timing the candidates on the first gn_step (autotune);
                                    1: one row block per CTA, chained launches; 2: persistent CTAs with a
                                    bulk-copy pipeline of row blocks; 3: staged tiles -- each CTA fetches
                                    the distinct (source, delay) history values of a tile of rows once into
                                    shared memory, then sums each row from there.  3 fails with GN_EINVAL
                                    if a single row needs more shared memory than a CTA may have
                                    (in-degree above about 20,000).  Every kernel sums a node's inputs
                                    in the same order, so results do not depend on this choice.  The
                                    environment variable GN_STEP_SHAPE=i picks the CTA shape of an
                                    explicitly chosen kernel 1, 3, 4 or 5 (default 0).  4: the whole
                                    network resident in one CTA's shared memory, many steps per launch.
                                    5: kernel 3's tiles in one persistent cooperative launch per call
                                    (up to 65,536 steps), each CTA holding its tile's keys and entries
                                    in shared memory for the whole launch, the CTAs meeting at a counting
                                    barrier in global memory between steps; 4 and 5 fail with GN_EINVAL
                                    if the network does not fit (5: every tile's CTA resident at once),
                                    and neither takes plastic weights.  Kernel 3 with static weights
                                    fetches its history values (all written two or more steps back)
                                    before it waits for the previous step; GN_STAGED_EARLY=0 makes it
                                    wait first */
    void *cuda_stream;           /* cudaStream_t to run on; NULL: the library makes its own */
    int32_t device;              /* CUDA device ordinal */
    int32_t model;               /* GN_MODEL_FHN (0), GN_MODEL_IZH (1) or GN_MODEL_HH (2) */
    gn_izh_params izh;           /* used when model == GN_MODEL_IZH (C > 0, tau_c > 0, all finite) */
    gn_hh_params hh;             /* used when model == GN_MODEL_HH (C > 0, tau_c > 0, all finite) */
    gn_stdp_params stdp;         /* plastic weights when stdp.enable != 0 (spiking models) */
    /* Heterogeneous cells (Sec. 3.1: cell types as parameter sets of one transition
     * function; spiking models): with 1 <= n_cell_types <= 8, node j takes parameter
     * set cell_type[j] (caller order) of izh_types or hh_types in place of izh / hh,
     * and an Izhikevich node starts at its set's v_r.  0: every node takes izh / hh. */
    int32_t n_cell_types;
    const gn_izh_params *izh_types;
    const gn_hh_params *hh_types;
    const uint8_t *cell_type;
} gn_net_desc;

/* A pulse of amplitude amp on node over [t_on_ms, t_off_ms): the steps
 * n with llround(t_on/dt) <= n < llround(t_off/dt). */
typedef struct {
    int32_t node;
    double t_on_ms, t_off_ms;
    float amp;
} gn_pulse;

/* Sizes and layout chosen at create time. */
typedef struct {
    int32_t n_nodes;
    int64_t n_edges;
    int32_t dim;
    int32_t ring_depth;
    int32_t max_delay;
    int32_t min_delay;
    int64_t n_clamped;           /* geometric delays that rounded below one step */
    int32_t edge_format;         /* 0: packed 32-bit (src << log2 R | D); 1: 64-bit (src, D) */
    int32_t n_blocks;            /* row blocks (kernels 1, 2) or tiles (kernel 3) of the step kernel */
    int32_t step_kernel;         /* 1 to 5 once chosen (0 before the first gn_step when autotuning) */
    int32_t step_threads;        /* CTA size of the chosen kernel */
    int32_t step_edges_per_thread; /* kernels 1, 2: edges per thread of a row block; 3: longest row summed
                                      by one thread (longer rows: 32 lane-strided pieces) */
    int32_t grid;                /* CTAs per step launch */
    int64_t step;                /* steps taken */
    int64_t samples;             /* samples produced */
    double v_rest, w_rest;
    size_t device_bytes;         /* device memory held by the handle */
    int64_t step_gathers;        /* history values fetched per step: n_edges for kernels 1 and 2; for
                                    kernel 3 the distinct (source, delay) pairs summed over its tiles */
    int64_t step_entries;        /* edge records read per step: n_edges for kernels 1 and 2; for kernel 3
                                    the stored entries including the padding of its slices */
    int64_t step_lane_slots;     /* kernel 3: lane slots (32 per slice of pieces); 0 for kernels 1 and 2 */
    int32_t step_cluster;        /* kernel 5: 1 if the grid runs as one thread-block cluster (at most 16 tiles,
                                    the cluster's own barrier between steps), 0 for the cooperative grid */
} gn_net_info;

typedef struct gn_net gn_net;

/* Build a network on the device: copy the inputs, quantise the delays in FP64
 * on the GPU (D = max(1, llround(|x_i - x_j| / (s dt))), Sec. 3.2.1, Eq. delaydist),
 * renumber the nodes in Morton order, build the by-target edge list (CSR) and
 * put every node at rest with a resting history.  *out receives the handle.
 * GN_EINVAL: bad descriptor (NaN position, speed <= 0, id out of range,
 * self-loop, dt <= 0, no unique rest point); GN_ERANGE: a delay does not fit
 * the ring; GN_ENOMEM / GN_ECUDA as named. */
GN_API gn_status gn_net_create(const gn_net_desc *desc, gn_net **out);

/* Free every device and host resource of the handle (NULL is a no-op). */
GN_API gn_status gn_net_destroy(gn_net *net);

GN_API gn_status gn_net_get_info(const gn_net *net, gn_net_info *info);

/* The whole-step delay of every edge, in the caller's edge order ([n_edges]). */
GN_API gn_status gn_get_delays(const gn_net *net, int32_t *out);

/* The isolated rest point (V*, W*) in FP64 (Sec. 3.1 FHN with S = U = 0). */
GN_API gn_status gn_get_rest(const gn_net *net, double *v_rest, double *w_rest);

/* Replace the pulse set (u_j of Eq. Htrans).  Pulses on the same node add. */
GN_API gn_status gn_set_stimulus(gn_net *net, const gn_pulse *pulses, int32_t n_pulses);

/* Background pulses: at every step a node starts, with probability
 * p = rate_hz * dt, a pulse of amplitude amp lasting llround(dur_ms/dt) steps;
 * an onset during a pulse restarts its count.  The draw at step n for node j is
 * the first word of Philox4x32-10 keyed by `seed` at counter (j, n, 1), compared
 * with floor(p 2^32).  rate_hz = 0 turns it off. */
GN_API gn_status gn_set_background(gn_net *net, double rate_hz, float amp, double dur_ms, uint64_t seed);

/* Advance n_steps steps of dt (asynchronous).  Each step is one launch of the
 * fused step kernel: delayed gather, FHN update, history write, readout, noise,
 * events and first arrivals. */
GN_API gn_status gn_step(gn_net *net, int64_t n_steps);

/* Wait for the net's stream; reports device-side errors. */
GN_API gn_status gn_synchronize(gn_net *net);

/* Copy up to max_samples observation rows not yet read, oldest first, into
 * out[k][n_nodes] (host, caller node order), and advance the read cursor.
 * *first_sample (may be NULL) receives the sample number of row 0 (sample k is
 * taken after step (k+1) * sample_every).  out == NULL discards the rows instead
 * of copying them.  If more than obs_capacity samples
 * were produced since the last read, the oldest are lost and GN_EOVERFLOW is
 * returned with the kept rows copied. */
GN_API gn_status gn_observe(gn_net *net, float *out, int64_t max_samples, int64_t *first_sample,
                     int64_t *written);

/* As gn_observe (the same rows, the read cursor advanced the same way), but the
 * copies are queued on a copy stream behind the steps taken so far and the call
 * returns at once, so later gn_step calls overlap them (with pinned `out`).  `out`
 * must stay valid until gn_observe_wait or gn_synchronize returns, and until then
 * the steps may produce at most obs_capacity - *written new samples (more would
 * wrap onto the device rows still being copied).  GN_EOVERFLOW as gn_observe. */
GN_API gn_status gn_observe_async(gn_net *net, float *out, int64_t max_samples, int64_t *first_sample,
                                  int64_t *written);
/* Wait for the copies gn_observe_async queued (not for later steps). */
GN_API gn_status gn_observe_wait(gn_net *net);

/* State relative to rest, caller node order.  Any pointer may be NULL. */
GN_API gn_status gn_get_state(gn_net *net, float *v, float *w, float *c, int32_t *bg_count, int64_t *step);

/* Set the dynamic state (initial conditions y_j(t0), Sec. 2) at step `step`:
 * hist[k][j] = v~_j(step - k) for k < depth (1 <= depth <= ring_depth; older slots
 * are set to rest), w~ and c~ (NULL = 0) and background counters (NULL = 0), all
 * in caller node order.  First arrivals are reset to -1, the event list is
 * cleared and the observation cursor moves to the first sample after `step`. */
GN_API gn_status gn_set_state(gn_net *net, const float *hist, int32_t depth, const float *w, const float *c,
                              const int32_t *bg_count, int64_t step);

/* Spiking models only (Izhikevich or Hodgkin-Huxley; GN_EINVAL otherwise): V, the
 * PSC variables r and p, in caller node order (any pointer may be NULL).
 * gn_get_state / gn_set_state carry W (0 for Hodgkin-Huxley) and calcium in w and
 * c, and the history is spd(V) in {0, 1}; gn_get_state's v is V as well. */
GN_API gn_status gn_get_izh_state(gn_net *net, float *V, float *r, float *p);
GN_API gn_status gn_set_izh_state(gn_net *net, const float *V, const float *r, const float *p);

/* Hodgkin-Huxley model only (GN_EINVAL otherwise): the gates m, n, h in caller node
 * order (any pointer may be NULL; a set leaves a NULL gate as it is). */
GN_API gn_status gn_get_hh_gates(gn_net *net, float *m, float *n, float *h);
GN_API gn_status gn_set_hh_gates(gn_net *net, const float *m, const float *n, const float *h);

/* History: out[k][j] = v~_j(step - k), k = 0..depth-1, depth <= ring_depth (spiking
 * models: spd(V) in {0, 1}). */
GN_API gn_status gn_get_history(gn_net *net, float *out, int32_t depth);

/* Plastic networks only (GN_EINVAL otherwise).  The current weights in the caller's
 * edge order ([n_edges]; set takes effect from the next step). */
GN_API gn_status gn_get_weights(gn_net *net, float *w);
GN_API gn_status gn_set_weights(gn_net *net, const float *w);
/* The time since the last spike, s_hist[k][j] = s_j(step - k) in ms, k < depth <=
 * ring_depth (k = 0: the current s).  The set rounds each value to whole steps and
 * keeps the spike history; call it after gn_set_state, which sets s to 0. */
GN_API gn_status gn_get_stdp_history(gn_net *net, float *s_hist, int32_t depth);
GN_API gn_status gn_set_stdp_history(gn_net *net, const float *s_hist, int32_t depth);

/* First step at which v~_j became non-zero ([n_nodes], -1 = not yet). */
GN_API gn_status gn_get_arrivals(gn_net *net, int64_t *first_arrival);

/* Events (upward crossings of theta), sorted by (step, node), caller node ids.
 * *n_total receives the number recorded; up to cap are copied.  GN_EOVERFLOW if
 * the device buffer overflowed (then the kept ones are returned). */
GN_API gn_status gn_get_events(gn_net *net, int32_t *node, int64_t *step, int64_t cap, int64_t *n_total);

/* Checkpoint: the dynamic state (history ring, w~, c~, background counters,
 * first arrivals, step counter).  With buf == NULL, *used receives the size
 * needed.  Restoring into a handle created from the same descriptor makes the
 * continuation bit-identical to an uninterrupted run. */
GN_API gn_status gn_save_state(gn_net *net, void *buf, size_t cap, size_t *used);
GN_API gn_status gn_load_state(gn_net *net, const void *buf, size_t size);

/* ---------------------------------------------------------------------------
 * Batched form: many independent networks (of any sizes) advanced together,
 * from captured CUDA graphs, by one of two kernels: a persistent launch per
 * gn_batch_step whose CTAs take networks from a work queue ordered largest first
 * and run all the requested steps of a network before taking the next (kernel 1),
 * or the staged tiles of every member, one launch per step (kernel 3, with the
 * schedules described at gn_batch_step).  Every network of a batch uses one node
 * model; spiking batches run the staged form only, and plastic weights are not
 * taken (GN_EINVAL).  The kernel, its CTA size and schedule are chosen by timing
 * the candidates on the first gn_batch_step.  Every network follows the
 * same model and conventions as gn_net (Sec. 2, 3.1, 3.2.1, 3.3); per-network
 * calls take the network's index in the descriptor array.
 * ------------------------------------------------------------------------- */
typedef struct gn_batch gn_batch;

typedef struct {
    int32_t n_nets;
    int64_t n_nodes;             /* over all networks */
    int64_t n_edges;
    int64_t step;                /* common step counter */
    int32_t cta_threads;         /* chosen CTA size (0 before the first step) */
    int32_t grid;                /* CTAs per launch: persistent CTAs (kernel 1) or tiles (kernel 3) */
    size_t device_bytes;
    int32_t step_kernel;         /* 1: persistent k_batch, one launch per gn_batch_step; 3: staged tiles of
                                    every member, one launch per step; 5: the staged tile step in one
                                    persistent cooperative launch per 64-step chunk; 0 before the first step */
    int32_t step_groups;         /* kernels 3 and 5: member groups, each stepped through a 64-step chunk at a
                                    time (1: every member every step; see gn_batch_step); else 0 */
    int32_t step_lanes;          /* kernels 3 and 5: groups stepped concurrently (3: one chain of launches
                                    each; 5: one lane of the launch's CTAs each); else 0 */
} gn_batch_info;

/* Copy and build n_nets networks on one device (descs[i].device must agree; the
 * stream of descs[0] is used; obs_capacity of descs[0] applies to all, 0 = 256).
 * Errors as gn_net_create, for the first network that fails. */
GN_API gn_status gn_batch_create(const gn_net_desc *descs, int32_t n_nets, gn_batch **out);
GN_API gn_status gn_batch_destroy(gn_batch *batch);
GN_API gn_status gn_batch_get_info(const gn_batch *batch, gn_batch_info *info);
GN_API gn_status gn_batch_get_net_info(const gn_batch *batch, int32_t net, gn_net_info *info);
GN_API gn_status gn_batch_get_delays(const gn_batch *batch, int32_t net, int32_t *out);

/* Replace every network's pulses at once: network i takes counts[i] consecutive
 * entries of `pulses` (caller node ids of network i). */
GN_API gn_status gn_batch_set_stimulus_all(gn_batch *batch, const gn_pulse *pulses, const int32_t *counts);
GN_API gn_status gn_batch_set_background(gn_batch *batch, int32_t net, double rate_hz, float amp, double dur_ms,
                                         uint64_t seed);

/* Advance every network n_steps (asynchronous): one persistent launch (kernel 1),
 * one launch per step replayed from a captured graph (kernel 3) or one persistent
 * cooperative launch per 64-step chunk (kernel 5, the same tile step), whichever
 * the first call measured faster; GN_BATCH_KERNEL=1 or 3 in the environment
 * restricts the choice to that kernel.  Kernel 3 has several schedules, also timed
 * on the first call: every member every step, or (L2 blocking) contiguous groups
 * of members, each group stepped through the 64 steps of a graph chunk at a time
 * so that its steps read from L2, with 1, 2 or 4 groups in flight at once (lanes:
 * one chain of launches each, on streams forked from the batch's stream).  Kernel
 * 5 runs the blocked schedule in 1, 2, 4 or 8 lanes of one launch's CTAs (every
 * CTA the device holds at once), a lane's CTAs meeting at a counting barrier in
 * global memory after each step instead of a launch boundary.  The groups in
 * flight share an L2 budget for their per-step working sets -- edge entries,
 * gather keys, live history slots, node state -- of GN_BATCH_GROUP_KB (default
 * 80 MB; 0 turns the blocking off); GN_BATCH_LANES=1..8 fixes the lanes,
 * GN_BATCH_KERNEL=4 takes kernel 3's blocked schedule and GN_BATCH_KERNEL=5
 * kernel 5, without timing.  The networks are independent, so neither the kernel
 * nor the schedule changes a result: all sum a node's inputs in the order of the
 * single-network kernels, and results are bit-identical either way.  Spiking
 * batches run kernel 3 or 5.  A bounded wait of kernel 5 that gives up (its copy
 * waits, its barrier polls) records a timeout that the next synchronising call
 * reports as GN_ETIMEOUT. */
GN_API gn_status gn_batch_step(gn_batch *batch, int64_t n_steps);
GN_API gn_status gn_batch_synchronize(gn_batch *batch);

/* Per-network views, as the gn_net calls of the same name. */
GN_API gn_status gn_batch_observe(gn_batch *batch, int32_t net, float *out, int64_t max_samples,
                                  int64_t *first_sample, int64_t *written);
GN_API gn_status gn_batch_get_state(gn_batch *batch, int32_t net, float *v, float *w, float *c, int32_t *bg_count,
                                    int64_t *step);
GN_API gn_status gn_batch_get_history(gn_batch *batch, int32_t net, float *out, int32_t depth);
GN_API gn_status gn_batch_get_izh_state(gn_batch *batch, int32_t net, float *V, float *r, float *p);
GN_API gn_status gn_batch_get_hh_gates(gn_batch *batch, int32_t net, float *m, float *n, float *h);
GN_API gn_status gn_batch_get_arrivals(gn_batch *batch, int32_t net, int64_t *first_arrival);
GN_API gn_status gn_batch_get_events(gn_batch *batch, int32_t net, int32_t *node, int64_t *step, int64_t cap,
                                     int64_t *n_total);

/* Advance every network n_steps like gn_batch_step, but without allocating any
 * memory: no cudaMalloc, cudaFree or other allocating routine is called.  This is
 * for callers that cannot allocate device memory while they step -- a real-time
 * control loop that must not take an allocator's latency or locks, or a program
 * whose device memory is handed out from a fixed arena owned by someone else.
 * gn_batch_step may allocate: on its first call it times candidate CTA sizes on
 * scratch copies of the state, and it instantiates a new CUDA graph whenever
 * n_steps changes.  This call launches the kernel directly, with the CTA size an
 * earlier gn_batch_step chose (or the default one), and takes the launch's work
 * queue -- its counter and largest-first schedule -- from a fixed device array
 * inside the library instead of the batch's memory.  The paper has no
 * counterpart; this is a deployment entry point.
 *   Limit: batches of at most 65,536 networks (GN_ERANGE beyond).
 *   The first call on a device looks up that array's device address (once per
 *   device, under a lock), so make the first call on each device before any stream
 *   capture begins.  Each call copies the batch's schedule into the array from the
 *   batch's own device memory (device to device, in stream order: the host does not
 *   wait) and advances the batch's step count on the host when the call is made.
 *   The array is shared by every call in the process and keeps the last call's
 *   contents (the counter is cleared and the schedule rewritten before each
 *   launch); calls that overlap on the GPU -- on different streams, or for
 *   different batches at the same time -- race on it and must be serialised. */
GN_API gn_status gn_batch_step_static(gn_batch *batch, int64_t n_steps);

/* Move the common step counter (clears every network's events and resets the
 * observation cursors), then set one network's state at that step as
 * gn_set_state does. */
GN_API gn_status gn_batch_set_step(gn_batch *batch, int64_t step);
GN_API gn_status gn_batch_set_state(gn_batch *batch, int32_t net, const float *hist, int32_t depth, const float *w,
                                    const float *c, const int32_t *bg_count);

/* ---------------------------------------------------------------------------
 * Connectivity estimator.  Correlating the activity of two cells is the common way
 * to map functional connections (Sec. 1); the framework's test networks exist to
 * score such mappings against a known topology (Sec. 3.5, Sec. 4).
 * ------------------------------------------------------------------------- */

/* Node-major traces of every network of a batch: out[(o_i + j) * n_samples + t] =
 * observation sample first_sample + t of node j (caller order) of network i, with
 * o_i the number of nodes of networks 0 .. i-1.  `out` is a device buffer of
 * (total nodes) x n_samples floats.  GN_ERANGE if a sample was not taken yet or no
 * longer held (obs_capacity). */
GN_API gn_status gn_batch_export_traces(gn_batch *batch, int64_t first_sample, int32_t n_samples, float *out);

/* Lagged normalised cross-correlation features of candidate pairs i -> j, all
 * pointers on the device.  traces [n_nodes][n_samples] (node-major), pos
 * [n_nodes][dim] (mm), pairs src/dst [n_pairs] (every entry in [0, n_nodes): the
 * kernel gathers traces and positions by them unchecked), radius [n_pairs] (the
 * candidate radius r_c of the pair's network).  With d = |x_i - x_j| and the first lag
 * l0 = floor((d / v_max) / sample_ms) (the shortest delay, Sec. 3.2.1), feature k < 32
 * is the Pearson correlation of y_i(t) and y_j(t + l0 + k) over their overlap, each
 * segment about its own mean (0 if one is constant); feature 32 is d / r_c.
 * features [n_pairs][33]; score [n_pairs] = max of features 0..31 (the plain
 * peak-correlation estimator).  Runs on `cuda_stream` (may be NULL); takes stream-
 * ordered scratch of about 3 x the traces (centred traces and their prefix sums),
 * GN_ECUDA if it cannot be allocated. */
GN_API gn_status gn_xcorr_features(const float *traces, int64_t n_nodes, int32_t n_samples, const double *pos,
                                   int32_t dim, int64_t n_pairs, const int32_t *src, const int32_t *dst,
                                   const double *radius, double v_max, double sample_ms, float *features,
                                   float *score, void *cuda_stream);

/* Learned estimator: an MLP in_dim -> 256 -> 256 -> 1 (ReLU, sigmoid output)
 * trained on labelled candidate pairs with binary cross-entropy and AdamW
 * (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay).  BF16 tensor-core GEMMs
 * with FP32 accumulation; inputs, weight copies, the first hidden activation and
 * the backward activations are BF16, masters and reductions FP32, every reduction
 * in a fixed order.  Parameters are exchanged as one packed FP32 host array
 * [W1 (in_dim x 256, row-major) | b1 (256) | W2 (256 x 256) | b2 | w3 (256) | b3 (1)];
 * X [rows][in_dim], y [rows] and p [B] are device buffers; with idx (device int64
 * [B], may be NULL; every entry in [0, rows): rows are gathered by it unchecked)
 * row b of the batch is X[idx[b]] / y[idx[b]], so a resident training set is
 * visited in any order without copies. */
typedef struct gn_mlp gn_mlp;
GN_API gn_status gn_mlp_create(int32_t in_dim, int32_t max_batch, const float *params, int32_t device,
                               void *cuda_stream, gn_mlp **out);
GN_API gn_status gn_mlp_destroy(gn_mlp *mlp);
GN_API gn_status gn_mlp_get_params(gn_mlp *mlp, float *params);
/* Gradients of the mean loss over the batch (packed layout, host) without an update. */
GN_API gn_status gn_mlp_gradients(gn_mlp *mlp, const float *X, const float *y, const int64_t *idx, int32_t B,
                                  float *grads, float *loss);
/* One AdamW step on one batch (B <= max_batch); *loss (may be NULL) receives the mean loss. */
GN_API gn_status gn_mlp_train_step(gn_mlp *mlp, const float *X, const float *y, const int64_t *idx, int32_t B,
                                   float lr, float weight_decay, float *loss);
/* n_batches AdamW steps in one call: step j trains on rows idx[j B .. (j + 1) B)
 * of X / y (idx: device int64 with n_batches * B entries, e.g. an epoch's
 * permutation).  One step is captured as a CUDA graph, the batch picked by a
 * device-side cursor, and replayed n_batches times, so the host issues one graph
 * launch per step; the result is bit-identical to n_batches gn_mlp_train_step calls
 * on the same slices.  losses (host [n_batches], may be NULL) receives each step's
 * mean loss, after which the call has synchronised; without it the call is
 * asynchronous. */
GN_API gn_status gn_mlp_train_epoch(gn_mlp *mlp, const float *X, const float *y, const int64_t *idx,
                                    int32_t n_batches, int32_t B, float lr, float weight_decay, float *losses);
/* Probabilities p = sigmoid(MLP(X)) for any number of rows (asynchronous). */
GN_API gn_status gn_mlp_infer(gn_mlp *mlp, const float *X, int64_t B, float *p);
GN_API gn_status gn_mlp_synchronize(gn_mlp *mlp);

/* Scores of a mapping (host buffers): area under the ROC curve (Mann-Whitney U
 * with mid-ranks for ties; NaN if one class is empty), F1 of "edge iff score >=
 * threshold", and the threshold among the scores that maximises F1. */
GN_API gn_status gn_score_auroc(const float *scores, const uint8_t *labels, int64_t n, double *auroc);
GN_API gn_status gn_score_f1(const float *scores, const uint8_t *labels, int64_t n, double threshold, double *f1);
GN_API gn_status gn_score_best_f1(const float *scores, const uint8_t *labels, int64_t n, double *threshold,
                                  double *f1);

/* Thread-local message of the last failing call ("" if none). */
GN_API const char *gn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GEONET_H */
