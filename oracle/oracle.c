/*
 * oracle.c -- plain, slow, FP64 reference of the delayed geometric-network
 * simulation of Buibas & Silva, "A framework for simulating and estimating the
 * state and functional topology of complex dynamic geometric networks"
 * (arXiv:0908.3934).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the timed
 * CPU baseline of the benchmark may load this library.  It shares no code,
 * header, table or helper with the CUDA library: the two sides meet only in
 * the seeded input generators.
 *
 * What it computes, in the paper's order:
 *   - geodesic delays tau_ij = |x_i - x_j| / s                (Eq. delaydist, Sec. 3.2.1;
 *     quantised to whole steps of dt                           Eq. gendelay, Sec. 2)
 *   - the delayed, weighted input of node j,
 *       S_j(t) = sum_{i -> j} w_ij * v_i(t - tau_ij)           (Eq. Yjset, Sec. 2)
 *   - the FitzHugh-Nagumo transition, forward Euler            (Eq. difform + the Euler form, Sec. 3.1;
 *       V' = V + dt (aV - bV^3 - cW + S + U)                    FHN pair and Eq. fnstate, Sec. 3.1)
 *       W' = W + dt  e (V + f - gW)
 *   - the control input U_j(t)                                 (u_j in Eq. Htrans, Sec. 2)
 *   - a linear low-pass readout of V and a noisy observation   (calcium model and fluorescence
 *       I = n c + b + N(0, gamma^2)                             readout, Sec. 3.3; Eq. obsfun, Sec. 2)
 *
 * Readings where the paper is silent (each is listed in the design notes):
 *   - D = max(1, llround(tau/dt)): half away from zero; a zero delay would need a
 *     same-step value inside an explicit step, so it is clamped to one step.
 *   - Coupling REST: S uses the voltage relative to the isolated rest point,
 *     v~ = V - V*, so an unstimulated network stays exactly at rest.  Coupling RAW
 *     uses V itself (V* for times before t = 0).
 *   - The state is held relative to the rest point (v~ = V - V*, w~ = W - W*);
 *     the FHN polynomial is expanded about (V*, W*) with the binomial theorem,
 *     the constant part being zero by definition of the rest point.
 *   - Jacobi step: every update reads only step-n values (Sec. 2, the component list
 *     under Eq. Hj advances each variable from time t).
 *   - Readout c: forward Euler of dc/dt = (v - c)/tau (the calcium model's Euler form
 *     with the voltage in place of the spike train), sampled every `sample_every` steps;
 *     y = gain (V* + c~) + offset + sigma xi.
 *   - Camera frame averaging (frame_average = 1; Sec. 3.3 notes that a camera slower
 *     than the step averages the calcium values of a frame): a sample reads the mean
 *     of c over the sample_every steps of its frame, the values after each step.  A
 *     run starts a new frame.
 *   - Events: upward crossing of V through theta (V(n) < theta <= V(n+1)).
 *   - Arrival: first step at which v~ becomes non-zero.
 *
 * Second node model (model = 1): the Izhikevich simple model with an alpha-function
 * post-synaptic current and the calcium readout, all in their forward-Euler forms
 * (Eq. izsimple / izpsc, Eq. alphapsc, Eq. spd, Eq. casimple, Sec. 3.1-3.3):
 *       V' = V + dt/C [k (V - Vr)(V - Vt) - W + r + U + I]   if V < V_peak, else V_reset
 *       W' = W + dt a (b (V - Vr) - W)                       if V < V_peak, else W + d
 *       r' = r + dt p
 *       p' = p + dt (-a_s^2 r - 2 a_s p + S),   S_j = sum_{i -> j} w_ij spd(V_i(t - tau_ij))
 *       c' = c + dt (-c / tau_c + spd(V)),      spd(V) = 1 if V >= V_peak else 0
 *       y  = gain c' + offset + sigma xi
 *   The history holds spd(V) (the only quantity another node reads, Sec. 3.2.1); the
 *   state V, W, r, p, c is absolute; the model starts from V = Vr, W = r = p = c = 0
 *   (the fixed point without input), with no spike before t = 0.  Events are spikes
 *   (V(n+1) >= V_peak) and the arrival of a node is its first spike.
 *
 * Third node model (model = 2): Hodgkin-Huxley (the paper names it, Sec. 3.1 and
 * 3.4, with four state variables {v, m, n, h}; the equations are the classic squid
 * axon ones in the modern convention, rest near -65 mV), with the same
 * alpha-function PSC, spike indicator and calcium readout as model 1:
 *       V' = V + dt/C [-gNa m^3 h (V - ENa) - gK n^4 (V - EK) - gL (V - EL) + r + U + I]
 *       x' = x + dt (alpha_x(V) (1 - x) - beta_x(V) x),   x in {m, n, h}
 *   alpha_m = 0.1 (V + 40) / (1 - e^-(V+40)/10), beta_m = 4 e^-(V+65)/18,
 *   alpha_h = 0.07 e^-(V+65)/20,                 beta_h = 1 / (1 + e^-(V+35)/10),
 *   alpha_n = 0.01 (V + 55) / (1 - e^-(V+55)/10), beta_n = 0.125 e^-(V+65)/80,
 *   the removable 0/0 at V = -40, -55 evaluated as x / (-expm1(-x / y)) (limit y).
 *   No reset: spd(V) = 1 while V >= V_peak; events are upward crossings of V_peak.
 *   The state starts at V = -65 mV with each gate at alpha / (alpha + beta) there.
 *
 * Plasticity (stdp = 1, spiking models; Sec. 3.2, the plasticity transition G_ij of
 * Eq. omegatrans): each node carries the time since its last spike,
 *       s_j' = (1 - spd(V_j)) (s_j + dt),                      s_j(0) = 0,
 *   and every weight evolves from step-n values, after w_ij(n) has fed S_j(n):
 *       q_ij = (s_i(t - tau_ij) - s_j(t)) max(spd(V_i(t - tau_ij)), spd(V_j(t)))
 *       w_ij' = w_ij + dt alpha sign(q_ij) exp(-beta |q_ij|)
 *   with s and spd before t = 0 taken as 0 (no spike yet).  alpha and beta are one
 *   pair for the whole network.
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), written from the
 * published definition; Box-Muller (1958) for the Gaussian.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared oracle.c -o liboracle.so -lm
 * (no FMA contraction: the delay quantisation must round exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL -1
#define ORC_ENOMEM -2
#define ORC_MAX_TYPES 8   /* cell types of a heterogeneous network */

/* ------------------------------------------------------------------------- */
/* Philox4x32-10 (Salmon et al., SC'11): 10 rounds of the 4x32 S-box
 * with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key increments
 * 0x9E3779B9 / 0xBB67AE85, the key being bumped before every round but the first. */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Counter layout shared by definition (not by code) with the CUDA side:
 *   ctr = {node, index_lo, index_hi, stream}, key = {seed_lo, seed_hi}. */
static void draw(uint64_t seed, uint32_t node, int64_t index, uint32_t stream, uint32_t out[4])
{
    uint32_t ctr[4] = {node, (uint32_t)((uint64_t)index & 0xffffffffu),
                       (uint32_t)((uint64_t)index >> 32), stream};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, out);
}

#define STREAM_BACKGROUND 1u
#define STREAM_OBSERVATION 2u

/* Standard normal from one Philox draw: Box-Muller on the top 23 bits of two words,
 * u = (k + 1/2) 2^-23, so u lies strictly inside (0, 1). */
double orc_gauss(uint64_t seed, uint32_t node, int64_t sample)
{
    uint32_t r[4];
    draw(seed, node, sample, STREAM_OBSERVATION, r);
    double u1 = ((double)(r[0] >> 9) + 0.5) * (1.0 / 8388608.0);
    double u2 = ((double)(r[1] >> 9) + 0.5) * (1.0 / 8388608.0);
    return sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
}

/* Per-step onset probability p = rate * dt, as a 32-bit threshold:
 * an onset happens at step n iff the first Philox word is below it. */
uint32_t orc_bg_threshold(double rate_hz, double dt_ms)
{
    double p = (rate_hz * dt_ms) / 1000.0;
    if (!(p > 0.0)) return 0u;
    double t = floor(ldexp(p, 32));
    if (t >= 4294967295.0) return 4294967295u;
    return (uint32_t)t;
}

int orc_bg_onset(uint64_t seed, uint32_t node, int64_t step, uint32_t threshold)
{
    uint32_t r[4];
    draw(seed, node, step, STREAM_BACKGROUND, r);
    return r[0] < threshold;
}

/* ------------------------------------------------------------------------- */
/* Rest point of the isolated FHN node (S = U = 0): the W-nullcline gives
 * W = (V + f)/g, and V solves a V - b V^3 - c (V + f)/g + I = 0.  For
 * a < c/g the left side is strictly decreasing, so the root is unique;
 * it is bracketed, bisected, then polished by Newton. */
int orc_rest_point(double a, double b, double c, double f, double g, double i_ext,
                   double *v_rest, double *w_rest)
{
    if (!(g > 0.0) || !(b > 0.0) || !(a < c / g)) return ORC_EINVAL;
    double lo = -1.0, hi = 1.0;
#define RP_F(v) (a * (v) - b * (v) * (v) * (v) - c * ((v) + f) / g + i_ext)
    while (RP_F(lo) < 0.0) lo *= 2.0;   /* F(-inf) = +inf */
    while (RP_F(hi) > 0.0) hi *= 2.0;   /* F(+inf) = -inf */
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (RP_F(mid) > 0.0) lo = mid; else hi = mid;
    }
    double v = 0.5 * (lo + hi);
    for (int it = 0; it < 3; ++it) {
        double fp = a - 3.0 * b * v * v - c / g;
        v = v - RP_F(v) / fp;
    }
#undef RP_F
    *v_rest = v;
    *w_rest = (v + f) / g;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
/* Delay quantisation: tau = |x_src - x_dst| / s (Eq. delaydist, Sec. 3.2.1),
 * D = max(1, llround(tau / dt)) with s*dt formed first.  Distances in mm,
 * speeds in m/s (= mm/ms), dt in ms.  `speed` may be NULL, then `speed_scalar`
 * applies to every edge.  clamped[e] = 1 where the rounded value was < 1. */
int orc_delays(int32_t n_nodes, int32_t dim, const double *pos, int64_t n_edges,
               const int32_t *src, const int32_t *dst, const double *speed,
               double speed_scalar, double dt_ms, int32_t *delay, uint8_t *clamped)
{
    if (dim < 1 || dim > 3 || !(dt_ms > 0.0)) return ORC_EINVAL;
    for (int64_t e = 0; e < n_edges; ++e) {
        int32_t i = src[e], j = dst[e];
        if (i < 0 || i >= n_nodes || j < 0 || j >= n_nodes) return ORC_EINVAL;
        double sum = 0.0;
        for (int k = 0; k < dim; ++k) {
            double diff = pos[(int64_t)i * dim + k] - pos[(int64_t)j * dim + k];
            sum = sum + diff * diff;
        }
        double dist = sqrt(sum);
        double s = speed ? speed[e] : speed_scalar;
        if (!(s > 0.0)) return ORC_EINVAL;
        double q = dist / (s * dt_ms);
        long long d = llround(q);
        uint8_t cl = 0;
        if (d < 1) { d = 1; cl = 1; }
        if (d > 2147483647LL) return ORC_EINVAL;
        delay[e] = (int32_t)d;
        if (clamped) clamped[e] = cl;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- */
typedef struct {
    int32_t n_nodes;
    int64_t n_edges;
    const int32_t *src;      /* [E] source i of edge i -> j */
    const int32_t *dst;      /* [E] target j */
    const double *weight;    /* [E] omega_ij */
    const int32_t *delay;    /* [E] whole steps, >= 1 */
    double dt_ms;
    /* FHN in the paper's notation (Sec. 3.1): dV = aV - bV^3 - cW + S + U + I_ext,
     * dW = e (V + f - gW). */
    double a, b, c, e, f, g, i_ext;
    int32_t coupling;        /* 0 = REST (v - V*), 1 = RAW (V) */
    double theta;            /* event threshold on V */
    /* readout */
    double tau_ms;
    int32_t sample_every;
    double gain, offset, sigma;
    uint64_t obs_seed;
    /* explicit pulses: amp on node during steps [on, off) */
    int32_t n_pulses;
    const int32_t *p_node;
    const int64_t *p_on;
    const int64_t *p_off;
    const double *p_amp;
    /* background: Bernoulli onsets per step, each starting a pulse of `bg_width`
     * steps of amplitude bg_amp; a new onset restarts the count (no stacking). */
    uint32_t bg_threshold;   /* 0 = off */
    double bg_amp;
    int32_t bg_width;
    uint64_t bg_seed;
    /* node model: 0 = FitzHugh-Nagumo (above), 1 = Izhikevich + alpha PSC + calcium */
    int32_t model;
    double iz_C, iz_k, iz_vr, iz_vt, iz_vpeak, iz_vreset, iz_a, iz_b, iz_d, iz_iext;
    double psc_a;            /* alpha-function rate a_s (1/ms) */
    double tau_c;            /* calcium removal time (ms) */
    /* model 2: Hodgkin-Huxley */
    double hh_C, hh_gna, hh_gk, hh_gl, hh_ena, hh_ek, hh_el, hh_vpeak, hh_iext;
    /* spike-time-dependent plasticity of every weight (spiking models only) */
    int32_t stdp;
    double stdp_alpha, stdp_beta;
    /* camera frame averaging: a sample reads the mean of the readout state over the
     * sample_every steps of its frame instead of its last value */
    int32_t frame_average;
    /* heterogeneous cells (spiking models): node j takes parameter set cell_type[j] of
     * n_types rows of `types`, each (C, k, v_r, v_t, v_peak, v_reset, a, b, d, i_ext,
     * psc_a, tau_c) for model 1 or (C, g_Na, g_K, g_L, E_Na, E_K, E_L, v_peak, i_ext,
     * psc_a, tau_c) for model 2, in place of the fields above */
    int32_t n_types;
    const double *types;
    const uint8_t *cell_type;
} orc_net;

typedef struct {
    double *v, *w, *c;        /* [N] final state relative to rest (required) */
    double *y;                /* [n_samples * N] observations, or NULL */
    double *y_clean;          /* [n_samples * N] observations without noise, or NULL */
    int32_t *first_arrival;   /* [N] first step n+1 with v~ != 0, -1 = none (or NULL) */
    double *first_value;      /* [N] v~ at that step (or NULL) */
    int32_t *ev_node;         /* [ev_cap] */
    int64_t *ev_step;         /* [ev_cap] */
    int64_t ev_cap;
    int64_t ev_count;         /* out: total events (may exceed ev_cap) */
    int32_t snap_every;       /* > 0: store the state after every snap_every steps */
    double *snap_v, *snap_w, *snap_c; /* [n_steps/snap_every * N] */
    int32_t *bg_count;        /* [N] final background counters (or NULL) */
    double *hist_out;         /* [hist_out_depth * N]: v~_j(n_end - k), k < hist_out_depth (or NULL) */
    int32_t hist_out_depth;   /* <= D_max + 1 */
    double *r, *p;            /* models 1, 2: [N] final PSC state (or NULL) */
    double *m, *n, *h;        /* model 2: [N] final gates (or NULL) */
    double *min_peak_gap;     /* model 1: [N] min over the run of |V - V_peak| (or NULL) */
    double *w_final;          /* stdp: [E] weights at the end (or NULL) */
    double *s;                /* stdp: [N] time since the last spike at the end (or NULL) */
    double *hist_s_out;       /* stdp: [hist_out_depth * N] s_j(n_end - k) (or NULL) */
} orc_out;

/* One Euler step of one node (the FHN transition about the rest point).
 * Expanding a(V*+v) - b(V*+v)^3 - c(W*+w) + I and dropping the rest-point
 * identity aV* - bV*^3 - cW* + I = 0 leaves
 *   a v - b (3 V*^2 v + 3 V* v^2 + v^3) - c w;
 * likewise e((V*+v) + f - g(W*+w)) = e (v - g w) since V* + f - g W* = 0. */
static void node_step(const orc_net *net, double v_rest, double v, double w, double c,
                      double S, double U, double *v1, double *w1, double *c1)
{
    double dt = net->dt_ms;
    double dv = net->a * v
              - net->b * (3.0 * v_rest * v_rest * v + 3.0 * v_rest * v * v + v * v * v)
              - net->c * w + S + U;
    double dw = net->e * (v - net->g * w);
    double vn = v + dt * dv;
    double wn = w + dt * dw;
    double cn = c + (dt / net->tau_ms) * (vn - c);
    *v1 = vn; *w1 = wn; *c1 = cn;
}

/* One Euler step of the Izhikevich + alpha-PSC + calcium node (model 1). */
static void izh_step(const orc_net *net, double V, double W, double r, double p, double c, double S, double U,
                     double *V1, double *W1, double *r1, double *p1, double *c1)
{
    double dt = net->dt_ms;
    double spike = V >= net->iz_vpeak ? 1.0 : 0.0;
    if (V < net->iz_vpeak) {
        *V1 = V + dt / net->iz_C * (net->iz_k * (V - net->iz_vr) * (V - net->iz_vt) - W + r + U + net->iz_iext);
        *W1 = W + dt * net->iz_a * (net->iz_b * (V - net->iz_vr) - W);
    } else {
        *V1 = net->iz_vreset;
        *W1 = W + net->iz_d;
    }
    *r1 = r + dt * p;
    *p1 = p + dt * (-net->psc_a * net->psc_a * r - 2.0 * net->psc_a * p + S);
    *c1 = c + dt * (-c / net->tau_c + spike);
}

/* x / (1 - exp(-x / y)), its limit y at x = 0 */
static double hh_trap(double x, double y)
{
    return x == 0.0 ? y : x / -expm1(-x / y);
}

static void hh_rates(double V, double *am, double *bm, double *ah, double *bh, double *an, double *bn)
{
    *am = 0.1 * hh_trap(V + 40.0, 10.0);
    *bm = 4.0 * exp(-(V + 65.0) / 18.0);
    *ah = 0.07 * exp(-(V + 65.0) / 20.0);
    *bh = 1.0 / (1.0 + exp(-(V + 35.0) / 10.0));
    *an = 0.01 * hh_trap(V + 55.0, 10.0);
    *bn = 0.125 * exp(-(V + 65.0) / 80.0);
}

/* Gates at rest: x_inf(-65 mV) = alpha / (alpha + beta). */
void orc_hh_rest_gates(double *m, double *n, double *h)
{
    double am, bm, ah, bh, an, bn;
    hh_rates(-65.0, &am, &bm, &ah, &bh, &an, &bn);
    *m = am / (am + bm);
    *n = an / (an + bn);
    *h = ah / (ah + bh);
}

/* One Euler step of the Hodgkin-Huxley + alpha-PSC + calcium node (model 2). */
static void hh_step(const orc_net *net, double V, double m, double n, double h, double r, double p, double c,
                    double S, double U, double *V1, double *m1, double *n1, double *h1, double *r1, double *p1,
                    double *c1)
{
    double dt = net->dt_ms;
    double am, bm, ah, bh, an, bn;
    hh_rates(V, &am, &bm, &ah, &bh, &an, &bn);
    double ina = net->hh_gna * m * m * m * h * (V - net->hh_ena);
    double ik = net->hh_gk * n * n * n * n * (V - net->hh_ek);
    double il = net->hh_gl * (V - net->hh_el);
    *V1 = V + dt / net->hh_C * (-ina - ik - il + r + U + net->hh_iext);
    *m1 = m + dt * (am * (1.0 - m) - bm * m);
    *n1 = n + dt * (an * (1.0 - n) - bn * n);
    *h1 = h + dt * (ah * (1.0 - h) - bh * h);
    *r1 = r + dt * p;
    *p1 = p + dt * (-net->psc_a * net->psc_a * r - 2.0 * net->psc_a * p + S);
    *c1 = c + dt * (-c / net->tau_c + (V >= net->hh_vpeak ? 1.0 : 0.0));
}

static double stimulus(const orc_net *net, int32_t j, int64_t n, int32_t *bg_count)
{
    double U = 0.0;
    for (int32_t p = 0; p < net->n_pulses; ++p)
        if (net->p_node[p] == j && net->p_on[p] <= n && n < net->p_off[p])
            U += net->p_amp[p];
    if (net->bg_threshold) {
        int32_t cnt = bg_count[j];
        if (orc_bg_onset(net->bg_seed, (uint32_t)j, n, net->bg_threshold)) cnt = net->bg_width;
        if (cnt > 0) {
            U += net->bg_amp;
            cnt -= 1;
        }
        bg_count[j] = cnt;
    }
    return U;
}

/* history accessor: full (dense) or circular of depth H */
typedef struct {
    double *buf;
    int64_t depth;   /* number of slots kept */
    int dense;       /* 1: slot = time index, buf holds every step */
    int32_t n;
} history;

static double hist_get(const history *h, int64_t t, int32_t i)
{
    if (t < 0) return 0.0;                      /* before t = 0 every node rests */
    int64_t slot = h->dense ? t : (t % h->depth);
    return h->buf[slot * h->n + i];
}

static void hist_put(history *h, int64_t t, int32_t i, double v)
{
    int64_t slot = h->dense ? t : (t % h->depth);
    h->buf[slot * h->n + i] = v;
}

/* Optional starting state at step n0 > 0 (restart): the state relative to rest,
 * the background counters and the history hist[k][j] = v~_j(n0 - k), k = 0..depth-1. */
typedef struct {
    int64_t n0;
    const double *v, *w, *c;
    const int32_t *bg_count;
    const double *hist;
    int32_t hist_depth;
    const double *r, *p;      /* models 1, 2: PSC state (NULL = 0) */
    const double *m, *n, *h;  /* model 2: gates (NULL = their values at -65 mV) */
    const double *w_edge;     /* stdp: [E] weights (NULL = the net's) */
    const double *s;          /* stdp: [N] time since the last spike (NULL = 0) */
    const double *hist_s;     /* stdp: [hist_depth * N] s_j(n0 - k) (NULL = 0) */
} orc_init;

static int simulate(const orc_net *net, int64_t n_steps, orc_out *out, int dense,
                    const orc_init *init)
{
    int32_t N = net->n_nodes;
    int64_t E = net->n_edges;
    const int izh = net->model == 1, hh = net->model == 2, spiking = izh || hh;
    const int stdp = net->stdp != 0;
    if (N <= 0 || E < 0 || n_steps < 0 || !(net->dt_ms > 0.0) || (net->model != 0 && !spiking))
        return ORC_EINVAL;
    if (stdp && (!spiking || !isfinite(net->stdp_alpha) || !(net->stdp_beta >= 0.0) || !isfinite(net->stdp_beta)))
        return ORC_EINVAL;
    if (izh && !(net->iz_C > 0.0)) return ORC_EINVAL;
    if (hh && !(net->hh_C > 0.0)) return ORC_EINVAL;
    if (spiking ? !(net->tau_c > 0.0) : !(net->tau_ms > 0.0)) return ORC_EINVAL;
    if (net->n_types < 0 || net->n_types > ORC_MAX_TYPES || (net->n_types > 0 && (!spiking || !net->types || !net->cell_type)))
        return ORC_EINVAL;
    /* the parameters of each cell type, as whole networks' fields */
    orc_net tnet[ORC_MAX_TYPES];
    for (int32_t t = 0; t < net->n_types; ++t) {
        const double *q = net->types + (size_t)t * (izh ? 12 : 11);
        tnet[t] = *net;
        if (izh) {
            tnet[t].iz_C = q[0]; tnet[t].iz_k = q[1]; tnet[t].iz_vr = q[2]; tnet[t].iz_vt = q[3];
            tnet[t].iz_vpeak = q[4]; tnet[t].iz_vreset = q[5]; tnet[t].iz_a = q[6]; tnet[t].iz_b = q[7];
            tnet[t].iz_d = q[8]; tnet[t].iz_iext = q[9]; tnet[t].psc_a = q[10]; tnet[t].tau_c = q[11];
        } else {
            tnet[t].hh_C = q[0]; tnet[t].hh_gna = q[1]; tnet[t].hh_gk = q[2]; tnet[t].hh_gl = q[3];
            tnet[t].hh_ena = q[4]; tnet[t].hh_ek = q[5]; tnet[t].hh_el = q[6]; tnet[t].hh_vpeak = q[7];
            tnet[t].hh_iext = q[8]; tnet[t].psc_a = q[9]; tnet[t].tau_c = q[10];
        }
        if ((izh && !(tnet[t].iz_C > 0.0)) || (hh && !(tnet[t].hh_C > 0.0)) || !(tnet[t].tau_c > 0.0)) return ORC_EINVAL;
    }
    for (int32_t j = 0; j < N && net->n_types > 0; ++j)
        if (net->cell_type[j] >= net->n_types) return ORC_EINVAL;
#define NODE_NET(j) (net->n_types > 0 ? &tnet[net->cell_type[j]] : net)
#define VPEAK(j) (hh ? NODE_NET(j)->hh_vpeak : NODE_NET(j)->iz_vpeak)
    double v_rest = 0.0, w_rest = 0.0;
    if (!spiking && orc_rest_point(net->a, net->b, net->c, net->f, net->g, net->i_ext, &v_rest, &w_rest))
        return ORC_EINVAL;
    int32_t dmax = 1;
    for (int64_t e = 0; e < E; ++e) {
        if (net->delay[e] < 1 || net->src[e] < 0 || net->src[e] >= N || net->dst[e] < 0 ||
            net->dst[e] >= N || net->src[e] == net->dst[e])
            return ORC_EINVAL;
        if (net->delay[e] > dmax) dmax = net->delay[e];
    }
    int64_t n0 = init ? init->n0 : 0;
    if (n0 < 0 || (init && dense)) return ORC_EINVAL;
    if (init && n0 > 0 && init->hist_depth < dmax + 1 && init->hist_depth < n0 + 1) return ORC_EINVAL;
    if (out->hist_out && (out->hist_out_depth < 1 || out->hist_out_depth > dmax + 1)) return ORC_EINVAL;
    history h;
    h.n = N;
    h.dense = dense;
    h.depth = dense ? (n_steps + 1) : ((int64_t)dmax + 1);
    h.buf = (double *)calloc((size_t)(h.depth * N), sizeof(double));
    double *v = (double *)calloc((size_t)N, sizeof(double));
    double *w = (double *)calloc((size_t)N, sizeof(double));
    double *c = (double *)calloc((size_t)N, sizeof(double));
    double *S = (double *)calloc((size_t)N, sizeof(double));
    int32_t *bgc = (int32_t *)calloc((size_t)N, sizeof(int32_t));
    double *r = (double *)calloc((size_t)N, sizeof(double));
    double *p = (double *)calloc((size_t)N, sizeof(double));
    double *gm = (double *)calloc((size_t)N, sizeof(double));
    double *gn = (double *)calloc((size_t)N, sizeof(double));
    double *gh = (double *)calloc((size_t)N, sizeof(double));
    /* STDP: the time since the last spike s_j, its history, and the evolving weights */
    history hs = h;
    hs.buf = stdp ? (double *)calloc((size_t)(h.depth * N), sizeof(double)) : NULL;
    double *sj = stdp ? (double *)calloc((size_t)N, sizeof(double)) : NULL;
    double *wcur = stdp ? (double *)malloc(sizeof(double) * (size_t)(E > 0 ? E : 1)) : NULL;
    if (!h.buf || !v || !w || !c || !S || !bgc || !r || !p || !gm || !gn || !gh || (stdp && (!hs.buf || !sj || !wcur))) {
        free(h.buf); free(v); free(w); free(c); free(S); free(bgc); free(r); free(p); free(gm); free(gn); free(gh);
        free(hs.buf); free(sj); free(wcur);
        return ORC_ENOMEM;
    }
    if (stdp)
        for (int64_t e = 0; e < E; ++e) wcur[e] = (init && init->w_edge) ? init->w_edge[e] : net->weight[e];
    const double *wgt = stdp ? wcur : net->weight;
    /* frame sums of the readout state (a run starts a new frame) */
    double *facc = (double *)calloc((size_t)N, sizeof(double));
    if (!facc) {
        free(h.buf); free(v); free(w); free(c); free(S); free(bgc); free(r); free(p); free(gm); free(gn); free(gh);
        free(hs.buf); free(sj); free(wcur);
        return ORC_ENOMEM;
    }
    if (izh)
        for (int32_t j = 0; j < N; ++j) v[j] = NODE_NET(j)->iz_vr;
    if (hh) {
        double m0, n0_, h0;
        orc_hh_rest_gates(&m0, &n0_, &h0);
        for (int32_t j = 0; j < N; ++j) {
            v[j] = -65.0;
            gm[j] = m0;
            gn[j] = n0_;
            gh[j] = h0;
        }
    }
    if (out->min_peak_gap)
        for (int32_t j = 0; j < N; ++j) out->min_peak_gap[j] = INFINITY;
    if (init) {
        for (int32_t j = 0; j < N; ++j) {
            v[j] = init->v[j];
            w[j] = init->w[j];
            c[j] = init->c[j];
            bgc[j] = init->bg_count ? init->bg_count[j] : 0;
            if (spiking) {
                r[j] = init->r ? init->r[j] : 0.0;
                p[j] = init->p ? init->p[j] : 0.0;
            }
            if (hh) {
                if (init->m) gm[j] = init->m[j];
                if (init->n) gn[j] = init->n[j];
                if (init->h) gh[j] = init->h[j];
            }
            if (stdp && init->s) sj[j] = init->s[j];
        }
        for (int64_t k = 1; k < h.depth && k < init->hist_depth; ++k)
            if (n0 - k >= 0)
                for (int32_t j = 0; j < N; ++j) {
                    hist_put(&h, n0 - k, j, init->hist[k * N + j]);
                    if (stdp) hist_put(&hs, n0 - k, j, init->hist_s ? init->hist_s[k * N + j] : 0.0);
                }
    }
    if (out->first_arrival)
        for (int32_t j = 0; j < N; ++j) out->first_arrival[j] = -1;
    if (out->first_value)
        for (int32_t j = 0; j < N; ++j) out->first_value[j] = 0.0;
    out->ev_count = 0;
    double v_theta = net->theta;
    int64_t snap_idx = 0;

    for (int64_t n = n0; n < n0 + n_steps; ++n) {
        /* record v~(n) (model 1: spd(V(n))) before anything reads the history of this step */
        for (int32_t j = 0; j < N; ++j) hist_put(&h, n, j, spiking ? (v[j] >= VPEAK(j) ? 1.0 : 0.0) : v[j]);
        if (stdp)
            for (int32_t j = 0; j < N; ++j) hist_put(&hs, n, j, sj[j]);
        /* S_j(n) = sum over edges i -> j of w_ij * v_i(n - D_ij) */
        for (int32_t j = 0; j < N; ++j) S[j] = 0.0;
        for (int64_t e = 0; e < E; ++e) {
            double past = hist_get(&h, n - net->delay[e], net->src[e]);
            if (!spiking && net->coupling == 1) past = v_rest + past;
            S[net->dst[e]] += wgt[e] * past;
            if (stdp) {
                /* Plasticity: q_ij = (s_i(t - tau_ij) - s_j(t)) max(spd(V_i(t - tau_ij)), spd(V_j(t)));
                 * w_ij' = w_ij + dt alpha sign(q_ij) exp(-beta |q_ij|), after w_ij(t) fed S. */
                double post = hist_get(&h, n, net->dst[e]);
                double gate = past > post ? past : post;
                double q = (hist_get(&hs, n - net->delay[e], net->src[e]) - sj[net->dst[e]]) * gate;
                if (q != 0.0)
                    wcur[e] += net->dt_ms * net->stdp_alpha * (q > 0.0 ? 1.0 : -1.0) * exp(-net->stdp_beta * fabs(q));
            }
        }
        int sample = ((n + 1) % net->sample_every) == 0;
        int64_t k = (n + 1) / net->sample_every - 1;            /* absolute sample number */
        int64_t k_out = (n + 1) / net->sample_every - n0 / net->sample_every - 1;  /* row of y */
        for (int32_t j = 0; j < N; ++j) {
            double U = stimulus(net, j, n, bgc);
            double v1, w1, c1;
            if (spiking) {
                double r1, p1;
                int spike;
                if (izh) {
                    izh_step(NODE_NET(j), v[j], w[j], r[j], p[j], c[j], S[j], U, &v1, &w1, &r1, &p1, &c1);
                    spike = v1 >= VPEAK(j);
                } else {
                    double m1, n1, h1;
                    hh_step(NODE_NET(j), v[j], gm[j], gn[j], gh[j], r[j], p[j], c[j], S[j], U, &v1, &m1, &n1, &h1, &r1, &p1,
                            &c1);
                    gm[j] = m1;
                    gn[j] = n1;
                    gh[j] = h1;
                    w1 = 0.0;
                    spike = v[j] < VPEAK(j) && v1 >= VPEAK(j);   /* an upward crossing (no reset) */
                }
                r[j] = r1;
                p[j] = p1;
                if (out->min_peak_gap) {
                    double gap = fabs(v1 - VPEAK(j));
                    if (gap < out->min_peak_gap[j]) out->min_peak_gap[j] = gap;
                }
                if (spike) {
                    if (out->ev_count < out->ev_cap) {
                        out->ev_node[out->ev_count] = j;
                        out->ev_step[out->ev_count] = n + 1;
                    }
                    out->ev_count++;
                }
                if (out->first_arrival && out->first_arrival[j] < 0 && spike) {
                    out->first_arrival[j] = (int32_t)(n + 1);
                    if (out->first_value) out->first_value[j] = v1;
                }
                facc[j] += c1;
                if (sample) {
                    double cbar = net->frame_average ? facc[j] / net->sample_every : c1;
                    facc[j] = 0.0;
                    double clean = net->gain * cbar + net->offset;
                    if (out->y_clean) out->y_clean[k_out * N + j] = clean;
                    if (out->y) out->y[k_out * N + j] = clean + net->sigma * orc_gauss(net->obs_seed, (uint32_t)j, k);
                }
                v[j] = v1; w[j] = w1; c[j] = c1;
                continue;
            }
            node_step(net, v_rest, v[j], w[j], c[j], S[j], U, &v1, &w1, &c1);
            /* event: V crosses theta upward between n and n+1 */
            if (v_rest + v[j] < v_theta && v_rest + v1 >= v_theta) {
                if (out->ev_count < out->ev_cap) {
                    out->ev_node[out->ev_count] = j;
                    out->ev_step[out->ev_count] = n + 1;
                }
                out->ev_count++;
            }
            if (out->first_arrival && out->first_arrival[j] < 0 && v1 != 0.0) {
                out->first_arrival[j] = (int32_t)(n + 1);
                if (out->first_value) out->first_value[j] = v1;
            }
            facc[j] += c1;
            if (sample) {
                double cbar = net->frame_average ? facc[j] / net->sample_every : c1;
                facc[j] = 0.0;
                double clean = net->gain * (v_rest + cbar) + net->offset;
                if (out->y_clean) out->y_clean[k_out * N + j] = clean;
                if (out->y) out->y[k_out * N + j] = clean + net->sigma * orc_gauss(net->obs_seed, (uint32_t)j, k);
            }
            v[j] = v1; w[j] = w1; c[j] = c1;
        }
        /* s_j(t + dt) = (1 - spd(V_j(t))) (s_j(t) + dt) */
        if (stdp)
            for (int32_t j = 0; j < N; ++j) sj[j] = hist_get(&h, n, j) > 0.0 ? 0.0 : sj[j] + net->dt_ms;
        if (out->snap_every > 0 && ((n + 1 - n0) % out->snap_every) == 0) {
            memcpy(out->snap_v + snap_idx * N, v, sizeof(double) * (size_t)N);
            memcpy(out->snap_w + snap_idx * N, w, sizeof(double) * (size_t)N);
            memcpy(out->snap_c + snap_idx * N, c, sizeof(double) * (size_t)N);
            snap_idx++;
        }
    }
    memcpy(out->v, v, sizeof(double) * (size_t)N);
    memcpy(out->w, w, sizeof(double) * (size_t)N);
    memcpy(out->c, c, sizeof(double) * (size_t)N);
    if (out->bg_count) memcpy(out->bg_count, bgc, sizeof(int32_t) * (size_t)N);
    if (out->r) memcpy(out->r, r, sizeof(double) * (size_t)N);
    if (out->p) memcpy(out->p, p, sizeof(double) * (size_t)N);
    if (out->m) memcpy(out->m, gm, sizeof(double) * (size_t)N);
    if (out->n) memcpy(out->n, gn, sizeof(double) * (size_t)N);
    if (out->h) memcpy(out->h, gh, sizeof(double) * (size_t)N);
    if (out->hist_out) {
        int64_t n_end = n0 + n_steps;
        for (int32_t k = 0; k < out->hist_out_depth; ++k)
            for (int32_t j = 0; j < N; ++j) {
                double now = spiking ? (v[j] >= VPEAK(j) ? 1.0 : 0.0) : v[j];
                out->hist_out[(int64_t)k * N + j] = (k == 0) ? now : hist_get(&h, n_end - k, j);
            }
    }
    if (stdp) {
        if (out->w_final) memcpy(out->w_final, wcur, sizeof(double) * (size_t)E);
        if (out->s) memcpy(out->s, sj, sizeof(double) * (size_t)N);
        if (out->hist_s_out && out->hist_out_depth >= 1) {
            int64_t n_end = n0 + n_steps;
            for (int32_t k = 0; k < out->hist_out_depth; ++k)
                for (int32_t j = 0; j < N; ++j)
                    out->hist_s_out[(int64_t)k * N + j] = (k == 0) ? sj[j] : hist_get(&hs, n_end - k, j);
        }
    }
    free(h.buf); free(v); free(w); free(c); free(S); free(bgc); free(r); free(p); free(gm); free(gn); free(gh);
    free(hs.buf); free(sj); free(wcur); free(facc);
    return ORC_OK;
#undef NODE_NET
#undef VPEAK
}

/* Circular history of depth D_max + 1 (the working oracle). */
int orc_simulate(const orc_net *net, int64_t n_steps, orc_out *out)
{
    return simulate(net, n_steps, out, 0, NULL);
}

/* The same, continuing from a given state at step n0 (used to check a long run
 * window by window from the state another implementation reached). */
int orc_simulate_from(const orc_net *net, const orc_init *init, int64_t n_steps, orc_out *out)
{
    return simulate(net, n_steps, out, 0, init);
}

/* Brute force: the whole history [n_steps + 1][N] kept, v_i(t - tau) read by
 * its time index directly, exactly as Eq. Yjset is written.  Tiny nets only. */
int orc_simulate_dense(const orc_net *net, int64_t n_steps, orc_out *out)
{
    return simulate(net, n_steps, out, 1, NULL);
}

/* Whole step of a time in ms: llround(t / dt), half away from zero. */
int64_t orc_ms_to_step(double t_ms, double dt_ms)
{
    return (int64_t)llround(t_ms / dt_ms);
}

int orc_rest_point_of(const orc_net *net, double *v_rest, double *w_rest)
{
    return orc_rest_point(net->a, net->b, net->c, net->f, net->g, net->i_ext, v_rest, w_rest);
}
