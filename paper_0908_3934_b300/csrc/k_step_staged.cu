// The staged step kernel: one launch advances every node by dt, one CTA per tile
// of consecutive target nodes (the layout is built by build_staged).
//
//   0. one thread starts bulk copies (cp.async.bulk, completion on an mbarrier)
//      of what does not change between steps -- the tile's gather keys and its
//      edge entries (weight, gather index) -- into shared memory, while the other
//      threads load the piece list and caller id of their row;
//   1. once the copies have landed, the CTA fetches each distinct history value its
//      edges read, v~_src(n - D) from ring slot (n - D) & (R - 1), once, into shared
//      memory.  Slot n - D (D >= 1) was written by step n - D - 1 <= n - 2, so a
//      kernel that gathers early (kEarly) does this and step 2 before it waits for
//      the previous step (griddepcontrol.wait), just before step 3, when step n - 1
//      is complete; the gathers of one step then overlap the end of the previous
//      one.  Every network with static weights gathers early.  A grid that
//      outnumbers the CTAs the device holds at once lets the next step start first
//      thing (kLaunchFirst: its first CTAs only fill the SMs this grid's last wave
//      leaves free); a smaller grid does so just before step 3, after its wait.
//      Plastic networks let the next step start at once and wait before step 1.
//      The gathers are sorted by (D, src), so a warp's 32 reads fall in a few lines
//      of one ring slot.  While they are in flight, a spiking node (Izhikevich,
//      Hodgkin-Huxley) runs every part of its update that does not read S -- all
//      but the PSC variable p;
//   2. each lane sums one piece of a row in a register, S_piece = sum_e w_e
//      v~_src(n - D_e) over its edges in order, all from shared memory (Eq. Yjset,
//      Sec. 2).  A row of at most kWarpRow edges is one piece; a longer row is 32
//      lane-strided pieces -- the summation order of every step kernel;
//   3. one thread per row combines its pieces (a long row's 32 by the butterfly
//      tree of a warp reduction) and runs the node update (a spiking node: p):
//      stimulus, FHN Euler step about the rest point (Sec. 3.1, Eq. fnstate),
//      history write, low-pass readout, noisy observation (Sec. 3.3), events and
//      first arrivals.
// Reads of step data are of step n (or older), writes are of step n + 1, and slots
// (n + 1) & (R - 1) and (n + 2) & (R - 1) are never read in step n because every
// delay is <= R - 2 (so step n's writes never meet step n + 1's early gathers).
// The copy wait is bounded: if it gives up, the CTA sets kStatusTimeout in the
// status word (the host reports GN_ETIMEOUT), waits once more for its copies and
// leaves its rows untouched.
#include "step_common.cuh"

namespace gn {
namespace {

using namespace step;


__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// threads per SM the register allocation must allow, with and without entry
// staging.  Without it, 1280 threads at 48 registers with 16-deep entry loads: on
// the 1M-node net 0.1023 ms per step in 256-row tiles (which shared memory holds 5
// to an SM anyway) against 0.1126 at 1536 threads and 40 registers with 8-deep
// loads, and 0.1048 at 1280 threads with 8-deep loads
constexpr int kThreadsSE = 1024;
constexpr int kThreadsL2 = 1280;
// plastic weights: 48 registers (one 4-byte spill) at 1280 threads per SM beat 56
// without spills at 1024 (1M-node net: 0.148 vs 0.160 ms per step)
constexpr int kThreadsPlastic = 1280;

// How a tile waits, before its node update, for the previous step to be complete
// everywhere: a launch of a chain waits for the previous grid (griddepcontrol.wait).
struct PdlWait {
    static constexpr bool kPdl = true;
    __device__ __forceinline__ bool operator()() const
    {
        pdl_wait();
        return true;
    }
};

// One tile's step (the CTA's work) for network `a`; `tile` indexes a.st_tile.
// `wait` is called by every thread before the node update (kEarly) and returns
// false if the CTA must give up; `phase` is the parity of the CTA's next copy
// completion (a kernel that runs one tile per CTA initialises the mbarrier for it;
// a persistent one, Wait::kPdl false, initialises it once and flips `phase` per
// use).  Returns false if the tile gave up (its rows are left untouched).
template <int kM, int T, bool kSE, bool kPacked, bool kStream, bool kEarly, bool kLaunchFirst, class Wait = PdlWait>
__device__ __forceinline__ bool staged_tile(const StepArgs &a, const int tile, const int k, Wait &wait,
                                            uint32_t &phase)
{
    // [mbarrier 16 B][keys][values (wide keys only)][entry weights][entry indices][piece sums];
    // without entry staging (kSE false) the entry arrays are absent
    constexpr bool kPl = (kM & kPlastic) != 0;
    static_assert(!(kPl && kSE), "plastic weights are written back to global memory: no entry staging");
    extern __shared__ __align__(128) unsigned char s_raw[];
    __shared__ int s_fail;
    __shared__ uint32_t s_post[kPl ? T : 1];  // plastic: each row's ring word of step n
    uint64_t *bar = reinterpret_cast<uint64_t *>(s_raw);
    uint32_t *s_key = reinterpret_cast<uint32_t *>(s_raw + 16);
    float *s_val = kPacked ? reinterpret_cast<float *>(s_key)
                           : reinterpret_cast<float *>(s_raw + 16 + static_cast<size_t>(a.st_ucap) * 8);
    float *s_w = reinterpret_cast<float *>(s_raw + 16 + static_cast<size_t>(a.st_ucap) * (kPacked ? 4 : 12));
    uint16_t *s_u = reinterpret_cast<uint16_t *>(s_w + a.st_xcap);
    float *s_part = kSE ? reinterpret_cast<float *>(s_u + a.st_xcap) : s_w;

    // kEarly (static weights, any node model): the gathers of step n read history slots
    // n - D <= n - 1, all written by step n - 2 or earlier, so the CTA fetches and
    // sums them before griddepcontrol.wait and waits only before the node update
    // (its rows' state is step n - 1's).  That needs step n - 2 complete when the
    // grid starts: with kLaunchFirst false the CTA lets the next grid start only
    // after its wait; with kLaunchFirst it does so at once (the next grid's prologue
    // overlaps this one), which the host allows only for a grid of more CTAs than
    // can be resident at once -- its last CTA then starts after another one has
    // passed the wait, so step n - 1 is complete before step n + 1 starts.
    static_assert(!kEarly || !kPl, "plastic weights are written by the previous step");
    static_assert(kEarly || kLaunchFirst, "a CTA that waits first lets the next grid start first");
    static_assert(kEarly || Wait::kPdl, "a persistent kernel gathers before it waits");
    if constexpr (kLaunchFirst && Wait::kPdl) pdl_launch_dependents();
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int4 td = __ldg(a.st_tile + tile);   // {r0, rows, u0, gathers}
    const int4 td2 = __ldg(a.st_tile2 + tile); // {s0, slices, x0, entries}
    const int nu = td.w, nx = td2.w;
    const uint32_t kbytes = static_cast<uint32_t>((nu + 3) & ~3) * (kPacked ? 4u : 8u);
    const uint32_t bytes = kbytes + (kSE ? static_cast<uint32_t>(nx) * 6u : 0u);
    if (t == 0) {
        s_fail = 0;
        if (bytes) {
            if constexpr (Wait::kPdl) {
                mbar_init(bar, 1);
                fence_barrier_init();
            } else {
                fence_async_shared();  // the previous tile's reads and writes of shared memory come first
            }
            mbar_arrive_expect_tx(bar, bytes);
            const char *keys = static_cast<const char *>(a.st_ukey) + static_cast<size_t>(td.z) * (kPacked ? 4 : 8);
            // a stream larger than L2 is read once per step: evict it first
            const uint64_t pol = kStream ? l2_evict_first() : l2_evict_last();
            if (kbytes) bulk_g2s_hint(s_key, keys, kbytes, bar, pol);
            if (kSE && nx) {
                bulk_g2s_hint(s_w, a.st_w + td2.z, static_cast<uint32_t>(nx) * 4u, bar, pol);
                bulk_g2s_hint(s_u, a.st_u + td2.z, static_cast<uint32_t>(nx) * 2u, bar, pol);
            }
        }
        if (!kSE && nx) {
            const uint64_t pol = kStream ? l2_evict_first() : l2_evict_last();
            bulk_prefetch_l2(a.st_w + td2.z, static_cast<uint32_t>(nx) * 4u, pol);
            bulk_prefetch_l2(a.st_u + td2.z, static_cast<uint32_t>(nx) * 2u, pol);
        }
    }
    const int r = td.x + t;
    const bool own = t < td.y;
    int q0 = 0, q1 = 0;
    int32_t orig = kLoad;
    if (own) {
        q0 = __ldg(a.st_rq + r);
        q1 = __ldg(a.st_rq + r + 1);
        orig = __ldg(a.perm + r);
    }
    int2 sd0 = make_int2(0, 0);
    if (warp < td2.y) sd0 = __ldg(a.st_slice + td2.x + warp);

    if constexpr (!kEarly) wait();
    const int64_t n = *a.d_step + k;  // the step counter changes only between graphs
    float v = 0.0f;
    float2 wc = make_float2(0.0f, 0.0f);
    int32_t cnt0 = kLoad;
    uint32_t word_now = 0;
    auto load_own = [&] {
        if (!own) return;
        if constexpr (kM == 0) v = a.ring[(n & a.ring_mask) * a.ring_stride + r];  // spiking models keep V apart
        if constexpr (kPl) {
            word_now = reinterpret_cast<const uint32_t *>(a.ring)[(n & a.ring_mask) * a.ring_stride + r];
            s_post[t] = word_now;
        }
        wc = a.wc[r];
        if (a.bg_thr) cnt0 = a.bgc[r];
    };
    if constexpr (!kEarly) load_own();
    if (t == 0 && bytes && !mbar_wait_bounded(bar, phase, a.wait_limit)) {
        atomicOr(a.status, kStatusTimeout);
        s_fail = 1;
        mbar_wait_bounded(bar, phase, kDefaultWaitLimit);  // the copies must land before the CTA leaves
    }
    if (bytes) phase ^= 1u;
    __syncthreads();
    if (s_fail) return false;

    // 1. the tile's distinct history values, copied asynchronously straight into
    // shared memory (packed keys are overwritten in place: a thread reads key u
    // before it issues the copy of value u); the live ring slots are kept in L2
    // ahead of the streamed edge data
    const uint32_t dmask = (1u << a.dbits) - 1u;
    const uint64_t pol_ring = l2_evict_last();
#pragma unroll 4
    for (int u = t; u < nu; u += T) {
        uint32_t src, d;
        if constexpr (kPacked) {
            const uint32_t kk = s_key[u];
            src = kk >> a.dbits;
            d = kk & dmask;
        } else {
            const uint2 kk = reinterpret_cast<const uint2 *>(s_key)[u];
            src = kk.x;
            d = kk.y;
        }
        const int64_t slot = (n - static_cast<int64_t>(d)) & a.ring_mask;
        cp_async4_hint(s_val + u, a.ring + slot * a.ring_stride + src, pol_ring);
    }
    // a spiking node's update reads S only in p: the rest runs while the gathers land
    float2 rp0 = make_float2(0.0f, 0.0f);
    if constexpr (kM != 0 && !kEarly)
        if (own) rp0 = spiking_begin<kM>(a, r, n, wc, orig, cnt0, word_now);
    cp_async_wait_all();
    __syncthreads();

    // 2. one piece per lane, 32 pieces per warp at a time
    for (int sl = warp; sl < td2.y; sl += T / 32) {
        const int2 sd = sl == warp ? sd0 : __ldg(a.st_slice + td2.x + sl);
        float acc = 0.0f;
        if constexpr (kPl) {
            // plastic weights: S from w_ij(n), then w_ij(n + 1) written back where a
            // spike gates it, over the piece's own entries (the slice's padding after
            // them, weight 0, is summed like the static kernel's but never updated)
            const uint32_t pi = __ldg(a.st_pinfo + 32 * (td2.x + sl) + lane);
            const int plen = static_cast<int>(pi & 0xffffu);
            const uint32_t post = s_post[pi >> 16];
            const int32_t k_post = static_cast<int32_t>(post >> 1);
            const uint32_t *s_word = reinterpret_cast<const uint32_t *>(s_val);
            float *wp = a.st_w + td2.z + sd.x + lane;
            const uint16_t *up = a.st_u + td2.z + sd.x + lane;
            auto entry = [&](int kk, float w, uint16_t u) {
                const uint32_t word = s_word[u];
                acc = __fadd_rn(acc, __fmul_rn(w, (word & 1u) ? 1.0f : 0.0f));
                if (((word | post) & 1u) && kk < plen) {
                    // q = (s_i(t - tau) - s_j(t)) max(spd_i, spd_j), both s in whole steps
                    const float q = static_cast<float>(static_cast<int32_t>(word >> 1) - k_post) * a.dt;
                    if (q != 0.0f) wp[kk * 32] = w + copysignf(a.stdp_dta * expf(-a.stdp_beta * fabsf(q)), q);
                }
            };
            int kk = 0;
            for (; kk + 8 <= sd.y; kk += 8) {
                float w8[8];
                uint16_t u8[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    w8[i] = __ldcs(wp + (kk + i) * 32);
                    u8[i] = __ldcs(up + (kk + i) * 32);
                }
#pragma unroll
                for (int i = 0; i < 8; ++i) entry(kk + i, w8[i], u8[i]);
            }
            for (; kk < sd.y; ++kk) entry(kk, __ldcs(wp + kk * 32), __ldcs(up + kk * 32));
        } else if constexpr (kSE) {
            const float *wp = s_w + sd.x + lane;
            const uint16_t *up = s_u + sd.x + lane;
#pragma unroll 4
            for (int kk = 0; kk < sd.y; ++kk) acc = __fadd_rn(acc, __fmul_rn(wp[kk * 32], s_val[up[kk * 32]]));
        } else {
            const float *wp = a.st_w + td2.z + sd.x + lane;
            const uint16_t *up = a.st_u + td2.z + sd.x + lane;
            int kk = 0;
            for (; kk + 16 <= sd.y; kk += 16) {
                float w8[16];
                uint16_t u8[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    w8[i] = __ldcs(wp + (kk + i) * 32);
                    u8[i] = __ldcs(up + (kk + i) * 32);
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) acc = __fadd_rn(acc, __fmul_rn(w8[i], s_val[u8[i]]));
            }
            for (; kk < sd.y; ++kk) acc = __fadd_rn(acc, __fmul_rn(__ldcs(wp + kk * 32), s_val[__ldcs(up + kk * 32)]));
        }
        s_part[sl * 32 + lane] = acc;
    }
    __syncthreads();

    // 3. row sums and the node update
    if constexpr (kEarly) {
        if (!wait()) return false;
        if constexpr (!kLaunchFirst && Wait::kPdl) pdl_launch_dependents();
        load_own();
    }
    if (own) {
        float S = 0.0f;
        if (q1 - q0 == 1) {
            S = s_part[__ldg(a.st_plist + q0)];
        } else if (q1 - q0 == 32) {
            float x[32];
#pragma unroll
            for (int l = 0; l < 32; ++l) x[l] = s_part[__ldg(a.st_plist + q0 + l)];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                for (int l = 0; l < o; ++l) x[l] = __fadd_rn(x[l], x[l + o]);
            S = x[0];
        }
        if constexpr (kM == 0)
            node_update<kM>(a, r, n, v, wc, S, orig, cnt0);
        else if constexpr (kEarly)  // the whole spiking update after the wait
            psc_finish(a, r, spiking_begin<kM>(a, r, n, wc, orig, cnt0, word_now), S);
        else
            psc_finish(a, r, rp0, S);
    }
    return true;
}

// kMode: 0 gathers after the grid wait (the next grid starts at once); 1 gathers
// early and lets the next grid start at once (a grid larger than the device holds);
// 2 gathers early and lets the next grid start only after its own wait (any grid)
template <int kM, int T, bool kSE, bool kPacked, bool kStream, int kMode>
__global__ void __launch_bounds__(T, (kSE ? kThreadsSE : (kM & kPlastic) ? kThreadsPlastic : kThreadsL2) / T)
    k_step_staged(const StepArgs a, const int k)
{
    PdlWait w;
    uint32_t phase = 0;
    staged_tile<kM, T, kSE, kPacked, kStream, kMode != 0, kMode != 2>(a, blockIdx.x, k, w, phase);
}

// Batched form, one launch per step over the tiles of every member network (all of
// node model kM): the CTA copies its network's arguments into shared memory, then
// runs the same tile step (tiles never straddle networks), gathering before the
// grid wait; kLaunchFirst as in staged_tile (a grid larger than the device holds).
template <int kM, int T, bool kPacked, bool kStream, bool kLaunchFirst>
__global__ void __launch_bounds__(T, kThreadsL2 / T) k_batch_staged(const StepArgs *__restrict__ nets,
                                                                    const int *__restrict__ tile_net, const int k)
{
    __shared__ StepArgs s_a;
    const uint32_t *src = reinterpret_cast<const uint32_t *>(nets + __ldg(tile_net + blockIdx.x));
    uint32_t *dst = reinterpret_cast<uint32_t *>(&s_a);
    for (int i = threadIdx.x; i < static_cast<int>(sizeof(StepArgs) / 4); i += T) dst[i] = __ldg(src + i);
    __syncthreads();
    PdlWait w;
    uint32_t phase = 0;
    staged_tile<kM, T, false, kPacked, kStream, true, kLaunchFirst>(s_a, blockIdx.x, k, w, phase);
}

// The lanes schedule of the batched form's L2 blocking, persistent: one cooperative
// launch steps every group n_steps times.  CTA b works in lane b % lanes and takes
// tiles b / lanes, b / lanes + C, ... of each group of its lane (C: the lane's
// CTAs); a lane runs its groups one after another (groups g = lane, lane + lanes,
// ...), each through all the steps, so a group's data stays in L2 across them.
// A lane's CTAs meet at a counting barrier in global memory (the lane's arrival
// count, on a line of its own).  After its tiles' node updates of the lane's j-th
// step (counted over its groups) a CTA adds 1 to the count; its node updates of step
// j wait until the count reaches j C, i.e. until step j - 1 is complete in the whole
// lane (slot n + 1, which step n writes, is read by step n - 1's longest delay).  Its
// gathers do not wait: they read history slots n - D, D >= 1, written by step n - 2
// or earlier, which the CTA's own wait in step n - 1 covered -- the argument of the
// early gathers in a chain of launches.  A CTA without a tile in a step still waits
// for step j - 1 before it arrives, so no CTA is two arrivals ahead of another and a
// count of (j + 1) C can only mean that every CTA has arrived for step j.  Memory
// order: the add is a release reduction (no reply awaited) after a CTA barrier;
// waits poll with relaxed loads and fence once the count is seen (acquire).  Waits
// are bounded: after `limit` polls, or once another CTA has set kStatusTimeout, the
// CTA gives up and returns.
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

__device__ __forceinline__ unsigned int ld_relaxed(const unsigned int *p)
{
    unsigned int v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Fire-and-forget add with release semantics (the CTA's writes before it, ordered by
// a CTA barrier, are visible to whoever observes the new count and then fences).
__device__ __forceinline__ void red_release_add(unsigned int *p, unsigned int v)
{
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Thread 0's wait until `count` reaches `target`: 1 on success, 0 on giving up.
__device__ __forceinline__ int lane_poll(const unsigned int *count, unsigned int target, uint32_t limit,
                                         unsigned int *status)
{
    for (uint32_t i = 0; i < limit; ++i) {
        if (ld_relaxed(count) >= target) {
            fence_acq_rel();
            return 1;
        }
        if ((i & 15u) == 15u && (ld_relaxed(status) & kStatusTimeout)) return 0;
        __nanosleep(64);
    }
    atomicOr(status, kStatusTimeout);
    return 0;
}

// The wait of one step (at most one poll loop per step; `done_here` is the thread's
// copy of its outcome).
struct LaneWait {
    static constexpr bool kPdl = false;
    const unsigned int *count;
    unsigned int target;
    uint32_t limit;
    unsigned int *status;
    int *s_ok;
    bool done_here;
    __device__ __forceinline__ bool operator()()
    {
        if (done_here) return true;
        if (threadIdx.x == 0) *s_ok = target == 0 ? 1 : lane_poll(count, target, limit, status);
        __syncthreads();
        done_here = *s_ok != 0;
        return done_here;
    }
};

template <int kM, int T, bool kPacked>
__global__ void __launch_bounds__(T, kThreadsL2 / T)
    k_batch_lanes(const StepArgs *__restrict__ nets, const int *__restrict__ tile_net, const int2 *__restrict__ groups,
                  const int n_groups, const int lanes, const int n_steps, unsigned int *__restrict__ counts,
                  unsigned int *status, const uint32_t limit)
{
    extern __shared__ __align__(128) unsigned char s_raw[];
    __shared__ StepArgs s_a;
    __shared__ int s_ok;
    const int lane = static_cast<int>(blockIdx.x) % lanes, me = static_cast<int>(blockIdx.x) / lanes;
    const unsigned int C = (gridDim.x - static_cast<unsigned int>(lane) + lanes - 1) / lanes;
    unsigned int *arrivals = counts + kLaneWords * lane;
    if (threadIdx.x == 0) {
        mbar_init(reinterpret_cast<uint64_t *>(s_raw), 1);
        fence_barrier_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    int cur = -1;
    unsigned int j = 0;
    for (int g = lane; g < n_groups; g += lanes) {
        const int2 gr = __ldg(groups + g);  // {first tile, tiles}
        for (int k = 0; k < n_steps; ++k, ++j) {
            LaneWait w{arrivals, j * C, limit, status, &s_ok, false};
            for (int i = me; i < gr.y; i += static_cast<int>(C)) {
                __syncthreads();  // the previous tile is done with shared memory
                const int net = __ldg(tile_net + gr.x + i);
                if (net != cur) {
                    const uint32_t *src = reinterpret_cast<const uint32_t *>(nets + net);
                    uint32_t *dst = reinterpret_cast<uint32_t *>(&s_a);
                    for (int x = threadIdx.x; x < static_cast<int>(sizeof(StepArgs) / 4); x += T) dst[x] = __ldg(src + x);
                    __syncthreads();
                    cur = net;
                }
                if (!staged_tile<kM, T, false, kPacked, false, true, false>(s_a, i, k, w, phase)) return;
            }
            if (!w()) return;
            __syncthreads();
            if (threadIdx.x == 0) red_release_add(arrivals, 1u);
        }
    }
}

// Persistent staged step of one network whose tiles the device holds all at once
// (kind 5): one cooperative launch of one CTA per tile runs n_steps steps.  The CTA
// copies its tile's gather keys and edge entries into shared memory once and keeps
// them for the whole launch (the gathered values have their own array), so a step is
// the gathers, the piece sums from shared memory, the wait for the previous step and
// the node update -- the tile step of the staged kernel with its entries staged, in the
// same summation order.  The CTAs meet at a counting barrier in global memory: after
// its node updates of step k a CTA adds 1 to the arrival count (a release reduction, no
// reply awaited), and its node updates of step k wait until the count reaches k C (C:
// the grid), i.e. until step k - 1 is complete everywhere (relaxed polls, then a
// fence).  A CTA arrives at step k only after that wait, so no CTA is two arrivals
// ahead and k C arrivals can only be every CTA's k.  Its gathers of step k read slots
// written in step k - 2 or earlier, covered by its own wait in step k - 1.  Bounded
// waits; a CTA that gives up sets kStatusTimeout and returns, and the others stop
// polling.
// kCluster: a network of at most 16 tiles runs as one thread-block cluster, and the
// step barrier is the cluster's own (barrier.cluster.arrive.release after the node
// updates of step k, barrier.cluster.wait.acquire before those of step k + 1, the
// next step's gathers and sums in between).  That barrier has no time limit, so every
// CTA passes every arrive and wait the same number of times: a CTA whose copy wait
// gave up (kStatusTimeout) runs the remaining steps' barriers without their work
// instead of returning, and it waits once more after the last arrive.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

template <int kM, int T, bool kPacked, bool kCluster>
__global__ void __launch_bounds__(T, 1)
    k_step_persist(const StepArgs a, const int n_steps, unsigned int *__restrict__ counts, const uint32_t limit)
{
    extern __shared__ __align__(128) unsigned char s_raw[];
    __shared__ int s_ok;
    uint64_t *bar = reinterpret_cast<uint64_t *>(s_raw);
    uint32_t *s_key = reinterpret_cast<uint32_t *>(s_raw + 16);
    float *s_val = reinterpret_cast<float *>(s_raw + 16 + static_cast<size_t>(a.st_ucap) * (kPacked ? 4 : 8));
    float *s_w = s_val + a.st_ucap;
    uint16_t *s_u = reinterpret_cast<uint16_t *>(s_w + a.st_xcap);
    float *s_part = reinterpret_cast<float *>(s_u + a.st_xcap);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int tile = blockIdx.x;
    const int4 td = __ldg(a.st_tile + tile);   // {r0, rows, u0, gathers}
    const int4 td2 = __ldg(a.st_tile2 + tile); // {s0, slices, x0, entries}
    const int nu = td.w, nx = td2.w;
    const uint32_t kbytes = static_cast<uint32_t>((nu + 3) & ~3) * (kPacked ? 4u : 8u);
    const uint32_t bytes = kbytes + static_cast<uint32_t>(nx) * 6u;
    if (t == 0) {
        s_ok = 1;
        if (bytes) {
            mbar_init(bar, 1);
            fence_barrier_init();
            mbar_arrive_expect_tx(bar, bytes);
            const char *keys = static_cast<const char *>(a.st_ukey) + static_cast<size_t>(td.z) * (kPacked ? 4 : 8);
            const uint64_t pol = l2_evict_last();
            if (kbytes) bulk_g2s_hint(s_key, keys, kbytes, bar, pol);
            if (nx) {
                bulk_g2s_hint(s_w, a.st_w + td2.z, static_cast<uint32_t>(nx) * 4u, bar, pol);
                bulk_g2s_hint(s_u, a.st_u + td2.z, static_cast<uint32_t>(nx) * 2u, bar, pol);
            }
        }
    }
    const int r = td.x + t;
    const bool own = t < td.y;
    int q0 = 0, q1 = 0;
    int32_t orig = kLoad;
    if (own) {
        q0 = __ldg(a.st_rq + r);
        q1 = __ldg(a.st_rq + r + 1);
        orig = __ldg(a.perm + r);
    }
    if (t == 0 && bytes && !mbar_wait_bounded(bar, 0, a.wait_limit)) {
        atomicOr(a.status, kStatusTimeout);
        s_ok = 0;
        mbar_wait_bounded(bar, 0, kDefaultWaitLimit);  // the copies must land before the CTA leaves
    }
    __syncthreads();
    const bool work = s_ok != 0;  // uniform over the CTA
    if constexpr (!kCluster) {
        if (!work) return;
    }

    unsigned int *arrivals = counts;
    const unsigned int C = gridDim.x;
    const uint32_t dmask = (1u << a.dbits) - 1u;
    const uint64_t pol_ring = l2_evict_last();
    const int64_t n0 = *a.d_step;  // the step counter changes only between launches
    for (int k = 0; k < n_steps; ++k) {
        const int64_t n = n0 + k;
        if (kCluster && !work) {  // a CTA that gave up keeps the cluster's barriers
            if (k > 0) cluster_wait();
            cluster_arrive();
            continue;
        }
        // 1. the tile's distinct history values
#pragma unroll 4
        for (int u = t; u < nu; u += T) {
            uint32_t src, d;
            if constexpr (kPacked) {
                const uint32_t kk = s_key[u];
                src = kk >> a.dbits;
                d = kk & dmask;
            } else {
                const uint2 kk = reinterpret_cast<const uint2 *>(s_key)[u];
                src = kk.x;
                d = kk.y;
            }
            const int64_t slot = (n - static_cast<int64_t>(d)) & a.ring_mask;
            cp_async4_hint(s_val + u, a.ring + slot * a.ring_stride + src, pol_ring);
        }
        cp_async_wait_all();
        __syncthreads();
        // 2. one piece per lane, 32 pieces per warp at a time, entries from shared memory
        for (int sl = warp; sl < td2.y; sl += T / 32) {
            const int2 sd = __ldg(a.st_slice + td2.x + sl);
            const float *wp = s_w + sd.x + lane;
            const uint16_t *up = s_u + sd.x + lane;
            float acc = 0.0f;
#pragma unroll 4
            for (int kk = 0; kk < sd.y; ++kk) acc = __fadd_rn(acc, __fmul_rn(wp[kk * 32], s_val[up[kk * 32]]));
            s_part[sl * 32 + lane] = acc;
        }
        __syncthreads();
        // 3. wait until step k - 1 is complete everywhere: k C arrivals
        if constexpr (kCluster) {
            if (k > 0) cluster_wait();
        } else {
            if (t == 0) s_ok = k == 0 ? 1 : lane_poll(arrivals, static_cast<unsigned int>(k) * C, limit, a.status);
            __syncthreads();
            if (!s_ok) return;
        }
        // 4. row sums and the node update of the own rows
        if (own) {
            float S = 0.0f;
            if (q1 - q0 == 1) {
                S = s_part[__ldg(a.st_plist + q0)];
            } else if (q1 - q0 == 32) {
                float x[32];
#pragma unroll
                for (int l = 0; l < 32; ++l) x[l] = s_part[__ldg(a.st_plist + q0 + l)];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1)
#pragma unroll
                    for (int l = 0; l < o; ++l) x[l] = __fadd_rn(x[l], x[l + o]);
                S = x[0];
            }
            const float2 wc = a.wc[r];
            const int32_t cnt0 = a.bg_thr ? a.bgc[r] : kLoad;
            if constexpr (kM == 0)
                node_update<kM>(a, r, n, a.ring[(n & a.ring_mask) * a.ring_stride + r], wc, S, orig, cnt0);
            else
                psc_finish(a, r, spiking_begin<kM>(a, r, n, wc, orig, cnt0, 0u), S);
        }
        // 5. arrive: this CTA's step k is complete
        if constexpr (kCluster) {
            cluster_arrive();
        } else {
            __syncthreads();
            if (t == 0) red_release_add(arrivals, 1u);
        }
    }
    if constexpr (kCluster) {
        if (n_steps > 0) cluster_wait();  // every CTA's last step is complete before any leaves
    }
}

template <int kM, int T, bool kSE, bool kPacked, bool kStream, int kMode>
cudaError_t launch_t(const StepArgs &a, int n_tiles, int k, size_t smem, cudaStream_t s)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(n_tiles));
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_step_staged<kM, T, kSE, kPacked, kStream, kMode>, a, k);
}

// One kernel instance: launch it, or (launch false) raise its dynamic shared-memory
// limit and report how many of its CTAs an SM holds.
template <int kM, int T, bool kSE, bool kPacked, bool kStream, int kMode>
cudaError_t instance(bool launch, const StepArgs *a, int n_tiles, int k, size_t smem, cudaStream_t s, int *per_sm)
{
    if (launch) return launch_t<kM, T, kSE, kPacked, kStream, kMode>(*a, n_tiles, k, smem, s);
    auto *fn = k_step_staged<kM, T, kSE, kPacked, kStream, kMode>;
    const cudaError_t e =
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    if (e != cudaSuccess || !per_sm) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, T, smem);
}

// The kernel instance of a shape, edge format and gather order (mode: see k_step_staged).
template <int kM, int T, bool kSE>
cudaError_t dispatch_fmt(bool launch, int mode, const StepArgs *a, int n_tiles, int k, bool packed,
                         bool stream_edges, size_t smem, cudaStream_t s, int *per_sm)
{
    if constexpr ((kM & kPlastic) != 0 && kSE) {
        return cudaErrorInvalidValue;  // plastic weights: entries are read from global memory
    } else {
        auto go = [&](auto e) -> cudaError_t {
            constexpr int E = decltype(e)::value;
            if (packed)
                return stream_edges ? instance<kM, T, kSE, true, true, E>(launch, a, n_tiles, k, smem, s, per_sm)
                                    : instance<kM, T, kSE, true, false, E>(launch, a, n_tiles, k, smem, s, per_sm);
            return stream_edges ? instance<kM, T, kSE, false, true, E>(launch, a, n_tiles, k, smem, s, per_sm)
                                : instance<kM, T, kSE, false, false, E>(launch, a, n_tiles, k, smem, s, per_sm);
        };
        if constexpr ((kM & kPlastic) == 0) {
            if (!launch) {  // every gather order may be launched
                cudaError_t e = go(std::integral_constant<int, 1>{});
                if (e == cudaSuccess) e = go(std::integral_constant<int, 2>{});
                if (e != cudaSuccess) return e;
                return go(std::integral_constant<int, 0>{});
            }
            if (mode == 1) return go(std::integral_constant<int, 1>{});
            if (mode == 2) return go(std::integral_constant<int, 2>{});
        } else if (mode != 0) {
            return cudaErrorInvalidValue;
        }
        return go(std::integral_constant<int, 0>{});
    }
}

cudaError_t dispatch(bool launch, const StagedShape &sh, int model, bool plastic, int early, const StepArgs *a,
                     int n_tiles, int k, bool packed, bool stream_edges, size_t smem, cudaStream_t s, int *per_sm)
{
    const bool se = sh.stage_entries != 0;
    return with_model_plastic(model, plastic, [&](auto m) {
        constexpr int M = decltype(m)::value;
        switch (sh.threads) {
            case 128:
                return se ? dispatch_fmt<M, 128, true>(launch, early, a, n_tiles, k, packed, stream_edges, smem, s, per_sm)
                          : dispatch_fmt<M, 128, false>(launch, early, a, n_tiles, k, packed, stream_edges, smem, s,
                                                        per_sm);
            case 256:
                return se ? dispatch_fmt<M, 256, true>(launch, early, a, n_tiles, k, packed, stream_edges, smem, s, per_sm)
                          : dispatch_fmt<M, 256, false>(launch, early, a, n_tiles, k, packed, stream_edges, smem, s,
                                                        per_sm);
            default: return cudaErrorInvalidValue;
        }
    });
}

}  // namespace

// {threads, gathers / edges / pieces per tile, stage entries}: shared memory per CTA
// on a net of mean in-degree 50 about 41, 13, 81, 26, 34 and 42 KB.  The last two
// let a tile of mean in-degree 50 reach its 256 rows (8192 edges stop it near 160),
// so all 8 warps have pieces to sum (1M-node net: 0.1169 ms per step with shape 3,
// 0.1392 with shape 4, 0.1126 with shape 5, which larger caps leave unchanged).  The
// last holds 1024 pieces, 32 rows of over kWarpRow edges (32 pieces each) per tile
// where the others stop at 8 or 16: at in-degree 100 (the 100k-node net) its tiles
// stop cutting short, 0.0336 ms per step against 0.0393 for the next shape; the last,
// 2048 pieces in 256-thread tiles, 0.0311.
const StagedShape kStagedShapes[kNumStagedShapes] = {
    {128, 3072, 4096, 256, 1}, {128, 3072, 4096, 256, 0}, {256, 6144, 8192, 512, 1},
    {256, 6144, 8192, 512, 0}, {256, 8192, 12288, 512, 0}, {256, 10240, 16384, 512, 0},
    {128, 4096, 8192, 1024, 1}, {256, 8192, 16384, 2048, 0}};

cudaError_t launch_step_staged(const StepArgs &a, int n_tiles, int k, const StagedShape &shape, bool packed,
                               bool stream_edges, size_t smem_bytes, int early, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    return dispatch(true, shape, a.model, a.stdp != 0, early, &a, n_tiles, k, packed, stream_edges, smem_bytes, s,
                    nullptr);
}

cudaError_t step_staged_prepare(const StagedShape &shape, int model, bool plastic, bool packed, bool stream_edges,
                                size_t smem_bytes, int *ctas_per_sm)
{
    return dispatch(false, shape, model, plastic, 0, nullptr, 0, 0, packed, stream_edges, smem_bytes, nullptr,
                    ctas_per_sm);
}

namespace {

template <int kM, bool kPacked, bool kStream, bool kFirst>
cudaError_t batch_staged_t(bool launch, const StepArgs *nets, const int *tile_net, int n_tiles, int k, size_t smem,
                           cudaStream_t s, int *per_sm)
{
    constexpr int T = kBatchStagedShape.threads;
    auto *fn = k_batch_staged<kM, T, kPacked, kStream, kFirst>;
    if (!launch) {
        const cudaError_t e =
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess || !per_sm) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, T, smem);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(n_tiles));
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, nets, tile_net, k);
}

cudaError_t batch_staged(bool launch, int model, bool first, const StepArgs *nets, const int *tile_net, int n_tiles,
                         int k, bool packed, bool stream_edges, size_t smem, cudaStream_t s, int *per_sm)
{
    return with_model(model, [&](auto m) {
        constexpr int M = decltype(m)::value;
        auto go = [&](auto f) -> cudaError_t {
            constexpr bool F = decltype(f)::value;
            if (packed)
                return stream_edges ? batch_staged_t<M, true, true, F>(launch, nets, tile_net, n_tiles, k, smem, s, per_sm)
                                    : batch_staged_t<M, true, false, F>(launch, nets, tile_net, n_tiles, k, smem, s,
                                                                        per_sm);
            return stream_edges ? batch_staged_t<M, false, true, F>(launch, nets, tile_net, n_tiles, k, smem, s, per_sm)
                                : batch_staged_t<M, false, false, F>(launch, nets, tile_net, n_tiles, k, smem, s, per_sm);
        };
        if (!launch) {  // both launch orders may be used
            const cudaError_t e = go(std::true_type{});
            if (e != cudaSuccess) return e;
            return go(std::false_type{});
        }
        return first ? go(std::true_type{}) : go(std::false_type{});
    });
}

template <int kM, bool kPacked>
cudaError_t batch_lanes_t(bool launch, const StepArgs *nets, const int *tile_net, const int2 *groups, int n_groups,
                          int lanes, int n_steps, unsigned int *counts, unsigned int *status, uint32_t limit, int grid,
                          size_t smem, cudaStream_t s, int *per_sm)
{
    constexpr int T = kBatchStagedShape.threads;
    auto *fn = k_batch_lanes<kM, T, kPacked>;
    if (!launch) {
        const cudaError_t e =
            cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess || !per_sm) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, T, smem);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(grid));
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident at once: the lane barriers need it
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, nets, tile_net, groups, n_groups, lanes, n_steps, counts, status, limit);
}

cudaError_t batch_lanes(bool launch, int model, const StepArgs *nets, const int *tile_net, const int2 *groups,
                        int n_groups, int lanes, int n_steps, unsigned int *counts, unsigned int *status,
                        uint32_t limit, bool packed, int grid, size_t smem, cudaStream_t s, int *per_sm)
{
    return with_model(model, [&](auto m) {
        constexpr int M = decltype(m)::value;
        return packed ? batch_lanes_t<M, true>(launch, nets, tile_net, groups, n_groups, lanes, n_steps, counts,
                                               status, limit, grid, smem, s, per_sm)
                      : batch_lanes_t<M, false>(launch, nets, tile_net, groups, n_groups, lanes, n_steps, counts,
                                                status, limit, grid, smem, s, per_sm);
    });
}

// One instance: launch it, or (launch false) raise its shared-memory limits and report
// how many of its CTAs an SM holds (kCluster: how many clusters of n_tiles CTAs the
// device holds at once).
template <int kM, int T, bool kPacked, bool kCluster>
cudaError_t persist_t(bool launch, const StepArgs *a, int n_tiles, int n_steps, unsigned int *counts, size_t smem,
                      cudaStream_t s, int *per_sm)
{
    auto *fn = k_step_persist<kM, T, kPacked, kCluster>;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(static_cast<unsigned>(n_tiles));
    cfg.blockDim = dim3(T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    if constexpr (kCluster) {
        attr[0].id = cudaLaunchAttributeClusterDimension;  // the whole grid is one cluster
        attr[0].val.clusterDim.x = static_cast<unsigned>(n_tiles);
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
    } else {
        attr[0].id = cudaLaunchAttributeCooperative;  // every CTA resident at once: the step barrier needs it
        attr[0].val.cooperative = 1;
    }
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (!launch) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        if (e != cudaSuccess || !per_sm) return e;
        if constexpr (kCluster) {
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveClusters(per_sm, fn, &cfg);
        }
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, fn, T, smem);
    }
    return cudaLaunchKernelEx(&cfg, fn, *a, n_steps, counts, a->wait_limit);
}

cudaError_t persist(bool launch, bool cluster, const StagedShape &sh, int model, const StepArgs *a, int n_tiles,
                    int n_steps, unsigned int *counts, bool packed, size_t smem, cudaStream_t s, int *per_sm)
{
    return with_model(model, [&](auto m) {
        constexpr int M = decltype(m)::value;
        auto go = [&](auto tt) -> cudaError_t {
            constexpr int T = decltype(tt)::value;
            if (cluster)
                return packed ? persist_t<M, T, true, true>(launch, a, n_tiles, n_steps, counts, smem, s, per_sm)
                              : persist_t<M, T, false, true>(launch, a, n_tiles, n_steps, counts, smem, s, per_sm);
            return packed ? persist_t<M, T, true, false>(launch, a, n_tiles, n_steps, counts, smem, s, per_sm)
                          : persist_t<M, T, false, false>(launch, a, n_tiles, n_steps, counts, smem, s, per_sm);
        };
        switch (sh.threads) {
            case 128: return go(std::integral_constant<int, 128>{});
            case 256: return go(std::integral_constant<int, 256>{});
            default: return cudaErrorInvalidValue;
        }
    });
}

}  // namespace

cudaError_t launch_step_persist(const StepArgs &a, int n_tiles, int n_steps, const StagedShape &shape, bool packed,
                                bool cluster, unsigned int *counts, size_t smem_bytes, cudaStream_t s)
{
    if (n_steps <= 0 || n_tiles <= 0) return cudaSuccess;
    if (cluster && n_tiles > kMaxClusterTiles) return cudaErrorInvalidValue;
    if (!cluster) {
        const cudaError_t e = cudaMemsetAsync(counts, 0, 64 * sizeof(unsigned int), s);
        if (e != cudaSuccess) return e;
    }
    return persist(true, cluster, shape, a.model, &a, n_tiles, n_steps, counts, packed, smem_bytes, s, nullptr);
}

cudaError_t step_persist_prepare(const StagedShape &shape, int model, bool packed, bool cluster, int n_tiles,
                                 size_t smem_bytes, int *fits)
{
    if (cluster && (n_tiles < 1 || n_tiles > kMaxClusterTiles)) return cudaErrorInvalidValue;
    return persist(false, cluster, shape, model, nullptr, n_tiles, 0, nullptr, packed, smem_bytes, nullptr, fits);
}

cudaError_t launch_batch_lanes(int model, const StepArgs *nets, const int *tile_net, const int2 *groups, int n_groups,
                               int lanes, int n_steps, unsigned int *counts, unsigned int *status, uint32_t limit,
                               bool packed, int grid, size_t smem_bytes, cudaStream_t s)
{
    if (n_steps <= 0 || n_groups <= 0) return cudaSuccess;
    if (lanes < 1 || lanes > kMaxBatchLanes || grid < lanes) return cudaErrorInvalidValue;
    return batch_lanes(true, model, nets, tile_net, groups, n_groups, lanes, n_steps, counts, status, limit, packed,
                       grid, smem_bytes, s, nullptr);
}

cudaError_t batch_lanes_prepare(int model, bool packed, size_t smem_bytes, int *ctas_per_sm)
{
    return batch_lanes(false, model, nullptr, nullptr, nullptr, 0, 1, 0, nullptr, nullptr, 0, packed, 0, smem_bytes,
                       nullptr, ctas_per_sm);
}

cudaError_t launch_batch_staged(int model, const StepArgs *nets, const int *tile_net, int n_tiles, int k, bool packed,
                                bool stream_edges, size_t smem_bytes, bool launch_first, cudaStream_t s)
{
    if (n_tiles <= 0) return cudaSuccess;
    return batch_staged(true, model, launch_first, nets, tile_net, n_tiles, k, packed, stream_edges, smem_bytes, s,
                        nullptr);
}

cudaError_t batch_staged_prepare(int model, bool packed, bool stream_edges, size_t smem_bytes, int *ctas_per_sm)
{
    return batch_staged(false, model, false, nullptr, nullptr, 0, 0, packed, stream_edges, smem_bytes, nullptr,
                        ctas_per_sm);
}

}  // namespace gn
