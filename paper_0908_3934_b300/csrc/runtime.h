// Internal host runtime shared by the single-network (net.cu) and batched
// (batch.cu) parts of libgeonet.so: error handling, device arrays, descriptor
// validation, delay quantisation and the host-side build of one network.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/geonet.h"
#include "internal.cuh"

namespace gnrt {

struct Fail {
    gn_status st;
};

// Record a message for gn_last_error() and throw; only guarded() catches it.
[[noreturn]] void fail(gn_status st, const char *fmt, ...);
void set_error(const std::string &msg);
const char *last_error();
void cuda_check(cudaError_t e, const char *what);

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev);
    ~DeviceGuard();
};

// A device allocation that keeps the owner's byte count (`total`) current: alloc
// adds its size, release subtracts it.
template <class T>
struct DevArray {
    T *p = nullptr;
    size_t n = 0;
    size_t *counted = nullptr;
    void alloc(size_t count, size_t *total)
    {
        n = count;
        if (count == 0) return;
        cuda_check(cudaMalloc(reinterpret_cast<void **>(&p), count * sizeof(T)), "cudaMalloc");
        *total += count * sizeof(T);
        counted = total;
    }
    void upload(const std::vector<T> &v, size_t *total)
    {
        alloc(v.size(), total);
        if (!v.empty()) cuda_check(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice), "H2D");
    }
    void release()
    {
        if (p) {
            cudaFree(p);
            if (counted) *counted -= n * sizeof(T);
        }
        p = nullptr;
        n = 0;
        counted = nullptr;
    }
};

gn_status guarded_call(void (*fn)(void *), void *ctx);

template <class F>
gn_status guarded(F &&f)
{
    return guarded_call([](void *c) { (*static_cast<F *>(c))(); }, &f);
}

// Rest point of the isolated FHN vertex (S = U = 0): W = (V + f)/g and
// a V - b V^3 - c (V + f)/g + I = 0, unique when g > 0, b > 0, a < c/g.
bool rest_point(const gn_fhn_params &p, double *v_out, double *w_out);

void validate_desc(const gn_net_desc *d);

// FP64 delay quantisation of several networks in one launch (geometric ones;
// explicit tables are copied).  delay[i] in caller edge order of network i.
void quantise_delays(const gn_net_desc *descs, int n_nets, cudaStream_t s, std::vector<std::vector<int32_t>> &delay,
                     std::vector<int64_t> &n_clamped);

// Host-side products of one network, ready to upload.
struct HostNet {
    int32_t N = 0, dim = 0;
    int64_t E = 0;
    int32_t R = 0, dbits = 0, dmax = 1, dmin = 1, stride = 0;
    int64_t n_clamped = 0;
    bool packed = true;
    int32_t model = GN_MODEL_FHN;
    double v_rest = 0.0, w_rest = 0.0;   // FHN: the rest point; Izhikevich: (v_r, 0)
    std::vector<int32_t> perm, inv, delay;   // perm: internal -> caller; delay: caller edge order
    std::vector<uint32_t> key;               // [E + pad] packed, or [2 (E + pad)] wide
    std::vector<float> w;                    // [E + pad]
    std::vector<float> bias;                 // [N], RAW coupling only
    std::vector<int32_t> row_ptr;            // [N + 1 + 8]
    std::vector<int32_t> blk;                // [n_blocks + 1]
    std::vector<int4> desc;                  // [n_blocks] {r0, r1, e0, e1}
    std::vector<int32_t> eorig;              // plastic nets: caller edge of each CSR position
    std::vector<uint8_t> cell;               // heterogeneous cells: parameter set of each node (internal order)
    std::vector<float> type_par;             // [n_types][gn::kTypeStride] derived per-set parameters
    std::vector<float> v0;                   // spiking models: starting V of each node (internal order)
    int n_blocks() const { return static_cast<int>(blk.size()) - 1; }
};

// Ring depth, renumbering, CSR by target (rows sorted by source), edge packing and
// row blocks of at most block_cap - 3 edges and block_rows rows.
void host_build(const gn_net_desc *d, std::vector<int32_t> delay, int64_t n_clamped, int block_cap, int block_rows,
                HostNet &h);

// Row blocks of consecutive rows with at most cap - 3 edges and max_rows rows
// (a longer row alone), and their {r0, r1, e0, e1} descriptors.
void make_blocks(const std::vector<int32_t> &row_ptr, int32_t N, int cap, int max_rows, std::vector<int32_t> &blk,
                 std::vector<int4> &desc);

// Staged layout of the by-target edge list (k_step_staged.cu).  Consecutive rows
// form a tile of at most `threads` rows.  A tile lists the distinct (source, delay)
// pairs its edges read -- its gathers -- sorted by (delay, source), so one CTA
// fetches each history value once per step into shared memory.  Every row is cut
// into pieces in the shared summation order (kWarpRow in internal.cuh): a row of at
// most kWarpRow edges is one piece, a longer row 32 lane-strided pieces.  A tile's
// pieces are sorted by length (longest first) and each lane of the CTA sums one
// piece, reading its edges as (weight, index of the gather) column by column in
// slices of 32 pieces.
//
// A tile's gather keys and its entries are contiguous and 16-byte aligned, so the
// CTA copies them into shared memory with two or three bulk copies: keys start at
// a multiple of 4 and are padded to a multiple of 4; entries come in slices of
// 32 x length.
struct StagedLayout {
    int threads = 0;
    std::vector<int4> tile;        // {first row, rows, first gather (multiple of 4), gathers}
    std::vector<int4> tile2;       // {first slice, slices, first entry, entries}
    std::vector<uint32_t> ukey;    // per gather: packed key, or {src, D} (wide)
    std::vector<int2> slice;       // {first entry relative to the tile's, length}: entries k * 32 + lane
    std::vector<float> w;          // entry weights (0 in the padding)
    std::vector<uint16_t> u;       // entry gather index within the tile (0 in the padding)
    std::vector<int32_t> rq;       // [N + 1] first piece-list entry of each row
    std::vector<uint16_t> plist;   // lane slot (32 * slice + lane) of each piece, rows in order
    // plastic nets only: the caller edge of each entry (-1: padding), and per lane slot
    // (32 * global slice + lane) its piece's length | local row << 16
    std::vector<int32_t> eidx;
    std::vector<uint32_t> pinfo;
    int max_u = 0, max_x = 0, max_p = 0;  // largest padded gather count, entries, lane slots of a tile
    // shared memory of one CTA: mbarrier, keys (wide keys need a separate value
    // array; packed values overwrite their keys), entry weights and indices when
    // they are staged, piece sums
    size_t smem_bytes(bool packed, bool stage_entries = true) const
    {
        return 16 + static_cast<size_t>(max_u) * (packed ? 4 : 12) +
               (stage_entries ? static_cast<size_t>(max_x) * 6 : 0) + static_cast<size_t>(max_p) * 4;
    }
};

// Build the staged layout from the CSR of `h`: tiles close at `threads` rows,
// `ucap` gathers, `ecap` edges or `pcap` pieces (a row that alone exceeds a cap
// gets a tile of its own).  Returns false if a tile would need more than 65535
// gathers or lane slots, or 2^31 entries in total.
bool build_staged(const HostNet &h, int threads, int ucap, int ecap, int pcap, StagedLayout &out);

// Scalar fields of the step arguments (FHN about the rest point, readout, sizes).
void fill_step_params(const gn_net_desc *d, const HostNet &h, gn::StepArgs &a);
// Per-set parameter rows of a heterogeneous network, in the order of the step
// arguments' scalar fields (Izhikevich: dt/C, k, v_r, v_t, v_peak, v_reset, dt a, b,
// d, i_ext; Hodgkin-Huxley: dt/C, g_Na, g_K, g_L, E_Na, E_K, E_L, v_peak, i_ext),
// then at gn::kTypeA2 for both: a_s^2, 2 a_s, 1/tau_c.
std::vector<float> cell_type_rows(const gn_net_desc *d);
// Hodgkin-Huxley gates at -65 mV, x = alpha / (alpha + beta) of the classic rates.
void hh_rest_gates(double *m, double *n, double *h);

// Pulses (caller node ids, ms) -> sorted by internal node, steps; invalid -> GN_EINVAL.
struct PulseTable {
    std::vector<int32_t> node;
    std::vector<int64_t> on, off;
    std::vector<float> amp;
};
PulseTable make_pulses(const gn_pulse *pulses, int32_t n, int32_t n_nodes, double dt, const std::vector<int32_t> &inv);

// Background onset threshold floor(p 2^32), p = rate * dt.
uint32_t background_threshold(double rate_hz, double dt_ms);

}  // namespace gnrt
