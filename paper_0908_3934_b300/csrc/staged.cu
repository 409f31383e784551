// Host builder of the staged edge layout (see StagedLayout in runtime.h and the
// kernel in k_step_staged.cu).
//
// The delayed input of Eq. Yjset (Sec. 2) reads, for every edge, one history
// value v~_src(n - D).  In a geometric network the targets of one tile share most
// sources, and many of their edges also share the delay, so a tile's gathers are
// far fewer than its edges; the builder lists them once per tile.
#include <algorithm>
#include <numeric>

#include "runtime.h"

namespace gnrt {

namespace {

// Open-addressing map from a (D, src) key to its gather index within the tile.
class TileSet {
public:
    explicit TileSet(size_t min_cap)
    {
        cap_ = 16;
        bits_ = 4;
        while (cap_ < 2 * min_cap + 2) {
            cap_ <<= 1;
            ++bits_;
        }
        key_.assign(cap_, 0);
        val_.assign(cap_, -1);
    }
    // slot of `k` (stored as k + 1; 0 marks an empty slot)
    size_t find(uint64_t k) const
    {
        size_t i = static_cast<size_t>((k * 0x9E3779B97F4A7C15ull) >> (64 - bits_));
        while (key_[i] && key_[i] != k + 1) i = (i + 1) & (cap_ - 1);
        return i;
    }
    // true if k was new
    bool insert(uint64_t k)
    {
        const size_t i = find(k);
        if (key_[i]) return false;
        key_[i] = k + 1;
        used_.push_back(i);
        return true;
    }
    size_t mark() const { return used_.size(); }
    void rollback(size_t mark)
    {
        for (size_t j = mark; j < used_.size(); ++j) key_[used_[j]] = 0;
        used_.resize(mark);
    }
    void keys(std::vector<uint64_t> &out) const
    {
        out.clear();
        for (size_t i : used_) out.push_back(key_[i] - 1);
    }
    void set_index(uint64_t k, int32_t v) { val_[find(k)] = v; }
    int32_t index(uint64_t k) const { return val_[find(k)]; }
    void clear()
    {
        for (size_t i : used_) {
            key_[i] = 0;
            val_[i] = -1;
        }
        used_.clear();
    }

private:
    size_t cap_ = 0;
    int bits_ = 0;
    std::vector<uint64_t> key_;
    std::vector<int32_t> val_;
    std::vector<size_t> used_;
};

struct Piece {
    int32_t len, first, stride;  // edges first, first + stride, ... (len of them) of the CSR
    int32_t row;                 // its row within the tile
};

// Pieces of a row of L edges, in the summation order every step kernel uses: one
// piece for a short row, 32 lane-strided pieces for a longer one.
int pieces_of(int32_t L) { return L == 0 ? 0 : L <= gn::kWarpRow ? 1 : 32; }

}  // namespace

bool build_staged(const HostNet &h, int threads, int ucap, int ecap, int pcap, StagedLayout &o)
{
    const int32_t N = h.N;
    o = StagedLayout{};
    o.threads = threads;
    const uint32_t dmask = (1u << h.dbits) - 1u;
    // (D << 32) | src: sorting the keys orders a tile's gathers by delay, then source
    auto edge_key = [&](int64_t p) -> uint64_t {
        uint32_t s, d;
        if (h.packed) {
            const uint32_t k = h.key[p];
            s = k >> h.dbits;
            d = k & dmask;
        } else {
            s = h.key[2 * p];
            d = h.key[2 * p + 1];
        }
        return (static_cast<uint64_t>(d) << 32) | s;
    };
    int32_t max_deg = 0;
    for (int32_t r = 0; r < N; ++r) max_deg = std::max(max_deg, h.row_ptr[r + 1] - h.row_ptr[r]);
    TileSet set(static_cast<size_t>(std::max(ucap, max_deg)));
    o.rq.assign(static_cast<size_t>(N) + 1, 0);
    std::vector<uint64_t> keys;
    std::vector<Piece> pcs;
    std::vector<int32_t> ord, lane_of;
    const int kw = h.packed ? 1 : 2;  // key words per gather
    auto pad_keys = [&] {
        while ((o.ukey.size() / kw) % 4) o.ukey.push_back(0);
    };

    int32_t r = 0;
    while (r < N) {
        const int32_t r0 = r;
        int nu = 0, np = 0;
        int64_t ne = 0;
        while (r < N && r - r0 < threads) {
            const int32_t e0 = h.row_ptr[r], e1 = h.row_ptr[r + 1];
            const int m = pieces_of(e1 - e0);
            const size_t mark = set.mark();
            int add = 0;
            for (int32_t e = e0; e < e1; ++e) add += set.insert(edge_key(e)) ? 1 : 0;
            if (r > r0 && (nu + add > ucap || np + m > pcap || ne + (e1 - e0) > ecap)) {
                set.rollback(mark);
                break;
            }
            nu += add;
            np += m;
            ne += e1 - e0;
            ++r;
        }
        const int ns = (np + 31) / 32;
        if (nu > 65535 || ns * 32 > 65535) return false;

        // the tile's gathers, sorted by (D, src)
        set.keys(keys);
        std::sort(keys.begin(), keys.end());
        for (int j = 0; j < nu; ++j) set.set_index(keys[j], j);
        o.tile.push_back(make_int4(r0, r - r0, static_cast<int>(o.ukey.size() / kw), nu));
        for (uint64_t k : keys) {
            const uint32_t s = static_cast<uint32_t>(k), d = static_cast<uint32_t>(k >> 32);
            if (h.packed) {
                o.ukey.push_back((s << h.dbits) | d);
            } else {
                o.ukey.push_back(s);
                o.ukey.push_back(d);
            }
        }
        pad_keys();

        // pieces: a short row whole, a longer one as lanes l = 0..31 taking edges l, l + 32, ...
        pcs.clear();
        for (int32_t rr = r0; rr < r; ++rr) {
            const int32_t e0 = h.row_ptr[rr], e1 = h.row_ptr[rr + 1];
            const int32_t L = e1 - e0;
            const int m = pieces_of(L);
            if (m == 1) pcs.push_back({L, e0, 1, rr - r0});
            for (int q = 0; q < m && m == 32; ++q) pcs.push_back({(L - q + 31) / 32, e0 + q, 32, rr - r0});
        }
        ord.resize(np);
        std::iota(ord.begin(), ord.end(), 0);
        std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return pcs[a].len > pcs[b].len; });
        lane_of.assign(np, 0);
        for (int i = 0; i < np; ++i) lane_of[ord[i]] = i;
        {
            int pi = 0;
            for (int32_t rr = r0; rr < r; ++rr) {
                o.rq[rr] = static_cast<int32_t>(o.plist.size());
                const int m = pieces_of(h.row_ptr[rr + 1] - h.row_ptr[rr]);
                for (int q = 0; q < m; ++q) o.plist.push_back(static_cast<uint16_t>(lane_of[pi++]));
            }
        }

        // slices of 32 pieces, entries column-major
        const bool plastic = !h.eorig.empty();
        const size_t x0 = o.w.size();
        for (int s = 0; s < ns; ++s) {
            const int32_t len = pcs[ord[32 * s]].len;
            const size_t off = o.w.size();
            if (off + static_cast<size_t>(len) * 32 >= (1ull << 31)) return false;
            o.slice.push_back(make_int2(static_cast<int>(off - x0), len));
            o.w.resize(off + static_cast<size_t>(len) * 32, 0.0f);
            o.u.resize(off + static_cast<size_t>(len) * 32, 0);
            if (plastic) o.eidx.resize(off + static_cast<size_t>(len) * 32, -1);
            for (int lane = 0; lane < 32; ++lane) {
                if (32 * s + lane >= np) {
                    if (plastic) o.pinfo.push_back(0u);
                    continue;
                }
                const Piece &pc = pcs[ord[32 * s + lane]];
                if (plastic) o.pinfo.push_back(static_cast<uint32_t>(pc.len) | (static_cast<uint32_t>(pc.row) << 16));
                for (int32_t k = 0; k < pc.len; ++k) {
                    const int64_t e = pc.first + static_cast<int64_t>(k) * pc.stride;
                    o.w[off + static_cast<size_t>(k) * 32 + lane] = h.w[e];
                    o.u[off + static_cast<size_t>(k) * 32 + lane] = static_cast<uint16_t>(set.index(edge_key(e)));
                    if (plastic) o.eidx[off + static_cast<size_t>(k) * 32 + lane] = h.eorig[e];
                }
            }
        }
        const int nx = static_cast<int>(o.w.size() - x0);
        o.tile2.push_back(make_int4(static_cast<int>(o.slice.size()) - ns, ns, static_cast<int>(x0), nx));
        o.max_u = std::max(o.max_u, (nu + 3) / 4 * 4);
        o.max_x = std::max(o.max_x, nx);
        o.max_p = std::max(o.max_p, ns * 32);
        set.clear();
    }
    o.rq[N] = static_cast<int32_t>(o.plist.size());
    // never-empty arrays keep every device pointer valid
    if (o.ukey.empty()) o.ukey.assign(4 * kw, 0);
    if (o.w.empty()) {
        o.w.push_back(0.0f);
        o.u.push_back(0);
        if (!h.eorig.empty()) o.eidx.push_back(-1);
    }
    if (o.plist.empty()) o.plist.push_back(0);
    if (o.slice.empty()) o.slice.push_back(make_int2(0, 0));
    if (!h.eorig.empty() && o.pinfo.empty()) o.pinfo.push_back(0u);
    return true;
}

}  // namespace gnrt
