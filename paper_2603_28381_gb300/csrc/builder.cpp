// builder.cpp -- host-side validation, levelization and device layout.
//
// Levelization follows the paper's stage (2) (Section 2.1): nets are grouped
// into levels so that the pins of level i only need arrival times of levels
// < i; it is computed once per netlist (Section 2.1, "needs to be computed only
// once").  Here it is a Kahn breadth-first sweep over the net graph: level 0
// for a net whose driver is not a cell output, else 1 + the largest level of
// the nets feeding the driver cell's inputs.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <numeric>

#include "sta_internal.h"

namespace sta {
namespace {

struct Roles {
    std::vector<int32_t> sink_net, drv_net, out_cell, in_cell, start_of, end_of;
};

bool fail(std::string& err, const std::string& msg) {
    err = msg;
    return false;
}

// Structural checks on the description; fills the role of every pin.
StaStatus check_netlist(const StaNetlistDesc& nl, const StaLibrary* lib, Roles& r, std::string& err) {
    const int32_t P = nl.num_pins, N = nl.num_nets, C = nl.num_cells;
    if (P < 0 || N < 0 || C < 0 || nl.num_start < 0 || nl.num_end < 0)
        return err = "negative size", STA_ERR_INVALID_ARG;
    if ((N > 0 && (!nl.net_ptr || !nl.net_pins)) || (C > 0 && (!nl.cell_type || !nl.cell_in_ptr ||
        !nl.cell_in_pins || !nl.cell_out_pin)) || (P > 0 && !nl.pin_cap) ||
        (nl.num_start > 0 && (!nl.start_pins || !nl.start_at || !nl.start_slew)) ||
        (nl.num_end > 0 && (!nl.end_pins || !nl.end_rat)))
        return err = "null array with non-zero size", STA_ERR_INVALID_ARG;
    if (!(std::isfinite(nl.r_per_um) && nl.r_per_um >= 0 && std::isfinite(nl.c_per_um) && nl.c_per_um >= 0))
        return err = "r_per_um / c_per_um must be finite and >= 0", STA_ERR_INVALID_ARG;
    r.sink_net.assign(P, -1);
    r.drv_net.assign(P, -1);
    r.out_cell.assign(P, -1);
    r.in_cell.assign(P, -1);
    r.start_of.assign(P, -1);
    r.end_of.assign(P, -1);
    if (N > 0 && nl.net_ptr[0] != 0) return err = "net_ptr[0] must be 0", STA_ERR_INVALID_ARG;
    for (int32_t n = 0; n < N; ++n) {
        const int32_t b = nl.net_ptr[n], e = nl.net_ptr[n + 1];
        if (e <= b) return err = "net " + std::to_string(n) + " has no driver", STA_ERR_INVALID_ARG;
        for (int32_t k = b; k < e; ++k) {
            const int32_t p = nl.net_pins[k];
            if (p < 0 || p >= P) return err = "net pin out of range", STA_ERR_INVALID_ARG;
            if (k == b) {
                if (r.drv_net[p] >= 0 || r.sink_net[p] >= 0)
                    return err = "pin " + std::to_string(p) + " on two nets", STA_ERR_INVALID_ARG;
                r.drv_net[p] = n;
            } else {
                if (r.sink_net[p] >= 0 || r.drv_net[p] >= 0)
                    return err = "pin " + std::to_string(p) + " on two nets", STA_ERR_INVALID_ARG;
                r.sink_net[p] = n;
            }
        }
    }
    for (int32_t c = 0; c < C; ++c) {
        const int32_t t = nl.cell_type[c], o = nl.cell_out_pin[c];
        const int32_t k = nl.cell_in_ptr[c + 1] - nl.cell_in_ptr[c];
        if (nl.cell_in_ptr[0] != 0 || k < 1 || k > STA_MAX_ARCS)
            return err = "cell " + std::to_string(c) + " must have 1..4 inputs", STA_ERR_INVALID_ARG;
        if (lib && (t < 0 || t >= lib->num_types || lib->type_num_arcs[t] != k))
            return err = "cell " + std::to_string(c) + " type / input count mismatch", STA_ERR_INVALID_ARG;
        if (o < 0 || o >= P || r.out_cell[o] >= 0)
            return err = "bad or repeated cell output pin", STA_ERR_INVALID_ARG;
        r.out_cell[o] = c;
        for (int32_t a = nl.cell_in_ptr[c]; a < nl.cell_in_ptr[c + 1]; ++a) {
            const int32_t p = nl.cell_in_pins[a];
            if (p < 0 || p >= P || r.in_cell[p] >= 0)
                return err = "bad or repeated cell input pin", STA_ERR_INVALID_ARG;
            r.in_cell[p] = c;
        }
    }
    for (int32_t s = 0; s < nl.num_start; ++s) {
        const int32_t p = nl.start_pins[s];
        if (p < 0 || p >= P || r.start_of[p] >= 0) return err = "bad or repeated startpoint", STA_ERR_INVALID_ARG;
        for (int q = 0; q < 4; ++q)
            if (!std::isfinite(nl.start_at[4 * s + q]) || !std::isfinite(nl.start_slew[4 * s + q]) ||
                nl.start_slew[4 * s + q] < 0)
                return err = "startpoint AT/slew must be finite, slew >= 0", STA_ERR_INVALID_ARG;
        r.start_of[p] = s;
    }
    for (int32_t e = 0; e < nl.num_end; ++e) {
        const int32_t p = nl.end_pins[e];
        if (p < 0 || p >= P || r.end_of[p] >= 0) return err = "bad or repeated endpoint", STA_ERR_INVALID_ARG;
        if (r.sink_net[p] < 0 || r.in_cell[p] >= 0)
            return err = "endpoint " + std::to_string(p) + " must be a net sink that is not a cell input",
                   STA_ERR_INVALID_ARG;
        for (int q = 0; q < 4; ++q)
            if (!std::isfinite(nl.end_rat[4 * e + q])) return err = "endpoint RAT must be finite", STA_ERR_INVALID_ARG;
        r.end_of[p] = e;
    }
    if (nl.end_clock && nl.num_end > 0) {
        std::vector<uint8_t> used(P, 0);
        for (int32_t e = 0; e < nl.num_end; ++e) {
            const int32_t k = nl.end_clock[e];
            if (k == -1) continue;
            if (k < -1 || k >= P) return err = "end_clock out of range", STA_ERR_INVALID_ARG;
            if (r.sink_net[k] < 0 || r.start_of[nl.net_pins[nl.net_ptr[r.sink_net[k]]]] < 0 || r.in_cell[k] < 0 ||
                nl.cell_in_ptr[r.in_cell[k] + 1] - nl.cell_in_ptr[r.in_cell[k]] != 1)
                return err = "capturing clock pin " + std::to_string(k) +
                             " must be the input of a one-input cell on a net driven by a startpoint",
                       STA_ERR_INVALID_ARG;
            if (used[k]++) return err = "clock pin " + std::to_string(k) + " captures two endpoints",
                                  STA_ERR_INVALID_ARG;
        }
    }
    for (int32_t p = 0; p < P; ++p) {
        const int nsrc = (r.start_of[p] >= 0) + (r.sink_net[p] >= 0) + (r.out_cell[p] >= 0);
        if (nsrc != 1)
            return err = "pin " + std::to_string(p) + " must have exactly one arrival source "
                         "(startpoint, net sink or cell output)", STA_ERR_INVALID_ARG;
        if (r.drv_net[p] >= 0 && r.in_cell[p] >= 0)
            return err = "pin " + std::to_string(p) + " drives a net and is a cell input", STA_ERR_INVALID_ARG;
        if (!(std::isfinite(nl.pin_cap[p]) && nl.pin_cap[p] >= 0))
            return err = "pin_cap must be finite and >= 0", STA_ERR_INVALID_ARG;
    }
    return STA_OK;
}

StaStatus check_library(const StaLibrary& lib, std::string& err) {
    if (lib.num_types < 1 || !lib.type_num_arcs || !lib.arc_unate || !lib.slew_index || !lib.load_index ||
        !lib.delay_tab || !lib.slew_tab)
        return err = "library arrays missing", STA_ERR_INVALID_ARG;
    for (int32_t t = 0; t < lib.num_types; ++t) {
        if (lib.type_num_arcs[t] < 1 || lib.type_num_arcs[t] > STA_MAX_ARCS)
            return err = "type_num_arcs must be 1..4", STA_ERR_INVALID_ARG;
        for (int a = 0; a < STA_MAX_ARCS; ++a)
            if (lib.arc_unate[t * STA_MAX_ARCS + a] != 1 && lib.arc_unate[t * STA_MAX_ARCS + a] != -1)
                return err = "arc_unate must be +1 or -1", STA_ERR_INVALID_ARG;
        for (int k = 0; k < STA_LUT; ++k) {
            const float s = lib.slew_index[t * STA_LUT + k], l = lib.load_index[t * STA_LUT + k];
            if (!std::isfinite(s) || !std::isfinite(l)) return err = "non-finite table index", STA_ERR_INVALID_ARG;
            if (k > 0 && !(s > lib.slew_index[t * STA_LUT + k - 1] && l > lib.load_index[t * STA_LUT + k - 1]))
                return err = "table indices must be strictly increasing", STA_ERR_INVALID_ARG;
        }
    }
    const size_t ntab = (size_t)lib.num_types * STA_MAX_ARCS * 2 * STA_LUT * STA_LUT;
    for (size_t i = 0; i < ntab; ++i)
        if (!std::isfinite(lib.delay_tab[i]) || !std::isfinite(lib.slew_tab[i]))
            return err = "non-finite table value", STA_ERR_INVALID_ARG;
    return STA_OK;
}

// Kahn sweep over "level nodes": description nets 0..N-1 then one node per
// dangling cell.  level = 0 without fanin nets, else 1 + max fanin level.
StaStatus kahn_levels(const StaNetlistDesc& nl, const Roles& r, const std::vector<int32_t>& dangling,
                      std::vector<int32_t>& level, int32_t& num_levels, std::string& err) {
    const int32_t N = nl.num_nets, D = (int32_t)dangling.size(), V = N + D;
    // fanin nets of each node
    auto node_cell = [&](int32_t v) -> int32_t {
        return v < N ? r.out_cell[nl.net_pins[nl.net_ptr[v]]] : dangling[v - N];
    };
    std::vector<int32_t> indeg(V, 0), fo_cnt(N + 1, 0);
    for (int32_t v = 0; v < V; ++v) {
        const int32_t c = node_cell(v);
        if (c < 0) continue;
        for (int32_t a = nl.cell_in_ptr[c]; a < nl.cell_in_ptr[c + 1]; ++a) {
            const int32_t m = r.sink_net[nl.cell_in_pins[a]];
            if (m >= 0) { ++indeg[v]; ++fo_cnt[m + 1]; }
        }
    }
    for (int32_t m = 0; m < N; ++m) fo_cnt[m + 1] += fo_cnt[m];
    std::vector<int32_t> fo(fo_cnt[N]), fill(fo_cnt.begin(), fo_cnt.end() - 1);
    for (int32_t v = 0; v < V; ++v) {
        const int32_t c = node_cell(v);
        if (c < 0) continue;
        for (int32_t a = nl.cell_in_ptr[c]; a < nl.cell_in_ptr[c + 1]; ++a) {
            const int32_t m = r.sink_net[nl.cell_in_pins[a]];
            if (m >= 0) fo[fill[m]++] = v;
        }
    }
    level.assign(V, 0);
    std::vector<int32_t> queue;
    queue.reserve(V);
    for (int32_t v = 0; v < V; ++v) if (indeg[v] == 0) queue.push_back(v);
    size_t head = 0;
    int32_t maxl = -1;
    while (head < queue.size()) {
        const int32_t m = queue[head++];
        maxl = std::max(maxl, level[m]);
        if (m >= N) continue;
        for (int32_t k = fo_cnt[m]; k < fo_cnt[m + 1]; ++k) {
            const int32_t v = fo[k];
            level[v] = std::max(level[v], level[m] + 1);
            if (--indeg[v] == 0) queue.push_back(v);
        }
    }
    if ((int32_t)queue.size() != V) return err = "timing graph has a cycle", STA_ERR_NOT_DAG;
    num_levels = maxl + 1;
    return STA_OK;
}

std::vector<int32_t> dangling_cells(const StaNetlistDesc& nl, const Roles& r) {
    std::vector<int32_t> d;
    for (int32_t c = 0; c < nl.num_cells; ++c)
        if (r.drv_net[nl.cell_out_pin[c]] < 0) d.push_back(c);
    return d;
}

}  // namespace

StaStatus levelize(const StaNetlistDesc& nl, const StaLibrary* lib, std::vector<int32_t>& net_level,
                   std::vector<int32_t>* dangling_out, std::vector<int32_t>* dangling_level,
                   int32_t& num_levels, std::string& err) {
    Roles r;
    StaStatus st = check_netlist(nl, lib, r, err);
    if (st != STA_OK) return st;
    std::vector<int32_t> dang = dangling_cells(nl, r), lv;
    st = kahn_levels(nl, r, dang, lv, num_levels, err);
    if (st != STA_OK) return st;
    net_level.assign(lv.begin(), lv.begin() + nl.num_nets);
    if (dangling_out) *dangling_out = dang;
    if (dangling_level) dangling_level->assign(lv.begin() + nl.num_nets, lv.end());
    return STA_OK;
}

namespace {

// Internal net order: level; within a level the nets of <= 32 pins before the
// larger ones, then by the latest position (in this order) of a net feeding the
// driver cell, then id; ids >= num_nets are dangling cells.  Grouping the nets
// that read the same, nearby producers makes a packed task wait for fewer
// producer tasks of the level before (1.8 instead of 6 on average at 500k pins).
struct NetOrder {
    std::vector<int32_t> order;   // internal -> level-node id
    std::vector<int32_t> level;   // per level-node
    int32_t L = 0;
};

StaStatus make_order(const StaNetlistDesc& nl, const Roles& r, const std::vector<int32_t>& dang,
                     NetOrder& no, std::string& err) {
    StaStatus st = kahn_levels(nl, r, dang, no.level, no.L, err);
    if (st != STA_OK) return st;
    const int32_t N = nl.num_nets, V = N + (int32_t)dang.size();
    std::vector<int64_t> key(V);
    for (int32_t v = 0; v < V; ++v) {
        const int32_t size = v < N ? nl.net_ptr[v + 1] - nl.net_ptr[v] : 1;
        key[v] = ((int64_t)no.level[v] << 33) | ((int64_t)(size > kWarpPins) << 32) | (int64_t)v;
    }
    no.order.resize(V);
    std::iota(no.order.begin(), no.order.end(), 0);
    std::sort(no.order.begin(), no.order.end(), [&](int32_t a, int32_t b) { return key[a] < key[b]; });
    // within each level: (size class, latest position of a fanin net (-1: none), id)
    std::vector<int64_t> pos(V, -1), fk(V, -1);
    size_t i = 0;
    while (i < no.order.size()) {
        size_t j = i;
        const int32_t l = no.level[no.order[i]];
        while (j < no.order.size() && no.level[no.order[j]] == l) ++j;
        for (size_t k = i; k < j; ++k) {
            const int32_t v = no.order[k];
            const int32_t c = v < N ? r.out_cell[nl.net_pins[nl.net_ptr[v]]] : dang[v - N];
            int64_t m = -1;
            if (c >= 0)
                for (int32_t a = nl.cell_in_ptr[c]; a < nl.cell_in_ptr[c + 1]; ++a) {
                    const int32_t f = r.sink_net[nl.cell_in_pins[a]];
                    if (f >= 0) m = std::max(m, pos[f]);
                }
            fk[v] = m;
        }
        std::sort(no.order.begin() + i, no.order.begin() + j, [&](int32_t a, int32_t b) {
            const int sa = (key[a] >> 32) & 1, sb = (key[b] >> 32) & 1;
            if (sa != sb) return sa < sb;
            if (fk[a] != fk[b]) return fk[a] < fk[b];
            return a < b;
        });
        for (size_t k = i; k < j; ++k) pos[no.order[k]] = (int64_t)k;
        i = j;
    }
    return STA_OK;
}

}  // namespace

StaStatus ordering(const StaNetlistDesc& nl, std::vector<int32_t>& net_level, int32_t& num_levels,
                   std::vector<int32_t>& net_order, std::vector<int32_t>& pin_order, std::string& err) {
    Roles r;
    StaStatus st = check_netlist(nl, nullptr, r, err);
    if (st != STA_OK) return st;
    std::vector<int32_t> dang = dangling_cells(nl, r);
    NetOrder no;
    st = make_order(nl, r, dang, no, err);
    if (st != STA_OK) return st;
    num_levels = no.L;
    net_level.assign(no.level.begin(), no.level.begin() + nl.num_nets);
    net_order.clear();
    pin_order.clear();
    for (int32_t v : no.order) {
        if (v >= nl.num_nets) continue;
        net_order.push_back(v);
        const int32_t b = nl.net_ptr[v], e = nl.net_ptr[v + 1];
        pin_order.push_back(nl.net_pins[b]);
        std::vector<int32_t> s(nl.net_pins + b + 1, nl.net_pins + e);
        std::sort(s.begin(), s.end());
        pin_order.insert(pin_order.end(), s.begin(), s.end());
    }
    return STA_OK;
}

StaStatus build_tasks(Layout& o, const TaskShape& sh, std::string& err) {
    if (sh.pack_pins < 1 || sh.pack_nets < 1 || sh.big < 1 || sh.chunk < 1)
        return err = "task shape: every field must be >= 1", STA_ERR_INVALID_ARG;
    const int32_t P = o.P, V = o.N, A = o.A;
    o.shape = sh;
    // forward: per level, packed nets of at most `big` pins (several nets while
    // they fit in pack_pins, at most pack_nets), then chunks of `chunk` sinks of
    // the larger nets
    std::vector<int32_t> pin_fprod(P, -1), net_step(V, -1);
    std::vector<int32_t> bigs;
    std::vector<std::vector<int32_t>> lvl_big(o.L), lvl_pack(o.L);  // pack: (n0, nn) pairs
    for (int32_t l = 0; l < o.L; ++l) {
        for (int32_t i = o.lvl_net[l]; i < o.lvl_net[l + 1];) {
            const int32_t sz = o.net_ptr[i + 1] - o.net_ptr[i];
            if (sz > sh.big) {
                lvl_big[l].push_back(i++);
                continue;
            }
            int32_t n0 = i, pins = 0, cnt = 0;
            while (i < o.lvl_net[l + 1] && cnt < sh.pack_nets) {
                const int32_t z = o.net_ptr[i + 1] - o.net_ptr[i];
                if (z > sh.big || (cnt > 0 && pins + z > sh.pack_pins)) break;
                pins += z;
                ++cnt;
                ++i;
            }
            lvl_pack[l].push_back(n0);
            lvl_pack[l].push_back(cnt);
        }
    }
    o.ftask.clear();
    o.lvl_ftask.assign(o.L + 1, 0);
    for (int32_t l = 0; l < o.L; ++l) {
        o.lvl_ftask[l] = (int32_t)(o.ftask.size() / 4);
        for (size_t k = 0; k < lvl_pack[l].size(); k += 2) {
            const int32_t n0 = lvl_pack[l][k], nn = lvl_pack[l][k + 1];
            const int32_t t = (int32_t)(o.ftask.size() / 4);
            const int32_t p0 = o.net_ptr[n0], p1 = o.net_ptr[n0 + nn];
            o.ftask.insert(o.ftask.end(), {n0, nn, p0, p1 - p0});
            for (int32_t p = p0; p < p1; ++p) pin_fprod[p] = t;
        }
        for (int32_t n : lvl_big[l]) {
            for (int32_t p0 = o.net_ptr[n] + 1; p0 < o.net_ptr[n + 1]; p0 += sh.chunk) {
                const int32_t cnt = std::min(sh.chunk, o.net_ptr[n + 1] - p0);
                const int32_t t = (int32_t)(o.ftask.size() / 4);
                o.ftask.insert(o.ftask.end(), {n, -1, p0, cnt});
                for (int32_t p = p0; p < p0 + cnt; ++p) pin_fprod[p] = t;
            }
            bigs.push_back(n);
        }
    }
    o.big_nets = bigs;
    o.TF = (int32_t)(o.ftask.size() / 4);
    o.lvl_ftask[o.L] = o.TF;
    // every pin on a net has exactly one forward task (its net's task, or the
    // chunk holding the sink; a large net's driver belongs to its chunks)
    for (int32_t n = 0; n < V; ++n)
        for (int32_t p = o.net_ptr[n] + 1; p < o.net_ptr[n + 1]; ++p)
            if (pin_fprod[p] < 0) return err = "internal: a sink without a forward task", STA_ERR_INVALID_ARG;
    o.arc_prod.resize(A);
    for (int32_t a = 0; a < A; ++a) o.arc_prod[a] = pin_fprod[o.arc_pin[a]];

    // backward: per level in reverse, partial chunks of the large nets, their
    // driver steps, the packed nets, then the gradient chunks of the large nets
    o.btask.clear();
    o.baux.clear();
    o.npart = 0;
    o.lvl_bsec.assign((size_t)o.L * 5, 0);
    for (int32_t l = o.L - 1; l >= 0; --l) {
        const size_t nb = lvl_big[l].size();
        int32_t* sec = &o.lvl_bsec[(size_t)l * 5];
        sec[0] = (int32_t)o.baux.size();
        std::vector<int32_t> first_ptask(nb), first_slot(nb), nchunks(nb), dtask(nb);
        for (size_t k = 0; k < nb; ++k) {
            const int32_t n = lvl_big[l][k];
            first_ptask[k] = (int32_t)o.baux.size();
            first_slot[k] = o.npart;
            for (int32_t p0 = o.net_ptr[n] + 1; p0 < o.net_ptr[n + 1]; p0 += sh.chunk) {
                const int32_t cnt = std::min(sh.chunk, o.net_ptr[n + 1] - p0);
                o.btask.insert(o.btask.end(), {n, -1, p0, cnt});
                o.baux.push_back(o.npart++);
            }
            nchunks[k] = o.npart - first_slot[k];
        }
        sec[1] = (int32_t)o.baux.size();
        for (size_t k = 0; k < nb; ++k) {
            const int32_t n = lvl_big[l][k];
            dtask[k] = (int32_t)o.baux.size();
            net_step[n] = dtask[k];
            o.btask.insert(o.btask.end(), {n, -2, first_slot[k], nchunks[k]});
            o.baux.push_back(first_ptask[k]);
        }
        sec[2] = (int32_t)o.baux.size();
        for (size_t k = 0; k < lvl_pack[l].size(); k += 2) {
            const int32_t n0 = lvl_pack[l][k], nn = lvl_pack[l][k + 1];
            const int32_t t = (int32_t)o.baux.size();
            o.btask.insert(o.btask.end(), {n0, nn, o.net_ptr[n0], o.net_ptr[n0 + nn] - o.net_ptr[n0]});
            o.baux.push_back(0);
            for (int32_t n = n0; n < n0 + nn; ++n) net_step[n] = t;
        }
        sec[3] = (int32_t)o.baux.size();
        for (size_t k = 0; k < nb; ++k) {
            const int32_t n = lvl_big[l][k];
            for (int32_t p0 = o.net_ptr[n] + 1; p0 < o.net_ptr[n + 1]; p0 += sh.chunk) {
                const int32_t cnt = std::min(sh.chunk, o.net_ptr[n + 1] - p0);
                o.btask.insert(o.btask.end(), {n, -3, p0, cnt});
                o.baux.push_back(dtask[k]);
            }
        }
        sec[4] = (int32_t)o.baux.size();
    }
    o.TB = (int32_t)o.baux.size();
    o.pin_cons.assign(P, -1);
    for (int32_t n = 0; n < V; ++n)
        for (int32_t a = o.net_arc_ptr[n]; a < o.net_arc_ptr[n + 1]; ++a) o.pin_cons[o.arc_pin[a]] = net_step[n];

    // dependency counts and consumer lists (distinct producer per consumer)
    auto build_edges = [](int32_t T, const std::vector<std::vector<int32_t>>& prods, std::vector<int32_t>& indeg,
                          std::vector<int32_t>& out_ptr, std::vector<int32_t>& out) {
        indeg.assign(T, 0);
        out_ptr.assign(T + 1, 0);
        for (int32_t t = 0; t < T; ++t) {
            indeg[t] = (int32_t)prods[t].size();
            for (int32_t q : prods[t]) ++out_ptr[q + 1];
        }
        for (int32_t t = 0; t < T; ++t) out_ptr[t + 1] += out_ptr[t];
        out.assign(out_ptr[T], 0);
        std::vector<int32_t> fill(out_ptr.begin(), out_ptr.end() - 1);
        for (int32_t t = 0; t < T; ++t)
            for (int32_t q : prods[t]) out[fill[q]++] = t;
    };
    auto uniq = [](std::vector<int32_t>& v) {
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
        if (!v.empty() && v.front() < 0) v.erase(v.begin());
    };
    {
        std::vector<std::vector<int32_t>> prods(o.TF);
        for (int32_t t = 0; t < o.TF; ++t) {
            const int32_t n0 = o.ftask[4 * t], nn = o.ftask[4 * t + 1] > 0 ? o.ftask[4 * t + 1] : 1;
            for (int32_t a = o.net_arc_ptr[n0]; a < o.net_arc_ptr[n0 + nn]; ++a) prods[t].push_back(o.arc_prod[a]);
            uniq(prods[t]);
        }
        build_edges(o.TF, prods, o.f_indeg, o.f_out_ptr, o.f_out);
    }
    {
        std::vector<std::vector<int32_t>> prods(o.TB);
        for (int32_t t = 0; t < o.TB; ++t) {
            const int32_t kind = o.btask[4 * t + 1], p0 = o.btask[4 * t + 2], np = o.btask[4 * t + 3];
            if (kind == -2) {
                for (int32_t k = 0; k < np; ++k) prods[t].push_back(o.baux[t] + k);
            } else if (kind == -3) {
                prods[t].push_back(o.baux[t]);
            } else {  // packed nets or a partial chunk: the arc steps that feed its sinks
                for (int32_t p = p0; p < p0 + np; ++p) prods[t].push_back(o.pin_cons[p]);
            }
            uniq(prods[t]);
        }
        build_edges(o.TB, prods, o.b_indeg, o.b_out_ptr, o.b_out);
    }

    // Every task may only wait for tasks listed before it: the dataflow
    // kernels rely on this for progress.
    for (int32_t t = 0; t < o.TF; ++t)
        for (int32_t k = o.f_out_ptr[t]; k < o.f_out_ptr[t + 1]; ++k)
            if (o.f_out[k] <= t) return err = "internal: forward dependency order", STA_ERR_INVALID_ARG;
    for (int32_t t = 0; t < o.TB; ++t)
        for (int32_t k = o.b_out_ptr[t]; k < o.b_out_ptr[t + 1]; ++k)
            if (o.b_out[k] <= t) return err = "internal: backward dependency order", STA_ERR_INVALID_ARG;
    for (int32_t t = 0; t < o.TF; ++t) {
        const int32_t n0 = o.ftask[4 * t], nn = o.ftask[4 * t + 1] > 0 ? o.ftask[4 * t + 1] : 1;
        for (int32_t n = n0; n < n0 + nn; ++n)
            for (int32_t a = o.net_arc_ptr[n]; a < o.net_arc_ptr[n + 1]; ++a)
                if (o.arc_prod[a] >= t) return err = "internal: forward task order", STA_ERR_INVALID_ARG;
    }
    for (int32_t t = 0; t < o.TB; ++t) {
        const int32_t kind = o.btask[4 * t + 1], p0 = o.btask[4 * t + 2], np = o.btask[4 * t + 3];
        if (kind == -2) {
            if (o.baux[t] + np > t) return err = "internal: backward task order", STA_ERR_INVALID_ARG;
            continue;
        }
        if (kind == -3 && o.baux[t] >= t) return err = "internal: backward task order", STA_ERR_INVALID_ARG;
        for (int32_t p = p0; p < p0 + np; ++p)
            if (o.pin_cons[p] >= t) return err = "internal: backward task order", STA_ERR_INVALID_ARG;
    }
    return STA_OK;
}

StaStatus build_layout(const StaNetlistDesc& nl, const StaLibrary& lib, Layout& out, std::string& err) {
    StaStatus st = check_library(lib, err);
    if (st != STA_OK) return st;
    Roles r;
    st = check_netlist(nl, &lib, r, err);
    if (st != STA_OK) return st;
    std::vector<int32_t> dang = dangling_cells(nl, r);
    NetOrder no;
    st = make_order(nl, r, dang, no, err);
    if (st != STA_OK) return st;

    const int32_t P = nl.num_pins, Nreal = nl.num_nets, V = (int32_t)no.order.size();
    Layout& o = out;
    o.P = P;
    o.Nreal = Nreal;
    o.N = V;
    o.L = no.L;
    o.E = nl.num_end;
    o.T = lib.num_types;
    o.r_per_um = nl.r_per_um;
    o.c_per_um = nl.c_per_um;

    // ---- pins ----
    std::vector<int32_t> internal(P, -1);
    o.pin_orig.clear();
    o.pin_orig.reserve(P);
    o.net_ptr.assign(V + 1, 0);
    o.net_drv.assign(V, -1);
    o.net_orig.assign(V, -1);
    o.net_arc_ptr.assign(V + 1, 0);
    o.arc_pin.clear();
    std::vector<int32_t> net_cell(V, -1);
    for (int32_t i = 0; i < V; ++i) {
        const int32_t v = no.order[i];
        o.net_ptr[i] = (int32_t)o.pin_orig.size();
        if (v < Nreal) o.net_orig[i] = v;
        if (v < Nreal) {
            const int32_t b = nl.net_ptr[v], e = nl.net_ptr[v + 1];
            o.pin_orig.push_back(nl.net_pins[b]);
            std::vector<int32_t> s(nl.net_pins + b + 1, nl.net_pins + e);
            std::sort(s.begin(), s.end());
            o.pin_orig.insert(o.pin_orig.end(), s.begin(), s.end());
            net_cell[i] = r.out_cell[nl.net_pins[b]];
        } else {
            net_cell[i] = dang[v - Nreal];
            o.pin_orig.push_back(nl.cell_out_pin[net_cell[i]]);
        }
    }
    o.net_ptr[V] = (int32_t)o.pin_orig.size();
    o.Pnet = o.net_ptr[V];
    for (int32_t p = 0; p < P; ++p)
        if (r.sink_net[p] < 0 && r.drv_net[p] < 0 && r.out_cell[p] < 0) o.pin_orig.push_back(p);
    if ((int32_t)o.pin_orig.size() != P) return err = "internal: pin layout size mismatch", STA_ERR_INVALID_ARG;
    for (int32_t i = 0; i < P; ++i) internal[o.pin_orig[i]] = i;

    // ---- arcs ----
    for (int32_t i = 0; i < V; ++i) {
        o.net_arc_ptr[i] = (int32_t)o.arc_pin.size();
        const int32_t c = net_cell[i];
        if (c >= 0) {
            o.net_drv[i] = nl.cell_type[c];
            for (int32_t a = nl.cell_in_ptr[c]; a < nl.cell_in_ptr[c + 1]; ++a)
                o.arc_pin.push_back(internal[nl.cell_in_pins[a]]);
        }
    }
    o.net_arc_ptr[V] = (int32_t)o.arc_pin.size();
    o.A = o.net_arc_ptr[V];
    // pins the forward pass writes: every sink, and the driver of a cell-driven net
    o.pin_keep.assign(P, 1);
    for (int32_t i = 0; i < V; ++i) {
        if (o.net_drv[i] >= 0) o.pin_keep[o.net_ptr[i]] = 0;
        for (int32_t p = o.net_ptr[i] + 1; p < o.net_ptr[i + 1]; ++p) o.pin_keep[p] = 0;
    }
    o.pin_mask.assign(((size_t)P + 3) / 4 * 4, 0);
    for (int32_t a = 0; a < o.A; ++a) {
        const int32_t p = o.arc_pin[a];
        o.pin_mask[p] = (uint8_t)((o.pin_keep[p] ? 0 : 1) | 2);
    }

    o.pin_cap.resize(P);
    for (int32_t i = 0; i < P; ++i) o.pin_cap[i] = nl.pin_cap[o.pin_orig[i]];

    // ---- tasks per level ----
    o.lvl_wtask.assign(o.L + 1, 0);
    o.lvl_ctask.assign(o.L + 1, 0);
    o.wtask.clear();
    o.ctask.clear();
    int32_t i = 0;
    for (int32_t l = 0; l < o.L; ++l) {
        o.lvl_wtask[l] = (int32_t)(o.wtask.size() / 2);
        o.lvl_ctask[l] = (int32_t)o.ctask.size();
        while (i < V && no.level[no.order[i]] == l) {
            const int32_t size = o.net_ptr[i + 1] - o.net_ptr[i];
            if (size > kWarpPins) {
                o.ctask.push_back(i);
                ++i;
                continue;
            }
            // greedy pack of consecutive small nets of this level
            int32_t n0 = i, pins = 0, cnt = 0;
            while (i < V && no.level[no.order[i]] == l && cnt < kWarpNets) {
                const int32_t sz = o.net_ptr[i + 1] - o.net_ptr[i];
                if (sz > kWarpPins || pins + sz > kWarpPins) break;
                pins += sz;
                ++cnt;
                ++i;
            }
            o.wtask.push_back(n0);
            o.wtask.push_back(cnt);
        }
    }
    if (i != V) return err = "internal: task layout did not cover every net", STA_ERR_INVALID_ARG;
    o.lvl_wtask[o.L] = (int32_t)(o.wtask.size() / 2);
    o.lvl_ctask[o.L] = (int32_t)o.ctask.size();
    // RC chunks of the large nets (a net's partial loads are combined in chunk order)
    o.rc_chunk.clear();
    o.rc_net.clear();
    o.rc_slots = 0;
    for (int32_t n : o.ctask) {
        const int32_t p0 = o.net_ptr[n] + 1, p1 = o.net_ptr[n + 1];
        const int32_t nch = (p1 - p0 + kRcChunk - 1) / kRcChunk;
        for (int32_t k = 0; k < nch; ++k) {
            const int32_t a = p0 + k * kRcChunk;
            o.rc_chunk.insert(o.rc_chunk.end(), {n, a, std::min(kRcChunk, p1 - a), nch == 1 ? -1 : o.rc_slots + k});
            o.rc_net.insert(o.rc_net.end(), {o.rc_slots, nch});
        }
        if (nch > 1) o.rc_slots += nch;
    }

    // ---- dataflow task lists ----
    o.lvl_net.assign(o.L + 1, V);
    for (int32_t k = V - 1; k >= 0; --k) o.lvl_net[no.level[no.order[k]]] = k;
    for (int32_t l = o.L - 1; l >= 0; --l) o.lvl_net[l] = std::min(o.lvl_net[l], o.lvl_net[l + 1]);
    st = build_tasks(o, TaskShape{}, err);
    if (st != STA_OK) return st;

    // ---- constant per-pin state ----
    const float inf = std::numeric_limits<float>::infinity();
    o.at0.assign((size_t)P * 4, 0.f);
    o.slew0.assign((size_t)P * 4, 0.f);
    o.rat0.resize((size_t)P * 4);
    for (int32_t p = 0; p < P; ++p) {
        o.rat0[4 * p + 0] = o.rat0[4 * p + 1] = -inf;
        o.rat0[4 * p + 2] = o.rat0[4 * p + 3] = inf;
    }
    for (int32_t s = 0; s < nl.num_start; ++s) {
        const int32_t p = internal[nl.start_pins[s]];
        for (int q = 0; q < 4; ++q) {
            o.at0[4 * (size_t)p + q] = nl.start_at[4 * s + q];
            o.slew0[4 * (size_t)p + q] = nl.start_slew[4 * s + q];
        }
    }
    o.ep_pin.resize(o.E);
    o.ep_rat.resize((size_t)o.E * 4);
    o.ep_clk.clear();
    for (int32_t e = 0; nl.end_clock && e < o.E; ++e)
        if (nl.end_clock[e] >= 0) {
            o.ep_clk.assign(o.E, -1);
            break;
        }
    for (int32_t e = 0; e < o.E; ++e) {
        const int32_t p = internal[nl.end_pins[e]];
        o.ep_pin[e] = p;
        if (!o.ep_clk.empty() && nl.end_clock[e] >= 0) o.ep_clk[e] = internal[nl.end_clock[e]];
        for (int q = 0; q < 4; ++q) {
            o.ep_rat[4 * (size_t)e + q] = nl.end_rat[4 * e + q];
            o.rat0[4 * (size_t)p + q] = nl.end_rat[4 * e + q];
        }
    }

    // ---- library ----
    const int32_t T = lib.num_types;
    o.lib_idx.assign((size_t)T * kLibStride, 0.f);
    o.lib_inv.assign((size_t)T * kLibStride, 0.f);
    o.lib_unate.assign(T, 0);
    o.lib_tab.resize((size_t)T * STA_MAX_ARCS * 2 * kTabPerArcRf);
    o.lib_cell.resize((size_t)T * STA_MAX_ARCS * 2 * 36 * 8);
    o.lib_col.resize((size_t)T * STA_MAX_ARCS * 2 * 6 * STA_LUT * 4);
    for (int32_t t = 0; t < T; ++t) {
        for (int k = 0; k < STA_LUT; ++k) {
            o.lib_idx[t * kLibStride + k] = lib.slew_index[t * STA_LUT + k];
            o.lib_idx[t * kLibStride + 8 + k] = lib.load_index[t * STA_LUT + k];
        }
        for (int k = 0; k + 1 < STA_LUT; ++k) {
            o.lib_inv[t * kLibStride + k] =
                (float)(1.0 / ((double)lib.slew_index[t * STA_LUT + k + 1] - lib.slew_index[t * STA_LUT + k]));
            o.lib_inv[t * kLibStride + 8 + k] =
                (float)(1.0 / ((double)lib.load_index[t * STA_LUT + k + 1] - lib.load_index[t * STA_LUT + k]));
        }
        for (int a = 0; a < STA_MAX_ARCS; ++a) {
            if (lib.arc_unate[t * STA_MAX_ARCS + a] < 0) o.lib_unate[t] |= 1 << a;
            for (int rf = 0; rf < 2; ++rf) {
                const size_t src = (((size_t)t * STA_MAX_ARCS + a) * 2 + rf) * STA_LUT * STA_LUT;
                float* dst = &o.lib_tab[(((size_t)t * STA_MAX_ARCS + a) * 2 + rf) * kTabPerArcRf];
                std::memcpy(dst, lib.delay_tab + src, sizeof(float) * STA_LUT * STA_LUT);
                std::memcpy(dst + STA_LUT * STA_LUT, lib.slew_tab + src, sizeof(float) * STA_LUT * STA_LUT);
                float* cell = &o.lib_cell[(((size_t)t * STA_MAX_ARCS + a) * 2 + rf) * 36 * 8];
                for (int i = 0; i < 6; ++i)
                    for (int j = 0; j < 6; ++j) {
                        float* q = cell + (i * 6 + j) * 8;
                        const float* dt = lib.delay_tab + src;
                        const float* st = lib.slew_tab + src;
                        q[0] = dt[i * STA_LUT + j];
                        q[1] = dt[i * STA_LUT + j + 1];
                        q[2] = dt[(i + 1) * STA_LUT + j];
                        q[3] = dt[(i + 1) * STA_LUT + j + 1];
                        q[4] = st[i * STA_LUT + j];
                        q[5] = st[i * STA_LUT + j + 1];
                        q[6] = st[(i + 1) * STA_LUT + j];
                        q[7] = st[(i + 1) * STA_LUT + j + 1];
                    }
                float* col = &o.lib_col[(((size_t)t * STA_MAX_ARCS + a) * 2 + rf) * 6 * STA_LUT * 4];
                for (int j = 0; j < 6; ++j)
                    for (int i = 0; i < STA_LUT; ++i) {
                        float* q = col + (j * STA_LUT + i) * 4;
                        q[0] = lib.delay_tab[src + i * STA_LUT + j];
                        q[1] = lib.delay_tab[src + i * STA_LUT + j + 1];
                        q[2] = lib.slew_tab[src + i * STA_LUT + j];
                        q[3] = lib.slew_tab[src + i * STA_LUT + j + 1];
                    }
            }
        }
    }

    // ---- per-net driver-cell record (one 32-byte load instead of dependent ones) ----
    o.net_desc.assign((size_t)o.N * 8, 0);
    for (int32_t n = 0; n < o.N; ++n) {
        int32_t* q = &o.net_desc[(size_t)n * 8];
        const int32_t t = o.net_drv[n];
        const int32_t a0 = o.net_arc_ptr[n], na = t >= 0 ? o.net_arc_ptr[n + 1] - a0 : 0;
        int32_t bits = t >= 0 ? (o.lib_unate[t] & 15) << 4 : 0;
        for (int32_t k = 0; k < na; ++k) {
            q[4 + k] = o.arc_pin[a0 + k];
            bits |= (o.arc_prod[a0 + k] >= 0 ? 1 : 0) << k;  // input written during the sweep
        }
        q[0] = t;
        q[1] = a0;
        q[2] = na;
        q[3] = bits;
    }
    return STA_OK;
}

StaStatus build_layout_shared(const StaNetlistDesc& nl, const StaLibrary& lib, std::shared_ptr<const Layout>& out,
                              std::string& err) {
    auto lay = std::make_shared<Layout>();
    const StaStatus st = build_layout(nl, lib, *lay, err);
    if (st == STA_OK) out = std::move(lay);
    return st;
}

StaStatus build_union(const StaNetlistDesc* const* nls, int32_t count, UnionNetlist& u, std::string& err) {
    if (!nls || count < 1) {
        err = "sta_create_multi: count >= 1 netlists";
        return STA_ERR_INVALID_ARG;
    }
    // sizes first (the arrays are read up to net_ptr[N] and cell_in_ptr[C], as by sta_create)
    int64_t P = 0, N = 0, C = 0, NP = 0, CI = 0, S = 0, E = 0;
    bool clocked = false;
    for (int32_t k = 0; k < count; ++k) {
        const StaNetlistDesc* d = nls[k];
        if (!d || d->num_pins < 0 || d->num_nets < 0 || d->num_cells < 0 || d->num_start < 0 || d->num_end < 0 ||
            !d->net_ptr || !d->cell_in_ptr) {
            err = "sta_create_multi: netlist " + std::to_string(k) + ": null description, array or negative size";
            return STA_ERR_INVALID_ARG;
        }
        if (d->net_ptr[0] != 0 || d->net_ptr[d->num_nets] < 0 || d->cell_in_ptr[0] != 0 ||
            d->cell_in_ptr[d->num_cells] < 0) {
            err = "sta_create_multi: netlist " + std::to_string(k) + ": net_ptr / cell_in_ptr must start at 0";
            return STA_ERR_INVALID_ARG;
        }
        if (d->r_per_um != nls[0]->r_per_um || d->c_per_um != nls[0]->c_per_um) {
            err = "sta_create_multi: every netlist must have the same r_per_um and c_per_um";
            return STA_ERR_INVALID_ARG;
        }
        P += d->num_pins;
        N += d->num_nets;
        C += d->num_cells;
        NP += d->net_ptr[d->num_nets];
        CI += d->cell_in_ptr[d->num_cells];
        S += d->num_start;
        E += d->num_end;
        clocked = clocked || d->end_clock;
    }
    if (P >= (1ll << 31) - 1 || NP >= (1ll << 31) - 1 || CI >= (1ll << 31) - 1 || N >= (1ll << 31) - 1 ||
        E >= (1ll << 31) - 1) {
        err = "sta_create_multi: the union exceeds 2^31 pins, nets or endpoints";
        return STA_ERR_INVALID_ARG;
    }
    u = UnionNetlist();
    u.net_ptr.reserve(N + 1);
    u.net_ptr.push_back(0);
    u.net_pins.reserve(NP);
    u.cell_type.reserve(C);
    u.cell_in_ptr.reserve(C + 1);
    u.cell_in_ptr.push_back(0);
    u.cell_in_pins.reserve(CI);
    u.cell_out_pin.reserve(C);
    u.pin_cap.reserve(P);
    u.pin_off.assign(1, 0);
    u.end_off.assign(1, 0);
    auto missing = [&](int32_t k, const char* what) {
        err = "sta_create_multi: netlist " + std::to_string(k) + ": null " + what;
        return STA_ERR_INVALID_ARG;
    };
    for (int32_t k = 0; k < count; ++k) {
        const StaNetlistDesc& d = *nls[k];
        const int32_t po = u.pin_off.back();
        const int32_t np = d.net_ptr[d.num_nets], ci = d.cell_in_ptr[d.num_cells];
        if ((np > 0 && !d.net_pins) || (d.num_cells > 0 && (!d.cell_type || !d.cell_out_pin)) ||
            (ci > 0 && !d.cell_in_pins))
            return missing(k, "net_pins / cell array");
        if ((d.num_pins > 0 && !d.pin_cap) || (d.num_start > 0 && (!d.start_pins || !d.start_at || !d.start_slew)) ||
            (d.num_end > 0 && (!d.end_pins || !d.end_rat)))
            return missing(k, "pin_cap / startpoint / endpoint array");
        const int32_t nb = (int32_t)u.net_pins.size(), cb = (int32_t)u.cell_in_pins.size();
        for (int32_t i = 1; i <= d.num_nets; ++i) u.net_ptr.push_back(nb + d.net_ptr[i]);
        for (int32_t i = 0; i < np; ++i) u.net_pins.push_back(po + d.net_pins[i]);
        for (int32_t i = 0; i < d.num_cells; ++i) {
            u.cell_type.push_back(d.cell_type[i]);
            u.cell_in_ptr.push_back(cb + d.cell_in_ptr[i + 1]);
            u.cell_out_pin.push_back(po + d.cell_out_pin[i]);
        }
        for (int32_t i = 0; i < ci; ++i) u.cell_in_pins.push_back(po + d.cell_in_pins[i]);
        u.pin_cap.insert(u.pin_cap.end(), d.pin_cap, d.pin_cap + d.num_pins);
        for (int32_t i = 0; i < d.num_start; ++i) u.start_pins.push_back(po + d.start_pins[i]);
        u.start_at.insert(u.start_at.end(), d.start_at, d.start_at + 4 * (size_t)d.num_start);
        u.start_slew.insert(u.start_slew.end(), d.start_slew, d.start_slew + 4 * (size_t)d.num_start);
        for (int32_t i = 0; i < d.num_end; ++i) {
            u.end_pins.push_back(po + d.end_pins[i]);
            // a clock pin index moves with its netlist; -1 (none) stays
            if (clocked) u.end_clock.push_back(d.end_clock && d.end_clock[i] >= 0 ? po + d.end_clock[i] : -1);
        }
        u.end_rat.insert(u.end_rat.end(), d.end_rat, d.end_rat + 4 * (size_t)d.num_end);
        u.pin_off.push_back(po + d.num_pins);
        u.end_off.push_back(u.end_off.back() + d.num_end);
    }
    StaNetlistDesc& o = u.nl;
    o.num_pins = (int32_t)P;
    o.num_nets = (int32_t)N;
    o.num_cells = (int32_t)C;
    o.net_ptr = u.net_ptr.data();
    o.net_pins = u.net_pins.data();
    o.cell_type = u.cell_type.data();
    o.cell_in_ptr = u.cell_in_ptr.data();
    o.cell_in_pins = u.cell_in_pins.data();
    o.cell_out_pin = u.cell_out_pin.data();
    o.pin_cap = u.pin_cap.data();
    o.num_start = (int32_t)S;
    o.start_pins = u.start_pins.data();
    o.start_at = u.start_at.data();
    o.start_slew = u.start_slew.data();
    o.num_end = (int32_t)E;
    o.end_pins = u.end_pins.data();
    o.end_rat = u.end_rat.data();
    o.r_per_um = nls[0]->r_per_um;
    o.c_per_um = nls[0]->c_per_um;
    o.end_clock = clocked ? u.end_clock.data() : nullptr;
    return STA_OK;
}

}  // namespace sta

std::vector<std::pair<const void*, size_t>> layout_host_buffers(const sta::Layout& L) {
    std::vector<std::pair<const void*, size_t>> out;
    auto add = [&](const auto& v) {
        if (!v.empty()) out.emplace_back(static_cast<const void*>(v.data()), v.size() * sizeof(v[0]));
    };
    add(L.net_ptr), add(L.net_drv), add(L.net_arc_ptr), add(L.arc_pin), add(L.pin_orig), add(L.pin_cap);
    add(L.wtask), add(L.ctask), add(L.rc_chunk), add(L.rc_net), add(L.ftask), add(L.arc_prod), add(L.btask);
    add(L.baux), add(L.pin_cons), add(L.pin_keep), add(L.grp_ep), add(L.pin_grp), add(L.pin_mask), add(L.f_indeg);
    add(L.f_out_ptr), add(L.f_out), add(L.b_indeg), add(L.b_out_ptr), add(L.b_out), add(L.at0), add(L.slew0);
    add(L.rat0), add(L.ep_pin), add(L.ep_rat), add(L.ep_clk), add(L.lib_idx), add(L.lib_inv), add(L.lib_unate);
    add(L.lib_tab), add(L.net_desc), add(L.lib_cell), add(L.lib_col);
    return out;
}

namespace sta {

void set_groups(Layout& o, const UnionNetlist& u) {
    o.G = (int32_t)u.pin_off.size() - 1;
    o.grp_ep = u.end_off;  // endpoints keep the description's order
    o.pin_grp.resize(o.P);
    for (int32_t p = 0; p < o.P; ++p) {
        const int32_t orig = o.pin_orig[p];
        o.pin_grp[p] = (int32_t)(std::upper_bound(u.pin_off.begin(), u.pin_off.end(), orig) - u.pin_off.begin()) - 1;
    }
}

}  // namespace sta
