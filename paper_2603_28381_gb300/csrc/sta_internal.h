// sta_internal.h -- layout shared by the host builder and the device kernels.
//
// Device layout ("internal order"), built once per netlist by builder.cpp:
//   nets    sorted by (level, size class, original id); size class 0 = at most
//           kWarpPins pins (packed several to a warp), 1 = larger (one thread
//           block each).  Every cell output that drives no net gets an internal
//           net with no sinks, so that every cell is evaluated by exactly one net.
//   pins    net-contiguous: each net's driver then its sinks by ascending
//           original id; pins on no net (asserted clock pins) come last.
//   arcs    grouped by the net their cell drives, in the cell's input order.
// All per-pin state is structure-of-arrays in internal order; float4 holds the
// four timing conditions (cond = 2*el + rf), float2 the two late ones.
#pragma once

#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include "sta.h"

namespace sta {

constexpr int kWarpPins = 32;       // nets of <= 32 pins go to warp tasks
constexpr int kWarpNets = 8;        // at most 8 nets per warp task (4 lanes per net)
constexpr int kBlock = 256;         // threads per block in every task kernel
constexpr int kWarpsPerBlock = kBlock / 32;
constexpr int kLibStride = 16;      // floats per type in lib_idx / lib_inv
constexpr int kTabPerArcRf = 2 * STA_LUT * STA_LUT;  // delay table then slew table
constexpr int kRedBlocks = 152;     // endpoint reduction partials of the batched schedule (one per SM)
constexpr int kEpBlocks = 4 * 152;  // endpoint reduction partials of one placement
constexpr float kKrc = 1e-3f;       // Ohm * fF in ps
constexpr int kPartFloats = 12;     // floats per backward partial (large nets)
constexpr uint32_t kUnwritten = 0x7fbadbadu;  // a NaN: "not written yet in this sweep"
constexpr int kRcChunk = 1024;      // sinks per block of the large nets' RC prologue

// Granularity of the dataflow tasks: nets of at most `big` pins are packed
// (consecutive nets of a level while their pins fit in pack_pins, at most
// pack_nets of them; a net larger than pack_pins gets a task alone); larger nets
// are split into chunks of `chunk` sinks.  The default is the single-placement
// shape (lane per pin: 32 pins, 8 nets); the batched schedule (lane per
// placement) uses smaller tasks.
struct TaskShape {
    int32_t pack_pins = kWarpPins;
    int32_t pack_nets = kWarpNets;
    int32_t big = kWarpPins;
    int32_t chunk = kWarpPins;
};

struct Layout {
    int32_t P = 0;       // pins
    int32_t Pnet = 0;    // pins on nets (prefix of the internal order)
    int32_t N = 0;       // internal nets (real + one per dangling cell output)
    int32_t Nreal = 0;   // nets of the description
    int32_t L = 0;       // levels
    int32_t A = 0;       // arcs
    int32_t E = 0;       // endpoints
    int32_t T = 0;       // library types

    std::vector<int32_t> net_ptr;      // [N+1] internal pin range
    std::vector<int32_t> net_drv;      // [N] cell type if cell-driven, -1 if asserted
    std::vector<int32_t> net_orig;     // [N] description net id, -1 for a dangling cell output
    std::vector<int32_t> net_arc_ptr;  // [N+1]
    std::vector<int32_t> arc_pin;      // [A] internal input pin of each arc
    std::vector<int32_t> pin_orig;     // [P] original id of each internal pin
    std::vector<float> pin_cap;        // [P]
    std::vector<int32_t> lvl_wtask;    // [L+1] warp-task ranges per level
    std::vector<int32_t> lvl_ctask;    // [L+1] block-task ranges per level
    std::vector<int32_t> wtask;        // [2*W] (first net, number of nets)
    std::vector<int32_t> ctask;        // [Cb] net of each block task
    // RC of the nets of more than 32 pins in chunks of kRcChunk sinks, one block
    // each: {net, first sink, sinks, partial slot (-1: the net's only chunk)} and
    // {first slot of the net, chunks of the net}
    std::vector<int32_t> rc_chunk;     // [4*K]
    std::vector<int32_t> rc_net;       // [2*K]
    int32_t rc_slots = 0;

    std::vector<int32_t> lvl_net;      // [L+1] first internal net of each level

    // dataflow schedule (one persistent kernel per sweep, tasks in topological order)
    TaskShape shape;
    std::vector<int32_t> big_nets;   // nets split into chunks (their load comes from a prologue)
    std::vector<int32_t> lvl_ftask;  // [L+1] forward tasks of each level
    std::vector<int32_t> lvl_bsec;   // [L][5] backward tasks of level l: partial chunks from [0],
                                     // driver steps from [1], packed nets from [2], gradient chunks
                                     // from [3], end [4]
    //   forward task  {first net, nets (> 0) | -1 for a 32-sink chunk of a large net, first pin, pins}
    //   backward task {net(s), kind, first pin, pins}: kind > 0 packed nets (= count), -1 partial
    //   chunk of a large net, -2 its driver step (first pin = first partial slot, pins = chunks),
    //   -3 gradient chunk; aux = partial slot (-1), first partial task (-2), driver task (-3)
    std::vector<int32_t> ftask;      // [4*TF]
    std::vector<int32_t> arc_prod;   // [A] forward task that writes the arc's input pin, -1 if asserted
    std::vector<int32_t> btask;      // [4*TB]
    std::vector<int32_t> baux;       // [TB]
    std::vector<int32_t> pin_cons;   // [P] backward task whose arc step writes the pin's RAT / adjoint
    std::vector<uint8_t> pin_keep;   // [P] 1 if no forward task writes the pin (asserted drivers, clock pins)
    // several netlists in one layout (sta_create_multi): G netlists, the
    // endpoint range of each (grp_ep [G+1], description order = layout order)
    // and the netlist of each device pin (pin_grp [P]); G = 1 and both empty
    // for one netlist
    int32_t G = 1;
    std::vector<int32_t> grp_ep, pin_grp;
    std::vector<uint8_t> pin_mask;   // [P rounded up to 4] bit 0: words of the pin the forward sweep polls
                                     // (a cell input it writes), bit 1: the backward's (a cell input)
    // dependency counts and consumer lists: a task may start once `indeg` of its
    // producers have published; a producer signals every task of its out list
    std::vector<int32_t> f_indeg, f_out_ptr, f_out;  // forward: [TF], [TF+1], [..]
    std::vector<int32_t> b_indeg, b_out_ptr, b_out;  // backward: [TB], [TB+1], [..]
    int32_t TF = 0, TB = 0, npart = 0;

    // constant per-pin state written once at creation
    std::vector<float> at0, slew0;     // [P*4] asserted values (0 elsewhere)
    std::vector<float> rat0;           // [P*4] endpoint constraint, else -inf/+inf
    std::vector<int32_t> ep_pin;       // [E] internal pin of each endpoint
    std::vector<float> ep_rat;         // [E*4]
    std::vector<int32_t> ep_clk;       // [E] internal capturing clock pin, -1 none; empty: ideal clock

    // library, device form
    std::vector<float> lib_idx;        // [T*16] slew index (0..6), load index (8..14)
    std::vector<float> lib_inv;        // [T*16] 1/(idx[k+1]-idx[k]) for k = 0..5 (slew), 8..13 (load)
    std::vector<int32_t> lib_unate;    // [T] bit a set = arc a negative unate
    std::vector<float> lib_tab;        // [T*4*2*98] per (type, arc, rf_out): delay 7x7, slew 7x7
    std::vector<int32_t> net_desc;     // [N*8] driver type (-1: asserted), first arc, arcs, bits 0-3 input
                                       // written during the sweep and 4-7 negative unate, input pins 0-3
    std::vector<float> lib_cell;       // [T*4*2*36*8] per (type, arc, rf_out, slew seg, load seg): the
                                       // four delay corners then the four slew corners (one 32-byte sector)
    std::vector<float> lib_col;        // [T*4*2*6*7*4] per (type, arc, rf_out, load seg j, slew row i):
                                       // delay at (i, j), (i, j+1), slew at (i, j), (i, j+1)

    float r_per_um = 0.f, c_per_um = 0.f;
};

// Validate and levelize (Kahn sweep over nets).  net_level receives the level
// of every description net and, if dangling != nullptr, of every dangling cell
// (cells whose output drives no net) in cell order.  Returns the level count
// through num_levels.
StaStatus levelize(const StaNetlistDesc& nl, const StaLibrary* lib, std::vector<int32_t>& net_level,
                   std::vector<int32_t>* dangling_cells, std::vector<int32_t>* dangling_level,
                   int32_t& num_levels, std::string& err);

// Full host-side layout for the device.
StaStatus build_layout(const StaNetlistDesc& nl, const StaLibrary& lib, Layout& out, std::string& err);

// (Re)build the dataflow task lists and dependency lists of a layout for a
// task shape.  Checks that every task only depends on tasks listed before it.
StaStatus build_tasks(Layout& o, const TaskShape& sh, std::string& err);

// Processing order of description nets and device pin order (sta_levelize).
StaStatus ordering(const StaNetlistDesc& nl, std::vector<int32_t>& net_level, int32_t& num_levels,
                   std::vector<int32_t>& net_order, std::vector<int32_t>& pin_order, std::string& err);

// The disjoint union of `count` netlists over one library (sta_create_multi):
// netlist k's pins, nets, cells, startpoints and endpoints follow those of
// netlists 0..k-1, its pin indices shifted by the pins before it.  The wire
// parameters must agree (INVALID_ARG otherwise); build_layout validates the rest.
struct UnionNetlist {
    std::vector<int32_t> net_ptr, net_pins, cell_type, cell_in_ptr, cell_in_pins, cell_out_pin, start_pins, end_pins,
        end_clock;
    std::vector<float> pin_cap, start_at, start_slew, end_rat;
    std::vector<int32_t> pin_off, end_off;  // [count + 1] first pin / endpoint of each netlist
    StaNetlistDesc nl{};
};
StaStatus build_union(const StaNetlistDesc* const* nls, int32_t count, UnionNetlist& u, std::string& err);

// The netlist groups of a union's layout: endpoint ranges and each device pin's netlist.
void set_groups(Layout& o, const UnionNetlist& u);

// A netlist's host layout built once and shared by the handles created from
// it with sta_create_from_layout: the serving layer keeps one per registered
// netlist, so that re-admitting an evicted netlist allocates and uploads
// without rebuilding the layout on the host.
StaStatus build_layout_shared(const StaNetlistDesc& nl, const StaLibrary& lib, std::shared_ptr<const Layout>& out,
                              std::string& err);

}  // namespace sta

// The host arrays of a layout that sta_create uploads, as (address, bytes):
// a caller that keeps a layout for many handles may page-lock them once, so
// that the uploads of each new handle run as asynchronous DMA.
std::vector<std::pair<const void*, size_t>> layout_host_buffers(const sta::Layout& L);

// sta_create on a layout from build_layout_shared (same options and errors).
// The handle shares the layout, which stays unmodified; a BATCH handle with
// its own task lists (batch_sweep LEVELS or DATAFLOW) works on a copy.  With
// pool (a cudaMemPool_t) its device memory comes from that stream-ordered pool
// and neither its creation nor sta_destroy synchronizes the whole device: the
// caller destroys it only once none of its work is in flight.
StaStatus sta_create_from_layout(std::shared_ptr<const sta::Layout> lay, const StaOptions* opts, void* pool,
                                 StaHandle** out);
