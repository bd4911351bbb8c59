/*
 * sta.h -- C ABI of libsta: levelized, differentiable static timing analysis
 * on one GB300 GPU (sm_103a).
 *
 * The method is Warp-STAR (arXiv 2603.28381): per-net Elmore RC (Eqs. 1-3,
 * Section 3.1.1), NLDM cell-arc table lookup and level-by-level arrival-time
 * propagation (Section 3.1.2), backward required-time propagation and slack
 * (Section 2.1, 3.1.2), and the LogSumExp-smoothed arrival time (Eq. 4,
 * Section 3.2) whose smoothed TNS/WNS is differentiated with respect to pin
 * positions (Section 3.2).
 *
 * Problem statement (Section 2.1): a netlist of pins, cells and nets forms a
 * DAG; a net has one driver pin (its first pin, Algorithm 1's netRoot) and any
 * number of sink pins; a cell has input pins and one output pin and one timing
 * arc from each input to the output.
 *
 * Conventions
 *   units       ps, fF, Ohm, um; Ohm * fF = 1e-3 ps.
 *   conditions  4 per pin, index cond = 2*el + rf, el 0 early / 1 late,
 *               rf 0 rise / 1 fall (Section 3.1.1).
 *   wires       every net is a star: one wire of Manhattan length d from the
 *               driver to each sink, resistance r*d, capacitance c*d split half
 *               at each end.
 *   pins        every pin has exactly one source of arrival time: it is a
 *               startpoint (asserted AT/slew), a net sink, or a cell output.
 *               Endpoints must be net sinks that are not cell inputs.
 *   ownership   all input arrays are caller-owned host memory and are copied by
 *               sta_create; the handle owns every device allocation it makes.
 *   streams     calls taking `stream` (a cudaStream_t, NULL = legacy default)
 *               are asynchronous on it unless stated otherwise.  A handle is
 *               not thread-safe; use one handle per host thread.
 *   errors      every call returns a StaStatus; sta_last_error() gives a
 *               human-readable message for the calling thread's last failure.
 *               No call aborts the process.
 */
#ifndef STA_H_
#define STA_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define STA_ABI_VERSION 5
#define STA_LUT 7       /* table points per axis */
#define STA_MAX_ARCS 4  /* arcs (input pins) per cell type */

typedef enum {
    STA_OK = 0,
    STA_ERR_INVALID_ARG = 1, /* malformed netlist / library / argument */
    STA_ERR_NOT_DAG = 2,     /* the timing graph has a cycle */
    STA_ERR_OOM = 3,         /* device or host allocation failed */
    STA_ERR_CUDA = 4,        /* a CUDA runtime call failed */
    STA_ERR_TIMEOUT = 5,     /* a bounded device-side wait expired; reported once, by the
                                next synchronizing call (sta_synchronize or a call with
                                host output); results since the previous report are invalid */
    STA_ERR_STATE = 6        /* call out of order (e.g. gradient before forward) */
} StaStatus;

/* Netlist in CSR form (Algorithm 1 inputs netlist / netlist_ind).  Host arrays,
 * read during sta_create / sta_levelize only. */
typedef struct {
    int32_t num_pins, num_nets, num_cells;
    const int32_t *net_ptr;      /* [num_nets+1] pin range of each net in net_pins */
    const int32_t *net_pins;     /* [net_ptr[num_nets]] first pin of a net = its driver */
    const int32_t *cell_type;    /* [num_cells] index into the library */
    const int32_t *cell_in_ptr;  /* [num_cells+1] input-pin range of each cell */
    const int32_t *cell_in_pins; /* [cell_in_ptr[num_cells]] input k uses arc k of the type */
    const int32_t *cell_out_pin; /* [num_cells] */
    const float *pin_cap;        /* [num_pins] pin capacitance, fF */
    int32_t num_start;
    const int32_t *start_pins;   /* [num_start] startpoints (primary inputs, clock pins) */
    const float *start_at;       /* [num_start][4] asserted arrival time, ps */
    const float *start_slew;     /* [num_start][4] asserted slew, ps */
    int32_t num_end;
    const int32_t *end_pins;     /* [num_end] endpoints (primary outputs, flop D pins) */
    const float *end_rat;        /* [num_end][4] required time: early = hold bound,
                                    late = setup bound, ps */
    float r_per_um, c_per_um;    /* wire resistance (Ohm/um) and capacitance (fF/um) */
    const int32_t *end_clock;    /* [num_end] or NULL (ideal clock).  Propagated clock: the
                                    clock pin of the flop that captures the endpoint, -1 for
                                    none.  The endpoint's early bound then adds that pin's
                                    late rising arrival (hold: latest capture edge) and its
                                    late bound the early rising arrival (setup: earliest
                                    edge); the adjoint of the smoothed loss follows the
                                    setup term into the clock wire.  A clock pin must be the
                                    input of a one-input cell (a flop's clock->Q arc) on a net
                                    driven by a startpoint (an unbuffered clock net) and
                                    capture at most one endpoint (STA_ERR_INVALID_ARG
                                    otherwise). */
} StaNetlistDesc;

/* Liberty-like library (Section 3.1.2): per type and arc, per output
 * transition, a 7x7 delay and output-slew table indexed [slew][load]. */
typedef struct {
    int32_t num_types;
    const int32_t *type_num_arcs; /* [num_types] number of input pins, 1..4 */
    const int8_t *arc_unate;      /* [num_types][4] +1 positive unate (out rise <- in rise),
                                     -1 negative unate (out rise <- in fall) */
    const float *slew_index;      /* [num_types][7] strictly increasing, ps */
    const float *load_index;      /* [num_types][7] strictly increasing, fF */
    const float *delay_tab;       /* [num_types][4][2][7][7] ps, [type][arc][rf_out][slew][load] */
    const float *slew_tab;        /* [num_types][4][2][7][7] ps */
} StaLibrary;

typedef struct {
    int32_t use_graphs;  /* 1 (default): replay each sweep as a CUDA graph */
    int32_t profile;     /* 1: bracket every launch with CUDA events (see sta_query_profile) */
    int32_t schedule;    /* STA_SCHED_DATAFLOW (default), STA_SCHED_LEVELS or STA_SCHED_BATCH */
    int32_t num_placements; /* STA_SCHED_BATCH: placements B analysed together (>= 1; 0 = 1) */
    int32_t tile_pins;   /* STA_SCHED_BATCH task shape: nets are packed into one task while
                            their pins total at most tile_pins (0 = default 4) */
    int32_t chunk;       /* STA_SCHED_BATCH task shape: nets of more than `chunk` sinks are
                            split into tasks of `chunk` sinks (0 = default 16) */
    int32_t batch_sweep; /* STA_SCHED_BATCH: STA_BATCH_LEVELS (default), STA_BATCH_DATAFLOW or
                            STA_BATCH_LANES */
    int32_t grid_blocks; /* dataflow sweeps: blocks of the persistent kernels (0 = every block
                            that fits on the device; fewer leave room for other work) */
} StaOptions;

/* StaOptions.schedule.  Both compute the same quantities: arrival, slew,
 * LSE and required times are bit-identical; gradient sums over the sinks of
 * nets of more than 32 pins are reassociated (32-sink partials here, a
 * 256-thread block reduction there), so gradients agree to rounding.
 *   DATAFLOW  one persistent kernel per sweep; warp-sized tasks taken from a
 *             queue in topological order, each waiting (bounded in time) only
 *             for the tasks that produce its inputs.
 *   LEVELS    one kernel launch per level per sweep (Section 3.1.2). */
#define STA_SCHED_DATAFLOW 0
#define STA_SCHED_LEVELS 1
/*   BATCH     B placements (position sets) of one netlist in every call: the
 *             dataflow sweeps with lanes mapped to placements (32 placements
 *             per warp task).  Every per-pin input and output gains a leading
 *             placement dimension: positions and gradients [B][num_pins][2],
 *             summaries [B][STA_SUM_COUNT], pin results [B][num_pins][k],
 *             endpoint slacks [B][num_end][2], loss weights w [B][2].
 *             A placement's results do not depend on B or on the other
 *             placements (bit-identical to the same placement alone). */
#define STA_SCHED_BATCH 2
/* StaOptions.batch_sweep: how the batched schedule orders its tasks.
 *   LEVELS    one launch per level (two per level in the backward where a level
 *             has nets split into chunks), replayed as a CUDA graph; the tasks
 *             of a level run without any waiting.
 *   DATAFLOW  one persistent launch per sweep whose tasks wait on the data
 *             words they read, as in STA_SCHED_DATAFLOW; a warp takes a task
 *             for 8 placements x 4 timing conditions.
 *   WIDE      as DATAFLOW, but every sweep takes a task for 32 placements
 *             per warp, each lane running the four timing conditions of its
 *             placement (more independent memory round trips per warp, the
 *             task's topology read once for 32 placements).
 * LEVELS, DATAFLOW and WIDE give bit-identical results.
 *   LANES     the placements as independent lanes of the single-placement
 *             dataflow sweeps (STA_SCHED_DATAFLOW): each placement has its own
 *             state, laid out as for one placement, and one persistent launch
 *             per sweep takes task t of every placement in turn.  A placement's
 *             results are bit-identical to the same placement in a
 *             single-placement handle.  tile_pins and chunk do not apply;
 *             sta_autotune is not available (STA_ERR_STATE). */
#define STA_BATCH_LEVELS 0
#define STA_BATCH_DATAFLOW 1
#define STA_BATCH_LANES 2
#define STA_BATCH_WIDE 3

typedef struct StaHandle StaHandle;

/* sta_forward flags */
#define STA_FWD_LSE 1u  /* also propagate LSE arrival times (needed before sta_backward_grad) */
#define STA_FWD_RAT 2u  /* also propagate required times and per-pin slack */
#define STA_FWD_RAT_EAGER 4u /* with STA_FWD_RAT: run the required-time sweep in this call, on
                                `stream`, instead of deferring it to the next gradient sweep or query */

/* summary slots written by sta_forward and read by sta_query_summary */
enum {
    STA_SUM_WNS_EARLY = 0, STA_SUM_TNS_EARLY = 1, /* hold: slack = AT - RAT_c */
    STA_SUM_WNS_LATE = 2, STA_SUM_TNS_LATE = 3,   /* setup: slack = RAT_c - AT */
    STA_SUM_TNS_GAMMA = 4, STA_SUM_WNS_GAMMA = 5, /* smoothed, from LSE arrival times */
    STA_SUM_LATE_VIOLATIONS = 6, STA_SUM_NUM_ENDPOINTS = 7,
    STA_SUM_COUNT = 8
};

/* Validate, levelize and lay out a netlist and library, copy them to the
 * current CUDA device and allocate every device buffer the analysis needs.
 * opts may be NULL.  On success *out owns the device memory (free with
 * sta_destroy).  Errors: INVALID_ARG (malformed input), NOT_DAG, OOM, CUDA. */
StaStatus sta_create(const StaNetlistDesc *nl, const StaLibrary *lib, const StaOptions *opts,
                     StaHandle **out);

/* Many netlists in one handle: the disjoint union of nls[0..count-1] (one
 * library, the same r_per_um and c_per_um), swept together, one launch per
 * sweep and one endpoint launch for all of them.  Netlist k's pins, nets,
 * cells, startpoints and endpoints follow those of netlists 0..k-1: positions
 * (sta_set_positions), pin queries, endpoint slacks and gradients are over the
 * union in that order, netlist k's pin i at the number of pins before it plus
 * i.  The endpoint reduction, the smoothed loss and its adjoint seeds are per
 * netlist: sta_query_summary writes [count][STA_SUM_COUNT], and
 * sta_backward_grad takes w [count][2] (the loss of netlist k weighted by
 * w[k]; the gradient of each netlist's pins is that of its own loss).  Every
 * result of netlist k equals that of the same netlist in its own handle.
 * opts may be NULL; only the DATAFLOW schedule (INVALID_ARG otherwise);
 * sta_query_slack is not available (STATE).  Errors as sta_create, and
 * INVALID_ARG for count < 1 or a null description. */
StaStatus sta_create_multi(const StaNetlistDesc *const *nls, int32_t count, const StaLibrary *lib,
                           const StaOptions *opts, StaHandle **out);

/* Set pin positions xy [num_pins][2] (um, the netlist's pin order).  xy is a
 * device pointer if on_device != 0 (8-byte aligned: it is read as float2;
 * INVALID_ARG otherwise, before any device work), else host memory (copied
 * through pinned staging inside this call).  The positions are copied; the
 * caller may reuse xy when the call's work on `stream` completes. */
StaStatus sta_set_positions(StaHandle *h, const float *xy, int on_device, void *stream);

/* One forward pass: net RC for every net (Eqs. 1-3), then, level by level,
 * cell-arc NLDM delays and slews, late max / early min arrival times and wire
 * propagation to sinks (Section 3.1.2); with STA_FWD_LSE also the LSE arrival
 * time of Eq. 4 with smoothing gamma (ps, > 0); then endpoint slacks, WNS, TNS
 * and their smoothed forms; with STA_FWD_RAT required times propagated back
 * level by level and per-pin slack.  Needs sta_set_positions first (STATE).
 * The required-time sweep runs on a stream owned by the handle, ordered after
 * this call's arrival-time pass; `stream` is free for further work (such as
 * sta_backward_grad) as soon as arrival times exist, and every later call on
 * the handle waits for the sweep where it needs to. */
StaStatus sta_forward(StaHandle *h, uint32_t flags, float gamma, void *stream);

/* Gradient of loss = w[0] * TNS_gamma + w[1] * WNS_gamma with respect to the
 * pin positions, by a hand-written adjoint swept over the levels in reverse
 * (Section 3.2).  w is a device pointer if w_on_device != 0, else host.  The
 * result goes to grad_xy [num_pins][2] in the netlist's pin order, a device
 * pointer if on_device != 0 (8-byte aligned; a device w 4-byte aligned; else
 * INVALID_ARG before any device work), else host memory (this call then
 * synchronizes `stream`).  Requires a preceding sta_forward with STA_FWD_LSE (STATE).
 * The sweep waits for the forward's arrival-time pass only, so it overlaps the
 * forward's required-time sweep on the GPU (operation fusion, Section 3.2).
 * Positions, forward state and the gradient buffer are shared by every call on
 * the handle: a later sta_set_positions / sta_forward waits for this sweep. */
StaStatus sta_backward_grad(StaHandle *h, const float *w, int w_on_device, float *grad_xy,
                            int on_device, void *stream);

/* Make `stream` wait (on the GPU, without blocking the host) for all work the
 * handle has queued so far, including the required-time sweep that runs on
 * the handle's own stream. */
StaStatus sta_stream_wait(StaHandle *h, void *stream);

/* Block until every sweep of the handle has finished.  Returns STA_ERR_TIMEOUT
 * if a bounded wait of the dataflow schedule expired since the last report
 * (each dependency wait gives up after 1 s; the sweep then ends with invalid
 * results instead of hanging), else STA_OK.  The handle stays usable. */
StaStatus sta_synchronize(StaHandle *h);

/* Test hook for the bounded waits (dataflow sweeps only: STA_SCHED_DATAFLOW, or
 * STA_SCHED_BATCH with STA_BATCH_DATAFLOW; else STA_ERR_STATE):
 * in the next sta_forward the wait of the sweep's last task for its input
 * words never succeeds, so it expires after its 1 s budget (the sweep ends with
 * invalid results) and the next synchronizing call returns STA_ERR_TIMEOUT.
 * No fault is involved; later calls are unaffected. */
StaStatus sta_debug_expire_wait(StaHandle *h);

/* Autotuner of the batched schedule (STA_SCHED_BATCH only, else STATE): for
 * every candidate (tile_pins[i], chunks[j], sweeps[k]) it rebuilds the task
 * lists, replays one step (forward with LSE and required times, then the
 * gradient sweep; smoothing gamma) as a CUDA graph reps times on the handle's
 * current positions (sta_set_positions first, else STATE) and times it with
 * CUDA events; then it keeps the fastest.  ms [n_tile][n_chunk][n_sweep]
 * receives the mean step times in ms (may be NULL); best[3] = the chosen
 * (tile_pins, chunk, batch_sweep).  Synchronizes the device; the analysis
 * state is reset (call sta_forward again).  Results do not depend on the shape
 * beyond rounding of sums over large nets. */
StaStatus sta_autotune(StaHandle *h, const int32_t *tile_pins, int32_t n_tile, const int32_t *chunks,
                       int32_t n_chunk, const int32_t *sweeps, int32_t n_sweep, int32_t reps, float gamma,
                       float *ms, int32_t *best);

/* Net RC results (Eqs. 1-3) of the latest forward pass or RC ablation run, in
 * the description's order: load [num_nets] (fF), wdelay and impulse
 * [num_pins] (ps; 0 at pins that are not sinks).  Any output may be NULL.
 * Host outputs; synchronizes the device.  Single-placement schedules only. */
StaStatus sta_query_net_rc(StaHandle *h, float *load, float *wdelay, float *impulse);

/* Ablation of the net-RC work decomposition (single-placement schedules, after
 * sta_set_positions): runs the RC of every net `reps` times with one scheme and
 * returns the mean time per run in *ms (may be NULL); the results are left for
 * sta_query_net_rc.  STA_RC_PIN: the pin-based warp tasks of the other kernels
 * (nets of <= 32 pins packed into warps, larger nets one block each, fixed-order
 * sums).  STA_RC_CTE: the collaborative task engagement of Algorithm 2 (a
 * block-wide task pool built by a Blelloch scan, a binary search per task,
 * shared-memory atomics for the loads).  The analysis state is reset (call
 * sta_forward again).  Synchronizes the device. */
#define STA_RC_PIN 0
#define STA_RC_CTE 1
StaStatus sta_ablation_net_rc(StaHandle *h, int32_t scheme, int32_t reps, float *ms);

/* Copy the STA_SUM_COUNT summary values (double) to out, a device pointer if
 * on_device != 0 (asynchronous), else host (synchronizes `stream`). */
StaStatus sta_query_summary(StaHandle *h, double *out, int on_device, void *stream);

/* Per-pin results in the netlist's pin order (any output may be NULL):
 * at, slew, rat [num_pins][4]; ats [num_pins][2] (late rise/fall LSE arrival);
 * slack [num_pins][2] (early, late; minimum over rise/fall).  Device pointers if
 * on_device != 0 (asynchronous; 4-byte aligned, slack 8-byte aligned, else
 * INVALID_ARG before any device work), else host (synchronizes `stream`). */
StaStatus sta_query_pins(StaHandle *h, float *at, float *slew, float *rat, float *ats,
                         float *slack, int on_device, void *stream);

/* Slack in one call (single-placement, single-netlist handles; host outputs, synchronizes
 * the legacy default stream after the handle's work): wns_tns [2][2] =
 * {early WNS, early TNS, late WNS, late TNS} (ps; TNS sums negative endpoint
 * slacks, WNS is the unclamped minimum); pin_slack [num_pins][2] and
 * endpoint_slack [num_end][2] (early, late), each may be NULL.  The per-pin
 * slacks need a forward pass with STA_FWD_RAT (STATE otherwise). */
StaStatus sta_query_slack(StaHandle *h, float *wns_tns, float *pin_slack, float *endpoint_slack);

/* Endpoint slacks [num_end][2] (early, late), in the order of end_pins. */
StaStatus sta_query_endpoints(StaHandle *h, float *slack, int on_device, void *stream);

/* Host-only levelization (no device use): the level of every net, computed by
 * a breadth-first (Kahn) sweep over nets: level 0 if the driver is not a cell
 * output, else 1 + the largest level among the nets feeding the driver cell's
 * inputs (Section 2.1 stage 2).  net_level [num_nets]; *num_levels = max + 1.
 * If net_order != NULL it receives the original net ids in processing order
 * (level; within a level nets of <= 32 pins before larger ones, then by the
 * largest position in this order of a net feeding the driver cell, -1 if none,
 * then original id), and
 * if pin_order != NULL [net_ptr[num_nets]] the original pin ids in device
 * layout order (each net's driver, then its sinks by ascending id). */
StaStatus sta_levelize(const StaNetlistDesc *nl, int32_t *net_level, int32_t *num_levels,
                       int32_t *net_order, int32_t *pin_order);

/* Host-only planning of the dataflow task lists for a task shape (no device
 * use): packed tasks of nets of at most chunk + 1 pins (while their pins fit in
 * tile_pins, at most tile_nets nets; a larger net alone), larger nets split into
 * chunks of `chunk` sinks.  The builder checks that every task depends only on
 * tasks listed before it and that every written pin has exactly one forward
 * task (INVALID_ARG "internal: ..." otherwise).  out8: forward tasks, backward
 * tasks, partial records, forward chunk tasks, most pins in a packed task, most
 * nets in a packed task, forward dependency edges, nets split into chunks. */
StaStatus sta_plan_tasks(const StaNetlistDesc *nl, const StaLibrary *lib, int32_t tile_pins,
                         int32_t tile_nets, int32_t chunk, int64_t *out8);

/* Sizes of a created handle: [0] pins, [1] nets (including one internal
 * net per cell output that drives no net), [2] levels, [3] arcs, [4] endpoints,
 * [5] warp tasks, [6] block tasks, [7] device bytes held. */
StaStatus sta_query_sizes(const StaHandle *h, int64_t *out8);

/* Kernel kinds reported by sta_query_profile. */
enum {
    STA_PROF_POSITIONS = 0,  /* gather of positions into device order */
    STA_PROF_NET_RC = 1,     /* Eqs. 1-3: every net (LEVELS), nets > 32 pins (DATAFLOW) */
    STA_PROF_FORWARD = 2,    /* forward propagation: one launch per level, or one persistent launch */
    STA_PROF_ENDPOINTS = 3,  /* endpoint slack / WNS / TNS reduction (two launches) */
    STA_PROF_REQUIRED = 4,   /* required-time sweep */
    STA_PROF_SEED = 5,       /* loss weights (and, LEVELS only, endpoint seeds) */
    STA_PROF_ADJOINT = 6,    /* adjoint sweep */
    STA_PROF_OUTPUT = 7,     /* BATCH: gradient from device layout to [B][num_pins][2] */
    STA_PROF_RESET = 8,      /* dataflow sweeps: marking the words their tasks poll as unwritten */
    STA_PROF_KINDS = 9
};

/* Per-kind launch counts of one set_positions + forward(LSE|RAT) +
 * backward_grad step (always), and, for a handle created with
 * StaOptions.profile = 1, the summed CUDA-event durations (ms) of the most
 * recent execution of each kind's launches, measured on the stream each kernel
 * ran on.  Synchronizes the device.  ms and launches have STA_PROF_KINDS
 * entries; ms may be NULL. */
StaStatus sta_query_profile(StaHandle *h, double *ms, int32_t *launches);

/* ---- Allocation-free endpoint summary.  The paper has no counterpart. ----
 *
 * For callers that cannot call cudaMalloc: code running while a stream is
 * being captured into a CUDA graph (allocation cannot be captured), and
 * processes whose device memory is fully reserved by another framework's pool
 * allocator.  Computes, from per-pin arrays the caller holds, the same
 * endpoint slacks, WNS, TNS and smoothed TNS/WNS that sta_forward reduces, and
 * allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 *
 * at       [num_pins][4] device, arrival times (cond = 2*el + rf); 16-byte aligned
 * ats      [num_pins][2] device, late rise/fall LSE arrival times, or NULL
 *          (then the smoothed slots of the summary are 0 / +inf); 8-byte aligned
 * end_pins [num_end] device, pin index of each endpoint; an index outside
 *          [0, num_pins) gives that endpoint NaN slacks and leaves it out of the
 *          summary (STA_SUM_NUM_ENDPOINTS counts the endpoints used)
 * end_rat  [num_end][4] device, endpoint constraints as in StaNetlistDesc;
 *          16-byte aligned
 * end_clk  [num_end] device, the capturing clock pin of each endpoint (-1: none),
 *          as StaNetlistDesc.end_clock, or NULL for an ideal clock.  A clocked
 *          endpoint's hold bound adds the clock pin's late rising arrival and its
 *          setup bound the early rising arrival, exactly as sta_forward does; a
 *          clock pin >= num_pins leaves the endpoint out like a bad end pin
 * ep_slack [num_end][2] device output (early, late), 8-byte aligned; summary
 *          [STA_SUM_COUNT] device output, 8-byte aligned, same slots as
 *          sta_query_summary.
 * Asynchronous on `stream`.  num_end may not exceed STA_NOALLOC_MAX_ENDPOINTS
 * and every pointer must have the alignment stated (end_pins and end_clk 4
 * bytes): otherwise STA_ERR_INVALID_ARG, before any device work (a sliced
 * tensor view may start off its element type's vector boundary).
 *
 * Scratch: a file-scope device array of STA_NOALLOC_MAX_ENDPOINTS / 256
 * partials (1 MiB) that every GPU loading libsta holds until the process
 * exits.  Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress); the first such lookup on a device may load the
 * library's device code, so make the first call before any stream capture.
 * All calls share the array and each call rewrites every partial it reads, so
 * nothing needs clearing, but calls that overlap on the GPU (concurrent
 * streams, or graphs replayed concurrently) race on it. */
#define STA_NOALLOC_MAX_ENDPOINTS (1 << 22)
StaStatus sta_endpoint_summary_noalloc(const float *at, const float *ats, int32_t num_pins,
                                       const int32_t *end_pins, const float *end_rat,
                                       const int32_t *end_clk, int32_t num_end, float gamma,
                                       float *ep_slack, double *summary, void *stream);

/* Handles with STA_BATCH_LANES: run only placements [0, lanes) (1 <= lanes <=
 * num_placements) from the next sta_set_positions on, until changed.  That call
 * and the following ones then take and give [lanes][...] arrays (positions
 * [lanes][num_pins][2], weights [lanes][2], gradients, summaries and queries
 * likewise) and the sweeps run those lanes only, so a call costs what its
 * placements need.  Results are those of each placement alone.
 * STA_ERR_STATE on other handles. */
StaStatus sta_set_active(StaHandle *h, int32_t lanes);

/* Release every resource of the handle (NULL is a no-op). */
void sta_destroy(StaHandle *h);

/* Message of the calling thread's last failed call ("" if none). */
const char *sta_last_error(void);

/* Dependent-load latency of the memory system, the unit of the sweeps' depth
 * floor (each level of a sweep needs at least one round trip through L2 after
 * its producers' stores).  One GPU thread follows a random single-cycle
 * permutation of bytes / 4 int32 indices (Sattolo's algorithm, fixed seed),
 * every load's address being the previous load's value, for `steps` loads
 * through L2 (ld.global.cg); the buffer is read once beforehand, so a buffer
 * well below the L2 size measures an L2 hit and one well above it mostly DRAM.
 * Writes nanoseconds per load (CUDA events around the chase) to
 * *ns_per_load.  Allocates and frees its own device buffer on the current
 * device and synchronizes it.  bytes in [64, 2^33], steps in [1, 10^7]
 * (STA_ERR_INVALID_ARG otherwise); STA_ERR_OOM / STA_ERR_CUDA on failure. */
StaStatus sta_measure_latency(int64_t bytes, int32_t steps, double *ns_per_load);

/* STA_ABI_VERSION of the loaded library. */
int sta_abi_version(void);


/* ---------------------------------------------------------------------------
 * Serving: netlists resident on the device under a memory budget, and a
 * request loop that runs STA / gradient requests on a pool of CUDA streams
 * ("slots").  A worker thread admits each request as soon as a slot is free
 * and its netlist is resident and idle, so requests on different netlists run
 * concurrently on the device; requests of one netlist run in order.  A
 * netlist that is not resident is created when the budget allows, evicting
 * idle netlists in least-recently-used order.  Requests of one netlist run one
 * after another on its resident copy, concurrently on several copies
 * (replicas), or together as the placements of one batched call (merge).  A
 * request's results equal those of the same request run alone.  All calls are
 * thread-safe.
 * ------------------------------------------------------------------------- */
typedef struct StaServer StaServer;

typedef struct {
    int32_t slots;        /* concurrent requests (0 = 4, at most 64) */
    int32_t sequential;   /* 1: the plain loop: one request at a time, in arrival order */
    int64_t budget_bytes; /* device bytes for resident netlists (0 = 150 GiB) */
    int32_t merge;        /* 0: one request per launch.  M in [1, 64]: pending requests of one
                             netlist with the same gamma and kind (forward / gradient) run
                             together, up to M at a time, as the lanes of one call of a lanes
                             handle (STA_BATCH_LANES with M placements, sta_set_active to
                             the requests present).  A lane's results are bit-identical to
                             the same request alone.  Not with sequential. */
    int32_t replicas;     /* resident copies of a netlist, at most (0 = 1): with R > 1, pending
                             requests of one netlist run concurrently on up to R copies (each
                             its own handle; copies beyond the first are made only while the
                             budget allows without evicting).  Not with sequential or merge. */
    int32_t reserved[2];
} StaServerOptions;

typedef struct {
    int32_t netlist;      /* id from sta_server_add_netlist */
    int32_t gradient;     /* 0: forward (AT, LSE-AT, required times, slacks, WNS/TNS);
                             1: forward and the gradient of w_tns TNS_gamma + w_wns WNS_gamma */
    float gamma;          /* smoothing, ps, > 0 */
    float w_tns, w_wns;
    const float *xy;      /* host [num_pins][2]; read until the request completes; pinned
                             memory keeps the copy asynchronous */
    float *grad;          /* host [num_pins][2] (gradient requests; may be NULL); pinned */
    double *summary;      /* host [STA_SUM_COUNT] (may be NULL); written before completion */
} StaServerRequest;

typedef struct {
    int64_t id;
    int32_t status;       /* StaStatus of the request */
    int32_t netlist;
    double t_submit, t_start, t_done; /* sta_server_clock() seconds: submitted, started, seen done */
    int32_t merged;       /* requests that ran in the same launch as this one (1: alone) */
    int32_t reserved;
} StaServerCompletion;

StaStatus sta_server_create(const StaServerOptions *opt, StaServer **out);
/* Register a netlist (arrays are copied) and build its host layout once (the
 * errors of sta_create are reported here); every resident copy is created from
 * that layout, so a netlist evicted under the budget comes back with device
 * allocations and uploads only.  preload != 0 also makes it resident now (OOM
 * if it does not fit), with its further copies (replicas) while the budget
 * allows without evicting.  *id identifies it in requests. */
StaStatus sta_server_add_netlist(StaServer *s, const StaNetlistDesc *nl, const StaLibrary *lib,
                                 int32_t preload, int32_t *id);
StaStatus sta_server_submit(StaServer *s, const StaServerRequest *req, int64_t *id);
/* Up to max completions (waiting up to wait_ms for the first one); *n = count. */
StaStatus sta_server_poll(StaServer *s, StaServerCompletion *out, int32_t max, int32_t *n,
                          int32_t wait_ms);
/* Device bytes a netlist takes when resident: an upper-bound estimate from its
 * sizes until it has been resident once, then the measured amount. */
StaStatus sta_server_netlist_bytes(StaServer *s, int32_t id, int64_t *bytes);
/* out4: resident netlists, resident device bytes, admissions, evictions */
StaStatus sta_server_stats(StaServer *s, int64_t *out4);
/* Finishes every submitted request, then frees everything. */
void sta_server_destroy(StaServer *s);
double sta_server_clock(void); /* steady clock, seconds */

#ifdef __cplusplus
}
#endif
#endif /* STA_H_ */
