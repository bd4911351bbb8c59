/*
 * sta_oracle.c -- plain, slow, FP64 reference static timing analysis.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this file's library.  It shares no
 * code, header, table or constant with the CUDA path, and the CUDA path never
 * calls it.
 *
 * What it computes (Warp-STAR, arXiv 2603.28381):
 *   - Elmore load / delay / second-moment impulse of an RC tree (Eqs. 1-3,
 *     Section 3.1.1), applied to every net modelled as a star: one wire of
 *     Manhattan length d from the driver to each sink, resistance r*d, its
 *     capacitance c*d split half at the driver node and half at the sink node.
 *   - NLDM cell-arc delay and output slew by bilinear inter/extrapolation of
 *     7x7 tables (Section 3.1.2).
 *   - forward arrival time (AT) and slew over the pin graph in topological
 *     order: late = max, early = min over a cell's arcs (Section 2.1, 3.1.2).
 *   - backward required time (RAT) and slack (Section 2.1, 3.1.2).
 *   - endpoint slack, WNS, TNS.
 *   - LogSumExp arrival times (Eq. 4, Section 3.2) in place of the late max at
 *     cell outputs, the smoothed TNS/WNS built from them, and the analytic
 *     adjoint of that loss with respect to every pin position.
 *
 * It walks the pin graph in Kahn topological order, not the GPU's levels.
 * Readings of points the paper leaves open:
 *   - segment of a table axis = largest k in [0,5] with idx[k] <= v (right
 *     continuous); outside the index range the edge segment is extended
 *     linearly (no clamping of the interpolated value).
 *   - late output slew = max, early = min over arcs (independent worst-slew
 *     merge); gradient of the late max goes to the first arc attaining it.
 *   - wire slew degradation: slew_sink = sqrt(slew_driver^2 + impulse^2).
 *   - LSE replaces only the late AT max at cell outputs (rise and fall); slews
 *     and the early mode stay hard.
 *   - endpoint slack uses the endpoint's own constraint: late = RAT_c - AT,
 *     early = AT - RAT_c, minimum over rise/fall.
 *   - TNS_gamma = sum_e softmin_gamma(s_e_rise, s_e_fall, 0) and
 *     WNS_gamma = softmin_gamma over every endpoint rise/fall slack, where
 *     softmin_gamma(x) = -LSE_gamma(-x) stabilised by the extremum as in Eq. 4.
 *   - sign(0) = 0 in the derivative of |x_s - x_d|.
 *   - propagated clock: an endpoint may name the clock pin of the flop that
 *     captures it.  Its hold bound (early required time) then adds that pin's
 *     late rising arrival and its setup bound (late required time) the early
 *     rising arrival (the latest and the earliest capture edge).  The clock pin
 *     must be a sink of a net driven by a startpoint, so its arrival is the
 *     startpoint's plus the wire delay and the setup term's adjoint goes to
 *     that wire delay.
 * Units: ps, fF, Ohm, um; Ohm*fF = 1e-3 ps.  Condition index = 2*el + rf with
 * el 0 early / 1 late and rf 0 rise / 1 fall.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_LUT 7
#define OR_MAXA 4
#define OR_KRC 1e-3 /* Ohm * fF in ps */

typedef struct {
    int P, N, C;
    const int *net_ptr, *net_pins;
    const int *cell_type, *cell_in_ptr, *cell_in_pins, *cell_out_pin;
    const float *pin_cap;
    int S;
    const int *start_pins;
    const float *start_at, *start_slew;
    int E;
    const int *end_pins;
    const float *end_rat;
    double r_per_um, c_per_um;
    int T;
    const int *type_num_arcs;
    const signed char *arc_unate;
    const float *slew_index, *load_index, *delay_tab, *slew_tab;
    const int *end_clk;  /* [E] capturing clock pin of each endpoint, -1 none; NULL = none */
} OrNetlist;

typedef struct {
    double *at, *slew, *rat;     /* [P][4] */
    double *ats;                 /* [P][2] late rise/fall LSE arrival time */
    double *pin_slack;           /* [P][2] (early, late) */
    double *ep_slack;            /* [E][2] (early, late) */
    double *summary;             /* [8] */
    double *grad;                /* [P][2] d loss / d (x, y) */
    double *net_load;            /* [N] */
    double *wdelay, *impulse;    /* [P] wire delay / impulse at sink pins */
    double *adel;                /* [A][4] cell arc delays, A = cell_in_ptr[C] */
    uint64_t *decision_hash;     /* every discrete choice the loss depends on */
} OrOut;

enum { OR_OK = 0, OR_EINVAL = -1, OR_ECYCLE = -2, OR_ENOMEM = -3 };

/* ------------------------------------------------------------------------ */
/* Eqs. 1-3 on an RC tree.                                                   */
/* ------------------------------------------------------------------------ */
/* Nodes 0..n-1 are ordered parent before child, parent[0] = -1 is the root
 * (the net's driver).  res[u] is the resistance of the edge parent(u) -> u
 * (Ohm), cap[u] the capacitance lumped at node u (fF).
 *   Load(u)  = Cap(u) + sum over children v of Load(v)                 (Eq. 1)
 *   Delay(u) = Delay(parent) + Res(parent -> u) * Load(u)              (Eq. 2,
 *              accumulated along the path, the Elmore delay of a tree)
 *   LD(u)    = Cap(u) * Delay(u) + sum over children v of LD(v)
 *   Beta(u)  = Beta(parent) + Res(parent -> u) * LD(u)
 *   Impulse(u) = sqrt(2 Beta(u) - Delay(u)^2)                           (Eq. 3,
 *              the second-moment form; for a single edge it is exactly
 *              sqrt(2 Res Cap Delay - Delay^2))
 * work must hold 2n doubles. */
void oracle_elmore_tree(int n, const int *parent, const double *res, const double *cap,
                        double *load, double *delay, double *impulse, double *work)
{
    double *ld = work, *beta = work + n;
    for (int u = 0; u < n; ++u) load[u] = cap[u];
    for (int u = n - 1; u >= 1; --u) load[parent[u]] += load[u];
    delay[0] = 0.0;
    for (int u = 1; u < n; ++u) delay[u] = delay[parent[u]] + res[u] * load[u] * OR_KRC;
    for (int u = 0; u < n; ++u) ld[u] = cap[u] * delay[u];
    for (int u = n - 1; u >= 1; --u) ld[parent[u]] += ld[u];
    beta[0] = 0.0;
    for (int u = 1; u < n; ++u) beta[u] = beta[parent[u]] + res[u] * ld[u] * OR_KRC;
    for (int u = 0; u < n; ++u) {
        double m = 2.0 * beta[u] - delay[u] * delay[u];
        impulse[u] = sqrt(m > 0.0 ? m : 0.0);
    }
}

/* ------------------------------------------------------------------------ */
/* NLDM bilinear inter/extrapolation (Section 3.1.2).                        */
/* ------------------------------------------------------------------------ */
static int axis_segment(const float *idx, double v)
{
    int k = 0;
    for (int j = 1; j <= OR_LUT - 2; ++j)
        if ((double)idx[j] <= v) k = j;
    return k;
}

/* tab is one 7x7 table [slew i][load j].  Returns T(s, l) and its partials. */
double oracle_nldm(const float *tab, const float *s_idx, const float *l_idx, double s, double l,
                   double *d_ds, double *d_dl, int *seg_s, int *seg_l)
{
    int i = axis_segment(s_idx, s), j = axis_segment(l_idx, l);
    double s0 = s_idx[i], s1 = s_idx[i + 1], l0 = l_idx[j], l1 = l_idx[j + 1];
    double t = (s - s0) / (s1 - s0), u = (l - l0) / (l1 - l0);
    double t00 = tab[i * OR_LUT + j], t01 = tab[i * OR_LUT + j + 1];
    double t10 = tab[(i + 1) * OR_LUT + j], t11 = tab[(i + 1) * OR_LUT + j + 1];
    double v = (1 - t) * (1 - u) * t00 + t * (1 - u) * t10 + (1 - t) * u * t01 + t * u * t11;
    if (d_ds) *d_ds = ((1 - u) * (t10 - t00) + u * (t11 - t01)) / (s1 - s0);
    if (d_dl) *d_dl = ((1 - t) * (t01 - t00) + t * (t11 - t10)) / (l1 - l0);
    if (seg_s) *seg_s = i;
    if (seg_l) *seg_l = j;
    return v;
}

/* Eq. 4: c + gamma * log sum exp((x_i - c) / gamma) with c = max x_i. */
double oracle_lse(int n, const double *x, double gamma)
{
    double c = -INFINITY, s = 0.0;
    for (int i = 0; i < n; ++i) if (x[i] > c) c = x[i];
    if (!(c > -INFINITY) || !isfinite(c)) return c;
    for (int i = 0; i < n; ++i) s += exp((x[i] - c) / gamma);
    return c + gamma * log(s);
}

/* softmin_gamma(x) = -LSE_gamma(-x). */
static double softmin(int n, const double *x, double gamma)
{
    double m = INFINITY, s = 0.0;
    for (int i = 0; i < n; ++i) if (x[i] < m) m = x[i];
    if (!isfinite(m)) return m;
    for (int i = 0; i < n; ++i) s += exp(-(x[i] - m) / gamma);
    return m - gamma * log(s);
}

static uint64_t fnv(uint64_t h, int64_t v)
{
    for (int b = 0; b < 8; ++b) { h ^= (uint64_t)((v >> (8 * b)) & 0xff); h *= 1099511628211ULL; }
    return h;
}

static int sgn(double v) { return (v > 0) - (v < 0); }

/* ------------------------------------------------------------------------ */
/* Levelization by memoised depth-first search (Section 2.1 stage 2):        */
/* level(net) = 0 if its driver is not a cell output, else 1 + the largest   */
/* level among the nets that feed the driver cell's inputs (inputs on no net */
/* count as -1).  Returns the number of levels, or a negative error.         */
/* ------------------------------------------------------------------------ */
int oracle_levels(const OrNetlist *nl, int *net_level)
{
    int P = nl->P, N = nl->N, C = nl->C;
    int *sink_net = malloc(sizeof(int) * (size_t)P), *out_cell = malloc(sizeof(int) * (size_t)P);
    int *state = calloc((size_t)N, sizeof(int)), *stack = malloc(sizeof(int) * (size_t)(N + 1));
    int *cursor = calloc((size_t)N, sizeof(int));
    int rc = OR_OK, maxl = -1;
    if (!sink_net || !out_cell || !state || !stack || !cursor) { rc = OR_ENOMEM; goto done; }
    for (int p = 0; p < P; ++p) sink_net[p] = out_cell[p] = -1;
    for (int n = 0; n < N; ++n)
        for (int k = nl->net_ptr[n] + 1; k < nl->net_ptr[n + 1]; ++k) sink_net[nl->net_pins[k]] = n;
    for (int c = 0; c < C; ++c) out_cell[nl->cell_out_pin[c]] = c;
    /* state: 0 unvisited, 1 on stack, 2 done */
    for (int root = 0; root < N; ++root) {
        if (state[root]) continue;
        int sp = 0;
        stack[sp++] = root;
        state[root] = 1;
        cursor[root] = 0;
        while (sp) {
            int n = stack[sp - 1];
            int c = out_cell[nl->net_pins[nl->net_ptr[n]]];
            int nin = c >= 0 ? nl->cell_in_ptr[c + 1] - nl->cell_in_ptr[c] : 0;
            if (cursor[n] < nin) {
                int pin = nl->cell_in_pins[nl->cell_in_ptr[c] + cursor[n]++];
                int m = sink_net[pin];
                if (m < 0 || state[m] == 2) continue;
                if (state[m] == 1) { rc = OR_ECYCLE; goto done; }
                state[m] = 1;
                cursor[m] = 0;
                stack[sp++] = m;
                continue;
            }
            int lv = 0;
            for (int k = 0; k < nin; ++k) {
                int m = sink_net[nl->cell_in_pins[nl->cell_in_ptr[c] + k]];
                if (m >= 0 && net_level[m] + 1 > lv) lv = net_level[m] + 1;
            }
            net_level[n] = lv;
            if (lv > maxl) maxl = lv;
            state[n] = 2;
            --sp;
        }
    }
done:
    free(sink_net); free(out_cell); free(state); free(stack); free(cursor);
    return rc == OR_OK ? maxl + 1 : rc;
}

/* ------------------------------------------------------------------------ */
/* Full STA + smoothed loss + adjoint.                                        */
/* ------------------------------------------------------------------------ */
int oracle_sta(const OrNetlist *nl, const double *xy, double gamma, double w_tns, double w_wns,
               OrOut *out)
{
    const int P = nl->P, N = nl->N, C = nl->C, E = nl->E;
    const int A = C ? nl->cell_in_ptr[C] : 0;
    const double r = nl->r_per_um, cw = nl->c_per_um;
    int rc = OR_OK;
    if (!(gamma > 0.0)) return OR_EINVAL;

    int *sink_net = malloc(sizeof(int) * (size_t)P), *drv_net = malloc(sizeof(int) * (size_t)P);
    int *out_cell = malloc(sizeof(int) * (size_t)P), *in_arc = malloc(sizeof(int) * (size_t)P);
    int *start_of = malloc(sizeof(int) * (size_t)P), *end_of = malloc(sizeof(int) * (size_t)P);
    int *indeg = calloc((size_t)P, sizeof(int)), *topo = malloc(sizeof(int) * (size_t)P);
    int *arc_cell = malloc(sizeof(int) * (size_t)(A + 1));
    double *at = malloc(sizeof(double) * 4 * (size_t)P), *sl = malloc(sizeof(double) * 4 * (size_t)P);
    double *rat = malloc(sizeof(double) * 4 * (size_t)P), *ats = malloc(sizeof(double) * 2 * (size_t)P);
    double *load = malloc(sizeof(double) * (size_t)N), *wd = calloc((size_t)P, sizeof(double));
    double *imp = calloc((size_t)P, sizeof(double)), *dist = calloc((size_t)P, sizeof(double));
    double *adel = malloc(sizeof(double) * 4 * (size_t)(A + 1));
    double *ga = calloc(2 * (size_t)P, sizeof(double)), *gs = calloc(2 * (size_t)P, sizeof(double));
    double *gwd = calloc((size_t)P, sizeof(double)), *gimp = calloc((size_t)P, sizeof(double));
    double *gload = calloc((size_t)P, sizeof(double));
    double *grad = calloc(2 * (size_t)P, sizeof(double));
    double *sm = malloc(sizeof(double) * 2 * (size_t)(E + 1));
    double *con = malloc(sizeof(double) * 4 * (size_t)(E + 1)); /* effective endpoint bounds */
    int maxdeg = 1;
    for (int n = 0; n < N; ++n)
        if (nl->net_ptr[n + 1] - nl->net_ptr[n] > maxdeg) maxdeg = nl->net_ptr[n + 1] - nl->net_ptr[n];
    int *tpar = malloc(sizeof(int) * (size_t)maxdeg);
    double *tres = malloc(sizeof(double) * (size_t)maxdeg), *tcap = malloc(sizeof(double) * (size_t)maxdeg);
    double *tload = malloc(sizeof(double) * (size_t)maxdeg), *tdel = malloc(sizeof(double) * (size_t)maxdeg);
    double *timp = malloc(sizeof(double) * (size_t)maxdeg), *twork = malloc(sizeof(double) * 2 * (size_t)maxdeg);
    if (!sink_net || !drv_net || !out_cell || !in_arc || !start_of || !end_of || !indeg || !topo ||
        !arc_cell || !at || !sl || !rat || !ats || !load || !wd || !imp || !dist || !adel || !ga ||
        !gs || !gwd || !gimp || !gload || !grad || !sm || !con || !tpar || !tres || !tcap || !tload ||
        !tdel || !timp || !twork) { rc = OR_ENOMEM; goto done; }

    /* ---- roles of every pin, with validation ---- */
    for (int p = 0; p < P; ++p) sink_net[p] = drv_net[p] = out_cell[p] = in_arc[p] = start_of[p] = end_of[p] = -1;
    for (int n = 0; n < N; ++n) {
        int b = nl->net_ptr[n], e = nl->net_ptr[n + 1];
        if (e <= b) { rc = OR_EINVAL; goto done; }
        for (int k = b; k < e; ++k) {
            int p = nl->net_pins[k];
            if (p < 0 || p >= P) { rc = OR_EINVAL; goto done; }
            if (k == b) { if (drv_net[p] >= 0) { rc = OR_EINVAL; goto done; } drv_net[p] = n; }
            else { if (sink_net[p] >= 0) { rc = OR_EINVAL; goto done; } sink_net[p] = n; }
        }
    }
    for (int c = 0; c < C; ++c) {
        int t = nl->cell_type[c], o = nl->cell_out_pin[c];
        int k = nl->cell_in_ptr[c + 1] - nl->cell_in_ptr[c];
        if (t < 0 || t >= nl->T || o < 0 || o >= P || k < 1 || k > OR_MAXA || k != nl->type_num_arcs[t] ||
            out_cell[o] >= 0) { rc = OR_EINVAL; goto done; }
        out_cell[o] = c;
        for (int a = nl->cell_in_ptr[c]; a < nl->cell_in_ptr[c + 1]; ++a) {
            int p = nl->cell_in_pins[a];
            if (p < 0 || p >= P || in_arc[p] >= 0) { rc = OR_EINVAL; goto done; }
            in_arc[p] = a;
            arc_cell[a] = c;
        }
    }
    for (int s = 0; s < nl->S; ++s) {
        int p = nl->start_pins[s];
        if (p < 0 || p >= P || start_of[p] >= 0) { rc = OR_EINVAL; goto done; }
        start_of[p] = s;
    }
    for (int e = 0; e < E; ++e) {
        int p = nl->end_pins[e];
        if (p < 0 || p >= P || end_of[p] >= 0) { rc = OR_EINVAL; goto done; }
        end_of[p] = e;
    }
    /* every pin has exactly one source of its arrival time */
    for (int p = 0; p < P; ++p) {
        int nsrc = (start_of[p] >= 0) + (sink_net[p] >= 0) + (out_cell[p] >= 0);
        if (nsrc != 1) { rc = OR_EINVAL; goto done; }
    }
    /* a capturing clock pin hangs on a net driven by a startpoint */
    for (int e = 0; nl->end_clk && e < E; ++e) {
        int k = nl->end_clk[e];
        if (k < -1 || k >= P) { rc = OR_EINVAL; goto done; }
        if (k >= 0 && (sink_net[k] < 0 || start_of[nl->net_pins[nl->net_ptr[sink_net[k]]]] < 0)) {
            rc = OR_EINVAL;
            goto done;
        }
    }

    /* ---- net RC (Eqs. 1-3) on each star ---- */
    for (int n = 0; n < N; ++n) {
        int b = nl->net_ptr[n], e = nl->net_ptr[n + 1], k = e - b;
        int d = nl->net_pins[b];
        tpar[0] = -1;
        tres[0] = 0.0;
        tcap[0] = nl->pin_cap[d];
        for (int i = 1; i < k; ++i) {
            int s = nl->net_pins[b + i];
            double len = fabs(xy[2 * s] - xy[2 * d]) + fabs(xy[2 * s + 1] - xy[2 * d + 1]);
            dist[s] = len;
            tpar[i] = 0;
            tres[i] = r * len;
            tcap[0] += 0.5 * cw * len;
            tcap[i] = nl->pin_cap[s] + 0.5 * cw * len;
        }
        oracle_elmore_tree(k, tpar, tres, tcap, tload, tdel, timp, twork);
        load[n] = tload[0];
        for (int i = 1; i < k; ++i) {
            int s = nl->net_pins[b + i];
            wd[s] = tdel[i];
            imp[s] = timp[i];
        }
    }

    /* ---- Kahn topological order of the pin graph ---- */
    for (int p = 0; p < P; ++p) {
        if (sink_net[p] >= 0) indeg[p] = 1;
        if (out_cell[p] >= 0) { int c = out_cell[p]; indeg[p] = nl->cell_in_ptr[c + 1] - nl->cell_in_ptr[c]; }
    }
    int head = 0, tail = 0;
    for (int p = 0; p < P; ++p) if (indeg[p] == 0) topo[tail++] = p;
    while (head < tail) {
        int p = topo[head++];
        if (drv_net[p] >= 0) {
            int n = drv_net[p];
            for (int k = nl->net_ptr[n] + 1; k < nl->net_ptr[n + 1]; ++k)
                if (--indeg[nl->net_pins[k]] == 0) topo[tail++] = nl->net_pins[k];
        }
        if (in_arc[p] >= 0) {
            int o = nl->cell_out_pin[arc_cell[in_arc[p]]];
            if (--indeg[o] == 0) topo[tail++] = o;
        }
    }
    if (tail != P) { rc = OR_ECYCLE; goto done; }

    /* ---- forward: AT, slew (4 conditions) and LSE arrival time ---- */
    uint64_t hash = 1469598103934665603ULL;
    for (int ti = 0; ti < P; ++ti) {
        int p = topo[ti];
        if (start_of[p] >= 0) {
            int s = start_of[p];
            for (int q = 0; q < 4; ++q) { at[4 * p + q] = nl->start_at[4 * s + q]; sl[4 * p + q] = nl->start_slew[4 * s + q]; }
            ats[2 * p] = at[4 * p + 2];
            ats[2 * p + 1] = at[4 * p + 3];
        } else if (sink_net[p] >= 0) {
            int d = nl->net_pins[nl->net_ptr[sink_net[p]]];
            for (int q = 0; q < 4; ++q) {
                at[4 * p + q] = at[4 * d + q] + wd[p];
                sl[4 * p + q] = sqrt(sl[4 * d + q] * sl[4 * d + q] + imp[p] * imp[p]);
            }
            ats[2 * p] = ats[2 * d] + wd[p];
            ats[2 * p + 1] = ats[2 * d + 1] + wd[p];
        } else {
            int c = out_cell[p], t = nl->cell_type[c];
            int a0 = nl->cell_in_ptr[c], a1 = nl->cell_in_ptr[c + 1];
            double ld = drv_net[p] >= 0 ? load[drv_net[p]] : nl->pin_cap[p];
            const float *si = nl->slew_index + OR_LUT * t, *li = nl->load_index + OR_LUT * t;
            for (int el = 0; el < 2; ++el)
                for (int rf = 0; rf < 2; ++rf) {
                    double best_at = el ? -INFINITY : INFINITY, best_sl = el ? -INFINITY : INFINITY;
                    double cand[OR_MAXA];
                    int argmax = -1;
                    for (int a = a0; a < a1; ++a) {
                        int ai = a - a0, i = nl->cell_in_pins[a];
                        int rfi = nl->arc_unate[OR_MAXA * t + ai] > 0 ? rf : 1 - rf;
                        size_t tab = ((size_t)(t * OR_MAXA + ai) * 2 + rf) * OR_LUT * OR_LUT;
                        int ks, kl;
                        double s_in = sl[4 * i + 2 * el + rfi];
                        double D = oracle_nldm(nl->delay_tab + tab, si, li, s_in, ld, NULL, NULL, &ks, &kl);
                        double S = oracle_nldm(nl->slew_tab + tab, si, li, s_in, ld, NULL, NULL, NULL, NULL);
                        adel[4 * a + 2 * el + rf] = D;
                        double v = at[4 * i + 2 * el + rfi] + D;
                        if (el) {
                            if (v > best_at) best_at = v;
                            if (S > best_sl) { best_sl = S; argmax = ai; }
                            cand[ai] = ats[2 * i + rfi] + D;
                            hash = fnv(hash, ks);
                            hash = fnv(hash, kl);
                        } else {
                            if (v < best_at) best_at = v;
                            if (S < best_sl) best_sl = S;
                        }
                    }
                    at[4 * p + 2 * el + rf] = best_at;
                    sl[4 * p + 2 * el + rf] = best_sl;
                    if (el) {
                        ats[2 * p + rf] = oracle_lse(a1 - a0, cand, gamma);
                        hash = fnv(hash, argmax);
                    }
                }
        }
    }
    for (int n = 0; n < N; ++n) {
        int d = nl->net_pins[nl->net_ptr[n]];
        for (int k = nl->net_ptr[n] + 1; k < nl->net_ptr[n + 1]; ++k) {
            int s = nl->net_pins[k];
            hash = fnv(hash, sgn(xy[2 * s] - xy[2 * d]));
            hash = fnv(hash, sgn(xy[2 * s + 1] - xy[2 * d + 1]));
        }
    }

    /* ---- endpoint bounds: the constraint plus the capturing clock's arrival ---- */
    for (int e = 0; e < E; ++e) {
        int k = nl->end_clk ? nl->end_clk[e] : -1;
        for (int q = 0; q < 4; ++q) {
            con[4 * e + q] = nl->end_rat[4 * e + q];
            if (k >= 0) con[4 * e + q] += q < 2 ? at[4 * k + 2] : at[4 * k + 0];
        }
    }

    /* ---- backward: required times in reverse topological order ---- */
    for (int p = 0; p < P; ++p) {
        rat[4 * p] = rat[4 * p + 1] = -INFINITY;
        rat[4 * p + 2] = rat[4 * p + 3] = INFINITY;
        if (end_of[p] >= 0)
            for (int q = 0; q < 4; ++q) rat[4 * p + q] = con[4 * end_of[p] + q];
    }
    for (int ti = P - 1; ti >= 0; --ti) {
        int p = topo[ti];
        if (drv_net[p] >= 0) {
            int n = drv_net[p];
            for (int k = nl->net_ptr[n] + 1; k < nl->net_ptr[n + 1]; ++k) {
                int s = nl->net_pins[k];
                for (int q = 0; q < 4; ++q) {
                    double v = rat[4 * s + q] - wd[s];
                    if (q < 2) { if (v > rat[4 * p + q]) rat[4 * p + q] = v; }
                    else if (v < rat[4 * p + q]) rat[4 * p + q] = v;
                }
            }
        }
        if (in_arc[p] >= 0) {
            int a = in_arc[p], c = arc_cell[a], t = nl->cell_type[c], ai = a - nl->cell_in_ptr[c];
            int o = nl->cell_out_pin[c];
            for (int el = 0; el < 2; ++el)
                for (int rf = 0; rf < 2; ++rf) {
                    int rfi = nl->arc_unate[OR_MAXA * t + ai] > 0 ? rf : 1 - rf;
                    double v = rat[4 * o + 2 * el + rf] - adel[4 * a + 2 * el + rf];
                    double *dst = &rat[4 * p + 2 * el + rfi];
                    if (el) { if (v < *dst) *dst = v; }
                    else if (v > *dst) *dst = v;
                }
        }
    }

    /* ---- slacks, WNS, TNS (hard) and the smoothed loss ---- */
    double wns[2] = {INFINITY, INFINITY}, tns[2] = {0.0, 0.0};
    int nviol = 0;
    for (int e = 0; e < E; ++e) {
        int p = nl->end_pins[e];
        const double *ce = con + 4 * e;
        double se = fmin(at[4 * p] - ce[0], at[4 * p + 1] - ce[1]);
        double sL = fmin(ce[2] - at[4 * p + 2], ce[3] - at[4 * p + 3]);
        if (out && out->ep_slack) { out->ep_slack[2 * e] = se; out->ep_slack[2 * e + 1] = sL; }
        if (se < wns[0]) wns[0] = se;
        if (sL < wns[1]) wns[1] = sL;
        if (se < 0) tns[0] += se;
        if (sL < 0) { tns[1] += sL; ++nviol; }
        sm[2 * e] = ce[2] - ats[2 * p];
        sm[2 * e + 1] = ce[3] - ats[2 * p + 1];
    }
    double tns_g = 0.0;
    for (int e = 0; e < E; ++e) {
        double trip[3] = {sm[2 * e], sm[2 * e + 1], 0.0};
        tns_g += softmin(3, trip, gamma);
    }
    double wns_g = softmin(2 * E, sm, gamma);

    /* ---- adjoint of loss = w_tns * TNS_gamma + w_wns * WNS_gamma ---- */
    for (int e = 0; e < E; ++e) {
        int p = nl->end_pins[e];
        double trip[3] = {sm[2 * e], sm[2 * e + 1], 0.0};
        double te = softmin(3, trip, gamma);
        for (int rf = 0; rf < 2; ++rf) {
            double s = sm[2 * e + rf];
            double dl_ds = w_tns * exp(-(s - te) / gamma);
            if (isfinite(wns_g)) dl_ds += w_wns * exp(-(s - wns_g) / gamma);
            ga[2 * p + rf] += -dl_ds; /* s = RAT_c - ATs */
            /* RAT_c = constraint + early rising arrival of the clock pin k =
             * its startpoint's arrival + wire delay of k */
            if (nl->end_clk && nl->end_clk[e] >= 0) gwd[nl->end_clk[e]] += dl_ds;
        }
    }
    for (int ti = P - 1; ti >= 0; --ti) {
        int p = topo[ti];
        if (sink_net[p] >= 0) {
            int d = nl->net_pins[nl->net_ptr[sink_net[p]]];
            for (int rf = 0; rf < 2; ++rf) {
                ga[2 * d + rf] += ga[2 * p + rf];
                gwd[p] += ga[2 * p + rf];
                double sp = sl[4 * p + 2 + rf], sd = sl[4 * d + 2 + rf];
                if (sp > 0.0) {
                    gs[2 * d + rf] += gs[2 * p + rf] * sd / sp;
                    gimp[p] += gs[2 * p + rf] * imp[p] / sp;
                }
            }
        } else if (out_cell[p] >= 0) {
            int c = out_cell[p], t = nl->cell_type[c];
            int a0 = nl->cell_in_ptr[c], a1 = nl->cell_in_ptr[c + 1];
            double ld = drv_net[p] >= 0 ? load[drv_net[p]] : nl->pin_cap[p];
            const float *si = nl->slew_index + OR_LUT * t, *li = nl->load_index + OR_LUT * t;
            for (int rf = 0; rf < 2; ++rf) {
                double best = -INFINITY, dss = 0.0, dsl = 0.0;
                int amax = -1;
                for (int a = a0; a < a1; ++a) {
                    int ai = a - a0, i = nl->cell_in_pins[a];
                    int rfi = nl->arc_unate[OR_MAXA * t + ai] > 0 ? rf : 1 - rf;
                    size_t tab = ((size_t)(t * OR_MAXA + ai) * 2 + rf) * OR_LUT * OR_LUT;
                    double s_in = sl[4 * i + 2 + rfi], dDs, dDl, dSs, dSl;
                    double D = oracle_nldm(nl->delay_tab + tab, si, li, s_in, ld, &dDs, &dDl, NULL, NULL);
                    double S = oracle_nldm(nl->slew_tab + tab, si, li, s_in, ld, &dSs, &dSl, NULL, NULL);
                    double w = exp((ats[2 * i + rfi] + D - ats[2 * p + rf]) / gamma);
                    double gD = ga[2 * p + rf] * w;
                    ga[2 * i + rfi] += gD;
                    gs[2 * i + rfi] += gD * dDs;
                    gload[p] += gD * dDl;
                    if (S > best) { best = S; amax = a; dss = dSs; dsl = dSl; }
                }
                if (amax >= 0) {
                    int i = nl->cell_in_pins[amax], ai = amax - a0;
                    int rfi = nl->arc_unate[OR_MAXA * t + ai] > 0 ? rf : 1 - rf;
                    gs[2 * i + rfi] += gs[2 * p + rf] * dss;
                    gload[p] += gs[2 * p + rf] * dsl;
                }
            }
        }
    }
    /* distances -> positions.  Delay_s = k r d (cap_s + c d / 2); on a star
     * Eq. 3 gives Impulse_s = Delay_s exactly (2 Beta = 2 Delay^2), so both
     * share dDelay/dd = k r (cap_s + c d).  Load(root) gains c per unit d. */
    for (int n = 0; n < N; ++n) {
        int d = nl->net_pins[nl->net_ptr[n]];
        for (int k = nl->net_ptr[n] + 1; k < nl->net_ptr[n + 1]; ++k) {
            int s = nl->net_pins[k];
            double gd = gload[d] * cw + (gwd[s] + gimp[s]) * OR_KRC * r * (nl->pin_cap[s] + cw * dist[s]);
            double sx = sgn(xy[2 * s] - xy[2 * d]), sy = sgn(xy[2 * s + 1] - xy[2 * d + 1]);
            grad[2 * s] += gd * sx;
            grad[2 * d] -= gd * sx;
            grad[2 * s + 1] += gd * sy;
            grad[2 * d + 1] -= gd * sy;
        }
    }

    if (out) {
        size_t P4 = 4 * (size_t)P, P2 = 2 * (size_t)P;
        if (out->at) memcpy(out->at, at, sizeof(double) * P4);
        if (out->slew) memcpy(out->slew, sl, sizeof(double) * P4);
        if (out->rat) memcpy(out->rat, rat, sizeof(double) * P4);
        if (out->ats) memcpy(out->ats, ats, sizeof(double) * P2);
        if (out->grad) memcpy(out->grad, grad, sizeof(double) * P2);
        if (out->net_load) memcpy(out->net_load, load, sizeof(double) * (size_t)N);
        if (out->wdelay) memcpy(out->wdelay, wd, sizeof(double) * (size_t)P);
        if (out->impulse) memcpy(out->impulse, imp, sizeof(double) * (size_t)P);
        if (out->adel && A) memcpy(out->adel, adel, sizeof(double) * 4 * (size_t)A);
        if (out->pin_slack)
            for (int p = 0; p < P; ++p) {
                out->pin_slack[2 * p] = fmin(at[4 * p] - rat[4 * p], at[4 * p + 1] - rat[4 * p + 1]);
                out->pin_slack[2 * p + 1] = fmin(rat[4 * p + 2] - at[4 * p + 2], rat[4 * p + 3] - at[4 * p + 3]);
            }
        if (out->summary) {
            out->summary[0] = wns[0];
            out->summary[1] = tns[0];
            out->summary[2] = wns[1];
            out->summary[3] = tns[1];
            out->summary[4] = tns_g;
            out->summary[5] = wns_g;
            out->summary[6] = w_tns * tns_g + (isfinite(wns_g) ? w_wns * wns_g : 0.0);
            out->summary[7] = nviol;
        }
        if (out->decision_hash) *out->decision_hash = hash;
    }
done:
    free(sink_net); free(drv_net); free(out_cell); free(in_arc); free(start_of); free(end_of);
    free(indeg); free(topo); free(arc_cell); free(at); free(sl); free(rat); free(ats); free(load);
    free(wd); free(imp); free(dist); free(adel); free(ga); free(gs); free(gwd); free(gimp);
    free(gload); free(grad); free(sm); free(con); free(tpar); free(tres); free(tcap); free(tload); free(tdel);
    free(timp); free(twork);
    return rc;
}
