/*
 * FP64 reference ("oracle") for the look-ahead eco-driving DP.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file: only the tests, the smoke check and the benchmark's CPU
 * baseline leg use it.  It shares no code, header or table with the CUDA
 * library.
 *
 * What it computes (A GPU Implementation of a Look-Ahead Optimal Controller
 * for Eco-Driving Based on Dynamic Programming, Zhu et al., ECC 2021):
 *   - the distance-domain dynamics x_{s+1} = f_s(x_s, u_s) of Eq. (3)-(5) for
 *     x = [v, soc, t] and u = [T_eng, T_bsg] (plus a brake flag),
 *   - the stage cost (gamma * mdot_f + 1 - gamma) * dt of Eq. (1), (2), (6),
 *   - the constraints of Eq. (7) and the traffic-light feasibility of Eq. (8),
 *   - the backward recursion of Eq. (9a)-(9d) with hard masks (infeasible =
 *     +inf) instead of the penalty functions phi,
 *   - a forward rollout that re-minimises at the continuous state.
 * The loops follow the serial architecture of Sec. IV (Fig. 5): states
 * (v, soc, t) outermost, then engine torque, motor torque and brake flag, with
 * the full model evaluated for every state-control pair and no early exits.
 *
 * Readings of points the paper leaves open are listed beside the code that
 * applies them.  Every grid is given per stage as explicit, strictly
 * increasing node arrays; uniform grids are one case of that.
 *
 * FP32-fragile decisions.  A decision whose FP64 outcome is within the FP32
 * resolution of its threshold (a phase boundary within phase_band seconds, an
 * acceleration/discriminant/radicand within fp_band of zero, an
 * interpolation fraction or grid-band edge within fp_band * (1 + scale) index
 * units of its threshold) is "fragile".  Mode NOMINAL takes every decision
 * at face value.  Mode LENIENT evaluates every combination of the fragile
 * decisions of a transition and keeps the smallest cost; mode STRICT keeps
 * the largest (+inf if any combination is infeasible).  The three modes bound
 * what a correct lower-precision implementation may return.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_OK 0
#define ORC_ERR_ARG 1
#define ORC_ERR_INFEASIBLE 4
#define ORC_ERR_OOM 2

#define ORC_NOMINAL 0
#define ORC_LENIENT 1
#define ORC_STRICT 2

/* Interpolation snapping (reading of the generic DP interpolation the paper
 * defers to): a fraction below 1e-5 of a cell is snapped to the node, and a
 * point up to 1e-5 of a cell outside the grid is clamped to the edge. */
#define SNAP 1e-5

typedef struct {
    int32_t n_stages;
    double ds;
    const double *grade;      /* [n_stages], fraction */
    /* per-stage grids, stage k = 0..n_stages, node arrays concatenated */
    const int32_t *nv;
    const double *v_nodes;
    const int32_t *nxi;
    const double *xi_nodes;
    const int32_t *nt;
    const double *t_nodes;
    /* controls */
    int32_t n_te;
    const double *te;
    int32_t n_tm;
    const double *tm;
    int32_t n_b;
    double brake_decel;
    double a_min, a_max;
    double mass, cda, crr, rho, g, r_wheel, gear, eta_motor;
    double voc, r0, cap_As;
    double fuel_coef[6];
    double fuel_scale, gamma;
    double soc_ref, w_soc, v_ref, w_v;
    int32_t n_lights;
    const int32_t *light_node;
    const double *cycle, *red, *offset;
    double fp_band;    /* relative FP32 resolution band, index units */
    double phase_band; /* seconds */
    /* prefix sums of the per-stage sizes: node arrays (N+1 entries each) and
     * value arrays (N+2 entries, stage k at V_off[k]) */
    const int64_t *v_off, *xi_off, *t_off, *V_off;
    /* paper variants (0 = the default readings):
     * light_model 1: the green indicator sampled on the time grid (Sec. III,
     *   Eq. 8): at a light node, every state with v > 0 at a red time node is
     *   infeasible, and arrivals are not checked at the continuous time;
     * light_model 2: the literal standstill step of Eq. (5c) (see transition);
     * torque_limits 1: speed-dependent torque limits (Eq. 7e, 7f),
     *   T_eng <= c0 + c1 w + c2 w^2 and |T_bsg| w <= bsg_power_max, with w the
     *   engine (= BSG) speed at the stage-start speed. */
    int32_t light_model;
    int32_t torque_limits;
    double te_max_coef[3];
    double bsg_power_max;
} orc_problem;

typedef struct {
    double v1, xi1, t1; /* next state */
    double dt;          /* driving time of the step, Eq. (2) */
    double wait;        /* standstill time at a red light before departing */
    double fuel_rate;   /* g/s while driving */
    double cost;        /* stage cost, Eq. (6) */
} orc_trans;

/* Decision bookkeeping for FP32-fragile comparisons. */
typedef struct {
    uint32_t mask; /* which fragile decisions to flip */
    int nf;        /* fragile decisions met so far */
} dec_ctx;

static int decide(dec_ctx *d, int nominal, int fragile)
{
    if (!fragile || d == NULL)
        return nominal;
    int flip = (d->nf < 31) ? (int)((d->mask >> d->nf) & 1u) : 0;
    d->nf++;
    return nominal ^ flip;
}

/* ---- grids --------------------------------------------------------------- */

static int64_t value_offset(const orc_problem *P, int stage) { return P->V_off[stage]; }

int64_t orc_value_offset(const orc_problem *P, int stage) { return value_offset(P, stage); }

/* ---- traffic lights (Fig. 3, Eq. 5c, Eq. 8) ------------------------------ */

static int light_at(const orc_problem *P, int node)
{
    for (int j = 0; j < P->n_lights; ++j)
        if (P->light_node[j] == node)
            return j;
    return -1;
}

/* Position inside the light cycle: ((t - offset) mod cycle) in [0, cycle).
 * Reading: red comes first after the offset and lasts red[j] seconds. */
static double phase_of(const orc_problem *P, int j, double t)
{
    double c = P->cycle[j];
    double ph = fmod(t - P->offset[j], c);
    if (ph < 0)
        ph += c;
    if (ph >= c)
        ph -= c;
    return ph;
}

int orc_is_red(const orc_problem *P, int j, double t)
{
    return phase_of(P, j, t) < P->red[j];
}

static int phase_fragile(const orc_problem *P, int j, double ph)
{
    double b = P->phase_band;
    return ph < b || fabs(ph - P->red[j]) < b || P->cycle[j] - ph < b;
}

/* ---- model: one distance step (Eq. 2, 5a-5c, 7) ---------------------------
 * Readings: P0 drivetrain with one total ratio gear/r_wheel; engine and motor
 * speeds are v * gear / r_wheel taken at the stage-start speed (the powertrain
 * model takes the current speed, Sec. IV); constant motor efficiency; battery
 * as a zeroth-order circuit, I = (Voc - sqrt(Voc^2 - 4 R0 P)) / (2 R0); no
 * auxiliary load.  Stopping: if v^2 + 2 ds a < 0 the step is infeasible,
 * except when the next node holds a light, where the vehicle stops at the
 * stop line (v' = 0, dt = 2 ds / v).  Red arrival: arriving at a light node
 * with v' > 0 while it is red is infeasible.  Departure: standing (v = 0) at
 * a light node while red, the vehicle waits for green, at a time-only cost
 * (1 - gamma) * wait and with the engine off.  Returns 1 when feasible. */
static int transition(const orc_problem *P, int k, double v, double xi, double t,
                      double Te, double Tm, int b, dec_ctx *d, orc_trans *o)
{
    const double M = P->mass;
    double p = P->grade[k];
    double sq = sqrt(1.0 + p * p);
    double sin_th = p / sq, cos_th = 1.0 / sq;
    double F_road = M * P->g * (P->crr * cos_th + sin_th) + 0.5 * P->rho * P->cda * v * v;
    double ratio = P->gear / P->r_wheel;
    double F_tr = (Te + Tm) * ratio - (b ? M * P->brake_decel : 0.0);
    double a = (F_tr - F_road) / M;
    double ea = P->fp_band * (fabs(F_tr) + fabs(F_road)) / M;
    double w = v * ratio;

    /* Eq. (7e), (7f) with speed-dependent limits (variant) */
    if (P->torque_limits) {
        const double *c = P->te_max_coef;
        double te_max = c[0] + c[1] * w + c[2] * w * w;
        if (decide(d, Te > te_max, fabs(Te - te_max) <= P->fp_band * (fabs(Te) + fabs(te_max) + 1.0)))
            return 0;
        double pm = fabs(Tm) * w;
        if (decide(d, pm > P->bsg_power_max, fabs(pm - P->bsg_power_max) <= P->fp_band * (pm + P->bsg_power_max + 1.0)))
            return 0;
    }

    /* Eq. (7d): comfort acceleration limits */
    if (decide(d, a < P->a_min, fabs(a - P->a_min) <= ea))
        return 0;
    if (decide(d, a > P->a_max, fabs(a - P->a_max) <= ea))
        return 0;

    /* the literal Eq. (5c) (variant light_model 2): standing at a light node,
     * a control without forward acceleration makes the step at zero speed
     * while the clock jumps to the end of red (zero time during green); the
     * engine is off at standstill (start-stop), so only T_eng = 0 realises it.
     * A departure needs green; there is no folded wait. */
    int lk = light_at(P, k);
    if (P->light_model == 2 && lk >= 0 && v == 0.0) {
        double ph = phase_of(P, lk, t);
        int red = decide(d, ph < P->red[lk], phase_fragile(P, lk, ph));
        double R0 = 2.0 * P->ds * a;
        double eR0 = P->fp_band * 2.0 * P->ds * fabs(a);
        if (decide(d, R0 <= 0.0, fabs(R0) <= eR0)) {
            if (Te != 0.0)
                return 0;
            double t_rg = 0.0;
            if (red) { /* a fragile boundary taken as red: the red that has just begun or is about to */
                if (ph < P->red[lk])
                    t_rg = P->red[lk] - ph;
                else if (ph > 0.5 * (P->red[lk] + P->cycle[lk]))
                    t_rg = P->red[lk] + (P->cycle[lk] - ph);
            }
            o->v1 = 0.0;
            o->xi1 = xi;
            o->t1 = t + t_rg;
            o->dt = 0.0;
            o->wait = t_rg;
            o->fuel_rate = 0.0;
            o->cost = (1.0 - P->gamma) * t_rg;
            return 1;
        }
        if (red)
            return 0;
    }

    /* waiting for green when standing at a light node */
    double wait = 0.0;
    if (P->light_model != 2 && lk >= 0 && v == 0.0) {
        double ph = phase_of(P, lk, t);
        int red = ph < P->red[lk];
        if (decide(d, red, phase_fragile(P, lk, ph))) {
            if (ph < P->red[lk])
                wait = P->red[lk] - ph;
            else if (ph > 0.5 * (P->red[lk] + P->cycle[lk]))
                wait = P->red[lk] + (P->cycle[lk] - ph); /* red is about to start */
            else
                wait = 0.0; /* green has just started */
        }
    }

    /* Eq. (5a) and Eq. (2) */
    double R = v * v + 2.0 * P->ds * a;
    double eR = P->fp_band * (v * v + 2.0 * P->ds * fabs(a));
    int next_light = light_at(P, k + 1);
    double v1, dt;
    if (decide(d, R < 0.0, fabs(R) <= eR)) {
        if (next_light >= 0 && v > 0.0) {
            v1 = 0.0;
            dt = 2.0 * P->ds / v;
        } else {
            return 0;
        }
    } else {
        v1 = sqrt(R > 0.0 ? R : 0.0);
        if (v + v1 <= 0.0)
            return 0;
        dt = 2.0 * P->ds / (v + v1);
    }
    double t1 = t + wait + dt;

    /* Eq. (5c), (7c), (8): no arrival at a light node during red unless
     * stopped at the line; evaluated at the continuous arrival time (with the
     * sampled indicator the value function carries the constraint instead). */
    if (P->light_model != 1 && next_light >= 0 && v1 > 0.0) {
        double ph = phase_of(P, next_light, t1);
        if (decide(d, ph < P->red[next_light], phase_fragile(P, next_light, ph)))
            return 0;
    }

    /* powertrain: fuel map and BSG power */
    double mf = 0.0;
    if (Te > 0.0) {
        const double *c = P->fuel_coef;
        mf = P->fuel_scale * (c[0] + c[1] * w + c[2] * Te + c[3] * w * Te + c[4] * w * w + c[5] * Te * Te);
    }
    double Pm = Tm * w;
    double Pb = Pm > 0.0 ? Pm / P->eta_motor : Pm * P->eta_motor;

    /* Eq. (5b): zeroth-order battery; infeasible if the power exceeds what
     * the circuit can deliver (negative discriminant). */
    double disc = P->voc * P->voc - 4.0 * P->r0 * Pb;
    double ed = P->fp_band * (P->voc * P->voc + 4.0 * P->r0 * fabs(Pb));
    if (decide(d, disc < 0.0, fabs(disc) <= ed))
        return 0;
    if (disc < 0.0)
        disc = 0.0;
    double I = (P->voc - sqrt(disc)) / (2.0 * P->r0);
    double dxi = dt * I / P->cap_As;

    o->v1 = v1;
    o->xi1 = xi - dxi;
    o->t1 = t1;
    o->dt = dt;
    o->wait = wait;
    o->fuel_rate = mf;
    /* Eq. (1)/(6): weighted fuel and time; waiting costs time only */
    o->cost = (P->gamma * mf + 1.0 - P->gamma) * dt + (1.0 - P->gamma) * wait;
    return 1;
}

/* ---- interpolation on a stage grid ---------------------------------------- */

/* Locate x on an increasing node array.  Returns 0 when x lies outside the
 * grid by more than SNAP of the end cell.  scale sets the FP32 band. */
static int locate(const double *nodes, int n, double x, double scale, double fp_band,
                  dec_ctx *d, int *i0, double *f)
{
    if (n == 1) {
        if (fabs(x - nodes[0]) <= 1e-12 * (1.0 + fabs(nodes[0]))) {
            *i0 = 0;
            *f = 0.0;
            return 1;
        }
        return 0;
    }
    double lo = nodes[0], hi = nodes[n - 1];
    double h0 = nodes[1] - nodes[0], h1 = nodes[n - 1] - nodes[n - 2];
    double eps = fp_band * (1.0 + fabs(scale));
    double below = (lo - x) / h0, above = (x - hi) / h1;
    if (decide(d, below > SNAP, fabs(below - SNAP) <= eps))
        return 0;
    if (decide(d, above > SNAP, fabs(above - SNAP) <= eps))
        return 0;
    if (x < lo)
        x = lo;
    if (x > hi)
        x = hi;
    int a = 0, b = n - 1; /* invariant nodes[a] <= x, and x < nodes[b] or b = n-1 */
    while (b - a > 1) {
        int m = (a + b) / 2;
        if (nodes[m] <= x)
            a = m;
        else
            b = m;
    }
    int i = a < n - 1 ? a : n - 2;
    double ff = (x - nodes[i]) / (nodes[i + 1] - nodes[i]);
    if (decide(d, ff < SNAP, fabs(ff - SNAP) <= eps))
        ff = 0.0;
    else if (decide(d, ff > 1.0 - SNAP, fabs(ff - (1.0 - SNAP)) <= eps))
        ff = 1.0;
    *i0 = i;
    *f = ff;
    return 1;
}

/* Trilinear interpolation of a stage value array; corners with weight
 * exactly 0 are skipped and any other +inf corner makes the result +inf. */
static double interp3(const orc_problem *P, int stage, const double *V, double v, double xi, double t,
                      const double scale[3], dec_ctx *d)
{
    int nv = P->nv[stage], nx = P->nxi[stage], nt = P->nt[stage];
    const double *vn = P->v_nodes + P->v_off[stage];
    const double *xn = P->xi_nodes + P->xi_off[stage];
    const double *tn = P->t_nodes + P->t_off[stage];
    int iv, ix, it;
    double fv, fx, ft;
    if (!locate(vn, nv, v, scale[0], P->fp_band, d, &iv, &fv))
        return INFINITY;
    if (!locate(xn, nx, xi, scale[1], P->fp_band, d, &ix, &fx))
        return INFINITY;
    if (!locate(tn, nt, t, scale[2], P->fp_band, d, &it, &ft))
        return INFINITY;
    double acc = 0.0;
    for (int a = 0; a < 2; ++a) {
        double wa = a ? fv : 1.0 - fv;
        if (wa == 0.0)
            continue;
        for (int b = 0; b < 2; ++b) {
            double wb = b ? fx : 1.0 - fx;
            if (wb == 0.0)
                continue;
            for (int c = 0; c < 2; ++c) {
                double wc = c ? ft : 1.0 - ft;
                if (wc == 0.0)
                    continue;
                double val = V[((int64_t)(iv + a) * nx + (ix + b)) * nt + (it + c)];
                if (isinf(val))
                    return INFINITY;
                acc += wa * wb * wc * val;
            }
        }
    }
    return acc;
}

/* Terminal cost c_T (Eq. 9a; reading: SoC shortfall and speed deviation). */
double orc_terminal_cost(const orc_problem *P, double v, double xi)
{
    double short_soc = P->soc_ref - xi;
    if (short_soc < 0.0)
        short_soc = 0.0;
    return P->w_soc * short_soc + P->w_v * (v - P->v_ref) * (v - P->v_ref);
}

/* One transition's cost-to-go term c + J_{k+1}(f(x, u)) under a decision
 * mask.  abs_scale: use absolute grid positions for the FP32 bands (states
 * off the grid, as in the rollout) instead of the step's shift. */
static double eval_once(const orc_problem *P, int k, const double *Vnext, double v, double xi, double t,
                        int ie, int im, int b, int abs_scale, dec_ctx *d, orc_trans *tr)
{
    if (!transition(P, k, v, xi, t, P->te[ie], P->tm[im], b, d, tr))
        return INFINITY;
    int s1 = k + 1;
    const double *vn = P->v_nodes + P->v_off[s1];
    const double *xn = P->xi_nodes + P->xi_off[s1];
    const double *tn = P->t_nodes + P->t_off[s1];
    int nv = P->nv[s1], nx = P->nxi[s1], nt = P->nt[s1];
    double hv = nv > 1 ? (vn[nv - 1] - vn[0]) / (nv - 1) : 1.0;
    double hx = nx > 1 ? (xn[nx - 1] - xn[0]) / (nx - 1) : 1.0;
    double ht = nt > 1 ? (tn[nt - 1] - tn[0]) / (nt - 1) : 1.0;
    double scale[3];
    scale[0] = (tr->v1 - vn[0]) / hv;
    if (abs_scale || tr->wait > 0.0) {
        scale[1] = (tr->xi1 - xn[0]) / hx;
        scale[2] = (tr->t1 - tn[0]) / ht;
    } else {
        scale[1] = (tr->xi1 - xi) / hx;
        scale[2] = (tr->t1 - t) / ht;
    }
    double J = interp3(P, s1, Vnext, tr->v1, tr->xi1, tr->t1, scale, d);
    if (isinf(J))
        return INFINITY;
    return tr->cost + J;
}

/* Evaluate a transition in the given mode; *nfrag returns how many fragile
 * decisions the nominal evaluation met. */
static double eval_mode(const orc_problem *P, int k, const double *Vnext, double v, double xi, double t,
                        int ie, int im, int b, int mode, int abs_scale, int *nfrag, orc_trans *tr_nom)
{
    dec_ctx d = {0u, 0};
    orc_trans tr;
    memset(&tr, 0, sizeof tr);
    double F0 = eval_once(P, k, Vnext, v, xi, t, ie, im, b, abs_scale, &d, &tr);
    if (tr_nom)
        *tr_nom = tr;
    if (nfrag)
        *nfrag = d.nf;
    if (mode == ORC_NOMINAL || d.nf == 0)
        return F0;
    int m = d.nf;
    double lo = F0, hi = F0;
    for (uint32_t mask = 1; mask < (1u << (m < 10 ? m : 10)); ++mask) {
        dec_ctx dd = {mask, 0};
        orc_trans t2;
        double F = eval_once(P, k, Vnext, v, xi, t, ie, im, b, abs_scale, &dd, &t2);
        if (dd.nf > m && dd.nf <= 10)
            m = dd.nf; /* a flipped branch met further fragile decisions */
        if (F < lo)
            lo = F;
        if (F > hi || isinf(F))
            hi = F;
    }
    if (m > 10)
        hi = INFINITY;
    return mode == ORC_LENIENT ? lo : hi;
}

/* ---- public entry points ---------------------------------------------------- */

/* One model step, for unit tests: out = {v1, xi1, t1, dt, wait, fuel_rate,
 * cost}; returns 1 if feasible (nominal decisions). */
int orc_model_step(const orc_problem *P, int k, double v, double xi, double t, double Te, double Tm,
                   int b, double *out)
{
    orc_trans tr;
    memset(&tr, 0, sizeof tr);
    int ok = transition(P, k, v, xi, t, Te, Tm, b, NULL, &tr);
    out[0] = tr.v1;
    out[1] = tr.xi1;
    out[2] = tr.t1;
    out[3] = tr.dt;
    out[4] = tr.wait;
    out[5] = tr.fuel_rate;
    out[6] = tr.cost;
    return ok;
}

/* One transition's value c + J_{k+1}(f(x, u)) in a mode (the quantity the
 * backward step minimises, Eq. 9b), for tests of the fragile-decision
 * bookkeeping; *nfrag receives the number of fragile decisions met by the
 * nominal evaluation (may be NULL). */
double orc_eval(const orc_problem *P, int k, int mode, const double *Vnext, double v, double xi, double t,
                int ie, int im, int b, int32_t *nfrag)
{
    int nf = 0;
    double F = eval_mode(P, k, Vnext, v, xi, t, ie, im, b, mode, 0, &nf, NULL);
    if (nfrag)
        *nfrag = nf;
    return F;
}

/* Interpolate a stage value array at a point (nominal decisions). */
double orc_interp(const orc_problem *P, int stage, const double *V, double v, double xi, double t)
{
    double scale[3] = {0.0, 0.0, 0.0};
    return interp3(P, stage, V, v, xi, t, scale, NULL);
}

/* Terminal values J_N = c_T on the last stage grid (Eq. 9a). */
int orc_terminal(const orc_problem *P, double *VN)
{
    int s = P->n_stages;
    const double *vn = P->v_nodes + P->v_off[s];
    const double *xn = P->xi_nodes + P->xi_off[s];
    int nv = P->nv[s], nx = P->nxi[s], nt = P->nt[s];
    for (int i = 0; i < nv; ++i)
        for (int j = 0; j < nx; ++j)
            for (int l = 0; l < nt; ++l)
                VN[((int64_t)i * nx + j) * nt + l] = orc_terminal_cost(P, vn[i], xn[j]);
    return ORC_OK;
}

/* One backward step of Eq. (9b)-(9d) at stage k.
 *   Vnext: J_{k+1} on the stage-(k+1) grid.
 *   idx:   NULL for every state of stage k (outputs hold nv*nxi*nt entries,
 *          t fastest), or n_idx flat state indices (outputs hold n_idx).
 *   Vout:  J_k (mode-dependent, +inf when infeasible).
 *   pi:    argmin control u = (ie * n_tm + im) * n_b + b, lowest u on ties,
 *          -1 when infeasible (may be NULL).
 *   second: the second-smallest transition value over distinct controls
 *          (may be NULL).
 *   nfrag: number of controls whose evaluation met a fragile decision (may
 *          be NULL).
 */
int orc_stage(const orc_problem *P, int k, int mode, const double *Vnext, int64_t n_idx, const int64_t *idx,
              double *Vout, int32_t *pi, double *second, int32_t *nfrag, int nthreads)
{
    if (k < 0 || k >= P->n_stages || !Vnext || !Vout)
        return ORC_ERR_ARG;
    int nv = P->nv[k], nx = P->nxi[k], nt = P->nt[k];
    const double *vn = P->v_nodes + P->v_off[k];
    const double *xn = P->xi_nodes + P->xi_off[k];
    const double *tn = P->t_nodes + P->t_off[k];
    int64_t total = idx ? n_idx : (int64_t)nv * nx * nt;
#ifdef _OPENMP
    if (nthreads > 0)
        omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 64)
#endif
    for (int64_t q = 0; q < total; ++q) {
        int64_t s = idx ? idx[q] : q;
        int i = (int)(s / ((int64_t)nx * nt));
        int j = (int)((s / nt) % nx);
        int l = (int)(s % nt);
        double v = vn[i], xi = xn[j], t = tn[l];
        double best = INFINITY, sec = INFINITY;
        int32_t bu = -1, nf_total = 0;
        /* Fig. 5: engine torque, motor torque, brake flag innermost */
        for (int ie = 0; ie < P->n_te; ++ie)
            for (int im = 0; im < P->n_tm; ++im)
                for (int b = 0; b < P->n_b; ++b) {
                    int nf = 0;
                    double F = eval_mode(P, k, Vnext, v, xi, t, ie, im, b, mode, 0, &nf, NULL);
                    nf_total += nf > 0;
                    if (F < best) {
                        sec = best;
                        best = F;
                        bu = (ie * P->n_tm + im) * P->n_b + b;
                    } else if (F < sec) {
                        sec = F;
                    }
                }
        /* sampled green indicator (variant): a state moving through a light
         * node at a red time node is infeasible; a time node within the phase
         * band of a boundary is fragile (green when lenient, red when strict) */
        int lk = P->light_model == 1 ? light_at(P, k) : -1;
        if (lk >= 0 && v > 0.0) {
            double ph = phase_of(P, lk, t);
            int red = ph < P->red[lk];
            if (phase_fragile(P, lk, ph) && mode != ORC_NOMINAL) {
                red = mode == ORC_STRICT;
                nf_total += 1;
            }
            if (red) {
                best = INFINITY;
                sec = INFINITY;
            }
        }
        Vout[q] = best;
        if (pi)
            pi[q] = isinf(best) ? -1 : bu;
        if (second)
            second[q] = sec;
        if (nfrag)
            nfrag[q] = nf_total;
    }
    return ORC_OK;
}

/* Full backward sweep in one mode: Vall holds J_0..J_N back to back (stage
 * k at orc_value_offset(k)), piall holds pi_0..pi_{N-1} with the same
 * offsets (may be NULL), secall likewise (may be NULL). */
int orc_solve(const orc_problem *P, int mode, double *Vall, int32_t *piall, double *secall, int nthreads)
{
    int N = P->n_stages;
    orc_terminal(P, Vall + value_offset(P, N));
    for (int k = N - 1; k >= 0; --k) {
        int64_t o = value_offset(P, k);
        int rc = orc_stage(P, k, mode, Vall + value_offset(P, k + 1), 0, NULL, Vall + o,
                           piall ? piall + o : NULL, secall ? secall + o : NULL, NULL, nthreads);
        if (rc)
            return rc;
    }
    return ORC_OK;
}

/* Forward rollout from x0 through J_1..J_N (Vall as in orc_solve): at every
 * stage re-minimise c + J_{k+1}(f(x, u)) over all controls at the continuous
 * state, apply the argmin (lowest u on ties) and accumulate.
 *   traj:  [(N+1) * 3] states (v, soc, t)
 *   u:     [N] controls; step: [N * 5] (dt, wait, fuel_g, cost, gap) where gap
 *          is (second - best) / |best| of that stage's minimisation
 *   totals: fuel_g, time_s, J (sum of stage costs + c_T(x_N))
 * Returns ORC_ERR_INFEASIBLE (and the stage in totals[3]) if no control is
 * feasible somewhere along the way. */
int orc_rollout(const orc_problem *P, const double *Vall, const double *x0, double *traj, int32_t *u,
                double *step, double *totals)
{
    int N = P->n_stages;
    double v = x0[0], xi = x0[1], t = x0[2];
    double fuel = 0.0, J = 0.0;
    traj[0] = v;
    traj[1] = xi;
    traj[2] = t;
    for (int k = 0; k < N; ++k) {
        const double *Vn = Vall + value_offset(P, k + 1);
        double best = INFINITY, sec = INFINITY;
        int bu = -1;
        orc_trans bt;
        memset(&bt, 0, sizeof bt);
        for (int ie = 0; ie < P->n_te; ++ie)
            for (int im = 0; im < P->n_tm; ++im)
                for (int b = 0; b < P->n_b; ++b) {
                    orc_trans tr;
                    double F = eval_mode(P, k, Vn, v, xi, t, ie, im, b, ORC_NOMINAL, 1, NULL, &tr);
                    if (F < best) {
                        sec = best;
                        best = F;
                        bu = (ie * P->n_tm + im) * P->n_b + b;
                        bt = tr;
                    } else if (F < sec) {
                        sec = F;
                    }
                }
        if (bu < 0) {
            totals[0] = fuel;
            totals[1] = t - x0[2];
            totals[2] = INFINITY;
            totals[3] = k;
            return ORC_ERR_INFEASIBLE;
        }
        u[k] = bu;
        double fuel_k = bt.fuel_rate * bt.dt;
        step[k * 5 + 0] = bt.dt;
        step[k * 5 + 1] = bt.wait;
        step[k * 5 + 2] = fuel_k;
        step[k * 5 + 3] = bt.cost;
        step[k * 5 + 4] = isinf(sec) ? INFINITY : (sec - best) / fabs(best);
        fuel += fuel_k;
        J += bt.cost;
        v = bt.v1;
        xi = bt.xi1;
        t = bt.t1;
        traj[(k + 1) * 3 + 0] = v;
        traj[(k + 1) * 3 + 1] = xi;
        traj[(k + 1) * 3 + 2] = t;
    }
    J += orc_terminal_cost(P, v, xi);
    totals[0] = fuel;
    totals[1] = t - x0[2];
    totals[2] = J;
    totals[3] = -1;
    return ORC_OK;
}

/* ---- adjoint: dJ_0(x0)/dtheta by the envelope theorem ------------------------
 * theta = (mass, CdA, Crr, R0, fuel_scale).  With the argmin fixed,
 *   J_k(s) = c(s, u*) + I_{k+1}[J_{k+1}](f(s, u*)),
 * where I_{k+1} is the trilinear interpolant on the stage-(k+1) grid, so
 *   dJ_0(x0) = sum_k sum_s lam_k(s) [dc/dtheta + grad I_{k+1} . df/dtheta],
 *   lam_0 = interpolation weights of x0, lam_{k+1}(n) = sum_s lam_k(s) w_n(f(s, u*)).
 * The derivatives of one step follow Eq. (2), (5a), (5b) and (6) by
 * differentiating through a, v', dt, I and the fuel map. */

typedef struct {
    double dv1[5], dxi1[5], dt1[5], dcost[5];
} orc_dstep;

/* One step with derivatives (nominal decisions).  Returns 1 if feasible. */
static int transition_grad(const orc_problem *P, int k, double v, double xi, double t, double Te, double Tm, int b,
                           orc_trans *o, orc_dstep *g)
{
    if (!transition(P, k, v, xi, t, Te, Tm, b, NULL, o))
        return 0;
    memset(g, 0, sizeof *g);
    const double M = P->mass;
    double p = P->grade[k];
    double sq = sqrt(1.0 + p * p);
    double cos_th = 1.0 / sq;
    double ratio = P->gear / P->r_wheel;
    double da[5] = {0, 0, 0, 0, 0}; /* d a / d theta */
    da[0] = -((Te + Tm) * ratio - 0.5 * P->rho * P->cda * v * v) / (M * M);
    da[1] = -0.5 * P->rho * v * v / M;
    da[2] = -P->g * cos_th;
    double ddt[5] = {0, 0, 0, 0, 0};
    if (o->v1 > 0.0) { /* v' = sqrt(v^2 + 2 ds a), dt = 2 ds / (v + v') */
        for (int q = 0; q < 5; ++q) {
            g->dv1[q] = P->ds * da[q] / o->v1;
            ddt[q] = -o->dt / (v + o->v1) * g->dv1[q];
        }
    } /* stopping at the line: v' = 0 and dt = 2 ds / v do not depend on theta */
    double w = v * ratio;
    double Pm = Tm * w;
    double Pb = Pm > 0.0 ? Pm / P->eta_motor : Pm * P->eta_motor;
    double D = P->voc * P->voc - 4.0 * P->r0 * Pb;
    double sD = sqrt(D > 0.0 ? D : 0.0);
    double I = (P->voc - sD) / (2.0 * P->r0);
    double dI_dR0 = sD > 0.0 ? (2.0 * P->r0 * Pb / sD - (P->voc - sD)) / (2.0 * P->r0 * P->r0) : 0.0;
    double poly = 0.0; /* fuel map without its scale */
    if (Te > 0.0) {
        const double *c = P->fuel_coef;
        poly = c[0] + c[1] * w + c[2] * Te + c[3] * w * Te + c[4] * w * w + c[5] * Te * Te;
    }
    for (int q = 0; q < 5; ++q) {
        double dI = q == 3 ? dI_dR0 : 0.0;
        double dmf = q == 4 ? poly : 0.0;
        g->dt1[q] = ddt[q];
        g->dxi1[q] = -(ddt[q] * I + o->dt * dI) / P->cap_As;
        g->dcost[q] = (P->gamma * o->fuel_rate + 1.0 - P->gamma) * ddt[q] + P->gamma * dmf * o->dt;
    }
    return 1;
}

/* Corners, weights and gradient of the trilinear interpolant at a point of a
 * stage grid (nominal snapping; along a snapped axis the interpolant is flat,
 * so its slope there is 0).  Returns 0 if the point is outside the grid, 2 if
 * a corner entering the value or the gradient is infeasible, 1 otherwise. */
static int interp_grad(const orc_problem *P, int stage, const double *V, double v, double xi, double t,
                       int64_t corner[8], double wgt[8], double grad[3], int *snapped)
{
    const double *nodes[3] = {P->v_nodes + P->v_off[stage], P->xi_nodes + P->xi_off[stage],
                              P->t_nodes + P->t_off[stage]};
    int n[3] = {P->nv[stage], P->nxi[stage], P->nt[stage]};
    double x[3] = {v, xi, t};
    int i0[3];
    double f[3], h[3];
    int snap[3];
    *snapped = 0;
    for (int a = 0; a < 3; ++a) {
        if (!locate(nodes[a], n[a], x[a], 0.0, 0.0, NULL, &i0[a], &f[a]))
            return 0;
        h[a] = n[a] > 1 ? nodes[a][i0[a] + 1] - nodes[a][i0[a]] : 1.0;
        /* recompute the raw fraction to know whether it was snapped */
        double raw = n[a] > 1 ? (fmin(fmax(x[a], nodes[a][0]), nodes[a][n[a] - 1]) - nodes[a][i0[a]]) / h[a] : 0.0;
        snap[a] = (f[a] != raw);
        *snapped |= snap[a];
    }
    int nv_ = n[0], nx = n[1], nt = n[2];
    int bad = 0;
    for (int q = 0; q < 8; ++q) {
        int a = (q >> 2) & 1, b = (q >> 1) & 1, c = q & 1;
        int iv = i0[0] + a, ix = i0[1] + b, it = i0[2] + c;
        if (iv >= nv_)
            iv = nv_ - 1;
        if (ix >= nx)
            ix = nx - 1;
        if (it >= nt)
            it = nt - 1;
        corner[q] = ((int64_t)iv * nx + ix) * nt + it;
        wgt[q] = (a ? f[0] : 1.0 - f[0]) * (b ? f[1] : 1.0 - f[1]) * (c ? f[2] : 1.0 - f[2]);
    }
    for (int a = 0; a < 3; ++a) {
        grad[a] = 0.0;
        if (snap[a] || n[a] == 1)
            continue;
        for (int q = 0; q < 8; ++q) {
            int bits[3] = {(q >> 2) & 1, (q >> 1) & 1, q & 1};
            if (!bits[a])
                continue;
            int lo = q & ~(1 << (2 - a));
            double wo = 1.0; /* weight of the other two axes */
            for (int o = 0; o < 3; ++o)
                if (o != a)
                    wo *= bits[o] ? f[o] : 1.0 - f[o];
            if (wo == 0.0)
                continue;
            double Vh = V[corner[q]], Vl = V[corner[lo]];
            if (isinf(Vh) || isinf(Vl))
                bad = 1;
            else
                grad[a] += wo * (Vh - Vl) / h[a];
        }
    }
    for (int q = 0; q < 8; ++q)
        if (wgt[q] != 0.0 && isinf(V[corner[q]]))
            bad = 1;
    return bad ? 2 : 1;
}

/* Forward lambda sweep.  Vall, piall as filled by orc_solve (nominal).
 * grad[5] receives dJ_0(x0)/dtheta.  diag[6]: number of (stage, state) pairs
 * on the lambda support, 1 if a snapped fraction was met on the support, 1 if
 * an infeasible corner entered a value or gradient, the smallest relative gap
 * (second - best) / |best| of the policy on the support (needs secall, else
 * NaN), the lambda mass (summed over stages; each stage carries mass 1) on
 * support states whose relative gap is at most 1e-4 (needs secall, else
 * NaN), and the lambda mass on support states whose successor met a snapped
 * fraction.  The two masses bound how much of the gradient rests on
 * decisions that a lower-precision solver may take differently.  support (optional, [total states of stages 0..N-1]) receives the
 * support as 0/1 flags, lam_out (optional, same size) the lambda of every
 * state (0 off the support).  Returns ORC_ERR_INFEASIBLE if the support
 * reaches an infeasible state. */
int orc_adjoint(const orc_problem *P, const double *Vall, const int32_t *piall, const double *secall,
                const double *x0, double *grad, double *diag, uint8_t *support, double *lam_out)
{
    int N = P->n_stages;
    double *lam = calloc((size_t)P->V_off[N + 1], sizeof(double));
    if (!lam)
        return ORC_ERR_OOM;
    for (int q = 0; q < 5; ++q)
        grad[q] = 0.0;
    diag[0] = 0;
    diag[1] = 0;
    diag[2] = 0;
    diag[3] = secall ? INFINITY : NAN;
    diag[4] = secall ? 0.0 : NAN;
    diag[5] = 0.0;
    /* lambda_0: interpolation weights of x0 on the stage-0 grid */
    {
        int64_t cn[8];
        double wg[8], gr[3];
        int sn;
        int rc = interp_grad(P, 0, Vall, x0[0], x0[1], x0[2], cn, wg, gr, &sn);
        if (rc == 0) {
            free(lam);
            return ORC_ERR_INFEASIBLE;
        }
        for (int q = 0; q < 8; ++q)
            if (wg[q] != 0.0)
                lam[cn[q]] += wg[q];
    }
    int status = ORC_OK;
    for (int k = 0; k < N && status == ORC_OK; ++k) {
        int nv = P->nv[k], nx = P->nxi[k], nt = P->nt[k];
        const double *vn = P->v_nodes + P->v_off[k];
        const double *xn = P->xi_nodes + P->xi_off[k];
        const double *tn = P->t_nodes + P->t_off[k];
        int64_t base = P->V_off[k];
        int64_t n_states = (int64_t)nv * nx * nt;
        const double *Vn = Vall + P->V_off[k + 1];
        for (int64_t s = 0; s < n_states; ++s) {
            double L = lam[base + s];
            if (L == 0.0)
                continue;
            diag[0] += 1;
            if (support)
                support[base + s] = 1;
            if (lam_out)
                lam_out[base + s] = L;
            int u = piall[base + s];
            if (u < 0) {
                status = ORC_ERR_INFEASIBLE;
                break;
            }
            if (secall) {
                double best = Vall[base + s];
                double gap = (secall[base + s] - best) / fabs(best);
                if (gap < diag[3])
                    diag[3] = gap;
                if (!(gap > 1e-4))
                    diag[4] += L;
            }
            int i = (int)(s / ((int64_t)nx * nt)), j = (int)((s / nt) % nx), l = (int)(s % nt);
            int bb = u % P->n_b, im = (u / P->n_b) % P->n_tm, ie = u / (P->n_b * P->n_tm);
            orc_trans tr;
            orc_dstep dg;
            if (!transition_grad(P, k, vn[i], xn[j], tn[l], P->te[ie], P->tm[im], bb, &tr, &dg)) {
                status = ORC_ERR_INFEASIBLE;
                break;
            }
            int64_t cn[8];
            double wg[8], gr[3];
            int sn;
            int rc = interp_grad(P, k + 1, Vn, tr.v1, tr.xi1, tr.t1, cn, wg, gr, &sn);
            if (rc == 0) {
                status = ORC_ERR_INFEASIBLE;
                break;
            }
            if (rc == 2)
                diag[2] = 1;
            if (sn) {
                diag[1] = 1;
                diag[5] += L;
            }
            for (int q = 0; q < 5; ++q)
                grad[q] += L * (dg.dcost[q] + gr[0] * dg.dv1[q] + gr[1] * dg.dxi1[q] + gr[2] * dg.dt1[q]);
            for (int q = 0; q < 8; ++q)
                if (wg[q] != 0.0)
                    lam[P->V_off[k + 1] + cn[q]] += L * wg[q];
        }
    }
    free(lam);
    return status;
}

/* Cost of a given control sequence from x0 (exact model, no grid): the
 * brute-force pin enumerates sequences with this.  Returns +inf if any step
 * is infeasible or leaves the state box [lo, hi] of the given stage grid. */
double orc_sequence_cost(const orc_problem *P, const double *x0, const int32_t *useq, double *xN)
{
    double v = x0[0], xi = x0[1], t = x0[2], J = 0.0;
    for (int k = 0; k < P->n_stages; ++k) {
        int u = useq[k];
        int b = u % P->n_b;
        int im = (u / P->n_b) % P->n_tm;
        int ie = u / (P->n_b * P->n_tm);
        orc_trans tr;
        if (!transition(P, k, v, xi, t, P->te[ie], P->tm[im], b, NULL, &tr))
            return INFINITY;
        int s1 = k + 1;
        const double *vn = P->v_nodes + P->v_off[s1];
        const double *xn = P->xi_nodes + P->xi_off[s1];
        const double *tn = P->t_nodes + P->t_off[s1];
        if (tr.v1 < vn[0] || tr.v1 > vn[P->nv[s1] - 1] || tr.xi1 < xn[0] || tr.xi1 > xn[P->nxi[s1] - 1] ||
            tr.t1 < tn[0] || tr.t1 > tn[P->nt[s1] - 1])
            return INFINITY;
        /* a path through a light node must meet it green, whichever way the
         * DP enforces it (continuous arrival check or sampled indicator) */
        int lj = light_at(P, s1);
        if (P->light_model == 1 && lj >= 0 && tr.v1 > 0.0 && orc_is_red(P, lj, tr.t1))
            return INFINITY;
        J += tr.cost;
        v = tr.v1;
        xi = tr.xi1;
        t = tr.t1;
    }
    if (xN) {
        xN[0] = v;
        xN[1] = xi;
        xN[2] = t;
    }
    return J + orc_terminal_cost(P, v, xi);
}
