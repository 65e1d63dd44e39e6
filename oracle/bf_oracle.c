/*
 * bf_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the
 * generalized Bellman-Ford method of symbolic optimal control
 * (Weber, Kreuzer, Knoll: "A generalized Bellman-Ford Algorithm for
 * Application in Symbolic Optimal Control", arXiv 2001.06231).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header, table or helper with
 * the CUDA library; it is written directly from the paper.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (no -ffast-math, no FMA
 * contraction), so every floating-point expression below is evaluated
 * exactly in the order it is written, with IEEE round-to-nearest.
 *
 * Contents
 *   orc_build_boxes   discrete abstraction of a sampled system (Sec. V-B):
 *                     a uniform cover of hyper-rectangles, a box
 *                     over-approximation of the attainable set per
 *                     (cell, input), quantised to integer cell ranges.
 *   orc_pred_build    the predecessor map pred(x,u) of Eq. (pred), exact,
 *                     as CSR lists (union over the inputs).
 *   orc_solve         Algorithm 1 (generalized Bellman-Ford-Yen) with
 *                     synchronous (Jacobi) rounds.
 *   orc_dijkstra      the generalized (min-max) Dijkstra algorithm that
 *                     Sec. IV cites for non-negative costs.
 *   orc_bellman_check the dynamic-programming operator P of
 *                     Eq. (dynamicprogramming) applied to a candidate V.
 *
 * Problem encoding (shared by every function)
 *   grid     D <= 4 dimensions, n[d] cells each, cell index
 *            c = i0 + n0*(i1 + n1*(i2 + n2*i3)); periodic[d] != 0 wraps.
 *   boxes    int16 [C][U][2][D]: lo[0..D-1], hi[0..D-1].  The successor set
 *            F(x,u) is every cell y with lo_d <= y_d <= hi_d in each dim
 *            (on a periodic dim, hi may exceed n-1 and indexes wrap).
 *            lo[0] == -32768 marks a box that leaves the grid: its successor
 *            is the overflow set, whose value is +inf (Sec. V-B cover).
 *   G        double [C][U]: the running cost g(x,y,u) = G(x,u) of Eq. (cost)
 *            for every successor y outside the successor class (below).
 *   cls, Gc  optional uint8 [C] and double [C][U]: a successor class R (the
 *            cells with cls[y] != 0) with its own running cost,
 *            g(x,y,u) = Gc(x,u) for y in R -- the form of g2 in Sec. VI-A
 *            (a reward -5 tau for successors over the fire, g1 elsewhere).
 *            NULL: g does not depend on y.
 *   terminal double [C]: the terminal cost G(x) of Eq. (cost).
 *   avoid    uint8 [C] or NULL: an avoid cell x is read as g(x,.,.) = +inf
 *            and g(.,x,.) = +inf with terminal +inf, so it keeps V = +inf.
 *   -0.0 in G or terminal is read as +0.0; NaN, -inf and finite values of
 *   magnitude above 2^64 are rejected (so no sum over at most |X| rounds can
 *   overflow).
 *
 * parity note: every function here is pinned by the CPU tests (worked
 * example of Fig. 2, brute force over memoryless controllers, min-max
 * Dijkstra, closed forms on 1-D chains, closed-form flows).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_BLOCKED (-32768)
#define ORC_HANDOVER 0xFF

enum { ORC_CONVERGED = 0, ORC_NEG_CYCLE = 1, ORC_ITER_CAP = 2 };
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2 };
enum { ORC_LINEAR2D = 1, ORC_UNICYCLE3D = 2, ORC_FIRE4D = 3 };

/* ------------------------------------------------------------------------ */
/* grid helpers                                                             */
/* ------------------------------------------------------------------------ */

static int64_t n_cells(int D, const int32_t *n)
{
    int64_t c = 1;
    for (int d = 0; d < D; ++d) c *= n[d];
    return c;
}

static void cell_coords(int D, const int32_t *n, int64_t c, int64_t *k)
{
    for (int d = 0; d < D; ++d) { k[d] = c % n[d]; c /= n[d]; }
}

static int64_t cell_index(int D, const int32_t *n, const int64_t *k)
{
    int64_t c = 0;
    for (int d = D - 1; d >= 0; --d) c = c * n[d] + k[d];
    return c;
}

/* Enumerate the cells of one box.  Calls back with the cell index.
 * Returns the number of cells (0 for a blocked box). */
typedef void (*cell_fn)(int64_t y, void *ctx);

static int64_t for_box(int D, const int32_t *n, const uint8_t *periodic,
                       const int16_t *box, cell_fn fn, void *ctx)
{
    if (box[0] == ORC_BLOCKED) return 0;
    int64_t lo[4], len[4], k[4], cnt = 1;
    for (int d = 0; d < D; ++d) {
        lo[d] = box[d];
        len[d] = (int64_t)box[D + d] - box[d] + 1;
        k[d] = 0;
        cnt *= len[d];
    }
    for (int64_t t = 0; t < cnt; ++t) {
        int64_t y[4];
        for (int d = 0; d < D; ++d) {
            int64_t v = lo[d] + k[d];
            if (periodic[d] && v >= n[d]) v -= n[d];
            y[d] = v;
        }
        fn(cell_index(D, n, y), ctx);
        for (int d = 0; d < D; ++d) {           /* odometer increment */
            if (++k[d] < len[d]) break;
            k[d] = 0;
        }
    }
    return cnt;
}

/* Validate boxes against the grid. Returns ORC_OK or ORC_EINVAL. */
static int check_boxes(int D, const int32_t *n, const uint8_t *periodic,
                       int64_t C, int U, const int16_t *boxes)
{
    for (int64_t p = 0; p < C * U; ++p) {
        const int16_t *b = boxes + p * 2 * D;
        if (b[0] == ORC_BLOCKED) continue;
        for (int d = 0; d < D; ++d) {
            int lo = b[d], hi = b[D + d];
            if (lo < 0 || lo >= n[d] || hi < lo) return ORC_EINVAL;
            if (periodic[d]) { if (hi - lo + 1 > n[d]) return ORC_EINVAL; }
            else if (hi >= n[d]) return ORC_EINVAL;
        }
    }
    return ORC_OK;
}

/* -0.0 -> +0.0; reject NaN and -inf.  Returns ORC_OK or ORC_EINVAL. */
static int clean_value(double v, double *out)
{
    if (isnan(v)) return ORC_EINVAL;
    if (isinf(v) && v < 0) return ORC_EINVAL;
    if (!isinf(v) && fabs(v) > 0x1p64) return ORC_EINVAL;   /* |finite| <= 2^64 */
    *out = (v == 0.0) ? 0.0 : v;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* orc_build_boxes: discrete abstraction of a sampled system (Sec. V)       */
/* ------------------------------------------------------------------------ */
/*
 * kind LINEAR2D (double integrator x0' = x1, x1' = u0).  The flow is linear,
 *   phi(tau,x,u) = (x0 + tau*x1 + tau^2/2*u0, x1 + tau*u0), so the image of a
 *   cell is the convex hull of the images of its 4 corners and the bounding
 *   box of those images is the exact hull in each coordinate.
 * kind UNICYCLE3D (x' = v cos th, y' = v sin th, th' = w; u = (v, w)).
 * kind FIRE4D (x' = V cos psi + wind, y' = V sin psi,
 *   psi' = (g/V) tan(phi), V' = a; u = (phi, a)).
 *   For these two the attainable set of a cell c +- eta/2 is
 *   over-approximated (Sec. V-B, box over-approximation of attainable sets)
 *   by the growth-bound box  phi(tau,c,u) +- r(tau), where r solves
 *   r' = L r + w, r(0) = eta/2, L the componentwise bound on the Jacobian
 *   (|d f_i / d x_j| off the diagonal) and w the disturbance bound.  Both
 *   ODEs are integrated with the classical 4th-order Runge-Kutta scheme over
 *   `substeps` equal steps.
 *
 * params
 *   UNICYCLE3D: param[0] = disturbance bound w (added to every component).
 *   FIRE4D:     param[0] = wind (added to x'), param[1] = gravity g,
 *               param[2] = V_lo, param[3] = V_hi (Jacobian bounds),
 *               param[4] = disturbance bound w.
 *
 * Quantisation (the cells meeting the over-approximation, half-open cells):
 *   eta_d = (ghi_d - glo_d) / n_d
 *   lo = floor((a - glo_d) / eta_d),  hi = floor((b - glo_d) / eta_d)
 *   non-periodic dim leaving [0, n-1] -> blocked (overflow set);
 *   periodic dim: a box of n or more cells is the full circle [0, n-1],
 *   otherwise lo is reduced mod n and hi = lo + (length - 1).
 */

static void rhs(int kind, const double *p, const double *x, const double *u,
                double *dx)
{
    if (kind == ORC_UNICYCLE3D) {
        dx[0] = u[0] * cos(x[2]);
        dx[1] = u[0] * sin(x[2]);
        dx[2] = u[1];
    } else { /* ORC_FIRE4D */
        dx[0] = x[3] * cos(x[2]) + p[0];
        dx[1] = x[3] * sin(x[2]);
        dx[2] = (p[1] / x[3]) * tan(u[0]);
        dx[3] = u[1];
    }
}

/* L (row-major DxD) and w (D) of the growth bound r' = L r + w. */
static void growth_matrix(int kind, const double *p, const double *u,
                          double *L, double *w)
{
    memset(L, 0, sizeof(double) * 16);
    if (kind == ORC_UNICYCLE3D) {
        /* |d(v cos th)/d th| <= |v|, |d(v sin th)/d th| <= |v| */
        double v = fabs(u[0]);
        L[0 * 3 + 2] = v;
        L[1 * 3 + 2] = v;
        w[0] = p[0]; w[1] = p[0]; w[2] = p[0];
    } else { /* ORC_FIRE4D, D = 4 */
        double vhi = p[3], vlo = p[2];
        L[0 * 4 + 2] = vhi;  L[0 * 4 + 3] = 1.0;   /* d/dpsi, d/dV of V cos psi */
        L[1 * 4 + 2] = vhi;  L[1 * 4 + 3] = 1.0;   /* same for V sin psi        */
        L[2 * 4 + 3] = (p[1] * tan(fabs(u[0]))) / (vlo * vlo); /* d/dV of (g/V) tan phi */
        w[0] = p[4]; w[1] = p[4]; w[2] = p[4]; w[3] = p[4];
    }
}

static void lin_rhs(int D, const double *L, const double *w, const double *r,
                    double *dr)
{
    for (int i = 0; i < D; ++i) {
        double s = w[i];
        for (int j = 0; j < D; ++j) s = s + L[i * D + j] * r[j];
        dr[i] = s;
    }
}

/* One classical RK4 integration of centre c and radius r over tau. */
static void rk4_flow(int kind, const double *p, int D, const double *u,
                     double tau, int substeps, double *c, double *r)
{
    double L[16], w[4];
    growth_matrix(kind, p, u, L, w);
    double h = tau / (double)substeps;
    double hh = h * 0.5, h6 = h / 6.0;
    for (int s = 0; s < substeps; ++s) {
        double k1[4], k2[4], k3[4], k4[4], t[4];
        double q1[4], q2[4], q3[4], q4[4], tr[4];
        rhs(kind, p, c, u, k1);           lin_rhs(D, L, w, r, q1);
        for (int i = 0; i < D; ++i) { t[i] = c[i] + hh * k1[i]; tr[i] = r[i] + hh * q1[i]; }
        rhs(kind, p, t, u, k2);           lin_rhs(D, L, w, tr, q2);
        for (int i = 0; i < D; ++i) { t[i] = c[i] + hh * k2[i]; tr[i] = r[i] + hh * q2[i]; }
        rhs(kind, p, t, u, k3);           lin_rhs(D, L, w, tr, q3);
        for (int i = 0; i < D; ++i) { t[i] = c[i] + h * k3[i];  tr[i] = r[i] + h * q3[i]; }
        rhs(kind, p, t, u, k4);           lin_rhs(D, L, w, tr, q4);
        for (int i = 0; i < D; ++i) {
            c[i] = c[i] + h6 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
            r[i] = r[i] + h6 * (q1[i] + 2.0 * q2[i] + 2.0 * q3[i] + q4[i]);
        }
    }
}

/* Quantise [a, b] on dim d into [lo, hi]; returns 0 if blocked. */
static int quantise(double a, double b, double glo, double eta, int32_t n,
                    int periodic, int *lo, int *hi)
{
    double fa = floor((a - glo) / eta);
    double fb = floor((b - glo) / eta);
    if (!(fa == fa) || !(fb == fb)) return 0;       /* NaN: treat as blocked */
    if (!periodic) {
        if (fa < 0.0 || fb > (double)(n - 1)) return 0;
        *lo = (int)fa; *hi = (int)fb;
        return 1;
    }
    double len = fb - fa + 1.0;
    if (len >= (double)n) { *lo = 0; *hi = n - 1; return 1; }
    double m = fmod(fa, (double)n);
    if (m < 0.0) m += (double)n;
    *lo = (int)m;
    *hi = (int)m + (int)len - 1;
    return 1;
}

int orc_build_boxes(int kind, const double *param, int substeps,
                    int D, const int32_t *n, const double *glo,
                    const double *ghi, const uint8_t *periodic,
                    int U, int udim, const double *inputs, double tau,
                    int16_t *boxes)
{
    if (kind == ORC_LINEAR2D && D != 2) return ORC_EINVAL;
    if (kind == ORC_UNICYCLE3D && D != 3) return ORC_EINVAL;
    if (kind == ORC_FIRE4D && D != 4) return ORC_EINVAL;
    if (kind < ORC_LINEAR2D || kind > ORC_FIRE4D) return ORC_EINVAL;
    if (udim < 1 || (kind != ORC_LINEAR2D && udim < 2)) return ORC_EINVAL;
    if (substeps < 1 && kind != ORC_LINEAR2D) return ORC_EINVAL;
    for (int d = 0; d < D; ++d)
        if (n[d] < 1 || n[d] > 16383) return ORC_EINVAL;

    int64_t C = n_cells(D, n);
    double eta[4];
    for (int d = 0; d < D; ++d) eta[d] = (ghi[d] - glo[d]) / (double)n[d];

    for (int64_t c = 0; c < C; ++c) {
        int64_t k[4];
        cell_coords(D, n, c, k);
        for (int ui = 0; ui < U; ++ui) {
            const double *u = inputs + (int64_t)ui * udim;
            int16_t *box = boxes + (c * U + ui) * 2 * D;
            double a[4], b[4];
            if (kind == ORC_LINEAR2D) {
                /* images of the 4 corners under the exact flow */
                double tt = 0.5 * tau * tau;
                for (int q = 0; q < 4; ++q) {
                    double x0 = glo[0] + (double)(k[0] + (q & 1)) * eta[0];
                    double x1 = glo[1] + (double)(k[1] + ((q >> 1) & 1)) * eta[1];
                    double y0 = (x0 + tau * x1) + tt * u[0];
                    double y1 = x1 + tau * u[0];
                    if (q == 0 || y0 < a[0]) a[0] = y0;
                    if (q == 0 || y0 > b[0]) b[0] = y0;
                    if (q == 0 || y1 < a[1]) a[1] = y1;
                    if (q == 0 || y1 > b[1]) b[1] = y1;
                }
            } else {
                double cc[4], rr[4];
                for (int d = 0; d < D; ++d) {
                    cc[d] = glo[d] + ((double)k[d] + 0.5) * eta[d];
                    rr[d] = eta[d] * 0.5;
                }
                rk4_flow(kind, param, D, u, tau, substeps, cc, rr);
                for (int d = 0; d < D; ++d) { a[d] = cc[d] - rr[d]; b[d] = cc[d] + rr[d]; }
            }
            int ok = 1, lo[4], hi[4];
            for (int d = 0; d < D && ok; ++d)
                ok = quantise(a[d], b[d], glo[d], eta[d], n[d], periodic[d], &lo[d], &hi[d]);
            if (!ok) {
                box[0] = ORC_BLOCKED;
                for (int d = 1; d < 2 * D; ++d) box[d] = 0;
            } else {
                for (int d = 0; d < D; ++d) { box[d] = (int16_t)lo[d]; box[D + d] = (int16_t)hi[d]; }
            }
        }
    }
    return ORC_OK;
}

/* Centre and radius after one sampling period, for the closed-form tests. */
int orc_flow(int kind, const double *param, int substeps, int D,
             const double *u, double tau, double *c, double *r)
{
    if (kind != ORC_UNICYCLE3D && kind != ORC_FIRE4D) return ORC_EINVAL;
    rk4_flow(kind, param, D, u, tau, substeps, c, r);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* orc_pred_build: pred(y) = { x : exists u, y in F(x,u) }  (Eq. pred)       */
/* ------------------------------------------------------------------------ */

struct pred_ctx {
    int64_t x;        /* current predecessor candidate */
    int64_t *stamp;   /* last x that touched y         */
    int64_t *count;   /* per-y counts / fill cursors   */
    int32_t *list;    /* CSR column array (fill pass)  */
    int fill;
};

static void pred_visit(int64_t y, void *vctx)
{
    struct pred_ctx *p = (struct pred_ctx *)vctx;
    if (p->stamp[y] == p->x) return;     /* x already listed for y */
    p->stamp[y] = p->x;
    if (p->fill) p->list[p->count[y]++] = (int32_t)p->x;
    else p->count[y]++;
}

/* Two passes: count, then fill.  row_ptr has C+1 entries; *col_out is
 * malloc'd (caller frees with orc_free).  Lists come out sorted by x. */
int orc_pred_build(int D, const int32_t *n, const uint8_t *periodic, int U,
                   const int16_t *boxes, int64_t *row_ptr, int32_t **col_out)
{
    int64_t C = n_cells(D, n);
    if (check_boxes(D, n, periodic, C, U, boxes) != ORC_OK) return ORC_EINVAL;
    int64_t *stamp = (int64_t *)malloc(sizeof(int64_t) * C);
    int64_t *cnt = (int64_t *)calloc(C + 1, sizeof(int64_t));
    if (!stamp || !cnt) { free(stamp); free(cnt); return ORC_ENOMEM; }
    struct pred_ctx ctx = { 0, stamp, cnt, NULL, 0 };
    for (int pass = 0; pass < 2; ++pass) {
        for (int64_t y = 0; y < C; ++y) stamp[y] = -1;
        if (pass == 1) {
            int64_t acc = 0;
            for (int64_t y = 0; y < C; ++y) { row_ptr[y] = acc; acc += cnt[y]; }
            row_ptr[C] = acc;
            ctx.list = (int32_t *)malloc(sizeof(int32_t) * (acc > 0 ? acc : 1));
            if (!ctx.list) { free(stamp); free(cnt); return ORC_ENOMEM; }
            for (int64_t y = 0; y < C; ++y) cnt[y] = row_ptr[y];
            ctx.fill = 1;
        }
        for (int64_t x = 0; x < C; ++x) {
            ctx.x = x;
            for (int u = 0; u < U; ++u)
                for_box(D, n, periodic, boxes + (x * U + u) * 2 * D, pred_visit, &ctx);
        }
    }
    *col_out = ctx.list;
    free(stamp);
    free(cnt);
    return ORC_OK;
}

void orc_free(void *p) { free(p); }

/* ------------------------------------------------------------------------ */
/* Algorithm 1: generalized Bellman-Ford-Yen, Jacobi rounds                  */
/* ------------------------------------------------------------------------ */
/*
 * Reading of Algorithm 1 used here (the paper notes that the processing
 * order of F1 is irrelevant): every d of one pass of the while-loop reads W
 * as it stood when the pass began; at the end of the pass, for each x in F1,
 *   W(x) <- min(W(x), min_u d(x,u)),
 *   mu(x) <- the lowest u attaining that minimum, if it is strictly below the
 *            old W(x) (line "if d < W(x)"); otherwise mu(x) is unchanged.
 * d(x,u) = sup_{y in F(x,u)} g(x,y,u) + W(y), computed literally, one sum
 * per successor, as the supremum of Algorithm 1's relaxation line.
 * F2 collects pred(x,.) of every x whose W changed; F1 <- F2; i <- i + 1.
 * The loop runs while F1 is non-empty and i < cap (cap = |X|, the paper's
 * negative-cycle test, or max_iters if smaller).
 */

struct sup_ctx {
    const double *W;
    const uint8_t *avoid;
    const uint8_t *cls;
    double g;      /* g(x,y,u) for y outside the successor class */
    double gc;     /* g(x,y,u) for y in the successor class      */
    double d;
    int any;
};

static void sup_visit(int64_t y, void *vctx)
{
    struct sup_ctx *s = (struct sup_ctx *)vctx;
    double gy = (s->cls && s->cls[y]) ? s->gc : s->g;          /* g(x,y,u) */
    if (s->avoid && s->avoid[y]) gy = INFINITY;
    double v = gy + s->W[y];
    if (!s->any || v > s->d) s->d = v;
    s->any = 1;
}

/* d(x,u) of Algorithm 1, reading W. */
static double relax_value(int D, const int32_t *n, const uint8_t *periodic,
                          int U, const int16_t *boxes, const double *G,
                          const uint8_t *cls, const double *Gc,
                          const uint8_t *avoid, const double *W,
                          int64_t x, int u)
{
    const int16_t *box = boxes + (x * U + u) * 2 * D;
    if (avoid && avoid[x]) return INFINITY;           /* g(x,.,.) = +inf */
    if (box[0] == ORC_BLOCKED) return INFINITY;       /* overflow set    */
    struct sup_ctx s = { W, avoid, cls, G[x * U + u], cls ? Gc[x * U + u] : 0.0, 0.0, 0 };
    for_box(D, n, periodic, box, sup_visit, &s);
    return s.d;
}

int orc_solve(int D, const int32_t *n, const uint8_t *periodic, int U,
              const int16_t *boxes, const double *G_in, const double *terminal,
              const uint8_t *avoid, const uint8_t *cls, const double *Gc_in,
              int64_t max_iters,
              const int64_t *pred_ptr, const int32_t *pred_col,
              double *V, uint8_t *mu, int64_t *iters, int32_t *status,
              int64_t *f1_trace, int64_t *chg_trace, int64_t trace_cap,
              uint8_t *f1_exit)
{
    int64_t C = n_cells(D, n);
    if (C <= 0 || U < 1 || U > 255 || D < 1 || D > 4) return ORC_EINVAL;
    if (check_boxes(D, n, periodic, C, U, boxes) != ORC_OK) return ORC_EINVAL;

    double *G = (double *)malloc(sizeof(double) * C * U);
    double *Gc = cls ? (double *)malloc(sizeof(double) * C * U) : NULL;
    double *Wn = (double *)malloc(sizeof(double) * C);
    uint8_t *inF2 = (uint8_t *)calloc(C, 1);
    int64_t *F1 = (int64_t *)malloc(sizeof(int64_t) * C);
    int64_t *F2 = (int64_t *)malloc(sizeof(int64_t) * C);
    int64_t *chg = (int64_t *)malloc(sizeof(int64_t) * C);
    uint8_t *chmu = (uint8_t *)malloc(C);
    int64_t *own_ptr = NULL;
    int32_t *own_col = NULL;
    int rc = ORC_OK;
    if (!G || !Wn || !inF2 || !F1 || !F2 || !chg || !chmu || (cls && !Gc)) { rc = ORC_ENOMEM; goto done; }
    for (int64_t p = 0; p < C * U; ++p)
        if (clean_value(G_in[p], &G[p]) != ORC_OK) { rc = ORC_EINVAL; goto done; }
    if (cls)
        for (int64_t p = 0; p < C * U; ++p)
            if (clean_value(Gc_in[p], &Gc[p]) != ORC_OK) { rc = ORC_EINVAL; goto done; }
    if (!pred_ptr) {
        own_ptr = (int64_t *)malloc(sizeof(int64_t) * (C + 1));
        if (!own_ptr) { rc = ORC_ENOMEM; goto done; }
        rc = orc_pred_build(D, n, periodic, U, boxes, own_ptr, &own_col);
        if (rc != ORC_OK) goto done;
        pred_ptr = own_ptr;
        pred_col = own_col;
    }

    /* lines 1-9: W = G (terminal), mu = U, F1 = union of pred over finite G */
    int64_t nF1 = 0, nF2 = 0;
    for (int64_t x = 0; x < C; ++x) {
        double t;
        if (clean_value(terminal[x], &t) != ORC_OK) { rc = ORC_EINVAL; goto done; }
        V[x] = (avoid && avoid[x]) ? INFINITY : t;
        mu[x] = ORC_HANDOVER;
    }
    for (int64_t y = 0; y < C; ++y) {
        if (!(V[y] < INFINITY)) continue;
        for (int64_t q = pred_ptr[y]; q < pred_ptr[y + 1]; ++q) {
            int64_t x = pred_col[q];
            if (!inF2[x]) { inF2[x] = 1; F1[nF1++] = x; }
        }
    }
    for (int64_t q = 0; q < nF1; ++q) inF2[F1[q]] = 0;

    int64_t cap = C;
    if (max_iters > 0 && max_iters < cap) cap = max_iters;
    int64_t i = 0;
    /* line 11: while F1 != empty and i < |X| */
    while (nF1 > 0 && i < cap) {
        int64_t nchg = 0;
        /* lines 12-18, synchronous: all d read the W of the round start */
        for (int64_t q = 0; q < nF1; ++q) {
            int64_t x = F1[q];
            double best = V[x];
            int bu = -1;
            for (int u = 0; u < U; ++u) {
                double d = relax_value(D, n, periodic, U, boxes, G, cls, Gc, avoid, V, x, u);
                if (d < best) { best = d; bu = u; }
            }
            if (bu >= 0) { Wn[x] = best; chmu[x] = (uint8_t)bu; chg[nchg++] = x; }
        }
        /* end of pass: commit W, mu; F2 = union of pred(x,.) of changed x */
        for (int64_t q = 0; q < nchg; ++q) {
            int64_t x = chg[q];
            V[x] = Wn[x];
            mu[x] = chmu[x];
        }
        nF2 = 0;
        for (int64_t q = 0; q < nchg; ++q) {
            int64_t y = chg[q];
            for (int64_t r = pred_ptr[y]; r < pred_ptr[y + 1]; ++r) {
                int64_t x = pred_col[r];
                if (!inF2[x]) { inF2[x] = 1; F2[nF2++] = x; }
            }
        }
        if (f1_trace && i < trace_cap) f1_trace[i] = nF1;
        if (chg_trace && i < trace_cap) chg_trace[i] = nchg;
        /* swap frontiers, clear F2 */
        for (int64_t q = 0; q < nF2; ++q) inF2[F2[q]] = 0;
        int64_t *tmp = F1; F1 = F2; F2 = tmp;
        nF1 = nF2;
        i = i + 1;
    }
    *iters = i;
    if (f1_exit) {                                   /* F1 when the loop ends */
        memset(f1_exit, 0, (size_t)C);
        for (int64_t q = 0; q < nF1; ++q) f1_exit[F1[q]] = 1;
    }
    if (nF1 == 0) *status = ORC_CONVERGED;
    else if (i >= C) *status = ORC_NEG_CYCLE;
    else *status = ORC_ITER_CAP;

done:
    free(G); free(Gc); free(Wn); free(inF2); free(F1); free(F2); free(chg); free(chmu);
    free(own_ptr); free(own_col);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* generalized min-max Dijkstra (costs >= 0), used only as a cross-check     */
/* ------------------------------------------------------------------------ */
/*
 * Settles cells in increasing W.  Each pair (x,u) counts its successors not
 * yet settled; when the last one, y, is settled, every successor value is
 * final and y holds the largest, so d(x,u) = G(x,u) + W(y).  Valid when
 * G >= 0 and the terminal cost is >= 0 (Sec. IV, generalized Dijkstra).
 */

struct heap { int64_t *cell; double *key; int64_t n, cap; };

static int heap_push(struct heap *h, int64_t c, double k)
{
    if (h->n == h->cap) {
        int64_t nc = h->cap ? 2 * h->cap : 1024;
        int64_t *a = (int64_t *)realloc(h->cell, sizeof(int64_t) * nc);
        if (!a) return ORC_ENOMEM;
        h->cell = a;
        double *b = (double *)realloc(h->key, sizeof(double) * nc);
        if (!b) return ORC_ENOMEM;
        h->key = b;
        h->cap = nc;
    }
    int64_t i = h->n++;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!(k < h->key[p])) break;
        h->cell[i] = h->cell[p]; h->key[i] = h->key[p];
        i = p;
    }
    h->cell[i] = c; h->key[i] = k;
    return ORC_OK;
}

static void heap_pop(struct heap *h, int64_t *c, double *k)
{
    *c = h->cell[0]; *k = h->key[0];
    int64_t last = --h->n;
    int64_t lc = h->cell[last];
    double lk = h->key[last];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        double mk = lk;
        if (l < h->n && h->key[l] < mk) { m = l; mk = h->key[l]; }
        if (r < h->n && h->key[r] < mk) { m = r; }
        if (m == i) break;
        h->cell[i] = h->cell[m]; h->key[i] = h->key[m];
        i = m;
    }
    if (h->n > 0) { h->cell[i] = lc; h->key[i] = lk; }
}

struct pp_ctx { int64_t pair; int64_t *cnt; int64_t *ptr; int64_t *list; int fill; };

static void pp_visit(int64_t y, void *vctx)
{
    struct pp_ctx *p = (struct pp_ctx *)vctx;
    if (p->fill) p->list[p->ptr[y]++] = p->pair;
    else p->cnt[y]++;
}

int orc_dijkstra(int D, const int32_t *n, const uint8_t *periodic, int U,
                 const int16_t *boxes, const double *G_in,
                 const double *terminal, const uint8_t *avoid,
                 double *V, uint8_t *mu)
{
    int64_t C = n_cells(D, n);
    if (check_boxes(D, n, periodic, C, U, boxes) != ORC_OK) return ORC_EINVAL;
    int rc = ORC_OK;
    int64_t *remain = (int64_t *)malloc(sizeof(int64_t) * C * U);
    int64_t *cnt = (int64_t *)calloc(C + 1, sizeof(int64_t));
    int64_t *ptr = (int64_t *)malloc(sizeof(int64_t) * (C + 1));
    uint8_t *done = (uint8_t *)calloc(C, 1);
    double *G = (double *)malloc(sizeof(double) * C * U);
    int64_t *list = NULL;
    struct heap h = { NULL, NULL, 0, 0 };
    if (!remain || !cnt || !ptr || !done || !G) { rc = ORC_ENOMEM; goto out; }
    for (int64_t p = 0; p < C * U; ++p) {
        if (clean_value(G_in[p], &G[p]) != ORC_OK || G[p] < 0) { rc = ORC_EINVAL; goto out; }
    }
    /* predecessor pairs per successor cell */
    struct pp_ctx pc = { 0, cnt, ptr, NULL, 0 };
    for (int64_t p = 0; p < C * U; ++p) {
        pc.pair = p;
        remain[p] = for_box(D, n, periodic, boxes + p * 2 * D, pp_visit, &pc);
        if (boxes[p * 2 * D] == ORC_BLOCKED) remain[p] = -1;   /* never fires */
    }
    int64_t acc = 0;
    for (int64_t y = 0; y < C; ++y) { ptr[y] = acc; acc += cnt[y]; }
    ptr[C] = acc;
    list = (int64_t *)malloc(sizeof(int64_t) * (acc > 0 ? acc : 1));
    if (!list) { rc = ORC_ENOMEM; goto out; }
    pc.list = list; pc.fill = 1;
    for (int64_t p = 0; p < C * U; ++p) {
        pc.pair = p;
        for_box(D, n, periodic, boxes + p * 2 * D, pp_visit, &pc);
    }
    for (int64_t y = C; y > 0; --y) ptr[y] = ptr[y - 1];
    ptr[0] = 0;

    for (int64_t x = 0; x < C; ++x) {
        double t;
        if (clean_value(terminal[x], &t) != ORC_OK || t < 0) { rc = ORC_EINVAL; goto out; }
        V[x] = (avoid && avoid[x]) ? INFINITY : t;
        mu[x] = ORC_HANDOVER;
        if (V[x] < INFINITY && heap_push(&h, x, V[x]) != ORC_OK) { rc = ORC_ENOMEM; goto out; }
    }
    while (h.n > 0) {
        int64_t y; double k;
        heap_pop(&h, &y, &k);
        if (done[y] || k != V[y]) continue;      /* stale entry */
        done[y] = 1;
        for (int64_t q = ptr[y]; q < ptr[y + 1]; ++q) {
            int64_t p = list[q];
            int64_t x = p / U;
            int u = (int)(p % U);
            if (--remain[p] != 0) continue;
            if (done[x] || (avoid && avoid[x])) continue;
            double d = G[p] + V[y];
            if (d < V[x]) {
                V[x] = d;
                mu[x] = (uint8_t)u;
                if (heap_push(&h, x, d) != ORC_OK) { rc = ORC_ENOMEM; goto out; }
            }
        }
    }
out:
    free(remain); free(cnt); free(ptr); free(done); free(G); free(list);
    free(h.cell); free(h.key);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Bellman check: P(V) = V (Eq. dynamicprogramming) and mu attains V         */
/* ------------------------------------------------------------------------ */
/*
 * For each listed cell x (all cells if cells == NULL):
 *   avoid x:        V(x) must be +inf;
 *   otherwise       V(x) == min(T(x), min_u d(x,u)) with d from V itself;
 *   mu(x) == U  ->  V(x) == T(x);
 *   mu(x) == u  ->  d(x,u) == V(x) < T(x).
 * Returns the number of violating cells in *nbad (first one in *first_bad).
 */
int orc_bellman_check(int D, const int32_t *n, const uint8_t *periodic, int U,
                      const int16_t *boxes, const double *G_in,
                      const double *terminal, const uint8_t *avoid,
                      const uint8_t *cls, const double *Gc_in,
                      const double *V, const uint8_t *mu,
                      const int64_t *cells, int64_t ncells,
                      int64_t *nbad, int64_t *first_bad)
{
    int64_t C = n_cells(D, n);
    if (check_boxes(D, n, periodic, C, U, boxes) != ORC_OK) return ORC_EINVAL;
    int64_t m = cells ? ncells : C;
    int64_t bad = 0;
    *first_bad = -1;
    double *Gx = (double *)malloc(sizeof(double) * 2 * U);
    if (!Gx) return ORC_ENOMEM;
    double *Gcx = Gx + U;
    for (int64_t q = 0; q < m; ++q) {
        int64_t x = cells ? cells[q] : q;
        int ok = 1;
        double t;
        if (clean_value(terminal[x], &t) != ORC_OK) { free(Gx); return ORC_EINVAL; }
        for (int u = 0; u < U; ++u) {
            if (clean_value(G_in[x * U + u], &Gx[u]) != ORC_OK) { free(Gx); return ORC_EINVAL; }
            Gcx[u] = 0.0;
            if (cls && clean_value(Gc_in[x * U + u], &Gcx[u]) != ORC_OK) { free(Gx); return ORC_EINVAL; }
        }
        if (avoid && avoid[x]) {
            ok = (V[x] == INFINITY) && mu[x] == ORC_HANDOVER;
        } else {
            double best = t;
            double dmu = INFINITY;
            for (int u = 0; u < U; ++u) {
                /* d(x,u) with the cleaned G(x,u) */
                const int16_t *box = boxes + (x * U + u) * 2 * D;
                double d = INFINITY;
                if (box[0] != ORC_BLOCKED) {
                    struct sup_ctx s = { V, avoid, cls, Gx[u], Gcx[u], 0.0, 0 };
                    for_box(D, n, periodic, box, sup_visit, &s);
                    d = s.d;
                }
                if (d < best) best = d;
                if (mu[x] == u) dmu = d;
            }
            if (!(best == V[x])) ok = 0;
            if (mu[x] == ORC_HANDOVER) { if (!(V[x] == t)) ok = 0; }
            else if (mu[x] >= U || !(dmu == V[x]) || !(V[x] < t)) ok = 0;
        }
        if (!ok) { if (bad == 0) *first_bad = x; ++bad; }
    }
    free(Gx);
    *nbad = bad;
    return ORC_OK;
}
