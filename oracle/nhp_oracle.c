/*
 * nhp_oracle.c -- TEST INFRASTRUCTURE ONLY (see nhp_oracle.h).
 *
 * A plain restatement of the paper's graph and its kernel-style processing,
 * written for a reader who checks it against the paper by eye:
 *   - geometry tables               Section V.C, eqs. 11-24
 *   - maneuver edges                Section V.D, eqs. 25-28, 30-31
 *   - obstacle rendering            Section VI (walls: Section V.C)
 *   - Star transition subgraph      Section V.A, Fig. 9, Table 1 (7 vertices,
 *                                   18 edges per cell)
 *   - maneuver-kernel relaxation    Section VIII.B, Insert 1 (two loops for
 *                                   turns, one for straights)
 *   - cycle order                   Section XVI.A
 *   - Dijkstra                      Section VIII.A
 *   - forward-tracking labels       Section X
 *   - soft obstacle image           Section VII
 * Readings where the paper is silent are stated where they are used.
 */
#include "nhp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define ORC_INF 0xFFFFFFFFu
#define ORC_HARD 0xFFFFu
#define ORC_NONE 0xFFFFu
#define ORC_PI 3.14159265358979323846

enum { LF = 0, SF = 1, RB = 2, RF = 3, SB = 4, LB = 5 };

struct orc_ctx {
    int lx, lt, nx, nt, mx, mt;
    int64_t nr;
    double R;
    int half;
    uint32_t step_s, step_a, ct;
    uint32_t cin[6], cout[6]; /* Star transition edges T->M_mu and M_mu->T (Fig. 9) */
    int32_t* beta;  /* beta(T), eq. 13 context */
    uint8_t* psi2;  /* 2*Psi(T), eq. 13 */
    uint8_t* iflag; /* I(T), eq. 19 */
    int8_t* jsign;  /* J(T), eq. 24 */
    int32_t* bsh;   /* B(y',T), eq. 22, stored [T*nx + y'] */
    uint32_t* wS;   /* straight step weight per heading */
    uint32_t wA;    /* turn step weight */
};

/* saturating uint32 addition: INF absorbs */
static uint32_t sadd(uint32_t a, uint32_t b) {
    uint64_t s = (uint64_t)a + (uint64_t)b;
    return s >= ORC_INF ? ORC_INF : (uint32_t)s;
}

static int64_t floor_half(int64_t z) { return z >= 0 ? z / 2 : -((-z + 1) / 2); }

static double heading(int T, int nt) { return (2.0 * ORC_PI) * (double)T / (double)nt; }

orc_ctx* orc_create(int nx_log2, int nt_log2, double R, int half_shift,
                    uint32_t step_straight, uint32_t step_scale, uint32_t ct) {
    if (nx_log2 < 2 || nx_log2 > 12 || nt_log2 < 2 || nt_log2 > 12 || !(R > 0)) return NULL;
    orc_ctx* c = (orc_ctx*)calloc(1, sizeof(orc_ctx));
    if (!c) return NULL;
    c->lx = nx_log2; c->lt = nt_log2;
    c->nx = 1 << nx_log2; c->nt = 1 << nt_log2;
    c->mx = c->nx - 1; c->mt = c->nt - 1;
    c->nr = (int64_t)c->nx * c->nx * c->nt;
    c->R = R; c->half = half_shift ? 1 : 0;
    c->step_s = step_straight; c->step_a = step_scale; c->ct = ct;
    for (int m = 0; m < 6; m++) { c->cin[m] = ct; c->cout[m] = 0; }
    int nt = c->nt, nx = c->nx;
    c->beta = (int32_t*)malloc(sizeof(int32_t) * nt);
    c->psi2 = (uint8_t*)malloc(nt);
    c->iflag = (uint8_t*)malloc(nt);
    c->jsign = (int8_t*)malloc(nt);
    c->bsh = (int32_t*)malloc(sizeof(int32_t) * (size_t)nt * nx);
    c->wS = (uint32_t*)malloc(sizeof(uint32_t) * nt);
    if (!c->beta || !c->psi2 || !c->iflag || !c->jsign || !c->bsh || !c->wS) {
        orc_destroy(c);
        return NULL;
    }
    for (int T = 0; T < nt; T++) {
        double th = heading(T, nt);
        double s = sin(th), co = cos(th);
        /* eqs. 11-13: alpha = R sin(theta); zeta(x) = round(2x)/2;
         * beta = floor(zeta(alpha)); Psi = zeta(alpha) - beta.  Without the
         * half-cell option beta is alpha rounded the usual way and Psi = 0. */
        double alpha = R * s;
        if (c->half) {
            long z = lround(2.0 * alpha);
            c->beta[T] = (int32_t)floor_half(z);
            c->psi2[T] = (uint8_t)(z & 1 ? 1 : 0);
        } else {
            c->beta[T] = (int32_t)lround(alpha);
            c->psi2[T] = 0;
        }
        /* eq. 19: I = 0 iff |tan theta| <= 1, decided on the integer heading:
         * the angular distance to the nearest multiple of pi is m*2pi/nt, and
         * m*2pi/nt <= pi/4  <=>  8m <= nt. */
        int r = T % (nt / 2);
        int m = r < nt / 2 - r ? r : nt / 2 - r;
        c->iflag[T] = (uint8_t)(8 * m <= nt ? 0 : 1);
        /* eq. 24: J = sign(cos) when I = 0, sign(sin) when I = 1. */
        if (c->iflag[T] == 0) {
            int d0 = T < nt - T ? T : nt - T; /* cos > 0 iff d0 < nt/4 */
            c->jsign[T] = (int8_t)(4 * d0 < nt ? 1 : -1);
        } else {
            c->jsign[T] = (int8_t)(2 * T < nt ? 1 : -1); /* sin > 0 iff 0 < T < nt/2 */
        }
        /* eq. 20: K = tan when I = 0, cot when I = 1;  eq. 22: B = round(y' K). */
        double K = c->iflag[T] == 0 ? s / co : co / s;
        for (int y = 0; y < nx; y++) c->bsh[(size_t)T * nx + y] = (int32_t)lround((double)y * K);
        /* Section V.D: a straight edge spans 1/|cos| (I = 0) or 1/|sin| (I = 1)
         * cells, i.e. 1/max(|cos|,|sin|); the weight is that length times the
         * straight step unit, rounded. */
        double len = 1.0 / fmax(fabs(co), fabs(s));
        c->wS[T] = (uint32_t)lround((double)step_straight * len);
    }
    /* Section V.D: a turn edge spans 2 pi R / N_theta. */
    c->wA = (uint32_t)lround((double)step_scale * (2.0 * ORC_PI) * R / (double)nt);
    return c;
}

/* Star transition edges per maneuver (Section V.A, Fig. 9): entering
 * maneuver mu from the transition state costs cin[mu], returning to it
 * cout[mu] (changing gear or steering, speeding up, slowing down).  Each sum
 * must stay below 2^28. */
int orc_set_transition(orc_ctx* c, const uint32_t* cin, const uint32_t* cout) {
    for (int m = 0; m < 6; m++)
        if ((uint64_t)cin[m] + cout[m] >= (1u << 28)) return -1;
    for (int m = 0; m < 6; m++) { c->cin[m] = cin[m]; c->cout[m] = cout[m]; }
    return 0;
}

void orc_destroy(orc_ctx* c) {
    if (!c) return;
    free(c->beta); free(c->psi2); free(c->iflag); free(c->jsign); free(c->bsh); free(c->wS);
    free(c);
}

void orc_tables(const orc_ctx* c, int32_t* beta, uint8_t* psi2, uint8_t* iflag,
                int8_t* jsign, int32_t* bshear, uint32_t* wS, uint32_t* wA) {
    if (beta) memcpy(beta, c->beta, sizeof(int32_t) * c->nt);
    if (psi2) memcpy(psi2, c->psi2, c->nt);
    if (iflag) memcpy(iflag, c->iflag, c->nt);
    if (jsign) memcpy(jsign, c->jsign, c->nt);
    if (bshear) memcpy(bshear, c->bsh, sizeof(int32_t) * (size_t)c->nt * c->nx);
    if (wS) memcpy(wS, c->wS, sizeof(uint32_t) * c->nt);
    if (wA) *wA = c->wA;
}

/* ---------------------------------------------------------------- indexing */

static int64_t cell_of(const orc_ctx* c, int i, int j, int T) {
    return (int64_t)(i & c->mx) + (int64_t)c->nx * ((int64_t)(j & c->mx) + (int64_t)c->nx * (T & c->mt));
}
static void coords(const orc_ctx* c, int64_t cell, int* i, int* j, int* T) {
    *i = (int)(cell & c->mx);
    *j = (int)((cell >> c->lx) & c->mx);
    *T = (int)(cell >> (2 * c->lx));
}
static int beta_at(const orc_ctx* c, int T) { return c->beta[T & c->mt]; }

/* ---------------------------------------------------------------- footprint
 * Reading of Section VI with Fig. 6: the vehicle is the closed rectangle
 * [-rear, front] x [-hw, hw] in vehicle coordinates (origin at the rear axle).
 * Pose (i, j, T) stands for the continuum pose (i + Psi_0, j + Psi_1, theta)
 * (eq. 16).  World cell (i+dx, j+dy) belongs to the footprint when its centre,
 * expressed in vehicle coordinates, lies in the rectangle (with a 1e-9-cell
 * tolerance so that exact rotations by multiples of 90 degrees keep their
 * boundary cells); the cell under the origin always belongs. */
static double psi_x(const orc_ctx* c, int T) { return c->psi2[T & c->mt] * 0.5; }
static double psi_y(const orc_ctx* c, int T) { return c->psi2[(T + c->nt / 4) & c->mt] * 0.5; }

static int in_footprint(const orc_ctx* c, int front, int rear, int hw, int T, int dx, int dy) {
    if (dx == 0 && dy == 0) return 1;
    const double eps = 1e-9;
    double th = heading(T, c->nt);
    double co = cos(th), s = sin(th);
    double px = (double)dx - psi_x(c, T), py = (double)dy - psi_y(c, T);
    double xv = co * px + s * py;
    double yv = -s * px + co * py;
    return xv >= -(double)rear - eps && xv <= (double)front + eps &&
           yv >= -(double)hw - eps && yv <= (double)hw + eps;
}

static int footprint_reach(int front, int rear, int hw) {
    int ext = front > rear ? front : rear;
    return (int)ceil(sqrt((double)ext * ext + (double)hw * hw)) + 2;
}

int orc_footprint(const orc_ctx* c, int front, int rear, int hw, int T,
                  int32_t* dx, int32_t* dy, int cap) {
    int lim = footprint_reach(front, rear, hw);
    int n = 0;
    for (int y = -lim; y <= lim; y++)
        for (int x = -lim; x <= lim; x++)
            if (in_footprint(c, front, rear, hw, T, x, y)) {
                if (n < cap) { dx[n] = x; dy[n] = y; }
                n++;
            }
    return n <= cap ? n : -n;
}

/* Section VI + walls of Section V.C: a one-cell hard wall at i = 0 and j = 0,
 * all coordinates modulo N_x; B is the maximum of the image over the
 * footprint (HARD = 0xFFFF is the largest value, so any hard cell wins). */
static uint16_t img_at(const orc_ctx* c, const uint16_t* img, int x, int y) {
    x &= c->mx; y &= c->mx;
    if (x == 0 || y == 0) return ORC_HARD;
    return img[(size_t)y * c->nx + x];
}

static uint16_t render_one(const orc_ctx* c, const uint16_t* img, const int32_t* dx,
                           const int32_t* dy, int n, int i, int j) {
    uint16_t m = 0;
    for (int k = 0; k < n; k++) {
        uint16_t v = img_at(c, img, i + dx[k], j + dy[k]);
        if (v > m) m = v;
    }
    return m;
}

int orc_render(const orc_ctx* c, const uint16_t* img, int front, int rear, int hw, uint16_t* B) {
    int lim = footprint_reach(front, rear, hw);
    int cap = (2 * lim + 1) * (2 * lim + 1);
    int32_t* dx = (int32_t*)malloc(sizeof(int32_t) * cap);
    int32_t* dy = (int32_t*)malloc(sizeof(int32_t) * cap);
    if (!dx || !dy) { free(dx); free(dy); return -1; }
    for (int T = 0; T < c->nt; T++) {
        int n = orc_footprint(c, front, rear, hw, T, dx, dy, cap);
        for (int j = 0; j < c->nx; j++)
            for (int i = 0; i < c->nx; i++)
                B[cell_of(c, i, j, T)] = render_one(c, img, dx, dy, n, i, j);
    }
    free(dx); free(dy);
    return 0;
}

/* Same volume, grouped by footprint rows: each row of the footprint is a run
 * of cells [lo, lo+w) at offset dy, and the maximum over a run is a sliding
 * window maximum of width w along image rows, which Section VI notes costs a
 * constant number of comparisons per sample regardless of the width (the van
 * Herk / Gil-Werman block method: prefix maxima from each block start and
 * suffix maxima from each block end, window = max(suffix at x, prefix at
 * x+w-1)).  Rows are cyclic (coordinates modulo Nx). */
static void window_max_rows(const orc_ctx* c, const uint16_t* img, int w, uint16_t* out,
                            uint16_t* ext, uint16_t* pre, uint16_t* suf) {
    int nx = c->nx;
    int len = nx + w - 1; /* the row extended cyclically */
    int nblk = (len + w - 1) / w;
    int plen = nblk * w;
    for (int y = 0; y < nx; y++) {
        for (int x = 0; x < plen; x++) ext[x] = x < len ? img_at(c, img, x, y) : 0;
        for (int b = 0; b < nblk; b++) {
            int a = b * w;
            pre[a] = ext[a];
            for (int x = a + 1; x < a + w; x++) pre[x] = ext[x] > pre[x - 1] ? ext[x] : pre[x - 1];
            suf[a + w - 1] = ext[a + w - 1];
            for (int x = a + w - 2; x >= a; x--) suf[x] = ext[x] > suf[x + 1] ? ext[x] : suf[x + 1];
        }
        for (int x = 0; x < nx; x++) {
            uint16_t s1 = suf[x], p1 = pre[x + w - 1];
            out[(size_t)y * nx + x] = s1 > p1 ? s1 : p1;
        }
    }
}

int orc_render_rows(const orc_ctx* c, const uint16_t* img, int front, int rear, int hw, uint16_t* B) {
    int lim = footprint_reach(front, rear, hw);
    int cap = (2 * lim + 1) * (2 * lim + 1);
    int nx = c->nx;
    size_t plane = (size_t)nx * nx;
    int wmax = 2 * lim + 1;
    int32_t* dx = (int32_t*)malloc(sizeof(int32_t) * cap);
    int32_t* dy = (int32_t*)malloc(sizeof(int32_t) * cap);
    uint16_t* win = (uint16_t*)malloc(sizeof(uint16_t) * plane * (size_t)(wmax + 1));
    uint8_t* have = (uint8_t*)malloc((size_t)wmax + 1);
    int buf = 2 * (nx + wmax) + 2 * wmax;
    uint16_t* ext = (uint16_t*)malloc(sizeof(uint16_t) * buf);
    uint16_t* pre = (uint16_t*)malloc(sizeof(uint16_t) * buf);
    uint16_t* suf = (uint16_t*)malloc(sizeof(uint16_t) * buf);
    if (!dx || !dy || !win || !have || !ext || !pre || !suf) {
        free(dx); free(dy); free(win); free(have); free(ext); free(pre); free(suf);
        return -1;
    }
    memset(have, 0, (size_t)wmax + 1);
    for (int T = 0; T < c->nt; T++) {
        int n = orc_footprint(c, front, rear, hw, T, dx, dy, cap);
        uint16_t* Bt = B + (size_t)T * plane;
        memset(Bt, 0, plane * sizeof(uint16_t));
        /* cells come sorted by dy then dx: split each dy into maximal runs */
        for (int k = 0; k < n;) {
            int e = k;
            while (e + 1 < n && dy[e + 1] == dy[k] && dx[e + 1] == dx[e] + 1) e++;
            int lo = dx[k], w = dx[e] - dx[k] + 1, ry = dy[k];
            if (!have[w]) { window_max_rows(c, img, w, win + (size_t)w * plane, ext, pre, suf); have[w] = 1; }
            const uint16_t* W = win + (size_t)w * plane;
            for (int j = 0; j < nx; j++) {
                const uint16_t* row = W + (size_t)((j + ry) & c->mx) * nx;
                uint16_t* out = Bt + (size_t)j * nx;
                for (int i = 0; i < nx; i++) {
                    uint16_t v = row[(i + lo) & c->mx];
                    if (v > out[i]) out[i] = v;
                }
            }
            k = e + 1;
        }
    }
    free(dx); free(dy); free(win); free(have); free(ext); free(pre); free(suf);
    return 0;
}

int orc_render_cells(const orc_ctx* c, const uint16_t* img, int front, int rear, int hw,
                     const int64_t* cells, int64_t n, uint16_t* out) {
    int lim = footprint_reach(front, rear, hw);
    int cap = (2 * lim + 1) * (2 * lim + 1);
    int32_t* dx = (int32_t*)malloc(sizeof(int32_t) * cap);
    int32_t* dy = (int32_t*)malloc(sizeof(int32_t) * cap);
    if (!dx || !dy) { free(dx); free(dy); return -1; }
    for (int64_t k = 0; k < n; k++) {
        int i, j, T;
        if (cells[k] < 0 || cells[k] >= c->nr) { free(dx); free(dy); return -1; }
        coords(c, cells[k], &i, &j, &T);
        int m = orc_footprint(c, front, rear, hw, T, dx, dy, cap);
        out[k] = render_one(c, img, dx, dy, m, i, j);
    }
    free(dx); free(dy);
    return 0;
}

/* ------------------------------------------------------------ maneuver edges */

static int is_turn(int mu) { return mu == LF || mu == LB || mu == RF || mu == RB; }

int64_t orc_succ(const orc_ctx* c, int mu, int64_t cell) {
    int i, j, T;
    coords(c, cell, &i, &j, &T);
    int q = c->nt / 4;
    if (is_turn(mu)) {
        /* eqs. 25-28: LEFT uses (beta_0, beta_3), RIGHT uses (beta_2, beta_1);
         * LF and RB step to T+1, LB and RF to T-1; beta_q^{+/-}(T) =
         * beta(T + qN/4 +/- 1) - beta(T + qN/4). */
        int qa = (mu == LF || mu == LB) ? 0 : 2;
        int qb = (mu == LF || mu == LB) ? 3 : 1;
        int step = (mu == LF || mu == RB) ? 1 : -1;
        int T2 = (T + step) & c->mt;
        int di = beta_at(c, T + step + qa * q) - beta_at(c, T + qa * q);
        int dj = beta_at(c, T + step + qb * q) - beta_at(c, T + qb * q);
        return cell_of(c, i + di, j + dj, T2);
    }
    /* eqs. 30-31; eq. 24 picks which of them is forward. */
    int plus = (c->jsign[T] >= 0) == (mu == SF);
    int step = plus ? 1 : -1;
    const int32_t* Bs = c->bsh + (size_t)T * c->nx;
    if (c->iflag[T] == 0) {
        int i2 = (i + step) & c->mx;
        return cell_of(c, i2, j + Bs[i2] - Bs[i], T);
    } else {
        int j2 = (j + step) & c->mx;
        return cell_of(c, i + Bs[j2] - Bs[j], j2, T);
    }
}

/* Edge weight of the maneuver edge leaving `cell` (Insert 1 charges the
 * obstacle value of the vertex being left): w * B >> 8 with B in Q8, or INF
 * when the cell is hard. */
uint32_t orc_edge(const orc_ctx* c, const uint16_t* B, int mu, int64_t cell) {
    uint16_t b = B[cell];
    if (b == ORC_HARD) return ORC_INF;
    uint32_t w = is_turn(mu) ? c->wA : c->wS[cell >> (2 * c->lx)];
    return (uint32_t)(((uint64_t)w * b) >> 8);
}

/* ------------------------------------------------- explicit Star graph (Fig. 9)
 * Per cell X: vertex T(X) (transition state) and M_mu(X) for the six
 * maneuvers; edges T->M_mu (weight cin[mu], ct by default), M_mu->T (weight
 * cout[mu], 0 by default), and the maneuver
 * edge M_mu(X) -> M_mu(succ_mu(X)) (weight orc_edge).  A hard cell has no
 * transition vertex: its T<->M edges are absent (weight INF). */
typedef struct {
    int64_t nr;
    uint32_t* succ[6];   /* maneuver edge targets  */
    uint32_t* w_mm[6];   /* maneuver edge weights  */
    uint32_t* w_tm[6];   /* T -> M_mu weights      */
    uint32_t* w_mt[6];   /* M_mu -> T weights      */
} star_graph;

static void graph_free(star_graph* g) {
    for (int m = 0; m < 6; m++) { free(g->succ[m]); free(g->w_mm[m]); free(g->w_tm[m]); free(g->w_mt[m]); }
}

static int graph_build(const orc_ctx* c, const uint16_t* B, star_graph* g) {
    memset(g, 0, sizeof(*g));
    if (c->nr > 0xFFFFFFFFll) return -1;
    g->nr = c->nr;
    for (int m = 0; m < 6; m++) {
        g->succ[m] = (uint32_t*)malloc(sizeof(uint32_t) * c->nr);
        g->w_mm[m] = (uint32_t*)malloc(sizeof(uint32_t) * c->nr);
        g->w_tm[m] = (uint32_t*)malloc(sizeof(uint32_t) * c->nr);
        g->w_mt[m] = (uint32_t*)malloc(sizeof(uint32_t) * c->nr);
        if (!g->succ[m] || !g->w_mm[m] || !g->w_tm[m] || !g->w_mt[m]) { graph_free(g); return -1; }
        for (int64_t x = 0; x < c->nr; x++) {
            int hard = B[x] == ORC_HARD;
            g->succ[m][x] = (uint32_t)orc_succ(c, m, x);
            g->w_mm[m][x] = orc_edge(c, B, m, x);
            g->w_tm[m][x] = hard ? ORC_INF : c->cin[m];
            g->w_mt[m][x] = hard ? ORC_INF : c->cout[m];
        }
    }
    return 0;
}

/* ------------------------------------------ relaxation along one maneuver cycle
 * Running a maneuver kernel (Section VIII.B) means: from any transition state
 * at its current value, enter the maneuver, follow its edges, and return to
 * the transition state wherever that improves the value.  On a cycle
 * c_0 .. c_{n-1} (c_{k+1} = succ(c_k)) this is, for each position p,
 *     V'(c_p) = min( V(c_p),  min_{d=1..n-1} V(c_{p-d}) + w_tm(c_{p-d})
 *                              + sum_{k=p-d}^{p-1} w_mm(c_k) + w_mt(c_p) )
 * with all V read at the start of the layer.  Longer segments wrap a full
 * cycle and cannot improve (every finite edge costs at least 1).
 * Tie reading: a label is written only on strict improvement, and among
 * equal-cost entries the one furthest upstream (largest d) is recorded; for
 * the straight lines, which start at the wall, this is exactly what the
 * sequential Insert 1 loop with a strict comparison records. */
typedef struct {
    const uint32_t* Vin;
    uint32_t* Vout;
    uint16_t* L;
    int mu;
    int64_t improved;
} layer_io;

/* The definition above, evaluated directly: O(n^2) per cycle. */
static void relax_cycle_definition(layer_io* io, int n, const int64_t* cell, const uint32_t* w_tm,
                                   const uint32_t* w_mm, const uint32_t* w_mt) {
    for (int p = 0; p < n; p++) {
        uint32_t best = ORC_INF;
        int bd = 0;
        uint32_t path = 0; /* sum of w_mm over positions p-d .. p-1 */
        for (int d = 1; d < n; d++) {
            int s = ((p - d) % n + n) % n;
            path = sadd(path, w_mm[s]);
            uint32_t cand = sadd(sadd(sadd(io->Vin[cell[s]], w_tm[s]), path), w_mt[p]);
            if (cand != ORC_INF && cand <= best) { best = cand; bd = d; }
        }
        if (best < io->Vin[cell[p]]) {
            io->Vout[cell[p]] = best;
            io->L[cell[p]] = (uint16_t)((io->mu << 13) | bd);
            io->improved++;
        }
    }
}

/* The same relaxation as the sequential loop of Insert 1 run over the cycle
 * twice (Section VIII.B): the first loop warms the carried value up, the
 * second stores.  The carry keeps the entry position; a new entry replaces it
 * only when strictly cheaper, so ties keep the earlier (further upstream)
 * entry. */
static void relax_cycle_scan(layer_io* io, int n, const int64_t* cell, const uint32_t* w_tm,
                             const uint32_t* w_mm, const uint32_t* w_mt) {
    uint32_t v = ORC_INF;
    int qe = 0;
    for (int q = 0; q < 2 * n; q++) {
        int k = q % n;
        uint32_t u = io->Vin[cell[k]];
        if (q >= n) {
            uint32_t cand = sadd(v, w_mt[k]);
            if (cand < u) {
                io->Vout[cell[k]] = cand;
                io->L[cell[k]] = (uint16_t)((io->mu << 13) | (q - qe));
                io->improved++;
            }
        }
        uint32_t t = sadd(u, w_tm[k]);
        if (t < v) { v = t; qe = q; }
        v = sadd(v, w_mm[k]);
    }
}

/* mode 0 / 2: explicit edge list, cycles found by following succ pointers. */
static int layer_edgelist(const star_graph* g, int mu, layer_io* io, int use_definition) {
    int64_t nr = g->nr;
    uint8_t* seen = (uint8_t*)calloc((size_t)nr, 1);
    int64_t* cyc = (int64_t*)malloc(sizeof(int64_t) * 8192);
    uint32_t* a = (uint32_t*)malloc(sizeof(uint32_t) * 3 * 8192);
    if (!seen || !cyc || !a) { free(seen); free(cyc); free(a); return -1; }
    uint32_t *wtm = a, *wmm = a + 8192, *wmt = a + 2 * 8192;
    for (int64_t x0 = 0; x0 < nr; x0++) {
        if (seen[x0]) continue;
        int n = 0;
        int64_t x = x0;
        while (!seen[x]) {
            if (n >= 8192) { free(seen); free(cyc); free(a); return -1; }
            seen[x] = 1;
            cyc[n] = x;
            wtm[n] = g->w_tm[mu][x];
            wmm[n] = g->w_mm[mu][x];
            wmt[n] = g->w_mt[mu][x];
            n++;
            x = g->succ[mu][x];
        }
        if (x != x0) { free(seen); free(cyc); free(a); return -1; } /* not a permutation */
        if (use_definition) relax_cycle_definition(io, n, cyc, wtm, wmm, wmt);
        else relax_cycle_scan(io, n, cyc, wtm, wmm, wmt);
    }
    free(seen); free(cyc); free(a);
    return 0;
}

/* mode 1: edges evaluated on the fly; all cycles of the maneuver advance in
 * lockstep (as the paper's threads do), each started at one cell of its own:
 * turn chains at their heading-0 cell, straight lines at their wall cell.
 * Each chain is checked to close after n steps.
 *
 * The chains of one layer touch disjoint cells (each cell lies on exactly
 * one chain of a maneuver, eqs. 18 and 23) and read only the layer's input
 * V, so they may run on several host threads (orc_set_threads; one by
 * default): the turn chains of each lockstep step, or whole heading planes
 * of straight lines.  Every chain does the same steps as on one thread. */
static int g_threads = 1;

void orc_set_threads(int n) { g_threads = n > 0 ? n : 1; }

/* One lockstep step q of the chains k in [0, nchains): returns the number
 * of cells improved. */
static int64_t lockstep_step(const orc_ctx* c, const uint16_t* B, int mu, layer_io* io, int n, int q,
                             int64_t nchains, int64_t* cur, uint32_t* v, int32_t* qe, int threads) {
    int64_t improved = 0;
#pragma omp parallel for reduction(+ : improved) num_threads(threads) if (threads > 1) schedule(static)
    for (int64_t k = 0; k < nchains; k++) {
        int64_t x = cur[k];
        int hard = B[x] == ORC_HARD;
        uint32_t u = io->Vin[x];
        if (q >= n) {
            uint32_t cand = hard ? ORC_INF : sadd(v[k], c->cout[mu]);
            if (cand < u) {
                io->Vout[x] = cand;
                io->L[x] = (uint16_t)((io->mu << 13) | (q - qe[k]));
                improved++;
            }
        }
        uint32_t t = hard ? ORC_INF : sadd(u, c->cin[mu]);
        if (t < v[k]) { v[k] = t; qe[k] = q; }
        v[k] = sadd(v[k], orc_edge(c, B, mu, x));
        cur[k] = orc_succ(c, mu, x);
    }
    return improved;
}

/* All chains of one heading plane (straights) or of the whole volume
 * (turns), started at plane `plane`'s wall cells or at heading 0. */
static int lockstep_plane(const orc_ctx* c, const uint16_t* B, int mu, layer_io* io, int plane, int threads,
                          int64_t* improved) {
    int nx = c->nx;
    int64_t nchains;
    int n;
    if (is_turn(mu)) { nchains = (int64_t)nx * nx; n = c->nt; }
    else { nchains = nx; n = nx; }
    int64_t* start = (int64_t*)malloc(sizeof(int64_t) * nchains);
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * nchains);
    uint32_t* v = (uint32_t*)malloc(sizeof(uint32_t) * nchains);
    int32_t* qe = (int32_t*)malloc(sizeof(int32_t) * nchains);
    if (!start || !cur || !v || !qe) { free(start); free(cur); free(v); free(qe); return -1; }
    int rc = 0;
    for (int64_t k = 0; k < nchains; k++) {
        if (is_turn(mu)) start[k] = k; /* cells of heading plane 0 */
        else start[k] = c->iflag[plane] == 0 ? cell_of(c, 0, (int)k, plane) : cell_of(c, (int)k, 0, plane);
        cur[k] = start[k];
        v[k] = ORC_INF;
        qe[k] = 0;
    }
    for (int q = 0; q < 2 * n; q++) {
        *improved += lockstep_step(c, B, mu, io, n, q, nchains, cur, v, qe, threads);
        if (q == n - 1)
            for (int64_t k = 0; k < nchains; k++)
                if (cur[k] != start[k]) rc = -1;
    }
    free(start); free(cur); free(v); free(qe);
    return rc;
}

static int layer_lockstep(const orc_ctx* c, const uint16_t* B, int mu, layer_io* io) {
    int64_t improved = 0;
    int rc = 0;
    if (is_turn(mu)) {
        rc = lockstep_plane(c, B, mu, io, 0, g_threads, &improved);
    } else {
        const int threads = g_threads;
#pragma omp parallel for reduction(+ : improved) reduction(| : rc) num_threads(threads) if (threads > 1) \
    schedule(dynamic, 1)
        for (int plane = 0; plane < c->nt; plane++) {
            int64_t imp = 0;
            rc |= lockstep_plane(c, B, mu, io, plane, 1, &imp);
            improved += imp;
        }
    }
    io->improved += improved;
    return rc;
}

static const int cycle_order[6] = {LF, SF, RB, RF, SB, LB}; /* Section XVI.A */

int orc_layers(const orc_ctx* c, const uint16_t* B, int first_layer, int n_layers, int mode,
               uint32_t* V, uint16_t* L, int64_t* improved) {
    if (mode < 0 || mode > 2 || n_layers < 0 || first_layer < 0) return -1;
    star_graph g;
    int have_graph = 0;
    if (mode != 1) {
        if (graph_build(c, B, &g) != 0) return -1;
        have_graph = 1;
    }
    uint32_t* Vin = (uint32_t*)malloc(sizeof(uint32_t) * c->nr);
    if (!Vin) { if (have_graph) graph_free(&g); return -1; }
    int rc = 0;
    for (int l = 0; l < n_layers && rc == 0; l++) {
        int mu = cycle_order[(first_layer + l) % 6];
        memcpy(Vin, V, sizeof(uint32_t) * c->nr);
        layer_io io = {Vin, V, L, mu, 0};
        if (mode == 1) rc = layer_lockstep(c, B, mu, &io);
        else rc = layer_edgelist(&g, mu, &io, mode == 2);
        if (improved) improved[l] = io.improved;
    }
    free(Vin);
    if (have_graph) graph_free(&g);
    return rc;
}

int orc_sweep(const orc_ctx* c, const uint16_t* B, int64_t start, int n_cycles, int mode,
              uint32_t* V, uint16_t* L, int64_t* improved) {
    if (start < 0 || start >= c->nr || B[start] == ORC_HARD || n_cycles < 0) return -1;
    for (int64_t x = 0; x < c->nr; x++) { V[x] = ORC_INF; L[x] = ORC_NONE; }
    V[start] = 0;
    return orc_layers(c, B, 0, 6 * n_cycles, mode, V, L, improved);
}

/* ------------------------------------------------ start state (Section XII)
 * A vehicle already under way when the plan starts: entry[mu] is what
 * entering maneuver mu at the start pose costs -- cin[mu] (ct) for a vehicle
 * at rest in the transition state, 0 for the maneuver in progress (no
 * transition cost for it), the rest of a transition in progress toward mu.
 * Reading of Section XII's "first maneuver kernel of that type without a
 * transition cost": every maneuver with entry[mu] < cin[mu] is first
 * followed from the start pose alone (the start layer, maneuvers in cycle
 * order, strict improvement; leaving the maneuver still costs cout[mu]),
 * then the N cycles run as from rest.  The start keeps V = 0, so entering at
 * cin[mu] stays possible and entries above it are refused. */
static int entries_ok(const orc_ctx* c, const uint32_t* entry) {
    for (int m = 0; m < 6; m++)
        if (entry[m] > c->cin[m]) return 0;
    return 1;
}

int orc_seed(const orc_ctx* c, const uint16_t* B, int64_t start, const uint32_t* entry, uint32_t* V,
             uint16_t* L) {
    if (start < 0 || start >= c->nr || B[start] == ORC_HARD || !entries_ok(c, entry)) return -1;
    for (int l = 0; l < 6; l++) {
        int mu = cycle_order[l];
        if (entry[mu] >= c->cin[mu]) continue;
        int n = is_turn(mu) ? c->nt : c->nx; /* the curve closes after n steps */
        uint32_t run = entry[mu];
        int64_t y = start;
        for (int d = 1; d < n; d++) {
            run = sadd(run, orc_edge(c, B, mu, y));
            y = orc_succ(c, mu, y);
            if (run == ORC_INF) break; /* a hard cell was left */
            uint32_t back = sadd(run, c->cout[mu]); /* back in the transition state */
            if (B[y] != ORC_HARD && back < V[y]) {
                V[y] = back;
                L[y] = (uint16_t)((mu << 13) | d);
            }
        }
    }
    return 0;
}

int orc_sweep_state(const orc_ctx* c, const uint16_t* B, int64_t start, const uint32_t* entry, int n_cycles,
                    int mode, uint32_t* V, uint16_t* L, int64_t* improved) {
    if (start < 0 || start >= c->nr || B[start] == ORC_HARD || n_cycles < 0 || !entries_ok(c, entry)) return -1;
    for (int64_t x = 0; x < c->nr; x++) { V[x] = ORC_INF; L[x] = ORC_NONE; }
    V[start] = 0;
    if (orc_seed(c, B, start, entry, V, L) != 0) return -1;
    return orc_layers(c, B, 0, 6 * n_cycles, mode, V, L, improved);
}

/* ----------------------------------------------------- Dijkstra (Section VIII.A)
 * Indexed binary heap kept in two arrays, heap position of a vertex and the
 * vertex at a heap position, keyed by the value array itself. */
typedef struct {
    uint32_t* key;
    int64_t* heap;
    int64_t* pos;
    int64_t n;
} iheap;

static void heap_swap(iheap* h, int64_t a, int64_t b) {
    int64_t va = h->heap[a], vb = h->heap[b];
    h->heap[a] = vb; h->heap[b] = va;
    h->pos[vb] = a; h->pos[va] = b;
}
static void heap_up(iheap* h, int64_t k) {
    while (k > 0) {
        int64_t p = (k - 1) / 2;
        if (h->key[h->heap[p]] <= h->key[h->heap[k]]) break;
        heap_swap(h, p, k);
        k = p;
    }
}
static void heap_down(iheap* h, int64_t k) {
    for (;;) {
        int64_t l = 2 * k + 1, r = l + 1, m = k;
        if (l < h->n && h->key[h->heap[l]] < h->key[h->heap[m]]) m = l;
        if (r < h->n && h->key[h->heap[r]] < h->key[h->heap[m]]) m = r;
        if (m == k) break;
        heap_swap(h, m, k);
        k = m;
    }
}

/* entry (optional): the start's own transition edges T(start) -> M_mu(start)
 * weigh entry[mu] instead of ct (the start state of Section XII). */
static int dijkstra_from(const orc_ctx* c, const uint16_t* B, int64_t start, const uint32_t* entry,
                         uint32_t* Vinf) {
    if (start < 0 || start >= c->nr || B[start] == ORC_HARD) return -1;
    star_graph g;
    if (graph_build(c, B, &g) != 0) return -1;
    int64_t nr = c->nr, nv = 7 * nr; /* vertex 0..nr-1: T(X); (1+mu)*nr + X: M_mu(X) */
    iheap h;
    h.key = (uint32_t*)malloc(sizeof(uint32_t) * nv);
    h.heap = (int64_t*)malloc(sizeof(int64_t) * nv);
    h.pos = (int64_t*)malloc(sizeof(int64_t) * nv);
    uint8_t* done = (uint8_t*)calloc((size_t)nv, 1);
    if (!h.key || !h.heap || !h.pos || !done) {
        free(h.key); free(h.heap); free(h.pos); free(done); graph_free(&g); return -1;
    }
    for (int64_t v = 0; v < nv; v++) { h.key[v] = ORC_INF; h.pos[v] = -1; }
    h.key[start] = 0;
    h.heap[0] = start; h.pos[start] = 0; h.n = 1;
#define RELAX(dst, w)                                                   \
    do {                                                                \
        uint32_t nd_ = sadd(du, (w));                                   \
        int64_t d_ = (dst);                                             \
        if (nd_ < h.key[d_] && !done[d_]) {                             \
            h.key[d_] = nd_;                                            \
            if (h.pos[d_] < 0) { h.heap[h.n] = d_; h.pos[d_] = h.n; h.n++; } \
            heap_up(&h, h.pos[d_]);                                     \
        }                                                               \
    } while (0)
    while (h.n > 0) {
        int64_t u = h.heap[0];
        heap_swap(&h, 0, h.n - 1);
        h.n--;
        h.pos[u] = -1;
        if (h.n > 0) heap_down(&h, 0);
        done[u] = 1;
        uint32_t du = h.key[u];
        if (du == ORC_INF) break;
        if (u < nr) {
            for (int m = 0; m < 6; m++)
                RELAX((1 + m) * nr + u, (entry && u == start) ? entry[m] : g.w_tm[m][u]);
        } else {
            int m = (int)(u / nr) - 1;
            int64_t x = u % nr;
            RELAX(x, g.w_mt[m][x]);
            RELAX((1 + m) * nr + g.succ[m][x], g.w_mm[m][x]);
        }
    }
#undef RELAX
    for (int64_t x = 0; x < nr; x++) Vinf[x] = B[x] == ORC_HARD ? ORC_INF : h.key[x];
    free(h.key); free(h.heap); free(h.pos); free(done); graph_free(&g);
    return 0;
}

int orc_dijkstra(const orc_ctx* c, const uint16_t* B, int64_t start, uint32_t* Vinf) {
    return dijkstra_from(c, B, start, NULL, Vinf);
}

int orc_dijkstra_state(const orc_ctx* c, const uint16_t* B, int64_t start, const uint32_t* entry,
                       uint32_t* Vinf) {
    if (!entries_ok(c, entry)) return -1;
    return dijkstra_from(c, B, start, entry, Vinf);
}

/* ------------------------------------------------------------ brute force
 * Enumerate every sequence of at most one maneuver segment per layer (layers
 * in the cycle order), every segment length 1..n-1, starting at T(start);
 * a path prefix that reaches (layer, cell) no cheaper than an earlier one is
 * dropped, because what can follow depends only on (layer, cell). */
typedef struct {
    const orc_ctx* c;
    const uint16_t* B;
    int layers;
    uint32_t* seen; /* [layer][cell] */
    uint32_t* best;
} bf_state;

static void bf_explore(bf_state* s, int layer, int64_t x, uint32_t cost) {
    const orc_ctx* c = s->c;
    uint32_t* sl = s->seen + (size_t)layer * c->nr;
    if (cost >= sl[x]) return;
    sl[x] = cost;
    if (cost < s->best[x]) s->best[x] = cost;
    if (layer == s->layers) return;
    bf_explore(s, layer + 1, x, cost); /* no segment in this layer */
    int mu = cycle_order[layer % 6];
    int n = is_turn(mu) ? c->nt : c->nx;
    uint32_t run = sadd(cost, c->cin[mu]);
    int64_t y = x;
    for (int d = 1; d < n; d++) {
        run = sadd(run, orc_edge(c, s->B, mu, y));
        y = orc_succ(c, mu, y);
        if (run == ORC_INF) break;
        if (s->B[y] != ORC_HARD) bf_explore(s, layer + 1, y, sadd(run, c->cout[mu]));
    }
}

/* With entry: before layer 0, at most one segment of any maneuver mu with
 * entry[mu] < cin[mu] leaves the start, entered at entry[mu] (the start layer). */
static int bruteforce_from(const orc_ctx* c, const uint16_t* B, int64_t start, const uint32_t* entry,
                           int n_cycles, uint32_t* Vbest) {
    if (start < 0 || start >= c->nr || B[start] == ORC_HARD) return -1;
    bf_state s = {c, B, 6 * n_cycles, NULL, Vbest};
    s.seen = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(s.layers + 1) * c->nr);
    if (!s.seen) return -1;
    for (int64_t k = 0; k < (int64_t)(s.layers + 1) * c->nr; k++) s.seen[k] = ORC_INF;
    for (int64_t x = 0; x < c->nr; x++) Vbest[x] = ORC_INF;
    bf_explore(&s, 0, start, 0);
    for (int mu = 0; entry && mu < 6; mu++) {
        if (entry[mu] >= c->cin[mu]) continue;
        int n = is_turn(mu) ? c->nt : c->nx;
        uint32_t run = entry[mu];
        int64_t y = start;
        for (int d = 1; d < n; d++) {
            run = sadd(run, orc_edge(c, B, mu, y));
            y = orc_succ(c, mu, y);
            if (run == ORC_INF) break;
            if (B[y] != ORC_HARD) bf_explore(&s, 0, y, sadd(run, c->cout[mu]));
        }
    }
    free(s.seen);
    return 0;
}

int orc_bruteforce(const orc_ctx* c, const uint16_t* B, int64_t start, int n_cycles, uint32_t* Vbest) {
    return bruteforce_from(c, B, start, NULL, n_cycles, Vbest);
}

int orc_bruteforce_state(const orc_ctx* c, const uint16_t* B, int64_t start, const uint32_t* entry,
                         int n_cycles, uint32_t* Vbest) {
    if (!entries_ok(c, entry)) return -1;
    return bruteforce_from(c, B, start, entry, n_cycles, Vbest);
}

/* ------------------------------------------------------------ extraction
 * Forward tracking (Section X): each label names the maneuver and how many
 * steps back its entry lies.  The entry is reached by walking the reverse
 * maneuver (eqs. 25-31 are exactly reversible: LF<->LB, RF<->RB, SF<->SB,
 * which in cycle-order numbering is mu -> 5 - mu). */
int orc_extract(const orc_ctx* c, const uint32_t* V, const uint16_t* L, int64_t goal,
                int64_t* seg, int cap) {
    if (goal < 0 || goal >= c->nr) return -3;
    if (V[goal] == ORC_INF) return -1;
    int n = 0;
    int64_t x = goal;
    int guard = 0;
    while (L[x] != ORC_NONE) {
        if (++guard > 1 << 20) return -3;
        int mu = L[x] >> 13, d = L[x] & 8191;
        if (mu > 5 || d == 0) return -3;
        int64_t e = x;
        for (int k = 0; k < d; k++) e = orc_succ(c, 5 - mu, e);
        if (n < cap) {
            int64_t* r = seg + 6 * (size_t)n;
            r[0] = mu; r[1] = e; r[2] = x; r[3] = d;
            r[4] = (int64_t)(V[x] & 0xFFFF); r[5] = (int64_t)(V[x] >> 16);
        }
        n++;
        x = e;
    }
    if (V[x] != 0) return -3;
    if (n > cap) return -2;
    for (int a = 0, b = n - 1; a < b; a++, b--)
        for (int k = 0; k < 6; k++) {
            int64_t t = seg[6 * a + k];
            seg[6 * a + k] = seg[6 * b + k];
            seg[6 * b + k] = t;
        }
    return n;
}

/* --------------------------------------------------------------- gear states
 * A gear penalty that depends on the pair of consecutive maneuvers needs the
 * transition state to remember the gear: two transition vertices per cell,
 * T_F (the last maneuver ran forward, LF SF RF) and T_R (reverse, LB SB RB).
 * Entering maneuver mu costs cin[mu] from the state of its own gear and
 * cin[mu] + pen from the other one; leaving mu costs cout[mu] and returns to
 * the state of mu's gear (the Star of Fig. 9 with its centre split in two).
 * Volumes: V[0 .. nr) is T_F, V[nr .. 2 nr) is T_R, L alike, a label being
 * (mu << 13) | (other << 12) | d, other = 1 when the segment was entered
 * from the other gear's state.  Kernel-style layers as in orc_layers (all
 * values read at the start of the layer); at one entry cell the own gear's
 * state wins a tie.  A segment may now run a whole cycle (d = n): going
 * once around a turn circle from T_F(x) reaches T_R(x), which with one
 * transition state could never pay off; so d <= n <= 4095 (grids up to
 * 2048).  start_gear: 0 the vehicle stands in forward gear, 1 in reverse, 2
 * at rest (both states 0 at the start). */
static int gear_of(int mu) { return (mu == LB || mu == SB || mu == RB) ? 1 : 0; }

static int layer_gear(const orc_ctx* c, const uint16_t* B, int mu, uint32_t pen, const uint32_t* Vin,
                      uint32_t* V, uint16_t* L) {
    int nx = c->nx, G = gear_of(mu);
    int64_t nr = c->nr, nchains;
    int n;
    if (is_turn(mu)) { nchains = (int64_t)nx * nx; n = c->nt; }
    else { nchains = nx; n = nx; }
    int nplanes = is_turn(mu) ? 1 : c->nt;
    const uint32_t* Vs = Vin + (G ? nr : 0); /* own gear */
    const uint32_t* Vo = Vin + (G ? 0 : nr); /* other gear */
    uint32_t* Vw = V + (G ? nr : 0);
    uint16_t* Lw = L + (G ? nr : 0);
    for (int plane = 0; plane < nplanes; plane++)
        for (int64_t k = 0; k < nchains; k++) {
            int64_t start;
            if (is_turn(mu)) start = k;
            else start = c->iflag[plane] == 0 ? cell_of(c, 0, (int)k, plane) : cell_of(c, (int)k, 0, plane);
            int64_t x = start;
            uint32_t v = ORC_INF;
            int qe = 0, vo = 0;
            for (int q = 0; q < 2 * n; q++) {
                int hard = B[x] == ORC_HARD;
                if (q >= n) {
                    uint32_t cand = hard ? ORC_INF : sadd(v, c->cout[mu]);
                    if (cand < Vs[x]) {
                        Vw[x] = cand;
                        Lw[x] = (uint16_t)((mu << 13) | (vo << 12) | (q - qe));
                    }
                }
                uint32_t ts = hard ? ORC_INF : sadd(Vs[x], c->cin[mu]);
                uint32_t to = hard ? ORC_INF : sadd(sadd(Vo[x], c->cin[mu]), pen);
                int oth = to < ts;
                uint32_t t = oth ? to : ts;
                if (t < v) { v = t; qe = q; vo = oth; }
                v = sadd(v, orc_edge(c, B, mu, x));
                x = orc_succ(c, mu, x);
            }
            if (x != start) return -1;
        }
    return 0;
}

static int gear_args_ok(const orc_ctx* c, const uint16_t* B, int64_t start, int start_gear) {
    return start >= 0 && start < c->nr && B[start] != ORC_HARD && start_gear >= 0 && start_gear <= 2 &&
           c->nx <= 2048 && c->nt <= 2048;
}

int orc_sweep_gear(const orc_ctx* c, const uint16_t* B, int64_t start, int start_gear, uint32_t pen,
                   int n_cycles, uint32_t* V, uint16_t* L) {
    if (!gear_args_ok(c, B, start, start_gear) || n_cycles < 0) return -1;
    int64_t nr = c->nr;
    for (int64_t x = 0; x < 2 * nr; x++) { V[x] = ORC_INF; L[x] = ORC_NONE; }
    if (start_gear != 1) V[start] = 0;
    if (start_gear != 0) V[nr + start] = 0;
    uint32_t* Vin = (uint32_t*)malloc(sizeof(uint32_t) * 2 * nr);
    if (!Vin) return -1;
    int rc = 0;
    for (int l = 0; l < 6 * n_cycles && rc == 0; l++) {
        memcpy(Vin, V, sizeof(uint32_t) * 2 * nr);
        rc = layer_gear(c, B, cycle_order[l % 6], pen, Vin, V, L);
    }
    free(Vin);
    return rc;
}

/* Dijkstra on the explicit graph: vertices T_F(x), T_R(x), M_mu(x).  A
 * segment moves at least one step (Insert 1 tests a cell for storing before
 * entering there), so a transition vertex leads straight over the first
 * maneuver edge: T_g(x) -> M_mu(succ(x)); otherwise T_F(x) -> M_mu(x) ->
 * T_R(x) would change gear without moving, which the sweeps never do. */
int orc_dijkstra_gear(const orc_ctx* c, const uint16_t* B, int64_t start, int start_gear, uint32_t pen,
                      uint32_t* Vinf) {
    if (!gear_args_ok(c, B, start, start_gear)) return -1;
    int64_t nr = c->nr, nv = 8 * nr; /* [0, nr) T_F, [nr, 2nr) T_R, (2+mu)*nr + x: M_mu(x) */
    iheap h;
    h.key = (uint32_t*)malloc(sizeof(uint32_t) * nv);
    h.heap = (int64_t*)malloc(sizeof(int64_t) * nv);
    h.pos = (int64_t*)malloc(sizeof(int64_t) * nv);
    uint8_t* done = (uint8_t*)calloc((size_t)nv, 1);
    if (!h.key || !h.heap || !h.pos || !done) { free(h.key); free(h.heap); free(h.pos); free(done); return -1; }
    for (int64_t v = 0; v < nv; v++) { h.key[v] = ORC_INF; h.pos[v] = -1; }
    h.n = 0;
    for (int g = 0; g < 2; g++) {
        if ((g == 0 && start_gear == 1) || (g == 1 && start_gear == 0)) continue;
        int64_t v = g * nr + start;
        h.key[v] = 0;
        h.heap[h.n] = v; h.pos[v] = h.n; h.n++;
    }
#define GRELAX(dst, w)                                                  \
    do {                                                                \
        uint32_t nd_ = sadd(du, (w));                                   \
        int64_t d_ = (dst);                                             \
        if (nd_ < h.key[d_] && !done[d_]) {                             \
            h.key[d_] = nd_;                                            \
            if (h.pos[d_] < 0) { h.heap[h.n] = d_; h.pos[d_] = h.n; h.n++; } \
            heap_up(&h, h.pos[d_]);                                     \
        }                                                               \
    } while (0)
    while (h.n > 0) {
        int64_t u = h.heap[0];
        heap_swap(&h, 0, h.n - 1);
        h.n--;
        h.pos[u] = -1;
        if (h.n > 0) heap_down(&h, 0);
        done[u] = 1;
        uint32_t du = h.key[u];
        if (du == ORC_INF) break;
        int64_t x = u % nr;
        int kind = (int)(u / nr);
        if (B[x] == ORC_HARD) continue;
        if (kind < 2) {
            for (int m = 0; m < 6; m++) {
                int64_t y = orc_succ(c, m, x);
                uint32_t w = sadd(gear_of(m) == kind ? c->cin[m] : sadd(c->cin[m], pen), orc_edge(c, B, m, x));
                if (B[y] != ORC_HARD) GRELAX((2 + m) * nr + y, w);
            }
        } else {
            int m = kind - 2;
            GRELAX(gear_of(m) * nr + x, c->cout[m]);
            int64_t y = orc_succ(c, m, x);
            uint32_t w = orc_edge(c, B, m, x);
            if (B[y] != ORC_HARD) GRELAX((2 + m) * nr + y, w);
        }
    }
#undef GRELAX
    for (int64_t x = 0; x < 2 * nr; x++) Vinf[x] = B[x % nr] == ORC_HARD ? ORC_INF : h.key[x];
    free(h.key); free(h.heap); free(h.pos); free(done);
    return 0;
}

/* Exhaustive search over layer-ordered segment sequences with the gear
 * state: best[g*nr + x] over sequences ending in state g at x. */
typedef struct {
    const orc_ctx* c;
    const uint16_t* B;
    uint32_t pen;
    int layers;
    uint32_t* seen; /* [layer][gear][cell] */
    uint32_t* best;
} bfg_state;

static void bfg_explore(bfg_state* s, int layer, int g, int64_t x, uint32_t cost) {
    const orc_ctx* c = s->c;
    int64_t nr = c->nr;
    uint32_t* sl = s->seen + ((size_t)layer * 2 + g) * nr;
    if (cost >= sl[x]) return;
    sl[x] = cost;
    if (cost < s->best[g * nr + x]) s->best[g * nr + x] = cost;
    if (layer == s->layers) return;
    bfg_explore(s, layer + 1, g, x, cost);
    int mu = cycle_order[layer % 6], G = gear_of(mu);
    int n = is_turn(mu) ? c->nt : c->nx;
    uint32_t run = sadd(cost, G == g ? c->cin[mu] : sadd(c->cin[mu], s->pen));
    int64_t y = x;
    for (int d = 1; d <= n; d++) { /* a whole cycle may change the gear state */
        run = sadd(run, orc_edge(c, s->B, mu, y));
        y = orc_succ(c, mu, y);
        if (run == ORC_INF) break;
        if (s->B[y] != ORC_HARD) bfg_explore(s, layer + 1, G, y, sadd(run, c->cout[mu]));
    }
}

int orc_bruteforce_gear(const orc_ctx* c, const uint16_t* B, int64_t start, int start_gear, uint32_t pen,
                        int n_cycles, uint32_t* Vbest) {
    if (!gear_args_ok(c, B, start, start_gear) || n_cycles < 0) return -1;
    int64_t nr = c->nr;
    bfg_state s = {c, B, pen, 6 * n_cycles, NULL, Vbest};
    s.seen = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(s.layers + 1) * 2 * nr);
    if (!s.seen) return -1;
    for (int64_t k = 0; k < (int64_t)(s.layers + 1) * 2 * nr; k++) s.seen[k] = ORC_INF;
    for (int64_t x = 0; x < 2 * nr; x++) Vbest[x] = ORC_INF;
    if (start_gear != 1) bfg_explore(&s, 0, 0, start, 0);
    if (start_gear != 0) bfg_explore(&s, 0, 1, start, 0);
    free(s.seen);
    return 0;
}

/* Label walk with gear states: from the cheaper state at the goal (forward
 * on a tie), each label names the maneuver, the steps back to its entry and
 * whether it entered from the other gear's state.  seg[k*7 + {mu, entry,
 * exit, d, cost_lo16, cost_hi16, entry_gear}] in driving order.  Returns the
 * segment count, -1 unreachable, -2 cap too small, -3 malformed labels. */
int orc_extract_gear(const orc_ctx* c, const uint32_t* V, const uint16_t* L, int64_t goal, int64_t* seg,
                     int cap) {
    if (goal < 0 || goal >= c->nr) return -3;
    int64_t nr = c->nr;
    int g = V[nr + goal] < V[goal] ? 1 : 0;
    if (V[g * nr + goal] == ORC_INF) return -1;
    int n = 0, guard = 0;
    int64_t x = goal;
    while (L[g * nr + x] != ORC_NONE) {
        if (++guard > 1 << 20) return -3;
        uint16_t lab = L[g * nr + x];
        int mu = lab >> 13, oth = (lab >> 12) & 1, d = lab & 4095;
        if (mu > 5 || d == 0 || gear_of(mu) != g) return -3;
        int64_t e = x;
        for (int k = 0; k < d; k++) e = orc_succ(c, 5 - mu, e);
        int ge = oth ? 1 - g : g;
        if (n < cap) {
            int64_t* r = seg + 7 * (size_t)n;
            uint32_t cost = V[g * nr + x];
            r[0] = mu; r[1] = e; r[2] = x; r[3] = d; r[4] = cost & 0xFFFF; r[5] = cost >> 16; r[6] = ge;
        }
        n++;
        x = e;
        g = ge;
    }
    if (V[g * nr + x] != 0) return -3;
    if (n > cap) return -2;
    for (int a2 = 0, b2 = n - 1; a2 < b2; a2++, b2--)
        for (int k = 0; k < 7; k++) {
            int64_t t = seg[7 * a2 + k];
            seg[7 * a2 + k] = seg[7 * b2 + k];
            seg[7 * b2 + k] = t;
        }
    return n;
}

/* ------------------------------------------------------- Compact graph
 * Section V.A, Fig. 12: three vertices per cell -- S (the straight maneuver
 * type, which is also the transition state), L (left turns, forward and
 * backward) and R (right turns) -- and ten edges: S -> L and S -> R (the
 * transition cost ct of plan creation), L -> S and R -> S (free), and the six
 * maneuver edges, straights within S, LF/LB within L, RF/RB within R.  So a
 * turn costs ct to start, a straight nothing, and a gear change within one
 * turn direction nothing (the flexibility the Compact graph gives up).
 * Readings for its kernel-style processing: the cycle order of Section
 * XVI.A; a turn layer enters its chain from the cell's own turn state free
 * or from S at ct (own state on a tie) and stores into its turn state and,
 * over the free edge back, into S; a straight layer moves within S; a
 * segment moves at least one step, and a whole turn circle from S back to
 * the same cell counts (it reaches the turn state; d <= n <= 2048).
 * Volumes: V[0, nr) S, [nr, 2nr) L, [2nr, 3nr) R; labels (mu << 13) |
 * (entered from S << 12) | d. */
static int compact_type(int mu) { return (mu == LF || mu == LB) ? 1 : (mu == RF || mu == RB) ? 2 : 0; }

static int layer_compact(const orc_ctx* c, const uint16_t* B, int mu, const uint32_t* Vin, uint32_t* V,
                         uint16_t* L) {
    int64_t nr = c->nr;
    int ty = compact_type(mu), n;
    int64_t nchains;
    if (is_turn(mu)) { nchains = (int64_t)c->nx * c->nx; n = c->nt; }
    else { nchains = c->nx; n = c->nx; }
    int nplanes = is_turn(mu) ? 1 : c->nt;
    for (int plane = 0; plane < nplanes; plane++)
        for (int64_t k = 0; k < nchains; k++) {
            int64_t start;
            if (is_turn(mu)) start = k;
            else start = c->iflag[plane] == 0 ? cell_of(c, 0, (int)k, plane) : cell_of(c, (int)k, 0, plane);
            int64_t x = start;
            uint32_t v = ORC_INF;
            int qe = 0, vs = 0;
            for (int q = 0; q < 2 * n; q++) {
                int hard = B[x] == ORC_HARD;
                uint32_t uT = Vin[ty * nr + x], uS = Vin[x];
                if (q >= n && !hard) {
                    uint16_t lab = (uint16_t)((mu << 13) | (vs << 12) | (q - qe));
                    if (v < uT && v < V[ty * nr + x]) { V[ty * nr + x] = v; L[ty * nr + x] = lab; }
                    if (ty != 0 && v < uS && v < V[x]) { V[x] = v; L[x] = lab; } /* back to S, free */
                }
                uint32_t tT = hard ? ORC_INF : uT;
                uint32_t tS = (hard || ty == 0) ? ORC_INF : sadd(uS, c->ct);
                int fromS = tS < tT;
                uint32_t t = fromS ? tS : tT;
                if (t < v) { v = t; qe = q; vs = fromS; }
                v = sadd(v, orc_edge(c, B, mu, x));
                x = orc_succ(c, mu, x);
            }
            if (x != start) return -1;
        }
    return 0;
}

int orc_sweep_compact(const orc_ctx* c, const uint16_t* B, int64_t start, int n_cycles, uint32_t* V,
                      uint16_t* L) {
    if (start < 0 || start >= c->nr || B[start] == ORC_HARD || n_cycles < 0 || c->nx > 2048 || c->nt > 2048)
        return -1;
    int64_t n3 = 3 * c->nr;
    for (int64_t x = 0; x < n3; x++) { V[x] = ORC_INF; L[x] = ORC_NONE; }
    V[start] = 0; /* the vehicle starts in S */
    uint32_t* Vin = (uint32_t*)malloc(sizeof(uint32_t) * n3);
    if (!Vin) return -1;
    int rc = 0;
    for (int l = 0; l < 6 * n_cycles && rc == 0; l++) {
        memcpy(Vin, V, sizeof(uint32_t) * n3);
        rc = layer_compact(c, B, cycle_order[l % 6], Vin, V, L);
    }
    free(Vin);
    return rc;
}

/* Dijkstra on the explicit Compact graph; a transition into a turn leads over
 * the turn's first edge (a segment moves at least one step). */
int orc_dijkstra_compact(const orc_ctx* c, const uint16_t* B, int64_t start, uint32_t* Vinf) {
    if (start < 0 || start >= c->nr || B[start] == ORC_HARD) return -1;
    int64_t nr = c->nr, nv = 3 * nr;
    iheap h;
    h.key = (uint32_t*)malloc(sizeof(uint32_t) * nv);
    h.heap = (int64_t*)malloc(sizeof(int64_t) * nv);
    h.pos = (int64_t*)malloc(sizeof(int64_t) * nv);
    uint8_t* done = (uint8_t*)calloc((size_t)nv, 1);
    if (!h.key || !h.heap || !h.pos || !done) { free(h.key); free(h.heap); free(h.pos); free(done); return -1; }
    for (int64_t v = 0; v < nv; v++) { h.key[v] = ORC_INF; h.pos[v] = -1; }
    h.key[start] = 0; h.heap[0] = start; h.pos[start] = 0; h.n = 1;
#define RC(dst, w)                                                      \
    do {                                                                \
        uint32_t nd_ = sadd(du, (w));                                   \
        int64_t d_ = (dst);                                             \
        if (nd_ < h.key[d_] && !done[d_]) {                             \
            h.key[d_] = nd_;                                            \
            if (h.pos[d_] < 0) { h.heap[h.n] = d_; h.pos[d_] = h.n; h.n++; } \
            heap_up(&h, h.pos[d_]);                                     \
        }                                                               \
    } while (0)
    static const int of_type[3][2] = {{SF, SB}, {LF, LB}, {RF, RB}};
    while (h.n > 0) {
        int64_t u = h.heap[0];
        heap_swap(&h, 0, h.n - 1);
        h.n--;
        h.pos[u] = -1;
        if (h.n > 0) heap_down(&h, 0);
        done[u] = 1;
        uint32_t du = h.key[u];
        if (du == ORC_INF) break;
        int ty = (int)(u / nr);
        int64_t x = u % nr;
        if (B[x] == ORC_HARD) continue;
        for (int k = 0; k < 2; k++) { /* maneuver edges within the vertex type */
            int mu = of_type[ty][k];
            int64_t y = orc_succ(c, mu, x);
            if (B[y] != ORC_HARD) RC(ty * nr + y, orc_edge(c, B, mu, x));
        }
        if (ty == 0) { /* S -> L, S -> R over the turn's first edge */
            for (int t2 = 1; t2 < 3; t2++)
                for (int k = 0; k < 2; k++) {
                    int mu = of_type[t2][k];
                    int64_t y = orc_succ(c, mu, x);
                    if (B[y] != ORC_HARD) RC(t2 * nr + y, sadd(c->ct, orc_edge(c, B, mu, x)));
                }
        } else {
            RC(x, 0u); /* back to S */
        }
    }
#undef RC
    for (int64_t x = 0; x < nv; x++) Vinf[x] = B[x % nr] == ORC_HARD ? ORC_INF : h.key[x];
    free(h.key); free(h.heap); free(h.pos); free(done);
    return 0;
}

/* Exhaustive search over layer-ordered segment sequences (tiny grids):
 * best[ty * nr + x] over sequences ending in vertex type ty at x. */
typedef struct {
    const orc_ctx* c;
    const uint16_t* B;
    int layers;
    uint32_t* seen; /* [layer][type][cell] */
    uint32_t* best;
} bfc_state;

static void bfc_explore(bfc_state* s, int layer, int ty, int64_t x, uint32_t cost) {
    const orc_ctx* c = s->c;
    int64_t nr = c->nr;
    uint32_t* sl = s->seen + ((size_t)layer * 3 + ty) * nr;
    if (cost >= sl[x]) return;
    sl[x] = cost;
    if (cost < s->best[ty * nr + x]) s->best[ty * nr + x] = cost;
    if (ty != 0) bfc_explore(s, layer, 0, x, cost); /* back to S, free */
    if (layer == s->layers) return;
    bfc_explore(s, layer + 1, ty, x, cost);
    int mu = cycle_order[layer % 6], T = compact_type(mu);
    if (T != ty && ty != 0) return;          /* a turn state enters only its own turns */
    if (T == 0 && ty != 0) return;
    uint32_t run = (T != 0 && ty == 0) ? sadd(cost, c->ct) : cost;
    int n = is_turn(mu) ? c->nt : c->nx;
    int64_t y = x;
    for (int d = 1; d <= n; d++) { /* a whole turn circle from S changes the vertex type */
        run = sadd(run, orc_edge(c, s->B, mu, y));
        y = orc_succ(c, mu, y);
        if (run == ORC_INF) break;
        if (s->B[y] != ORC_HARD) bfc_explore(s, layer + 1, T, y, run);
    }
}

int orc_bruteforce_compact(const orc_ctx* c, const uint16_t* B, int64_t start, int n_cycles, uint32_t* Vbest) {
    if (start < 0 || start >= c->nr || B[start] == ORC_HARD || n_cycles < 0) return -1;
    int64_t nr = c->nr;
    bfc_state s = {c, B, 6 * n_cycles, NULL, Vbest};
    s.seen = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(s.layers + 1) * 3 * nr);
    if (!s.seen) return -1;
    for (int64_t k = 0; k < (int64_t)(s.layers + 1) * 3 * nr; k++) s.seen[k] = ORC_INF;
    for (int64_t x = 0; x < 3 * nr; x++) Vbest[x] = ORC_INF;
    bfc_explore(&s, 0, 0, start, 0);
    free(s.seen);
    return 0;
}

/* Label walk from S(goal): seg[k*6 + {mu, entry, exit, d, cost, entered_from_S}]. */
int orc_extract_compact(const orc_ctx* c, const uint32_t* V, const uint16_t* L, int64_t goal, int64_t* seg,
                        int cap) {
    if (goal < 0 || goal >= c->nr) return -3;
    int64_t nr = c->nr;
    if (V[goal] == ORC_INF) return -1;
    int ty = 0, n = 0, guard = 0;
    int64_t x = goal;
    while (L[ty * nr + x] != ORC_NONE) {
        if (++guard > 1 << 20) return -3;
        uint16_t lab = L[ty * nr + x];
        int mu = lab >> 13, fs = (lab >> 12) & 1, d = lab & 4095;
        int T = compact_type(mu);
        if (mu > 5 || d == 0 || (ty != 0 && T != ty)) return -3;
        int64_t e = x;
        for (int k = 0; k < d; k++) e = orc_succ(c, 5 - mu, e);
        if (n < cap) {
            int64_t* r = seg + 6 * (size_t)n;
            r[0] = mu; r[1] = e; r[2] = x; r[3] = d; r[4] = V[ty * nr + x]; r[5] = fs;
        }
        n++;
        x = e;
        ty = fs ? 0 : T;
    }
    if (V[ty * nr + x] != 0) return -3;
    if (n > cap) return -2;
    for (int a2 = 0, b2 = n - 1; a2 < b2; a2++, b2--)
        for (int k = 0; k < 6; k++) {
            int64_t t = seg[6 * a2 + k];
            seg[6 * a2 + k] = seg[6 * b2 + k];
            seg[6 * b2 + k] = t;
        }
    return n;
}

/* ------------------------------------------------- 4D generalisation (App. F)
 * Curvature as a fourth state dimension: 2M+1 levels kappa = -M .. M (index
 * K = kappa + M) of the 3D volume, curvature k = kappa / (M R).  Readings of
 * App. F where it is silent:
 *   - extremal controls: the turns of the 3D model at the steering limits
 *     (LF, LB at kappa = +M; RF, RB at -M), the straights at kappa = 0, and
 *     clothoids that change the curvature one level per arc length L (cells)
 *     at the other levels: family C1 with dk/ds = +1/(M R L), family C2 with
 *     dk/ds = -1/(M R L), each driven forward and backward (time reversal:
 *     C1F raises kappa, C1B lowers it, C2F lowers it, C2B raises it);
 *   - a clothoid chain is named by its pose (x0, y0, theta0) at kappa = 0;
 *     at level kappa it is at (x0 + round X, y0 + round Y, theta0 + round
 *     Psi) with s = kappa L (C1) or -kappa L (C2), Psi = +-a s^2, a = 1 /
 *     (2 M R L), X = int_0^s cos(theta0 +- a sigma^2) dsigma, Y the sine
 *     (App. F's per-level map, a bijection per level), integrals by
 *     composite Simpson with 64 |kappa| intervals, headings Psi * N_theta /
 *     (2 pi), rounding half away from zero;
 *   - a clothoid step costs round(step_scale * L) * B >> 8 of the cell left
 *     (B does not depend on the curvature), entering a clothoid ctc, leaving
 *     it nothing; the 3D maneuvers keep their Star costs;
 *   - chains of a clothoid are open (kappa runs from one steering limit to
 *     the other): one pass from their first level;
 *   - cycle order: C1F, C2F, C1B, C2B, then the 3D order LF SF RB RF SB LB
 *     (maneuver ids 6, 8, 7, 9, 0 .. 5);
 *   - labels (mu << 12) | d.  The start and the goal name their level. */
struct orc4 {
    const orc_ctx* c;
    int M, nk;
    double L;
    uint32_t wC, ctc;
    int16_t* dx; /* [f][K][T0] */
    int16_t* dy;
    int32_t* dth; /* [f][K] */
};

static double clothoid_f(int f, int xy, double th0, double a, double sg) {
    double ang = f == 0 ? th0 + a * sg * sg : th0 - a * sg * sg;
    return xy == 0 ? cos(ang) : sin(ang);
}

/* int_0^s of cos or sin (xy) of theta0 +- a sigma^2, composite Simpson */
static double clothoid_int(int f, int xy, double th0, double a, double s, int n) {
    double h = s / n, acc = clothoid_f(f, xy, th0, a, 0.0) + clothoid_f(f, xy, th0, a, s);
    for (int i = 1; i < n; i++) acc += (i & 1 ? 4.0 : 2.0) * clothoid_f(f, xy, th0, a, i * h);
    return acc * h / 3.0;
}

orc4* orc4_create(const orc_ctx* c, int M, double L, uint32_t ctc) {
    if (M < 1 || M > 1000 || !(L > 0.0) || L > 4.0 || ctc >= (1u << 28)) return NULL;
    orc4* q = (orc4*)calloc(1, sizeof(orc4));
    if (!q) return NULL;
    q->c = c; q->M = M; q->nk = 2 * M + 1; q->L = L; q->ctc = ctc;
    q->wC = (uint32_t)lround((double)c->step_a * L);
    if (q->wC == 0) q->wC = 1;
    size_t n = (size_t)2 * q->nk * c->nt;
    q->dx = (int16_t*)malloc(sizeof(int16_t) * n);
    q->dy = (int16_t*)malloc(sizeof(int16_t) * n);
    q->dth = (int32_t*)malloc(sizeof(int32_t) * 2 * q->nk);
    if (!q->dx || !q->dy || !q->dth) { orc4_destroy(q); return NULL; }
    double a = 1.0 / (2.0 * M * c->R * L);
    for (int f = 0; f < 2; f++)
        for (int K = 0; K < q->nk; K++) {
            int kap = K - M;
            double s = f == 0 ? kap * L : -kap * L;
            double psi = f == 0 ? a * s * s : -a * s * s;
            q->dth[f * q->nk + K] = (int32_t)lround(psi * c->nt / (2.0 * ORC_PI));
            int nint = 64 * (kap < 0 ? -kap : kap);
            for (int T0 = 0; T0 < c->nt; T0++) {
                size_t at = ((size_t)f * q->nk + K) * c->nt + T0;
                if (kap == 0) { q->dx[at] = 0; q->dy[at] = 0; continue; }
                double th0 = heading(T0, c->nt);
                q->dx[at] = (int16_t)lround(clothoid_int(f, 0, th0, a, s, nint));
                q->dy[at] = (int16_t)lround(clothoid_int(f, 1, th0, a, s, nint));
            }
        }
    return q;
}

void orc4_destroy(orc4* q) {
    if (!q) return;
    free(q->dx); free(q->dy); free(q->dth); free(q);
}

void orc4_tables(const orc4* q, int16_t* dx, int16_t* dy, int32_t* dth) {
    size_t n = (size_t)2 * q->nk * q->c->nt;
    memcpy(dx, q->dx, sizeof(int16_t) * n);
    memcpy(dy, q->dy, sizeof(int16_t) * n);
    memcpy(dth, q->dth, sizeof(int32_t) * 2 * q->nk);
}

static int m4_level(const orc4* q, int mu) { /* level of a 3D maneuver */
    if (mu == LF || mu == LB) return q->nk - 1;
    if (mu == RF || mu == RB) return 0;
    return q->M;
}
static int m4_family(int mu) { return (mu == 6 || mu == 7) ? 0 : 1; }
static int m4_dir(int mu) { return (mu == 6 || mu == 9) ? 1 : -1; } /* kappa step */

/* Cell (3D index) of clothoid family f's chain (i0, j0, T0) at level K. */
static int64_t m4_chain_cell(const orc4* q, int f, int i0, int j0, int T0, int K) {
    const orc_ctx* c = q->c;
    size_t at = ((size_t)f * q->nk + K) * c->nt + T0;
    return cell_of(c, i0 + q->dx[at], j0 + q->dy[at], T0 + q->dth[f * q->nk + K]);
}

/* Successor of 4D cell (3D cell x at level K) along maneuver mu; -1 none. */
int64_t orc4_succ(const orc4* q, int mu, int64_t x4) {
    const orc_ctx* c = q->c;
    int64_t nr = c->nr;
    int K = (int)(x4 / nr);
    int64_t x = x4 % nr;
    if (mu < 6) {
        if (K != m4_level(q, mu)) return -1;
        return (int64_t)K * nr + orc_succ(c, mu, x);
    }
    int f = m4_family(mu), K2 = K + m4_dir(mu);
    if (K2 < 0 || K2 >= q->nk) return -1;
    int i, j, T;
    coords(c, x, &i, &j, &T);
    int T0 = (T - q->dth[f * q->nk + K]) & c->mt;
    size_t at = ((size_t)f * q->nk + K) * c->nt + T0;
    return (int64_t)K2 * nr + m4_chain_cell(q, f, i - q->dx[at], j - q->dy[at], T0, K2);
}

static uint32_t m4_edge(const orc4* q, const uint16_t* B, int mu, int64_t x4) {
    int64_t x = x4 % q->c->nr;
    if (mu < 6) return orc_edge(q->c, B, mu, x);
    if (B[x] == ORC_HARD) return ORC_INF;
    return (uint32_t)(((uint64_t)q->wC * B[x]) >> 8);
}
static uint32_t m4_cin(const orc4* q, int mu) { return mu < 6 ? q->c->cin[mu] : q->ctc; }
static uint32_t m4_cout(const orc4* q, int mu) { return mu < 6 ? q->c->cout[mu] : 0u; }

static const int cycle4[10] = {6, 8, 7, 9, LF, SF, RB, RF, SB, LB};

/* One maneuver layer on the 4D volumes (values read at the start of the
 * layer).  Cyclic chains (turns, straights) take two loops as in
 * layer_lockstep; clothoid chains are open and take one pass. */
static int layer4(const orc4* q, const uint16_t* B, int mu, const uint32_t* Vin, uint32_t* V, uint16_t* L) {
    const orc_ctx* c = q->c;
    int64_t nr = c->nr;
    int64_t* cyc = (int64_t*)malloc(sizeof(int64_t) * (size_t)(c->nx > c->nt ? c->nx : c->nt) * 2 + 64 +
                                    sizeof(int64_t) * q->nk);
    if (!cyc) return -1;
    int rc = 0;
    if (mu < 6) {
        int K = m4_level(q, mu), n;
        int64_t nchains;
        if (is_turn(mu)) { nchains = (int64_t)c->nx * c->nx; n = c->nt; }
        else { nchains = c->nx; n = c->nx; }
        int nplanes = is_turn(mu) ? 1 : c->nt;
        for (int plane = 0; plane < nplanes && rc == 0; plane++)
            for (int64_t k = 0; k < nchains && rc == 0; k++) {
                int64_t x = is_turn(mu) ? k
                            : (c->iflag[plane] == 0 ? cell_of(c, 0, (int)k, plane) : cell_of(c, (int)k, 0, plane));
                for (int t = 0; t < n; t++) { cyc[t] = (int64_t)K * nr + x; x = orc_succ(c, mu, x); }
                if ((int64_t)K * nr + x != cyc[0]) rc = -1;
                uint32_t v = ORC_INF;
                int qe = 0;
                for (int qq = 0; qq < 2 * n; qq++) {
                    int64_t y = cyc[qq % n];
                    int hard = B[y % nr] == ORC_HARD;
                    if (qq >= n) {
                        uint32_t cand = hard ? ORC_INF : sadd(v, m4_cout(q, mu));
                        if (cand < Vin[y] && cand < V[y]) {
                            V[y] = cand;
                            L[y] = (uint16_t)((mu << 12) | (qq - qe));
                        }
                    }
                    uint32_t t = hard ? ORC_INF : sadd(Vin[y], m4_cin(q, mu));
                    if (t < v) { v = t; qe = qq; }
                    v = sadd(v, m4_edge(q, B, mu, y));
                }
            }
    } else {
        int f = m4_family(mu), dir = m4_dir(mu);
        for (int T0 = 0; T0 < c->nt; T0++)
            for (int j0 = 0; j0 < c->nx; j0++)
                for (int i0 = 0; i0 < c->nx; i0++) {
                    uint32_t v = ORC_INF;
                    int qe = 0;
                    for (int qq = 0; qq < q->nk; qq++) {
                        int K = dir > 0 ? qq : q->nk - 1 - qq;
                        int64_t y = (int64_t)K * nr + m4_chain_cell(q, f, i0, j0, T0, K);
                        int hard = B[y % nr] == ORC_HARD;
                        uint32_t cand = hard ? ORC_INF : sadd(v, m4_cout(q, mu));
                        if (cand < Vin[y] && cand < V[y]) {
                            V[y] = cand;
                            L[y] = (uint16_t)((mu << 12) | (qq - qe));
                        }
                        uint32_t t = hard ? ORC_INF : sadd(Vin[y], m4_cin(q, mu));
                        if (t < v) { v = t; qe = qq; }
                        v = sadd(v, m4_edge(q, B, mu, y));
                    }
                }
    }
    free(cyc);
    return rc;
}

int orc4_sweep(const orc4* q, const uint16_t* B, int64_t start4, int n_cycles, uint32_t* V, uint16_t* L) {
    const orc_ctx* c = q->c;
    int64_t n4 = c->nr * q->nk;
    if (start4 < 0 || start4 >= n4 || B[start4 % c->nr] == ORC_HARD || n_cycles < 0) return -1;
    if (c->nx > 2048 || c->nt > 2048) return -1;
    for (int64_t x = 0; x < n4; x++) { V[x] = ORC_INF; L[x] = ORC_NONE; }
    V[start4] = 0;
    uint32_t* Vin = (uint32_t*)malloc(sizeof(uint32_t) * n4);
    if (!Vin) return -1;
    int rc = 0;
    for (int l = 0; l < 10 * n_cycles && rc == 0; l++) {
        memcpy(Vin, V, sizeof(uint32_t) * n4);
        rc = layer4(q, B, cycle4[l % 10], Vin, V, L);
    }
    free(Vin);
    return rc;
}

/* Dijkstra on the explicit 4D Star graph: T(x4) and M_mu(x4) for the
 * maneuvers that exist at x4's level. */
int orc4_dijkstra(const orc4* q, const uint16_t* B, int64_t start4, uint32_t* Vinf) {
    const orc_ctx* c = q->c;
    int64_t n4 = c->nr * q->nk, nv = 11 * n4; /* [0, n4) T, (1+mu)*n4 + x4: M_mu */
    if (start4 < 0 || start4 >= n4 || B[start4 % c->nr] == ORC_HARD) return -1;
    iheap h;
    h.key = (uint32_t*)malloc(sizeof(uint32_t) * nv);
    h.heap = (int64_t*)malloc(sizeof(int64_t) * nv);
    h.pos = (int64_t*)malloc(sizeof(int64_t) * nv);
    uint8_t* done = (uint8_t*)calloc((size_t)nv, 1);
    if (!h.key || !h.heap || !h.pos || !done) { free(h.key); free(h.heap); free(h.pos); free(done); return -1; }
    for (int64_t v = 0; v < nv; v++) { h.key[v] = ORC_INF; h.pos[v] = -1; }
    h.key[start4] = 0; h.heap[0] = start4; h.pos[start4] = 0; h.n = 1;
#define R4(dst, w)                                                      \
    do {                                                                \
        uint32_t nd_ = sadd(du, (w));                                   \
        int64_t d_ = (dst);                                             \
        if (nd_ < h.key[d_] && !done[d_]) {                             \
            h.key[d_] = nd_;                                            \
            if (h.pos[d_] < 0) { h.heap[h.n] = d_; h.pos[d_] = h.n; h.n++; } \
            heap_up(&h, h.pos[d_]);                                     \
        }                                                               \
    } while (0)
    while (h.n > 0) {
        int64_t u = h.heap[0];
        heap_swap(&h, 0, h.n - 1);
        h.n--;
        h.pos[u] = -1;
        if (h.n > 0) heap_down(&h, 0);
        done[u] = 1;
        uint32_t du = h.key[u];
        if (du == ORC_INF) break;
        int64_t x4 = u % n4;
        int kind = (int)(u / n4);
        if (B[x4 % c->nr] == ORC_HARD) continue;
        if (kind == 0) {
            for (int m = 0; m < 10; m++) {
                if (m < 6 && x4 / c->nr != m4_level(q, m)) continue;
                R4((1 + m) * n4 + x4, m4_cin(q, m));
            }
        } else {
            int m = kind - 1;
            R4(x4, m4_cout(q, m));
            int64_t y4 = orc4_succ(q, m, x4);
            if (y4 >= 0 && B[y4 % c->nr] != ORC_HARD) R4((1 + m) * n4 + y4, m4_edge(q, B, m, x4));
        }
    }
#undef R4
    for (int64_t x = 0; x < n4; x++) Vinf[x] = B[x % c->nr] == ORC_HARD ? ORC_INF : h.key[x];
    free(h.key); free(h.heap); free(h.pos); free(done);
    return 0;
}

/* Exhaustive search over layer-ordered segment sequences (tiny grids). */
typedef struct {
    const orc4* q;
    const uint16_t* B;
    int layers;
    uint32_t* seen;
    uint32_t* best;
} bf4_state;

static void bf4_explore(bf4_state* s, int layer, int64_t x4, uint32_t cost) {
    const orc4* q = s->q;
    int64_t n4 = q->c->nr * q->nk;
    uint32_t* sl = s->seen + (size_t)layer * n4;
    if (cost >= sl[x4]) return;
    sl[x4] = cost;
    if (cost < s->best[x4]) s->best[x4] = cost;
    if (layer == s->layers) return;
    bf4_explore(s, layer + 1, x4, cost);
    int mu = cycle4[layer % 10];
    if (mu < 6 && x4 / q->c->nr != m4_level(q, mu)) return;
    int n = mu < 6 ? (is_turn(mu) ? q->c->nt : q->c->nx) : q->nk;
    uint32_t run = sadd(cost, m4_cin(q, mu));
    int64_t y = x4;
    for (int d = 1; d < n; d++) {
        run = sadd(run, m4_edge(q, s->B, mu, y));
        y = orc4_succ(q, mu, y);
        if (y < 0 || run == ORC_INF) break;
        if (s->B[y % q->c->nr] != ORC_HARD) bf4_explore(s, layer + 1, y, sadd(run, m4_cout(q, mu)));
    }
}

int orc4_bruteforce(const orc4* q, const uint16_t* B, int64_t start4, int n_cycles, uint32_t* Vbest) {
    int64_t n4 = q->c->nr * q->nk;
    if (start4 < 0 || start4 >= n4 || B[start4 % q->c->nr] == ORC_HARD || n_cycles < 0) return -1;
    bf4_state s = {q, B, 10 * n_cycles, NULL, Vbest};
    s.seen = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)(s.layers + 1) * n4);
    if (!s.seen) return -1;
    for (int64_t k = 0; k < (int64_t)(s.layers + 1) * n4; k++) s.seen[k] = ORC_INF;
    for (int64_t x = 0; x < n4; x++) Vbest[x] = ORC_INF;
    bf4_explore(&s, 0, start4, 0);
    free(s.seen);
    return 0;
}

/* Label walk in 4D: seg[k*5 + {mu, entry4, exit4, d, cost}], driving order. */
int orc4_extract(const orc4* q, const uint32_t* V, const uint16_t* L, int64_t goal4, int64_t* seg, int cap) {
    int64_t n4 = q->c->nr * q->nk;
    if (goal4 < 0 || goal4 >= n4) return -3;
    if (V[goal4] == ORC_INF) return -1;
    static const int rev4[10] = {LB, SB, RF, RB, SF, LF, 7, 6, 9, 8};
    int n = 0, guard = 0;
    int64_t x = goal4;
    while (L[x] != ORC_NONE) {
        if (++guard > 1 << 20) return -3;
        int mu = L[x] >> 12, d = L[x] & 4095;
        if (mu > 9 || d == 0) return -3;
        int64_t e = x;
        for (int k = 0; k < d && e >= 0; k++) e = orc4_succ(q, rev4[mu], e);
        if (e < 0) return -3;
        if (n < cap) {
            int64_t* r = seg + 5 * (size_t)n;
            r[0] = mu; r[1] = e; r[2] = x; r[3] = d; r[4] = V[x];
        }
        n++;
        x = e;
    }
    if (V[x] != 0) return -3;
    if (n > cap) return -2;
    for (int a2 = 0, b2 = n - 1; a2 < b2; a2++, b2--)
        for (int k = 0; k < 5; k++) {
            int64_t t = seg[5 * a2 + k];
            seg[5 * a2 + k] = seg[5 * b2 + k];
            seg[5 * b2 + k] = t;
        }
    return n;
}

/* ------------------------------------------------------------ goal search
 * Section IX: a goal set instead of one exact pose, each pose scored by a
 * reward that falls with its distance from an ideal pose; the best pose
 * maximises reward minus cost.  Reading (the form of the neighbourhood
 * search in Appendix G): the score to minimise is
 *     V(x) + bias_g + w_xy * (|dx| + |dy|) + w_theta * |dtheta|
 * over every goal g and every reached pose x of its box |dx|, |dy| <= r_xy
 * (inside the grid; the grid does not wrap) and |dtheta| <= r_theta (modulo
 * N_theta, 2 r_theta < N_theta).  Ties go to the earlier goal, within a goal
 * to the ideal pose itself, then to the box in raster order (dtheta, then
 * dy, then dx increasing).  goals[g*8 + {x, y, theta, r_xy, r_theta, w_xy,
 * w_theta, bias}].  Returns 0 with *cell and *score set, -1 if no pose of
 * any box was reached, -2 for a malformed goal. */
int orc_goal_search(const orc_ctx* c, const uint32_t* V, const int64_t* goals, int n, int64_t* cell,
                    uint64_t* score) {
    uint64_t best = UINT64_MAX;
    int64_t at = -1;
    for (int g = 0; g < n; g++) {
        const int64_t* q = goals + 8 * (size_t)g;
        int gx = (int)q[0], gy = (int)q[1], gt = (int)q[2], r = (int)q[3], rt = (int)q[4];
        uint64_t wxy = (uint64_t)q[5], wt = (uint64_t)q[6], bias = (uint64_t)q[7];
        if (gx < 0 || gx >= c->nx || gy < 0 || gy >= c->nx || gt < 0 || gt >= c->nt) return -2;
        if (r < 0 || r > 255 || rt < 0 || rt > 255 || 2 * rt >= c->nt) return -2;
        if (q[5] < 0 || q[5] > 0xFFFFFFFFll || q[6] < 0 || q[6] > 0xFFFFFFFFll || q[7] < 0 || q[7] > 0xFFFFFFFFll)
            return -2;
        for (int pass = 0; pass < 2; pass++) /* the ideal pose, then the box */
            for (int dt = -rt; dt <= rt; dt++)
                for (int dy = -r; dy <= r; dy++)
                    for (int dx = -r; dx <= r; dx++) {
                        if (pass == 0 && (dx || dy || dt)) continue;
                        int x = gx + dx, y = gy + dy;
                        if (x < 0 || x >= c->nx || y < 0 || y >= c->nx) continue;
                        int64_t k = cell_of(c, x, y, gt + dt);
                        if (V[k] == ORC_INF) continue;
                        uint64_t sc = (uint64_t)V[k] + bias + wxy * (uint64_t)(abs(dx) + abs(dy)) +
                                      wt * (uint64_t)abs(dt);
                        if (sc < best) { best = sc; at = k; }
                    }
    }
    if (at < 0) return -1;
    *cell = at;
    *score = best;
    return 0;
}

/* ------------------------------------------------------ direction penalties
 * Section XVI, Fig. 19: costs that encode which side of the road to drive on
 * and which way to move in an area.  Reading: a field gives each cell a
 * preferred heading (0xFFFF: none); a pose whose own cell has one and whose
 * heading differs from it by more than tol heading steps (circular distance)
 * has its obstacle value scaled, B = min(floor(B * pen / 256), 0xFFFE), so
 * every step there costs pen/256 times more; hard poses stay hard.  Applied
 * to a rendered B.  Returns -1 for a heading >= N_theta other than 0xFFFF,
 * tol outside [0, N_theta/2] or pen outside [256, 65535]. */
int orc_direction(const orc_ctx* c, uint16_t* B, const uint16_t* heading, int tol, uint32_t pen) {
    if (tol < 0 || tol > c->nt / 2 || pen < 256 || pen > 65535) return -1;
    for (int64_t k = 0; k < (int64_t)c->nx * c->nx; k++)
        if (heading[k] != 0xFFFF && heading[k] >= c->nt) return -1;
    for (int T = 0; T < c->nt; T++)
        for (int j = 0; j < c->nx; j++)
            for (int i = 0; i < c->nx; i++) {
                uint16_t h = heading[(size_t)j * c->nx + i];
                int64_t k = cell_of(c, i, j, T);
                if (h == 0xFFFF || B[k] == ORC_HARD) continue;
                int d = abs(T - (int)h);
                if (c->nt - d < d) d = c->nt - d;
                if (d <= tol) continue;
                uint32_t v = (uint32_t)B[k] * pen / 256u;
                B[k] = (uint16_t)(v < 0xFFFEu ? v : 0xFFFEu);
            }
    return 0;
}

/* ----------------------------------------------------------- soft obstacles
 * Only distances below the radius matter, and any occupied cell at squared
 * distance < r^2 lies inside the (2r-1)^2 window, so the window search gives
 * the exact penalty.  Cells outside the image do not count as occupied. */
void orc_soft_image(int nx, const uint8_t* occ, int radius, int soft_max, uint16_t* img) {
    int r2 = radius * radius;
    for (int y = 0; y < nx; y++)
        for (int x = 0; x < nx; x++) {
            if (occ[(size_t)y * nx + x]) { img[(size_t)y * nx + x] = ORC_HARD; continue; }
            int best = -1;
            for (int yy = y - radius + 1; yy <= y + radius - 1; yy++)
                for (int xx = x - radius + 1; xx <= x + radius - 1; xx++)
                    if (yy >= 0 && yy < nx && xx >= 0 && xx < nx && occ[(size_t)yy * nx + xx]) {
                        int d2 = (xx - x) * (xx - x) + (yy - y) * (yy - y);
                        if (best < 0 || d2 < best) best = d2;
                    }
            int pen = (best >= 0 && best < r2) ? soft_max * (r2 - best) / r2 : 0;
            img[(size_t)y * nx + x] = (uint16_t)(256 + pen);
        }
}

/* ------------------------------------------------------------------------
 * Maneuver-count reachability (Appendix C, Insert 2): hard obstacles only,
 * every maneuver edge free, every transition one maneuver.  reach_m is the
 * set of poses reachable from the start with at most m maneuvers; a cycle
 * takes every maneuver from reach_m at once (each of the six maneuver
 * kernels reads the previous cycle's reachability and the results are
 * combined), so reach_{m+1} = reach_m united with, for every maneuver,
 * the cells that follow a cell of reach_m along that maneuver's curve
 * without meeting a hard cell.  A curve is followed for at most one period
 * (N_theta steps for turns, Nx for straights, which meet the wall earlier).
 * count[x] = the smallest m with x in reach_m, 255 if none up to N.
 */
int orc_reach(const orc_ctx* c, const uint16_t* B, int64_t start, int n_cycles, uint8_t* count) {
    if (!c || !B || !count || start < 0 || start >= c->nr || n_cycles < 0 || n_cycles > 254) return -1;
    if (B[start] == ORC_HARD) return -1;
    for (int64_t x = 0; x < c->nr; x++) count[x] = 255;
    count[start] = 0;
    for (int m = 0; m < n_cycles; m++) {
        for (int mu = 0; mu < 6; mu++) {
            const int period = is_turn(mu) ? c->nt : c->nx;
            for (int64_t x = 0; x < c->nr; x++) {
                if (count[x] > m || B[x] == ORC_HARD) continue; /* entries: reach_m */
                int64_t y = x;
                for (int k = 1; k < period; k++) {
                    y = orc_succ(c, mu, y);
                    if (B[y] == ORC_HARD) break;
                    /* a cell of reach_m starts its own walk; everything beyond
                     * it is covered there (it is an entry of the same curve) */
                    if (count[y] <= m) break;
                    if (count[y] > m + 1) count[y] = (uint8_t)(m + 1);
                }
            }
        }
    }
    return 0;
}

/* Back-track a minimal maneuver sequence to `goal` (the paper does this on
 * the host from the kept reachability volumes).  Canonical choice, also used
 * by the library: at each level, the first maneuver in cycle order (LF, SF,
 * RB, RF, SB, LB) whose curve, walked upstream from the current cell without
 * meeting a hard cell, reaches a cell of the previous level; the nearest such
 * cell is the segment's entry.  Writes seg[k*4 + {mu, entry, exit, steps}] in
 * driving order.  Returns the number of segments, -1 if the goal is not
 * reachable within the counts, -2 if cap is too small, -3 if the counts are
 * inconsistent. */
int orc_reach_extract(const orc_ctx* c, const uint16_t* B, const uint8_t* count, int64_t goal,
                      int64_t* seg, int cap) {
    if (!c || !B || !count || goal < 0 || goal >= c->nr) return -3;
    if (count[goal] == 255) return -1;
    int n = 0;
    int64_t x = goal;
    for (int m = count[goal]; m > 0; m--) {
        int found = 0;
        for (int mu = 0; mu < 6 && !found; mu++) {
            const int period = is_turn(mu) ? c->nt : c->nx;
            int64_t y = x;
            for (int d = 1; d < period; d++) {
                y = orc_succ(c, 5 - mu, y); /* the reverse maneuver walks the curve upstream */
                if (B[y] == ORC_HARD) break;
                if (count[y] <= m - 1) {
                    if (n < cap) {
                        int64_t* r = seg + 4 * (size_t)n;
                        r[0] = mu; r[1] = y; r[2] = x; r[3] = d;
                    }
                    n++;
                    x = y;
                    found = 1;
                    break;
                }
            }
        }
        if (!found) return -3;
    }
    if (n > cap) return -2;
    for (int a = 0, b = n - 1; a < b; a++, b--)
        for (int k = 0; k < 4; k++) {
            int64_t t = seg[4 * a + k];
            seg[4 * a + k] = seg[4 * b + k];
            seg[4 * b + k] = t;
        }
    return n;
}
