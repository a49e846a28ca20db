/* cpu_sweep.c -- the kernel-style sweep on all host cores: a timed CPU
 * baseline, TEST AND MEASUREMENT INFRASTRUCTURE ONLY.
 *
 * Not the oracle, and not part of the planner.  It is the CPU counterpart of
 * the paper's kernel-style timings (the Kern.CPU rows of Table 5): the same
 * layered relaxation as Section VIII.B-C (Insert 1), one maneuver layer after
 * another in the cycle order of Section XVI.A, with the curves of a layer
 * spread over OpenMP threads.  bench.py times it beside the single-threaded
 * oracle; tests/test_cpu_sweep.py checks its V and L against the oracle's
 * sweep, value for value and label for label.
 *
 * The geometry arrives as tables (beta, iflag, jsign, the straight-line
 * shear B(y', T), the step weights), computed by the caller from eqs. 11-24.
 *
 * Curves of a layer (Section V.C):
 *   turn      chain (x', y') walked from its heading-0 cell (x', y', 0): at
 *             step k it is at heading T_k = +-k and cell
 *             (x' + beta(T_k + a N/4) - beta(a N/4), y' + beta(T_k + b N/4) -
 *             beta(b N/4)), (a, b) = (0, 3) for left turns, (2, 1) for right
 *             turns (eqs. 18, 25-28).  The chain is a cycle of N_theta cells;
 *             it is walked twice, the second loop stores (Section VIII.C).
 *             A thread takes a whole row of chains (fixed y') in lockstep, so
 *             at each step it touches one row segment of one heading plane.
 *   straight  line k of plane T walked from its wall cell: shallow planes
 *             (I = 0) cell (i_s, k + B(i_s)), steep planes (I = 1) cell
 *             (k + B(j_s), j_s), with i_s (j_s) = +-s by eq. 24 (eqs. 23,
 *             30-31).  The wall row and column are hard, so what is carried
 *             into the wall cell never matters and one pass suffices.
 *             A thread takes a whole plane.
 * Every cell of a layer lies on exactly one curve, and a curve reads a cell
 * before it may write it, so the layer runs in place.
 *
 * Arithmetic: uint32 with PLAN_INF = 0xFFFFFFFF absorbing (saturating adds);
 * edge cost (w B) >> 8, INF for hard cells; strict improvements only; labels
 * (mu << 13) | d, d the steps since the entry.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#define CS_INF 0xFFFFFFFFu
#define CS_HARD 0xFFFFu
#define CS_NONE 0xFFFFu

enum { LF = 0, SF = 1, RB = 2, RF = 3, SB = 4, LB = 5 };

static inline uint32_t cs_add(uint32_t a, uint32_t b) {
    uint64_t s = (uint64_t)a + b;
    return s >= CS_INF ? CS_INF : (uint32_t)s;
}

static inline uint32_t cs_edge(uint16_t b, uint32_t w) {
    return b == CS_HARD ? CS_INF : (uint32_t)(((uint64_t)w * b) >> 8);
}

typedef struct {
    int lx, lt, nx, nt, mx, mt;
    const int32_t* beta;
    const uint8_t* iflag;
    const int8_t* jsign;
    const int32_t* bshear;
    const uint32_t* wS;
    uint32_t wA;
    const uint32_t* cin;
    const uint32_t* cout;
    const uint16_t* B;
    uint32_t* V;
    uint16_t* L;
} cs_ctx;

/* One step of a curve at cell x, position q: store when the carried value
 * (plus leaving) is strictly better, then enter or carry on. */
static inline void cs_step(const cs_ctx* c, int64_t x, int q, int store, int mu, uint32_t w, uint32_t* v,
                           int* qe, int64_t* nimp) {
    const uint16_t b = c->B[x];
    const int hard = b == CS_HARD;
    const uint32_t u = c->V[x];
    if (store) {
        const uint32_t cand = hard ? CS_INF : cs_add(*v, c->cout[mu]);
        if (cand < u) {
            c->V[x] = cand;
            c->L[x] = (uint16_t)((mu << 13) | (q - *qe));
            (*nimp)++;
        }
    }
    const uint32_t t = hard ? CS_INF : cs_add(u, c->cin[mu]);
    if (t < *v) {
        *v = t;
        *qe = q;
    }
    *v = cs_add(*v, cs_edge(b, w));
}

static int64_t cs_turn_layer(const cs_ctx* c, int mu) {
    const int n = c->nt, nx = c->nx, Q = c->nt / 4;
    const int a = (mu == LF || mu == LB) ? 0 : 2, bq = (mu == LF || mu == LB) ? 3 : 1;
    const int step = (mu == LF || mu == RB) ? 1 : -1;
    const int64_t nxy = (int64_t)nx * nx;
    int64_t nimp = 0;
#pragma omp parallel reduction(+ : nimp)
    {
        uint32_t* v = (uint32_t*)malloc(sizeof(uint32_t) * nx);
        int* qe = (int*)malloc(sizeof(int) * nx);
#pragma omp for schedule(dynamic, 4)
        for (int yq = 0; yq < nx; yq++) {
            for (int xq = 0; xq < nx; xq++) { v[xq] = CS_INF; qe[xq] = 0; }
            for (int q = 0; q < 2 * n; q++) {
                const int T = (step * q) & c->mt;
                const int di = c->beta[(T + a * Q) & c->mt] - c->beta[(a * Q) & c->mt];
                const int dj = c->beta[(T + bq * Q) & c->mt] - c->beta[(bq * Q) & c->mt];
                const int64_t row = (int64_t)T * nxy + ((int64_t)((yq + dj) & c->mx) << c->lx);
                for (int xq = 0; xq < nx; xq++)
                    cs_step(c, row + ((xq + di) & c->mx), q, q >= n, mu, c->wA, &v[xq], &qe[xq], &nimp);
            }
        }
        free(v);
        free(qe);
    }
    return nimp;
}

static int64_t cs_straight_layer(const cs_ctx* c, int mu) {
    const int nx = c->nx;
    const int64_t nxy = (int64_t)nx * nx;
    int64_t nimp = 0;
#pragma omp parallel reduction(+ : nimp)
    {
        uint32_t* v = (uint32_t*)malloc(sizeof(uint32_t) * nx);
        int* qe = (int*)malloc(sizeof(int) * nx);
#pragma omp for schedule(dynamic, 1)
        for (int T = 0; T < c->nt; T++) {
            const int plus = (c->jsign[T] >= 0) == (mu == SF);
            const int step = plus ? 1 : -1;
            const int32_t* Bs = c->bshear + (int64_t)T * nx;
            const uint32_t w = c->wS[T];
            const int64_t base = (int64_t)T * nxy;
            for (int k = 0; k < nx; k++) { v[k] = CS_INF; qe[k] = 0; }
            for (int s = 0; s < nx; s++) {
                const int y = (step * s) & c->mx;  /* y' along the line, from the wall cell */
                if (c->iflag[T] == 0) {
                    for (int k = 0; k < nx; k++)
                        cs_step(c, base + y + ((int64_t)((k + Bs[y]) & c->mx) << c->lx), s, 1, mu, w, &v[k], &qe[k],
                                &nimp);
                } else {
                    const int64_t row = base + ((int64_t)y << c->lx);
                    for (int k = 0; k < nx; k++)
                        cs_step(c, row + ((k + Bs[y]) & c->mx), s, 1, mu, w, &v[k], &qe[k], &nimp);
                }
            }
        }
        free(v);
        free(qe);
    }
    return nimp;
}

/* V, L: caller-owned volumes of nx*nx*nt cells (idx = x + nx*(y + nx*T)),
 * initialised here (V = INF but V[start] = 0, L = NONE).  improved[6N]
 * (optional) receives the strictly improved cells per layer.  threads <= 0:
 * the OpenMP default.  Returns the thread count used, or -1 on bad input. */
int cs_sweep(int nx_log2, int nt_log2, const int32_t* beta, const uint8_t* iflag, const int8_t* jsign,
             const int32_t* bshear, const uint32_t* wS, uint32_t wA, const uint32_t* cin, const uint32_t* cout,
             const uint16_t* B, int64_t start, int n_cycles, int threads, uint32_t* V, uint16_t* L,
             int64_t* improved) {
    if (nx_log2 < 2 || nx_log2 > 12 || nt_log2 < 2 || nt_log2 > 10 || n_cycles < 0) return -1;
    cs_ctx c;
    c.lx = nx_log2;
    c.lt = nt_log2;
    c.nx = 1 << nx_log2;
    c.nt = 1 << nt_log2;
    c.mx = c.nx - 1;
    c.mt = c.nt - 1;
    c.beta = beta;
    c.iflag = iflag;
    c.jsign = jsign;
    c.bshear = bshear;
    c.wS = wS;
    c.wA = wA;
    c.cin = cin;
    c.cout = cout;
    c.B = B;
    c.V = V;
    c.L = L;
    const int64_t nr = (int64_t)c.nx * c.nx * c.nt;
    if (start < 0 || start >= nr || B[start] == CS_HARD) return -1;
    int used = 1;
#ifdef _OPENMP
    if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
    }
#pragma omp parallel for schedule(static)
#endif
    for (int64_t x = 0; x < nr; x++) {
        V[x] = CS_INF;
        L[x] = CS_NONE;
    }
    V[start] = 0;
    static const int order[6] = {LF, SF, RB, RF, SB, LB};
    for (int l = 0; l < 6 * n_cycles; l++) {
        const int mu = order[l % 6];
        const int64_t n = (mu == SF || mu == SB) ? cs_straight_layer(&c, mu) : cs_turn_layer(&c, mu);
        if (improved) improved[l] = n;
    }
    return used;
}
