/*
 * nhp_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Plain, slow, single-threaded CPU oracle for the kernel-style N-turn sweep of
 * Nister et al., "Nonholonomic Motion Planning as Efficient as Piano Mover's"
 * (arXiv 2306.01301).  It exists to check the CUDA library bit for bit.  It
 * shares no code, header, table or constant with the library under
 * paper_2306_01301_b300/; only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline leg may load it.
 *
 * Conventions (all integer, all exact):
 *   cell index  idx = i + Nx*(j + Nx*T)   (i = x column, j = y row, T = heading)
 *   value INF   0xFFFFFFFF, saturating uint32 addition
 *   obstacle    uint16 Q8 reciprocal velocity, 256 = free, 0xFFFF = HARD
 *   label       (mu << 13) | d, NONE = 0xFFFF; mu is the cycle-order index
 *               LF=0 SF=1 RB=2 RF=3 SB=4 LB=5 (Section XVI.A), d = steps
 *               from the entry cell of the maneuver segment to this cell.
 */
#ifndef NHP_ORACLE_H
#define NHP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_ctx orc_ctx;

/* Grid + vehicle + cost description.  R in cells, costs in integer units. */
orc_ctx* orc_create(int nx_log2, int nt_log2, double R, int half_shift,
                    uint32_t step_straight, uint32_t step_scale, uint32_t ct);
void     orc_destroy(orc_ctx* c);
/* Per-maneuver Star transition edges (Section V.A, Fig. 9): T -> M_mu costs
 * cin[mu], M_mu -> T costs cout[mu]; by default cin = ct, cout = 0.  Every
 * function below uses them.  Returns -1 if some cin + cout >= 2^28. */
int      orc_set_transition(orc_ctx* c, const uint32_t* cin, const uint32_t* cout);

/* Geometry tables (Section V.C, eqs. 11-24).  Arrays are caller-owned:
 * beta[nt], psi2[nt] (2*Psi), iflag[nt], jsign[nt], bshear[nt*nx] (B(y',T) at
 * [T*nx + y']), wS[nt]; *wA gets the turn step weight. */
void orc_tables(const orc_ctx* c, int32_t* beta, uint8_t* psi2, uint8_t* iflag,
                int8_t* jsign, int32_t* bshear, uint32_t* wS, uint32_t* wA);

/* Footprint offsets of heading T (Section VI; rectangle read of Fig. 6):
 * writes up to cap (dx,dy) pairs, returns the count (or -needed if cap small). */
int orc_footprint(const orc_ctx* c, int front, int rear, int hw, int T,
                  int32_t* dx, int32_t* dy, int cap);

/* Obstacle volume B (Section VI), full volume or selected cells. */
int orc_render(const orc_ctx* c, const uint16_t* img, int front, int rear, int hw,
               uint16_t* B);
/* The same B computed row run by row run with sliding-window maxima
 * (Section VI's constant-cost max filter); used for large grids. */
int orc_render_rows(const orc_ctx* c, const uint16_t* img, int front, int rear,
                    int hw, uint16_t* B);
int orc_render_cells(const orc_ctx* c, const uint16_t* img, int front, int rear,
                     int hw, const int64_t* cells, int64_t n, uint16_t* out);

/* Successor of cell under maneuver mu (eqs. 25-28, 30-31). */
int64_t orc_succ(const orc_ctx* c, int mu, int64_t cell);

/* Edge weight leaving cell under maneuver mu (Section V.D + Insert 1). */
uint32_t orc_edge(const orc_ctx* c, const uint16_t* B, int mu, int64_t cell);

/* Layered relaxation (Section VIII.B), N cycles in the order of Section XVI.A.
 * mode 0: explicit Star-graph edge list, cycles found by pointer following;
 * mode 1: same relaxation, edges evaluated on the fly, chains in lockstep;
 * mode 2: explicit edge list, each cycle relaxed by the O(n^2) definition.
 * improved[6N] (optional) receives the number of strictly improved cells per
 * layer.  Returns 0, or -1 on bad input / allocation failure. */
int orc_sweep(const orc_ctx* c, const uint16_t* B, int64_t start, int n_cycles,
              int mode, uint32_t* V, uint16_t* L, int64_t* improved);

/* Host threads for mode 1 (default 1): independent chains of a layer run
 * on several threads; the results do not depend on the count. */
void orc_set_threads(int n);

/* Continue an existing (V, L) by more layers starting at layer index
 * first_layer (so first_layer % 6 selects the maneuver). */
int orc_layers(const orc_ctx* c, const uint16_t* B, int first_layer, int n_layers,
               int mode, uint32_t* V, uint16_t* L, int64_t* improved);

/* Full Dijkstra on the explicit Star graph (Section VIII.A): V_inf. */
int orc_dijkstra(const orc_ctx* c, const uint16_t* B, int64_t start, uint32_t* Vinf);

/* Exhaustive search over layer-ordered segment sequences (tiny grids). */
int orc_bruteforce(const orc_ctx* c, const uint16_t* B, int64_t start, int n_cycles,
                   uint32_t* Vbest);

/* Start state (Section XII): entry[mu] = cost of entering maneuver mu at the
 * start (<= cin[mu]).  orc_seed applies the start layer -- each maneuver with
 * entry[mu] < ct followed from the start alone -- to (V, L); orc_sweep_state
 * is orc_sweep with the start layer before the N cycles.  Dijkstra and the
 * exhaustive search with the start's transition edges weighted by entry. */
int orc_seed(const orc_ctx* c, const uint16_t* B, int64_t start, const uint32_t* entry,
             uint32_t* V, uint16_t* L);
int orc_sweep_state(const orc_ctx* c, const uint16_t* B, int64_t start, const uint32_t* entry,
                    int n_cycles, int mode, uint32_t* V, uint16_t* L, int64_t* improved);
int orc_dijkstra_state(const orc_ctx* c, const uint16_t* B, int64_t start, const uint32_t* entry,
                       uint32_t* Vinf);
int orc_bruteforce_state(const orc_ctx* c, const uint16_t* B, int64_t start, const uint32_t* entry,
                         int n_cycles, uint32_t* Vbest);
/* Gear states: two transition vertices per cell (forward / reverse gear of
 * the last maneuver); entering a maneuver of the other gear costs pen more.
 * V, L hold 2 * nr entries (forward state first); labels (mu << 13) |
 * (entered from the other state << 12) | d.  start_gear 0 forward, 1 reverse,
 * 2 at rest.  Sweep, Dijkstra, exhaustive search and label walk
 * (seg[k*7 + {mu, entry, exit, d, cost_lo16, cost_hi16, entry_gear}]). */
int orc_sweep_gear(const orc_ctx* c, const uint16_t* B, int64_t start, int start_gear, uint32_t pen,
                   int n_cycles, uint32_t* V, uint16_t* L);
int orc_dijkstra_gear(const orc_ctx* c, const uint16_t* B, int64_t start, int start_gear, uint32_t pen,
                      uint32_t* Vinf);
int orc_bruteforce_gear(const orc_ctx* c, const uint16_t* B, int64_t start, int start_gear, uint32_t pen,
                        int n_cycles, uint32_t* Vbest);
int orc_extract_gear(const orc_ctx* c, const uint32_t* V, const uint16_t* L, int64_t goal, int64_t* seg,
                     int cap);
/* Compact graph (Section V.A, Fig. 12): vertices S (straight = transition
 * state), L, R per cell; V, L hold 3 * nr entries (S, L, R); labels (mu <<
 * 13) | (entered from S << 12) | d.  Sweep (kernel-style layers), Dijkstra,
 * exhaustive search and the label walk from S(goal) (seg[k*6 + {mu, entry,
 * exit, d, cost, entered_from_S}]). */
int orc_sweep_compact(const orc_ctx* c, const uint16_t* B, int64_t start, int n_cycles, uint32_t* V,
                      uint16_t* L);
int orc_dijkstra_compact(const orc_ctx* c, const uint16_t* B, int64_t start, uint32_t* Vinf);
int orc_bruteforce_compact(const orc_ctx* c, const uint16_t* B, int64_t start, int n_cycles, uint32_t* Vbest);
int orc_extract_compact(const orc_ctx* c, const uint32_t* V, const uint16_t* L, int64_t goal, int64_t* seg,
                        int cap);
/* 4D generalisation (App. F): 2M+1 curvature levels of the 3D volume,
 * clothoid maneuvers between them (ids 6 C1F, 7 C1B, 8 C2F, 9 C2B), the 3D
 * turns at the steering limits and the straights at zero curvature.  4D
 * cells are K * nr + 3D cell (K = kappa + M); labels (mu << 12) | d.
 * orc4_tables: dx, dy [2][2M+1][N_theta], dth [2][2M+1].  Extract rows
 * seg[k*5 + {mu, entry4, exit4, d, cost}]. */
typedef struct orc4 orc4;
orc4*   orc4_create(const orc_ctx* c, int M, double L, uint32_t ct_clothoid);
void    orc4_destroy(orc4* q);
void    orc4_tables(const orc4* q, int16_t* dx, int16_t* dy, int32_t* dth);
int64_t orc4_succ(const orc4* q, int mu, int64_t cell4);
int     orc4_sweep(const orc4* q, const uint16_t* B, int64_t start4, int n_cycles, uint32_t* V, uint16_t* L);
int     orc4_dijkstra(const orc4* q, const uint16_t* B, int64_t start4, uint32_t* Vinf);
int     orc4_bruteforce(const orc4* q, const uint16_t* B, int64_t start4, int n_cycles, uint32_t* Vbest);
int     orc4_extract(const orc4* q, const uint32_t* V, const uint16_t* L, int64_t goal4, int64_t* seg, int cap);
/* Goal search over a goal set (Section IX): the reached pose minimising
 * V + bias + w_xy (|dx|+|dy|) + w_theta |dtheta| over every goal's box;
 * goals[g*8 + {x, y, theta, r_xy, r_theta, w_xy, w_theta, bias}].  Returns 0
 * (*cell, *score), -1 nothing reached, -2 malformed goal. */
int orc_goal_search(const orc_ctx* c, const uint32_t* V, const int64_t* goals, int n,
                    int64_t* cell, uint64_t* score);
/* Label walk from goal (Section X, forward tracking).  Writes segments in
 * driving order: seg[k*6 + {mu, entry, exit, d, cost_lo16, cost_hi16}] as
 * int64.  Returns segment count, -1 unreachable, -2 cap too small, -3
 * malformed labels. */
int orc_extract(const orc_ctx* c, const uint32_t* V, const uint16_t* L, int64_t goal,
                int64_t* seg, int cap);

/* Maneuver-count reachability (Appendix C, Insert 2): count[x] = fewest
 * maneuvers from start to x over hard obstacles only, every maneuver of a
 * cycle taken from the previous cycle's reachable set; 255 if more than
 * n_cycles.  Returns 0, or -1 for bad arguments / a hard start. */
int orc_reach(const orc_ctx* c, const uint16_t* B, int64_t start, int n_cycles, uint8_t* count);

/* Canonical back-track of a fewest-maneuver sequence to goal (driving
 * order, seg[k*4 + {mu, entry, exit, steps}]).  Returns the segment count,
 * -1 unreachable, -2 cap too small, -3 inconsistent counts. */
int orc_reach_extract(const orc_ctx* c, const uint16_t* B, const uint8_t* count, int64_t goal,
                      int64_t* seg, int cap);

/* Direction penalties (Section XVI, Fig. 19) on a rendered B: poses whose
 * heading is more than tol steps (circular) from their cell's preferred
 * heading (heading[j*Nx + i], 0xFFFF none) get B = min(B*pen/256, 0xFFFE);
 * hard stays hard.  Returns 0, -1 for bad arguments. */
int orc_direction(const orc_ctx* c, uint16_t* B, const uint16_t* heading, int tol, uint32_t pen);
/* Soft-obstacle image (Section VII): HARD where occ != 0, else 256 + pen with
 * pen = soft_max*(r2-d2)/r2 for squared Euclidean distance d2 < r2 to the
 * nearest occupied cell, else 256. */
void orc_soft_image(int nx, const uint8_t* occ, int radius, int soft_max, uint16_t* img);

#ifdef __cplusplus
}
#endif
#endif
