// footprint.h -- host-side geometry shared by plan_create and the
// allocation-free renderer (private): the eq. 13 half-cell shift and the
// vehicle footprint's row runs.
#pragma once
#include <math.h>

#include <algorithm>

#include "internal.h"

namespace nhp {

// Section V.C, eqs. 11-13: beta(T) = floor(zeta(R sin theta)) and the
// residual Psi(T) = zeta - beta in {0, 1/2}, with zeta(x) = round(2x)/2
// (round half away from zero); psi2 = 2 Psi.  Without the half shift beta is
// the plainly rounded sinusoid and Psi = 0.  Either output may be null.
inline void shift_tables(double R, int nt, bool half, int* beta, int* psi2) {
    const double kPi = 3.14159265358979323846;
    for (int T = 0; T < nt; T++) {
        const double alpha = R * sin((2.0 * kPi) * (double)T / (double)nt);
        int b, q = 0;
        if (half) {
            const long z = lround(2.0 * alpha);
            b = (int)(z >= 0 ? z / 2 : -((-z + 1) / 2));
            q = (int)(z & 1);
        } else {
            b = (int)lround(alpha);
        }
        if (beta) beta[T] = b;
        if (psi2) psi2[T] = q;
    }
}

// Footprint (Section VI, Fig. 6): the closed rectangle [-rear, front] x
// [-hw, hw] in vehicle coordinates, placed at the continuum pose of eq. 16
// (i + Psi_0, j + Psi_1, theta), Psi_0(T) = psi2[T]/2, Psi_1(T) =
// psi2[T + N_theta/4]/2.  World cell (i+dx, j+dy) is covered when its centre
// lies in the rectangle (1e-9-cell tolerance, so exact multiples of 90
// degrees keep their edge cells); the cell under the origin is always
// covered.  Heading by heading, row by row: cell(dx, dy) for every covered
// cell, run(Run) for every maximal run of a row (the sparse-table windows
// of render.cu: level lvl with windows at lo and hi2), end(T) after each
// heading.  `row` holds reach_width(f) flags.  Returns false when a callback
// does.
inline int reach_width(const plan_footprint& f) {
    const int ext = std::max(f.front, f.rear);
    return 2 * ((int)ceil(sqrt((double)ext * ext + (double)f.half_width * f.half_width)) + 2) + 1;
}

template <class CellFn, class RunFn, class EndFn>
bool footprint_rows(int lx, int nt, const plan_footprint& f, const int* psi2, char* row, CellFn&& cell,
                    RunFn&& run, EndFn&& end) {
    const double kPi = 3.14159265358979323846;
    const int nx = 1 << lx;
    const int lim = (reach_width(f) - 1) / 2;
    const double eps = 1e-9;
    for (int T = 0; T < nt; T++) {
        const double th = (2.0 * kPi) * (double)T / (double)nt;
        const double c = cos(th), s = sin(th);
        const double px0 = 0.5 * psi2[T], py0 = 0.5 * psi2[(T + nt / 4) % nt];
        for (int dy = -lim; dy <= lim; dy++) {
            for (int dx = -lim; dx <= lim; dx++) {
                bool in = dx == 0 && dy == 0;
                if (!in) {
                    const double ax = (double)dx - px0, ay = (double)dy - py0;
                    const double xv = c * ax + s * ay, yv = -s * ax + c * ay;
                    in = xv >= -(double)f.rear - eps && xv <= (double)f.front + eps &&
                         yv >= -(double)f.half_width - eps && yv <= (double)f.half_width + eps;
                }
                row[dx + lim] = in;
                if (in && !cell(dx, dy)) return false;
            }
            for (int a = 0; a <= 2 * lim;) {
                if (!row[a]) { a++; continue; }
                int b = a;
                while (b + 1 <= 2 * lim && row[b + 1]) b++;
                const int lo = a - lim, hi = b - lim, w = hi - lo + 1;
                Run r;
                r.dy = (int16_t)dy;
                r.lo = (int16_t)lo;
                if (w >= nx) {  // covers the whole (cyclic) row
                    r.lvl = (int16_t)lx;
                    r.hi2 = (int16_t)lo;
                } else {
                    int lvl = 0;
                    while ((2 << lvl) <= w) lvl++;
                    r.lvl = (int16_t)lvl;
                    r.hi2 = (int16_t)(hi - (1 << lvl) + 1);
                }
                if (!run(r)) return false;
                a = b + 1;
            }
        }
        if (!end(T)) return false;
    }
    return true;
}

}  // namespace nhp
