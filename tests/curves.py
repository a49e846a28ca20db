"""Closed-form shortest paths of the continuum vehicle in free space, written
for the tests from the published constructions (Appendix B, Theorems 2-3):

* Dubins (1957): forward only; a shortest path is one of LSL, RSR, LSR, RSL,
  RLR, LRL (Theorem 2).
* Reeds-Shepp (1990), with the family reduction of Sussmann-Tang (1991) the
  paper cites: forward and reverse; a shortest path is one of the CSC, CCC,
  CC|CC, C|CC|C, C|C_{pi/2}SC, CSC_{pi/2}|C and C|C_{pi/2}SC_{pi/2}|C words and
  their time-flipped and reflected variants (Theorem 3).

Formulation followed: the segment lengths (t, u, v) of the base words are
Reeds and Shepp's closed forms (section 8 of their paper, formulas 8.1 to
8.11), named here in their word notation with p/m for the + and - gears
(L+S+L+ is `_LpSpLp`, L+R-L is `_LpRmL`, ...), with the helper that both
four-arc words share (`_tau_omega`); every other word follows from a base
word by the time-flip, reflection and backwards symmetries of their section
7.  Base words plus symmetries is also how the common open-source
implementations of Reeds-Shepp curves organise the computation, so the
layout below resembles them; the formulas are the paper's.  The Dubins words
are the six tangent constructions of Dubins (1957) in the normalised frame
(start at the origin, goal at distance d on the x axis).

Lengths are in units of the turn radius; `*_path` functions return the
shortest word as a list of (kind, signed length) segments with kind in
{"L", "R", "S"} and the sign giving the gear, so that tests can also drive
the path forward and count its maneuvers.  Pure Python and math only: the
oracle and the library share none of this code.
"""
from __future__ import annotations

import math

PI = math.pi
EPS = 1e-10


def mod2pi(x: float) -> float:
    """Angle in [-pi, pi)."""
    v = math.fmod(x, 2 * PI)
    if v < -PI:
        v += 2 * PI
    elif v >= PI:
        v -= 2 * PI
    return v


def polar(x: float, y: float):
    return math.hypot(x, y), math.atan2(y, x)


# ------------------------------------------------------------------ Dubins
def _dubins_words(alpha: float, beta: float, d: float):
    """Candidate (word, t, p, q) in the normalised frame (start at the
    origin heading alpha, goal at (d, 0) heading beta)."""
    sa, sb, ca, cb = math.sin(alpha), math.sin(beta), math.cos(alpha), math.cos(beta)
    cab = math.cos(alpha - beta)
    out = []
    # LSL
    p2 = 2 + d * d - 2 * cab + 2 * d * (sa - sb)
    if p2 >= 0:
        tmp = math.atan2(cb - ca, d + sa - sb)
        out.append(("LSL", (tmp - alpha) % (2 * PI), math.sqrt(p2), (beta - tmp) % (2 * PI)))
    # RSR
    p2 = 2 + d * d - 2 * cab + 2 * d * (sb - sa)
    if p2 >= 0:
        tmp = math.atan2(ca - cb, d - sa + sb)
        out.append(("RSR", (alpha - tmp) % (2 * PI), math.sqrt(p2), (tmp - beta) % (2 * PI)))
    # LSR
    p2 = -2 + d * d + 2 * cab + 2 * d * (sa + sb)
    if p2 >= 0:
        p = math.sqrt(p2)
        tmp = math.atan2(-ca - cb, d + sa + sb) - math.atan2(-2.0, p)
        out.append(("LSR", (tmp - alpha) % (2 * PI), p, (tmp - beta) % (2 * PI)))
    # RSL
    p2 = -2 + d * d + 2 * cab - 2 * d * (sa + sb)
    if p2 >= 0:
        p = math.sqrt(p2)
        tmp = math.atan2(ca + cb, d - sa - sb) - math.atan2(2.0, p)
        out.append(("RSL", (alpha - tmp) % (2 * PI), p, (beta - tmp) % (2 * PI)))
    # RLR
    c = (6.0 - d * d + 2 * cab + 2 * d * (sa - sb)) / 8.0
    if abs(c) <= 1:
        p = (2 * PI - math.acos(c)) % (2 * PI)
        t = (alpha - math.atan2(ca - cb, d - sa + sb) + p / 2) % (2 * PI)
        out.append(("RLR", t, p, (alpha - beta - t + p) % (2 * PI)))
    # LRL
    c = (6.0 - d * d + 2 * cab + 2 * d * (sb - sa)) / 8.0
    if abs(c) <= 1:
        p = (2 * PI - math.acos(c)) % (2 * PI)
        t = (-alpha - math.atan2(ca - cb, d + sa - sb) + p / 2) % (2 * PI)
        out.append(("LRL", t, p, ((beta - alpha) - t + p) % (2 * PI)))
    return out


def dubins_path(q0, q1, R: float):
    """Shortest forward-only path from q0 = (x, y, theta) to q1."""
    dx, dy = q1[0] - q0[0], q1[1] - q0[1]
    D = math.hypot(dx, dy)
    d = D / R
    th = math.atan2(dy, dx) if D > 0 else 0.0
    alpha, beta = (q0[2] - th) % (2 * PI), (q1[2] - th) % (2 * PI)
    best = None
    for word, t, p, q in _dubins_words(alpha, beta, d):
        L = t + p + q
        if best is None or L < best[0]:
            best = (L, [(word[0], t * R), (word[1], p * R), (word[2], q * R)])
    return best[1]


# ------------------------------------------------------------- Reeds-Shepp
def _tau_omega(u, v, xi, eta, phi):
    delta = mod2pi(u - v)
    A = math.sin(u) - math.sin(delta)
    B = math.cos(u) - math.cos(delta) - 1
    t1 = math.atan2(eta * A - xi * B, xi * A + eta * B)
    t2 = 2 * (math.cos(delta) - math.cos(v) - math.cos(u)) + 3
    tau = mod2pi(t1 + PI) if t2 < 0 else mod2pi(t1)
    omega = mod2pi(tau - u + v - phi)
    return tau, omega


def _LpSpLp(x, y, phi):
    u, t = polar(x - math.sin(phi), y - 1 + math.cos(phi))
    if t >= -EPS:
        v = mod2pi(phi - t)
        if v >= -EPS:
            return t, u, v
    return None


def _LpSpRp(x, y, phi):
    u1, t1 = polar(x + math.sin(phi), y - 1 - math.cos(phi))
    u1 = u1 * u1
    if u1 >= 4:
        u = math.sqrt(u1 - 4)
        theta = math.atan2(2, u)
        t = mod2pi(t1 + theta)
        v = mod2pi(t - phi)
        if t >= -EPS and v >= -EPS:
            return t, u, v
    return None


def _LpRmL(x, y, phi):
    xi, eta = x - math.sin(phi), y - 1 + math.cos(phi)
    u1, theta = polar(xi, eta)
    if u1 <= 4:
        u = -2 * math.asin(u1 / 4)
        t = mod2pi(theta + u / 2 + PI)
        v = mod2pi(phi - t + u)
        if t >= -EPS and u <= EPS:
            return t, u, v
    return None


def _LpRupLumRm(x, y, phi):
    xi, eta = x + math.sin(phi), y - 1 - math.cos(phi)
    rho = 0.25 * (2 + math.hypot(xi, eta))
    if rho <= 1:
        u = math.acos(rho)
        t, v = _tau_omega(u, -u, xi, eta, phi)
        if t >= -EPS and v <= EPS:
            return t, u, v
    return None


def _LpRumLumRp(x, y, phi):
    xi, eta = x + math.sin(phi), y - 1 - math.cos(phi)
    rho = (20 - xi * xi - eta * eta) / 16
    if 0 <= rho <= 1:
        u = -math.acos(rho)
        if u >= -PI / 2:
            t, v = _tau_omega(u, u, xi, eta, phi)
            if t >= -EPS and v >= -EPS:
                return t, u, v
    return None


def _LpRmSmLm(x, y, phi):
    xi, eta = x - math.sin(phi), y - 1 + math.cos(phi)
    rho, theta = polar(xi, eta)
    if rho >= 2:
        r = math.sqrt(rho * rho - 4)
        u = 2 - r
        t = mod2pi(theta + math.atan2(r, -2))
        v = mod2pi(phi - PI / 2 - t)
        if t >= -EPS and u <= EPS and v <= EPS:
            return t, u, v
    return None


def _LpRmSmRm(x, y, phi):
    xi, eta = x + math.sin(phi), y - 1 - math.cos(phi)
    rho, theta = polar(-eta, xi)
    if rho >= 2:
        t = theta
        u = 2 - rho
        v = mod2pi(t + PI / 2 - phi)
        if t >= -EPS and u <= EPS and v <= EPS:
            return t, u, v
    return None


def _LpRmSLmRp(x, y, phi):
    xi, eta = x + math.sin(phi), y - 1 - math.cos(phi)
    rho, _ = polar(xi, eta)
    if rho >= 2:
        u = 4 - math.sqrt(rho * rho - 4)
        if u <= EPS:
            t = mod2pi(math.atan2((4 - u) * xi - 2 * eta, -2 * xi + (u - 4) * eta))
            v = mod2pi(t - phi)
            if t >= -EPS and v >= -EPS:
                return t, u, v
    return None


def _flip(word):  # time flip: every gear reversed
    return [(k, -s) for k, s in word]


def _reflect(word):  # reflect: left and right exchanged
    return [({"L": "R", "R": "L"}.get(k, k), s) for k, s in word]


def _candidates(x, y, phi):
    """All Reeds-Shepp words reaching (x, y, phi) from the origin (unit radius)."""
    out = []

    def add(fn, shape, xx, yy, pp, flip, refl, backwards=False):
        r = fn(xx, yy, pp)
        if r is None:
            return
        t, u, v = r
        word = shape(t, u, v)
        if backwards:
            word = list(reversed(word))
        if flip:
            word = _flip(word)
        if refl:
            word = _reflect(word)
        out.append(word)

    sym = [(x, y, phi, False, False), (-x, y, -phi, True, False), (x, -y, -phi, False, True),
           (-x, -y, phi, True, True)]
    xb = x * math.cos(phi) + y * math.sin(phi)
    yb = x * math.sin(phi) - y * math.cos(phi)
    symb = [(xb, yb, phi, False, False), (-xb, yb, -phi, True, False), (xb, -yb, -phi, False, True),
            (-xb, -yb, phi, True, True)]
    for xx, yy, pp, f, r in sym:  # CSC
        add(_LpSpLp, lambda t, u, v: [("L", t), ("S", u), ("L", v)], xx, yy, pp, f, r)
        add(_LpSpRp, lambda t, u, v: [("L", t), ("S", u), ("R", v)], xx, yy, pp, f, r)
    for xx, yy, pp, f, r in sym:  # CCC
        add(_LpRmL, lambda t, u, v: [("L", t), ("R", u), ("L", v)], xx, yy, pp, f, r)
    for xx, yy, pp, f, r in symb:
        add(_LpRmL, lambda t, u, v: [("L", t), ("R", u), ("L", v)], xx, yy, pp, f, r, backwards=True)
    for xx, yy, pp, f, r in sym:  # CCCC
        add(_LpRupLumRm, lambda t, u, v: [("L", t), ("R", u), ("L", -u), ("R", v)], xx, yy, pp, f, r)
        add(_LpRumLumRp, lambda t, u, v: [("L", t), ("R", u), ("L", u), ("R", v)], xx, yy, pp, f, r)
    for xx, yy, pp, f, r in sym:  # CCSC
        add(_LpRmSmLm, lambda t, u, v: [("L", t), ("R", -PI / 2), ("S", u), ("L", v)], xx, yy, pp, f, r)
        add(_LpRmSmRm, lambda t, u, v: [("L", t), ("R", -PI / 2), ("S", u), ("R", v)], xx, yy, pp, f, r)
    for xx, yy, pp, f, r in symb:
        add(_LpRmSmLm, lambda t, u, v: [("L", t), ("R", -PI / 2), ("S", u), ("L", v)], xx, yy, pp, f, r,
            backwards=True)
        add(_LpRmSmRm, lambda t, u, v: [("L", t), ("R", -PI / 2), ("S", u), ("R", v)], xx, yy, pp, f, r,
            backwards=True)
    for xx, yy, pp, f, r in sym:  # CCSCC
        add(_LpRmSLmRp, lambda t, u, v: [("L", t), ("R", -PI / 2), ("S", u), ("L", -PI / 2), ("R", v)],
            xx, yy, pp, f, r)
    return out


def reeds_shepp_path(q0, q1, R: float):
    """Shortest path with reversals from q0 = (x, y, theta) to q1, as
    (kind, signed length) segments (lengths in the units of the input)."""
    dx, dy = q1[0] - q0[0], q1[1] - q0[1]
    c, s = math.cos(q0[2]), math.sin(q0[2])
    x, y = (c * dx + s * dy) / R, (-s * dx + c * dy) / R
    phi = q1[2] - q0[2]
    best, bestL = None, math.inf
    for word in _candidates(x, y, phi):
        L = sum(abs(v) for _, v in word)
        if L < bestL:
            best, bestL = word, L
    return [(k, v * R) for k, v in best]


def length(path) -> float:
    return sum(abs(v) for _, v in path)


def maneuvers(path, tol=1e-9) -> int:
    """Maneuvers of a path: maximal runs of the same kind and gear, zero-length
    segments dropped."""
    m, last = 0, None
    for k, v in path:
        if abs(v) <= tol:
            continue
        key = (k, v > 0)
        if key != last:
            m += 1
            last = key
    return m


def drive(q, path, R: float):
    """End pose of a path driven from q: L/R arcs of radius R (signed arc
    length: + forward), S straight."""
    x, y, th = q
    for k, v in path:
        if k == "S":
            x, y = x + v * math.cos(th), y + v * math.sin(th)
            continue
        ang = v / R  # signed turned angle for forward motion on a left arc
        if k == "L":
            cx, cy = x - R * math.sin(th), y + R * math.cos(th)
            th = th + ang
            x, y = cx + R * math.sin(th), cy - R * math.cos(th)
        else:
            cx, cy = x + R * math.sin(th), y - R * math.cos(th)
            th = th - ang
            x, y = cx - R * math.sin(th), cy + R * math.cos(th)
    return x, y, th
