"""Scheme algebra of the paper -- TEST INFRASTRUCTURE ONLY.

The paper describes every 2-D lifting scheme as a chain of 4x4 polyphase
matrices of bivariate Laurent polynomials acting on the quadruple
x = [LL, HL, LH, HH]^T (Sec. 2.3-2.4), separated by barriers "|".  This
module writes those matrices down (Sec. 2.5 Sweldens, Sec. 2.6 Iwahashi,
Sec. 3.1 Explosive, Sec. 3.2 Monolithic, Sec. 2.3 Polyphase, Sec. 4 the
starred variants) so that tests can check, independently of any kernel:

  * the operation and barrier counts of the paper's Table
    "Number of operations and memory barriers" (Sec. 5);
  * S_U T_P = N_{P,U} (Sec. 3.2) and that every scheme's product equals the
    separable Sweldens product;
  * applying a scheme's matrices, one step at a time, to a symmetrically
    extended image gives the separable oracle's result.

Polynomial convention.  A monomial c*z^e applied to a polyphase component X
at index i reads c*X[i+e]; z_m is the horizontal variable, z_n the vertical
one (Sec. 2, Eq. of H(z_m,z_n)), and X* denotes the transposed filter.  The
quadruple (n, m) holds samples rows 2n..2n+1 x columns 2m..2m+1, so the
predict reads the even neighbours at offsets 0 and +1 and the update reads
the odd neighbours at -1 and 0.  This is the paper's P = -1/2(1+z^-1),
U = 1/4(1+z) with H placed after L (the JPEG 2000 origin), i.e. z -> 1/z;
every count and identity below is unchanged by that relabelling.
"""
from __future__ import annotations

from fractions import Fraction
from typing import Dict, List, Sequence, Tuple

Mono = Tuple[int, int]  # (vertical exponent, horizontal exponent)


class LP:
    """Bivariate Laurent polynomial: {(ev, eh): coefficient}."""

    __slots__ = ("t",)

    def __init__(self, terms: Dict[Mono, object] | None = None):
        self.t = {k: v for k, v in (terms or {}).items() if v != 0}

    @staticmethod
    def const(c) -> "LP":
        return LP({(0, 0): c})

    def __add__(self, o: "LP") -> "LP":
        r = dict(self.t)
        for k, v in o.t.items():
            r[k] = r.get(k, 0) + v
        return LP(r)

    def __neg__(self) -> "LP":
        return LP({k: -v for k, v in self.t.items()})

    def __sub__(self, o: "LP") -> "LP":
        return self + (-o)

    def __mul__(self, o: "LP") -> "LP":
        r: Dict[Mono, object] = {}
        for (a1, b1), v1 in self.t.items():
            for (a2, b2), v2 in o.t.items():
                k = (a1 + a2, b1 + b2)
                r[k] = r.get(k, 0) + v1 * v2
        return LP(r)

    def nterms(self, tol: float = 0.0) -> int:
        return sum(1 for v in self.t.values() if abs(v) > tol)

    def close(self, o: "LP", tol: float) -> bool:
        keys = set(self.t) | set(o.t)
        return all(abs(self.t.get(k, 0) - o.t.get(k, 0)) <= tol for k in keys)


ZERO = LP()
ONE = LP.const(1)


def horiz(taps: Dict[int, object]) -> LP:
    """1-D operator along z_m (horizontal), e.g. P."""
    return LP({(0, e): c for e, c in taps.items()})


def vert(taps: Dict[int, object]) -> LP:
    """The transposed operator along z_n (vertical), e.g. P*."""
    return LP({(e, 0): c for e, c in taps.items()})


Mat = List[List[LP]]


def eye() -> Mat:
    return [[ONE if i == j else ZERO for j in range(4)] for i in range(4)]


def matmul(a: Mat, b: Mat) -> Mat:
    r = [[ZERO] * 4 for _ in range(4)]
    for i in range(4):
        for j in range(4):
            s = ZERO
            for k in range(4):
                if a[i][k].t and b[k][j].t:
                    s = s + a[i][k] * b[k][j]
            r[i][j] = s
    return r


def with_entries(entries: Dict[Tuple[int, int], LP]) -> Mat:
    m = eye()
    for (i, j), v in entries.items():
        m[i][j] = v
    return m


LL, HL, LH, HH = 0, 1, 2, 3


# ---------------------------------------------------------------------------
# Wavelets (Sec. 5), in the convention of the module docstring.  Each is a
# list of (P taps, U taps) pairs, plus the scaling of the low / high band.
# ---------------------------------------------------------------------------

def cdf53():
    h = Fraction(1, 2)
    q = Fraction(1, 4)
    return [({0: -h, 1: -h}, {-1: q, 0: q})]


def cdf97(alpha, beta, gamma, delta):
    return [({0: alpha, 1: alpha}, {-1: beta, 0: beta}),
            ({0: gamma, 1: gamma}, {-1: delta, 0: delta})]


def dd137():
    return [({-1: Fraction(1, 16), 0: Fraction(-9, 16), 1: Fraction(-9, 16), 2: Fraction(1, 16)},
             {-2: Fraction(-1, 32), -1: Fraction(9, 32), 0: Fraction(9, 32), 1: Fraction(-1, 32)})]


def split0(taps: Dict[int, object]):
    """Scalar split of Sec. 4: X = X0 + X1 with X0 the z^0 monomial."""
    x0 = {0: taps[0]} if taps.get(0, 0) != 0 else {}
    x1 = {e: c for e, c in taps.items() if e != 0}
    return x0, x1


# ---------------------------------------------------------------------------
# The step matrices.  p, u are 1-D tap dicts; X = horiz(x), X* = vert(x).
# ---------------------------------------------------------------------------

def T_H(p):  # Sec. 2.5, T^H_P
    P = horiz(p)
    return with_entries({(HL, LL): P, (HH, LH): P})


def T_V(p):  # T^V_P
    Ps = vert(p)
    return with_entries({(LH, LL): Ps, (HH, HL): Ps})


def S_H(u):  # S^H_U
    U = horiz(u)
    return with_entries({(LL, HL): U, (LH, HH): U})


def S_V(u):  # S^V_U
    Us = vert(u)
    return with_entries({(LL, LH): Us, (HL, HH): Us})


def T_I(p):  # Sec. 2.6, T^I_P
    P, Ps = horiz(p), vert(p)
    return with_entries({(HH, LL): P * Ps, (HH, HL): Ps, (HH, LH): P})


def R_I(p, u):  # R^I_{P,U}
    return with_entries({(HL, LL): horiz(p), (HL, HH): vert(u),
                         (LH, LL): vert(p), (LH, HH): horiz(u)})


def S_I(u):  # S^I_U
    U, Us = horiz(u), vert(u)
    return with_entries({(LL, HL): U, (LL, LH): Us, (LL, HH): -(U * Us)})


def T_E(p):  # Sec. 3.1, T^E_P
    P, Ps = horiz(p), vert(p)
    return with_entries({(HL, LL): P, (LH, LL): Ps, (HH, LL): -(P * Ps)})


def R_E(p, u):  # R^E_{P,U}
    return with_entries({(LL, HL): horiz(u), (LL, LH): vert(u),
                         (HH, HL): vert(p), (HH, LH): horiz(p)})


def S_E(u):  # S^E_U
    U, Us = horiz(u), vert(u)
    return with_entries({(LL, HH): U * Us, (HL, HH): Us, (LH, HH): U})


def T_M(p):  # Sec. 3.2, T_P (Monolithic predict)
    P, Ps = horiz(p), vert(p)
    return with_entries({(HL, LL): P, (LH, LL): Ps, (HH, LL): P * Ps, (HH, HL): Ps, (HH, LH): P})


def S_M(u):  # S_U (Monolithic update)
    U, Us = horiz(u), vert(u)
    return with_entries({(LL, HL): U, (LL, LH): Us, (LL, HH): U * Us, (HL, HH): Us, (LH, HH): U})


def N_PU(p, u):  # Sec. 2.3, the Polyphase matrix with V = PU + 1
    P, Ps, U, Us = horiz(p), vert(p), horiz(u), vert(u)
    V, Vs = P * U + ONE, Ps * Us + ONE
    return [[Vs * V, Vs * U, Us * V, Us * U],
            [Vs * P, Vs, Us * P, Us],
            [Ps * V, Ps * U, V, U],
            [Ps * P, Ps, P, ONE]]


def scaling(slo, shi) -> Mat:
    m = [[ZERO] * 4 for _ in range(4)]
    for i, s in enumerate((slo * slo, shi * slo, slo * shi, shi * shi)):
        m[i][i] = LP.const(s)
    return m


# ---------------------------------------------------------------------------
# Schemes: for one predict/update pair, a list of segments; a segment is
# (barrier_before, [matrices in the order they are applied]).
# ---------------------------------------------------------------------------

SCHEMES = ["Sweldens", "Iwahashi", "Iwahashi*", "Explosive", "Explosive*",
           "Monolithic", "Monolithic*", "Polyphase", "Polyphase*", "Convolution"]


def scheme_pair(name: str, p, u) -> List[Tuple[bool, List[Mat]]]:
    p0, p1 = split0(p)
    u0, u1 = split0(u)
    if name == "Sweldens":  # y = S^V_U | S^H_U | T^V_P | T^H_P | x
        return [(True, [T_H(p)]), (True, [T_V(p)]), (True, [S_H(u)]), (True, [S_V(u)])]
    if name == "Iwahashi":  # y = S^I_U | R^I | T^I_P | x
        return [(True, [T_I(p)]), (True, [R_I(p, u)]), (True, [S_I(u)])]
    if name == "Iwahashi*":  # y = S^V_U0 S^H_U0 S^I_U1 | R^I | T^I_P1 | T^V_P0 T^H_P0 x
        return [(False, [T_H(p0), T_V(p0)]), (True, [T_I(p1)]), (True, [R_I(p1, u1)]),
                (True, [S_I(u1), S_H(u0), S_V(u0)])]
    if name == "Explosive":  # y = S^E_U | R^E | T^E_P | x
        return [(True, [T_E(p)]), (True, [R_E(p, u)]), (True, [S_E(u)])]
    if name == "Explosive*":
        return [(False, [T_H(p0), T_V(p0)]), (True, [T_E(p1)]), (True, [R_E(p1, u1)]),
                (True, [S_E(u1), S_H(u0), S_V(u0)])]
    if name == "Monolithic":  # y = S_U | T_P | x
        return [(True, [T_M(p)]), (True, [S_M(u)])]
    if name == "Monolithic*":
        # y = S^V_U0 S^H_U0 S_U1 | T^V_P0 T^H_P0 T_P1 x, with the initial
        # barrier after the load implied (the Table counts two barriers).
        return [(True, [T_M(p1), T_H(p0), T_V(p0)]), (True, [S_M(u1), S_H(u0), S_V(u0)])]
    if name == "Polyphase":  # y = N | x
        return [(True, [N_PU(p, u)])]
    if name == "Polyphase*":  # y = S^V_U0 S^H_U0 N_{P1,U1} | T^V_P0 T^H_P0 x
        return [(False, [T_H(p0), T_V(p0)]), (True, [N_PU(p1, u1)]), (False, [S_H(u0), S_V(u0)])]
    raise KeyError(name)


def product(mats: Sequence[Mat]) -> Mat:
    """Matrix of applying ``mats`` in order (the first is applied first)."""
    r = eye()
    for m in mats:
        r = matmul(m, r)
    return r


def scheme_matrices(name: str, pairs) -> List[Mat]:
    out: List[Mat] = []
    for p, u in pairs:
        for _, seg in scheme_pair(name, p, u):
            out.extend(seg)
    return out


def full_matrix(pairs) -> Mat:
    """The unscaled 2-D polyphase matrix of the transform (separable)."""
    return product(scheme_matrices("Sweldens", pairs))


def _count_minus_identity(m: Mat, tol: float) -> int:
    n = 0
    for i in range(4):
        for j in range(4):
            e = m[i][j] - ONE if i == j else m[i][j]
            n += e.nterms(tol)
    return n


def op_count(name: str, pairs, tol: float = 1e-12) -> int:
    """MAC count per quadruple (scaling omitted, Sec. 5): the monomials of
    every step matrix minus its identity; Convolution counts every monomial
    of the full matrix (the four 2-D FIR filters)."""
    if name == "Convolution":
        m = full_matrix(pairs)
        return sum(m[i][j].nterms(tol) for i in range(4) for j in range(4))
    return sum(_count_minus_identity(m, tol) for m in scheme_matrices(name, pairs))


def barrier_count(name: str, npairs: int) -> int:
    """Barriers of the scheme; connected schemes add theirs (Sec. 4), except
    that Convolution is one filtering step with one initial barrier."""
    if name == "Convolution":
        return 1
    per = sum(1 for b, _ in scheme_pair(name, {0: 1, 1: 1}, {-1: 1, 0: 1}) if b)
    return per * npairs


# ---------------------------------------------------------------------------
# Applying matrices to images (polyphase components of a WSS-extended image)
# ---------------------------------------------------------------------------

def apply_matrix(m: Mat, comps, margin: int):
    """comps: four numpy arrays (LL, HL, LH, HH) on the same quad grid, with
    ``margin`` quads of extension on every side.  Returns the four outputs;
    entries within the stencil reach of the edge are not meaningful."""
    import numpy as np
    H, W = comps[0].shape
    out = []
    for i in range(4):
        acc = np.zeros((H, W))
        for j in range(4):
            for (ev, eh), c in m[i][j].t.items():
                shifted = np.zeros((H, W))
                ys = slice(max(0, -ev), min(H, H - ev))
                xs = slice(max(0, -eh), min(W, W - eh))
                yd = slice(max(0, ev), min(H, H + ev))
                xd = slice(max(0, eh), min(W, W + eh))
                shifted[ys, xs] = comps[j][yd, xd]
                acc += float(c) * shifted
        out.append(acc)
    return out
