"""Exact Riemann solver for the ideal ultra-relativistic (conformal) fluid,
eps = 3P, with a passively conserved particle density n.

TEST INFRASTRUCTURE ONLY.  Sec. III of the paper validates the inviscid limit
of the method against the analytic solution of the relativistic Riemann
problem; this module computes that solution so the oracle can be pinned to
it.  It is derived here from the conservation laws, not taken from a code:

* shock between states a (upstream) and b (downstream): the relative velocity
  of the two fluids is v_ab^2 = (P_b - P_a)(e_b - e_a) / ((e_a + P_b)(e_b + P_a)),
  which for e = 3P is 3 (P_b - P_a)^2 / ((3 P_a + P_b)(3 P_b + P_a)); the
  shock moves relative to the upstream fluid at
  V^2 = (P_b - P_a)(e_b + P_a) / ((e_b - e_a)(e_a + P_b)) = (3 P_b + P_a) / (3 (3 P_a + P_b));
  n follows from the continuity of n gamma (v - v_shock).
* rarefaction: sound speed c_s = 1/sqrt(3); the Riemann invariants are
  J+- = artanh(v) +- (sqrt(3)/4) ln P; the fan is self-similar with
  x/t = (v -+ c_s)/(1 -+ v c_s); n ~ P^(3/4) (isentropic, n ~ s ~ T^3).
* the star pressure P* is found by bisection on v*_left(P) = v*_right(P).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

CS = 1.0 / np.sqrt(3.0)


def _add(a, b):
    return (a + b) / (1.0 + a * b)


def _vrel(Pa, Pb):
    return np.sqrt(3.0 * (Pb - Pa) ** 2 / ((3.0 * Pa + Pb) * (3.0 * Pb + Pa)))


def _vshock_rel(Pa, Pb):
    """shock speed relative to the upstream fluid a, with downstream pressure Pb"""
    return np.sqrt((3.0 * Pb + Pa) / (3.0 * (3.0 * Pa + Pb)))


def _v_left_star(P, PL, vL):
    if P <= PL:
        return np.tanh(np.arctanh(vL) + np.sqrt(3.0) / 4.0 * np.log(PL / P))
    return _add(vL, -_vrel(PL, P))


def _v_right_star(P, PR, vR):
    if P <= PR:
        return np.tanh(np.arctanh(vR) - np.sqrt(3.0) / 4.0 * np.log(PR / P))
    return _add(vR, _vrel(PR, P))


def _gamma(v):
    return 1.0 / np.sqrt(1.0 - v * v)


@dataclass
class RiemannSolution:
    PL: float
    vL: float
    nL: float
    PR: float
    vR: float
    nR: float
    Pstar: float
    vstar: float
    nLstar: float
    nRstar: float
    left_kind: str          # "shock" or "rarefaction"
    right_kind: str
    left_speeds: tuple      # (head, tail) or (shock, shock)
    right_speeds: tuple

    def sample(self, xi: np.ndarray):
        """(P, v, n) at similarity coordinates xi = (x - x0) / t."""
        xi = np.asarray(xi, np.float64)
        P = np.empty_like(xi)
        v = np.empty_like(xi)
        n = np.empty_like(xi)
        for k, s in enumerate(xi.flat):
            P.flat[k], v.flat[k], n.flat[k] = self._sample1(s)
        return P, v, n

    def _sample1(self, s):
        if s <= self.vstar:
            if self.left_kind == "shock":
                if s < self.left_speeds[0]:
                    return self.PL, self.vL, self.nL
                return self.Pstar, self.vstar, self.nLstar
            head, tail = self.left_speeds
            if s < head:
                return self.PL, self.vL, self.nL
            if s > tail:
                return self.Pstar, self.vstar, self.nLstar
            v = (s + CS) / (1.0 + s * CS)
            P = self.PL * np.exp(4.0 / np.sqrt(3.0) * (np.arctanh(self.vL) - np.arctanh(v)))
            return P, v, self.nL * (P / self.PL) ** 0.75
        if self.right_kind == "shock":
            if s > self.right_speeds[0]:
                return self.PR, self.vR, self.nR
            return self.Pstar, self.vstar, self.nRstar
        tail, head = self.right_speeds
        if s > head:
            return self.PR, self.vR, self.nR
        if s < tail:
            return self.Pstar, self.vstar, self.nRstar
        v = (s - CS) / (1.0 - s * CS)
        P = self.PR * np.exp(4.0 / np.sqrt(3.0) * (np.arctanh(v) - np.arctanh(self.vR)))
        return P, v, self.nR * (P / self.PR) ** 0.75


def solve(PL, vL, nL, PR, vR, nR) -> RiemannSolution:
    lo = np.log(min(PL, PR)) - 40.0
    hi = np.log(max(PL, PR)) + 40.0
    for _ in range(300):
        m = 0.5 * (lo + hi)
        P = np.exp(m)
        if _v_left_star(P, PL, vL) - _v_right_star(P, PR, vR) > 0.0:
            lo = m
        else:
            hi = m
    Ps = np.exp(0.5 * (lo + hi))
    vs = 0.5 * (_v_left_star(Ps, PL, vL) + _v_right_star(Ps, PR, vR))
    gs = _gamma(vs)
    if Ps > PL:
        sL = _add(vL, -_vshock_rel(PL, Ps))
        nLs = nL * _gamma(vL) * (vL - sL) / (gs * (vs - sL))
        lk, lsp = "shock", (sL, sL)
    else:
        nLs = nL * (Ps / PL) ** 0.75
        lk, lsp = "rarefaction", (_add(vL, -CS), _add(vs, -CS))
    if Ps > PR:
        sR = _add(vR, _vshock_rel(PR, Ps))
        nRs = nR * _gamma(vR) * (vR - sR) / (gs * (vs - sR))
        rk, rsp = "shock", (sR, sR)
    else:
        nRs = nR * (Ps / PR) ** 0.75
        rk, rsp = "rarefaction", (_add(vs, CS), _add(vR, CS))
    return RiemannSolution(PL, vL, nL, PR, vR, nR, Ps, vs, nLs, nRs, lk, rk, lsp, rsp)


def conserved_fluxes(P, v, n):
    """lab-frame densities (T00, T01, N0) and fluxes (T01, T11, N1) of an
    ideal e = 3P fluid moving along x"""
    g2 = 1.0 / (1.0 - v * v)
    w = 4.0 * P
    T00 = w * g2 - P
    T01 = w * g2 * v
    T11 = w * g2 * v * v + P
    N0 = n * np.sqrt(g2)
    N1 = N0 * v
    return (T00, T01, N0), (T01, T11, N1)
