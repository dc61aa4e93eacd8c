"""Pins of the oracle's lattice tables against what the paper fixes.

Sec. II.A, Eqs. 42-46 (extended D3Q19 lattice, weights and constants) and
Eqs. 59-60 (number-distribution weights), with the global lattice constant
nu = sqrt(13), i.e. c_a = sqrt(13)/nu = 1 and c_t/c_0 = sqrt(27/13).
"""
from fractions import Fraction as Fr
import itertools
import math

import numpy as np

NU = math.sqrt(13.0)


def test_lattice_constant(orc):
    assert abs(orc.nu() - NU) < 1e-15


def test_weights_are_the_printed_formulas_at_nu_1(orc):
    # Eqs. 43-45 with c_t^2/c_0^2 = 27/nu^2 and c_a^2 = 13/nu^2 (Eq. 46), in
    # exact rational arithmetic (nu^2 = 13): the weights do not depend on nu and
    # are w0 = -539/676, w_axis = 99/338, w_diag = 9/2704.
    nu2 = Fr(13)
    r2, ca2 = Fr(27) / nu2, Fr(13) / nu2
    w0 = 1 + 7 * r2 * nu2 / 676 - r2 / ca2
    w1 = r2 / (1014 * ca2) * (169 - 2 * ca2 * nu2)
    w2 = r2 * nu2 / 8112
    assert (w0, w1, w2) == (Fr(-539, 676), Fr(99, 338), Fr(9, 2704))
    _, _, w, _, _ = orc.lattice()
    assert abs(w[0] - float(w0)) < 1e-15
    assert np.allclose(w[1:7], float(w1), rtol=0, atol=1e-16)
    assert np.allclose(w[7:], float(w2), rtol=0, atol=1e-17)


def test_velocity_set_is_the_extended_fully_symmetric_set(orc):
    e, c, _, _, xi0 = orc.lattice()
    ca = np.sqrt(13.0) / NU
    assert np.all(e[0] == 0) and np.all(c[0] == 0)
    axis = {tuple(v) for v in e[1:7]}
    diag = {tuple(v) for v in e[7:]}
    # fully symmetric: all sign flips and permutations of (1,0,0) and (1,1,0)
    fs = lambda base: {tuple(s * x for s, x in zip(signs, perm))
                       for perm in itertools.permutations(base)
                       for signs in itertools.product((1, -1), repeat=3)}
    assert axis == fs((1, 0, 0)) and len(axis) == 6
    assert diag == fs((1, 1, 0)) and len(diag) == 12
    # speeds: c_a on the axes, 2 c_a per component on the diagonals (Eq. 42)
    assert np.allclose(np.abs(c[1:7]).sum(1), ca, rtol=1e-15)
    assert np.allclose(np.abs(c[7:]).sum(1), 4 * ca, rtol=1e-15)
    assert abs(xi0 - np.sqrt(27.0) / NU) < 1e-15


def test_quadrature_moments(orc):
    _, c, w, _, xi0 = orc.lattice()
    assert abs(w.sum() - 1.0) < 1e-15
    # second moments isotropic: sum w c_a c_b = (9 / nu^2) delta_ab
    M2 = np.einsum("i,ia,ib->ab", w, c, c)
    assert np.allclose(M2, 9.0 / NU ** 2 * np.eye(3), rtol=0, atol=1e-14)
    # odd moments vanish
    assert np.allclose(np.einsum("i,ia->a", w, c), 0, atol=1e-15)
    assert np.allclose(np.einsum("i,ia,ib,ic->abc", w, c, c, c), 0, atol=1e-12)
    # fourth moments that fix the equilibrium: 171/nu^4 (aaaa), 36/nu^4 (aabb)
    assert abs(np.sum(w * c[:, 0] ** 4) - 171.0 / NU ** 4) < 1e-14
    assert abs(np.sum(w * c[:, 0] ** 2 * c[:, 1] ** 2) - 36.0 / NU ** 4) < 1e-14
    # the lattice constants make the U^a U^b coefficient of T^{ab} and of
    # T^{00} equal (Sec. II): xi0^2 = 3 sigma2
    assert abs(xi0 ** 2 - 3 * M2[0, 0]) < 1e-12


def test_number_weights(orc):
    # Eqs. 59-60 with c_a^2 = 13/nu^2 = 1: sum w' = 1, sum w' c_a c_b = delta_ab/3,
    # and every weight is non-negative
    ca2 = Fr(1)
    wh0, wh1, wh2 = Fr(1, 10), Fr(6, 35) - 1 / (42 * ca2), 1 / (84 * ca2) - Fr(3, 280)
    assert wh0 + 6 * wh1 + 12 * wh2 == 1
    assert 2 * wh1 * ca2 + 8 * wh2 * 4 * ca2 == Fr(1, 3)
    assert min(wh0, wh1, wh2) >= 0
    _, c, _, wh, _ = orc.lattice()
    assert abs(wh[0] - 0.1) < 1e-16
    assert np.allclose(wh[1:7], float(wh1), atol=1e-16)
    assert np.allclose(wh[7:], float(wh2), atol=1e-16)
    assert np.allclose(np.einsum("i,ia,ib->ab", wh, c, c), np.eye(3) / 3, atol=1e-14)
