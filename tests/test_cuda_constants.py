"""The lattice constants of the CUDA library, read as text from
rlb_consts.h, against the oracle's lattice (itself pinned to the paper's
formulas): xi0 = c_t/c_0, c_0/c_t, (c_0/c_t) nu, 4/xi0, nu^2, nu^6, the
weights w_i and w'_i, and the equilibrium coefficients 1/sigma2,
4 sigma2/m22 and 4 sigma2/(m4 - m22) of the moment-matched f^eq, for the
extended (Lat<0>) and the basic (Lat<1>) lattice; float copies equal the
doubles rounded to float."""
import math
import os
import re

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(__file__), "..", "paper_1302_1125_gb300", "csrc", "rlb_consts.h")


def _eval(expr, env):
    expr = re.sub(r"(\d)f\b", r"\1", expr.strip())
    assert re.fullmatch(r"[\w\s.+\-*/()]+", expr), expr
    return float(eval(expr, {"__builtins__": {}}, env))


def _constants():
    text = open(SRC).read()
    env = {}
    for decl in re.findall(r"^constexpr double ([^;]+);", text, re.M):
        for part in re.split(r",\s*(?=k\w+ = )", decl):
            name, expr = part.split(" = ")
            env[name.strip()] = _eval(expr, env)
    lats = {}
    for lat, body in re.findall(r"struct Lat<(\d)> \{(.*?)\n\};", text, re.S):
        d = {}
        for decl in re.findall(r"static constexpr (?:double|float|int) ([^;]+);", body):
            for part in re.split(r",\s*(?=\w+ = )", decl):
                name, expr = part.split(" = ")
                d[name.strip()] = _eval(expr, {**env, **d})
        lats[int(lat)] = d
    return env, lats


@pytest.mark.parametrize("model", [0, 1])
def test_lattice_constants_match_the_oracle(orc, model):
    env, lats = _constants()
    L = lats[model]
    e, c, w, wh, xi0 = orc.lattice(model)
    nu = orc.nu(model)
    sigma2 = float((w * c[:, 0] ** 2).sum())
    m22 = float((w * c[:, 0] ** 2 * c[:, 1] ** 2).sum())
    m4 = float((w * c[:, 0] ** 4).sum())
    close = lambda a, b: a == pytest.approx(b, rel=1e-13, abs=1e-16)   # the oracle forms them by formula
    assert close(L["xi0"], xi0) and close(L["xi0sq"], xi0 * xi0)
    assert close(L["c0ct"], 1.0 / xi0) and close(L["omegaC"], nu / xi0)
    assert close(L["four_over_xi0"], 4.0 / xi0)
    assert close(L["nu2"], nu ** 2) and close(L["nu6"], nu ** 6)
    assert close(L["inv_sigma2"], 1.0 / sigma2)
    assert close(L["a2f"], 4.0 * sigma2 / m22) and close(L["a3f"], 4.0 * sigma2 / (m4 - m22))
    # population order: rest, six axis populations, twelve diagonals
    for k, i in (("0", 0), ("1", 1), ("2", 7)):
        assert close(L["w" + k], w[i]) and close(L["wh" + k], wh[i])
    assert L["dmag"] == np.abs(c[7:, :]).max()
    for f, dname in (("f_inv_sigma2", "inv_sigma2"), ("f_a2f", "a2f"), ("f_a3f", "a3f"), ("f_nu2", "nu2")):
        assert np.float32(L[f]) == np.float32(L[dname]), f


def test_shared_constants(orc):
    env, _ = _constants()
    e, c, w, wh, xi0 = orc.lattice(0)
    assert env["kPi2Over16"] == pytest.approx(math.pi ** 2 / 16.0, rel=1e-15)     # 1/(d_G/pi^2)
    assert env["kXi0"] == pytest.approx(xi0, rel=1e-15)
    assert env["kOmegaC"] == pytest.approx(13.0 / math.sqrt(27.0), rel=1e-15)


@pytest.mark.parametrize("model", [0, 1])
def test_velocity_table_matches_the_oracle(orc, model):
    """kDir of rlb_device.cuh (the extended lattice's integer vectors, population
    order rest, axes, diagonals; the basic lattice halves the diagonals)"""
    text = open(os.path.join(os.path.dirname(SRC), "rlb_device.cuh")).read()
    m = re.search(r"constexpr Dir kDir\[19\] = \{(.*?)\};", text, re.S)
    assert m
    kdir = np.array([int(v) for v in re.findall(r"-?\d+", m.group(1))]).reshape(19, 3)
    if model == 1:
        kdir[7:] //= 2
    e, c, w, wh, xi0 = orc.lattice(model)
    assert np.array_equal(kdir, np.rint(c).astype(int)) and np.allclose(c, kdir, rtol=0, atol=1e-15)
