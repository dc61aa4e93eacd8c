"""The population classes of the exact symmetry reductions, read from the
CUDA sources (the class representatives of rlb_classes.cuh and the member
table of rlb_aux.cu), checked against the oracle's lattice:

* 1-D (u_y = u_z = 0, fields uniform in y and z): every member of a class has
  its representative's f and h weights and c_x; the 7 classes partition the
  19 populations with multiplicities 1, 1, 1, 4, 4, 4, 4.
* 2-D (u_z = 0, fields uniform in z): every member is its representative's
  mirror image under z -> -z; the 14 classes partition the 19 populations.
* Representatives are the first population of their class.
"""
import os
import re

import numpy as np
import pytest

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_1302_1125_gb300", "csrc")


def read(name):
    with open(os.path.join(CSRC, name)) as fh:
        return fh.read()


def int_list(text):
    return [int(v) for v in re.findall(r"-?\d+", text)]


def reps(np_):
    src = read("rlb_classes.cuh")
    m = re.search(r"constexpr int r\[%d\] = \{([^}]*)\}" % np_, src)
    assert m, np_
    return int_list(m.group(1))


def members():
    src = read("rlb_aux.cu")
    m = re.search(r"kMember\[2\]\[12\]\[2\] = \{(.*?)\};", src, re.S)
    assert m
    vals = int_list(m.group(1))
    assert len(vals) == 2 * 12 * 2
    table = np.array(vals).reshape(2, 12, 2)
    one_d = [tuple(p) for p in table[0]]
    two_d = [tuple(p) for p in table[1][:5]]
    return one_d, two_d


def classes(rep_list, pairs):
    cl = {r: [r] for r in rep_list}
    for r, mbr in pairs:
        assert r in cl, (r, mbr)
        cl[r].append(mbr)
    return cl


@pytest.fixture(scope="module")
def lattice(orc):
    e, c, w, wh, xi0 = orc.lattice(0)
    return c, w, wh


def check_partition(cl):
    pops = sorted(p for v in cl.values() for p in v)
    assert pops == list(range(19))
    for r, v in cl.items():
        assert r == min(v)          # the representative is the first population


def test_one_d_classes(lattice):
    c, w, wh = lattice
    one_d, _ = members()
    cl = classes(reps(7), one_d)
    check_partition(cl)
    assert [len(cl[r]) for r in reps(7)] == [1, 1, 1, 4, 4, 4, 4]
    for r, v in cl.items():
        for m in v:
            assert w[m] == w[r] and wh[m] == wh[r] and c[m][0] == c[r][0], (r, m)


def test_two_d_classes(lattice):
    c, w, wh = lattice
    _, two_d = members()
    cl = classes(reps(14), two_d)
    check_partition(cl)
    assert [len(cl[r]) for r in reps(14)] == [1, 1, 1, 1, 1, 2, 1, 1, 1, 1, 2, 2, 2, 2]
    for r, mbr in two_d:
        assert np.array_equal(c[mbr], c[r] * np.array([1, 1, -1])) and c[r][2] != 0, (r, mbr)
        assert w[mbr] == w[r] and wh[mbr] == wh[r]
    # no two representatives are mirror images of each other
    rs = reps(14)
    for a in rs:
        for b in rs:
            if a != b:
                assert not np.array_equal(c[a], c[b] * np.array([1, 1, -1])), (a, b)


def test_one_d_representatives_distinct(lattice):
    """two representatives never share weight and c_x (else they would be one class)"""
    c, w, wh = lattice
    rs = reps(7)
    keys = [(w[r], wh[r], c[r][0]) for r in rs]
    assert len(set(keys)) == len(keys)
