"""Host logic of the batched-tube path, without a GPU: the job plan of the
persistent launch (rlb_batch_plan) and the argument checks of
rlb_batch_create, which run before any CUDA call.

The plan is checked against what it must satisfy rather than against a
second copy of the algorithm: every tube with steps runs in exactly one job,
jobs respect their capacity, the tube order is the documented one, the
per-cluster tables partition the jobs, the reported critical path is the
largest per-cluster cost, and the greedy longest-first assignment is within
Graham's 4/3 bound of the best possible makespan.
"""
import math

import numpy as np
import pytest

from paper_1302_1125_gb300 import build as B
from paper_1302_1125_gb300 import rlb
from paper_1302_1125_gb300 import workloads as W


@pytest.fixture(scope="module", autouse=True)
def lib():
    B.build()
    return rlb.lib()


def tuning(threads=256, bound=256, cluster=1, ppt=1):
    return rlb.rlb_batch_tuning(threads, bound, cluster, ppt, 0.0)


def check_plan(nx, steps, t, ncl):
    order, jobs, cl, crit = rlb.rlb_batch_plan(nx, steps, t, ncl)
    nx, steps = np.asarray(nx), np.asarray(steps)
    B_ = nx.size
    assert sorted(order.tolist()) == list(range(B_))
    # documented order: steps desc, nx desc, id asc; zero-step tubes last
    keys = [(-steps[i], -nx[i], i) for i in order]
    assert keys == sorted(keys)
    per_pass = t.cluster * t.threads
    cap = per_pass * t.pairs_per_thread
    seen = []
    cost = []
    for first, count, jsteps, pairs in jobs:
        assert 1 <= count <= 32
        ids = order[first:first + count]
        seen.extend(ids.tolist())
        assert pairs == sum((nx[i] + 1) // 2 for i in ids)
        assert count == 1 or pairs <= cap
        assert jsteps == max(steps[i] for i in ids)
        cost.append(jsteps * math.ceil(pairs / per_pass))
    active = [i for i in range(B_) if steps[i] > 0]
    assert sorted(seen) == sorted(active)
    # consecutive positions in the order: jobs cover a prefix of it
    firsts = sorted(j[0] for j in jobs)
    assert firsts == sorted(set(firsts))
    assert cl[0] == 0 and cl[-1] == len(jobs) and np.all(np.diff(cl) >= 0)
    loads = [sum(cost[cl[c]:cl[c + 1]]) for c in range(ncl)]
    assert crit == max(loads)
    # jobs of a cluster run longest first
    for c in range(ncl):
        cc = cost[cl[c]:cl[c + 1]]
        assert cc == sorted(cc, reverse=True)
    if cost:
        lower = max(sum(cost) / ncl, max(cost))    # no schedule beats this
        assert crit <= (4.0 / 3.0) * lower + 1e-9
    return order, jobs, cl, crit


@pytest.mark.parametrize("t,ncl", [(tuning(), 304), (tuning(128, 512, 2), 150), (tuning(512, 512, 8, 2), 19),
                                   (tuning(256, 384, 4, 4), 38), (tuning(32, 256, 1), 7)])
def test_plan_of_the_512_tube_sweep(t, ncl):
    s = W.batch_tubes()
    check_plan(s.nx, s.steps, t, ncl)


def test_plan_groups_short_tubes_and_skips_idle_ones():
    nx = [10, 12, 9, 500, 11, 3, 1, 600]
    steps = [40, 40, 36, 2000, 44, 0, 4, 2400]
    order, jobs, cl, crit = check_plan(nx, steps, tuning(32, 256, 1), 3)
    # 2 long tubes alone, the 5 short active ones in one job, tube 5 idle
    assert len(jobs) == 3
    assert order[-1] == 5
    short = [j for j in jobs if j[1] > 1]
    assert len(short) == 1 and short[0][1] == 5


def test_plan_caps_tubes_per_job():
    nx = [2] * 100
    steps = [5] * 100
    order, jobs, cl, crit = check_plan(nx, steps, tuning(512, 512, 8, 4), 2)
    assert all(j[1] <= 32 for j in jobs) and len(jobs) == 4


def test_plan_more_clusters_than_jobs():
    order, jobs, cl, crit = check_plan([64, 64], [10, 10], tuning(), 16)
    assert crit == 10 and len(jobs) == 1


def test_plan_brute_force_optimum_small():
    """Tiny instances: the plan's makespan is within 4/3 of the true optimum
    over all assignments of its jobs (exhaustive)."""
    import itertools
    rng = np.random.default_rng(5)
    for _ in range(20):
        nx = rng.integers(64, 2000, 6)
        steps = 4 * nx
        t = tuning(64, 256, 1)
        order, jobs, cl, crit = check_plan(nx, steps, t, 3)
        cost = [j[2] * math.ceil(j[3] / 64) for j in jobs]
        best = min(max(sum(c for c, a in zip(cost, asg) if a == k) for k in range(3))
                   for asg in itertools.product(range(3), repeat=len(cost)))
        assert crit <= (4.0 / 3.0) * best + 1e-9


@pytest.mark.parametrize("t,why", [(tuning(48), "multiple of 32"), (tuning(512, 256), "multiple of 32"),
                                   (tuning(256, 300), "bound"), (tuning(256, 256, 3), "cluster"),
                                   (tuning(256, 256, 1, 0), "pairs_per_thread")])
def test_plan_rejects_bad_tunings(t, why):
    with pytest.raises(rlb.RLBError) as e:
        rlb.rlb_batch_plan([64], [1], t, 4)
    assert e.value.status == rlb.RLB_E_INVALID
    assert why in rlb.batch_last_error()


def test_plan_rejects_bad_inputs():
    for nx, st, ncl in (([0], [1], 4), ([4], [-1], 4), ([4], [2 ** 31], 4), ([4], [1], 0)):
        with pytest.raises(rlb.RLBError) as e:
            rlb.rlb_batch_plan(nx, st, tuning(), ncl)
        assert e.value.status == rlb.RLB_E_INVALID


@pytest.mark.parametrize("kw,expect", [
    (dict(nx=[]), rlb.RLB_E_INVALID),
    (dict(nx=[0, 4]), rlb.RLB_E_INVALID),
    (dict(eta=[-0.1, 0.1]), rlb.RLB_E_INVALID),
    (dict(zeta=[0.0, math.inf]), rlb.RLB_E_INVALID),
    (dict(limiter=4), rlb.RLB_E_INVALID),
    (dict(precision=rlb.FP64), rlb.RLB_E_INVALID),
    (dict(euler_mode=1), rlb.RLB_E_INVALID),
    (dict(dt_over_dx=0.73), rlb.RLB_E_UNSTABLE),
    (dict(alpha_override=1.0), rlb.RLB_E_UNSTABLE),
    (dict(zeta=[0.0, 1e6]), rlb.RLB_E_UNSTABLE),
    (dict(symmetry_1d=2), rlb.RLB_E_INVALID),
])
def test_batch_create_validates_on_the_host(kw, expect):
    import ctypes as C
    nx = np.asarray(kw.get("nx", [64, 80]), np.int32)
    eta = np.asarray(kw.get("eta", [0.1] * max(nx.size, 1)), np.float64)
    zeta = np.asarray(kw.get("zeta", [0.0] * max(nx.size, 1)), np.float64)
    o = rlb.make_options(dt_over_dx=kw.get("dt_over_dx", 0.25), alpha_override=kw.get("alpha_override", -1.0),
                         euler_mode=kw.get("euler_mode", 0), precision=kw.get("precision", rlb.FP32_STORAGE),
                         symmetry_1d=kw.get("symmetry_1d", 0))
    h = C.c_void_p()
    dp, ip = C.POINTER(C.c_double), C.POINTER(C.c_int)
    st = rlb.lib().rlb_batch_create(int(nx.size), nx.ctypes.data_as(ip), eta.ctypes.data_as(dp),
                                    zeta.ctypes.data_as(dp), kw.get("limiter", 0), C.byref(o), C.byref(h))
    assert st == expect
    assert h.value is None
    assert rlb.batch_last_error() != "no error"


def test_batch_null_handles_are_rejected():
    L = rlb.lib()
    assert L.rlb_batch_step(None, None) == rlb.RLB_E_INVALID
    assert L.rlb_batch_init(None, None, None, None, 0) == rlb.RLB_E_INVALID
    assert L.rlb_batch_total_cells(None) == 0
    L.rlb_batch_destroy(None)


def test_batch_parameters_are_sized_before_the_library_reads_them():
    """the binding broadcasts eta/s and zeta/s to one value per tube and
    refuses arrays of another length (the library reads B values of each)"""
    with pytest.raises(ValueError):
        rlb.Batch([64, 80, 96], [0.1, 0.2], [0.0, 0.0, 0.0])
    with pytest.raises(ValueError):
        rlb.Batch([64, 80], [0.1, 0.2], [0.0, 0.0, 0.0])
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        # sizes accepted: the call reaches the library, which needs a device
        with pytest.raises(rlb.RLBError) as e:
            rlb.Batch([64, 80], 0.1, 0.0)
        assert e.value.status == rlb.RLB_E_CUDA


def test_plan_step_counts_are_sized_before_the_library_reads_them():
    t = rlb.rlb_batch_tuning(256, 256, 1, 1, 0.0)
    with pytest.raises(ValueError):
        rlb.rlb_batch_plan([64, 80, 96], [10, 20], t, 4)
    assert rlb.rlb_batch_plan([64, 80, 96], 10, t, 4)[3] == 10     # a scalar applies to all tubes


def test_batch_from_spec_marshals_through_to_the_library():
    """the 512-tube recipe's arrays pass the binding's checks and reach
    rlb_batch_create (which, without a device, answers RLB_E_CUDA)"""
    from paper_1302_1125_gb300 import workloads as W
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    for spec in (W.batch_tubes(), W.batch_tubes(count=8, seed=3)):
        with pytest.raises(rlb.RLBError) as e:
            rlb.Batch.from_spec(spec)
        assert e.value.status == rlb.RLB_E_CUDA
        with pytest.raises(rlb.RLBError) as e:
            rlb.Batch.from_spec(spec, symmetry_1d=1)
        assert e.value.status == rlb.RLB_E_CUDA
