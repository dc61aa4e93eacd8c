"""Runs the paper's two fastest 1-D shock tubes (Sec. III) in whichever
oracle library RLB_ORACLE_LIB names and prints one JSON line of outcomes.
Called in a subprocess by tests/test_oracle_ultrarelativistic.py, once per
reading of the paper compiled into a private copy of the oracle."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1302_1125_gb300 import workloads as W  # noqa: E402

# (name, P ratio, eta/s, alpha, Euler mode): Sec. III's beta ~ 0.99 run and
# its inviscid beta ~ 0.9 run, 800 cells, open ends, dt/dx 0.25
RUNS = (("beta099", 1e5, 0.01, 0.2, 0), ("beta09_inviscid", 1e3, 0.0, 0.2, 1))


def run(ratio, eta, alpha, euler, steps=1000, chunk=5):
    w = W.riemann_tube(800, ratio, 2.0, eta_over_s=eta, alpha_override=alpha, dt_over_dx=0.25)
    p = oracle.Params(nx=800, dt=0.25, eta_over_s=eta, alpha_override=alpha, euler_mode=euler)
    s = oracle.init(p, *w.fields())
    for k in range(0, steps, chunk):
        oracle.step(s, chunk)
        if s.nonphysical:
            return {"physical": False, "by_step": k + chunk}
    m = oracle.macroscopic(s)
    return {"physical": True, "max_u": float(m[2].max()), "max_gamma": float(m[5].max())}


if __name__ == "__main__":
    oracle.set_threads(min(16, os.cpu_count() or 1))
    print(json.dumps({name: run(r, e, a, eu) for name, r, e, a, eu in RUNS}))
