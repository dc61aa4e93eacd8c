"""Error norms of the parity tests.

The FP32-storage bound is a per-field L1 relative error, sum |a - b| / sum |b|
over the grid, for each macroscopic field on its own: the scalars n and e,
the velocity component u_x (the fields the FP64 parity names), and the
velocity as one vector field, sum |u_a - u_b| / sum |u_b| with |.| the
Euclidean length in each cell.  The vector norm covers u_y and u_z without
measuring a secondary component against its own, possibly vanishing, scale
(u_y near a symmetric cloud, u_y and u_z of a tube); where the reference
velocity is zero everywhere, the GPU velocity is measured against the scale
of gamma instead, sum |u_a| / sum gamma.
"""
import numpy as np


def l1rel(got, ref) -> float:
    """sum |got - ref| / sum |ref|"""
    return float(np.sum(np.abs(got - ref)) / max(np.sum(np.abs(ref)), 1e-300))


def l1_fields(got, ref) -> dict:
    """per-field L1 relative errors of the (6, N) macroscopic arrays got and
    ref (n, e, u_x, u_y, u_z, gamma): keys "n", "e", "u_x", "u" (vector)"""
    out = {"n": l1rel(got[0], ref[0]), "e": l1rel(got[1], ref[1])}
    ux = np.sum(np.abs(ref[2]))
    out["u_x"] = l1rel(got[2], ref[2]) if ux > 0.0 else float(np.sum(np.abs(got[2])) / np.sum(np.abs(ref[5])))
    du = np.sqrt(np.sum((got[2:5] - ref[2:5]) ** 2, axis=0)).sum()
    u = np.sqrt(np.sum(ref[2:5] ** 2, axis=0)).sum()
    out["u"] = float(du / u) if u > 0.0 else float(np.sqrt(np.sum(got[2:5] ** 2, axis=0)).sum() / np.sum(ref[5]))
    return out
