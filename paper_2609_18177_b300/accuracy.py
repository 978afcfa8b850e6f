"""The accuracy contract of the FP32 and served results against FP64.

Error norm.  Each scalar conserved field (density, depth, energy, rho*Y, the
advected quantity) is measured by its relative L1 error sum|a - b| / sum|b|
over the nodes.  The momentum is measured as one vector per node:
sum ||a_m - b_m||_2 / sum ||b_m||_2, so that a momentum component that is
nearly zero everywhere (hv of a dam break before the flow meets the bump)
is weighed against the momentum of the flow rather than against itself.

Tolerances (frozen after measurement; relative L1 in the norm above, every
quantity of every result must meet the one of its workload):

    smooth runs (advection, entropy waves)           1e-5
    shock, wet-dry and reactive runs                 5e-3

The second figure sits above the scheme's own sensitivity: the FP64 oracle run
from its input moved by a relative 2^-24 (half an FP32 ulp) moves by up to
1.9e-3 (momentum) and 5.8e-4 (depth) on the dam break over a bump at T = 0.1
(n = 274..1024), because rounding-level differences grow about 2x per step at
the head of the rarefaction (tests/test_oracle_sensitivity.py).  No FP32 path
can come closer to FP64 than FP64 comes to itself under such a change.
"""
import numpy as np

TOL_SMOOTH = 1e-5
TOL_SHOCK = 5e-3

ADVECTION, EULER, SWE, REACTIVE = 0, 1, 2, 3


def quantities(system, dim):
    """Names and field indices of the measured quantities: scalars as (name, [c]),
    the momentum as ("momentum", [1, .., dim])."""
    if system == ADVECTION:
        return [("u", [0])]
    mom = ("momentum", list(range(1, dim + 1)))
    if system == SWE:
        return [("h", [0]), mom]
    out = [("rho", [0]), mom, ("E", [dim + 1])]
    if system == REACTIVE:
        out.append(("rhoY", [dim + 2]))
    return out


def contract_l1(a, b, system, dim):
    """Relative L1 errors of a against the reference b (arrays [m][...]) per
    quantity, and their maximum under "max"."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    m = b.shape[0]
    a2, b2 = a.reshape(m, -1), b.reshape(m, -1)
    out = {}
    for name, idx in quantities(system, dim):
        if len(idx) == 1:
            num = np.abs(a2[idx[0]] - b2[idx[0]]).sum()
            den = np.abs(b2[idx[0]]).sum()
        else:
            num = np.sqrt(((a2[idx] - b2[idx]) ** 2).sum(axis=0)).sum()
            den = np.sqrt((b2[idx] ** 2).sum(axis=0)).sum()
        out[name] = float(num / den) if den > 0 else float(num)
    out["max"] = max(out.values())
    return out


def contract_l1_torch(a, b, system, dim):
    """contract_l1 on torch tensors (any device), reduced in FP64."""
    import torch
    a = a.to(torch.float64)
    b = b.to(torch.float64)
    m = b.shape[0]
    a2, b2 = a.reshape(m, -1), b.reshape(m, -1)
    out = {}
    for name, idx in quantities(system, dim):
        if len(idx) == 1:
            num = (a2[idx[0]] - b2[idx[0]]).abs().sum()
            den = b2[idx[0]].abs().sum()
        else:
            num = ((a2[idx] - b2[idx]) ** 2).sum(dim=0).sqrt().sum()
            den = (b2[idx] ** 2).sum(dim=0).sqrt().sum()
        out[name] = float(num / den) if float(den) > 0 else float(num)
    out["max"] = max(out.values())
    return out
