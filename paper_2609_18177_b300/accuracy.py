"""The accuracy contract of the FP32 and served results against FP64.

Error norm.  Each scalar conserved field (density, depth, energy, the
advected quantity) is measured by its relative L1 error sum|a - b| / sum|b|
over the nodes.  The momentum is measured as one vector per node:
sum ||a_m - b_m||_2 / sum ||b_m||_2, so that a momentum component that is
nearly zero everywhere (hv of a dam break before the flow meets the bump)
is weighed against the momentum of the flow rather than against itself.  The
unburnt-gas density rho*Y (0 <= rho*Y <= rho) is measured against the
density, sum|a_rhoY - b_rhoY| / sum|b_rho|: once the gas has burnt out rho*Y
is ~0 everywhere (an FP64 run decays it towards 1e-300, an FP32 run stops at
its smallest normal numbers), and a ratio to its own sum would divide by
nothing.

Tolerances (frozen after measurement; relative L1 in the norm above, every
quantity of every result must meet the one of its workload):

    smooth runs (advection of smooth data, entropy waves)     1e-5
    shock and wet-dry runs (Euler, shallow water)             1e-2
    reactive Euler (detonations)                              5e-2

They sit above the scheme's own sensitivity, measured as the move of the FP64
solution when its input is moved by a relative 2^-24 (half an FP32 ulp):
rounding-level differences grow at rarefaction heads and shocks
(tests/test_oracle_sensitivity.py), up to 1.9e-3 (momentum) on the dam break
over a bump at T = 0.1 and 4.4e-3 on 5,000-step dam breaks; on 5,000-step
reactive circles (Example 5.12 constants) the FP64 momentum moves by 3.3e-2 to
5.8e-2.  No FP32 path can come closer to FP64 than FP64 comes to itself
under such a change.  Measured FP32 errors: 8192^2 Riemann 3.1e-5 after 20
steps; batched dam breaks <= 1.8e-3; served Euler / shallow water / reactive
requests of up to 5,000 steps <= 3.0e-3 / 4.2e-3 / 1.5e-2.
"""
import numpy as np

TOL_SMOOTH = 1e-5
TOL_SHOCK = 1e-2
TOL_REACTIVE = 5e-2

ADVECTION, EULER, SWE, REACTIVE = 0, 1, 2, 3


def tolerance(system):
    """The frozen tolerance of a (non-smooth) run of the given system."""
    return TOL_REACTIVE if system == REACTIVE else TOL_SHOCK


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
            den = np.abs(b2[0 if name == "rhoY" else idx[0]]).sum()
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
            den = b2[0 if name == "rhoY" else idx[0]].abs().sum()
        else:
            num = ((a2[idx] - b2[idx]) ** 2).sum(dim=0).sqrt().sum()
            den = (b2[idx] ** 2).sum(dim=0).sqrt().sum()
        out[name] = float(num / den) if float(den) > 0 else float(num)
    out["max"] = max(out.values())
    return out
