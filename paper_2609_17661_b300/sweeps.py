"""Parameter sweeps over the ensemble engine: one line per parameter set,
all advanced together, with the diagnostics the paper follows in its
eta_min and mass-ratio studies (Sec. 4.2 on the mass ratio, App. C on the
drag-time floor eta_min): the circuit potential V_c after every step and the
pair creation rate averaged over a light-crossing time of the line.

The sweep only builds the lines and reads the record; every step runs in the
ensemble's kernels and the record is kept on the device
(``pic1d_ens_record`` / ``pic1d_ens_history``).  Reproducing the paper's
figures needs production-length runs and is not the point here.
"""
from __future__ import annotations

import itertools


def eta_mass_sweep(base_cfg: dict, eta_mins, mass_ratios, steps: int, theta, states=None, window=None):
    """Run one line per (eta_min, mass_ratio) of the grid from `base_cfg`
    (drag law SURROGATE, the network `theta` shared by all lines) for
    `steps` steps; `states` maps a line's config to its initial particle
    state (default: an empty line).  Returns one dict per line with the
    parameters and its record (vc, pairs, pair_rate, window)."""
    from . import Ensemble

    grid = list(itertools.product(eta_mins, mass_ratios))
    cfgs = []
    for k, (eta, mr) in enumerate(grid):
        c = dict(base_cfg)
        c.update(eta_min=float(eta), mass_ratio=float(mr), seed=int(base_cfg.get("seed", 1)) + k)
        cfgs.append(c)
    ens = Ensemble(cfgs)
    try:
        ens.lines[0].sur_set_params(theta)
        if states is not None:
            for ln, c in zip(ens.lines, cfgs):
                ln.set_state(states(c))
        ens.record(steps)
        ens.step(steps)
        out = []
        for k, ((eta, mr), c) in enumerate(zip(grid, cfgs)):
            h = ens.history(k, window)
            out.append(dict(eta_min=float(eta), mass_ratio=float(mr), cfg=c, **h))
        return out
    finally:
        ens.close()
