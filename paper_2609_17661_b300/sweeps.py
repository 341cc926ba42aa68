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


def sweep_configs(base_cfg: dict, eta_mins, mass_ratios):
    """[(eta_min, mass_ratio, config)] of the grid, one line each (seed
    advanced per line)."""
    out = []
    for k, (eta, mr) in enumerate(itertools.product(eta_mins, mass_ratios)):
        c = dict(base_cfg)
        c.update(eta_min=float(eta), mass_ratio=float(mr), seed=int(base_cfg.get("seed", 1)) + k)
        out.append((float(eta), float(mr), c))
    return out


def eta_mass_sweep(base_cfg: dict, eta_mins, mass_ratios, steps: int, theta, states=None, window=None,
                   rank: int = 0, world: int = 1, weights=None):
    """Run one line per (eta_min, mass_ratio) of the grid from `base_cfg`
    (drag law SURROGATE, the network `theta` shared by all lines) for
    `steps` steps; `states` maps a line's config to its initial particle
    state (default: an empty line).  In a job of `world` ranks, this rank
    runs its share of the grid (``shard.shard_lines`` by `weights`, one per
    grid point, equal by default).  Returns one dict per line run here with
    the grid index, the parameters and its record (vc, pairs, pair_rate,
    window)."""
    from . import Ensemble
    from .shard import my_lines

    grid = sweep_configs(base_cfg, eta_mins, mass_ratios)
    mine = my_lines(weights if weights is not None else [1.0] * len(grid), rank, world)
    if not mine:
        return []
    grid = [grid[k] for k in mine]
    cfgs = [c for _, _, c in grid]
    ens = Ensemble(cfgs)
    try:
        ens.lines[0].sur_set_params(theta)
        if states is not None:
            for ln, c in zip(ens.lines, cfgs):
                ln.set_state(states(c))
        ens.record(steps)
        ens.step(steps)
        out = []
        for k, (g, (eta, mr, c)) in enumerate(zip(mine, grid)):
            h = ens.history(k, window)
            out.append(dict(index=g, eta_min=eta, mass_ratio=mr, cfg=c, **h))
        return out
    finally:
        ens.close()
