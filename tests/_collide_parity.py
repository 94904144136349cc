"""Collide-stream parity against the FP64 oracle (Sec. 2.1: Eqs. lbm,
BGKequilibrium, rho_u and the Guo term; half-way bounce-back), shared by the
in-process tests and by a child process that loads another build of the
library (IBM_LBM_LIBRARY), e.g. the one compiled with IBM_FORCE_IDX64.

Run as ``python -m tests._collide_parity`` it checks the three small
lattices and prints one line per geometry."""
import numpy as np

import oracle as O
from paper_1704_04551_gb300 import inputs as I
from tests._cases import LATTICES, fluid_mask, shape


def check_collide_parity(binding, lat, steps=3, seed=11, tol=2e-7, markers=None):
    """Random populations, then `steps` collide-stream stages (even, odd,
    ...): populations and moments element by element against the oracle.
    With markers = (X, F) (tracers with fixed forces) every step is
    spread, collide, interpolate, so that the collision reads a force
    density on the touched tiles and the interpolation clears it."""
    sim = binding.Simulation(lat)
    ora = O.Oracle(lat)
    fl = fluid_mask(lat)
    f0 = I.random_populations(shape(lat), seed, amp=0.02)
    f0[:, ~fl] = 0.0
    sim.set_populations(f0)
    ora.set_populations(f0)
    X, F = markers if markers is not None else (np.zeros((3, 0)), None)
    sim.set_markers(None, [], X)
    ora.set_bodies([], X)
    if F is not None:
        sim.set_marker_forces(F)
        ora.set_marker_forces(F)
    worst = 0.0
    for s in range(steps):
        if F is not None:
            sim.stage(binding.STAGE_SPREAD)
            ora.stage_spread()
        sim.stage(binding.STAGE_COLLIDE)
        ora.stage_collide_stream()
        fg, fo = sim.populations(), ora.populations()
        err = np.abs(fg[:, fl] - fo[:, fl]).max()
        rg, ug = sim.fields()
        ro, uo = ora.fields()
        err = max(err, np.abs(rg[fl] - ro[fl]).max(), np.abs(ug[:, fl] - uo[:, fl]).max())
        assert err < tol, f'step {s}: {err}'
        worst = max(worst, err)
        if F is not None:
            sim.stage(binding.STAGE_INTERP)
            ora.stage_interpolate()
    sim.close()
    return worst


def main():
    from paper_1704_04551_gb300 import binding
    binding.load()
    for geom, lat in LATTICES.items():
        err = check_collide_parity(binding, lat)
        print(f'{geom} ok {err:.3e}')


if __name__ == '__main__':
    main()
