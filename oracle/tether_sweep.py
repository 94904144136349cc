"""Stability sweep of the penalty tether stiffness kappa for the rigid
ellipsoid in shear (the rigid-body reading of Sec. 2.3, Eq. FSIRigid, with
the 32^3 Couette cell, 6 x 3 x 3 ellipsoid of 812 markers, walls at
-/+0.02, tau = 0.8), run on the FP64 oracle. For each kappa the oracle runs
up to `steps` coupled steps and records the first step at which the
result is unstable: a non-finite field, |u| > 0.4, or a marker more than
2 lattice units from its tethered reference point (the tether has let go).

TEST INFRASTRUCTURE: calls only the oracle. Writes the summary table that
backs the choice kappa = 0.02:

    python oracle/tether_sweep.py --steps 6000 > profiles/tether_stability_oracle.md
"""
import argparse
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_1704_04551_gb300 import inputs as I  # noqa: E402


def run(kappa, steps, every=50):
    w = I.shear_ellipsoid(n=32, steps=steps, kappa=kappa)
    o = O.Oracle.from_workload(w)
    R0 = None
    for s in range(every, steps + every, every):
        o.step(every)
        _, u = o.fields()
        X, _, _ = o.markers()
        b = o.body(0)
        R = I.quat_to_matrix(np.array(b['quat']))
        if R0 is None:
            ref = np.linalg.solve(I.quat_to_matrix(np.array(w['bodies'][0]['quat'])),
                                  w['X'] - np.array(w['bodies'][0]['center'])[:, None])
            R0 = ref
        Xref = R @ R0 + np.array(b['center'])[:, None]
        gap = float(np.abs(X - Xref).max())
        umax = float(np.sqrt((u * u).sum(axis=0)).max())
        if not np.isfinite(u).all() or umax > 0.4 or not np.isfinite(gap) or gap > 2.0:
            return s, umax, gap
    return None, umax, gap


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--steps', type=int, default=6000)
    ap.add_argument('--kappa', type=float, nargs='*', default=[0.005, 0.02, 0.05, 0.5])
    a = ap.parse_args()
    threads = O.set_threads(0)
    print('# Tether stiffness stability sweep (FP64 oracle)\n')
    print('Rigid prolate ellipsoid 6 x 3 x 3 (812 markers, neutrally buoyant) in the 32^3 Couette cell,')
    print('walls at -/+0.02, tau = 0.8, penalty tether F = -kappa (X - X_ref) (the rigid reading of')
    print(f'Sec. 2.3). Up to {a.steps} coupled steps per kappa; unstable = a non-finite field, |u| > 0.4, or a')
    print(f'marker more than 2 lu from its tethered point. Oracle threads: {threads}. Command:\n')
    print(f'    python oracle/tether_sweep.py --steps {a.steps} > profiles/tether_stability_oracle.md\n')
    print('| kappa | unstable at step | max \\|u\\| at the end or at failure | max marker-tether gap (lu) | run s |')
    print('|---|---|---|---|---|')
    for k in a.kappa:
        t0 = time.time()
        s, umax, gap = run(k, a.steps)
        print(f'| {k:g} | {s if s is not None else "stable"} | {umax:.3e} | {gap:.3e} | {time.time() - t0:.0f} |',
              flush=True)


if __name__ == '__main__':
    main()
