"""Kernel paths that the small coupled parity tests do not reach, each
against the FP64 oracle through the C ABI:

* the collide variant with 64-bit element offsets (taken when 19 N >= 2^32,
  i.e. only above ~600^3 cells), from a build with IBM_FORCE_IDX64 that
  selects it on small lattices (Sec. 2.1, Eqs. lbm, rho_u, Guo term);
* the collide on a lattice wide enough for full 128-cell blocks, a ragged
  x block and many row blocks, with a spread force density on touched
  tiles, over even and odd steps;
* the membrane force scatter in fixed point (taken once a previous step set
  the body's scale) and its float redo (taken when a contribution outgrows
  that scale) (Sec. 2.2, Eqs. membrane-potential .. volumeEnergy);
* both families of transfer kernels: launches of fewer than 512 marker
  groups take four lanes per marker in large blocks, launches of more take
  one thread per marker with bank-sorted shared-memory atomics; spreading
  and interpolation with shared-memory boxes, through each family
  (Sec. 2.3, Eqs. ibmForceSpread, ibmVelocityInterpret);
* the fused coupling kernel of membrane suspensions (interpolation, forces
  and spreading per body between two collisions, two force-density
  buffers), which ibm_lbm_step takes for chunks of 16 and 64 steps, against
  the same steps run stage by stage with the separate kernels and against
  the oracle.
Tolerances as in test_gpu_parity.py."""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
from paper_1704_04551_gb300 import inputs as I
from tests._cases import WIDE, cluster_tracers, membrane_case, shape, wide_tracers
from tests._collide_parity import check_collide_parity

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

@pytest.mark.parametrize('geom', list(WIDE))
def test_collide_wide_lattice_with_force_density(cuda_lib, geom):
    lat = WIDE[geom]
    check_collide_parity(cuda_lib, lat, steps=3, seed=13, markers=wide_tracers(lat, 3000, 14))


def test_collide_64bit_offsets_variant(cuda_lib):
    """The same collide parity on a library built with IBM_FORCE_IDX64, run
    in a child process that loads that build."""
    from paper_1704_04551_gb300 import build
    out = os.path.join(build.BUILD, 'idx64', 'libibmlbm.so')
    os.makedirs(os.path.dirname(out), exist_ok=True)
    build.build(extra=['-DIBM_FORCE_IDX64'], out=out)
    env = dict(os.environ, IBM_LBM_LIBRARY=out, PYTHONPATH=ROOT + os.pathsep + os.environ.get('PYTHONPATH', ''))
    r = subprocess.run([sys.executable, '-m', 'tests._collide_parity'], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.count(' ok ') == 3, r.stdout


@pytest.mark.parametrize('n_clusters', [40, 600])
@pytest.mark.parametrize('geom', list(WIDE))
def test_transfer_kernel_families(cuda_lib, geom, n_clusters):
    """Spreading, then interpolation and advection through the boxes the
    spreading computed, for 40 groups (four-lanes kernels) and 600 groups
    (sorted kernels), against the oracle."""
    from paper_1704_04551_gb300.binding import Simulation
    lat = WIDE[geom]
    X, F = cluster_tracers(lat, n_clusters, 31 + n_clusters)
    sim, ora = Simulation(lat), O.Oracle(lat)
    sim.set_markers(None, [], X)
    ora.set_bodies([], X)
    sim.set_marker_forces(F)
    ora.set_marker_forces(F)
    sim.stage(cuda_lib.STAGE_SPREAD)
    ora.stage_spread()
    gg, go = sim.force_density(), ora.force_density()
    assert np.abs(gg - go).max() < 2e-5 * np.abs(go).max()
    assert np.allclose(gg.sum(1), go.sum(1), rtol=1e-5, atol=1e-9)
    rho, u = I.random_fields(shape(lat), 32)
    sim.set_lattice(rho, u)
    ora.set_equilibrium(rho, u)
    sim.stage(cuda_lib.STAGE_INTERP)
    ora.stage_interpolate()
    Xg, Ug, _ = sim.markers()
    Xo, Uo, _ = ora.markers()
    assert np.abs(Ug - Uo).max() < 2e-5 * np.abs(Uo).max()
    assert np.abs(Xg - Xo).max() < 1e-6


def test_membrane_forces_fixed_point_after_steps(cuda_lib):
    """After three coupled steps every body has a scale from its previous
    forces, so the FORCES stage scatters in fixed point; the result matches
    the oracle's forces at the GPU's current positions."""
    w = membrane_case()
    w['lattice'] = dict(w['lattice'], body_force=[2e-6, 0, 0])
    sim = cuda_lib.Simulation.from_workload(w)
    sim.step(3)
    Xg = sim.markers()[0]
    ora = O.Oracle.from_workload(dict(w, X=Xg))
    sim.stage(cuda_lib.STAGE_FORCES)
    ora.stage_forces()
    Fg, Fo = sim.markers()[2], ora.markers()[2]
    scale = np.abs(Fo).max()
    assert scale > 1e-5
    assert np.abs(Fg - Fo).max() < 1e-4 * scale


def test_membrane_forces_overflow_redo(cuda_lib):
    """Bodies one step away from their rest shape set a tiny scale; a random
    flow then displaces the vertices by ~1e-2 lu, so this step's
    contributions exceed the fixed-point headroom by orders of magnitude
    and every block redoes its scatter with float atomics."""
    w = membrane_case(deform=1e-7)
    sim = cuda_lib.Simulation.from_workload(w)
    sim.step(1)
    rng = np.random.default_rng(5)
    u = 0.02 * (2 * rng.random((3, sim.N)) - 1)
    sim.set_lattice(None, u)
    sim.stage(cuda_lib.STAGE_SPREAD)   # stencil boxes at the current positions
    sim.stage(cuda_lib.STAGE_INTERP)   # advect by the random flow
    Xg = sim.markers()[0]
    ora = O.Oracle.from_workload(dict(w, X=Xg))
    sim.stage(cuda_lib.STAGE_FORCES)
    ora.stage_forces()
    Fg, Fo = sim.markers()[2], ora.markers()[2]
    scale = np.abs(Fo).max()
    assert scale > 1e-4
    assert np.abs(Fg - Fo).max() < 1e-4 * scale


def test_fused_membrane_chunks_match_stages_and_oracle(cuda_lib):
    """98 steps of deformed membranes in a tube through ibm_lbm_step (one
    fused chunk of 64 steps, two of 16, two single steps) against the same
    steps stage by stage, and against the FP64 oracle. Several groups add
    into shared cells with float atomics, so the two GPU paths agree to
    rounding (the bound of the serving identity test), not bit for bit."""
    w = membrane_case()
    w['lattice'] = dict(w['lattice'], body_force=[2e-6, 0, 0])
    steps = 98
    a = cuda_lib.Simulation.from_workload(w)
    a.step(steps)
    b = cuda_lib.Simulation.from_workload(w)
    for _ in range(steps):
        for st in (cuda_lib.STAGE_FORCES, cuda_lib.STAGE_SPREAD, cuda_lib.STAGE_COLLIDE, cuda_lib.STAGE_INTERP):
            b.stage(st)
    ua, ub = a.fields()[1], b.fields()[1]
    Xa, Ua, Fa = a.markers()
    Xb, Ub, Fb = b.markers()
    from tests._cases import fluid_mask, rel_l2
    fl = fluid_mask(w['lattice'])
    assert rel_l2(ua[:, fl], ub[:, fl]) < 1e-6
    assert np.abs(Xa - Xb).max() < 1e-7
    assert np.abs(Fa - Fb).max() < 1e-4 * np.abs(Fb).max()
    assert a.diagnostics()['steps'] == steps
    ora = O.Oracle.from_workload(w)
    ora.step(steps)
    uo = ora.fields()[1]
    Xo, _, Fo = ora.markers()
    assert rel_l2(ua[:, fl], uo[:, fl]) < 1e-5
    assert np.abs(Xa - Xo).max() < 1e-5
    assert np.abs(Fa - Fo).max() < 1e-3 * np.abs(Fo).max()


def test_fused_path_timing_mode(cuda_lib):
    """ibm_lbm_set_timing_fused: a membrane suspension times its fused steps
    (starting at an even AA step, all but the last of the call's steps, the
    last one separate): forces and spreading slots zero, collisions and fused
    kernels timed; the results equal those of the graph path to rounding. A
    handle with tracers only is still timed stage by stage."""
    w = membrane_case()
    w['lattice'] = dict(w['lattice'], body_force=[2e-6, 0, 0])
    steps = 20
    a = cuda_lib.Simulation.from_workload(w)
    a.step(steps)
    b = cuda_lib.Simulation.from_workload(w)
    b.set_timing(steps, fused=True)
    b.step(steps)
    t = b.timing()
    b.set_timing(0)
    assert t['steps'] == steps - 2
    assert t['forces_ms'] == 0.0 and t['spread_ms'] == 0.0
    assert t['collide_ms'] > 0.0 and t['interp_ms'] > 0.0
    from tests._cases import fluid_mask, rel_l2
    fl = fluid_mask(w['lattice'])
    assert rel_l2(a.fields()[1][:, fl], b.fields()[1][:, fl]) < 1e-6
    assert np.abs(a.markers()[0] - b.markers()[0]).max() < 1e-7
    assert b.diagnostics()['steps'] == steps
    lat = WIDE['periodic']
    X, F = wide_tracers(lat, 500, 3)
    c = cuda_lib.Simulation(lat)
    c.set_markers(None, [], X)
    c.set_timing(4, fused=True)
    c.step(4)
    tc = c.timing()
    assert tc['steps'] == 4 and tc['spread_ms'] > 0.0

