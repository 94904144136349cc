"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances (FP32 arithmetic on FP64 inputs):
  * populations after a few collide-stream stages: the kernel works on the
    deviations d_i = f_i - w_i (|d| <= ~0.01 here) with ~20 FP32 operations
    per value, so |f_gpu - f_oracle| <= 20 * 2^-24 * 0.01 * steps ~ 1e-8;
    the test allows 2e-7.
  * spread force density / interpolated velocity: 64 FP32 products and sums
    of weights in [0, 1/2] -> relative error ~ 64 * 2^-24 ~ 4e-6 of the
    largest value; the test allows 2e-5.
  * membrane forces: FP32 geometry from FP64 differences; the force terms
    are differences of O(1) quantities under deformations of ~0.1, so the
    relative error is ~1e-6; the test allows 1e-4 of max |F|.
  * whole coupled runs: relative L2 velocity error <= 1e-5 for FP32 storage
    and <= 1e-3 for FP16-deviation storage (the stated targets).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1704_04551_gb300 import inputs as I
from tests._cases import LATTICES, fluid_mask, markers_inside, membrane_case, rel_l2, shape

pytestmark = pytest.mark.gpu


def _pair(lat, storage='f32'):
    from paper_1704_04551_gb300.binding import Simulation
    return Simulation(lat, storage=storage), O.Oracle(lat)


@pytest.mark.parametrize('geom', list(LATTICES))
def test_collide_stream_matches_oracle(cuda_lib, geom):
    lat = LATTICES[geom]
    sim, ora = _pair(lat)
    sim.set_markers(None, [], np.zeros((3, 0)))
    ora.set_bodies([], np.zeros((3, 0)))
    fl = fluid_mask(lat)
    f0 = I.random_populations(shape(lat), 11, amp=0.02)
    f0[:, ~fl] = 0.0
    sim.set_populations(f0)
    ora.set_populations(f0)
    assert np.abs(sim.populations()[:, fl] - f0[:, fl]).max() < 1e-8
    for s in range(3):   # even, odd, even: both AA parities and the swapped layout
        sim.stage(cuda_lib.STAGE_COLLIDE)
        ora.stage_collide_stream()
        fg, fo = sim.populations(), ora.populations()
        assert np.abs(fg[:, fl] - fo[:, fl]).max() < 2e-7, f'step {s}'
        rg, ug = sim.fields()
        ro, uo = ora.fields()
        assert np.abs(rg[fl] - ro[fl]).max() < 2e-7
        assert np.abs(ug[:, fl] - uo[:, fl]).max() < 2e-7


@pytest.mark.parametrize('geom', list(LATTICES))
def test_spread_matches_oracle(cuda_lib, geom):
    lat = LATTICES[geom]
    sim, ora = _pair(lat)
    X = markers_inside(lat, 300, 5)
    F = 1e-3 * (2 * np.random.default_rng(6).random(X.shape) - 1)
    sim.set_markers(None, [], X)
    ora.set_bodies([], X)
    sim.set_marker_forces(F)
    ora.set_marker_forces(F)
    sim.stage(cuda_lib.STAGE_SPREAD)
    ora.stage_spread()
    gg, go = sim.force_density(), ora.force_density()
    assert np.abs(gg - go).max() < 2e-5 * np.abs(go).max()
    assert np.allclose(gg.sum(1), go.sum(1), rtol=1e-5, atol=1e-9)


@pytest.mark.parametrize('geom', list(LATTICES))
def test_interpolate_matches_oracle(cuda_lib, geom):
    lat = LATTICES[geom]
    sim, ora = _pair(lat)
    X = markers_inside(lat, 300, 7)
    rho, u = I.random_fields(shape(lat), 8)
    sim.set_lattice(rho, u)
    ora.set_equilibrium(rho, u)
    sim.set_markers(None, [], X)
    ora.set_bodies([], X)
    sim.stage(cuda_lib.STAGE_INTERP)
    ora.stage_interpolate()
    Xg, Ug, _ = sim.markers()
    Xo, Uo, _ = ora.markers()
    assert np.abs(Ug - Uo).max() < 2e-5 * np.abs(Uo).max()
    assert np.abs(Xg - Xo).max() < 1e-6


_membrane_case = membrane_case


def test_membrane_forces_match_oracle(cuda_lib):
    from paper_1704_04551_gb300.binding import Simulation
    w = _membrane_case()
    sim = Simulation.from_workload(w)
    ora = O.Oracle.from_workload(w)
    sim.stage(cuda_lib.STAGE_FORCES)
    ora.stage_forces()
    _, _, Fg = sim.markers()
    _, _, Fo = ora.markers()
    scale = np.abs(Fo).max()
    assert scale > 1e-5
    assert np.abs(Fg - Fo).max() < 1e-4 * scale
    # each term alone
    for term in ('kBT_p', 'k_b', 'k_l', 'k_g', 'k_v'):
        w2 = dict(w)
        zero = dict(kBT_p=0.0, k_b=0.0, k_l=0.0, k_g=0.0, k_v=0.0)
        zero[term] = 3e-3
        w2['bodies'] = [dict(b, **zero) for b in w['bodies']]
        sim = Simulation.from_workload(w2)
        ora = O.Oracle.from_workload(w2)
        sim.stage(cuda_lib.STAGE_FORCES)
        ora.stage_forces()
        Fg, Fo = sim.markers()[2], ora.markers()[2]
        scale = np.abs(Fo).max()
        assert np.abs(Fg - Fo).max() < 1e-4 * scale, term


def test_rigid_tether_forces_and_pose(cuda_lib):
    from paper_1704_04551_gb300.binding import Simulation
    w = I.shear_ellipsoid(n=24, axes=(5.0, 2.5, 2.5), seed=31)
    sim = Simulation.from_workload(w)
    ora = O.Oracle.from_workload(w)
    # displace the markers with a non-uniform flow, then tether forces
    rng = np.random.default_rng(3)
    u = 0.01 * (2 * rng.random((3, sim.N)) - 1)
    sim.set_lattice(None, u)
    ora.set_equilibrium(None, u)
    sim.stage(cuda_lib.STAGE_INTERP)
    ora.stage_interpolate()
    sim.stage(cuda_lib.STAGE_FORCES)
    ora.stage_forces()
    Xg, _, Fg = sim.markers()
    Xo, _, Fo = ora.markers()
    assert np.abs(Xg - Xo).max() < 1e-6
    assert np.abs(Fg - Fo).max() < 1e-4 * np.abs(Fo).max()
    bg, bo = sim.bodies()[0], ora.body(0)
    for k in ('center', 'quat', 'vel', 'omega'):
        assert np.allclose(bg[k], bo[k], rtol=1e-5, atol=1e-9), k


def _run_pair(w, steps, storage='f32'):
    from paper_1704_04551_gb300.binding import Simulation
    sim = Simulation.from_workload(w, storage=storage)
    ora = O.Oracle.from_workload(w)
    sim.step(steps)
    ora.step(steps)
    return sim, ora


def test_coupled_rigid_ellipsoid_500_steps(cuda_lib):
    """Rigid prolate ellipsoid 6x3x3 (812 markers) in a 32^3 Couette cell,
    tau = 0.8, walls at -/+0.02: 500 coupled steps."""
    w = I.shear_ellipsoid(n=32, steps=500)
    sim, ora = _run_pair(w, 500)
    _, ug = sim.fields()
    _, uo = ora.fields()
    assert rel_l2(ug, uo) < 1e-5
    Xg, Ug, Fg = sim.markers()
    Xo, Uo, Fo = ora.markers()
    assert np.abs(Xg - Xo).max() < 1e-5
    assert rel_l2(Ug, Uo) < 1e-4
    bg, bo = sim.bodies()[0], ora.body(0)
    assert np.allclose(bg['omega'], bo['omega'], rtol=1e-3, atol=1e-9)
    assert np.allclose(bg['quat'], bo['quat'], atol=1e-6)


def test_coupled_membranes_tube(cuda_lib):
    """Three deformed red-cell membranes in a 40^3 tube (R = 16), 60 steps."""
    w = _membrane_case()
    w['lattice'] = dict(w['lattice'], body_force=[2e-6, 0, 0])
    sim, ora = _run_pair(w, 60)
    fl = fluid_mask(w['lattice'])
    _, ug = sim.fields()
    _, uo = ora.fields()
    assert rel_l2(ug[:, fl], uo[:, fl]) < 1e-5
    Xg, _, Fg = sim.markers()
    Xo, _, Fo = ora.markers()
    assert np.abs(Xg - Xo).max() < 1e-5
    assert np.abs(Fg - Fo).max() < 1e-3 * np.abs(Fo).max()


@pytest.mark.parametrize('storage,tol', [('f16', 1e-3), ('bf16', 3e-2)])
def test_half_storage_error_bound(cuda_lib, storage, tol):
    """FP16 deviation storage meets the 1e-3 relative L2 velocity target;
    BF16 (8-bit significand) is only checked against a loose bound."""
    w = I.shear_ellipsoid(n=32, steps=300)
    sim, ora = _run_pair(w, 300, storage=storage)
    _, ug = sim.fields()
    _, uo = ora.fields()
    assert rel_l2(ug, uo) < tol


def test_step_graph_matches_stages(cuda_lib):
    """ibm_lbm_step (CUDA-graph chunks) and stage-by-stage execution agree."""
    from paper_1704_04551_gb300.binding import Simulation
    w = I.shear_ellipsoid(n=24, axes=(5.0, 2.5, 2.5), seed=9)
    a = Simulation.from_workload(w)
    b = Simulation.from_workload(w)
    a.step(37)
    for _ in range(37):
        for st in (cuda_lib.STAGE_FORCES, cuda_lib.STAGE_SPREAD, cuda_lib.STAGE_COLLIDE, cuda_lib.STAGE_INTERP):
            b.stage(st)
    assert np.abs(a.populations() - b.populations()).max() < 1e-9
    assert np.abs(a.markers()[0] - b.markers()[0]).max() < 1e-9
    assert a.diagnostics()['steps'] == 37


def test_mass_and_momentum_laws_on_gpu(cuda_lib):
    """Periodic box with a uniform force: FP64 mass stays constant and the
    momentum grows by N g0 per step (Guo forcing)."""
    from paper_1704_04551_gb300.binding import Simulation
    lat = dict(nx=48, ny=20, nz=18, tau=0.9, geometry=0, body_force=[1e-5, -2e-5, 3e-6])
    sim = Simulation(lat)
    sim.set_markers(None, [], np.zeros((3, 0)))
    rho, u = I.random_fields(shape(lat), 4)
    sim.set_lattice(rho, u)
    sim.step(1)
    d1 = sim.diagnostics()
    sim.step(40)
    d2 = sim.diagnostics()
    N = np.prod(shape(lat))
    assert d2['fluid_cells'] == N
    assert abs(d2['mass'] - d1['mass']) < 1e-6 * N
    assert np.allclose(d2['momentum'] - d1['momentum'], 40 * N * np.array(lat['body_force']), rtol=2e-3)


def test_errors_are_reported(cuda_lib):
    from paper_1704_04551_gb300.binding import IbmLbmError, Simulation
    sim = Simulation(LATTICES['periodic'])
    with pytest.raises(IbmLbmError):
        sim.set_markers(None, [dict(kind=0, first=0, count=5)], np.zeros((3, 5)))  # membrane without mesh
    with pytest.raises(IbmLbmError):
        sim.set_markers(None, [dict(kind=1, first=0, count=5, mass=1.0, inertia=[1, 1, 1])], np.zeros((3, 3)))
    with pytest.raises(IbmLbmError):
        sim.step(-1)
    for bad in (np.nan, np.inf, 2.0 ** 30):  # floor(X) must fit an int32
        X = np.full((3, 4), 5.0)
        X[1, 2] = bad
        with pytest.raises(IbmLbmError) as e:
            sim.set_markers(None, [], X)
        assert e.value.code == cuda_lib.E_ARG
    sim.set_markers(None, [], np.zeros((3, 0)))
    sim.step(0)


def test_positions_round_trip_and_unwrapped_coordinates(cuda_lib):
    """set/get returns the FP64 positions unchanged, negative and far
    unwrapped coordinates included; markers moved by whole periods on the
    periodic lattice spread and interpolate exactly as the unshifted ones
    (the stencil cache floors negative coordinates correctly)."""
    lat = LATTICES['periodic']
    nx, ny, nz = shape(lat)
    rng = np.random.default_rng(12)
    X = np.concatenate([rng.uniform(-3e5, 3e5, (3, 50)), rng.uniform(-2, 2, (3, 50)),
                        np.round(rng.uniform(-100, 100, (3, 20)) * 2.0 ** 32) / 2.0 ** 32], axis=1)
    sim = cuda_lib.Simulation(lat)
    sim.set_markers(None, [], X)
    Xg, _, _ = sim.markers()
    assert np.array_equal(Xg, X)
    X0 = np.round(markers_inside(lat, 200, 9) * 2.0 ** 32) / 2.0 ** 32  # so that X0 + shift is exact
    shift = np.array([-nx, 2 * ny, -3 * nz], dtype=float)[:, None]
    F = 1e-3 * (2 * rng.random(X0.shape) - 1)
    rho, u = I.random_fields(shape(lat), 3)
    out = []
    for Xs in (X0, X0 + shift):
        s = cuda_lib.Simulation(lat)
        s.set_lattice(rho, u)
        s.set_markers(None, [], Xs)
        s.set_marker_forces(F)
        s.stage(cuda_lib.STAGE_SPREAD)
        g = s.force_density()
        s.stage(cuda_lib.STAGE_INTERP)
        Xa, U, _ = s.markers()
        out.append((g, U, Xa - Xs))
    (g0, U0, d0), (g1, U1, d1) = out
    assert np.abs(g1 - g0).max() <= 1e-6 * np.abs(g0).max()  # same sums, another order of float atomics
    assert np.array_equal(U1, U0)
    assert np.abs(d1 - d0).max() <= 2.0 ** -32


def test_rigid_direct_forcing_stage_and_coupled(cuda_lib):
    """The paper's direct FSI forcing (Eq. FSIRigid) for a rigid ellipsoid:
    one interpolation + forces stage in a random flow (marker forces, the
    rigidly moved markers, the new pose), then 300 coupled steps in a
    Couette cell, against the oracle."""
    from paper_1704_04551_gb300.binding import Simulation
    w = I.shear_ellipsoid(n=24, axes=(5.0, 2.5, 2.5), seed=33, direct=True)
    sim = Simulation.from_workload(w)
    ora = O.Oracle.from_workload(w)
    rng = np.random.default_rng(4)
    u = 0.01 * (2 * rng.random((3, sim.N)) - 1)
    sim.set_lattice(None, u)
    ora.set_equilibrium(None, u)
    sim.stage(cuda_lib.STAGE_INTERP)
    ora.stage_interpolate()
    sim.stage(cuda_lib.STAGE_FORCES)
    ora.stage_forces()
    Xg, _, Fg = sim.markers()
    Xo, _, Fo = ora.markers()
    assert np.abs(Fg - Fo).max() < 1e-4 * np.abs(Fo).max()
    assert np.abs(Xg - Xo).max() < 1e-9
    bg, bo = sim.bodies()[0], ora.body(0)
    for k in ('center', 'quat', 'vel', 'omega'):
        assert np.allclose(bg[k], bo[k], rtol=1e-5, atol=1e-10), k
    w = I.shear_ellipsoid(n=32, steps=300, direct=True, couette_init=True)
    sim, ora = _run_pair(w, 300)
    _, ug = sim.fields()
    _, uo = ora.fields()
    assert rel_l2(ug, uo) < 1e-5
    Xg, _, _ = sim.markers()
    Xo, _, _ = ora.markers()
    assert np.abs(Xg - Xo).max() < 1e-5
    bg, bo = sim.bodies()[0], ora.body(0)
    assert np.allclose(bg['omega'], bo['omega'], rtol=1e-3, atol=1e-9)
    assert np.allclose(bg['quat'], bo['quat'], atol=1e-6)
