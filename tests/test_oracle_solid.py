"""Pins of the oracle's solid-only dynamics (the membrane stretching
validation of Sec. 3.2: velocity Verlet with viscous damping, no fluid):
exact kinematics under a constant force, the damped terminal velocity,
momentum conservation of the internal forces, and monotone relaxation of a
deformed red-cell membrane to its rest shape."""
import numpy as np

import oracle as O
from paper_1704_04551_gb300 import inputs as I

LAT = dict(nx=40, ny=40, nz=40, tau=1.0, geometry=0)


def _cell(deform, seed=3, freq=5):
    w = I.rbc_tube(n=40, radius=18.0, n_cells=1, seed=seed, freq=freq, steps=0)
    rng = np.random.default_rng(seed)
    X = w['X'] + deform * rng.standard_normal(w['X'].shape)
    b = dict(w['bodies'][0], kBT_p=2e-3, k_b=1e-3, k_l=5e-3, k_g=4e-3, k_v=3e-3)
    o = O.Oracle(LAT)
    o.set_mesh(w['mesh']['tris'], w['mesh']['rest_X'])
    o.set_bodies([b], X)
    return o, X, b


def test_constant_force_kinematics_are_exact():
    """Velocity Verlet integrates a constant force exactly:
    X = X0 + a t^2 / 2, v = a t (tracers: no forces of their own)."""
    rng = np.random.default_rng(1)
    X0 = 10 + 5 * rng.random((3, 7))
    f = 1e-3 * (2 * rng.random((3, 7)) - 1)
    o = O.Oracle(LAT)
    o.set_bodies([], X0)
    m, dt, n = 2.5, 0.4, 30
    v = o.solid_steps(n, dt, 0.0, m, f)
    X, _, _ = o.markers()
    t = n * dt
    assert np.allclose(v, f / m * t, rtol=1e-13, atol=0)
    assert np.allclose(X, X0 + 0.5 * f / m * t * t, rtol=1e-14, atol=1e-13)


def test_damped_terminal_velocity():
    """With damping gamma the velocity under a constant force tends to
    f / (m gamma), geometrically with ratio (1 - gamma dt/2)/(1 + gamma dt/2)."""
    X0 = np.full((3, 1), 20.0)
    f = np.array([[2e-3], [-1e-3], [5e-4]])
    o = O.Oracle(LAT)
    o.set_bodies([], X0)
    m, dt, g = 1.5, 0.5, 0.2
    v = o.solid_steps(200, dt, g, m, f)
    assert np.allclose(v, f / (m * g), rtol=1e-12)
    v1 = O.Oracle(LAT)
    v1.set_bodies([], X0)
    v_one = v1.solid_steps(1, dt, g, m, f)
    r = (1 - g * dt / 2) / (1 + g * dt / 2)
    assert np.allclose(v_one, f / (m * g) * (1 - r), rtol=1e-13)


def test_internal_forces_conserve_momentum():
    o, X, b = _cell(0.1)
    v = o.solid_steps(50, 0.5, 0.0, 1.0)
    assert np.abs(v.sum(axis=1)).max() < 1e-13
    assert np.abs(v).max() > 1e-4


def test_deformed_membrane_relaxes_monotonically():
    o, X, b = _cell(0.15)
    energies, v = [], None
    for _ in range(20):
        Xc, _, _ = o.markers()
        energies.append(o.membrane_energy(0, Xc))
        v = o.solid_steps(50, 0.5, 0.05, 1.0, v=v)
    e = np.array(energies)
    assert np.all(np.diff(e) < 0)
    # close to the rest energy (the k_p/l terms) and nearly force-free at the end
    rest = o.membrane_energy(0, _cell(0.0)[1])
    assert (e[-1] - rest) < 1e-3 * (e[0] - rest)
