"""Pins of the oracle's direct FSI forcing for rigid bodies (Eq. FSIRigid):
nodal force on the solid kappa (u(X) - U(X)) (kappa the volume a marker
stands for, rho_f = dt = 1), the opposite force on the fluid, Newton-Euler
update, markers carried rigidly by the body. Checked against closed forms
(uniform flow, pure spin), momentum exchange and rigidity."""
import math

import numpy as np

import oracle as O
from paper_1704_04551_gb300 import inputs as I

LAT = dict(nx=20, ny=18, nz=16, tau=0.8, geometry=0)


def _body(kappa=0.3, vel=(0.0, 0.0, 0.0), omega=(0.0, 0.0, 0.0), quat=None):
    q = np.array([0.9, 0.1, -0.3, 0.2]) if quat is None else np.asarray(quat, dtype=float)
    q = q / np.linalg.norm(q)
    X, b = I.rigid_ellipsoid([9.3, 8.6, 7.7], (4.0, 2.5, 2.0), q, 0, freq=5, kappa=kappa)
    b = dict(b, kind=3, vel=list(vel), omega=list(omega))
    return X, b


def _oracle(X, b, u0=None):
    o = O.Oracle(LAT)
    N = LAT['nx'] * LAT['ny'] * LAT['nz']
    u = None if u0 is None else np.tile(np.asarray(u0, dtype=float)[:, None], (1, N))
    o.set_equilibrium(None, u)
    o.set_bodies([b], X)
    return o


def test_body_moving_with_uniform_flow_feels_no_force():
    U0 = np.array([0.012, -0.007, 0.004])
    X, b = _body(vel=U0)
    o = _oracle(X, b, U0)
    o.stage_interpolate()  # U_k = U0 exactly (partition of unity); markers stay put
    Xa, U, _ = o.markers()
    assert np.abs(Xa - X).max() == 0.0
    assert np.allclose(U, U0[:, None], atol=1e-15)
    o.stage_forces()
    Xb, _, F = o.markers()
    assert np.abs(F).max() < 1e-15
    body = o.body(0)
    assert np.allclose(body['vel'], U0, atol=1e-16)
    assert np.allclose(Xb - X, U0[:, None], atol=1e-13)  # carried rigidly by V dt


def test_body_at_rest_in_uniform_flow_closed_form():
    """F_B = M kappa U0, so the body velocity jumps to M kappa U0 / m and the
    fluid receives -kappa U0 at every marker."""
    U0 = np.array([0.01, 0.0, -0.004])
    kappa = 0.3
    X, b = _body(kappa=kappa)
    o = _oracle(X, b, U0)
    o.stage_interpolate()
    o.stage_forces()
    _, _, F = o.markers()
    M = X.shape[1]
    assert np.allclose(F, -kappa * U0[:, None], atol=1e-16)
    assert np.allclose(o.body(0)['vel'], M * kappa * U0 / b['mass'], rtol=1e-14)


def test_spinning_body_in_fluid_at_rest_torque_closed_form():
    """u = 0: f_k = -kappa (omega x r_k), torque T = -kappa sum r x (omega x r)
    = -kappa sum (|r|^2 omega - r (r . omega)); the body-frame update then
    follows Euler's equation."""
    omega = np.array([0.002, -0.001, 0.003])
    kappa = 0.3
    X, b = _body(kappa=kappa, omega=omega)
    o = _oracle(X, b)
    o.stage_interpolate()
    o.stage_forces()
    _, _, F = o.markers()
    r = X - np.array(b['center'])[:, None]
    f_solid = -kappa * np.cross(omega, r.T).T
    assert np.allclose(F, -f_solid, atol=1e-16)
    T = -kappa * ((r * r).sum(axis=0).sum() * omega - r @ (r.T @ omega))
    # Euler's equations with torque, per component in the body frame:
    # I1 dw1 = t1 + (I2 - I3) w2 w3 and cyclic shifts (dt = 1)
    R = I.quat_to_matrix(b['quat'])
    w, t = R.T @ omega, R.T @ T
    nb = R.T @ np.array(o.body(0)['omega'])
    I1, I2, I3 = b['inertia']
    expect = (t[0] + (I2 - I3) * w[1] * w[2], t[1] + (I3 - I1) * w[2] * w[0], t[2] + (I1 - I2) * w[0] * w[1])
    got = (I1 * (nb[0] - w[0]), I2 * (nb[1] - w[1]), I3 * (nb[2] - w[2]))
    for g, e in zip(got, expect):
        assert abs(g - e) <= 1e-10 * abs(e) + 1e-22


def test_momentum_exchange_and_rigidity_over_coupled_steps():
    """Over coupled steps in a shear flow: the fluid's force on each step is
    exactly minus the body's momentum change, and the marker cloud stays
    rigid (all pairwise distances preserved)."""
    lat = dict(LAT, geometry=1, wall_u=[-0.01, 0.01])
    X, b = _body(kappa=0.25)
    o = O.Oracle(lat)
    nx, ny, nz = lat['nx'], lat['ny'], lat['nz']
    u0 = np.zeros((3, nz, ny, nx))
    u0[0] = (0.01 * (2.0 * (np.arange(ny) + 0.5) / ny - 1.0))[None, :, None]  # Couette profile
    o.set_equilibrium(None, u0.reshape(3, -1))
    o.set_bodies([b], X)
    d0 = np.linalg.norm(X[:, :, None] - X[:, None, :], axis=0)
    for _ in range(12):
        v0 = np.array(o.body(0)['vel'])
        o.step(1)
        _, _, F = o.markers()
        dv = np.array(o.body(0)['vel']) - v0
        assert np.allclose(b['mass'] * dv, -F.sum(axis=1), rtol=1e-12, atol=1e-12 * np.abs(F).sum())
    Xs, _, _ = o.markers()
    d1 = np.linalg.norm(Xs[:, :, None] - Xs[:, None, :], axis=0)
    assert np.abs(d1 - d0).max() < 1e-12
    assert np.abs(o.body(0)['omega']).max() > 1e-6  # the shear turns it
    assert math.isclose(np.linalg.norm(o.body(0)['quat']), 1.0, rel_tol=1e-14)
