"""Pins of the oracle's rigid-body rotation (Sec. 2.3: the body is advanced by
Newton's second law; Eq. FSIRigid gives its force). The explicit step
advances the body-frame angular velocity by Euler's equations and the
orientation quaternion by q += (0, omega) q / 2 with omega in the world
frame. Neither half is pinned by a sphere (isotropic inertia) or a spin about
a principal axis, where the gyroscopic term vanishes. Here a torque-free
body with three distinct principal moments, spun off every principal axis:

* Euler's equations for one step, written out per component from the
  textbook form I_1 dw_1/dt = (I_2 - I_3) w_2 w_3 and its cyclic shifts;
* conservation of the world-frame angular momentum L = R(q) I w_b. With the
  right signs the explicit step changes L only at second order in |w| per
  step; a flipped gyroscopic term, or the quaternion multiplied on the body
  side, changes it at first order (checked by hand against mutated copies
  of the oracle: 400x and 70x larger after one step)."""
import numpy as np

import oracle as O
from paper_1704_04551_gb300 import inputs as I

LAT = dict(nx=12, ny=12, nz=12, tau=0.8, geometry=0)
INERTIA = (50.0, 80.0, 130.0)


def _free_body(quat, omega):
    q = np.asarray(quat, dtype=float)
    q = q / np.linalg.norm(q)
    # kappa = 0: the tether carries no force, so the body is torque-free and
    # the fluid stays at rest
    X, b = I.rigid_ellipsoid([6.0, 6.0, 6.0], (3.0, 2.0, 1.5), q, 0, freq=3, kappa=0.0)
    b = dict(b, inertia=list(INERTIA), omega=list(omega))
    o = O.Oracle(LAT)
    o.set_equilibrium(None, None)
    o.set_bodies([b], X)
    return o, b


def test_euler_equations_one_step_per_component():
    """Identity orientation, so world and body frames coincide:
    I1 (w1' - w1) = (I2 - I3) w2 w3, I2 (w2' - w2) = (I3 - I1) w3 w1,
    I3 (w3' - w3) = (I1 - I2) w1 w2 (explicit step, dt = 1)."""
    w1, w2, w3 = 0.004, -0.003, 0.005
    o, _ = _free_body([1.0, 0.0, 0.0, 0.0], [w1, w2, w3])
    o.stage_forces()
    n1, n2, n3 = o.body(0)['omega']
    I1, I2, I3 = INERTIA
    expect = ((I2 - I3) * w2 * w3, (I3 - I1) * w3 * w1, (I1 - I2) * w1 * w2)
    got = (I1 * (n1 - w1), I2 * (n2 - w2), I3 * (n3 - w3))
    for g, e in zip(got, expect):
        assert abs(g - e) <= 1e-12 * abs(e)
    # the opposite sign of the gyroscopic term would give -expect
    assert all(abs(e) > 1e-4 for e in expect)


def test_euler_equations_rotated_body_frame():
    """The same law for a rotated body: the world-frame omega is taken to the
    body frame by R(q)^T before Euler's equations and back after."""
    q = np.array([0.8, 0.3, -0.4, 0.33])
    q = q / np.linalg.norm(q)
    Rm = I.quat_to_matrix(q)
    w_world = np.array([0.002, 0.006, -0.004])
    o, _ = _free_body(q, w_world)
    o.stage_forces()
    wb = Rm.T @ w_world
    nb = Rm.T @ np.array(o.body(0)['omega'])
    I1, I2, I3 = INERTIA
    expect = ((I2 - I3) * wb[1] * wb[2], (I3 - I1) * wb[2] * wb[0], (I1 - I2) * wb[0] * wb[1])
    got = (I1 * (nb[0] - wb[0]), I2 * (nb[1] - wb[1]), I3 * (nb[2] - wb[2]))
    for g, e in zip(got, expect):
        assert abs(g - e) <= 1e-10 * abs(e)


def test_orientation_turns_about_world_omega():
    """One step turns a body-fixed vector r_w by omega x r_w (world frame) up
    to second order in |omega|."""
    q = np.array([0.8, 0.3, -0.4, 0.33])
    q = q / np.linalg.norm(q)
    w = np.array([0.004, -0.003, 0.005])
    o, _ = _free_body(q, w)
    r_body = np.array([1.0, -2.0, 0.5])
    r0 = I.quat_to_matrix(q) @ r_body
    o.stage_forces()
    r1 = I.quat_to_matrix(np.array(o.body(0)['quat'])) @ r_body
    turn = np.array([w[1] * r0[2] - w[2] * r0[1], w[2] * r0[0] - w[0] * r0[2], w[0] * r0[1] - w[1] * r0[0]])
    err = np.linalg.norm(r1 - (r0 + turn))
    wn = np.linalg.norm(w)
    assert err < wn * wn * np.linalg.norm(r0)
    assert np.linalg.norm(turn) > 50 * wn * wn * np.linalg.norm(r0)


def test_world_angular_momentum_conserved_torque_free():
    """L = R(q) diag(I) w_b over 1000 explicit steps of about 7e-3 rad each
    (7 rad in all): the change per step stays below |w|^2 |L| and the total
    drift below 2 %. The flipped gyroscopic term breaks both within one step
    (5e-3 |L|) and the body-side quaternion product within 100 steps."""
    q = np.array([0.8, 0.3, -0.4, 0.33])
    w = np.array([0.004, -0.003, 0.005])
    o, _ = _free_body(q, w)
    Iv = np.array(INERTIA)

    def L():
        B = o.body(0)
        R = I.quat_to_matrix(np.array(B['quat']))
        return R @ (Iv * (R.T @ np.array(B['omega'])))

    L0 = L()
    nL = np.linalg.norm(L0)
    wn2 = float(w @ w)
    prev = L0
    worst_step, worst = 0.0, 0.0
    for _ in range(1000):
        o.stage_forces()
        cur = L()
        worst_step = max(worst_step, np.linalg.norm(cur - prev) / nL)
        worst = max(worst, np.linalg.norm(cur - L0) / nL)
        prev = cur
    assert worst_step < wn2
    assert worst < 0.02
    B = o.body(0)
    assert abs(np.linalg.norm(B['quat']) - 1.0) < 1e-14
    assert np.allclose(B['center'], [6.0, 6.0, 6.0], atol=0.0)  # no force, no drift
