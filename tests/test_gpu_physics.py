"""Physics-level GPU checks: the Jeffery orbit (Sec. 3.1) and the full-size
tube workload checked through properties that hold at any size and through
outputs the FP64 oracle computes one body / one marker at a time."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1704_04551_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _in_plane_angle(q):
    R = I.quat_to_matrix(q)
    return math.atan2(R[1, 0], R[0, 0])  # major (body x) axis in the flow-gradient plane


def _jeffery_period(scale, direct=False):
    """Measured in-plane orbit period of the paper's Jeffery case (Sec. 3.1)
    at `scale` times its resolution: a = 6 s, b = c = 4.5 s, channel height
    60 s, grid 60 s x 60 s x 30 s, walls at -/+0.01, nu = s/6 (Re = aU/nu =
    0.36 at every scale), 812 s^2 markers, fluid started from the Couette
    profile; penalty tether (default) or the direct FSI forcing of Eq.
    FSIRigid. Returns (measured, closed form)."""
    from paper_1704_04551_gb300.binding import Simulation
    a, b, U = 6.0 * scale, 4.5 * scale, 0.01
    H, nz = int(round(60 * scale)), int(round(30 * scale))
    tau = 0.5 + 3 * (scale / 6.0)
    w = I.shear_ellipsoid(n=H, ny=H, nz=nz, tau=tau, wall_speed=U, axes=(a, b, b), seed=7,
                          quat=[1.0, 0.0, 0.0, 0.0], freq=int(round(9 * scale)), couette_init=True, direct=direct)
    T = I.jeffery_period(2 * U / H, a / b)
    sim = Simulation.from_workload(w)
    stride = max(100, int(T / 400))
    theta, t, prev = [0.0], [0], 0.0
    for k in range(int(1.2 * T / stride) + 1):
        sim.step(stride)
        ang = _in_plane_angle(sim.bodies()[0]['quat'])
        theta.append(theta[-1] + (ang - prev + math.pi) % (2 * math.pi) - math.pi)
        prev = ang
        t.append((k + 1) * stride)
        if theta[-1] < -2 * math.pi:
            break
    theta = np.array(theta)
    t = np.array(t, dtype=float)
    # the shear turns the body clockwise; a full period is the time the
    # major axis needs to turn by -2 pi
    i = int(np.argmax(theta <= -2 * math.pi))
    assert theta[i] <= -2 * math.pi, 'orbit too slow'
    f = (theta[i - 1] + 2 * math.pi) / (theta[i - 1] - theta[i])
    return t[i - 1] + f * stride, T


def test_jeffery_period_converges_to_closed_form(cuda_lib):
    """Jeffery's orbit T = (2 pi / gamma)(r + 1/r), gamma = 2U/H (Eq.
    jefferyOrbit): within 3 % at the paper's resolution (the paper reports a
    2.62 % mean angle error there), within 1 % at twice that resolution, and
    the error falls as the grid is refined (the paper: eps ~ N^-0.96)."""
    errs = {}
    for s in (1.0, 2.0):
        T_meas, T = _jeffery_period(s)
        errs[s] = abs(T_meas - T) / T
        print(f'Jeffery period, scale {s}: measured {T_meas:.0f} steps, closed form {T:.0f}, rel. error {errs[s]:.4f}')
    assert errs[1.0] < 0.03
    assert errs[2.0] < 0.01
    assert errs[2.0] < 0.6 * errs[1.0]


def test_jeffery_period_direct_forcing(cuda_lib):
    """With the paper's own rigid coupling (direct FSI forcing, Eq.
    FSIRigid) the period is within 1 % of the closed form already at the
    paper's resolution (measured 0.31 %; 0.35 % and 0.37 % at 1.5x and 2x:
    a residual that does not shrink with the grid, i.e. not discretisation
    error — the walls at 5 semi-axes confine the flow, which the closed form
    ignores)."""
    T_meas, T = _jeffery_period(1.0, direct=True)
    err = abs(T_meas - T) / T
    print(f'Jeffery period, direct forcing: measured {T_meas:.0f} steps, closed form {T:.0f}, rel. error {err:.4f}')
    assert err < 0.01


def test_full_size_tube_properties(cuda_lib):
    """256^3 tube, 3000 red cells, FP32, the launch configuration the
    benchmark times: mass conservation, finite fields, sampled membrane
    forces against the oracle body by body, sampled interpolated velocities
    against the delta-weighted sum of the returned fields."""
    from paper_1704_04551_gb300.binding import Simulation
    w = I.rbc_tube(n=256, radius=120.0, n_cells=3000, seed=1706)
    sim = Simulation.from_workload(w)
    d0 = sim.diagnostics()
    sim.step(20)
    d1 = sim.diagnostics()
    assert d1['fluid_cells'] == d0['fluid_cells']
    assert abs(d1['mass'] - d0['mass']) < 1e-6 * d0['mass']
    assert np.isfinite(d1['umax']) and d1['umax'] < 0.01
    X, U, F = sim.markers()
    # sampled bodies: the oracle's analytic membrane forces at the same positions
    ora = O.Oracle(dict(nx=8, ny=8, nz=8, tau=1.0, geometry=0))
    ora.set_mesh(w['mesh']['tris'], w['mesh']['rest_X'])
    V = w['mesh']['rest_X'].shape[1]
    rng = np.random.default_rng(0)
    for b in rng.choice(len(w['bodies']), 10, replace=False):
        body = dict(w['bodies'][b], first=0)
        Xb = X[:, w['bodies'][b]['first']:w['bodies'][b]['first'] + V]
        ora.set_bodies([body], Xb)
        # F of the last step was computed at the positions before the last advection
        Fo = ora.membrane_forces(0, Xb - U[:, w['bodies'][b]['first']:w['bodies'][b]['first'] + V])
        Fg = F[:, w['bodies'][b]['first']:w['bodies'][b]['first'] + V]
        scale = np.abs(Fo).max()
        err = np.abs(Fg - Fo).max()
        # FP32 floor: the area terms take A_t - A_t0 from FP32 areas, whose
        # rounding (2^-24 A_t, A_t ~ 0.4) times k_l (~3e-3) and |dA/dx| (~1)
        # over the ~6 triangles at a vertex gives ~5e-10 absolute
        print(f'body {b}: max|F| {scale:.3e}, max|dF| {err:.3e}')
        assert err < 1e-3 * scale + 2e-9, (b, err, scale)
    # sampled markers: U_k = sum_x u(x) delta(x - X_k) over fluid nodes, at the
    # position before the last advection, with the fields of that collision
    _, u = sim.fields()
    n = 256
    for k in rng.choice(X.shape[1], 200, replace=False):
        Xk = X[:, k] - U[:, k]
        base = np.floor(Xk).astype(int) - 1
        acc = np.zeros(3)
        for cz in range(4):
            for cy in range(4):
                for cx in range(4):
                    nxi, nyi, nzi = base + np.array([cx, cy, cz])
                    if (nyi - 127.5) ** 2 + (nzi - 127.5) ** 2 > 120.0 ** 2:
                        continue
                    wgt = O.phi(nxi - Xk[0]) * O.phi(nyi - Xk[1]) * O.phi(nzi - Xk[2])
                    acc += wgt * u[:, (nxi % n) + n * (nyi + n * nzi)]
        assert np.allclose(U[:, k], acc, rtol=2e-5, atol=1e-12), k
