"""Pins of the oracle's filament forces (bead chains: Eq. inPlanePotential
bonds, Eq. bendingEnergyWorm angles with theta0 = 180 degrees) and Morse
excluded volume (Eq. morsePotential), against the energy by central
differences, closed forms, conservation laws and special cases."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1704_04551_gb300 import inputs as I


def _chain_oracle(X, kBT_p, k_b, l0=1.0, lattice=None):
    lattice = lattice or dict(nx=16, ny=16, nz=16, tau=1.0, geometry=0)
    o = O.Oracle(lattice)
    body = I._body(I.BODY_FILAMENT, 0, X.shape[1], kBT_p=kBT_p, k_b=k_b, l0=l0)
    o.set_bodies([body], X)
    return o


def _bent_chain(n=9, seed=3, l0=1.0):
    rng = np.random.default_rng(seed)
    X, _ = I.filament(0, n, [2.0, 3.0, 4.0], [1.0, 0.3, -0.2], l0=l0)
    return X + 0.15 * rng.standard_normal(X.shape)


def _fd_forces(energy, X, h=1e-6):
    F = np.zeros_like(X)
    for a in range(3):
        for k in range(X.shape[1]):
            Xp, Xm = X.copy(), X.copy()
            Xp[a, k] += h
            Xm[a, k] -= h
            F[a, k] = -(energy(Xp) - energy(Xm)) / (2 * h)
    return F


@pytest.mark.parametrize('kBT_p,k_b', [(3e-3, 0.0), (0.0, 2e-3), (3e-3, 2e-3)])
def test_filament_forces_are_minus_energy_gradient(kBT_p, k_b):
    X = _bent_chain()
    o = _chain_oracle(X, kBT_p, k_b)
    F = o.filament_forces(0, X)
    Ffd = _fd_forces(lambda Y: o.filament_energy(0, Y), X)
    assert np.abs(F).max() > 1e-5
    assert np.allclose(F, Ffd, rtol=1e-5, atol=1e-10 * np.abs(F).max() + 1e-12)


def test_filament_forces_conserve_momentum_and_angular_momentum():
    X = _bent_chain(n=12, seed=5)
    F = _chain_oracle(X, 3e-3, 2e-3).filament_forces(0, X)
    assert np.abs(F.sum(axis=1)).max() < 1e-14
    torque = np.cross(X.T, F.T).sum(axis=0)
    assert np.abs(torque).max() < 1e-13


def test_straight_chain_at_rest_length_is_force_free():
    X, _ = I.filament(0, 10, [1.0, 2.0, 3.0], [0.3, -1.0, 0.5], l0=0.8)
    o = _chain_oracle(X, 3e-3, 2e-3, l0=0.8)
    assert np.abs(o.filament_forces(0, X)).max() < 1e-15
    # each bond at x = 1/2: WLC part kBT/p l_m / 4 = kBT/p l0 / 2, POW part k_p / l0 = 1.25 kBT/p l0
    assert abs(o.filament_energy(0, X) - 9 * 1.75 * 3e-3 * 0.8) < 1e-15


def test_right_angle_bend_energy_and_force():
    """Three beads with a 90-degree angle: U = k_b (pi/2)^2; each end bead is
    pushed to open the angle with |F| = 2 k_b (pi/2) / (bond length)."""
    X = np.array([[1.0, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 1.0, 0.0]]).T.copy()
    k_b = 1e-3
    o = _chain_oracle(X, 0.0, k_b)
    assert abs(o.filament_energy(0, X) - k_b * (math.pi / 2) ** 2) < 1e-15
    F = o.filament_forces(0, X)
    # end bead a = (1,0,0): force along -y (opening the angle), magnitude k_b * pi / |u|
    assert np.allclose(F[:, 0], [0.0, -k_b * math.pi, 0.0], atol=1e-15)
    assert np.allclose(F[:, 2], [-k_b * math.pi, 0.0, 0.0], atol=1e-15)


def test_bond_force_vanishes_at_rest_and_restores():
    X = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]]).T.copy()
    for l, sign in ((1.0, 0), (1.2, 1), (0.8, -1)):
        Y = X.copy()
        Y[0, 1] = l
        F = _chain_oracle(Y, 3e-3, 0.0).filament_forces(0, Y)
        if sign == 0:
            assert abs(F[0, 1]) < 1e-17
        else:
            assert np.sign(F[0, 0]) == sign and np.sign(F[0, 1]) == -sign  # stretched: pulled together


# ------------------------------------------------------------------- Morse
MORSE = dict(D0=2e-3, alpha=0.6, r0=1.3, rc=1.3)


def _morse_oracle(X, bodies, lattice=None):
    lattice = lattice or dict(nx=12, ny=10, nz=9, tau=1.0, geometry=0)
    o = O.Oracle(lattice)
    o.set_bodies(bodies, X)
    o.set_morse(**MORSE)
    return o


def _two_chains(d=1.0, lattice_shift=0.0):
    A, ba = I.filament(0, 4, [3.0 + lattice_shift, 4.0, 4.0], [1, 0, 0], l0=0.5, kBT_p=1e-3)
    B, bb = I.filament(4, 4, [3.2 + lattice_shift, 4.0 + d, 4.3], [1, 0.2, 0], l0=0.5, kBT_p=1e-3)
    return np.concatenate([A, B], axis=1), [ba, bb]


def test_morse_forces_are_minus_energy_gradient():
    X, bodies = _two_chains(d=0.9)
    o = _morse_oracle(X, bodies)
    F = o.morse_forces(X)
    Ffd = _fd_forces(o.morse_energy, X)
    assert np.abs(F).max() > 1e-5
    assert np.allclose(F, Ffd, rtol=1e-5, atol=1e-9 * np.abs(F).max())
    assert np.abs(F.sum(axis=1)).max() < 1e-15  # pairwise, equal and opposite


def test_morse_pair_closed_form_and_cutoff():
    """One pair of beads of different bodies: |F| = 2 alpha D0 (e^2 - e),
    e = exp(-alpha (r - r0)), repulsive below r0; nothing at r >= rc."""
    for r in (0.5, 1.0, 1.29, 1.3, 2.0):
        # two two-bead chains whose second beads are far from everything
        X = np.array([[2.0, 3.0, 1.0], [2.0, 3.0, -6.0], [2.0 + r, 3.0, 1.0], [2.0 + r, 3.0, 8.0]]).T.copy()
        bodies = [I._body(I.BODY_FILAMENT, 0, 2, l0=1.0), I._body(I.BODY_FILAMENT, 2, 2, l0=1.0)]
        o = _morse_oracle(X, bodies, lattice=dict(nx=40, ny=40, nz=40, tau=1.0, geometry=2, tube_radius=19.0))
        F = o.morse_forces(X)
        e = math.exp(-MORSE['alpha'] * (r - MORSE['r0']))
        mag = 2 * MORSE['alpha'] * MORSE['D0'] * (e * e - e) if r < MORSE['rc'] else 0.0
        assert abs(F[0, 0] + mag) < 1e-15 and abs(F[0, 2] - mag) < 1e-15, r
        assert np.abs(F[1:, :]).max() < 1e-15
        if r < MORSE['r0']:
            assert F[0, 0] < 0 < F[0, 2]


def test_morse_skips_same_body_rigid_and_tracers():
    X, bodies = _two_chains(d=0.9)
    o = _morse_oracle(X, [dict(bodies[0], count=8)])  # one body: no pairs
    assert np.abs(o.morse_forces(X)).max() == 0.0
    rigid = I._body(I.BODY_RIGID, 4, 4, kappa=0.01, mass=1.0, inertia=[1.0, 1.0, 1.0])
    o = _morse_oracle(X, [bodies[0], rigid])  # rigid markers do not take part
    assert np.abs(o.morse_forces(X)).max() == 0.0
    o = _morse_oracle(X, [bodies[0]])  # the rest are tracers
    assert np.abs(o.morse_forces(X)).max() == 0.0


def test_morse_uses_the_nearest_periodic_image():
    """A pair straddling the periodic x boundary feels the same force as the
    same pair in the middle of the box."""
    lat = dict(nx=12, ny=10, nz=9, tau=1.0, geometry=0)
    X, bodies = _two_chains(d=0.9)
    Fc = _morse_oracle(X, bodies, lat).morse_forces(X)
    Xw = X.copy()
    Xw[0, 4:] -= 12.0  # second chain one period to the left
    Fw = _morse_oracle(Xw, bodies, lat).morse_forces(Xw)
    assert np.allclose(Fc, Fw, atol=1e-15)
    assert np.abs(Fc).max() > 1e-5
