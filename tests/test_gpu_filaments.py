"""GPU parity of the filament forces (bead chains, Sec. 2.2) and of the Morse
excluded volume between bodies (Eq. morsePotential), through the C ABI,
against the FP64 oracle: forces of one stage for several geometries and
bin layouts (including fewer than three bins on a periodic axis), then a
coupled run of red cells and filaments in a channel.

Tolerances: FP32 force arithmetic on positions rounded once to FP32
fractions (~3e-8 lu), so forces agree to ~1e-6 of their scale; the bounds
are 1e-4 of the largest force. The coupled run uses the coupled-parity
bounds of the other tests (relative L2 of u 1e-5, marker positions 1e-5 lu).
"""
import numpy as np
import pytest

import oracle as O
from paper_1704_04551_gb300 import inputs as I
from tests._cases import fluid_mask, rel_l2

pytestmark = pytest.mark.gpu


def _forces_pair(cuda_lib, w):
    from paper_1704_04551_gb300.binding import Simulation
    sim = Simulation.from_workload(w)
    ora = O.Oracle.from_workload(w)
    sim.stage(cuda_lib.STAGE_FORCES)
    ora.stage_forces()
    return sim.markers()[2], ora.markers()[2]


def _chains(lat, n_chains, beads, l0, seed, noise, moduli, inside=None):
    """Bent chains at random positions and directions (unwrapped positions
    may leave the box on periodic axes)."""
    rng = np.random.default_rng(seed)
    Xs, bodies, first = [], [], 0
    while len(bodies) < n_chains:
        start = rng.random(3) * np.array([lat['nx'], lat['ny'], lat['nz']])
        d = rng.standard_normal(3)
        X, b = I.filament(first, beads, start, d, l0=l0, **moduli)
        X = X + noise * rng.standard_normal(X.shape)
        if inside is not None and not inside(X):
            continue
        Xs.append(X)
        bodies.append(b)
        first += beads
    return np.concatenate(Xs, axis=1), bodies


def test_filament_forces_match_oracle(cuda_lib):
    lat = dict(nx=40, ny=12, nz=10, tau=0.8, geometry=0)
    X, bodies = _chains(lat, 6, 17, 0.9, seed=11, noise=0.2, moduli=dict(kBT_p=3e-3, k_b=2e-3))
    bodies[1]['k_b'] = 0.0  # stretching only
    bodies[2]['kBT_p'] = 0.0  # bending only
    w = dict(lattice=lat, mesh=None, bodies=bodies, X=X)
    Fg, Fo = _forces_pair(cuda_lib, w)
    scale = np.abs(Fo).max()
    assert scale > 1e-4
    assert np.abs(Fg - Fo).max() < 1e-4 * scale
    # a straight chain at its rest length carries no force
    Xs, bs = I.filament(0, 20, [3.0, 4.0, 5.0], [1.0, 0.5, 0.2], l0=0.8, kBT_p=3e-3, k_b=2e-3)
    Fg, _ = _forces_pair(cuda_lib, dict(lattice=lat, mesh=None, bodies=[bs], X=Xs))
    assert np.abs(Fg).max() < 1e-6 * 3e-3


MORSE_CASES = {
    'periodic': (dict(nx=24, ny=20, nz=18, tau=1.0, geometry=0), dict(D0=2e-3, alpha=0.6, r0=1.3, rc=1.3)),
    'ywalls': (dict(nx=24, ny=20, nz=18, tau=1.0, geometry=1), dict(D0=2e-3, alpha=0.6, r0=1.3, rc=1.3)),
    'tube': (dict(nx=24, ny=21, nz=21, tau=1.0, geometry=2, tube_radius=9.5), dict(D0=2e-3, alpha=0.6, r0=1.3, rc=1.3)),
    'few_bins': (dict(nx=16, ny=5, nz=4, tau=1.0, geometry=0), dict(D0=2e-3, alpha=0.6, r0=2.1, rc=2.1)),
}


@pytest.mark.parametrize('case', list(MORSE_CASES))
def test_morse_forces_match_oracle(cuda_lib, case):
    """Bead chains with no forces of their own, packed densely: the marker
    forces are the Morse forces alone (pairs across periodic boundaries,
    near walls, and with fewer than three bins on an axis)."""
    lat, morse = MORSE_CASES[case]
    inside = None
    if lat['geometry'] == 1:
        inside = lambda X: X[1].min() > 0.0 and X[1].max() < lat['ny'] - 1.0
    if lat['geometry'] == 2:
        yc = zc = (lat['ny'] - 1) / 2
        inside = lambda X: ((X[1] - yc) ** 2 + (X[2] - zc) ** 2).max() < (lat['tube_radius'] - 1.0) ** 2
    X, bodies = _chains(lat, 60, 8, 0.7, seed=17, noise=0.1, moduli={}, inside=inside)
    w = dict(lattice=lat, mesh=None, bodies=bodies, X=X, morse=morse)
    Fg, Fo = _forces_pair(cuda_lib, w)
    scale = np.abs(Fo).max()
    assert scale > 1e-5, 'no pair within the cutoff'
    assert np.abs(Fg - Fo).max() < 1e-4 * scale
    assert np.abs(Fg.sum(axis=1)).max() < 1e-4 * scale  # equal and opposite pairs


def _sliding_chains(lat, morse, seed):
    """Dense bead chains (no forces of their own) pushed in different
    directions, so that neighbours change while they move."""
    X, bodies = _chains(lat, 60, 8, 0.7, seed=seed, noise=0.1, moduli={})
    rng = np.random.default_rng(seed + 1)
    push = np.concatenate([np.repeat(rng.standard_normal((3, 1)), 8, axis=1) for _ in bodies], axis=1)
    return dict(lattice=lat, mesh=None, bodies=bodies, X=X, morse=morse), 4e-3 * push


def test_morse_lists_follow_moving_markers(cuda_lib):
    """Solid-only steps of sliding chains (terminal speed ~0.02 lu per step,
    so the lists are rebuilt many times): the trajectory with Morse forces
    matches the oracle's, which sums every pair directly."""
    from paper_1704_04551_gb300.binding import Simulation
    lat, morse = MORSE_CASES['periodic']
    w, push = _sliding_chains(lat, dict(morse, D0=5e-4), seed=23)
    sim = Simulation.from_workload(w)
    ora = O.Oracle.from_workload(w)
    v = None
    for _ in range(4):
        sim.solid_steps(15, 1.0, 0.2, 1.0, push)
        v = ora.solid_steps(15, 1.0, 0.2, 1.0, push, v=v)
    Xg, _, Fg = sim.markers()
    Xo, _, Fo = ora.markers()
    assert np.abs(Xo - w['X']).max() > 1.0  # moved by several list skins (0.2 lu)
    assert np.abs(Xg - Xo).max() < 1e-4
    assert np.abs(Fo).max() > 1e-5, 'no pair within the cutoff'
    assert np.abs(Fg - Fo).max() < 1e-3 * np.abs(Fo).max()


def test_morse_list_overflow_uses_the_full_gather(cuda_lib):
    """A cutoff wide enough that markers have more neighbours within
    rc + skin than a list holds: the forces still match the oracle, at the
    first stage and after the markers have moved."""
    from paper_1704_04551_gb300.binding import Simulation
    lat, _ = MORSE_CASES['periodic']
    w, push = _sliding_chains(lat, dict(D0=1e-6, alpha=0.6, r0=5.0, rc=5.0), seed=29)
    sim = Simulation.from_workload(w)
    ora = O.Oracle.from_workload(w)
    d = np.linalg.norm(w['X'][:, :, None] - w['X'][:, None, :], axis=0)  # no image needed for a lower bound
    assert (d < 6.5).sum(axis=1).max() > 60  # well above the 48 entries of a list
    sim.stage(cuda_lib.STAGE_FORCES)
    ora.stage_forces()
    Fg, Fo = sim.markers()[2], ora.markers()[2]
    assert np.abs(Fg - Fo).max() < 1e-4 * np.abs(Fo).max()
    sim.solid_steps(10, 1.0, 0.2, 1.0, push)
    ora.solid_steps(10, 1.0, 0.2, 1.0, push)
    Xg, _, Fg = sim.markers()
    Xo, _, Fo = ora.markers()
    assert np.abs(Xg - Xo).max() < 1e-4
    assert np.abs(Fg - Fo).max() < 1e-3 * np.abs(Fo).max()


def test_coupled_cells_and_filaments_match_oracle(cuda_lib):
    """Three red cells and six 12-bead filaments in a 48 x 40 x 40 channel
    with Morse excluded volume (lattice parameters of the mixed suspension),
    60 coupled steps."""
    from paper_1704_04551_gb300.binding import Simulation
    w = I.mixed_suspension(shape=(48, 40, 40), n_cells=3, n_filaments=6, beads=12, seed=5)
    w['lattice'] = dict(w['lattice'], body_force=[2e-6, 0.0, 0.0])
    # stiffer than physical so that every term matters within 60 steps
    for b in w['bodies']:
        if b['kind'] == I.BODY_FILAMENT:
            b.update(kBT_p=2e-3, k_b=1e-3)
    w['morse'] = dict(D0=1e-3, alpha=0.6, r0=1.32, rc=1.32)
    rng = np.random.default_rng(6)
    w['X'] = w['X'] + 0.05 * rng.standard_normal(w['X'].shape)
    sim = Simulation.from_workload(w)
    ora = O.Oracle.from_workload(w)
    sim.step(60)
    ora.step(60)
    fl = fluid_mask(w['lattice'])
    _, ug = sim.fields()
    _, uo = ora.fields()
    assert rel_l2(ug[:, fl], uo[:, fl]) < 1e-5
    Xg, _, Fg = sim.markers()
    Xo, _, Fo = ora.markers()
    assert np.abs(Xg - Xo).max() < 1e-5
    assert np.abs(Fg - Fo).max() < 1e-3 * np.abs(Fo).max()


def test_morse_and_filament_errors(cuda_lib):
    from paper_1704_04551_gb300.binding import E_ARG, IbmLbmError, Simulation
    lat = dict(nx=16, ny=8, nz=8, tau=1.0, geometry=0)
    sim = Simulation(lat)
    sim.set_lattice()
    with pytest.raises(IbmLbmError) as e:
        sim.set_morse(1e-3, 0.0, 1.0, 1.0)  # alpha must be positive
    assert e.value.code == E_ARG
    sim.set_morse(1e-3, 0.5, 1.0, 0.0)  # rc <= 0: switched off
    X, b = I.filament(0, 1, [3.0, 3.0, 3.0], [1, 0, 0], l0=1.0)
    with pytest.raises(IbmLbmError) as e:
        sim.set_markers(None, [b], X)  # a filament needs two beads
    assert e.value.code == E_ARG
    X, b = I.filament(0, 4, [3.0, 3.0, 3.0], [1, 0, 0], l0=1.0)
    with pytest.raises(IbmLbmError) as e:
        sim.set_markers(None, [dict(b, l0=0.0)], X)  # and a positive rest length
    assert e.value.code == E_ARG
