"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks a property that an independent fact determines (a moment
identity, a closed-form flow, a conservation law, a printed number, a
finite-difference derivative, a polyhedron with known area/volume/angles),
chosen so that a dropped term, a wrong sign or index, or a transposed operand
in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1704_04551_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    out = {}
    with open(os.path.join(HERE, 'golden', 'paper_cases.txt')) as f:
        for line in f:
            line = line.split('#', 1)[0].strip()
            if line:
                k, v = line.split()
                out[k] = float(v)
    return out


# ----------------------------------------------------------------------------
# D3Q19 lattice, equilibrium and Guo forcing (Sec. 2.1)
# ----------------------------------------------------------------------------
def test_lattice_isotropy():
    c, w = O.lattice()
    c = c.astype(np.float64)
    cs2 = 1.0 / 3.0  # Eq. viscosity: nu = cs^2 (tau - 1/2) = (tau - 1/2)/3
    assert abs(w.sum() - 1) < 1e-15
    assert np.abs(w @ c).max() < 1e-16
    m2 = np.einsum('i,ia,ib->ab', w, c, c)
    assert np.allclose(m2, cs2 * np.eye(3), atol=1e-15)
    m4 = np.einsum('i,ia,ib,ic,id->abcd', w, c, c, c, c)
    d = np.eye(3)
    iso = cs2 ** 2 * (np.einsum('ab,cd->abcd', d, d) + np.einsum('ac,bd->abcd', d, d)
                      + np.einsum('ad,bc->abcd', d, d))
    assert np.allclose(m4, iso, atol=1e-15)
    # every velocity has its opposite; 19 distinct vectors of norm^2 0, 1 or 2
    assert len({tuple(v) for v in c.astype(int)}) == 19
    for v in c:
        assert any((v == -u).all() for u in c)
    assert sorted(set((c ** 2).sum(1))) == [0, 1, 2]


@pytest.mark.parametrize('seed', range(4))
def test_equilibrium_moments(seed):
    rng = np.random.default_rng(seed)
    rho = 1 + 0.1 * rng.random()
    u = 0.1 * (2 * rng.random(3) - 1)
    c, _ = O.lattice()
    feq = O.equilibrium(rho, u)
    cs2 = 1.0 / 3.0
    assert abs(feq.sum() - rho) < 1e-14
    assert np.allclose(feq @ c, rho * u, atol=1e-15)
    P = np.einsum('i,ia,ib->ab', feq, c, c)
    assert np.allclose(P, rho * cs2 * np.eye(3) + rho * np.outer(u, u), atol=1e-14)


@pytest.mark.parametrize('tau', [0.6, 0.8, 1.0, 1.7])
def test_guo_moments(tau):
    rng = np.random.default_rng(int(tau * 10))
    u = 0.05 * (2 * rng.random(3) - 1)
    g = 1e-3 * (2 * rng.random(3) - 1)
    c, _ = O.lattice()
    F = O.guo(tau, u, g)
    pre = 1 - 1 / (2 * tau)
    assert abs(F.sum()) < 1e-17
    assert np.allclose(F @ c, pre * g, atol=1e-17)
    P = np.einsum('i,ia,ib->ab', F, c, c)
    assert np.allclose(P, pre * (np.outer(u, g) + np.outer(g, u)), atol=1e-17)


# ----------------------------------------------------------------------------
# delta kernel (Eq. deltaPhiSimple)
# ----------------------------------------------------------------------------
def test_phi_partition_of_unity_and_support():
    rng = np.random.default_rng(5)
    for X in 50 * rng.random(200) - 25:
        nodes = np.floor(X) - 1 + np.arange(4)
        assert abs(sum(O.phi(n - X) for n in nodes) - 1.0) < 1e-15
        # nodes outside the 4-point stencil carry no weight
        assert O.phi(np.floor(X) - 2 - X) == 0.0 or abs(np.floor(X) - 2 - X) == 2.0
        assert O.phi(np.floor(X) + 3 - X) == 0.0
    for r in np.linspace(-2, 2, 41):
        assert O.phi(r) == pytest.approx(O.phi(-r), abs=1e-16)
        assert O.phi(r) >= 0.0
    assert O.phi(2.0 + 1e-12) == 0.0


def _oracle(shape, geometry=0, tau=0.8, **kw):
    lat = dict(nx=shape[0], ny=shape[1], nz=shape[2], tau=tau, geometry=geometry, **kw)
    o = O.Oracle(lat)
    return o


@pytest.mark.parametrize('geometry', [0, 1, 2])
def test_spread_total_and_interp_adjoint(geometry):
    """sum_x g(x) = sum_k F_k (markers away from walls) and
    sum_x u(x).g(x) = sum_k U_k.F_k for any field u (same stencil, Eqs.
    ibmVelocityInterpret / ibmForceSpread are adjoint)."""
    shape = (12, 11, 13)
    kw = dict(tube_radius=5.0) if geometry == 2 else {}
    o = _oracle(shape, geometry, **kw)
    M = 30
    rng = np.random.default_rng(geometry)
    if geometry == 2:
        # inside the tube, at least 2 lu from the wall
        r = 2.9 * np.sqrt(rng.random(M))
        th = 2 * np.pi * rng.random(M)
        X = np.stack([12 * rng.random(M), 5 + r * np.cos(th), 6 + r * np.sin(th)])
    else:
        X = I.tracer_markers(shape, M, 4, margin=2.5)
    o.set_bodies([], X)
    F = 1e-3 * (2 * rng.random((3, M)) - 1)
    o.set_marker_forces(F)
    o.stage_spread()
    g = o.force_density()
    assert np.allclose(g.sum(1), F.sum(1), rtol=1e-13, atol=1e-18)
    rho0, u0 = I.random_fields(shape, 7)
    o.set_equilibrium(rho0, u0)   # the moments read by interpolation are rho0, u0
    o.stage_interpolate()
    Xn, U, _ = o.markers()
    fluid = np.abs(g).sum(0) > 0
    lhs = np.einsum('an,an->', u0[:, fluid], g[:, fluid])
    rhs = np.einsum('ak,ak->', U, F)
    assert lhs == pytest.approx(rhs, rel=1e-12)
    assert np.allclose(Xn, X + U, atol=1e-15)


def test_interpolate_constant_field_and_wall_truncation():
    shape = (10, 10, 10)
    o = _oracle(shape, 0)
    X = I.tracer_markers(shape, 20, 1)
    o.set_bodies([], X)
    N = 1000
    u = np.tile(np.array([0.01, -0.02, 0.005])[:, None], (1, N))
    o.set_equilibrium(None, u)
    o.stage_interpolate()
    _, U, _ = o.markers()
    assert np.allclose(U, u[:, :20], atol=1e-16)
    # next to a wall the stencil nodes inside the wall are dropped: a marker
    # at y = 0.25 loses the node y = -1 (weight phi(1.25))
    o = _oracle(shape, 1)
    Xw = np.array([[5.0], [0.25], [5.0]])
    o.set_bodies([], Xw)
    o.set_equilibrium(None, u)
    o.stage_interpolate()
    _, U, _ = o.markers()
    kept = 1.0 - O.phi(1.25)
    assert np.allclose(U[:, 0], u[:, 0] * kept, atol=1e-16)


# ----------------------------------------------------------------------------
# collision + streaming
# ----------------------------------------------------------------------------
@pytest.mark.parametrize('geometry', [0, 1, 2])
def test_mass_conservation(geometry):
    shape = (7, 9, 8)
    kw = dict(tube_radius=3.6) if geometry == 2 else {}
    if geometry == 1:
        kw['wall_u'] = [-0.01, 0.03]
    o = _oracle(shape, geometry, tau=0.73, **kw)
    o.set_bodies([], np.zeros((3, 0)))
    f = I.random_populations(shape, 3)
    o.set_equilibrium()            # zero solid cells
    solid = o.populations()[0] == 0
    f[:, solid] = 0.0
    o.set_populations(f)
    m0 = f.sum()
    o.step(25)
    assert abs(o.populations().sum() - m0) < 1e-12 * m0


def test_uniform_force_momentum_growth():
    """Periodic box, uniform force density g0: the collision-time momentum
    sum_x rho u grows by exactly N g0 per step (Guo forcing, Eq. rho_u)."""
    shape = (5, 6, 7)
    g0 = np.array([1e-5, -2e-5, 3e-6])
    o = _oracle(shape, 0, tau=0.9, body_force=list(g0))
    o.set_bodies([], np.zeros((3, 0)))
    rho0, u0 = I.random_fields(shape, 2)
    o.set_equilibrium(rho0, u0)
    N = np.prod(shape)
    o.step(1)
    p1 = o.conserved()
    o.step(4)
    p5 = o.conserved()
    assert np.allclose(p5[1:] - p1[1:], 4 * N * g0, rtol=1e-10, atol=1e-16)
    assert p5[0] == pytest.approx(p1[0], rel=1e-14)


def test_streaming_brute_force_tau1():
    """With tau = 1 and no force, f_i(x + c_i, t+1) = f_i^eq(rho(x), u(x)):
    checked against np.roll streaming of the equilibrium of each cell."""
    shape = (4, 5, 3)
    o = _oracle(shape, 0, tau=1.0)
    o.set_bodies([], np.zeros((3, 0)))
    f = I.random_populations(shape, 8, amp=0.05)
    o.set_populations(f)
    o.step(1)
    c, _ = O.lattice()
    rho = f.sum(0)
    u = (c.T.astype(float) @ f) / rho
    N = f.shape[1]
    feq = np.stack([O.equilibrium(rho[n], u[:, n]) for n in range(N)], axis=1)
    nx, ny, nz = shape
    expect = np.empty_like(feq)
    for i in range(19):
        a = feq[i].reshape(nz, ny, nx)
        a = np.roll(a, shift=(c[i, 2], c[i, 1], c[i, 0]), axis=(0, 1, 2))
        expect[i] = a.ravel()
    assert np.allclose(o.populations(), expect, atol=1e-15)


def test_couette_exact():
    """Half-way bounce-back with moving walls reproduces the linear Couette
    profile u_x = U_w (2 (y + 1/2)/H - 1) with H = ny (walls at y=-1/2, ny-1/2)."""
    ny, Uw = 10, 0.02
    o = _oracle((3, ny, 3), 1, tau=0.8, wall_u=[-Uw, Uw])
    o.set_bodies([], np.zeros((3, 0)))
    o.step(4000)
    _, u = o.fields()
    ux = u[0].reshape(3, ny, 3)[1, :, 1]
    y = np.arange(ny)
    assert np.abs(ux - Uw * (2 * (y + 0.5) / ny - 1)).max() < 1e-12
    assert np.abs(u[1:]).max() < 1e-15


def test_poiseuille_exact_at_magic_tau():
    """Body-force-driven channel: u_x = g (y+1/2)(H-y-1/2)/(2 nu) is exact for
    BGK with half-way bounce-back when (tau - 1/2)^2 = 3/16."""
    ny = 8
    tau = 0.5 + math.sqrt(3 / 16)
    nu = (tau - 0.5) / 3
    g0 = 1e-6
    o = _oracle((3, ny, 3), 1, tau=tau, body_force=[g0, 0, 0])
    o.set_bodies([], np.zeros((3, 0)))
    o.step(6000)
    _, u = o.fields()
    ux = u[0].reshape(3, ny, 3)[1, :, 1]
    y = np.arange(ny)
    ex = g0 * (y + 0.5) * (ny - y - 0.5) / (2 * nu)
    assert np.abs(ux - ex).max() < 1e-9 * ex.max()


def test_tube_flow_symmetric_and_below_hagen_poiseuille():
    """Tube along x (staircase bounce-back): the steady profile is symmetric
    under y <-> z and stays close to the Hagen-Poiseuille maximum g R^2/(4 nu)."""
    n, R = 12, 5.0
    tau = 1.0
    nu = (tau - 0.5) / 3
    g0 = 1e-6
    o = _oracle((4, n, n), 2, tau=tau, tube_radius=R, body_force=[g0, 0, 0])
    o.set_bodies([], np.zeros((3, 0)))
    o.step(3000)
    _, u = o.fields()
    ux = u[0].reshape(n, n, 4)[:, :, 0]  # [z][y]
    assert np.abs(ux - ux.T).max() < 1e-13
    umax = g0 * R * R / (4 * nu)
    assert 0.7 * umax < ux.max() < 1.3 * umax


# ----------------------------------------------------------------------------
# membrane model (Sec. 2.2)
# ----------------------------------------------------------------------------
def _octahedron():
    V = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]], float)
    T = []
    for sx in (0, 1):
        for sy in (2, 3):
            for sz in (4, 5):
                tri = [sx, sy, sz]
                a, b, c = V[tri]
                if np.dot(np.cross(b - a, c - a), a + b + c) < 0:
                    tri = [sx, sz, sy]
                T.append(tri)
    return V.T.copy(), np.array(T, dtype=np.int32)


def test_mesh_rest_state_octahedron():
    """Regular octahedron |x|+|y|+|z| = 1: area 4 sqrt(3), volume 4/3, and
    the angle between adjacent outward face normals arccos(1/3) > 0 (convex)."""
    X, T = _octahedron()
    o = _oracle((8, 8, 8), 0)
    o.set_mesh(T, X)
    r = o.mesh_rest()
    assert r['A0'] == pytest.approx(4 * math.sqrt(3), rel=1e-14)
    assert r['V0'] == pytest.approx(4 / 3, rel=1e-14)
    assert r['l0_mean'] == pytest.approx(math.sqrt(2), rel=1e-14)
    # a rotated, translated copy has the same angles, lengths, area, volume
    body = I._body(I.BODY_MEMBRANE, 0, 6, k_b=1.0, k_l=1.0, k_g=1.0, k_v=1.0)
    o.set_bodies([body], X)
    Rm = I.quat_to_matrix(I.random_quaternion(np.random.default_rng(1)))
    assert o.membrane_energy(0, Rm @ X + 3.0) == pytest.approx(0.0, abs=1e-14)


def test_octahedron_dihedral_value():
    """Bending energy with k_b = 1 of the regular octahedron measured
    against the rest angles of a flattened one (vertices +-z moved to
    +-eps z): all 12 edges change angle from arccos(1/3) (regular) to the
    flattened value; check the regular angle itself through a mesh whose
    rest shape is the regular octahedron and a deformed copy with known
    angles: scaling z by s changes the angle at an equatorial edge... use the
    exact identity instead: for the regular octahedron each dihedral has
    cos(theta) = 1/3, so U_bend relative to theta0 = 0 (a rest shape with all
    angles zero does not exist) equals 12 (1 - 1/3); obtain theta0 = 0 by
    comparing two octahedra whose normals are equal: none. Hence test the
    angle through the energy difference of a rigidly rotated copy (zero) and
    through the sign: inflating one vertex outward increases convexity."""
    X, T = _octahedron()
    o = _oracle((8, 8, 8), 0)
    o.set_mesh(T, X)
    body = I._body(I.BODY_MEMBRANE, 0, 6, k_b=1.0)
    o.set_bodies([body], X)
    # pull vertex +z outward along z: the four edges at that vertex fold
    # more sharply (their dihedral grows), the equatorial edges flatten.
    Xp = X.copy()
    Xp[2, 4] = 1.5
    e = o.membrane_energy(0, Xp)
    # closed form: edges at the apex: cos(theta) between faces (1,0,1.5)...
    def normal(a, b, c):
        n = np.cross(b - a, c - a)
        return n / np.linalg.norm(n)
    P = Xp.T
    th0 = math.acos(1 / 3)
    total = 0.0
    for tri1, tri2 in _octa_edge_pairs(T):
        n1 = normal(*P[list(tri1)])
        n2 = normal(*P[list(tri2)])
        th = math.acos(np.clip(np.dot(n1, n2), -1, 1))  # all angles here lie in (0, pi)
        total += 1 - math.cos(th - th0)
    assert e == pytest.approx(total, rel=1e-12)


def _octa_edge_pairs(T):
    pairs = {}
    for t in T:
        for s in range(3):
            key = tuple(sorted((t[s], t[(s + 1) % 3])))
            pairs.setdefault(key, []).append(tuple(t))
    assert len(pairs) == 12 and all(len(v) == 2 for v in pairs.values())
    return [tuple(v) for v in pairs.values()]


def _fd_check(S, T, X, moduli, h=1e-6):
    o = _oracle((8, 8, 8), 0)
    o.set_mesh(T, S)
    body = I._body(I.BODY_MEMBRANE, 0, S.shape[1], **moduli)
    o.set_bodies([body], X)
    F = o.membrane_forces(0, X)
    Ffd = np.zeros_like(X)
    for a in range(3):
        for v in range(X.shape[1]):
            Xp = X.copy(); Xp[a, v] += h
            Xm = X.copy(); Xm[a, v] -= h
            Ffd[a, v] = -(o.membrane_energy(0, Xp) - o.membrane_energy(0, Xm)) / (2 * h)
    return o, F, Ffd


@pytest.mark.parametrize('term', ['stretch', 'bend', 'local', 'global', 'volume', 'all'])
def test_membrane_forces_are_minus_energy_gradient(term):
    """F = -grad U by central differences for each term of Eq.
    membrane-potential separately and together, on a randomly deformed
    42-vertex geodesic ellipsoid."""
    S, T = I.geodesic_sphere(2)
    S = (S * np.array([3.0, 2.5, 2.0])).T.copy()
    rng = np.random.default_rng(0)
    X = S + 0.15 * rng.standard_normal(S.shape) + 4.0
    full = dict(kBT_p=0.3, k_b=0.7, k_l=0.5, k_g=0.9, k_v=0.4)
    key = dict(stretch='kBT_p', bend='k_b', local='k_l', volume='k_v')
    if term == 'all':
        mod = full
    elif term == 'global':
        mod = dict(k_g=0.9)
    else:
        mod = {key[term]: full[key[term]]}
    o, F, Ffd = _fd_check(S, T, X, mod)
    assert np.abs(F).max() > 1e-4
    assert np.abs(F - Ffd).max() < 2e-7 * np.abs(F).max()
    # internal forces: no net force, no net torque
    assert np.abs(F.sum(1)).max() < 1e-13 * np.abs(F).max() * X.shape[1]
    tq = np.cross(X.T, F.T).sum(0)
    assert np.abs(tq).max() < 1e-12 * np.abs(F).max() * X.shape[1] * 10


def test_membrane_rest_shape_is_force_free_and_invariant():
    rest, T = I.rbc_rest_shape(16.0)
    o = _oracle((8, 8, 8), 0)
    o.set_mesh(T, rest)
    body = I._body(I.BODY_MEMBRANE, 0, rest.shape[1], kBT_p=1e-4, k_b=2e-5, k_l=3e-3, k_g=3e-3, k_v=2e-5)
    q = I.random_quaternion(np.random.default_rng(2))
    X = I.quat_to_matrix(q) @ rest + np.array([[40.3], [-7.1], [12.9]])
    o.set_bodies([body], X)
    F = o.membrane_forces(0, X)
    assert np.abs(F).max() < 1e-14
    # the stretching term keeps a nonzero value at rest; a rigid motion of
    # the rest shape leaves the total energy unchanged
    assert o.membrane_energy(0, X) == pytest.approx(o.membrane_energy(0, rest), rel=1e-12)
    # the 642-vertex template: V - E + F = 2 and E = 3F/2
    r = o.mesh_rest()
    assert rest.shape[1] == 642 and T.shape[0] == 1280
    assert r['A0'] > 0 and r['V0'] > 0


def test_shear_modulus_closed_form_and_paper_meshes():
    """Eq. shearModulus with x0 = 1/2 and the zero-force k_p reduces to
    mu0 = 1.25 sqrt(3) (kBT/p) / l0. The paper keeps mu0 = 6 uN/m for three
    meshes with the printed kBT/p (Sec. 3.2); the implied l0 must match the
    edge length of an 8 um cell's surface triangulated with that many nodes."""
    G = golden()
    for l0 in (0.3, 1.0, 2.5):
        assert O.shear_modulus(0.7, l0, 0.5) == pytest.approx(1.25 * math.sqrt(3) * 0.7 / l0, rel=1e-14)
    # a cell surface of area ~135 um^2 (diameter 8 um) with N nodes has ~2N
    # triangles; equilateral edge l = sqrt(4 A_t / sqrt(3))
    area = 135e-12 * (G['rbc_diameter'] / 7.82e-6) ** 2
    for N in (1320, 2562, 10242):
        kbtp = G[f'rbc_kBTp_{N}']
        l0 = 1.25 * math.sqrt(3) * kbtp / G['rbc_mu0']
        assert O.shear_modulus(kbtp, l0, 0.5) == pytest.approx(G['rbc_mu0'], rel=1e-12)
        l_mesh = math.sqrt(4 * area / (2 * N) / math.sqrt(3))
        assert abs(l0 / l_mesh - 1) < 0.1
    # the paper's 1320-node mesh: V - E + F = 2 with E = 3F/2
    assert G['mesh_1320_bonds'] == 1.5 * G['mesh_1320_triangles']
    assert 1320 - G['mesh_1320_bonds'] + G['mesh_1320_triangles'] == 2


def test_jeffery_case_parameters():
    """gamma = 2U/H and Re = aU/nu reproduce the printed 0.00033 and 0.36
    (Sec. 3.1), and nu = (tau - 1/2)/3 gives tau = 1 for nu = 1/6."""
    G = golden()
    gamma = 2 * G['jeffery_U'] / G['jeffery_H']
    assert gamma == pytest.approx(G['jeffery_gamma'], rel=0.02)
    assert G['jeffery_a'] * G['jeffery_U'] / G['jeffery_nu'] == pytest.approx(G['jeffery_Re'], rel=1e-9)
    assert (G['casestudy_tau'] - 0.5) / 3 == pytest.approx(1 / 6)
    # case-study units: nu_phys = nu_lu dx^2/dt ~ 1e-6 m^2/s (water)
    nu_phys = (1 / 6) * G['casestudy_dx'] ** 2 / G['casestudy_dt']
    assert nu_phys == pytest.approx(1.0e-6, rel=0.01)


# ----------------------------------------------------------------------------
# rigid body (Sec. 2.3, penalty reading)
# ----------------------------------------------------------------------------
def test_rigid_tether_rest_and_reaction():
    w = I.shear_ellipsoid(n=16, axes=(4.0, 2.0, 2.0), seed=3)
    o = O.Oracle.from_workload(w)
    o.stage_forces()
    _, _, F = o.markers()
    assert np.abs(F).max() < 1e-14          # markers on their reference points
    b = o.body(0)
    assert np.allclose(b['vel'], 0) and np.allclose(b['omega'], 0)
    # displace all markers by d: F = -kappa d on every marker, the body is
    # pulled by +kappa M d and moves one step with v = kappa M d / mass
    d = np.array([0.01, -0.02, 0.005])
    w2 = dict(w)
    o2 = O.Oracle.from_workload(w2)
    # same references, markers shifted: set the body from the original
    # positions, then shift the markers through one interpolation in a
    # uniform flow u = d (interpolation of a constant field is exact)
    N = o2.N
    o2.set_equilibrium(None, np.tile(d[:, None], (1, N)))
    o2.stage_interpolate()
    X2, _, _ = o2.markers()
    assert np.allclose(X2, w['X'] + d[:, None], atol=1e-14)
    o2.stage_forces()
    _, _, F2 = o2.markers()
    kappa, M = w['bodies'][0]['kappa'], w['X'].shape[1]
    assert np.allclose(F2, -kappa * d[:, None], atol=1e-15)
    b2 = o2.body(0)
    mass = w['bodies'][0]['mass']
    assert np.allclose(b2['vel'], kappa * M * d / mass, rtol=1e-12)
    assert np.allclose(b2['center'], np.array(w['bodies'][0]['center']) + kappa * M * d / mass, rtol=1e-12)
    # a uniform shift exerts no torque about the centre for a centred mesh
    assert np.abs(b2['omega']).max() < 1e-12


def test_sphere_in_couette_rotates_at_half_shear():
    """A neutrally buoyant sphere (r = 1) in Couette flow spins at gamma/2
    about the vorticity axis (the r = 1 limit of Jeffery's orbit, Sec. 3.1)."""
    n, Uw = 24, 0.01
    w = I.shear_ellipsoid(n=n, axes=(3.0, 3.0, 3.0), wall_speed=Uw, seed=4, freq=6, quat=[1, 0, 0, 0])
    o = O.Oracle.from_workload(w)
    o.step(2000)
    b = o.body(0)
    gamma = 2 * Uw / n
    assert b['omega'][2] == pytest.approx(-gamma / 2, rel=0.05)
    assert abs(b['omega'][0]) < 0.05 * gamma and abs(b['omega'][1]) < 0.05 * gamma
