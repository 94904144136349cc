"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only *generates inputs*: lattice sizes and boundary settings,
Lagrangian marker meshes (geodesic spheres mapped to ellipsoids or to the
biconcave red-cell shape), seeded placements and orientations, and body
parameters converted to lattice units. It holds none of the coupled step's
arithmetic (no collision, no delta kernel, no membrane forces, no rest-state
derivation): each side computes those from these arrays on its own.

Workloads (shapes of the paper's cases, Sec. 3):
  * ``shear_ellipsoid``: rigid prolate ellipsoid in a wall-driven shear cell
    (the Jeffery-orbit validation of Sec. 3.1, Eq. jefferyOrbit).
  * ``rbc_tube``: red-cell membranes in a tube driven by a body force (the
    blood-flow cases of Sec. 3.3 / 3.4, membrane model of Sec. 2.2).
  * ``serving_stream``: many independent shear cells arriving over time.

Every array is float64 unless stated; marker positions are SoA ``[3][M]``.
"""
from __future__ import annotations

import math
import numpy as np

# Body kinds understood by both sides.
BODY_MEMBRANE = 0
BODY_RIGID = 1
BODY_FILAMENT = 2
BODY_RIGID_DIRECT = 3

# Geometry codes.
GEOM_PERIODIC = 0
GEOM_YWALLS = 1
GEOM_TUBE = 2


# ----------------------------------------------------------------------------
# meshes
# ----------------------------------------------------------------------------
def _icosahedron():
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([
        [-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
        [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
        [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([
        [0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
        [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
        [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
        [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v, f


def geodesic_sphere(freq: int):
    """Class-I geodesic sphere: each icosahedron face split into freq^2
    triangles, vertices projected to the unit sphere.

    Returns (verts [V,3], tris [T,3] int32) with V = 10 freq^2 + 2,
    T = 20 freq^2, triangles counter-clockwise seen from outside.
    freq = 8 gives the 642-vertex mesh, freq = 9 the 812-vertex mesh.
    """
    iv, faces = _icosahedron()
    key_to_id = {}
    verts = []

    def vid(p):
        q = p / np.linalg.norm(p)
        k = tuple(np.round(q * 1e9).astype(np.int64))
        if k not in key_to_id:
            key_to_id[k] = len(verts)
            verts.append(q)
        return key_to_id[k]

    tris = []
    n = freq
    for (ia, ib, ic) in faces:
        A, B, C = iv[ia], iv[ib], iv[ic]
        grid = {}
        for i in range(n + 1):
            for j in range(n + 1 - i):
                grid[(i, j)] = vid(A + (B - A) * (i / n) + (C - A) * (j / n))
        for i in range(n):
            for j in range(n - i):
                tris.append((grid[(i, j)], grid[(i + 1, j)], grid[(i, j + 1)]))
                if i + j < n - 1:
                    tris.append((grid[(i + 1, j)], grid[(i + 1, j + 1)], grid[(i, j + 1)]))
    V = np.array(verts)
    T = np.array(tris, dtype=np.int64)
    # outward orientation
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    s = np.einsum('ij,ij->i', np.cross(b - a, c - a), a + b + c)
    flip = s < 0
    T[flip] = T[flip][:, [0, 2, 1]]
    # Order vertices along a space-filling (Morton) curve so that
    # consecutive markers are spatially close; this only permutes the input.
    q = np.floor((V + 1.0) * 0.5 * 1023.0).astype(np.int64)
    code = np.zeros(len(V), dtype=np.int64)
    for bit in range(10):
        for ax in range(3):
            code |= ((q[:, ax] >> bit) & 1) << (3 * bit + ax)
    order = np.argsort(code, kind='stable')
    inv = np.empty_like(order)
    inv[order] = np.arange(len(order))
    V = V[order]
    T = inv[T]
    return V, T.astype(np.int32)


def quat_to_matrix(q):
    w, x, y, z = q
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])


def random_quaternion(rng):
    """Uniformly distributed unit quaternion (w, x, y, z)."""
    u1, u2, u3 = rng.random(3)
    q = np.array([
        math.sqrt(u1) * math.cos(2 * math.pi * u3),
        math.sqrt(1 - u1) * math.sin(2 * math.pi * u2),
        math.sqrt(1 - u1) * math.cos(2 * math.pi * u2),
        math.sqrt(u1) * math.sin(2 * math.pi * u3)])
    if q[0] < 0:
        q = -q
    return q


# Evans-Fung biconcave profile (published fit, normalised by the radius R0):
# half-thickness z(rho) = (R0/2) sqrt(1-rho^2) (c0 + c1 rho^2 + c2 rho^4).
EF_C = (0.207161, 2.002558, -1.122762)


def rbc_rest_shape(diameter: float, freq: int = 8):
    """Biconcave red-cell rest shape of the given diameter, in its own frame
    (symmetry axis z, centred at the origin). Returns (X [3,V], tris [T,3])."""
    S, T = geodesic_sphere(freq)
    R0 = 0.5 * diameter
    rho2 = np.clip(S[:, 0] ** 2 + S[:, 1] ** 2, 0.0, 1.0)
    c0, c1, c2 = EF_C
    h = 0.5 * R0 * np.sqrt(1.0 - rho2) * (c0 + c1 * rho2 + c2 * rho2 * rho2)
    X = np.stack([R0 * S[:, 0], R0 * S[:, 1], np.sign(S[:, 2]) * h])
    return X, T


# ----------------------------------------------------------------------------
# unit conversion (paper Table tab:paraPtlCellMix, Sec. 3.2) -> lattice units
# ----------------------------------------------------------------------------
def lattice_units(dx_m: float, tau: float, nu_phys: float = 1.0e-6, rho_phys: float = 1000.0):
    nu_lu = (tau - 0.5) / 3.0
    dt = nu_lu * dx_m * dx_m / nu_phys
    mass = rho_phys * dx_m ** 3
    force = mass * dx_m / (dt * dt)
    return dict(dx=dx_m, dt=dt, force=force, energy=force * dx_m)


def rbc_moduli_lattice(dx_m: float, tau: float):
    """The paper's red-cell moduli (kBT/p, k_b, k_g = k_l, k_v) in lattice units."""
    u = lattice_units(dx_m, tau)
    return dict(kBT_p=1.0e-12 / u['force'],
                k_b=2.3e-19 / u['energy'],
                k_l=2.1e-4 / (u['force'] / dx_m),
                k_g=2.1e-4 / (u['force'] / dx_m),
                k_v=2.2 / (u['force'] / dx_m ** 2))


def filament_moduli_lattice(dx_m: float, tau: float, k_b_J: float = 4.1e-20):
    """The paper's filament parameters (Table tab:paraPtlCellMix: kBT/p =
    1.36e-12 N, bending k_b in [4.1e-20, 4.1e-18] J) in lattice units."""
    u = lattice_units(dx_m, tau)
    return dict(kBT_p=1.36e-12 / u['force'], k_b=k_b_J / u['energy'])


def morse_lattice(dx_m: float, tau: float):
    """The paper's Morse parameters (D0 = 1.2e-18 J, alpha = 0.5 per um,
    r0 = rc = 0.66 um) in lattice units."""
    u = lattice_units(dx_m, tau)
    return dict(D0=1.2e-18 / u['energy'], alpha=0.5e6 * dx_m, r0=0.66e-6 / dx_m, rc=0.66e-6 / dx_m)


# ----------------------------------------------------------------------------
# bodies
# ----------------------------------------------------------------------------
def _body(kind, first, count, **kw):
    b = dict(kind=kind, first=int(first), count=int(count),
             kBT_p=0.0, k_b=0.0, k_l=0.0, k_g=0.0, k_v=0.0, kappa=0.0, mass=0.0,
             inertia=[0.0, 0.0, 0.0], center=[0.0, 0.0, 0.0], quat=[1.0, 0.0, 0.0, 0.0],
             vel=[0.0, 0.0, 0.0], omega=[0.0, 0.0, 0.0], l0=0.0)
    b.update(kw)
    return b


def filament(first, n_beads, start, direction, l0=1.0, kBT_p=0.0, k_b=0.0):
    """A straight bead chain (its rest state: bonds of length l0, angles of
    180 degrees) from `start` along `direction`."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    X = (np.asarray(start, dtype=np.float64)[:, None] + l0 * d[:, None] * np.arange(n_beads)[None, :]).copy()
    return X, _body(BODY_FILAMENT, first, n_beads, kBT_p=kBT_p, k_b=k_b, l0=l0)


def rigid_ellipsoid(center, axes, quat, first, freq=9, kappa=0.02, direct=False):
    """Markers on a rigid ellipsoid surface and its body record (neutrally
    buoyant, unit fluid density). direct=True selects the direct FSI forcing
    (Eq. FSIRigid) with each marker standing for an equal share of the
    surface times one lattice spacing (kappa is then ignored)."""
    S, _ = geodesic_sphere(freq)
    a, b, c = axes
    local = S * np.array([a, b, c])
    R = quat_to_matrix(quat)
    X = (local @ R.T + np.asarray(center)).T.copy()
    mass = 4.0 / 3.0 * math.pi * a * b * c
    inertia = [mass * (b * b + c * c) / 5, mass * (a * a + c * c) / 5, mass * (a * a + b * b) / 5]
    if direct:
        kappa = ellipsoid_area(a, b, c) / X.shape[1]
    body = _body(BODY_RIGID_DIRECT if direct else BODY_RIGID, first, X.shape[1], kappa=kappa, mass=mass,
                 inertia=inertia, center=list(map(float, center)), quat=list(map(float, quat)))
    return X, body


def shear_ellipsoid(n=32, ny=None, nz=None, tau=0.8, wall_speed=0.02, axes=(6.0, 3.0, 3.0),
                    seed=1705, kappa=0.02, freq=9, steps=500, quat=None, couette_init=False, direct=False):
    """Rigid prolate ellipsoid centred in a Couette cell: periodic x and z,
    y-walls moving at -/+ wall_speed. With couette_init the fluid starts
    from the linear wall-driven profile u_x = U (2 (y + 1/2)/H - 1) instead
    of rest (no start-up transient)."""
    ny = ny or n
    nz = nz or n
    rng = np.random.default_rng(seed)
    q = random_quaternion(rng) if quat is None else np.asarray(quat, dtype=np.float64)
    center = np.array([(n - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0])
    X, body = rigid_ellipsoid(center, axes, q, 0, freq=freq, kappa=kappa, direct=direct)
    lattice = dict(nx=n, ny=ny, nz=nz, tau=tau, geometry=GEOM_YWALLS,
                   wall_u=[-wall_speed, wall_speed], tube_radius=0.0, body_force=[0.0, 0.0, 0.0])
    w = dict(name=f'shear_ellipsoid_{n}x{ny}x{nz}', lattice=lattice, mesh=None,
             bodies=[body], X=X, steps=steps, seed=seed)
    if couette_init:
        y = np.arange(ny, dtype=np.float64)
        prof = wall_speed * (2.0 * (y + 0.5) / ny - 1.0)
        u0 = np.zeros((3, nz, ny, n))
        u0[0] = prof[None, :, None]
        w['u0'] = u0.reshape(3, -1)
    return w


def rbc_tube(n=256, radius=120.0, n_cells=3000, diameter=16.0, tau=1.0, reynolds=1.0,
             seed=1706, dx_m=0.5e-6, jitter=0.2, freq=8, steps=2000):
    """Red-cell membranes in a tube along x (bounce-back wall, periodic in x),
    driven by a uniform body force chosen for the requested centreline
    Reynolds number Re = u_c (2R) / nu, u_c = g R^2 / (4 nu)."""
    rng = np.random.default_rng(seed)
    rest, tris = rbc_rest_shape(diameter, freq)
    nu = (tau - 0.5) / 3.0
    u_c = reynolds * nu / (2.0 * radius)
    g0 = 4.0 * nu * u_c / (radius * radius)
    mod = rbc_moduli_lattice(dx_m, tau)
    centers, quats = place_cells_in_tube(rng, n, radius, n_cells, diameter)
    V = rest.shape[1]
    X = np.empty((3, V * len(centers)))
    bodies = []
    for k, (c, q) in enumerate(zip(centers, quats)):
        R = quat_to_matrix(q)
        X[:, k * V:(k + 1) * V] = (R @ rest) + c[:, None]
        s = 1.0 + jitter * (2.0 * rng.random(5) - 1.0)
        bodies.append(_body(BODY_MEMBRANE, k * V, V, kBT_p=mod['kBT_p'] * s[0], k_b=mod['k_b'] * s[1],
                            k_l=mod['k_l'] * s[2], k_g=mod['k_g'] * s[3], k_v=mod['k_v'] * s[4],
                            center=list(map(float, c)), quat=list(map(float, q))))
    lattice = dict(nx=n, ny=n, nz=n, tau=tau, geometry=GEOM_TUBE, wall_u=[0.0, 0.0],
                   tube_radius=float(radius), body_force=[g0, 0.0, 0.0])
    return dict(name=f'rbc_tube_{n}^3_R{radius:g}_{len(centers)}cells', lattice=lattice,
                mesh=dict(rest_X=rest, tris=tris), bodies=bodies, X=X, steps=steps, seed=seed)


def place_cells_in_tube(rng, n, radius, n_cells, diameter, max_tilt_deg=40.0, tries=5):
    """Seeded non-overlapping placement of red cells in a tube along x.

    Candidate slots form stacks: columns on a hexagonal grid of the tube
    cross-section (spacing D + 2) and, along each column, slots every
    ~2.3 half-thicknesses. A seeded random subset of the slots is filled
    with cells whose symmetry axis lies along x (these cannot overlap).
    Then, in a seeded random order, each cell is given a random spin about
    its axis, a random tilt of the axis away from x (up to
    ``max_tilt_deg``) and a small positional jitter; the move is kept only if
    the cell's bounding oblate spheroid (inflated by 0.5 lu) overlaps
    neither another cell nor the wall on a voxel occupancy grid, else the
    tilt is halved a few times and finally the untilted pose is kept."""
    a = 0.5 * diameter + 0.5
    cz = 0.33 * 0.5 * diameter + 0.5
    yc = zc = (n - 1) / 2.0
    iy, iz = np.meshgrid(np.arange(n), np.arange(n), indexing='ij')
    wall = (iy - yc) ** 2 + (iz - zc) ** 2 > (radius - 0.5) ** 2
    occ = np.broadcast_to(wall[None], (n, n, n)).copy()  # [x][y][z]
    sp = diameter + 2.0
    r_max = radius - a - 0.5
    cols = []
    m = int(r_max // sp) + 2
    for i in range(-m, m + 1):
        for j in range(-m, m + 1):
            y = sp * (i + 0.5 * j)
            z = sp * (j * math.sqrt(3.0) / 2.0)
            if y * y + z * z <= r_max * r_max + 1e-9:
                cols.append((y, z))
    per_col = max(1, int(n // (2.0 * cz + 0.25)))
    dxs = n / per_col
    slots = [(k * dxs, y, z) for (y, z) in cols for k in range(per_col)]
    if len(slots) < n_cells:
        raise RuntimeError(f'only {len(slots)} slots for {n_cells} cells')
    pick = sorted(rng.permutation(len(slots))[:n_cells])
    ext = int(math.ceil(a)) + 1
    off = np.arange(-ext, ext + 1)
    ox, oy, oz = np.meshgrid(off, off, off, indexing='ij')
    pts = np.stack([ox.ravel(), oy.ravel(), oz.ravel()], axis=1).astype(np.float64)
    q_align = np.array([math.cos(math.pi / 4), 0.0, math.sin(math.pi / 4), 0.0])  # body z -> world x

    def footprint(c, q):
        R = quat_to_matrix(q)
        p = pts + np.floor(c)
        d = (p - c) @ R
        inside = (d[:, 0] ** 2 + d[:, 1] ** 2) / (a * a) + d[:, 2] ** 2 / (cz * cz) <= 1.0
        idx = p[inside].astype(np.int64)
        if idx[:, 1].min() < 0 or idx[:, 2].min() < 0 or idx[:, 1].max() >= n or idx[:, 2].max() >= n:
            return None
        return idx[:, 0] % n, idx[:, 1], idx[:, 2]

    centers, quats, feet = [], [], []
    for s_id in pick:
        x0, y0, z0 = slots[s_id]
        spin = 2 * math.pi * rng.random()
        q = _qmul(q_align, np.array([math.cos(spin / 2), 0.0, 0.0, math.sin(spin / 2)]))
        c = np.array([x0, yc + y0, zc + z0])
        fp = footprint(c, q)
        if fp is None or occ[fp].any():
            raise RuntimeError('stack slot overlaps')
        occ[fp] = True
        centers.append(c)
        quats.append(q)
        feet.append(fp)
    for k in rng.permutation(len(centers)):
        occ[feet[k]] = False
        tilt = math.radians(max_tilt_deg) * math.sqrt(rng.random())
        azim = 2 * math.pi * rng.random()
        jit = (rng.random(3) - 0.5) * np.array([0.5, 1.0, 1.0])
        for t in range(tries):
            tl = tilt * (0.5 ** t)
            ax = np.array([0.0, math.cos(azim), math.sin(azim)])
            q_tilt = np.concatenate([[math.cos(tl / 2)], math.sin(tl / 2) * np.cross([1.0, 0.0, 0.0], ax)])
            q = _qmul(q_tilt, quats[k])
            q /= np.linalg.norm(q)
            c = centers[k] + jit
            fp = footprint(c, q)
            if fp is not None and not occ[fp].any():
                centers[k], quats[k], feet[k] = c, q, fp
                break
        occ[feet[k]] = True
    quats = [q if q[0] >= 0 else -q for q in quats]
    return centers, quats


def place_cells_in_channel(rng, shape, x_range, n_cells, diameter, max_tilt_deg=40.0, tries=5):
    """Seeded non-overlapping placement of red cells in a channel (walls at
    y = -1/2 and ny - 1/2, periodic x and z) within x_range, the same scheme
    as place_cells_in_tube: stacks of slots on a hexagonal grid of the
    cross-section (spacing D + 2) filled at random with cells whose axis lies
    along x, then a random spin, tilt (up to max_tilt_deg) and jitter kept
    only where the cell's inflated bounding spheroid stays clear."""
    nx, ny, nz = shape
    a = 0.5 * diameter + 0.5
    cz = 0.33 * 0.5 * diameter + 0.5
    occ = np.zeros((nx, ny, nz), dtype=bool)
    sp = diameter + 2.0
    cols = []
    for j in range(int(nz / (sp * math.sqrt(3.0) / 2.0)) + 1):
        z = a + 0.5 + sp * j * math.sqrt(3.0) / 2.0
        for i in range(int(ny / sp) + 1):
            y = a + 0.5 + sp * (i + 0.5 * (j % 2))
            if y <= ny - 1.5 - a and z <= nz - 1.5 - a:
                cols.append((y, z))
    x0, x1 = x_range
    per_col = max(1, int((x1 - x0) // (2.0 * cz + 0.25)))
    dxs = (x1 - x0) / per_col
    slots = [(x0 + (k + 0.5) * dxs, y, z) for (y, z) in cols for k in range(per_col)]
    if len(slots) < n_cells:
        raise RuntimeError(f'only {len(slots)} slots for {n_cells} cells')
    pick = sorted(rng.permutation(len(slots))[:n_cells])
    ext = int(math.ceil(a)) + 1
    off = np.arange(-ext, ext + 1)
    ox, oy, oz = np.meshgrid(off, off, off, indexing='ij')
    pts = np.stack([ox.ravel(), oy.ravel(), oz.ravel()], axis=1).astype(np.float64)
    q_align = np.array([math.cos(math.pi / 4), 0.0, math.sin(math.pi / 4), 0.0])  # body z -> world x

    def footprint(c, q):
        R = quat_to_matrix(q)
        p = pts + np.floor(c)
        d = (p - c) @ R
        inside = (d[:, 0] ** 2 + d[:, 1] ** 2) / (a * a) + d[:, 2] ** 2 / (cz * cz) <= 1.0
        idx = p[inside].astype(np.int64)
        if idx[:, 1].min() < 0 or idx[:, 1].max() >= ny or idx[:, 0].min() < x0 - 1 or idx[:, 0].max() > x1:
            return None
        return idx[:, 0] % nx, idx[:, 1], idx[:, 2] % nz

    centers, quats, feet = [], [], []
    for s_id in pick:
        xs, y0, z0 = slots[s_id]
        spin = 2 * math.pi * rng.random()
        q = _qmul(q_align, np.array([math.cos(spin / 2), 0.0, 0.0, math.sin(spin / 2)]))
        c = np.array([xs, y0, z0])
        fp = footprint(c, q)
        if fp is None or occ[fp].any():
            raise RuntimeError('stack slot overlaps')
        occ[fp] = True
        centers.append(c)
        quats.append(q)
        feet.append(fp)
    for k in rng.permutation(len(centers)):
        occ[feet[k]] = False
        tilt = math.radians(max_tilt_deg) * math.sqrt(rng.random())
        azim = 2 * math.pi * rng.random()
        jit = (rng.random(3) - 0.5) * np.array([0.5, 1.0, 1.0])
        for t in range(tries):
            tl = tilt * (0.5 ** t)
            ax = np.array([0.0, math.cos(azim), math.sin(azim)])
            q_tilt = np.concatenate([[math.cos(tl / 2)], math.sin(tl / 2) * np.cross([1.0, 0.0, 0.0], ax)])
            q = _qmul(q_tilt, quats[k])
            q /= np.linalg.norm(q)
            c = centers[k] + jit
            fp = footprint(c, q)
            if fp is not None and not occ[fp].any():
                centers[k], quats[k], feet[k] = c, q, fp
                break
        occ[feet[k]] = True
    quats = [q if q[0] >= 0 else -q for q in quats]
    return centers, quats


def mixed_suspension(shape=(512, 512, 512), n_cells=20000, n_filaments=4000, beads=50, diameter=16.0,
                     tau=1.0, wall_shear_rate=1000.0, seed=1709, dx_m=0.5e-6, jitter=0.2, freq=8,
                     filament_spacing=3.0, steps=1000, morse=True):
    """Red cells and flexible filaments in a channel (walls at rest at
    y = -1/2 and ny - 1/2, periodic x and z), driven by a uniform body force
    whose plane-Poiseuille wall shear rate is `wall_shear_rate` (1/s).
    Filaments (bond length 1 lu, the lattice spacing) lie straight along x
    in a slab at the channel inlet, on a jittered grid of the
    cross-section, half with bending stiffness 10 kBT and half 1000 kBT
    (4.1e-20 and 4.1e-18 J); cells fill the rest of the channel. Markers:
    cells first, then filaments; Morse excluded volume between bodies."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    u = lattice_units(dx_m, tau)
    nu = (tau - 0.5) / 3.0
    g0 = 2.0 * nu * (wall_shear_rate * u['dt']) / ny
    rest, tris = rbc_rest_shape(diameter, freq)
    mod = rbc_moduli_lattice(dx_m, tau)
    slab = beads + 2.0
    centers, quats = place_cells_in_channel(rng, shape, (slab + 1.0, nx - 1.0), n_cells, diameter)
    V = rest.shape[1]
    M = V * len(centers) + beads * n_filaments
    X = np.empty((3, M))
    bodies = []
    for k, (c, q) in enumerate(zip(centers, quats)):
        R = quat_to_matrix(q)
        X[:, k * V:(k + 1) * V] = (R @ rest) + c[:, None]
        s = 1.0 + jitter * (2.0 * rng.random(5) - 1.0)
        bodies.append(_body(BODY_MEMBRANE, k * V, V, kBT_p=mod['kBT_p'] * s[0], k_b=mod['k_b'] * s[1],
                            k_l=mod['k_l'] * s[2], k_g=mod['k_g'] * s[3], k_v=mod['k_v'] * s[4],
                            center=list(map(float, c)), quat=list(map(float, q))))
    # filament grid on the cross-section, away from the walls
    gy = np.arange(1.5, ny - 1.5, filament_spacing)
    gz = np.arange(0.5, nz - 0.5, filament_spacing)
    grid = np.array([(y, z) for z in gz for y in gy])
    if len(grid) < n_filaments:
        raise RuntimeError(f'only {len(grid)} filament sites for {n_filaments} filaments')
    sites = grid[np.sort(rng.permutation(len(grid))[:n_filaments])]
    soft = filament_moduli_lattice(dx_m, tau, 4.1e-20)
    stiff = filament_moduli_lattice(dx_m, tau, 4.1e-18)
    first = V * len(centers)
    for f, (y, z) in enumerate(sites):
        mod_f = soft if f % 2 == 0 else stiff
        start = [1.0 + 0.5 * rng.random(), y + 0.4 * (rng.random() - 0.5), z + 0.4 * (rng.random() - 0.5)]
        Xf, bf = filament(first, beads, start, [1.0, 0.0, 0.0], l0=1.0, kBT_p=mod_f['kBT_p'], k_b=mod_f['k_b'])
        X[:, first:first + beads] = Xf
        bodies.append(bf)
        first += beads
    lattice = dict(nx=nx, ny=ny, nz=nz, tau=tau, geometry=GEOM_YWALLS, wall_u=[0.0, 0.0],
                   tube_radius=0.0, body_force=[g0, 0.0, 0.0])
    w = dict(name=f'mixed_channel_{nx}x{ny}x{nz}_{len(centers)}cells_{n_filaments}x{beads}filaments',
             lattice=lattice, mesh=dict(rest_X=rest, tris=tris), bodies=bodies, X=X, steps=steps, seed=seed)
    if morse:
        w['morse'] = morse_lattice(dx_m, tau)
    return w


def _qmul(p, q):
    w1, x1, y1, z1 = p
    w2, x2, y2, z2 = q
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2,
                     w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2,
                     w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


# ----------------------------------------------------------------------------
# lattice states
# ----------------------------------------------------------------------------
def random_fields(shape, seed, u_amp=0.02, rho_amp=0.01):
    """Smooth-ish random density/velocity fields [N], [3][N] (x fastest)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    N = nx * ny * nz
    rho = 1.0 + rho_amp * (2 * rng.random(N) - 1)
    u = u_amp * (2 * rng.random((3, N)) - 1)
    return rho, u


def random_populations(shape, seed, amp=0.005):
    """A random (non-equilibrium) population state [19][N] around the D3Q19
    rest weights w_0 = 1/3, w_axis = 1/18, w_diag = 1/36 (ordering as in the
    public header: 0 rest, 1..6 axis, 7..18 face diagonals)."""
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    w = np.array([1 / 3] + [1 / 18] * 6 + [1 / 36] * 12)
    return w[:, None] * (1.0 + amp * (2 * rng.random((19, nx * ny * nz)) - 1))


def tracer_markers(shape, M, seed, margin=0.0):
    """Random marker positions inside the box [margin, n-1-margin]."""
    rng = np.random.default_rng(seed)
    lo = np.full(3, margin)
    hi = np.array(shape, dtype=np.float64) - 1.0 - margin
    return (lo[:, None] + (hi - lo)[:, None] * rng.random((3, M)))


# ----------------------------------------------------------------------------
# serving stream
# ----------------------------------------------------------------------------
def jeffery_period(gamma, r):
    """Closed-form Jeffery period T = (2 pi / gamma)(r + 1/r) (Sec. 3.1)."""
    return 2.0 * math.pi / gamma * (r + 1.0 / r)


def ellipsoid_area(a, b, c):
    """Surface area of an ellipsoid, Thomsen's approximation (relative error
    below 1.1 %)."""
    p = 1.6075
    return 4.0 * math.pi * (((a * b) ** p + (a * c) ** p + (b * c) ** p) / 3.0) ** (1.0 / p)


def serving_stream(n_cases=512, seed=1708, periods=2.0, L_min=24, L_max=96, rate=None,
                   period_scale=1.0, tau=0.8, kappa=0.02, freq=9):
    """Independent rigid-ellipsoid shear cells arriving by a seeded Poisson
    process. L ~ U{L_min..L_max}, aspect r ~ U[1.5, 5], shear rate
    gamma ~ logU[1e-4, 1e-3]; a = 0.1875 L, b = c = max(a / r, 1.5).
    Each runs ceil(periods * period_scale * T) steps; the tether stiffness per
    marker scales with the body's surface area. ``rate`` is the mean
    arrival rate in cases per second (None: all arrive at t = 0)."""
    rng = np.random.default_rng(seed)
    cases = []
    t = 0.0
    for k in range(n_cases):
        L = int(rng.integers(L_min, L_max + 1))
        r = float(rng.uniform(1.5, 5.0))
        gamma = float(math.exp(rng.uniform(math.log(1e-4), math.log(1e-3))))
        a = 0.1875 * L
        b = max(a / r, 1.5)
        wall = 0.5 * gamma * L
        steps = int(math.ceil(periods * period_scale * jeffery_period(gamma, a / b)))
        # the same penalty stiffness per unit surface area as the 6 x 3 x 3
        # body with `kappa` per marker: with a fixed marker count a thin body
        # packs its markers ~0.3 lu apart and a fixed per-marker kappa makes
        # the explicit coupling unstable
        k_m = kappa * ellipsoid_area(a, b, b) / ellipsoid_area(6.0, 3.0, 3.0)
        case = shear_ellipsoid(n=L, tau=tau, wall_speed=wall, axes=(a, b, b),
                               seed=seed * 1000 + k, kappa=k_m, freq=freq, steps=steps)
        if rate is not None:
            t += float(rng.exponential(1.0 / rate))
        case['arrival'] = t
        case['gamma'] = gamma
        case['aspect'] = a / b
        cases.append(case)
    return cases
