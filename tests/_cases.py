"""Small seeded cases shared by the GPU parity tests (sizes the FP64 oracle
finishes in seconds, spanning several 32-wide x tiles plus a ragged tail)."""
import numpy as np

from paper_1704_04551_gb300 import inputs as I

LATTICES = {
    'periodic': dict(nx=40, ny=12, nz=10, tau=0.8, geometry=0, body_force=[2e-6, -1e-6, 5e-7]),
    'ywalls': dict(nx=40, ny=11, nz=9, tau=0.7, geometry=1, wall_u=[-0.015, 0.02], body_force=[1e-6, 0, 0]),
    'tube': dict(nx=37, ny=14, nz=13, tau=1.0, geometry=2, tube_radius=5.6, body_force=[3e-6, 0, 0]),
}


def shape(lat):
    return (lat['nx'], lat['ny'], lat['nz'])


def fluid_mask(lat):
    nx, ny, nz = shape(lat)
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing='ij')
    if lat['geometry'] == 2:
        yc, zc = (ny - 1) / 2, (nz - 1) / 2
        m = (y - yc) ** 2 + (z - zc) ** 2 <= lat['tube_radius'] ** 2
    else:
        m = np.ones_like(x, dtype=bool)
    return m.ravel()


def markers_inside(lat, M, seed):
    """Random marker positions in the fluid (some within 2 lu of walls,
    some across periodic boundaries)."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape(lat)
    if lat['geometry'] == 2:
        r = (lat['tube_radius'] - 0.5) * np.sqrt(rng.random(M))
        th = 2 * np.pi * rng.random(M)
        return np.stack([nx * rng.random(M) - 0.5 * nx * (rng.random(M) < 0.1),
                         (ny - 1) / 2 + r * np.cos(th), (nz - 1) / 2 + r * np.sin(th)])
    X = np.stack([nx * rng.random(M), (ny - 1) * rng.random(M), nz * rng.random(M)])
    X[0, : M // 10] += nx * 2.0  # unwrapped positions beyond the box
    X[2, : M // 10] -= nz
    if lat['geometry'] == 0:
        X[1, : M // 10] -= ny
    return X


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def membrane_case(n=40, R=16.0, cells=3, seed=21, deform=0.08):
    """Three red-cell membranes in a 40^3 tube, vertices displaced by
    `deform` lu (Gaussian), with moduli stiffer than the physical ones so
    that every force term is visible."""
    w = I.rbc_tube(n=n, radius=R, n_cells=cells, seed=seed, steps=0)
    rng = np.random.default_rng(seed + 1)
    w['X'] = w['X'] + deform * rng.standard_normal(w['X'].shape)
    for b in w['bodies']:
        b.update(kBT_p=2e-3, k_b=1e-3, k_l=5e-3, k_g=4e-3, k_v=3e-3)
    return w


# lattices wide enough for full 128-cell blocks, a ragged x block, several
# 64-cell warps per row and many row blocks
WIDE = {
    'periodic': dict(nx=160, ny=40, nz=36, tau=0.8, geometry=0, body_force=[2e-6, -1e-6, 5e-7]),
    'ywalls': dict(nx=160, ny=38, nz=36, tau=0.7, geometry=1, wall_u=[-0.015, 0.02], body_force=[1e-6, 0, 0]),
    'tube': dict(nx=160, ny=40, nz=40, tau=1.0, geometry=2, tube_radius=18.5, body_force=[3e-6, 0, 0]),
}


def wide_tracers(lat, M, seed):
    """Marker positions in the fluid of a WIDE lattice, with forces."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape(lat)
    if lat['geometry'] == 2:
        r = (lat['tube_radius'] - 1.0) * np.sqrt(rng.random(M))
        th = 2 * np.pi * rng.random(M)
        X = np.stack([nx * rng.random(M), (ny - 1) / 2 + r * np.cos(th), (nz - 1) / 2 + r * np.sin(th)])
    else:
        X = np.stack([nx * rng.random(M), (ny - 1) * rng.random(M), nz * rng.random(M)])
    F = 2e-3 * (2 * rng.random((3, M)) - 1)
    return X, F



def cluster_tracers(lat, n_clusters, seed, per=256, half=2.5):
    """Tracers in runs of `per` (one transfer group each) packed into cubes
    of side 2 * half around random centres in the fluid, so that every
    group's stencils fit a shared-memory box; the last run is ragged. Some
    clusters sit across periodic boundaries and within 2 lu of walls."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape(lat)
    n = n_clusters
    if lat['geometry'] == 2:
        r = (lat["tube_radius"] - 1.5 * half - 0.5) * np.sqrt(rng.random(n))
        th = 2 * np.pi * rng.random(n)
        C = np.stack([nx * rng.random(n), (ny - 1) / 2 + r * np.cos(th), (nz - 1) / 2 + r * np.sin(th)])
    else:
        C = np.stack([nx * rng.random(n), half + (ny - 1 - 2 * half) * rng.random(n), nz * rng.random(n)])
        if lat['geometry'] == 0:
            C[1] = ny * rng.random(n)
    X = np.repeat(C, per, axis=1) + rng.uniform(-half, half, (3, n * per))
    X = X[:, : n * per - per // 3]
    F = 2e-3 * (2 * rng.random(X.shape) - 1)
    return X, F
