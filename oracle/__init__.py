"""ctypes binding of the FP64 CPU oracle (``ibm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg use it to check and time against; the product
path (the CUDA library and its binding) never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, 'ibm_oracle.c')
_HDR = os.path.join(_HERE, 'ibm_oracle.h')
_LIB = os.path.join(_HERE, 'liboracle.so')


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, -O2, no fast-math), with OpenMP
    over its independent loops (lattice z slabs, markers, bodies) when the
    compiler has it; the results do not depend on the thread count."""
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR), os.path.getmtime(__file__))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f'.{os.getpid()}.tmp'
        base = ['gcc', '-O2', '-std=c11', '-D_DEFAULT_SOURCE', '-fPIC', '-shared', '-o', tmp, _SRC, '-lm']
        try:
            subprocess.check_call(base[:1] + ['-fopenmp'] + base[1:], stderr=subprocess.DEVNULL)
        except subprocess.CalledProcessError:
            subprocess.check_call(base)
        os.replace(tmp, _LIB)
    return _LIB


class _Config(C.Structure):
    _fields_ = [('nx', C.c_int32), ('ny', C.c_int32), ('nz', C.c_int32), ('geometry', C.c_int32),
                ('tau', C.c_double), ('wall_u', C.c_double * 2), ('tube_radius', C.c_double),
                ('body_force', C.c_double * 3)]


class _Body(C.Structure):
    _fields_ = [('kind', C.c_int32), ('pad', C.c_int32), ('first', C.c_int64), ('count', C.c_int64),
                ('kBT_p', C.c_double), ('k_b', C.c_double), ('k_l', C.c_double), ('k_g', C.c_double),
                ('k_v', C.c_double), ('kappa', C.c_double), ('mass', C.c_double),
                ('inertia', C.c_double * 3), ('center', C.c_double * 3), ('quat', C.c_double * 4),
                ('vel', C.c_double * 3), ('omega', C.c_double * 3), ('l0', C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        L.ora_create.restype = P
        L.ora_create.argtypes = [C.POINTER(_Config)]
        L.ora_destroy.argtypes = [P]
        for name in ('ora_set_equilibrium',):
            getattr(L, name).argtypes = [P, P, P]
        L.ora_set_populations.argtypes = [P, P]
        L.ora_get_populations.argtypes = [P, P]
        L.ora_get_fields.argtypes = [P, P, P]
        L.ora_get_force_density.argtypes = [P, P]
        L.ora_conserved.argtypes = [P, P]
        L.ora_set_mesh.argtypes = [P, C.c_int32, C.c_int32, P, P]
        L.ora_set_mesh.restype = C.c_int
        L.ora_set_bodies.argtypes = [P, C.c_int32, P, C.c_int64, P]
        L.ora_set_bodies.restype = C.c_int
        L.ora_get_markers.argtypes = [P, P, P, P]
        L.ora_set_marker_forces.argtypes = [P, P]
        L.ora_get_body.argtypes = [P, C.c_int32, C.POINTER(_Body)]
        for name in ('ora_stage_forces', 'ora_stage_spread', 'ora_stage_collide_stream',
                     'ora_stage_interpolate'):
            getattr(L, name).argtypes = [P]
        L.ora_step.argtypes = [P, C.c_int64]
        L.ora_set_threads.argtypes = [C.c_int]
        L.ora_set_threads.restype = C.c_int
        L.ora_solid_steps.argtypes = [P, C.c_int64, C.c_double, C.c_double, C.c_double, P, P]
        L.ora_phi.restype = C.c_double
        L.ora_phi.argtypes = [C.c_double]
        L.ora_lattice.argtypes = [P, P]
        L.ora_equilibrium.argtypes = [C.c_double, P, P]
        L.ora_guo.argtypes = [C.c_double, P, P, P]
        L.ora_membrane_energy.restype = C.c_double
        L.ora_membrane_energy.argtypes = [P, C.c_int32, P]
        L.ora_membrane_forces.argtypes = [P, C.c_int32, P, P]
        L.ora_mesh_rest.argtypes = [P, P]
        L.ora_shear_modulus.restype = C.c_double
        L.ora_shear_modulus.argtypes = [C.c_double, C.c_double, C.c_double]
        L.ora_filament_energy.restype = C.c_double
        L.ora_filament_energy.argtypes = [P, C.c_int32, P]
        L.ora_filament_forces.argtypes = [P, C.c_int32, P, P]
        L.ora_set_morse.argtypes = [P, C.c_double, C.c_double, C.c_double, C.c_double]
        L.ora_morse_energy.restype = C.c_double
        L.ora_morse_energy.argtypes = [P, P]
        L.ora_morse_forces.argtypes = [P, P, P]
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------- pure helpers
def set_threads(n: int = 0) -> int:
    """Threads the oracle's loops use (n <= 0: leave as is); returns the
    count in effect (1 without OpenMP)."""
    return int(lib().ora_set_threads(int(n)))


def phi(r: float) -> float:
    return lib().ora_phi(float(r))


def lattice():
    c = np.zeros((19, 3), dtype=np.int32)
    w = np.zeros(19)
    lib().ora_lattice(_p(c), _p(w))
    return c, w


def equilibrium(rho, u):
    u = _f64(u)
    out = np.zeros(19)
    lib().ora_equilibrium(float(rho), _p(u), _p(out))
    return out


def guo(tau, u, g):
    u, g = _f64(u), _f64(g)
    out = np.zeros(19)
    lib().ora_guo(float(tau), _p(u), _p(g), _p(out))
    return out


def shear_modulus(kBT_p, l0, x0=0.5):
    return lib().ora_shear_modulus(kBT_p, l0, x0)


def make_body(d) -> _Body:
    b = _Body()
    b.kind, b.first, b.count = int(d['kind']), int(d['first']), int(d['count'])
    for k in ('kBT_p', 'k_b', 'k_l', 'k_g', 'k_v', 'kappa', 'mass'):
        setattr(b, k, float(d[k]))
    b.l0 = float(d.get('l0', 0.0))
    for k, n in (('inertia', 3), ('center', 3), ('quat', 4), ('vel', 3), ('omega', 3)):
        arr = getattr(b, k)
        for i in range(n):
            arr[i] = float(d[k][i])
    return b


def body_dict(b: _Body):
    return dict(kind=b.kind, first=b.first, count=b.count,
                center=list(b.center), quat=list(b.quat), vel=list(b.vel), omega=list(b.omega))


class Oracle:
    """FP64 reference simulation of one lattice with its markers."""

    def __init__(self, lattice: dict):
        cfg = _Config()
        cfg.nx, cfg.ny, cfg.nz = int(lattice['nx']), int(lattice['ny']), int(lattice['nz'])
        cfg.geometry = int(lattice['geometry'])
        cfg.tau = float(lattice['tau'])
        cfg.wall_u[0], cfg.wall_u[1] = map(float, lattice.get('wall_u', (0.0, 0.0)))
        cfg.tube_radius = float(lattice.get('tube_radius', 0.0))
        for i, v in enumerate(lattice.get('body_force', (0.0, 0.0, 0.0))):
            cfg.body_force[i] = float(v)
        self.shape = (cfg.nx, cfg.ny, cfg.nz)
        self.N = cfg.nx * cfg.ny * cfg.nz
        self.M = 0
        self._h = lib().ora_create(C.byref(cfg))

    def __del__(self):
        if getattr(self, '_h', None):
            lib().ora_destroy(self._h)
            self._h = None

    @classmethod
    def from_workload(cls, w: dict):
        o = cls(w['lattice'])
        o.set_equilibrium(w.get('rho0'), w.get('u0'))
        if w.get('mesh') is not None:
            o.set_mesh(w['mesh']['tris'], w['mesh']['rest_X'])
        o.set_bodies(w.get('bodies', []), w['X'])
        if w.get('morse') is not None:
            o.set_morse(**w['morse'])
        return o

    # lattice
    def set_equilibrium(self, rho=None, u=None):
        rho = None if rho is None else _f64(rho)
        u = None if u is None else _f64(u)
        lib().ora_set_equilibrium(self._h, _p(rho), _p(u))

    def set_populations(self, f):
        f = _f64(f)
        assert f.shape == (19, self.N)
        lib().ora_set_populations(self._h, _p(f))

    def populations(self):
        f = np.zeros((19, self.N))
        lib().ora_get_populations(self._h, _p(f))
        return f

    def fields(self):
        rho = np.zeros(self.N)
        u = np.zeros((3, self.N))
        lib().ora_get_fields(self._h, _p(rho), _p(u))
        return rho, u

    def force_density(self):
        g = np.zeros((3, self.N))
        lib().ora_get_force_density(self._h, _p(g))
        return g

    def conserved(self):
        out = np.zeros(4)
        lib().ora_conserved(self._h, _p(out))
        return out

    # markers
    def set_mesh(self, tris, rest_X):
        tris = np.ascontiguousarray(tris, dtype=np.int32)
        rest_X = _f64(rest_X)
        rc = lib().ora_set_mesh(self._h, rest_X.shape[1], tris.shape[0], _p(tris), _p(rest_X))
        if rc != 0:
            raise ValueError('mesh is not a closed, consistently oriented manifold')
        self.nv = rest_X.shape[1]

    def set_bodies(self, bodies, X):
        X = _f64(X)
        self.M = X.shape[1]
        arr = (_Body * max(1, len(bodies)))()
        for i, d in enumerate(bodies):
            arr[i] = make_body(d)
        rc = lib().ora_set_bodies(self._h, len(bodies), arr, self.M, _p(X))
        if rc != 0:
            raise ValueError(f'bad body description ({rc})')

    def markers(self):
        X = np.zeros((3, self.M))
        U = np.zeros((3, self.M))
        F = np.zeros((3, self.M))
        lib().ora_get_markers(self._h, _p(X), _p(U), _p(F))
        return X, U, F

    def set_marker_forces(self, F):
        F = _f64(F)
        assert F.shape == (3, self.M)
        lib().ora_set_marker_forces(self._h, _p(F))

    def body(self, b):
        out = _Body()
        lib().ora_get_body(self._h, b, C.byref(out))
        return body_dict(out)

    def membrane_energy(self, b, Xb):
        return lib().ora_membrane_energy(self._h, b, _p(_f64(Xb)))

    def membrane_forces(self, b, Xb):
        Xb = _f64(Xb)
        F = np.zeros_like(Xb)
        lib().ora_membrane_forces(self._h, b, _p(Xb), _p(F))
        return F

    def filament_energy(self, b, Xb):
        return lib().ora_filament_energy(self._h, b, _p(_f64(Xb)))

    def filament_forces(self, b, Xb):
        Xb = _f64(Xb)
        F = np.zeros_like(Xb)
        lib().ora_filament_forces(self._h, b, _p(Xb), _p(F))
        return F

    def set_morse(self, D0, alpha, r0, rc):
        lib().ora_set_morse(self._h, float(D0), float(alpha), float(r0), float(rc))

    def morse_energy(self, X):
        return lib().ora_morse_energy(self._h, _p(_f64(X)))

    def morse_forces(self, X):
        X = _f64(X)
        F = np.zeros_like(X)
        lib().ora_morse_forces(self._h, _p(X), _p(F))
        return F

    def mesh_rest(self):
        out = np.zeros(3)
        lib().ora_mesh_rest(self._h, _p(out))
        return dict(A0=out[0], V0=out[1], l0_mean=out[2])

    # stepping
    def stage_forces(self):
        lib().ora_stage_forces(self._h)

    def stage_spread(self):
        lib().ora_stage_spread(self._h)

    def stage_collide_stream(self):
        lib().ora_stage_collide_stream(self._h)

    def stage_interpolate(self):
        lib().ora_stage_interpolate(self._h)

    def step(self, n=1):
        lib().ora_step(self._h, int(n))

    def solid_steps(self, n, dt, gamma, mass, f_ext=None, v=None):
        """Solid-only velocity-Verlet steps; returns the velocities [3][M]."""
        v = np.zeros((3, self.M)) if v is None else _f64(v).copy()
        fe = None if f_ext is None else _f64(f_ext)
        lib().ora_solid_steps(self._h, int(n), float(dt), float(gamma), float(mass), _p(fe), _p(v))
        return v
