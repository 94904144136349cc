"""Thin ctypes binding of ``libibmlbm.so`` (C ABI in ``include/ibm_lbm.h``).

The functions keep the C names (``ibm_lbm_create``, ``ibm_lbm_step`` ...) and
only marshal arguments: every stage of the coupled step runs in the CUDA
library. PyTorch is used for plumbing only: the device memory the library
asks for comes from torch's caching allocator (through the C allocator
callbacks), and the work is ordered on a ``torch.cuda.Stream``.

The library must have been built (``paper_1704_04551_gb300.build.build()``,
or ``__graft_entry__.build()``); loading fails loudly otherwise — there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get('IBM_LBM_LIBRARY') or os.path.join(_HERE, 'libibmlbm.so')

OK, E_ARG, E_NOMEM, E_CUDA, E_UNSTABLE, E_TIMEOUT, E_STATE = 0, -1, -2, -3, -4, -5, -6
STORE_F32, STORE_F16_DEV, STORE_BF16_DEV = 0, 1, 2
STORAGE = {'f32': STORE_F32, 'f16': STORE_F16_DEV, 'bf16': STORE_BF16_DEV}
STAGE_FORCES, STAGE_SPREAD, STAGE_COLLIDE, STAGE_INTERP = 0, 1, 2, 3


class IbmLbmError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f'ibm_lbm error {code}: {msg}')
        self.code = code


class Config(C.Structure):
    _fields_ = [('nx', C.c_int32), ('ny', C.c_int32), ('nz', C.c_int32), ('geometry', C.c_int32),
                ('tau', C.c_double), ('wall_u', C.c_double * 2), ('tube_radius', C.c_double),
                ('body_force', C.c_double * 3), ('storage', C.c_int32), ('device', C.c_int32)]


class Body(C.Structure):
    _fields_ = [('kind', C.c_int32), ('pad', C.c_int32), ('first', C.c_int64), ('count', C.c_int64),
                ('kBT_p', C.c_double), ('k_b', C.c_double), ('k_l', C.c_double), ('k_g', C.c_double),
                ('k_v', C.c_double), ('kappa', C.c_double), ('mass', C.c_double),
                ('inertia', C.c_double * 3), ('center', C.c_double * 3), ('quat', C.c_double * 4),
                ('vel', C.c_double * 3), ('omega', C.c_double * 3), ('l0', C.c_double)]


class Mesh(C.Structure):
    _fields_ = [('n_vertices', C.c_int32), ('n_triangles', C.c_int32),
                ('tris', C.c_void_p), ('rest_X', C.c_void_p)]


class ServerConfig(C.Structure):
    _fields_ = [('device_mem_budget', C.c_size_t), ('max_active', C.c_int32), ('chunk_steps', C.c_int32),
                ('device', C.c_int32)]


class Case(C.Structure):
    _fields_ = [('lattice', Config), ('rho0', C.c_void_p), ('u0', C.c_void_p), ('mesh', C.POINTER(Mesh)),
                ('n_bodies', C.c_int32), ('bodies', C.c_void_p), ('n_markers', C.c_int64), ('X', C.c_void_p),
                ('n_steps', C.c_int64)]


CASE_PENDING, CASE_RUNNING, CASE_DONE = 0, 1, 2

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [('alloc', ALLOC_FN), ('release', RELEASE_FN), ('ctx', C.c_void_p)]


_lib = None


def load():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f'{LIB_PATH} is missing: build it with paper_1704_04551_gb300.build.build()')
    L = C.CDLL(LIB_PATH)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        'ibm_lbm_create': ([C.POINTER(Config), C.POINTER(Allocator), P, C.POINTER(P)], C.c_int),
        'ibm_lbm_destroy': ([P], C.c_int),
        'ibm_lbm_set_lattice': ([P, P, P], C.c_int),
        'ibm_lbm_set_populations': ([P, P], C.c_int),
        'ibm_lbm_get_populations': ([P, P], C.c_int),
        'ibm_lbm_set_markers': ([P, C.POINTER(Mesh), I32, P, I64, P], C.c_int),
        'ibm_lbm_set_morse': ([P, D, D, D, D], C.c_int),
        'ibm_lbm_solid_steps': ([P, I64, D, D, D, P], C.c_int),
        'ibm_lbm_step': ([P, I64], C.c_int),
        'ibm_lbm_step_async': ([P, I64], C.c_int),
        'ibm_lbm_synchronize': ([P], C.c_int),
        'ibm_lbm_get_fields': ([P, P, P], C.c_int),
        'ibm_lbm_get_markers': ([P, P, P, P], C.c_int),
        'ibm_lbm_get_bodies': ([P, P, I32], C.c_int),
        'ibm_lbm_get_diagnostics': ([P, P], C.c_int),
        'ibm_lbm_run_stage': ([P, I32], C.c_int),
        'ibm_lbm_set_marker_forces': ([P, P], C.c_int),
        'ibm_lbm_get_force_density': ([P, P], C.c_int),
        'ibm_lbm_set_timing': ([P, I64], C.c_int),
        'ibm_lbm_get_timing': ([P, P], C.c_int),
        'ibm_lbm_set_timing_fused': ([P, I32], C.c_int),
        'ibm_lbm_spread_noalloc': ([P, P, I64, I32, I32, I32, I32, D, P, P], C.c_int),
        'ibm_lbm_stream': ([P], P),
        'ibm_lbm_device_bytes': ([P], C.c_size_t),
        'ibm_lbm_last_error': ([P], C.c_char_p),
        'ibm_lbm_version': ([], C.c_char_p),
        'ibm_lbm_server_create': ([C.POINTER(ServerConfig), C.POINTER(Allocator), P, C.POINTER(P)], C.c_int),
        'ibm_lbm_server_destroy': ([P], C.c_int),
        'ibm_lbm_server_submit': ([P, C.POINTER(Case), C.POINTER(C.c_uint64)], C.c_int),
        'ibm_lbm_server_advance': ([P, C.POINTER(I32), C.POINTER(I32), C.POINTER(I32)], C.c_int),
        'ibm_lbm_server_poll': ([P, C.c_uint64, C.POINTER(I32), C.POINTER(I64)], C.c_int),
        'ibm_lbm_server_result': ([P, C.c_uint64, P, P, P, P, P, I32], C.c_int),
        'ibm_lbm_server_last_error': ([P], C.c_char_p),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def exported_symbols():
    """Names declared in the public header (for the ABI check)."""
    hdr = os.path.join(os.path.dirname(_HERE), 'include', 'ibm_lbm.h')
    import re
    names = []
    with open(hdr) as f:
        for m in re.finditer(r'^\s*(?:const\s+)?[\w\s\*]+?\b(ibm_lbm_\w+)\s*\(', f.read(), re.M):
            names.append(m.group(1))
    return sorted(set(names))


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
# the C entry points under their own names (argument marshalling only)
# ---------------------------------------------------------------------------
def _check(h, rc):
    if rc != OK:
        msg = load().ibm_lbm_last_error(h)
        raise IbmLbmError(rc, msg.decode() if msg else '')
    return rc


def ibm_lbm_create(cfg: Config, allocator: Allocator | None, stream: int | None):
    out = C.c_void_p()
    rc = load().ibm_lbm_create(C.byref(cfg), C.byref(allocator) if allocator is not None else None,
                               C.c_void_p(stream) if stream else None, C.byref(out))
    if rc != OK:
        raise IbmLbmError(rc, 'create failed (invalid config, allocation or CUDA error)')
    return out


def ibm_lbm_destroy(h):
    return load().ibm_lbm_destroy(h)


def ibm_lbm_set_lattice(h, rho=None, u=None):
    rho = None if rho is None else _f64(rho)
    u = None if u is None else _f64(u)
    return _check(h, load().ibm_lbm_set_lattice(h, _p(rho), _p(u)))


def ibm_lbm_set_populations(h, f):
    return _check(h, load().ibm_lbm_set_populations(h, _p(_f64(f))))


def ibm_lbm_get_populations(h, f):
    return _check(h, load().ibm_lbm_get_populations(h, _p(f)))


def ibm_lbm_set_markers(h, mesh: Mesh | None, bodies, X):
    """bodies: a list of Body records, or the structured array body_array
    returns (the same bytes, filled without a Python object per body)."""
    X = _f64(X)
    if isinstance(bodies, np.ndarray):
        assert bodies.dtype == BODY_DTYPE and bodies.flags.c_contiguous
        n = len(bodies)
        arr = bodies if n else np.zeros(1, dtype=BODY_DTYPE)
        ptr = arr.ctypes.data
    else:
        n = len(bodies)
        arr = (Body * max(1, n))(*bodies) if bodies else (Body * 1)()
        ptr = C.cast(arr, C.c_void_p)
    return _check(h, load().ibm_lbm_set_markers(h, C.byref(mesh) if mesh is not None else None,
                                                n, ptr, X.shape[1], _p(X)))


def ibm_lbm_set_morse(h, D0, alpha, r0, rc):
    return _check(h, load().ibm_lbm_set_morse(h, float(D0), float(alpha), float(r0), float(rc)))


def ibm_lbm_solid_steps(h, n, dt, gamma, mass, f_ext=None):
    fe = None if f_ext is None else _f64(f_ext)
    return _check(h, load().ibm_lbm_solid_steps(h, int(n), float(dt), float(gamma), float(mass), _p(fe)))


def ibm_lbm_step(h, n):
    return _check(h, load().ibm_lbm_step(h, int(n)))


def ibm_lbm_step_async(h, n):
    return _check(h, load().ibm_lbm_step_async(h, int(n)))


def ibm_lbm_synchronize(h):
    return _check(h, load().ibm_lbm_synchronize(h))


def ibm_lbm_get_fields(h, rho, u):
    return _check(h, load().ibm_lbm_get_fields(h, _p(rho), _p(u)))


def ibm_lbm_get_markers(h, X, U, F):
    return _check(h, load().ibm_lbm_get_markers(h, _p(X), _p(U), _p(F)))


def ibm_lbm_get_bodies(h, n):
    arr = (Body * max(1, n))()
    _check(h, load().ibm_lbm_get_bodies(h, arr, n))
    return [arr[i] for i in range(n)]


def ibm_lbm_get_diagnostics(h):
    out = np.zeros(8)
    _check(h, load().ibm_lbm_get_diagnostics(h, _p(out)))
    return out


def ibm_lbm_run_stage(h, stage):
    return _check(h, load().ibm_lbm_run_stage(h, int(stage)))


def ibm_lbm_set_marker_forces(h, F):
    return _check(h, load().ibm_lbm_set_marker_forces(h, _p(_f64(F))))


def ibm_lbm_get_force_density(h, g):
    return _check(h, load().ibm_lbm_get_force_density(h, _p(g)))


def ibm_lbm_set_timing(h, max_steps):
    return _check(h, load().ibm_lbm_set_timing(h, int(max_steps)))


def ibm_lbm_set_timing_fused(h, on):
    return _check(h, load().ibm_lbm_set_timing_fused(h, 1 if on else 0))


def ibm_lbm_get_timing(h):
    out = np.zeros(6)
    _check(h, load().ibm_lbm_get_timing(h, _p(out)))
    return out


def ibm_lbm_spread_noalloc(X_ptr, F_ptr, n_markers, nx, ny, nz, geometry, tube_radius, g_ptr, stream=None):
    """Spreading without device allocation; all pointers are device
    addresses owned by the caller (see the header for the contract)."""
    return load().ibm_lbm_spread_noalloc(C.c_void_p(X_ptr), C.c_void_p(F_ptr), int(n_markers), int(nx), int(ny),
                                         int(nz), int(geometry), float(tube_radius), C.c_void_p(g_ptr),
                                         C.c_void_p(stream) if stream else None)


def ibm_lbm_stream(h):
    return load().ibm_lbm_stream(h)


def ibm_lbm_device_bytes(h):
    return load().ibm_lbm_device_bytes(h)


def ibm_lbm_last_error(h):
    return load().ibm_lbm_last_error(h).decode()


def ibm_lbm_version():
    return load().ibm_lbm_version().decode()


def _server_check(s, rc):
    if rc != OK:
        msg = load().ibm_lbm_server_last_error(s)
        raise IbmLbmError(rc, msg.decode() if msg else '')
    return rc


def ibm_lbm_server_create(cfg: ServerConfig, allocator: Allocator | None, stream: int | None):
    out = C.c_void_p()
    rc = load().ibm_lbm_server_create(C.byref(cfg), C.byref(allocator) if allocator else None, stream, C.byref(out))
    if rc != OK:
        raise IbmLbmError(rc, 'ibm_lbm_server_create failed')
    return out


def ibm_lbm_server_destroy(s):
    return load().ibm_lbm_server_destroy(s)


def ibm_lbm_server_submit(s, case: Case):
    cid = C.c_uint64()
    _server_check(s, load().ibm_lbm_server_submit(s, C.byref(case), C.byref(cid)))
    return cid.value


def ibm_lbm_server_advance(s):
    """Returns (rc, n_running, n_pending, n_done); rc is OK or E_UNSTABLE."""
    r, p, d = C.c_int32(), C.c_int32(), C.c_int32()
    rc = load().ibm_lbm_server_advance(s, C.byref(r), C.byref(p), C.byref(d))
    if rc not in (OK, E_UNSTABLE):
        _server_check(s, rc)
    return rc, r.value, p.value, d.value


def ibm_lbm_server_poll(s, cid):
    st, n = C.c_int32(), C.c_int64()
    _server_check(s, load().ibm_lbm_server_poll(s, cid, C.byref(st), C.byref(n)))
    return st.value, n.value


def ibm_lbm_server_result(s, cid, rho, u, X, U, bodies_n):
    arr = (Body * bodies_n)() if bodies_n else None
    _server_check(s, load().ibm_lbm_server_result(s, cid, _p(rho), _p(u), _p(X), _p(U), arr, bodies_n))
    return list(arr) if arr is not None else []


def ibm_lbm_server_last_error(s):
    return load().ibm_lbm_server_last_error(s).decode()


# ---------------------------------------------------------------------------
# convenience: one simulation handle with torch-provided memory and stream
# ---------------------------------------------------------------------------
class TorchMemory:
    """Device memory from torch's caching allocator, handed to the library
    through the C allocator callbacks."""

    def __init__(self, device):
        import torch
        self._torch = torch
        self.device = device
        self.live = {}
        self._alloc = ALLOC_FN(self._on_alloc)
        self._release = RELEASE_FN(self._on_release)
        self.struct = Allocator(self._alloc, self._release, None)

    def _on_alloc(self, nbytes, ctx):
        try:
            t = self._torch.empty(int(nbytes), dtype=self._torch.uint8, device=self.device)
        except Exception:  # out of memory: the library reports E_NOMEM
            return None
        p = t.data_ptr()
        self.live[p] = t
        return p

    def _on_release(self, ptr, ctx):
        self.live.pop(ptr, None)


def make_config(lattice: dict, storage='f32', device=0) -> Config:
    cfg = Config()
    cfg.nx, cfg.ny, cfg.nz = int(lattice['nx']), int(lattice['ny']), int(lattice['nz'])
    cfg.geometry = int(lattice['geometry'])
    cfg.tau = float(lattice['tau'])
    wu = lattice.get('wall_u', (0.0, 0.0))
    cfg.wall_u[0], cfg.wall_u[1] = float(wu[0]), float(wu[1])
    cfg.tube_radius = float(lattice.get('tube_radius', 0.0))
    for i, v in enumerate(lattice.get('body_force', (0.0, 0.0, 0.0))):
        cfg.body_force[i] = float(v)
    cfg.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
    cfg.device = int(device)
    return cfg


_BODY_SCALARS = ('kBT_p', 'k_b', 'k_l', 'k_g', 'k_v', 'kappa', 'mass')
_BODY_VECTORS = (('inertia', 3), ('center', 3), ('quat', 4), ('vel', 3), ('omega', 3))
# ibm_lbm_body as a numpy record (naturally aligned, no padding beyond `pad`)
BODY_DTYPE = np.dtype([('kind', '<i4'), ('pad', '<i4'), ('first', '<i8'), ('count', '<i8')] +
                      [(k, '<f8') for k in _BODY_SCALARS] + [(k, '<f8', (n,)) for k, n in _BODY_VECTORS] +
                      [('l0', '<f8')])


def body_array(bodies) -> np.ndarray:
    """Body dicts (as make_body takes them) as one ibm_lbm_body array."""
    if not bodies:
        return np.zeros(0, dtype=BODY_DTYPE)
    z3, q0 = (0.0, 0.0, 0.0), (1.0, 0.0, 0.0, 0.0)
    rows = [(d['kind'], 0, d['first'], d['count'], d.get('kBT_p', 0.0), d.get('k_b', 0.0), d.get('k_l', 0.0),
             d.get('k_g', 0.0), d.get('k_v', 0.0), d.get('kappa', 0.0), d.get('mass', 0.0),
             tuple(d.get('inertia', z3))[:3], tuple(d.get('center', z3))[:3], tuple(d.get('quat', q0))[:4],
             tuple(d.get('vel', z3))[:3], tuple(d.get('omega', z3))[:3], d.get('l0', 0.0)) for d in bodies]
    return np.array(rows, dtype=BODY_DTYPE)


def make_body(d) -> Body:
    b = Body()
    b.kind, b.first, b.count = int(d['kind']), int(d['first']), int(d['count'])
    for k in ('kBT_p', 'k_b', 'k_l', 'k_g', 'k_v', 'kappa', 'mass', 'l0'):
        setattr(b, k, float(d.get(k, 0.0)))
    for k, n in (('inertia', 3), ('center', 3), ('quat', 4), ('vel', 3), ('omega', 3)):
        arr = getattr(b, k)
        vals = d.get(k, [1.0, 0, 0, 0] if k == 'quat' else [0.0] * n)
        for i in range(n):
            arr[i] = float(vals[i])
    return b


class Simulation:
    """One lattice with its markers on one GPU (wraps an ibm_lbm handle)."""

    def __init__(self, lattice: dict, storage='f32', device=0, use_torch=True, stream=None, memory=None):
        """memory: an object with an ``Allocator`` in ``.struct`` (default:
        TorchMemory when use_torch, else cudaMalloc inside the library)."""
        self.shape = (int(lattice['nx']), int(lattice['ny']), int(lattice['nz']))
        self.N = int(np.prod(self.shape))
        self.M = 0
        self.n_bodies = 0
        self._mem = memory
        self._stream_obj = None
        if use_torch:
            import torch
            dev = torch.device('cuda', device)
            if self._mem is None:
                self._mem = TorchMemory(dev)
            if stream is None:
                self._stream_obj = torch.cuda.Stream(device=dev)
                stream = self._stream_obj.cuda_stream
        self.h = ibm_lbm_create(make_config(lattice, storage, device),
                                self._mem.struct if self._mem else None, stream)

    def close(self):
        if getattr(self, 'h', None):
            ibm_lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    @classmethod
    def from_workload(cls, w: dict, storage='f32', device=0, **kw):
        s = cls(w['lattice'], storage=storage, device=device, **kw)
        s.set_lattice(w.get('rho0'), w.get('u0'))
        if w.get('morse') is not None:
            s.set_morse(**w['morse'])
        s.set_markers(w.get('mesh'), w.get('bodies', []), w['X'])
        return s

    # lattice
    def set_lattice(self, rho=None, u=None):
        ibm_lbm_set_lattice(self.h, rho, u)

    def set_populations(self, f):
        ibm_lbm_set_populations(self.h, f)

    def populations(self):
        f = np.zeros((19, self.N))
        ibm_lbm_get_populations(self.h, f)
        return f

    def fields(self):
        rho = np.zeros(self.N)
        u = np.zeros((3, self.N))
        ibm_lbm_get_fields(self.h, rho, u)
        return rho, u

    def force_density(self):
        g = np.zeros((3, self.N))
        ibm_lbm_get_force_density(self.h, g)
        return g

    # markers
    def set_markers(self, mesh, bodies, X):
        X = _f64(X)
        m = None
        self._mesh_arrays = None
        if mesh is not None:
            tris = np.ascontiguousarray(mesh['tris'], dtype=np.int32)
            rest = _f64(mesh['rest_X'])
            self._mesh_arrays = (tris, rest)
            m = Mesh(rest.shape[1], tris.shape[0], tris.ctypes.data, rest.ctypes.data)
        ibm_lbm_set_markers(self.h, m, body_array(bodies), X)
        self.M = X.shape[1]
        self.n_bodies = len(bodies)

    def set_morse(self, D0, alpha, r0, rc):
        ibm_lbm_set_morse(self.h, D0, alpha, r0, rc)

    def solid_steps(self, n, dt, gamma, mass, f_ext=None):
        """Solid-only damped velocity-Verlet steps of the markers (no fluid)."""
        ibm_lbm_solid_steps(self.h, n, dt, gamma, mass, f_ext)

    def set_marker_forces(self, F):
        ibm_lbm_set_marker_forces(self.h, F)

    def markers(self):
        X = np.zeros((3, self.M))
        U = np.zeros((3, self.M))
        F = np.zeros((3, self.M))
        ibm_lbm_get_markers(self.h, X, U, F)
        return X, U, F

    def bodies(self):
        out = []
        for b in ibm_lbm_get_bodies(self.h, self.n_bodies):
            out.append(dict(kind=b.kind, first=b.first, count=b.count, center=list(b.center),
                            quat=list(b.quat), vel=list(b.vel), omega=list(b.omega)))
        return out

    def diagnostics(self):
        d = ibm_lbm_get_diagnostics(self.h)
        return dict(mass=d[0], momentum=d[1:4].copy(), umax=d[4], steps=int(d[5]), fluid_cells=int(d[6]))

    # stepping
    def step(self, n=1):
        ibm_lbm_step(self.h, n)

    def step_async(self, n=1):
        ibm_lbm_step_async(self.h, n)

    def synchronize(self):
        ibm_lbm_synchronize(self.h)

    def stage(self, stage):
        ibm_lbm_run_stage(self.h, stage)

    def set_timing(self, max_steps, fused=False):
        ibm_lbm_set_timing(self.h, max_steps)
        ibm_lbm_set_timing_fused(self.h, fused)

    def timing(self):
        t = ibm_lbm_get_timing(self.h)
        return dict(forces_ms=t[0], spread_ms=t[1], collide_ms=t[2], interp_ms=t[3], steps=int(t[4]),
                    collide_odd_ms=t[5])

    @property
    def stream(self):
        return ibm_lbm_stream(self.h)

    @property
    def device_bytes(self):
        return ibm_lbm_device_bytes(self.h)


class Server:
    """Continuous batching of independent simulations on one GPU (wraps an
    ibm_lbm_server). Cases are workload dicts as for Simulation.from_workload
    plus a step count."""

    def __init__(self, device_mem_budget, max_active=64, chunk_steps=100, device=0, use_torch=True, stream=None,
                 memory=None):
        self._mem = memory
        self._stream_obj = None
        if use_torch:
            import torch
            dev = torch.device('cuda', device)
            if self._mem is None:
                self._mem = TorchMemory(dev)
            if stream is None:
                self._stream_obj = torch.cuda.Stream(device=dev)
                stream = self._stream_obj.cuda_stream
        cfg = ServerConfig(int(device_mem_budget), int(max_active), int(chunk_steps), int(device))
        self.device = device
        self.s = ibm_lbm_server_create(cfg, self._mem.struct if self._mem else None, stream)
        self.meta = {}

    def close(self):
        if getattr(self, 's', None):
            ibm_lbm_server_destroy(self.s)
            self.s = None

    def __del__(self):
        self.close()

    def submit(self, w: dict, n_steps: int) -> int:
        lat = w['lattice']
        N = int(lat['nx']) * int(lat['ny']) * int(lat['nz'])
        X = _f64(w['X'])
        keep = [X]
        case = Case()
        case.lattice = make_config(lat, 'f32', self.device)
        for name in ('rho0', 'u0'):
            if w.get(name) is not None:
                a = _f64(w[name])
                keep.append(a)
                setattr(case, name, a.ctypes.data)
        mesh = w.get('mesh')
        if mesh is not None:
            tris = np.ascontiguousarray(mesh['tris'], dtype=np.int32)
            rest = _f64(mesh['rest_X'])
            keep += [tris, rest]
            m = Mesh(rest.shape[1], tris.shape[0], tris.ctypes.data, rest.ctypes.data)
            keep.append(m)
            case.mesh = C.pointer(m)
        bodies = w.get('bodies', [])
        barr = (Body * len(bodies))(*[make_body(b) for b in bodies]) if bodies else None
        keep.append(barr)
        case.n_bodies = len(bodies)
        case.bodies = C.cast(barr, C.c_void_p) if barr is not None else None
        case.n_markers = X.shape[1]
        case.X = X.ctypes.data
        case.n_steps = int(n_steps)
        cid = ibm_lbm_server_submit(self.s, case)  # arrays are copied by the call
        self.meta[cid] = (N, X.shape[1], len(bodies))
        return cid

    def advance(self):
        """One chunk for all admitted cases; returns (rc, running, pending, done)."""
        return ibm_lbm_server_advance(self.s)

    def poll(self, cid):
        return ibm_lbm_server_poll(self.s, cid)

    def result(self, cid):
        N, M, nb = self.meta[cid]
        rho, u = np.zeros(N), np.zeros((3, N))
        X, U = np.zeros((3, M)), np.zeros((3, M))
        bodies = ibm_lbm_server_result(self.s, cid, rho, u, X, U, nb)
        del self.meta[cid]
        return dict(rho=rho, u=u, X=X, U=U,
                    bodies=[dict(center=list(b.center), quat=list(b.quat), vel=list(b.vel), omega=list(b.omega))
                            for b in bodies])
