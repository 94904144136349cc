"""Failure paths, made on the host (no GPU fault): an allocator callback
that runs out of memory, a flow that leaves the stability bound, and a
served case that goes unstable beside healthy ones.

* E_NOMEM: ibm_lbm_create and ibm_lbm_set_markers return it when the
  caller's allocator returns NULL at any of their allocations, release
  everything they took, and leave a usable handle; a server whose allocator
  refuses keeps the case waiting and admits it once memory is there.
* E_UNSTABLE: the FP64 check at the end of ibm_lbm_step flags |u| > 0.4
  (0.45 here, in a periodic box without markers: a uniform flow that the
  collision leaves unchanged, so no marker position ever enters an index).
* A served case started at |u| = 0.45 is retired with E_UNSTABLE while the
  cases beside it finish exactly as they do alone."""
import numpy as np
import pytest

from tests._cases import LATTICES, markers_inside, membrane_case

pytestmark = pytest.mark.gpu


def _flaky(binding):
    class Flaky(binding.TorchMemory):
        """torch-backed allocator that returns NULL from call `fail_at` on."""

        def __init__(self, dev):
            super().__init__(dev)
            self.calls = 0
            self.fail_at = None

        def _on_alloc(self, nbytes, ctx):
            self.calls += 1
            if self.fail_at is not None and self.calls >= self.fail_at:
                return None
            return super()._on_alloc(nbytes, ctx)

    import torch
    return Flaky(torch.device('cuda', 0))


def test_create_reports_nomem_and_releases(cuda_lib):
    lat = LATTICES['tube']
    probe = _flaky(cuda_lib)
    sim = cuda_lib.Simulation(lat, memory=probe)
    n_create = probe.calls
    sim.close()
    assert n_create >= 3 and not probe.live
    for k in range(1, n_create + 1):
        mem = _flaky(cuda_lib)
        mem.fail_at = k
        with pytest.raises(cuda_lib.IbmLbmError) as e:
            cuda_lib.Simulation(lat, memory=mem)
        assert e.value.code == cuda_lib.E_NOMEM, k
        assert not mem.live, f'allocation {k}: {len(mem.live)} buffers not released'


def test_set_markers_reports_nomem_and_handle_stays_usable(cuda_lib):
    w = membrane_case()
    mem = _flaky(cuda_lib)
    sim = cuda_lib.Simulation(w['lattice'], memory=mem)
    lattice_buffers = set(mem.live)
    c0 = mem.calls
    sim.set_markers(w['mesh'], w['bodies'], w['X'])
    n_markers = mem.calls - c0
    assert n_markers >= 5
    for k in range(1, n_markers + 1):
        mem.fail_at = mem.calls + k
        with pytest.raises(cuda_lib.IbmLbmError) as e:
            sim.set_markers(w['mesh'], w['bodies'], w['X'])
        assert e.value.code == cuda_lib.E_NOMEM, k
        assert set(mem.live) == lattice_buffers, f'allocation {k}: marker buffers left behind'
        mem.fail_at = None
        sim.step(2)  # a lattice without markers steps
    mem.fail_at = None
    sim.set_markers(w['mesh'], w['bodies'], w['X'])
    sim.step(3)
    d = sim.diagnostics()
    assert np.isfinite(d['mass']) and d['steps'] >= 3
    X = sim.markers()[0]
    assert np.isfinite(X).all() and np.abs(X - w['X']).max() < 0.1


def test_server_waits_for_memory_then_admits(cuda_lib):
    mem = _flaky(cuda_lib)
    srv = cuda_lib.Server(1 << 33, max_active=4, chunk_steps=4, memory=mem)
    lat = LATTICES['periodic']
    w = dict(lattice=lat, mesh=None, bodies=[], X=markers_inside(lat, 50, 3))
    mem.fail_at = mem.calls + 1  # every allocation from now on fails
    cid = srv.submit(w, 8)
    for _ in range(3):
        rc, running, pending, done = srv.advance()
        assert rc == cuda_lib.OK and running == 0 and pending == 1
    mem.fail_at = None
    for _ in range(10):
        rc, running, pending, done = srv.advance()
        assert rc == cuda_lib.OK
        if done:
            break
    assert done == 1
    r = srv.result(cid)
    alone = cuda_lib.Simulation.from_workload(w)
    alone.step(8)
    assert np.array_equal(r['u'], alone.fields()[1])
    srv.close()
    assert not mem.live


def test_step_reports_unstable_flow(cuda_lib):
    lat = dict(nx=16, ny=12, nz=10, tau=0.8, geometry=0)
    sim = cuda_lib.Simulation(lat)
    sim.set_markers(None, [], np.zeros((3, 0)))
    u = np.zeros((3, sim.N))
    u[0] = 0.45
    sim.set_lattice(None, u)
    with pytest.raises(cuda_lib.IbmLbmError) as e:
        sim.step(1)
    assert e.value.code == cuda_lib.E_UNSTABLE
    u[0] = 0.05  # the same handle recovers with a stable state
    sim.set_lattice(None, u)
    sim.step(4)
    assert abs(sim.diagnostics()['umax'] - 0.05) < 1e-6


def test_server_retires_unstable_case_neighbours_unchanged(cuda_lib):
    lat = dict(nx=16, ny=12, nz=10, tau=0.8, geometry=0)
    N = 16 * 12 * 10
    bad_u = np.zeros((3, N))
    bad_u[0] = 0.45
    bad = dict(lattice=lat, mesh=None, bodies=[], X=np.zeros((3, 0)), u0=bad_u)
    ok_lat = LATTICES['periodic']
    good = dict(lattice=ok_lat, mesh=None, bodies=[], X=markers_inside(ok_lat, 80, 8))
    srv = cuda_lib.Server(1 << 33, max_active=4, chunk_steps=4)
    ids = [srv.submit(good, 12), srv.submit(bad, 6), srv.submit(good, 10)]
    seen_unstable = False
    for _ in range(50):
        rc, running, pending, done = srv.advance()
        assert rc in (cuda_lib.OK, cuda_lib.E_UNSTABLE)
        seen_unstable |= rc == cuda_lib.E_UNSTABLE
        if running == 0 and pending == 0:
            break
    assert seen_unstable
    res = [srv.result(i) for i in ids]
    assert np.abs(res[1]['u'][0]).max() > 0.4  # the unstable result is still kept
    for r, n in ((res[0], 12), (res[2], 10)):
        alone = cuda_lib.Simulation.from_workload(good)
        alone.step(n)
        rho, u = alone.fields()
        X = alone.markers()[0]
        assert np.array_equal(r['u'], u) and np.array_equal(r['rho'], rho) and np.array_equal(r['X'], X)
    srv.close()
