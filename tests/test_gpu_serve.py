"""Serving (continuous batching of independent simulations on one GPU): a
case's result does not depend on which other cases it is batched with or on
when it is admitted; the batched path agrees with the single-lattice path
and with the FP64 oracle; admission honours the slots and the memory
budget; invalid requests are reported."""
import numpy as np
import pytest

import oracle as O
from paper_1704_04551_gb300 import inputs as I
from tests._cases import LATTICES, fluid_mask, markers_inside, rel_l2

pytestmark = pytest.mark.gpu


def _membranes(n_steps):
    w = I.rbc_tube(n=40, radius=16.0, n_cells=3, seed=21, steps=0)
    rng = np.random.default_rng(22)
    w['X'] = w['X'] + 0.08 * rng.standard_normal(w['X'].shape)
    for b in w['bodies']:
        b.update(kBT_p=2e-3, k_b=1e-3, k_l=5e-3, k_g=4e-3, k_v=3e-3)
    w['lattice'] = dict(w['lattice'], body_force=[2e-6, 0, 0])
    return w, n_steps


def _tracers(n_steps):
    lat = LATTICES['periodic']
    return dict(lattice=lat, mesh=None, bodies=[], X=markers_inside(lat, 300, 5)), n_steps


def _mix():
    """Four different cases, step counts that end mid-chunk, odd and even."""
    return [
        (I.shear_ellipsoid(n=24, axes=(5.0, 2.5, 2.5), seed=41), 70),
        _membranes(46),
        _tracers(33),
        (I.shear_ellipsoid(n=28, ny=24, nz=20, tau=0.9, axes=(6.0, 2.0, 2.0), seed=42, couette_init=True), 90),
    ]


def _serve(cases, max_active, budget=1 << 34, chunk=8):
    from paper_1704_04551_gb300.binding import OK, Server
    srv = Server(budget, max_active=max_active, chunk_steps=chunk)
    ids = [srv.submit(w, n) for w, n in cases]
    most = 0
    for _ in range(100000):
        rc, running, pending, done = srv.advance()
        assert rc == OK
        most = max(most, running)
        if running == 0 and pending == 0:
            break
    assert done == len(cases)
    out = [srv.result(i) for i in ids]
    srv.close()
    return out, most


def _same(a, b, exact):
    """Bit-identical where one marker group covers all markers. Several
    groups add their boxes into the force density with float atomics, so a
    cell two groups reach sums in either order and its bits may differ at
    rounding level from run to run (batched or not): there the bound is
    1e-6 relative L2 on u and 1e-7 lu on marker positions (FP32 rounding of
    U ~ 1e-3 over ~50 advection steps, amplified by the stiff membranes)."""
    if exact:
        for k in ('rho', 'u', 'X', 'U'):
            assert np.array_equal(a[k], b[k]), k
        for ba, bb in zip(a['bodies'], b['bodies']):
            for k in ('center', 'quat', 'vel', 'omega'):
                assert ba[k] == bb[k], k
        return
    assert rel_l2(a['u'], b['u']) < 1e-6
    assert rel_l2(a['rho'], b['rho']) < 1e-7
    assert np.abs(a['X'] - b['X']).max() < 1e-7


def test_case_alone_equals_case_in_mix(cuda_lib):
    """The batched kernels run each case's own arithmetic on its own arrays:
    alone, batched with all others, or admitted late behind a two-slot limit,
    a case's result is the same (bit-identical for the single-group rigid
    ellipsoids)."""
    cases = _mix()
    exact = [True, False, False, True]
    alone = [_serve([c], 1)[0][0] for c in cases]
    mixed, most = _serve(cases, 8)
    assert most == len(cases)
    queued, most2 = _serve(cases, 2)
    assert most2 == 2
    for a, m, q, e in zip(alone, mixed, queued, exact):
        _same(a, m, e)
        _same(a, q, e)


def test_served_case_matches_handle_and_oracle(cuda_lib):
    """A served rigid-ellipsoid shear cell and served membranes agree with the
    single-lattice handle (same device bodies, different launch shapes) and
    with the FP64 oracle within the coupled-parity tolerances."""
    from paper_1704_04551_gb300.binding import Simulation
    cases = [(I.shear_ellipsoid(n=32, steps=200), 200), _membranes(60)]
    served, _ = _serve(cases, 4, chunk=16)
    for (w, n), r in zip(cases, served):
        sim = Simulation.from_workload(w)
        sim.step(n)
        rho_h, u_h = sim.fields()
        X_h, U_h, _ = sim.markers()
        assert rel_l2(r['u'], u_h) < 1e-6
        assert np.abs(r['X'] - X_h).max() < 1e-7
        ora = O.Oracle.from_workload(w)
        ora.step(n)
        fl = fluid_mask(w['lattice'])
        _, uo = ora.fields()
        Xo, _, _ = ora.markers()
        assert rel_l2(r['u'][:, fl], uo[:, fl]) < 1e-5
        assert np.abs(r['X'] - Xo).max() < 1e-5
    bo = O.Oracle.from_workload(cases[0][0])
    bo.step(cases[0][1])
    assert np.allclose(served[0]['bodies'][0]['quat'], bo.body(0)['quat'], atol=1e-6)


def test_admission_honours_memory_budget(cuda_lib):
    """Identical cases under a budget of three cases' device memory: never
    more than three run at once, all finish, in submission order."""
    from paper_1704_04551_gb300.binding import OK, Server, Simulation, CASE_DONE
    w = I.shear_ellipsoid(n=24, axes=(5.0, 2.5, 2.5), seed=43)
    one = Simulation.from_workload(w).device_bytes
    srv = Server(3 * one, max_active=8, chunk_steps=4)
    ids = [srv.submit(w, 12 + 4 * k) for k in range(7)]
    most, order = 0, []
    for _ in range(1000):
        rc, running, pending, _ = srv.advance()
        assert rc == OK
        most = max(most, running)
        for i in ids:
            if i not in order and srv.poll(i)[0] == CASE_DONE:
                order.append(i)
        if running == 0 and pending == 0:
            break
    assert 1 <= most <= 3
    assert order == ids
    for i in ids:
        assert srv.poll(i)[1] >= 12
        srv.result(i)
    srv.close()


def test_server_reports_invalid_requests(cuda_lib):
    from paper_1704_04551_gb300.binding import E_ARG, E_STATE, IbmLbmError, Server
    w = I.shear_ellipsoid(n=24, seed=44)
    srv = Server(1 << 30, max_active=2, chunk_steps=4)
    cid = srv.submit(w, 8)
    with pytest.raises(IbmLbmError) as e:
        srv.result(cid)  # not finished
    assert e.value.code == E_STATE
    with pytest.raises(IbmLbmError) as e:
        srv.poll(cid + 100)
    assert e.value.code == E_ARG
    srv.meta[cid]  # still known
    srv.close()
    small = Server(1 << 16, max_active=2, chunk_steps=4)
    with pytest.raises(IbmLbmError) as e:
        small.submit(w, 8)  # can never fit the budget
    assert e.value.code == E_ARG
    small.close()
    from paper_1704_04551_gb300 import binding as B
    with pytest.raises(IbmLbmError):
        B.ibm_lbm_server_create(B.ServerConfig(1 << 20, 1, 3, 0), None, None)  # odd chunk
