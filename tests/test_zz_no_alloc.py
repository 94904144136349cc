"""ibm_lbm_spread_noalloc: spreading for callers that cannot allocate device
memory (e.g. a framework that has reserved the GPU's memory for its own pool,
or a loop that may not pay for allocation). It must give the same force
density as the SPREAD stage of a handle, on two calls in a row (the second
call must not see the first call's sums), without the library allocating.

Named to be collected last: a failure here leaves every other test run.
"""
import numpy as np
import pytest

from tests._cases import LATTICES, markers_inside, shape

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize('geom', list(LATTICES))
def test_spread_noalloc_matches_handle_spread(cuda_lib, geom):
    import torch
    binding = cuda_lib
    lat = LATTICES[geom]
    nx, ny, nz = shape(lat)
    N = nx * ny * nz
    X = markers_inside(lat, 300, 5)
    M = X.shape[1]
    rng = np.random.default_rng(17)
    sim = binding.Simulation(lat)
    sim.set_markers(None, [], X)
    dev = torch.device('cuda', 0)
    Xd = torch.tensor(X, dtype=torch.float64, device=dev)
    g = torch.empty((3, N), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    for call in range(2):
        F = 1e-3 * (2 * rng.random((3, M)) - 1)
        # existing entry points: set forces, SPREAD stage, read the density;
        # set_lattice then clears it for the next call (within a step the
        # collision consumes it and the interpolation clears it, but the
        # interpolation would also move these markers)
        sim.set_marker_forces(F)
        sim.stage(binding.STAGE_SPREAD)
        g_ref = sim.force_density()
        sim.set_lattice()
        Fd = torch.tensor(F, dtype=torch.float64, device=dev)
        g.fill_(float('nan'))
        rc = binding.ibm_lbm_spread_noalloc(Xd.data_ptr(), Fd.data_ptr(), M, nx, ny, nz, lat['geometry'],
                                            lat.get('tube_radius', 0.0), g.data_ptr(), stream.cuda_stream)
        assert rc == binding.OK
        torch.cuda.synchronize(dev)
        g_new = g.cpu().numpy()
        assert np.isfinite(g_new).all()
        # the tolerance of the spread parity tests
        assert np.abs(g_new - g_ref).max() < 2e-5 * np.abs(g_ref).max(), f'call {call}'


def test_spread_noalloc_allocates_no_device_memory(cuda_lib):
    """The point of the entry point: once the library's device code is loaded
    (the first call), further calls leave the device's free memory as it
    was. Torch's own buffers are created before the measurement."""
    import torch
    binding = cuda_lib
    lat = LATTICES['tube']
    nx, ny, nz = shape(lat)
    X = markers_inside(lat, 300, 5)
    M = X.shape[1]
    dev = torch.device('cuda', 0)
    Xd = torch.tensor(X, dtype=torch.float64, device=dev)
    Fd = torch.full((3, M), 1e-3, dtype=torch.float64, device=dev)
    g = torch.empty((3, nx * ny * nz), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def call():
        return binding.ibm_lbm_spread_noalloc(Xd.data_ptr(), Fd.data_ptr(), M, nx, ny, nz, lat['geometry'],
                                              lat.get('tube_radius', 0.0), g.data_ptr(), stream.cuda_stream)

    assert call() == binding.OK
    torch.cuda.synchronize(dev)
    free0 = torch.cuda.mem_get_info(dev)[0]
    for _ in range(5):
        assert call() == binding.OK
    torch.cuda.synchronize(dev)
    assert torch.cuda.mem_get_info(dev)[0] == free0


def test_spread_noalloc_skips_markers_outside_the_position_bound(cuda_lib):
    """Positions are read on the device only: a marker that is not finite or
    lies at |x| >= 2^30 contributes nothing, and the others are unaffected."""
    import torch
    binding = cuda_lib
    lat = LATTICES['periodic']
    nx, ny, nz = shape(lat)
    X = markers_inside(lat, 40, 5)
    M = X.shape[1]
    F = np.full((3, M), 1e-3)
    dev = torch.device('cuda', 0)
    stream = torch.cuda.current_stream(dev)
    g = torch.empty((3, nx * ny * nz), dtype=torch.float64, device=dev)

    def spread(Xh, Fh):
        Xd = torch.tensor(Xh, dtype=torch.float64, device=dev)
        Fd = torch.tensor(Fh, dtype=torch.float64, device=dev)
        rc = binding.ibm_lbm_spread_noalloc(Xd.data_ptr(), Fd.data_ptr(), Xh.shape[1], nx, ny, nz,
                                            lat['geometry'], 0.0, g.data_ptr(), stream.cuda_stream)
        assert rc == binding.OK
        torch.cuda.synchronize(dev)
        return g.cpu().numpy()

    ref = spread(X, F)
    bad = np.array([[np.nan, 2.0 ** 30, -3.0e12], [1.0, 2.0, 3.0], [np.inf, 1.0, 2.0]])
    got = spread(np.concatenate([X, bad], axis=1), np.concatenate([F, np.full((3, 3), 1e-3)], axis=1))
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()


def test_spread_noalloc_rejects_oversized_lattice(cuda_lib):
    binding = cuda_lib
    import torch
    dev = torch.device('cuda', 0)
    X = torch.zeros((3, 1), dtype=torch.float64, device=dev)
    g = torch.zeros(3, dtype=torch.float64, device=dev)
    rc = binding.ibm_lbm_spread_noalloc(X.data_ptr(), X.data_ptr(), 1, 128, 128, 128, 0, 0.0, g.data_ptr())
    assert rc == binding.E_ARG
    rc = binding.ibm_lbm_spread_noalloc(X.data_ptr(), X.data_ptr(), 1, 2, 8, 8, 0, 0.0, g.data_ptr())
    assert rc == binding.E_ARG
