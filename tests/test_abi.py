"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point that include/ibm_lbm.h declares (no compute calls)."""
import ctypes
import os
import subprocess

import pytest

from paper_1704_04551_gb300 import binding, build


@pytest.fixture(scope='module')
def libpath():
    return build.build()


def test_header_declares_the_boundary(libpath):
    names = binding.exported_symbols()
    for required in ('ibm_lbm_create', 'ibm_lbm_destroy', 'ibm_lbm_set_lattice', 'ibm_lbm_set_markers',
                     'ibm_lbm_step', 'ibm_lbm_get_fields', 'ibm_lbm_get_markers'):
        assert required in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in binding.exported_symbols():
        assert hasattr(lib, name), name
    out = subprocess.run(['nm', '-D', '--defined-only', libpath], capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    for name in binding.exported_symbols():
        assert name in exported, name


def test_binding_signatures_load(libpath):
    L = binding.load()
    assert binding.ibm_lbm_version().startswith('ibm_lbm')
    assert L.ibm_lbm_last_error(None) == b'null handle'
    # invalid configs are rejected before any device work
    cfg = binding.Config()
    cfg.nx = cfg.ny = cfg.nz = 2
    cfg.tau = 0.8
    out = ctypes.c_void_p()
    assert L.ibm_lbm_create(ctypes.byref(cfg), None, None, ctypes.byref(out)) == binding.E_ARG
    cfg.nx = cfg.ny = cfg.nz = 8
    cfg.tau = 0.4
    assert L.ibm_lbm_create(ctypes.byref(cfg), None, None, ctypes.byref(out)) == binding.E_ARG
    assert L.ibm_lbm_destroy(None) == 0
    # timing controls on a NULL handle are argument errors, not crashes
    assert L.ibm_lbm_set_timing(None, 4) == binding.E_ARG
    assert L.ibm_lbm_set_timing_fused(None, 1) == binding.E_ARG


def test_calls_without_a_device_fail_with_a_status(libpath):
    """With no CUDA device, a valid configuration is refused with an error
    code (no abort, no handle), and so is a server."""
    torch = pytest.importorskip('torch')
    if torch.cuda.is_available():
        pytest.skip('a CUDA device is present')
    L = binding.load()
    cfg = binding.Config()
    cfg.nx = cfg.ny = cfg.nz = 16
    cfg.tau = 0.8
    out = ctypes.c_void_p()
    rc = L.ibm_lbm_create(ctypes.byref(cfg), None, None, ctypes.byref(out))
    assert rc in (binding.E_CUDA, binding.E_NOMEM)
    assert not out.value


def test_body_array_matches_the_ctypes_records():
    """The numpy body records passed to ibm_lbm_set_markers have the C
    layout of ibm_lbm_body: same size and offsets, and the same bytes as the
    per-body ctypes records, for every body kind."""
    from paper_1704_04551_gb300 import inputs as I
    assert binding.BODY_DTYPE.itemsize == ctypes.sizeof(binding.Body)
    for name, _ in binding.Body._fields_:
        assert binding.BODY_DTYPE.fields[name][1] == getattr(binding.Body, name).offset, name
    cases = [I.rbc_tube(n=40, radius=18.0, n_cells=2, seed=3, freq=5, steps=0)['bodies'],
             I.shear_ellipsoid(n=24, seed=3)['bodies'], I.shear_ellipsoid(n=24, seed=3, direct=True)['bodies'],
             I.mixed_suspension(shape=(48, 40, 40), n_cells=2, n_filaments=3, beads=6, seed=5)['bodies']]
    for bodies in cases:
        ref = (binding.Body * len(bodies))(*[binding.make_body(b) for b in bodies])
        assert binding.body_array(bodies).tobytes() == ctypes.string_at(ctypes.addressof(ref), ctypes.sizeof(ref))
    assert binding.body_array([]).shape == (0,)
