"""The C-ABI library builds, loads and exports every entry point include/crp.h declares;
argument checks fire before any device work (runs without a GPU)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "crp.h")


@pytest.fixture(scope="module")
def L():
    from paper_1410_5323_gb300 import build

    build.build()
    import paper_1410_5323_gb300 as crp

    return crp.lib()


def _declared():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(crp_\w+)\s*\(", text, re.M)))


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n


def test_error_strings(L):
    for code in (0, -1, -2, -3, -4, -5, -6, -7):
        assert L.crp_error_string(code)
    assert b"unknown" in L.crp_error_string(-99)
    assert L.crp_version().startswith(b"crp")


def test_null_and_range_arguments_rejected_before_device_work(L):
    h = C.c_void_p()
    org = (C.c_double * 3)(0, 0, 0)
    g = np.zeros((2, 2, 2, 3), dtype=np.float32)
    assert L.crp_field_create(None, 1, 0, 2, 2, 2, 1.0, org, 1.0, C.byref(h)) == -1
    assert L.crp_field_create(g.ctypes.data, 1, 0, 0, 2, 2, 1.0, org, 1.0, C.byref(h)) == -1
    assert L.crp_field_create(g.ctypes.data, 1, 0, 2, 2, 2, -1.0, org, 1.0, C.byref(h)) == -1
    assert L.crp_field_create(g.ctypes.data, 9, 0, 2, 2, 2, 1.0, org, 1.0, C.byref(h)) == -1
    assert L.crp_field_create(g.ctypes.data, 2, 0, 2, 2, 2, 1.0, org, 0.0, C.byref(h)) == -1
    assert b"scale" in L.crp_last_error_detail()
    m = np.ones((2, 2, 2), dtype=np.float32)
    fake = C.c_void_p(8)         # never dereferenced: every check below fails first
    assert L.crp_field_modulate(None, m.ctypes.data, 1, 0, 2, 2, 2, 1.0, org) == -1
    assert L.crp_field_modulate(fake, None, 1, 0, 2, 2, 2, 1.0, org) == -1
    assert L.crp_field_modulate(fake, m.ctypes.data, 0, 0, 2, 2, 2, 1.0, org) == -1     # F64
    assert L.crp_field_modulate(fake, m.ctypes.data, 1, 0, 2, 0, 2, 1.0, org) == -1
    assert L.crp_field_modulate(fake, m.ctypes.data, 1, 0, 2, 2, 2, 0.0, org) == -1
    assert b"spacing" in L.crp_last_error_detail()
    sz = (C.c_double * 3)(1.0, 0.0, 1.0)
    assert L.crp_sim_set_boundary(None, 1, org, sz) == -1
    assert L.crp_sim_set_boundary(fake, 7, org, sz) == -1                    # unknown kind
    assert L.crp_sim_set_boundary(fake, 1, org, sz) == -1                    # a size of 0
    assert L.crp_sim_set_boundary(fake, 1, None, sz) == -1
    lay = C.c_int32(0)
    assert L.crp_sim_grid_layout(None, C.byref(lay)) == -1
    assert L.crp_sim_grid_layout(fake, None) == -1
    assert L.crp_lens_set_group(None, 16) == -1
    assert L.crp_lens_set_group(fake, 12) == -1                               # not 4, 8, 16, 32
    import paper_1410_5323_gb300 as crp
    sp = crp.Spectrum.of([(4, 2, 1.0)], 1.8, 1e19, 1e18, 1e21)
    xs = np.zeros(4)
    assert L.crp_source_sample(None, C.byref(sp), xs.ctypes.data, xs.ctypes.data, xs.ctypes.data, None, 0, 4, None) == -1
    bad = crp.Spectrum.of([(4, 5, 1.0)], 1.8, 1e19, 1e18, 1e21)       # Z > A
    assert L.crp_source_sample(fake, C.byref(bad), xs.ctypes.data, xs.ctypes.data, xs.ctypes.data, None, 0, 4, None) == -1
    bad = crp.Spectrum.of([(4, 2, 1.0)], 1.8, 1e19, 1e21, 1e18)       # e_min > e_max
    assert L.crp_source_sample(fake, C.byref(bad), xs.ctypes.data, xs.ctypes.data, xs.ctypes.data, None, 0, 4, None) == -1
    assert L.crp_source_sample(fake, C.byref(sp), None, xs.ctypes.data, xs.ctypes.data, None, 0, 4, None) == -1
    assert L.crp_healpix_ring(0, xs.ctypes.data, 1, xs.ctypes.data, None) == -1       # nside 0
    assert L.crp_healpix_ring(8, None, 1, xs.ctypes.data, None) == -1
    assert L.crp_arrival_map(fake, 9000, 1e18, xs.ctypes.data, None) == -1             # nside too large
    assert L.crp_arrival_map(None, 8, 1e18, xs.ctypes.data, None) == -1
    rp = np.array([0, 1, 1], np.int64)
    cl = np.array([0], np.int32)
    vl = np.ones(1, np.float32)
    assert L.crp_lens_create(0, 1, rp.ctypes.data, cl.ctypes.data, vl.ctypes.data, None, C.byref(h)) == -1
    assert L.crp_lens_create(2, 1, None, cl.ctypes.data, vl.ctypes.data, None, C.byref(h)) == -1
    bad_rp = np.array([1, 1, 1], np.int64)                                   # does not start at 0
    assert L.crp_lens_create(2, 1, bad_rp.ctypes.data, cl.ctypes.data, vl.ctypes.data, None, C.byref(h)) == -1
    bad_cl = np.array([2], np.int32)                                         # column out of range
    assert L.crp_lens_create(2, 1, rp.ctypes.data, bad_cl.ctypes.data, vl.ctypes.data, None, C.byref(h)) == -1
    ed = np.array([2.0, 1.0])                                                # edges decrease
    assert L.crp_lens_create(2, 1, rp.ctypes.data, cl.ctypes.data, vl.ctypes.data, ed.ctypes.data, C.byref(h)) == -1
    assert L.crp_lens_apply(None, xs.ctypes.data, xs.ctypes.data, 1, None) == -1
    assert L.crp_lens_destroy(None) == -1
    assert L.crp_debug_fail_allocations(-1) == -1
    assert L.crp_debug_fail_allocations(0) == 0
    assert L.crp_selftest_wait(0, -1, None) == -1                            # limit < 1
    assert L.crp_sim_create(None, 0, None, 1, 10, C.byref(h)) == -1
    assert L.crp_tables_create(1, 1, 1, 6.0, 25.0, None, None, None, None, C.byref(h)) == -1
    assert L.crp_propagate(None, None, 1e-4, 1.0, 2.0, 3.0, None) == -1
    assert L.crp_sync(None, 0.0) == -1
    assert L.crp_field_destroy(None) == -1


def test_tables_reject_non_finite_rows(L):
    h = C.c_void_p()
    n_sp, nn = 4, 3
    ll = np.zeros((n_sp, nn))
    lp = np.zeros((n_sp, nn))
    hl = np.ones(n_sp, dtype=np.uint8)
    hp = np.zeros(n_sp, dtype=np.uint8)
    ll[2, 1] = np.inf
    rc = L.crp_tables_create(1, 1, nn, 6.0, 25.0, ll.ctypes.data, lp.ctypes.data, hl.ctypes.data,
                             hp.ctypes.data, C.byref(h))
    assert rc == -1


def test_no_cpu_fallback_without_device(L):
    """With no usable CUDA device a valid call reports a CUDA error instead of computing."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = C.c_void_p()
    org = (C.c_double * 3)(0, 0, 0)
    g = np.zeros((2, 2, 2, 3), dtype=np.float32)
    assert L.crp_field_create(g.ctypes.data, 1, 0, 2, 2, 2, 1.0, org, 1.0, C.byref(h)) == -3


def test_binding_raises_when_library_missing(monkeypatch, tmp_path):
    from paper_1410_5323_gb300 import api

    monkeypatch.setattr(api, "_lib", None)
    monkeypatch.setattr(api, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="missing"):
        api.lib()
