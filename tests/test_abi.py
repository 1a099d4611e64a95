"""The C ABI loads, exports every symbol include/cosparse.h declares, and
rejects bad arguments on the host without touching a GPU."""
import ctypes
import os
import re

import pytest

import paper_1312_4746_gb300 as cs
from paper_1312_4746_gb300 import build as csbuild

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "cosparse.h")


@pytest.fixture(scope="module")
def L():
    csbuild.build()
    return cs.lib()


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(cs_[a-z0-9_]+)\s*\(", txt)))


def test_header_symbols_exported(L):
    names = _declared()
    assert len(names) >= 9
    for n in names:
        assert hasattr(L, n), f"{n} declared in cosparse.h but not exported"
    assert set(names) == set(cs.EXPORTS)


def test_version_and_defaults(L):
    assert "sm_103a" in cs.version()
    p = cs.Params.default()
    assert p.p == 7 and p.tau == 0.1 and p.sigma_c2 == 1.3 and p.alpha == 1.3
    assert p.d_min == 1.0 and p.kappa_beta == 1.0 and p.mode == 0 and p.precision == 0
    assert p.codes_form == cs.CODES_AUTO and p.l_tol == 1e-3 and p.iota_sigma == 0.01
    assert p.rho_variance == 0 and p.patch_order == 0
    assert ctypes.sizeof(cs.Params) == 4 * 4 + 7 * 8 + 2 * 4
    sp = cs.SegParams.default()
    assert ctypes.sizeof(cs.SegParams) == 3 * 8 + 2 * 4
    assert sp.lam == 1.0 and sp.nu == 0.0 and sp.gamma == 5.0 and sp.iterations == 300
    up = cs.UnsupParams.default()
    assert ctypes.sizeof(cs.UnsupParams) == 4 * 4 + 8
    assert (up.n_colour, up.n_texture, up.kmeans_iterations, up.kmedians_iterations,
            up.beta) == (4, 4, 10, 10, 1.0)


def test_null_ctx_rejected(L):
    p = cs.Params.default()
    assert L.cs_codes(None, None, 4, 4, None, 8, None, ctypes.byref(p), None, None, None,
                      None) == cs.CS_ERR_INVALID_ARG
    assert b"ctx" in L.cs_last_error(None)
    off = (ctypes.c_int32 * 3)(0, 1, 2)
    assert L.cs_likelihood(None, None, 4, 4, None, 8, 2, off, None, ctypes.byref(p), None, None,
                           None, None) == cs.CS_ERR_INVALID_ARG
    assert L.cs_cosupport(None, None, 4, 8, 0.1, None, None) == cs.CS_ERR_INVALID_ARG
    assert L.cs_sync_status(None, None) == cs.CS_ERR_INVALID_ARG
    init = (ctypes.c_int32 * 2)(0, 1)
    assert L.cs_kmeans(None, None, 4, 2, init, 1, None, None, None) == cs.CS_ERR_INVALID_ARG
    assert L.cs_kmedians(None, None, 4, 3, 2, init, 1, None, None, None) == cs.CS_ERR_INVALID_ARG
    up = cs.UnsupParams.default()
    assert L.cs_unsup_data_term(None, None, 4, 4, None, 8, None, ctypes.byref(p), ctypes.byref(up),
                                init, init, None, None, None, None, None,
                                None) == cs.CS_ERR_INVALID_ARG
    h = ctypes.c_void_p()
    assert L.cs_create(None, 0) == cs.CS_ERR_INVALID_ARG
    L.cs_destroy(None)  # no-op


def test_create_bad_device_no_gpu(L):
    h = ctypes.c_void_p()
    assert L.cs_create(ctypes.byref(h), 9999) == cs.CS_ERR_INVALID_ARG
    assert not h.value


def test_batch_null_args_no_gpu(L):
    p = cs.Params.default()
    b = ctypes.c_void_p()
    imgs = (cs.Image * 1)()
    assert L.cs_batch_create(None, imgs, 1, None, 8, None, ctypes.byref(p), 0,
                             ctypes.byref(b)) == cs.CS_ERR_INVALID_ARG
    assert b"ctx" in L.cs_last_error(None)
    assert L.cs_batch_run(None, None) == cs.CS_ERR_INVALID_ARG
    assert L.cs_batch_config(None, None, None, None, None, None, None) == cs.CS_ERR_INVALID_ARG
    assert L.cs_batch_set_config(None, 1, 0, 0) == cs.CS_ERR_INVALID_ARG
    assert L.cs_batch_data_term(None, imgs, 1, None, 8, None, ctypes.byref(p),
                                None) == cs.CS_ERR_INVALID_ARG
    L.cs_batch_destroy(None)  # no-op


def test_image_struct_layout():
    # cs_image: pointer, 4 x int32, then six pointers (64-bit ABI)
    assert ctypes.sizeof(cs.Image) == 8 + 16 + 6 * 8
    assert cs.Image.label_off.offset == 24


def test_surrogate_file_args_no_gpu(L, tmp_path):
    assert L.cs_surrogate_save(None, b"x") == cs.CS_ERR_INVALID_ARG
    assert L.cs_surrogate_load(None, str(tmp_path / "missing").encode()) == cs.CS_ERR_INVALID_ARG
    assert b"ctx" in L.cs_last_error(None)
