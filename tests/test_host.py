"""CPU-side checks: the library builds, loads and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*TG_API\s+(?:const\s+)?[a-z_0-9]+\s*\*?\s*(tg_[a-z_0-9]+)\s*\(", src, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2402_14415_gb300.builder import build
    path = build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["tg_create", "tg_destroy", "tg_query", "tg_query_backward", "tg_adam_step", "tg_locate",
                 "tg_batch_bin", "tg_query_binned", "tg_query_backward_binned"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2402_14415_gb300 import binding
    assert set(binding.exported_symbols()) <= set(declared_functions())


def test_status_strings(lib):
    lib.tg_status_string.restype = ctypes.c_char_p
    assert lib.tg_status_string(0) == b"TG_OK"
    assert lib.tg_status_string(3) == b"TG_EBUDGET"


def test_invalid_arguments_are_rejected_without_a_gpu(lib):
    """Argument checks run on the host before any device call."""
    h = ctypes.c_void_p()
    lib.tg_create.argtypes = [ctypes.c_int] * 5 + [ctypes.c_uint64, ctypes.c_float, ctypes.POINTER(ctypes.c_void_p)]
    assert lib.tg_create(4, 8, 2, 1, 0, 0, 0.0, ctypes.byref(h)) == 1      # dim
    assert lib.tg_create(3, 8, 3, 1, 0, 0, 0.0, ctypes.byref(h)) == 1      # order
    assert lib.tg_create(3, 1, 2, 1, 0, 0, 0.0, ctypes.byref(h)) == 1      # res
    assert lib.tg_create(3, 8, 2, 5, 0, 0, 0.0, ctypes.byref(h)) == 1      # channels
    assert lib.tg_create(3, 8, 2, 1, 7, 0, 0.0, ctypes.byref(h)) == 1      # dtype
    lib.tg_query.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                             ctypes.c_void_p]
    assert lib.tg_query(None, None, 0, None, None, None) == 1
    for fn in ("tg_batch_gather", "tg_batch_scatter"):
        f = getattr(lib, fn)
        f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        assert f(None, None, 1, None, None) == 1
    lib.tg_cancel.argtypes = [ctypes.c_void_p, ctypes.c_int64]
    assert lib.tg_cancel(None, 1) == 1
    for fn, args in (("tg_extract_mesh", [ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_void_p,
                                          ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p]),):
        f = getattr(lib, fn)
        f.argtypes = args
        assert f(None, 16, 0.0, None, 0, None, None) == 1
    lib.tg_chamfer.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                               ctypes.c_void_p]
    assert lib.tg_chamfer(None, 1, None, 1, None, None) == 1
    lib.tg_measure_fp32_peak.argtypes = [ctypes.c_void_p]
    assert lib.tg_measure_fp32_peak(None) == 1


def test_fit_job_descriptions_are_checked_on_the_host(lib):
    """The server and its submission queue are host objects: bad descriptions, unknown flags and jobs that can
    never fit the budget are refused at submission, before anything touches the device."""
    from paper_2402_14415_gb300.binding import FitDesc
    s = ctypes.c_void_p()
    lib.tg_server_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
    lib.tg_server_destroy.argtypes = [ctypes.c_void_p]
    lib.tg_fit_job.argtypes = [ctypes.c_void_p, ctypes.POINTER(FitDesc), ctypes.POINTER(ctypes.c_int64)]
    assert lib.tg_server_create(0, 1, ctypes.byref(s)) == 1          # empty budget
    assert lib.tg_server_create(1 << 30, 0, ctypes.byref(s)) == 1    # no running slot
    assert lib.tg_server_create(1 << 30, 4, ctypes.byref(s)) == 0
    sph = (ctypes.c_float * 4)(0.5, 0.5, 0.5, 0.3)
    cdf = (ctypes.c_float * 1)(1.0)
    jid = ctypes.c_int64(-1)

    def desc(**kw):
        d = FitDesc(res=64, order=2, dtype=0, seed=0, n_spheres=1, n_boxes=0,
                    spheres=ctypes.cast(sph, ctypes.c_void_p), boxes=None, area_cdf=ctypes.cast(cdf, ctypes.c_void_p),
                    points_per_step=1 << 16, eval_points=1 << 14, eval_every=10, max_steps=100, tol=0.0, lr=1e-2,
                    lambda_eik=0.1, init_std=0.0, k_weight=0.0, lambda_tv=0.0, flags=0)
        for k, v in kw.items():
            setattr(d, k, v)
        return d

    try:
        assert lib.tg_fit_job(s, None, ctypes.byref(jid)) == 1
        assert lib.tg_fit_job(s, ctypes.byref(desc(flags=4)), ctypes.byref(jid)) == 1     # unknown flag bit
        assert lib.tg_fit_job(s, ctypes.byref(desc(dtype=7)), ctypes.byref(jid)) == 1
        assert lib.tg_fit_job(s, ctypes.byref(desc(order=3)), ctypes.byref(jid)) == 1
        assert lib.tg_fit_job(s, ctypes.byref(desc(res=1)), ctypes.byref(jid)) == 1
        assert lib.tg_fit_job(s, ctypes.byref(desc(area_cdf=None)), ctypes.byref(jid)) == 1
        assert lib.tg_fit_job(s, ctypes.byref(desc(n_spheres=0)), ctypes.byref(jid)) == 1  # no surface to sample
        # 1024^3 order 2 in FP32: 10.7 G coefficients x 16 bytes, far over the 1 GiB budget
        assert lib.tg_fit_job(s, ctypes.byref(desc(res=1024)), ctypes.byref(jid)) == 3
        assert jid.value == -1                                                             # nothing was queued
    finally:
        assert lib.tg_server_destroy(s) == 0


def test_product_path_has_no_oracle_reference():
    """The package and the CUDA sources never import or link the oracle."""
    pkg = os.path.join(ROOT, "paper_2402_14415_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt and "tg_oracle" not in txt, f


def test_binding_has_no_cpu_path(lib, monkeypatch):
    """A host tensor is refused before any library call, and without the built library every call raises:
    there is no CPU fallback behind the binding."""
    import torch
    from paper_2402_14415_gb300 import binding
    with pytest.raises(ValueError, match="no CPU path"):
        binding.tg_locate(3, 8, torch.rand((10, 3)))
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding, "LIB_PATH", os.path.join(ROOT, "paper_2402_14415_gb300", "_build", "absent.so"))
    with pytest.raises(ImportError):
        binding.tg_locate(3, 8, torch.rand((10, 3)))
