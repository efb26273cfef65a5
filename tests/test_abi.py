"""CPU-only checks of the C-ABI boundary: the library builds and loads, it
exports every entry point include/mips.h declares, argument errors come
back as status codes without touching a GPU, and the product path never
reaches the oracle."""
import ctypes
import os
import re

import pytest

from paper_1706_01449_gb300 import build, mips

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_entry_points():
    src = open(os.path.join(ROOT, "include", "mips.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mips_[a-z_0-9]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    lib = mips.load()
    names = declared_entry_points()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(mips.EXPORTS) == names


def test_version_and_defaults():
    lib = mips.load()
    assert lib.mips_version() >= 100
    opt = mips.Options()
    lib.mips_default_options(ctypes.byref(opt))
    assert opt.dtype == mips.DTYPES["bf16"] and opt.kmeans_iters == 3
    assert abs(opt.sample_frac - 0.005) < 1e-12
    assert opt.kmeans_spherical == 0


def test_argument_errors_need_no_gpu():
    lib = mips.load()
    h = ctypes.c_void_p()
    opt = mips.Options()
    lib.mips_default_options(ctypes.byref(opt))
    st = lib.mips_build_index(None, 10, 4, 2, ctypes.byref(opt), None, ctypes.byref(h))
    assert st == mips.MIPS_ERR_ARG and "null" in mips.last_error()
    fake = ctypes.c_void_p(16)
    assert lib.mips_build_index(fake, 10, 0, 2, ctypes.byref(opt), None, ctypes.byref(h)) == mips.MIPS_ERR_ARG
    assert lib.mips_build_index(fake, 10, 129, 2, ctypes.byref(opt), None, ctypes.byref(h)) == mips.MIPS_ERR_ARG
    assert lib.mips_build_index(fake, 0, 4, 2, ctypes.byref(opt), None, ctypes.byref(h)) == mips.MIPS_ERR_ARG
    assert lib.mips_build_index(fake, 10, 4, 0, ctypes.byref(opt), None, ctypes.byref(h)) == mips.MIPS_ERR_ARG
    for field, bad in (("kmeans_iters", 101), ("kmeans_iters", -1), ("block_items", -5), ("sample_frac", 0.0),
                       ("sample_frac", 1.5), ("sample_frac", float("nan")), ("kmeans_spherical", 2)):
        o2 = mips.Options()
        lib.mips_default_options(ctypes.byref(o2))
        setattr(o2, field, bad)
        assert lib.mips_build_index(fake, 10, 4, 2, ctypes.byref(o2), None, ctypes.byref(h)) == mips.MIPS_ERR_ARG, field
    o2 = mips.Options()
    lib.mips_default_options(ctypes.byref(o2))
    o2.dtype = 7  # not a mips_dtype
    assert lib.mips_build_index(fake, 10, 4, 2, ctypes.byref(o2), None, ctypes.byref(h)) == mips.MIPS_ERR_ARG
    assert lib.mips_build_index(fake, 10, 4, 4097, ctypes.byref(opt), None, ctypes.byref(h)) == mips.MIPS_ERR_ARG
    assert lib.mips_topk(None, fake, 4, 1, fake, fake, None) == mips.MIPS_ERR_ARG
    assert lib.mips_topk_maximus(None, fake, 4, 1, fake, fake, None) == mips.MIPS_ERR_ARG
    assert lib.mips_select(None, fake, 4, 1, fake, fake, None, None) == mips.MIPS_ERR_ARG
    assert lib.mips_sync(None, None) == mips.MIPS_ERR_ARG
    assert lib.mips_topk_graph(None, fake, 4, 1, 0, fake, fake, None) == mips.MIPS_ERR_ARG
    assert lib.mips_autotune(None, fake, 4, 1, None, None) == mips.MIPS_ERR_ARG
    assert lib.mips_fit_clusters(None, fake, 4, None) == mips.MIPS_ERR_ARG
    assert lib.mips_fit_clusters(None, None, 0, None) == mips.MIPS_ERR_ARG
    srv = ctypes.c_void_p()
    sopt = mips.ServerOptions(0, 2, 1024, 0)
    assert lib.mips_server_create(None, ctypes.byref(sopt), ctypes.byref(srv)) == mips.MIPS_ERR_ARG
    rid = ctypes.c_int64()
    assert lib.mips_server_submit(None, fake, 1, 1, fake, fake, ctypes.byref(rid)) == mips.MIPS_ERR_ARG
    assert lib.mips_server_wait(None, 0, 0.0, None) == mips.MIPS_ERR_ARG
    assert lib.mips_server_destroy(None) == mips.MIPS_OK
    lib.mips_free_index(None)


def test_product_path_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_1706_01449_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for fn in files:
            if fn.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, fn)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), fn
                assert "mips_oracle" not in text, fn


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(mips, "_lib", None)
    monkeypatch.setattr(mips, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(ImportError):
        mips.load()


def test_wait_expiry_hook_checks_its_limit():
    lib = mips.load()
    assert lib.mips_test_expire_next_wait(10) == mips.MIPS_ERR_ARG
    assert lib.mips_test_expire_next_wait(5_000_000_000) == mips.MIPS_ERR_ARG
