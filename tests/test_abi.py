"""The C-ABI library loads and exports every symbol include/momenti.h
declares; argument checks that need no GPU."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def mom():
    from paper_2502_14446_gb300 import build_ext
    build_ext.build()
    from paper_2502_14446_gb300 import momenti
    return momenti


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "momenti.h")).read()
    return sorted(set(re.findall(r"\b(momenti_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("momenti_create", "momenti_hash_all", "momenti_verify", "momenti_topk"):
        assert name in syms


def test_library_exports_every_declared_symbol(mom):
    for name in declared_symbols():
        assert hasattr(mom.lib, name), name
    assert sorted(mom.EXPORTS) == declared_symbols()


def test_struct_layouts(mom):
    assert C.sizeof(mom.momenti_motif) == 48
    assert C.sizeof(mom.momenti_params) == 80


def test_default_params_are_the_papers(mom):
    p = mom.default_params()
    assert (p.K, p.L, p.delta, p.r) == (8, 200, 0.01, 0.0)
    assert p.excl == -1


@pytest.mark.parametrize("bad", [dict(w=1), dict(d=0), dict(k=0), dict(delta=0.0),
                                 dict(delta=1.0), dict(K=9), dict(K=0), dict(L=-1),
                                 dict(precision=7), dict(delta_mode=3),
                                 dict(K=7, flags=4)])           # tensoring needs an even K
def test_create_rejects_bad_parameters(mom, bad):
    p = mom.default_params(**bad)
    h = C.c_void_p()
    assert mom.lib.momenti_create(C.byref(h), C.byref(p)) == mom.ERR_ARG


def test_calls_out_of_order(mom):
    p = mom.default_params(w=10, d=1, k=1)
    h = C.c_void_p()
    assert mom.lib.momenti_create(C.byref(h), C.byref(p)) == mom.OK
    out = (mom.momenti_motif * 1)()
    n = C.c_int32()
    assert mom.lib.momenti_topk(h, out, C.byref(n), None) == mom.ERR_STATE
    assert mom.lib.momenti_verify(h, None, 0, None, None, None, 0) == mom.ERR_STATE
    assert mom.lib.momenti_set_hash_params(h, 1, 1, 8, 11, None, None) == mom.ERR_ARG
    assert b"set_hash_params" in mom.lib.momenti_last_error(h)
    assert mom.lib.momenti_hash_all(h, None, 0, 100, 1, 100, 0, None) == mom.ERR_ARG
    mom.lib.momenti_destroy(h)
    mom.lib.momenti_destroy(None)


def test_window_limit_of_the_index_sort(mom):
    # at most 65535 * 2048 windows: the sort's tiles of 2048 windows sit on
    # the grid's y dimension; the check precedes any read of the series or
    # any device call
    w = 10
    p = mom.default_params(w=w, d=1, k=1)
    h = C.c_void_p()
    assert mom.lib.momenti_create(C.byref(h), C.byref(p)) == mom.OK
    dummy = (C.c_float * 4)()
    n = 65535 * 2048 + w - 1          # exactly 65535 * 2048 windows
    assert mom.lib.momenti_hash_all(h, dummy, mom.F32, n, 1, n, 0, None) == mom.ERR_ARG
    assert b"too many windows" in mom.lib.momenti_last_error(h)
    mom.lib.momenti_destroy(h)


def test_header_names_every_timed_kernel():
    # momenti_time_kernel documents the names it accepts: exactly the
    # names the sources pass to the launch accounting
    csrc = os.path.join(ROOT, "paper_2502_14446_gb300", "csrc")
    used = set()
    for fn in os.listdir(csrc):
        if fn.endswith(".cu") or fn.endswith(".cuh"):
            used |= set(re.findall(r'MOMENTI_LAUNCH\("([a-z0-9_]+)"', open(os.path.join(csrc, fn)).read()))
    text = open(os.path.join(ROOT, "include", "momenti.h")).read()
    block = re.search(r"Kernel names:(.*?)\*/", text, re.S).group(1)
    listed = set(re.findall(r"[a-z0-9_]+", block.replace("*", " ")))
    assert used and listed == used


def test_plain_c_client(mom, tmp_path):
    # the header is C99 and the library links and answers from a C program
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pkg = os.path.dirname(mom.LIB_PATH)
    exe = str(tmp_path / "c_client")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
                    os.path.join(ROOT, "tests", "c_client.c"), "-I", os.path.join(ROOT, "include"),
                    "-L", pkg, "-lmomenti", f"-Wl,-rpath,{pkg}", "-lm", "-o", exe],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "FAIL" not in r.stdout and r.stdout.count("ok ") == 9


def test_binding_fails_loudly_without_the_library(tmp_path):
    # no CPU fallback: a copy of the binding next to no libmomenti.so
    # refuses to import
    import shutil
    import subprocess
    import sys
    pkg = tmp_path / "nolib"
    pkg.mkdir()
    shutil.copy(os.path.join(ROOT, "paper_2502_14446_gb300", "momenti.py"), pkg / "momenti.py")
    r = subprocess.run([sys.executable, "-c", "import momenti"], cwd=str(pkg),
                       capture_output=True, text=True, timeout=120)
    assert r.returncode != 0
    assert "ImportError" in r.stderr and "libmomenti.so is missing" in r.stderr


def test_topk_batch_argument_errors(mom):
    P = C.POINTER
    one = (mom.momenti_params * 1)(mom.default_params(w=10, d=1, k=3))
    series = (C.c_void_p * 1)(None)
    dtype, n, D = (C.c_int32 * 1)(0), (C.c_int64 * 1)(100), (C.c_int32 * 1)(1)
    out = (mom.momenti_motif * 3)()
    n_out, rc = (C.c_int32 * 1)(), (C.c_int32 * 1)()
    call = mom.lib.momenti_topk_batch
    assert call(-1, one, series, dtype, n, D, 0, 1, out, 3, n_out, None, rc, None, 0) == mom.ERR_ARG
    assert call(0, None, None, None, None, None, 0, 1, None, 0, None, None, None, None, 0) == mom.OK
    assert call(1, None, series, dtype, n, D, 0, 1, out, 3, n_out, None, rc, None, 0) == mom.ERR_ARG
    # k = 3 motifs do not fit an output stride of 2
    assert call(1, one, series, dtype, n, D, 0, 1, out, 2, n_out, None, rc, None, 0) == mom.ERR_ARG


def test_no_device_is_an_error_not_a_fallback(mom):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    x = np.arange(200, dtype=np.float32)
    one = (mom.momenti_params * 1)(mom.default_params(w=10, d=1, k=1))
    series = (C.c_void_p * 1)(x.ctypes.data)
    dtype, n, D = (C.c_int32 * 1)(0), (C.c_int64 * 1)(200), (C.c_int32 * 1)(1)
    out = (mom.momenti_motif * 1)()
    n_out, rc = (C.c_int32 * 1)(), (C.c_int32 * 1)()
    r = mom.lib.momenti_topk_batch(1, one, series, dtype, n, D, 0, 1, out, 1, n_out, None, rc,
                                   None, 0)
    assert r == mom.ERR_CUDA
    with mom.Momenti(w=10, d=1, k=1, delta=0.1) as h:
        with pytest.raises(mom.MomentiError):
            h.hash_all(x.reshape(1, -1))
