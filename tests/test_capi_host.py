"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every function include/seird.h declares; argument validation happens
before any device call."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_01839_gb300 import build
    path = build.build()
    return C.CDLL(path)


def declared():
    txt = open(os.path.join(ROOT, "include", "seird.h")).read()
    return sorted(set(re.findall(r"\b(seird_[a-z0-9_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert "seird_create" in names and "seird_step" in names and "seird_run" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2208_01839_gb300 import seird as S
    for n in declared():
        assert hasattr(S._lib, n)


def test_default_options_match_the_paper_gmres_settings():
    from paper_2208_01839_gb300 import seird as S
    o = S.default_options()
    # Section 3.2: rtol 1e-5, atol 1e-50, dtol 1e5, at most 200 outer iterations
    assert o.gmres_rtol == 1e-5 and o.gmres_atol == 1e-50 and o.gmres_dtol == 1e5 and o.gmres_maxit == 200
    assert o.gmres_restart == 30 and o.quadrature == 0 and o.precision == 0


def test_null_arguments_are_rejected_without_a_device(lib):
    from paper_2208_01839_gb300 import seird as S
    h = C.c_void_p()
    rc = S._create(None, None, None, C.byref(h))
    assert rc == -1 and not h.value
    assert b"NULL" in S._last_error(None)
    assert S._bsr_spmv(-1, None, None, None, None, None, None) == -1
    assert S._bsr_spmv(0, None, None, None, None, None, None) == 0
    assert S._bsr_spmv(3, None, None, None, None, None, None) == -1


def test_bad_meshes_are_rejected_before_any_device_call():
    import numpy as np
    from paper_2208_01839_gb300 import inputs as I
    from paper_2208_01839_gb300 import seird as S
    xy, tri = I.structured_mesh(4)
    cw = tri[:, ::-1].copy()
    with pytest.raises(S.SeirdError) as e:
        S.Solver(xy, cw, I.params_square())
    assert e.value.code == -1 and "counter-clockwise" in str(e.value)
    bad = tri.copy()
    bad[0, 0] = 99
    with pytest.raises(S.SeirdError) as e:
        S.Solver(xy, bad, I.params_square())
    assert "out of range" in str(e.value)
    owner = np.zeros(len(xy), dtype=np.int32)
    owner[0] = 2  # part 1 empty
    with pytest.raises(S.SeirdError) as e:
        S.Solver(xy, tri, I.params_square(), owner=owner)
    assert "owns no node" in str(e.value)
