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


class _FakeDeviceTensor:
    """Stands in for a CUDA tensor in the placement check; its address is never used."""
    dtype = "torch.float64"
    is_cuda = True

    def __init__(self, n):
        self.n = n

    def data_ptr(self):
        return 16

    def is_contiguous(self):
        return True

    def numel(self):
        return self.n


def test_binding_refuses_wrong_sizes_types_and_placements_before_the_call():
    """The library reads and writes 5 n values behind each state pointer; the
    binding refuses anything else before it calls the library."""
    import numpy as np
    from paper_2208_01839_gb300 import inputs as I
    from paper_2208_01839_gb300 import seird as S
    xy, tri = I.structured_mesh(4)
    n = len(xy)
    with pytest.raises(ValueError, match="xy must be"):
        S.Solver(xy[:, :1], tri, I.params_square())
    with pytest.raises(ValueError, match="beta_field"):
        S.Solver(xy, tri, I.params_square(), beta_field=np.ones(n - 1))
    with pytest.raises(ValueError, match="owner"):
        S.Solver(xy, tri, I.params_square(), owner=np.zeros(n + 1, np.int32))
    sv = S.Solver.__new__(S.Solver)  # no context: whatever passes the checks reaches the library's NULL check
    sv.n, sv.n_samples, sv._h = n, 1, None
    u = np.ones((n, 5))
    with pytest.raises(ValueError, match="expected %d values, got %d" % (5 * n, 5 * n - 5)):
        sv.set_state(u[:-1])
    with pytest.raises(TypeError, match="float64"):
        sv.set_state(u.astype(np.float32))
    with pytest.raises(ValueError, match="C-contiguous"):
        sv.set_state(np.asfortranarray(u))
    with pytest.raises(ValueError, match="out"):
        sv.get_state(np.empty((n, 4)))
    with pytest.raises(ValueError, match="all be host arrays or all device tensors"):
        sv.residual(u, u, out=_FakeDeviceTensor(5 * n))
    with pytest.raises(ValueError, match="all be host arrays or all device tensors"):
        sv.linear_solve(_FakeDeviceTensor(5 * n), out=u.copy())
    with pytest.raises(ValueError, match="I_hat"):
        sv.adjoint(4, [0, 1], [2, 4], np.zeros((2, 3)), np.zeros((2, 2)))
    with pytest.raises(S.SeirdError) as e:  # well-formed arguments reach the library
        sv.set_state(u)
    assert e.value.code == -1
