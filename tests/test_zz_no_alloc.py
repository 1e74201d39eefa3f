"""The allocation-free residual entry point (seird_residual_noalloc).

Some callers cannot call cudaMalloc: a framework that owns all device memory
through its own arena, or a loop that must never allocate.  They cannot create
a context (creating one allocates), so the library gives them one entry point
that evaluates the residual F(u; u_prev) on a mesh held in their own device
memory and keeps its scratch in a fixed device array.  These tests call it
through the C ABI, for both quadrature rules, and compare it with the
context-based seird_eval_residual and with the CPU oracle, within the residual
tolerance of the parity tests, on two calls in a row (the second call reuses
the scratch the first one left behind); one call runs on a side stream, and a
state with N <= 0 returns SEIRD_ENONFINITE without spoiling the next call.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import numpy as np
import pytest

from oracle import seird_oracle as O
from paper_2208_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2208_01839_gb300 import build as _b  # noqa: E402

_b.build()
from paper_2208_01839_gb300 import seird as S  # noqa: E402


def incidence(n, tri):
    """Node -> (3*t + a) entries, grouped by node, ascending t within a node."""
    flat = tri.ravel().astype(np.int64)
    order = np.argsort(flat, kind="stable")  # stable: ascending 3t+a inside each node
    ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(ptr, flat + 1, 1)
    return np.cumsum(ptr).astype(np.int32), order.astype(np.int32)


def scale(xy, tri, params, U, dt):
    """Magnitude of the terms each residual entry sums (as in the parity tests)."""
    m = O.residual(xy, tri, params, 0.0, np.abs(U), np.zeros_like(U))
    return np.abs(m).max() * (1.0 + dt)


def _cases():
    sq = I.square_workload(33)
    xy, tri, _ = I.irregular_mesh(3, 3000)
    dens = I.urban_density(3)
    U0 = I.urban_ic(xy, dens, 3)
    p = I.params_ontario(float(U0.sum(axis=1).max()))
    return [("square33", sq.xy, sq.tri, sq.params, sq.U0, 1.0, None),
            ("irregular3k", xy, tri, p, U0, 0.5, I.smooth_field(xy, 3))]


@pytest.mark.parametrize("quadrature", [0, 1], ids=["deg5", "vertex"])
@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_noalloc_residual_matches_context_and_oracle_on_two_calls(case, quadrature):
    name, xy, tri, params, U0, dt, bf = case
    rule = "deg5" if quadrature == 0 else "vertex"
    rng = np.random.default_rng(11)
    U1 = U0 * (1.0 + 0.05 * rng.standard_normal(U0.shape)) + 1.0
    U2 = U1 * (1.0 + 0.05 * rng.standard_normal(U0.shape)) + 0.5
    with S.Solver(xy, tri, params, beta_field=bf, dt=dt, n_subdomains=3, quadrature=quadrature) as sv:
        ref1 = sv.residual(U1, U0)
        ref2 = sv.residual(U2, U1)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    ptr, inc = incidence(len(xy), tri)
    xy_d, tri_d, ptr_d, inc_d = d(xy), d(tri.astype(np.int32)), d(ptr), d(inc)
    bf_d = None if bf is None else d(bf)
    F = torch.full((len(xy), 5), np.nan, dtype=torch.float64, device="cuda")
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    for U, Up, ref in ((U1, U0, ref1), (U2, U1, ref2)):
        S.residual_noalloc(xy_d, tri_d, ptr_d, inc_d, params, d(U), d(Up), F, dt, quadrature=quadrature,
                           beta_field=bf_d, norm2=nrm)
        got = F.cpu().numpy()
        tol = 1e-12 * scale(xy, tri, params, U, dt)
        assert np.abs(got - ref).max() <= tol, name
        orc = O.residual(xy, tri, params, dt, U, Up, bf, rule)
        assert np.abs(got - orc).max() <= tol, name
        assert abs(nrm.item() - float((ref ** 2).sum())) <= 1e-10 * float((ref ** 2).sum())
    # without a norm output the call still fills F
    S.residual_noalloc(xy_d, tri_d, ptr_d, inc_d, params, d(U1), d(U0), F, dt, quadrature=quadrature,
                       beta_field=bf_d)
    assert np.abs(F.cpu().numpy() - ref1).max() <= 1e-12 * scale(xy, tri, params, U1, dt)


def test_noalloc_on_a_side_stream_and_after_a_nonpositive_density():
    """Inputs written on a non-blocking side stream and the call made on that
    stream; then a state whose density vanishes on a patch of triangles gives
    SEIRD_ENONFINITE (1/N undefined), and the next call with a valid state
    succeeds and matches the oracle again (the error word starts at zero on
    every call)."""
    name, xy, tri, params, U0, dt, bf = _cases()[1]
    U1 = U0 * 1.02 + 0.5
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    ptr, inc = incidence(len(xy), tri)
    tol = 1e-12 * scale(xy, tri, params, U1, dt)
    ref = O.residual(xy, tri, params, dt, U1, U0, bf)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        xy_d, tri_d, ptr_d, inc_d = d(xy), d(tri.astype(np.int32)), d(ptr), d(inc)
        bf_d, u_d, up_d = d(bf), d(U1), d(U0)
        F = torch.full((len(xy), 5), np.nan, dtype=torch.float64, device="cuda")
        S.residual_noalloc(xy_d, tri_d, ptr_d, inc_d, params, u_d, up_d, F, dt, beta_field=bf_d, stream=side)
    side.synchronize()
    assert np.abs(F.cpu().numpy() - ref).max() <= tol
    # host-prepared bad state: every compartment zero on the nodes of a few triangles
    bad = U1.copy()
    bad[np.unique(tri[:40])] = 0.0
    with pytest.raises(S.SeirdError) as ei:
        S.residual_noalloc(xy_d, tri_d, ptr_d, inc_d, params, d(bad), up_d, F, dt, beta_field=bf_d)
    assert ei.value.code == -7
    S.residual_noalloc(xy_d, tri_d, ptr_d, inc_d, params, u_d, up_d, F, dt, beta_field=bf_d)
    assert np.abs(F.cpu().numpy() - ref).max() <= tol


def test_noalloc_rejects_meshes_beyond_its_scratch():
    xy, tri = I.structured_mesh(4)
    d = lambda a: torch.tensor(np.ascontiguousarray(a), device="cuda")
    ptr, inc = incidence(len(xy), tri)
    args = [d(xy), d(tri.astype(np.int32)), d(ptr), d(inc)]
    p = S.params_struct(I.params_square())
    u = d(np.ones((len(xy), 5)))
    F = torch.empty_like(u)
    import ctypes as C
    rc = S._residual_noalloc(S.NOALLOC_MAX_NODES, S.NOALLOC_MAX_TRIS + 1, *(a.data_ptr() for a in args), C.byref(p),
                             None, 1.0, 0, u.data_ptr(), u.data_ptr(), F.data_ptr(), None, None)
    assert rc == -1
    assert b"at most 65536 triangles" in S._last_error(None)
