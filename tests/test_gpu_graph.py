"""GMRES restart cycles captured into CUDA graphs (options.graph = 1).

A captured cycle launches the same kernels with the same arguments as the
eager loop; only the convergence test of each iteration moves from the host
into the Givens kernel, which arms the next iteration's conditional node.  So:
  * states and Newton/GMRES iteration counts are bit for bit those of
    graph = 0 (FP64 and mixed; additive, multiplicative and hybrid two-grid;
    several restart cycles; a cycle cut short by the iteration limit);
  * the roots are the oracle's (<= 1e-9 relative L2 per compartment);
  * the kernel launch count is the eager loop's: iterations after convergence
    launch nothing;
  * divergence past dtol is reported as by the eager loop;
  * the adjoint, whose transposed solves run eagerly, gives the same gradient.
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


def rel_l2_per_comp(a, b):
    return [float(np.linalg.norm(a[:, c] - b[:, c]) / max(np.linalg.norm(b[:, c]), 1e-300)) for c in range(5)]


def _problem(seed=3, n_target=3000):
    xy, tri, _ = I.irregular_mesh(seed, n_target)
    dens = I.urban_density(seed)
    U0 = I.urban_ic(xy, dens, seed)
    p = I.params_ontario(float(U0.sum(axis=1).max()))
    atol = 1e-14 * np.linalg.norm(O.residual(xy, tri, p, 0.0, np.abs(U0), np.zeros_like(U0)))
    return xy, tri, p, U0, I.smooth_field(xy, seed), atol


def _solver(P, **kw):
    xy, tri, p, _, bf, atol = P
    opts = dict(dt=0.5, overlap=2, coarse=1, newton_rtol=1e-12, newton_atol=atol, gmres_rtol=1e-12,
                gmres_restart=30, gmres_maxit=2000, newton_maxit=100)
    opts.update(kw)
    return S.Solver(xy, tri, p, beta_field=bf, owner=I.box_partition(xy, 3, 2), **opts)


def _run(P, n_steps, **kw):
    with _solver(P, **kw) as sv:
        sv.set_state(P[3])
        l0 = S.launch_count()
        stats = sv.run(n_steps)
        launches = S.launch_count() - l0
        return sv.get_state(), [(s["newton_its"], s["gmres_its"]) for s in stats], launches


@pytest.mark.parametrize("precision,coarse,restart,one_pass", [(0, 1, 30, 1), (1, 2, 30, 1), (0, 2, 5, 0),
                                                               (0, 3, 8, 1), (1, 1, 4, 0)])
def test_captured_cycles_repeat_the_eager_loop(precision, coarse, restart, one_pass):
    P = _problem()
    kw = dict(precision=precision, coarse=coarse, gmres_restart=restart, gmres_one_pass=one_pass)
    U_e, its_e, l_e = _run(P, 3, graph=0, **kw)
    U_g, its_g, l_g = _run(P, 3, graph=1, **kw)
    assert its_g == its_e
    assert np.array_equal(U_g, U_e)
    assert l_g == l_e, (l_g, l_e)
    if restart < 30:  # the case exercises restarts
        assert max(g for _, g in its_e) > restart


def test_captured_cycles_reach_the_oracle_roots():
    P = _problem(seed=5, n_target=2500)
    xy, tri, p, U0, bf, atol = P
    U_ref, _ = O.run(xy, tri, p, 0.5, U0, 3, rtol=1e-12, atol=atol, bfield=bf)
    U_g, _, _ = _run(P, 3, graph=1, coarse=2)
    assert max(rel_l2_per_comp(U_g, U_ref)) <= 1e-9, rel_l2_per_comp(U_g, U_ref)


def test_cycle_cut_short_by_the_iteration_limit():
    """gmres_maxit = 7 with restart 5: a full cycle, then a cycle of two iterations."""
    P = _problem(seed=4, n_target=1500)
    out = {}
    for graph in (0, 1):
        with _solver(P, graph=graph, gmres_restart=5, gmres_maxit=7) as sv:
            U = P[3] * 1.01
            sv.jacobian(U)
            sv.precond_setup()
            b = np.random.default_rng(0).standard_normal(U.shape)
            x = np.empty_like(b)
            with pytest.raises(S.SeirdError):  # the limit is reached, x is the iterate there
                sv.linear_solve(b, out=x)
            out[graph] = x
    assert np.array_equal(out[0], out[1])
    assert np.all(np.isfinite(out[1])) and np.abs(out[1]).max() > 0


def test_divergence_is_reported():
    """A dtol far below 1 is crossed at the first iteration (the estimate starts at ||b||)."""
    P = _problem(seed=4, n_target=1500)
    for graph in (0, 1):
        with _solver(P, graph=graph, gmres_dtol=1e-8) as sv:
            sv.set_state(P[3])
            with pytest.raises(S.SeirdError, match="dtol"):
                sv.step()


def test_adjoint_with_captured_forward_cycles():
    from oracle import seird_adjoint as A
    P = _problem(seed=4, n_target=220)
    xy, tri, p, U0, bf, _ = P
    rng = np.random.default_rng(4)
    nodes = np.sort(rng.choice(len(xy), 12, replace=False))
    steps = [2, 4]
    S_obs = A.forward_states(xy, tri, p, 0.5, U0, 4, bfield=bf)
    Ih = np.array([S_obs[s][nodes, 2] * 1.1 for s in steps])
    Dh = np.array([S_obs[s][nodes, 4] * 0.9 for s in steps])
    res = {}
    for graph in (0, 1):
        with _solver(P, graph=graph, overlap=1, gmres_restart=40, gmres_maxit=3000, newton_rtol=1e-13) as sv:
            sv.set_state(U0)
            res[graph] = sv.adjoint(4, nodes, steps, Ih, Dh, lin_rtol=1e-12)
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])
