"""The paper's variants on the GPU against the oracle's restatements.

* Picard matrix of Eq. weak_vec_implicit (options.nonlinear = 1): block by
  block against the oracle's matrix built from B(u) as printed, within the
  assembly tolerance of the parity tests (1e-12 of the largest entry).
* Picard steps reach the backward-Euler root the Newton oracle computes
  (<= 1e-9 relative L2 per compartment, FP64 and mixed), and with the paper's
  stopping rule on eps (Eq. picardtol) they take the oracle Picard iteration's
  number of iterations and end at its iterate.
* Sigmoid transmission (Eq. beta_ie, Eq. beta_x) across the schedule's midpoint
  against the oracle run with beta(t^{n+1}) and the nodal beta(x).
"""
import numpy as np
import pytest

from oracle import seird_oracle as O
from oracle import seird_variants as V
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


def _irregular(seed=3, n_target=3000, alpha=0.0, mu=0.0):
    xy, tri, _ = I.irregular_mesh(seed, n_target)
    dens = I.urban_density(seed)
    U0 = I.urban_ic(xy, dens, seed)
    p = I.params_ontario(float(U0.sum(axis=1).max()))
    p.alpha, p.mu = alpha, mu
    return xy, tri, p, U0, I.smooth_field(xy, seed)


def _floor(xy, tri, p, U0):
    return 1e-14 * np.linalg.norm(O.residual(xy, tri, p, 0.0, np.abs(U0), np.zeros_like(U0)))


def _solver(xy, tri, p, bf, dt, **kw):
    opts = dict(dt=dt, overlap=2, coarse=1, newton_rtol=1e-12, gmres_rtol=1e-12, gmres_restart=30,
                gmres_maxit=2000, newton_maxit=200)
    opts.update(kw)
    return S.Solver(xy, tri, p, beta_field=bf, owner=I.box_partition(xy, 3, 2), **opts)


@pytest.mark.parametrize("rule", [0, 1])
def test_picard_matrix_matches_oracle(rule):
    xy, tri, p, U0, bf = _irregular(alpha=0.01, mu=0.002)
    rng = np.random.default_rng(4)
    U = U0 * (1.0 + 0.05 * rng.standard_normal(U0.shape)) + 1.0
    P = V.picard_matrix(xy, tri, p, 0.5, U, bfield=bf, rule="deg5" if rule == 0 else "vertex")
    rp, col, val = O.to_bsr(P)
    with _solver(xy, tri, p, bf, 0.5, nonlinear=1, quadrature=rule) as sv:
        sv.jacobian(U)
        grp, gcol, gval = sv.get_jacobian()
        x = rng.standard_normal(U.shape)
        y = sv.apply_jacobian(x)
    # the BSR pattern is the mesh's node graph (every block carries mass entries)
    assert np.array_equal(grp, rp) and np.array_equal(gcol, col)
    assert np.abs(gval - val).max() <= 1e-12 * np.abs(val).max()
    ref = (P @ x.ravel()).reshape(U.shape)
    assert np.all(np.abs(y - ref).ravel() <= 1e-12 * (abs(P) @ np.abs(x).ravel()) + 1e-300)


@pytest.mark.parametrize("precision", [0, 1])
def test_picard_steps_reach_the_newton_root(precision):
    xy, tri, p, U0, bf = _irregular()
    atol = _floor(xy, tri, p, U0)
    U_ref, _ = O.run(xy, tri, p, 0.5, U0, 3, rtol=1e-12, atol=atol, bfield=bf)
    with _solver(xy, tri, p, bf, 0.5, nonlinear=1, precision=precision, newton_atol=atol) as sv:
        sv.set_state(U0)
        stats = [sv.step() for _ in range(3)]
        got = sv.get_state()
    assert max(rel_l2_per_comp(got, U_ref)) <= 1e-9, (rel_l2_per_comp(got, U_ref), stats)


def test_picard_eps_rule_follows_the_oracle_iteration():
    wl = I.square_workload(17, N0=2000.0)
    Uo, io = V.picard_step(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, eps_tol=1e-8)
    with S.Solver(wl.xy, wl.tri, wl.params, owner=wl.owner, dt=wl.dt, overlap=1, coarse=1, nonlinear=1,
                  picard_tol=1e-8, gmres_rtol=1e-13, gmres_maxit=2000, newton_maxit=200) as sv:
        sv.set_state(wl.U0)
        st = sv.step()
        got = sv.get_state()
    assert st["newton_its"] == io["its"], (st, io["its"])
    assert abs(st["eps_update"] - io["eps"][-1]) <= 1e-6 * io["eps"][-1]
    assert max(rel_l2_per_comp(got, Uo)) <= 1e-9


def test_beta_schedule_across_its_midpoint():
    xy, tri, p, U0, _ = _irregular(seed=5, n_target=2500)
    nmax = float(U0.sum(axis=1).max())
    sched = dict(b0=0.101, b1=0.05, t_mid=130.0, beta_central=7.5 / nmax, beta_eastern=9.0 / nmax,
                 beta_western=5.0 / nmax, x_eastern=0.65, x_western=0.35, k_eastern=25.0, k_western=50.0)
    dt, t0, n = 0.5, 128.0, 8
    atol = _floor(xy, tri, p, U0)
    U_ref = V.schedule_run(xy, tri, p, dt, U0, t0, n, sched, rtol=1e-12, atol=atol)
    with _solver(xy, tri, p, None, dt, newton_atol=atol) as sv:
        sv.set_beta_schedule(sched)
        sv.set_state(U0, t=t0)
        sv.run(n)
        got = sv.get_state()
        # the adjoint takes constant rates only
        with pytest.raises(S.SeirdError):
            sv.adjoint(2, [0], [1], np.zeros((1, 1)), np.zeros((1, 1)))
        # schedule off: the params' constant rates again
        sv.set_beta_schedule(None)
        sv.set_state(U0, t=t0)
        sv.step()
        got_off = sv.get_state()
    assert max(rel_l2_per_comp(got, U_ref)) <= 1e-9, rel_l2_per_comp(got, U_ref)
    U_off, _ = O.newton_step(xy, tri, p, dt, U0, rtol=1e-12, atol=atol)
    assert max(rel_l2_per_comp(got_off, U_off)) <= 1e-9
