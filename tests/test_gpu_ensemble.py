"""Ensembles (seird_create_ensemble): independent samples on one mesh, with
their own rates, solved as one block-diagonal system.

* The residual and the Jacobian of the ensemble are, sample by sample, the
  oracle's residual and Jacobian at that sample's rates (assembly tolerance
  1e-12 of the summed terms), and no block couples two samples.
* Steps: every sample's state is the oracle root at its rates (<= 1e-9
  relative L2 per compartment, FP64 and mixed).
* An ensemble of one sample reproduces the single-problem context bit for bit.
* With options.graph (GMRES cycles replayed as captured CUDA graphs) the
  ensemble's states equal the eager loop's bit for bit.
* Rates of an ensemble are fixed: set_params and the beta schedule are refused.
* The ensemble adjoint gives every sample's gradient: sample by sample it is the
  oracle's adjoint at that sample's rates and observations (1e-7 of the largest
  scaled component, as the single-context adjoint test).
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


def _problem(n_samples=4, seed=6, n_target=1500):
    xy, tri, _ = I.irregular_mesh(seed, n_target)
    dens = I.urban_density(seed)
    U0 = I.urban_ic(xy, dens, seed)
    base = I.params_ontario(float(U0.sum(axis=1).max()))
    samples = I.rate_samples(base, n_samples, seed)
    return xy, tri, samples, U0, I.smooth_field(xy, seed)


def _opts(**kw):
    o = dict(dt=0.5, overlap=2, coarse=1, newton_rtol=1e-12, gmres_rtol=1e-12, gmres_restart=30, gmres_maxit=2000)
    o.update(kw)
    return o


def test_ensemble_assembly_is_blockwise_the_oracle():
    xy, tri, samples, U0, bf = _problem()
    n, B = len(xy), len(samples)
    rng = np.random.default_rng(1)
    U = np.concatenate([U0 * (1.0 + 0.05 * rng.standard_normal(U0.shape)) + 1.0 for _ in range(B)])
    Un = np.concatenate([U0] * B)
    with S.Solver(xy, tri, samples, beta_field=bf, owner=I.box_partition(xy, 2, 2), **_opts()) as sv:
        F = sv.residual(U, Un)
        sv.jacobian(U)
        rp, col, val = sv.get_jacobian()
    for k, p in enumerate(samples):
        sl = slice(k * n, (k + 1) * n)
        ref = O.residual(xy, tri, p, 0.5, U[sl], Un[sl], bfield=bf)
        scale = np.abs(O.residual(xy, tri, p, 0.0, np.abs(U[sl]), np.zeros_like(U0))).max() * 1.5
        assert np.abs(F[sl] - ref).max() <= 1e-12 * scale, k
        J = O.jacobian(xy, tri, p, 0.5, U[sl], bfield=bf)
        jrp, jcol, jval = O.to_bsr(J)
        a, b = rp[k * n], rp[(k + 1) * n]
        assert np.array_equal(rp[k * n:(k + 1) * n + 1] - a, jrp)
        assert np.array_equal(col[a:b] - k * n, jcol)  # no block leaves the sample
        assert np.abs(val[a:b] - jval).max() <= 1e-12 * np.abs(jval).max(), k


@pytest.mark.parametrize("precision,fill", [(0, 0), (1, 0), (0, 1)])
def test_ensemble_steps_match_per_sample_oracle(precision, fill):
    xy, tri, samples, U0, bf = _problem()
    n = len(xy)
    atol = 1e-14 * np.linalg.norm(O.residual(xy, tri, samples[0], 0.0, np.abs(U0), np.zeros_like(U0)))
    with S.Solver(xy, tri, samples, beta_field=bf, owner=I.box_partition(xy, 2, 2),
                  **_opts(precision=precision, newton_atol=atol * np.sqrt(len(samples)), ilu_fill=fill)) as sv:
        sv.set_state(np.concatenate([U0] * len(samples)))
        sv.run(3)
        got = sv.get_state()
    for k, p in enumerate(samples):
        ref, _ = O.run(xy, tri, p, 0.5, U0, 3, rtol=1e-12, atol=atol, bfield=bf)
        assert max(rel_l2_per_comp(got[k * n:(k + 1) * n], ref)) <= 1e-9, (k, rel_l2_per_comp(got[k * n:(k + 1) * n], ref))


@pytest.mark.parametrize("precision", [0, 1])
def test_ensemble_under_captured_gmres_cycles(precision):
    """options.graph on an ensemble: each GMRES restart cycle of the block-diagonal
    system is one replay of a captured CUDA graph.  The states equal the eager
    ensemble's bit for bit (same kernels, same launch shapes, same order of
    sums), and every sample is the oracle root at its rates."""
    xy, tri, samples, U0, bf = _problem()
    n = len(xy)
    atol = 1e-14 * np.linalg.norm(O.residual(xy, tri, samples[0], 0.0, np.abs(U0), np.zeros_like(U0)))
    out = {}
    for graph in (0, 1):
        with S.Solver(xy, tri, samples, beta_field=bf, owner=I.box_partition(xy, 2, 2),
                      **_opts(precision=precision, graph=graph, newton_atol=atol * np.sqrt(len(samples)))) as sv:
            sv.set_state(np.concatenate([U0] * len(samples)))
            stats = sv.run(3)
            out[graph] = (sv.get_state(), [s["gmres_its"] for s in stats])
    assert np.array_equal(out[0][0], out[1][0])
    assert out[0][1] == out[1][1]
    got = out[1][0]
    for k, p in enumerate(samples):
        ref, _ = O.run(xy, tri, p, 0.5, U0, 3, rtol=1e-12, atol=atol, bfield=bf)
        assert max(rel_l2_per_comp(got[k * n:(k + 1) * n], ref)) <= 1e-9, k


def test_ensemble_of_one_is_the_single_problem():
    xy, tri, samples, U0, bf = _problem(n_samples=1)
    kw = _opts(newton_rtol=1e-10, gmres_rtol=1e-8, n_subdomains=4)
    with S.Solver(xy, tri, samples, beta_field=bf, **kw) as e, S.Solver(xy, tri, samples[0], beta_field=bf, **kw) as s:
        for sv in (e, s):
            sv.set_state(U0)
            sv.run(2)
        assert np.array_equal(e.get_state(), s.get_state())


def test_ensemble_rates_are_fixed():
    xy, tri, samples, U0, _ = _problem(n_samples=2, n_target=400)
    with S.Solver(xy, tri, samples, **_opts()) as sv:
        with pytest.raises(S.SeirdError):
            sv.set_params(samples[0])
        with pytest.raises(S.SeirdError):
            sv.set_beta_schedule(dict(b0=0.1, b1=0.05, t_mid=1.0, beta_central=1.0, beta_eastern=1.0,
                                      beta_western=1.0, x_eastern=0.6, x_western=0.4, k_eastern=5.0, k_western=10.0))


def test_ensemble_adjoint_is_per_sample_oracle_adjoint():
    from oracle import seird_adjoint as A
    xy, tri, samples, U0, bf = _problem(n_samples=2, seed=4, n_target=220)
    n, N, dt = len(xy), 6, 0.5
    rng = np.random.default_rng(4)
    obs = [np.sort(rng.choice(n, 12, replace=False)) for _ in samples]
    steps = [2, 4, 6]
    atol = 1e-15 * np.linalg.norm(O.residual(xy, tri, samples[0], 0.0, np.abs(U0), np.zeros_like(U0)))
    refs, I_hat, D_hat = [], [], []
    for k, p in enumerate(samples):
        # observations from a run at perturbed rates, as in the single-context tests
        p_obs = A.with_params(p, A.params_vector(p) * (1.0 + 0.2 * rng.uniform(-1, 1, 10)))
        S_obs = A.forward_states(xy, tri, p_obs, dt, U0, N, bfield=bf)
        Ih = np.array([S_obs[s][obs[k], 2] for s in steps])
        Dh = np.array([S_obs[s][obs[k], 4] for s in steps])
        Sx = A.forward_states(xy, tri, p, dt, U0, N, bfield=bf, rtol=1e-13, atol=atol)
        refs.append(A.adjoint_gradient(xy, tri, p, dt, Sx, obs[k], steps, Ih, Dh, bfield=bf))
        I_hat.append(Ih)
        D_hat.append(Dh)
    nodes = np.concatenate([obs[k] + k * n for k in range(len(samples))])
    with S.Solver(xy, tri, samples, beta_field=bf, owner=I.box_partition(xy, 3, 2),
                  **_opts(newton_rtol=1e-13, newton_atol=atol, gmres_restart=40, gmres_maxit=3000, overlap=1)) as sv:
        sv.set_state(np.concatenate([U0] * len(samples)))
        j, g, gb = sv.adjoint(N, nodes, steps, np.concatenate(I_hat, axis=1), np.concatenate(D_hat, axis=1),
                              lin_rtol=1e-12)
    assert g.shape == (len(samples), 10)
    assert abs(j - sum(r[0] for r in refs)) <= 1e-9 * sum(r[0] for r in refs)
    for k, p in enumerate(samples):
        _, g_ref, gb_ref = refs[k]
        scale = np.abs(g_ref * A.params_vector(p)).max()
        assert np.all(np.abs(g[k] - g_ref) * np.abs(A.params_vector(p)) <= 1e-7 * scale), (k, g[k], g_ref)
        gbk = gb[k * n:(k + 1) * n]
        assert np.linalg.norm(gbk - gb_ref) <= 1e-7 * np.linalg.norm(gb_ref), k
