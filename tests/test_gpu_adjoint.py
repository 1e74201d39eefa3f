"""Discrete adjoint on the GPU (seird_adjoint) against the CPU oracle's adjoint,
central finite differences of GPU forward runs, checkpoint recomputation, and
the torch.autograd bridge."""
import numpy as np
import pytest

from oracle import seird_adjoint as A
from oracle import seird_oracle as O
from paper_2208_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2208_01839_gb300 import build as _b  # noqa: E402

_b.build()
from paper_2208_01839_gb300 import autograd as AG  # noqa: E402
from paper_2208_01839_gb300 import seird as S  # noqa: E402


def _problem(seed=4, n_target=220, N=6, obs_every=2, n_obs=12):
    xy, tri, _ = I.irregular_mesh(seed, n_target)
    dens = I.urban_density(seed)
    U0 = I.urban_ic(xy, dens, seed, width=0.08, frac=0.05)
    p = I.params_ontario(float(U0.sum(axis=1).max()), nu=(4e-4, 5e-4, 1e-4, 3e-4))
    bf = I.smooth_field(xy, seed)
    rng = np.random.default_rng(seed)
    obs_nodes = rng.choice(len(xy), n_obs, replace=False)
    obs_steps = list(range(obs_every, N + 1, obs_every))
    p_obs = A.with_params(p, A.params_vector(p) * (1.0 + 0.2 * rng.uniform(-1, 1, 10)))
    S_obs = A.forward_states(xy, tri, p_obs, 0.5, U0, N, bfield=bf)
    I_hat = np.array([S_obs[k][obs_nodes, 2] for k in obs_steps])
    D_hat = np.array([S_obs[k][obs_nodes, 4] for k in obs_steps])
    return dict(xy=xy, tri=tri, p=p, bf=bf, dt=0.5, N=N, U0=U0, obs_nodes=obs_nodes, obs_steps=obs_steps,
                I_hat=I_hat, D_hat=D_hat)


def _floor(P):
    return 1e-15 * np.linalg.norm(O.residual(P["xy"], P["tri"], P["p"], 0.0, np.abs(P["U0"]), np.zeros_like(P["U0"])))


def _solver(P, **kw):
    opts = dict(dt=P["dt"], overlap=1, coarse=1, newton_rtol=1e-13, newton_atol=_floor(P), gmres_rtol=1e-12,
                gmres_maxit=3000, gmres_restart=40)
    opts.update(kw)
    return S.Solver(P["xy"], P["tri"], P["p"], beta_field=P["bf"], owner=I.box_partition(P["xy"], 3, 2), **opts)


def _adjoint(sv, P, **kw):
    sv.set_state(P["U0"])
    return sv.adjoint(P["N"], P["obs_nodes"], P["obs_steps"], P["I_hat"], P["D_hat"], lin_rtol=1e-12, **kw)


@pytest.mark.parametrize("coarse,fill", [(1, 0), (2, 0), (2, 2)])
def test_gpu_adjoint_matches_oracle_adjoint(coarse, fill):
    """Also with the multiplicative two-grid: the transposed solves then use the
    two-grid built from J^T (its J Z update included); and with block ILU(2)
    factors of J^T on the fill pattern."""
    P = _problem()
    Sx = A.forward_states(P["xy"], P["tri"], P["p"], P["dt"], P["U0"], P["N"], bfield=P["bf"], rtol=1e-13,
                          atol=_floor(P))
    j_ref, g_ref, gb_ref = A.adjoint_gradient(P["xy"], P["tri"], P["p"], P["dt"], Sx, P["obs_nodes"],
                                              P["obs_steps"], P["I_hat"], P["D_hat"], bfield=P["bf"])
    with _solver(P, coarse=coarse, ilu_fill=fill) as sv:
        j, g, gb = _adjoint(sv, P)
        U_after = sv.get_state()
    assert abs(j - j_ref) <= 1e-9 * j_ref
    scale = np.abs(g_ref * A.params_vector(P["p"]))
    for k in range(10):
        assert abs(g[k] - g_ref[k]) * abs(A.params_vector(P["p"])[k]) <= 1e-7 * scale.max(), (A.PARAM_NAMES[k], g[k], g_ref[k])
    assert np.linalg.norm(gb - gb_ref) <= 1e-7 * np.linalg.norm(gb_ref)
    assert np.array_equal(U_after, P["U0"])  # the state is restored


def test_checkpoint_recomputation_is_exact():
    P = _problem(seed=5, N=7, obs_every=1)
    with _solver(P) as sv:
        j1, g1, gb1 = _adjoint(sv, P, checkpoint_every=1)
        j3, g3, gb3 = _adjoint(sv, P, checkpoint_every=3)
    assert j1 == j3
    assert np.array_equal(g1, g3) and np.array_equal(gb1, gb3)


def _gpu_misfit(sv, P, vec=None, bf=None):
    p = A.with_params(P["p"], A.params_vector(P["p"]) if vec is None else vec)
    sv.set_params(dict(A=p.A, beta_i=p.beta_i, beta_e=p.beta_e, sigma=p.sigma, gamma_e=p.gamma_e,
                       gamma_r=p.gamma_r, gamma_d=p.gamma_d, alpha=p.alpha, mu=p.mu, nu=p.nu),
                  beta_field=P["bf"] if bf is None else bf)
    sv.set_state(P["U0"])
    j = 0.0
    for k in range(1, P["N"] + 1):
        sv.step()
        if k in P["obs_steps"]:
            U = sv.get_state()
            r = P["obs_steps"].index(k)
            j += np.sum((U[P["obs_nodes"], 2] - P["I_hat"][r]) ** 2) + np.sum((U[P["obs_nodes"], 4] - P["D_hat"][r]) ** 2)
    return j


def test_gpu_adjoint_matches_central_differences():
    """Relative step 1e-6 on each rate and along a smooth field direction; the
    forward runs solve Newton to 1e-13 so that FD noise stays far below 1e-5."""
    P = _problem(seed=7, n_target=2500, N=8, obs_every=2, n_obs=50)
    with _solver(P) as sv:
        j, g, gb = _adjoint(sv, P)
        v0 = A.params_vector(P["p"])
        for k in range(10):
            h = 1e-6 * abs(v0[k])
            vp, vm = v0.copy(), v0.copy()
            vp[k] += h
            vm[k] -= h
            fd = (_gpu_misfit(sv, P, vp) - _gpu_misfit(sv, P, vm)) / (2 * h)
            tol = 1e-5 * max(abs(g[k]), 1e-3 * np.abs(g * v0).max() / abs(v0[k]))
            assert abs(fd - g[k]) <= tol, (A.PARAM_NAMES[k], fd, g[k])
        v = I.smooth_field(P["xy"], 99, lo=-1.0, hi=1.0)
        h = 1e-6
        fd = (_gpu_misfit(sv, P, bf=P["bf"] + h * v) - _gpu_misfit(sv, P, bf=P["bf"] - h * v)) / (2 * h)
        assert abs(fd - gb @ v) <= 1e-5 * abs(gb @ v), (fd, gb @ v)


def test_autograd_bridge():
    P = _problem(seed=8)
    spec = dict(n_steps=P["N"], obs_nodes=P["obs_nodes"], obs_steps=P["obs_steps"], I_hat=P["I_hat"],
                D_hat=P["D_hat"], lin_rtol=1e-12)
    with _solver(P) as sv:
        rates = torch.tensor(A.params_vector(P["p"]), dtype=torch.float64, requires_grad=True)
        field = torch.tensor(P["bf"], dtype=torch.float64, requires_grad=True)
        j = AG.misfit(sv, P["U0"], rates, field, P["p"], spec)
        gr, gf = torch.autograd.grad(3.0 * j, (rates, field))
        j2, g2, gb2 = _adjoint(sv, P)
    assert abs(j.item() - j2) <= 1e-12 * j2
    assert np.allclose(gr.numpy(), 3.0 * g2, rtol=1e-12, atol=0)
    assert np.allclose(gf.numpy(), 3.0 * gb2, rtol=1e-12, atol=0)
