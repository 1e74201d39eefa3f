"""Pins of the oracle's discrete adjoint against central finite differences of
the misfit (forward runs of the oracle itself, Newton to 1e-13)."""
import numpy as np

from oracle import seird_adjoint as A
from oracle import seird_oracle as O
from paper_2208_01839_gb300 import inputs as I


def _problem(seed=4):
    xy, tri, _ = I.irregular_mesh(seed, 220)
    dens = I.urban_density(seed)
    U0 = I.urban_ic(xy, dens, seed, width=0.08, frac=0.05)
    p = I.params_ontario(float(U0.sum(axis=1).max()), nu=(4e-4, 5e-4, 1e-4, 3e-4))
    bf = I.smooth_field(xy, seed)
    dt, N = 0.5, 6
    rng = np.random.default_rng(seed)
    obs_nodes = rng.choice(len(xy), 12, replace=False)
    obs_steps = [2, 4, 6]
    # observations from a run at perturbed rates, so the misfit is not zero
    p_obs = A.with_params(p, A.params_vector(p) * (1.0 + 0.2 * rng.uniform(-1, 1, 10)))
    S_obs = A.forward_states(xy, tri, p_obs, dt, U0, N, bfield=bf)
    I_hat = np.array([S_obs[k][obs_nodes, 2] for k in obs_steps])
    D_hat = np.array([S_obs[k][obs_nodes, 4] for k in obs_steps])
    return xy, tri, p, bf, dt, N, U0, obs_nodes, obs_steps, I_hat, D_hat


def _floor(xy, tri, p, U0):
    return 1e-15 * np.linalg.norm(O.residual(xy, tri, p, 0.0, np.abs(U0), np.zeros_like(U0)))


def _J(xy, tri, p, bf, dt, N, U0, obs_nodes, obs_steps, I_hat, D_hat, atol):
    S = A.forward_states(xy, tri, p, dt, U0, N, bfield=bf, rtol=1e-13, atol=atol)
    return A.misfit(S, obs_nodes, obs_steps, I_hat, D_hat)


def test_adjoint_gradient_matches_central_differences():
    xy, tri, p, bf, dt, N, U0, obs_nodes, obs_steps, I_hat, D_hat = _problem()
    atol = _floor(xy, tri, p, U0)
    S = A.forward_states(xy, tri, p, dt, U0, N, bfield=bf, rtol=1e-13, atol=atol)
    j, g, gb = A.adjoint_gradient(xy, tri, p, dt, S, obs_nodes, obs_steps, I_hat, D_hat, bfield=bf)
    assert j > 0
    v0 = A.params_vector(p)
    for k in range(10):
        h = 1e-6 * abs(v0[k])
        vp, vm = v0.copy(), v0.copy()
        vp[k] += h
        vm[k] -= h
        jp = _J(xy, tri, A.with_params(p, vp), bf, dt, N, U0, obs_nodes, obs_steps, I_hat, D_hat, atol)
        jm = _J(xy, tri, A.with_params(p, vm), bf, dt, N, U0, obs_nodes, obs_steps, I_hat, D_hat, atol)
        fd = (jp - jm) / (2 * h)
        assert abs(fd - g[k]) <= 1e-5 * max(abs(g[k]), 1e-3 * np.abs(g * v0).max() / abs(v0[k])), (A.PARAM_NAMES[k], fd, g[k])
    # per-node transmission field: directional derivative along a smooth direction
    v = I.smooth_field(xy, 99, lo=-1.0, hi=1.0)
    h = 1e-6
    jp = _J(xy, tri, p, bf + h * v, dt, N, U0, obs_nodes, obs_steps, I_hat, D_hat, atol)
    jm = _J(xy, tri, p, bf - h * v, dt, N, U0, obs_nodes, obs_steps, I_hat, D_hat, atol)
    fd = (jp - jm) / (2 * h)
    assert abs(fd - gb @ v) <= 1e-5 * abs(gb @ v), (fd, gb @ v)


def test_field_term_uses_the_affine_dependence_on_b():
    """F is affine in the transmission field, so lambda^T dF/db . v equals
    lambda^T (F(b = v) - F(b = 0)) exactly, for any lambda and state."""
    xy, tri, p, bf, dt, N, U0, *_ = _problem(6)
    rng = np.random.default_rng(1)
    lam = rng.standard_normal(U0.shape)
    v = rng.standard_normal(len(xy))
    lhs = A.field_gradient_term(xy, tri, p, dt, U0, lam) @ v
    rhs = np.sum(lam * (O.residual(xy, tri, p, dt, U0, U0, bfield=v) - O.residual(xy, tri, p, dt, U0, U0, bfield=0 * v)))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1e-300) * 1e3
