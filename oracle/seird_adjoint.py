"""CPU oracle for the discrete adjoint of a SEIRD backward-Euler run.

TEST INFRASTRUCTURE ONLY (see seird_oracle's header): only the tests and the
CPU-baseline legs of bench.py use it.  Plain FP64 NumPy/SciPy.

Problem.  States U^0 (given), U^1..U^N with F(U^k; U^{k-1}, p) = 0 (the
discrete system of Eq. weakform, one Newton-solved step each).  Misfit of
observed infected and deceased densities at observation nodes and steps:

    j = sum_{k in steps} sum_{i in nodes} (U^k_{i,I} - Ihat_{k,i})^2 + (U^k_{i,D} - Dhat_{k,i})^2.

Discrete adjoint (Lagrangian j + sum_k lambda_k^T F^k): F^{k+1} depends on
U^k only through -M U^k (M the consistent mass, per compartment), so for
k = N, ..., 1

    J_k^T lambda_k = -dj/dU^k + M lambda_{k+1},   lambda_{N+1} = 0,
    dj/dp = sum_k lambda_k^T dF^k/dp.

The gradient parameters are the rates the paper calibrates (Section 4.2):
beta_I, beta_E, sigma, gamma_E, gamma_R, gamma_D and nubar_S..nubar_R, plus a
per-node P1 transmission multiplier b (Eq. beta_ie/beta_x, frozen in time).
F is linear in each of them, so dF/dp_k at a state U is the residual of that
state with the unit parameter set {p_k = 1, all others 0} and U^n = U (the
mass term vanishes), and F is affine in b, which the tests use as a pin.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import seird_oracle as O

PARAM_NAMES = ("beta_i", "beta_e", "sigma", "gamma_e", "gamma_r", "gamma_d", "nu_S", "nu_E", "nu_I", "nu_R")


class _P:
    """Minimal parameter record (same attribute names as the inputs' Params)."""

    def __init__(self, **kw):
        self.A = kw.get("A", 0.0)
        for k in ("beta_i", "beta_e", "sigma", "gamma_e", "gamma_r", "gamma_d", "alpha", "mu"):
            setattr(self, k, kw.get(k, 0.0))
        self.nu = tuple(kw.get("nu", (0.0, 0.0, 0.0, 0.0)))


def unit_params(p, name):
    """Every gradient parameter 0 except ``name`` = 1; the Allee A is kept."""
    q = _P(A=p.A)
    if name.startswith("nu_"):
        nu = [0.0, 0.0, 0.0, 0.0]
        nu["SEIR".index(name[3])] = 1.0
        q.nu = tuple(nu)
    else:
        setattr(q, name, 1.0)
    return q


def params_vector(p):
    return np.array([p.beta_i, p.beta_e, p.sigma, p.gamma_e, p.gamma_r, p.gamma_d] + list(p.nu))


def with_params(p, vec):
    q = _P(A=p.A, alpha=p.alpha, mu=p.mu)
    for k, v in zip(PARAM_NAMES[:6], vec[:6]):
        setattr(q, k, float(v))
    q.nu = tuple(float(v) for v in vec[6:10])
    return q


def forward_states(xy, tri, p, dt, U0, n_steps, bfield=None, rtol=1e-13, atol=0.0, rule="deg5"):
    states = [U0.copy()]
    for _ in range(n_steps):
        U, info = O.newton_step(xy, tri, p, dt, states[-1], rtol=rtol, atol=atol, bfield=bfield, rule=rule)
        if not info["converged"]:
            raise RuntimeError("oracle Newton did not converge")
        states.append(U)
    return states


def misfit(states, obs_nodes, obs_steps, I_hat, D_hat):
    j = 0.0
    for r, k in enumerate(obs_steps):
        U = states[k]
        j += np.sum((U[obs_nodes, 2] - I_hat[r]) ** 2) + np.sum((U[obs_nodes, 4] - D_hat[r]) ** 2)
    return j


def mass_apply(xy, tri, V):
    """M V with the consistent P1 mass, per compartment (the dt = 0 residual)."""
    area, _ = O.geometry(xy, tri)
    out = np.zeros_like(V)
    Ve = V[tri]  # [m, 3, 5]
    s = Ve.sum(axis=1)  # [m, 5]
    np.add.at(out, tri, (area / 12.0)[:, None, None] * (Ve + s[:, None, :]))
    return out


def field_gradient_term(xy, tri, p, dt, U, lam, rule="deg5"):
    """lambda^T dF/db_j for every node j: dt int phi_j kappa s (beta_I i + beta_E e) (lambda_S - lambda_E)_h."""
    area, _ = O.geometry(xy, tri)
    L, W = O.quad_rule(rule)
    out = np.zeros(len(xy))
    Ue = U[tri]
    Le = lam[tri]
    for q in range(len(W)):
        uq = np.einsum("a,tac->tc", L[q], Ue)
        lq = np.einsum("a,tac->tc", L[q], Le)
        N = uq.sum(axis=1)
        kappa = 1.0 - p.A / N
        f = p.beta_i * uq[:, 2] + p.beta_e * uq[:, 1]
        val = dt * W[q] * area * kappa * uq[:, 0] * f * (lq[:, 0] - lq[:, 1])
        np.add.at(out, tri, val[:, None] * L[q][None, :])
    return out


def adjoint_gradient(xy, tri, p, dt, states, obs_nodes, obs_steps, I_hat, D_hat, bfield=None, rule="deg5"):
    """(misfit, d misfit / d p [10], d misfit / d b [n]) by the discrete adjoint."""
    n = len(xy)
    N = len(states) - 1
    obs_at = {k: r for r, k in enumerate(obs_steps)}
    lam_next = np.zeros((n, 5))
    g = np.zeros(len(PARAM_NAMES))
    gb = np.zeros(n)
    units = [unit_params(p, nm) for nm in PARAM_NAMES]
    for k in range(N, 0, -1):
        dj = np.zeros((n, 5))
        if k in obs_at:
            r = obs_at[k]
            dj[obs_nodes, 2] = 2.0 * (states[k][obs_nodes, 2] - I_hat[r])
            dj[obs_nodes, 4] = 2.0 * (states[k][obs_nodes, 4] - D_hat[r])
        rhs = -dj + mass_apply(xy, tri, lam_next)
        Jk = O.jacobian(xy, tri, p, dt, states[k], bfield=bfield, rule=rule)
        lam = spla.splu(Jk.T.tocsc()).solve(rhs.ravel()).reshape(n, 5)
        for i, q in enumerate(units):
            dF = O.residual(xy, tri, q, dt, states[k], states[k], bfield=bfield, rule=rule)
            g[i] += np.sum(lam * dF)
        gb += field_gradient_term(xy, tri, p, dt, states[k], lam, rule)
        lam_next = lam
    return misfit(states, obs_nodes, obs_steps, I_hat, D_hat), g, gb
