"""CPU oracle for the paper's solver and model variants.

TEST INFRASTRUCTURE ONLY (see seird_oracle's header): only the tests and the
CPU-baseline legs of bench.py use it.  Plain FP64 NumPy/SciPy.

1. Picard linearisation, Eq. weak_vec_implicit.  The coefficient terms nu(u)
   (Eq. vec_component1) and B(u) (Eq. vec_component2) are frozen at the
   previous iterate u^k and the new iterate solves the linear system

       (u^{k+1}, v) + dt (nu(u^k) grad u^{k+1}, grad v) - dt (B(u^k) u^{k+1}, v) = (u^n, v),

   started from u^{k,0} = u^n and stopped when the update measure
   eps = ||u^{k+1} - u^k||_2 / ||u^n||_2 (Eq. picardtol) reaches the tolerance.
   Since B(u) u is the reaction vector of Eq. seird1-5, the fixed point is the
   root of the backward-Euler system of Eq. weakform.
     * coupled: the five compartments in one linear system (the fully coupled
       alternative Section 2.2 mentions);
     * decoupled: each compartment's equation solved on its own inside a Picard
       iteration, in the order S, E, I, R, D, with the off-diagonal couplings
       B_{cc'} u_{c'} taken from the newest values available (Gauss-Seidel).
       The paper decouples the compartments without giving their order; this
       is the reading used here.

2. Sigmoid transmission schedule of the Southern Ontario study, Eq. beta_ie
   and Eq. beta_x: beta_I(x, t) = beta_E(x, t) = beta(t) beta(x).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import seird_oracle as O

S, E, I, R, D = range(5)


# ---------------------------------------------------------------------------
# Picard linearisation
# ---------------------------------------------------------------------------

def coefficient_matrix(u, p, b=1.0):
    """B(u) [..., 5, 5] of Eq. vec_component2, entry by entry as the paper prints it,
    with kappa = 1 - A/N and b multiplying beta_I and beta_E."""
    s, e, i = u[..., S], u[..., E], u[..., I]
    N = u.sum(axis=-1)
    kappa = 1.0 - p.A / N
    bi = p.beta_i * b
    be = p.beta_e * b
    B = np.zeros(u.shape + (5,))
    B[..., S, S] = p.alpha - p.mu - kappa * be * e - kappa * bi * i
    for c in (E, I, R, D):
        B[..., S, c] = p.alpha
    B[..., E, S] = kappa * bi * i
    B[..., E, E] = kappa * be * s - p.mu - p.sigma - p.gamma_e
    B[..., I, E] = p.sigma
    B[..., I, I] = -p.gamma_r - p.gamma_d - p.mu
    B[..., R, E] = p.gamma_e
    B[..., R, I] = p.gamma_r
    B[..., R, R] = -p.mu
    B[..., D, I] = p.gamma_d
    return B


def mass_matrix(xy, tri):
    """Consistent P1 mass matrix (n x n), (phi_a, phi_b)_T = |T| (1 + delta_ab) / 12."""
    n = len(xy)
    area, _ = O.geometry(xy, tri)
    Me = area[:, None, None] * (np.ones((3, 3)) + np.eye(3))[None] / 12.0
    rows = np.broadcast_to(tri[:, :, None], Me.shape).ravel()
    cols = np.broadcast_to(tri[:, None, :], Me.shape).ravel()
    return sp.coo_matrix((Me.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def picard_matrix(xy, tri, p, dt, U, bfield=None, rule="deg5"):
    """The matrix of Eq. weak_vec_implicit at the frozen iterate U, as CSR on the
    node-major index 5*node + c:  M (x) I + dt nubar_c (N_h grad phi_b, grad phi_a)
    - dt int B_{cc'}(u_h) phi_a phi_b."""
    n = len(xy)
    m = len(tri)
    area, g = O.geometry(xy, tri)
    nu = np.array([p.nu[0], p.nu[1], p.nu[2], p.nu[3], 0.0])
    Ue = U[tri]
    blocks = np.zeros((m, 3, 3, 5, 5))
    Me = (np.ones((3, 3)) + np.eye(3)) / 12.0
    blocks += (area[:, None, None] * Me[None])[:, :, :, None, None] * np.eye(5)
    # nu(u^k): N_h of the frozen iterate, exact on P1 (mean over the triangle)
    Nbar = Ue.sum(axis=2).mean(axis=1)
    K = np.einsum("tax,tbx->tab", g, g) * (area * Nbar)[:, None, None]
    blocks += dt * K[:, :, :, None, None] * np.diag(nu)[None, None, None]
    L, W = O.quad_rule(rule)
    for q in range(len(W)):
        uq = np.einsum("a,tac->tc", L[q], Ue)
        bq = 1.0 if bfield is None else bfield[tri] @ L[q]
        Bq = coefficient_matrix(uq, p, bq)
        wab = np.outer(L[q], L[q])
        blocks -= (dt * W[q] * area)[:, None, None, None, None] * wab[None, :, :, None, None] * Bq[:, None, None]
    rows = 5 * tri[:, :, None, None, None] + np.arange(5)[None, None, None, :, None]
    cols = 5 * tri[:, None, :, None, None] + np.arange(5)[None, None, None, None, :]
    rows = np.broadcast_to(rows, blocks.shape).ravel()
    cols = np.broadcast_to(cols, blocks.shape).ravel()
    P = sp.coo_matrix((blocks.ravel(), (rows, cols)), shape=(5 * n, 5 * n)).tocsr()
    P.sum_duplicates()
    return P


def picard_step(xy, tri, p, dt, Un, eps_tol=1e-8, maxit=200, decoupled=False, bfield=None, rule="deg5",
                rtol=None, atol=0.0):
    """One backward-Euler step by Picard iteration (Eq. weak_vec_implicit) from u^{n+1,0} = u^n.

    Stops when eps = ||U^{k+1} - U^k|| / ||U^n|| <= eps_tol (Eq. picardtol), or, when
    ``rtol`` is given, when ||F(U^{k+1})|| <= rtol ||F(U^n)|| + atol instead.
    Returns (U, info) with info["its"] and info["eps"] (one entry per iteration).
    """
    n = len(xy)
    Mn = mass_matrix(xy, tri) @ Un  # (u^n, phi_i) per compartment [n, 5]
    unorm = np.linalg.norm(Un)
    f0 = np.linalg.norm(O.residual(xy, tri, p, dt, Un, Un, bfield, rule)) if rtol is not None else None
    U = Un.copy()
    info = {"its": 0, "eps": [], "converged": False}
    for k in range(maxit):
        P = picard_matrix(xy, tri, p, dt, U, bfield, rule)
        if not decoupled:
            Unew = spla.splu(P.tocsc()).solve(Mn.ravel()).reshape(n, 5)
        else:
            Unew = U.copy()
            for c in range(5):
                idx = 5 * np.arange(n) + c
                Pcc = P[idx][:, idx]
                rhs = Mn[:, c].copy()
                for c2 in range(5):
                    if c2 != c:
                        rhs -= P[idx][:, 5 * np.arange(n) + c2] @ Unew[:, c2]
                Unew[:, c] = spla.splu(Pcc.tocsc()).solve(rhs)
        eps = np.linalg.norm(Unew - U) / unorm
        info["eps"].append(eps)
        U = Unew
        info["its"] = k + 1
        if rtol is None:
            done = eps <= eps_tol
        else:
            done = np.linalg.norm(O.residual(xy, tri, p, dt, U, Un, bfield, rule)) <= rtol * f0 + atol
        if done:
            info["converged"] = True
            break
    return U, info


# ---------------------------------------------------------------------------
# sigmoid transmission schedule
# ---------------------------------------------------------------------------

PAPER_TIME_SCHEDULE = dict(b0=0.101, b1=0.05, t_mid=130.0)  # Eq. beta_ie
PAPER_SLOPES = dict(k_eastern=5.0, k_western=10.0)          # Eq. beta_x


def beta_time(t, b0, b1, t_mid):
    """beta(t) of Eq. beta_ie: b0 - b1 / (1 + exp(t_mid - t))."""
    return b0 - b1 / (1.0 + np.exp(t_mid - t))


def beta_space(x, beta_central, beta_eastern, beta_western, x_eastern, x_western, k_eastern, k_western):
    """beta(x) of Eq. beta_x along the first coordinate."""
    east = (beta_eastern - beta_central) / (1.0 + np.exp(-k_eastern * (x - x_eastern)))
    west = (beta_western - beta_central) / (1.0 + np.exp(k_western * (x - x_western)))
    return beta_central + east + west


class _Rates:
    def __init__(self, p, beta):
        for k in ("A", "sigma", "gamma_e", "gamma_r", "gamma_d", "alpha", "mu", "nu"):
            setattr(self, k, getattr(p, k))
        self.beta_i = beta
        self.beta_e = beta


def schedule_run(xy, tri, p, dt, U0, t0, n_steps, sched, **newton_kw):
    """n_steps backward-Euler steps from time t0 with beta_I = beta_E = beta(t^{k+1}) beta(x):
    beta(t) at the end of each step, beta(x) at the nodes (a P1 field).  ``sched`` holds the
    keyword arguments of beta_time and beta_space."""
    bx = beta_space(xy[:, 0], sched["beta_central"], sched["beta_eastern"], sched["beta_western"],
                    sched["x_eastern"], sched["x_western"], sched["k_eastern"], sched["k_western"])
    U = U0.copy()
    for k in range(n_steps):
        bt = beta_time(t0 + (k + 1) * dt, sched["b0"], sched["b1"], sched["t_mid"])
        U, info = O.newton_step(xy, tri, _Rates(p, bt), dt, U, bfield=bx, **newton_kw)
        if not info["converged"]:
            raise RuntimeError("oracle Newton did not converge")
    return U
