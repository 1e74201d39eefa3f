"""Pins of the oracle's paper variants (Picard linearisation, sigmoid transmission).

* B(u) as printed (Eq. vec_component2) times u is the reaction vector of
  Eq. seird1-5, written out independently in the Newton oracle.
* The Picard matrix at U applied to U, minus the mass term of u^n, is the
  residual of Eq. weakform: the Picard fixed point is the backward-Euler root.
* On a linear problem (no transmission, no Allee term, no diffusion) the Picard
  matrix is the Jacobian.
* With alpha = 0 the coupling of B(u) is lower triangular in the order S, E,
  I, R, D, so the decoupled Gauss-Seidel Picard iterates equal the coupled ones.
* Picard (coupled and decoupled) reaches the Newton root (the cross-check of
  the two iterations).
* beta(t) and beta(x) take the values the closed forms of Eq. beta_ie and
  Eq. beta_x fix at their centres and limits; a flat schedule reduces to a run
  with constant rates.
"""
import numpy as np
import pytest

from oracle import seird_oracle as O
from oracle import seird_variants as V
from paper_2208_01839_gb300 import inputs as I


class _P:
    def __init__(self, **kw):
        self.__dict__.update(kw)


def _params(alpha=0.0, mu=0.0, A=8.9e-3):
    return _P(A=A, beta_i=0.03, beta_e=0.02, sigma=1 / 5, gamma_e=1 / 15, gamma_r=1 / 11, gamma_d=1 / 750,
              alpha=alpha, mu=mu, nu=(4.5e-4, 4.5e-4, 1e-5, 4.5e-4))


def _mesh_state(seed=2, n_target=300):
    xy, tri, _ = I.irregular_mesh(seed, n_target)
    rng = np.random.default_rng(seed)
    Un = rng.uniform(0.5, 3.0, (len(xy), 5))
    U = Un * rng.uniform(0.9, 1.1, Un.shape)
    return xy, tri, U, Un, I.smooth_field(xy, seed)


def test_coefficient_matrix_times_state_is_the_reaction():
    rng = np.random.default_rng(0)
    u = rng.uniform(0.1, 5.0, (200, 5))
    b = rng.uniform(0.5, 1.5, 200)
    for p in (_params(), _params(alpha=0.01, mu=0.003)):
        Bu = np.einsum("kcd,kd->kc", V.coefficient_matrix(u, p, b), u)
        Rv = O.reaction(u, p, b)
        assert np.abs(Bu - Rv).max() <= 1e-14 * np.abs(Rv).max()


@pytest.mark.parametrize("rule", ["deg5", "vertex"])
def test_picard_fixed_point_is_the_backward_euler_root(rule):
    xy, tri, U, Un, bf = _mesh_state()
    p = _params(alpha=0.01, mu=0.003)
    dt = 0.7
    P = V.picard_matrix(xy, tri, p, dt, U, bfield=bf, rule=rule)
    lhs = (P @ U.ravel()).reshape(U.shape) - V.mass_matrix(xy, tri) @ Un
    F = O.residual(xy, tri, p, dt, U, Un, bfield=bf, rule=rule)
    assert np.abs(lhs - F).max() <= 1e-12 * np.abs(V.mass_matrix(xy, tri) @ U).max()


def test_picard_matrix_is_the_jacobian_of_a_linear_problem():
    xy, tri, U, Un, _ = _mesh_state(seed=3)
    p = _params(alpha=0.01, mu=0.003, A=0.0)
    p.beta_i = p.beta_e = 0.0
    p.nu = (0.0, 0.0, 0.0, 0.0)
    P = V.picard_matrix(xy, tri, p, 0.5, U)
    J = O.jacobian(xy, tri, p, 0.5, U)
    assert abs(P - J).max() <= 1e-15 * abs(J).max()
    # with transmission on, they differ (the Jacobian carries the coefficient derivatives)
    q = _params()
    assert abs(V.picard_matrix(xy, tri, q, 0.5, U) - O.jacobian(xy, tri, q, 0.5, U)).max() > 1e-6


def test_decoupled_gauss_seidel_equals_coupled_when_alpha_is_zero():
    wl = I.square_workload(9, N0=2000.0)
    for its in (1, 3):
        Uc, _ = V.picard_step(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, eps_tol=0.0, maxit=its)
        Ud, _ = V.picard_step(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, eps_tol=0.0, maxit=its, decoupled=True)
        assert np.abs(Uc - Ud).max() <= 1e-11 * np.abs(Uc).max()


def test_picard_reaches_the_newton_root():
    wl = I.square_workload(9, N0=2000.0)
    Un_, _ = O.newton_step(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, rtol=1e-14)
    Uc, ic = V.picard_step(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, eps_tol=1e-15)
    assert ic["converged"]
    assert np.linalg.norm(Uc - Un_) <= 1e-10 * np.linalg.norm(Un_)
    # the update measure falls geometrically (a contraction, not Newton's quadratic rate)
    e = np.array(ic["eps"])
    assert e[-1] < 1e-15 and np.all(e[1:6] < e[:5])
    # decoupled with alpha != 0 (the order then matters for the iterates, not the root)
    xy, tri, U, Un, bf = _mesh_state(seed=5, n_target=150)
    p = _params(alpha=0.02, mu=0.004)
    Ur, _ = O.newton_step(xy, tri, p, 0.5, Un, rtol=1e-14, bfield=bf)
    Ud, idd = V.picard_step(xy, tri, p, 0.5, Un, eps_tol=1e-15, decoupled=True, bfield=bf)
    assert idd["converged"]
    assert np.linalg.norm(Ud - Ur) <= 1e-10 * np.linalg.norm(Ur)


def test_beta_time_closed_form_values():
    s = V.PAPER_TIME_SCHEDULE
    assert V.beta_time(s["t_mid"], **s) == s["b0"] - 0.5 * s["b1"]
    assert abs(V.beta_time(0.0, **s) - 0.101) < 1e-50 + 1e-15
    assert abs(V.beta_time(400.0, **s) - 0.051) < 1e-15
    t = np.linspace(0, 260, 261)
    assert np.all(np.diff(V.beta_time(t, **s)) <= 0)  # saturates in FP64 far from t_mid
    t = np.linspace(100, 160, 61)
    assert np.all(np.diff(V.beta_time(t, **s)) < 0)
    # symmetry of the logistic about t_mid: beta(t_mid + h) + beta(t_mid - h) = 2 b0 - b1
    h = np.array([0.5, 3.0, 11.0])
    assert np.allclose(V.beta_time(s["t_mid"] + h, **s) + V.beta_time(s["t_mid"] - h, **s),
                       2 * s["b0"] - s["b1"], rtol=0, atol=1e-16)


def test_beta_space_regions():
    kw = dict(beta_central=2.0, beta_eastern=3.0, beta_western=1.0, x_eastern=0.7, x_western=0.3,
              k_eastern=200.0, k_western=400.0)
    assert abs(V.beta_space(0.5, **kw) - 2.0) < 1e-12    # central region
    assert abs(V.beta_space(1.0, **kw) - 3.0) < 1e-12    # east of x_eastern
    assert abs(V.beta_space(0.0, **kw) - 1.0) < 1e-12    # west of x_western
    assert abs(V.beta_space(0.7, **kw) - 2.5) < 1e-12    # half way at the eastern boundary
    assert abs(V.beta_space(0.3, **kw) - 1.5) < 1e-12    # half way at the western boundary


def test_flat_schedule_reduces_to_constant_rates():
    wl = I.square_workload(9, N0=2000.0)
    beta = wl.params.beta_i
    sched = dict(b0=1.0, b1=0.0, t_mid=5.0, beta_central=beta, beta_eastern=beta, beta_western=beta,
                 x_eastern=0.7, x_western=0.3, k_eastern=5.0, k_western=10.0)
    Us = V.schedule_run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 0.0, 3, sched, rtol=1e-13)
    Uc, _ = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 3, rtol=1e-13)
    assert np.linalg.norm(Us - Uc) <= 1e-11 * np.linalg.norm(Uc)
