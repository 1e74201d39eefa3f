"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something outside itself: exactness
of the quadrature rule, exact integrals of P1 functions, discrete conservation
(Section 2.1: an isolated domain keeps its total population), the exact
deceased-row identity, the homogeneous-start reduction to the ODE and its
first-order convergence (Appendix B.4, Table order_time), closed-form
identities of the ODE, manufactured-solution spatial order 2 (Appendix B.1/B.3,
Table ord_spatial_2), brute-force dense Newton, finite-difference Jacobians,
mesh symmetry, and the defining properties of ILU(0), ILU(k) (its pattern
against the fill-path characterisation, its product against the matrix on the
pattern, its exact limit), RAS and the coarse space (Section 3).
"""
import json
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.integrate import solve_ivp
from scipy.optimize import fsolve

from oracle import seird_oracle as O
from paper_2208_01839_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# quadrature and P1 geometry
# ---------------------------------------------------------------------------

def test_quadrature_degree5_exact_on_monomials():
    """Radon's rule integrates x^a y^b exactly for a+b <= 5 on the reference
    triangle (exact value a! b! / (a+b+2)!) and is not exact at degree 6."""
    L, W = O.quad_rule("deg5")
    assert abs(W.sum() - 1.0) < 1e-15
    x, y = L[:, 1], L[:, 2]
    for a in range(7):
        for b in range(7 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            approx = 0.5 * np.sum(W * x ** a * y ** b)
            if a + b <= 5:
                assert abs(approx - exact) < 1e-15, (a, b)
    worst = max(abs(0.5 * np.sum(W * x ** a * y ** (6 - a)) - math.factorial(a) * math.factorial(6 - a) / math.factorial(8))
                for a in range(7))
    assert worst > 1e-6
    Lv, Wv = O.quad_rule("vertex")
    assert abs(0.5 * np.sum(Wv * Lv[:, 1]) - 1.0 / 6.0) < 1e-15
    assert abs(0.5 * np.sum(Wv * Lv[:, 1] ** 2) - 1.0 / 12.0) > 1e-3


def test_p1_gradients_reproduce_linear_functions():
    xy, tri, _ = I.irregular_mesh(3, 400)
    area, g = O.geometry(xy, tri)
    f = 2.0 + 3.0 * xy[:, 0] - 5.0 * xy[:, 1]
    grad = np.einsum("ta,tax->tx", f[tri], g)
    assert np.allclose(grad, [3.0, -5.0], atol=1e-10)
    assert np.allclose(g.sum(axis=1), 0.0, atol=1e-9)
    p = I.random_polygon(3)
    assert area.sum() < 1.0 and area.min() > 0


def _linear_state(xy):
    U = np.zeros((len(xy), 5))
    U[:, 0] = 2.0 + xy[:, 0]
    U[:, 1] = 1.0 + xy[:, 1]
    U[:, 2] = 0.5 + xy[:, 0]
    U[:, 3] = 0.3
    U[:, 4] = 0.1
    return U


def test_consistent_mass_integrates_p1_products_exactly():
    """With dt = 0 the residual is M (U - U^n); for U - U^n = x (all c) and the
    weights y, sum_i y_i F_ic = int x y = 1/4 on the unit square (exact for the
    consistent mass, not for a lumped one)."""
    xy, tri = I.structured_mesh(9)
    p = I.params_square()
    U = np.repeat(xy[:, 0:1], 5, axis=1)
    F = O.residual(xy, tri, p, 0.0, U, np.zeros_like(U))
    assert np.allclose(xy[:, 1] @ F, 0.25, rtol=0, atol=1e-14)
    assert np.allclose(F.sum(axis=0), 0.5, atol=1e-14)  # int x = 1/2


def test_diffusion_term_against_exact_integrals():
    """Reaction off, U = U^n linear: sum_i v_i F_ic = dt nubar_c int N grad u_c . grad v
    for P1 v, with N = s+e+i+r+d linear (Eq. weakform, no-flux boundary)."""
    xy, tri = I.structured_mesh(11)
    p = I.Params(A=0.0, beta_i=0.0, beta_e=0.0, sigma=0.0, gamma_e=0.0, gamma_r=0.0, gamma_d=0.0,
                 nu=(0.7, 1.3, 0.2, 2.9))
    U = _linear_state(xy)
    dt = 0.37
    F = O.residual(xy, tri, p, dt, U, U)
    # N = 3.9 + 2x + y ; int_N = 3.9 + 1 + 0.5
    intN = 5.4
    assert abs(xy[:, 0] @ F[:, 0] - dt * 0.7 * intN) < 1e-12      # grad s = (1,0), v = x
    assert abs(xy[:, 1] @ F[:, 1] - dt * 1.3 * intN) < 1e-12      # grad e = (0,1), v = y
    assert abs(xy[:, 0] @ F[:, 2] - dt * 0.2 * intN) < 1e-12      # grad i = (1,0), v = x
    assert abs(xy[:, 1] @ F[:, 0]) < 1e-12                        # grad s . grad y = 0
    assert np.allclose(F.sum(axis=0), 0.0, atol=1e-12)            # no flux: constants annihilated
    assert np.allclose(F[:, 3:], 0.0, atol=1e-13)                 # r constant, nubar_D = 0


# ---------------------------------------------------------------------------
# conservation and the D-row identity
# ---------------------------------------------------------------------------

def test_residual_sum_equals_mass_change_identity():
    """alpha = mu = 0: sum_c R_c = 0 pointwise and sum_i grad phi_i = 0, so
    sum_{i,c} F_ic = sum_c int (u_c - u_c^n) for ANY state (Section 2.1)."""
    xy, tri, _ = I.irregular_mesh(5, 300)
    rng = np.random.default_rng(1)
    U = rng.uniform(100, 1000, (len(xy), 5))
    Un = rng.uniform(100, 1000, (len(xy), 5))
    p = I.params_square()
    bf = I.smooth_field(xy, 2)
    F = O.residual(xy, tri, p, 0.8, U, Un, bfield=bf)
    Fm = O.residual(xy, tri, p, 0.0, U, Un)
    assert abs(F.sum() - Fm.sum()) <= 1e-12 * np.abs(F).sum()
    pv = I.params_square(alpha=0.01)
    Fa = O.residual(xy, tri, pv, 0.8, U, Un, bfield=bf)
    assert abs(Fa.sum() - Fm.sum()) > 1e-3  # births break it, as they should


def test_total_population_conserved_over_steps():
    wl = I.square_workload(17)
    U, infos = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 3)
    area, _ = O.geometry(wl.xy, wl.tri)
    w = np.zeros(wl.n)
    np.add.at(w, wl.tri, np.repeat(area[:, None] / 3.0, 3, axis=1))  # int phi_i
    tot0 = w @ wl.U0.sum(axis=1)
    tot = w @ U.sum(axis=1)
    assert abs(tot - tot0) <= 1e-11 * tot0
    assert all(i["converged"] for i in infos)


def test_paper_density_stays_nonnegative():
    """At the paper's square density N = 2000 (Section 4.1) the growth rate
    times dt stays below 1 and the steps keep every compartment nonnegative;
    at N = 1e4 (kappa beta N dt ~ 3.6) backward Euler flips the sign of the
    exposed compartment's growth phase, so negativity there is expected."""
    wl = I.square_workload(17, N0=2000.0)
    U, infos = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 4)
    assert U.min() >= 0.0
    wl2 = I.square_workload(17)
    U2, _ = O.run(wl2.xy, wl2.tri, wl2.params, wl2.dt, wl2.U0, 1)
    assert U2[:, 1].min() < 0.0


def test_deceased_row_identity_degree5():
    """The degree-5 rule integrates gamma_D i phi_j exactly, so at the root
    d^{n+1} = d^n + dt gamma_D i^{n+1} node by node (Eq. seird5)."""
    wl = I.square_workload(17)
    Un = wl.U0.copy()
    Un[:, 4] = 3.0
    U, info = O.newton_step(wl.xy, wl.tri, wl.params, wl.dt, Un, rtol=1e-13)
    lhs = U[:, 4] - Un[:, 4] - wl.dt * wl.params.gamma_d * U[:, 2]
    assert np.abs(lhs).max() < 1e-9 * np.abs(U[:, 4]).max()
    # the vertex rule lumps (gamma_D i, phi_j) while (d - d^n, phi_j) keeps the
    # consistent mass, so the nodewise identity must fail for it
    Uv, _ = O.newton_step(wl.xy, wl.tri, wl.params, wl.dt, Un, rtol=1e-13, rule="vertex")
    lhs_v = Uv[:, 4] - Un[:, 4] - wl.dt * wl.params.gamma_d * Uv[:, 2]
    assert np.abs(lhs_v).max() > 1e-6 * np.abs(Uv[:, 4] - Un[:, 4]).max()


# ---------------------------------------------------------------------------
# homogeneous start -> ODE (Appendix B.4)
# ---------------------------------------------------------------------------

def _ode_params():
    return I.params_square(beta_e=2.0e-4)


def test_homogeneous_start_is_the_ode_backward_euler_step():
    """Uniform U^0 under no-flux: grad u = 0 and the discrete system collapses
    to u - u^n = dt R(u) at every node."""
    p = _ode_params()
    xy, tri, _ = I.irregular_mesh(11, 120)
    U0 = I.uniform_ic(len(xy), 2000.0, 0.1)
    dt = 0.5
    U = U0
    for _ in range(3):
        un = U[0].copy()
        U, info = O.newton_step(xy, tri, p, dt, U, rtol=1e-13)
        ref = fsolve(lambda v: v - un - dt * O.reaction(v, p), un, xtol=1e-12)
        assert np.abs(U - ref[None]).max() <= 1e-10 * np.abs(ref).max()
        assert np.ptp(U, axis=0).max() <= 1e-10 * np.abs(ref).max()


def _ode_rhs(p):
    def f(t, v):
        return O.reaction(v, p)
    return f


def test_backward_euler_first_order_against_dop853():
    """The homogeneous PDE recursion converges at order 1 in dt to a high-order
    ODE solution (Table order_time reports p = 1 for backward Euler)."""
    gold = _gold("convergence_orders.json")
    p = _ode_params()
    xy, tri = I.structured_mesh(3)
    U0 = I.uniform_ic(len(xy), 2000.0, 0.1)
    T = 12.0
    ref = solve_ivp(_ode_rhs(p), (0, T), U0[0], method="DOP853", rtol=1e-12, atol=1e-10).y[:, -1]
    errs = []
    for dt in (0.4, 0.2, 0.1):
        U, _ = O.run(xy, tri, p, dt, U0, int(round(T / dt)), rtol=1e-13)
        errs.append(np.linalg.norm(U[0] - ref) / np.linalg.norm(ref))
    orders = [math.log(errs[k] / errs[k + 1], 2.0) for k in range(len(errs) - 1)]
    for o in orders:
        assert abs(o - gold["temporal_order"]) < gold["tolerance_time"], orders


def test_ode_closed_form_identities():
    """Integrated forms of Eq. seird1-5 at constant N (alpha = mu = 0):
    ln(s0/s) = kappa (beta_I int i + beta_E int e), d - d0 = gamma_D int i,
    (s+e) - (s0+e0) = -(sigma+gamma_E) int e, r - r0 = gamma_E int e + gamma_R int i,
    and N constant.  Checked on a DOP853 solution of the oracle's reaction()."""
    p = _ode_params()
    N0 = 2000.0
    v0 = np.array([1800.0, 50.0, 150.0, 0.0, 0.0])

    def f(t, w):
        u = w[:5]
        return np.concatenate([O.reaction(u, p), [u[1], u[2]]])

    sol = solve_ivp(f, (0, 40.0), np.concatenate([v0, [0.0, 0.0]]), method="DOP853", rtol=1e-12, atol=1e-9)
    s, e, i, r, d, Ie, Ii = sol.y[:, -1]
    kappa = 1.0 - p.A / N0
    assert abs(s + e + i + r + d - N0) < 1e-8 * N0
    assert abs(math.log(v0[0] / s) - kappa * (p.beta_i * Ii + p.beta_e * Ie)) < 1e-9
    assert abs((d - v0[4]) - p.gamma_d * Ii) < 1e-8 * N0
    assert abs((s + e) - (v0[0] + v0[1]) + (p.sigma + p.gamma_e) * Ie) < 1e-8 * N0
    assert abs((r - v0[3]) - (p.gamma_e * Ie + p.gamma_r * Ii)) < 1e-8 * N0


# ---------------------------------------------------------------------------
# manufactured solution: spatial order 2 (Appendix B.1 / B.3)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("variant", ["paper", "diffusive"])
def test_mms_spatial_order_two(variant):
    from tests.mms_helpers import build_load, l2_error
    gold = _gold("convergence_orders.json")
    p = I.params_square(A=100.0)  # Appendix B.3: Table 1 square values with A = 100
    dt = 1.0
    if variant == "diffusive":
        p = I.params_square(A=100.0, nu=(4e-4, 6e-4, 2e-4, 5e-4))
    exact, forcing = build_load(p, dt, 0.0)
    errs = []
    for nside in (9, 17, 33):
        xy, tri = I.structured_mesh(nside)
        U0 = exact(xy, 0.0)
        U1, info = O.newton_step(xy, tri, p, dt, U0, rtol=1e-12, forcing=forcing)
        assert info["converged"]
        e, ref = l2_error(xy, tri, U1, exact, dt)
        errs.append(e.sum() / ref.sum())
    orders = [math.log(errs[k] / errs[k + 1], 2.0) for k in range(len(errs) - 1)]
    assert abs(orders[-1] - gold["spatial_order"]) < gold["tolerance_space"], (errs, orders)


# ---------------------------------------------------------------------------
# Jacobian and brute-force Newton
# ---------------------------------------------------------------------------

def test_jacobian_matches_central_differences():
    xy, tri, _ = I.irregular_mesh(21, 60)
    rng = np.random.default_rng(4)
    p = I.params_square(beta_e=2.5e-4, alpha=0.01, mu=0.003, nu=(3e-3, 2e-3, 1e-3, 4e-3))
    U = rng.uniform(200, 900, (len(xy), 5))
    Un = rng.uniform(200, 900, (len(xy), 5))
    bf = I.smooth_field(xy, 9)
    dt = 0.7
    J = O.jacobian(xy, tri, p, dt, U, bfield=bf).toarray()
    x = U.ravel()
    for k in rng.choice(x.size, 40, replace=False):
        h = 1e-5 * abs(x[k])
        xp, xm = x.copy(), x.copy()
        xp[k] += h
        xm[k] -= h
        col = (O.residual(xy, tri, p, dt, xp.reshape(U.shape), Un, bf).ravel()
               - O.residual(xy, tri, p, dt, xm.reshape(U.shape), Un, bf).ravel()) / (2 * h)
        assert np.abs(col - J[:, k]).max() <= 1e-6 * max(np.abs(J[:, k]).max(), 1e-300)


def test_brute_force_dense_newton_matches_sparse_newton():
    wl = I.square_workload(7)
    p = wl.params
    U_s, info = O.newton_step(wl.xy, wl.tri, p, wl.dt, wl.U0, rtol=1e-13)
    U_d = O.dense_fd_newton_step(wl.xy, wl.tri, p, wl.dt, wl.U0, rtol=1e-13)
    for c in range(5):
        ref = np.linalg.norm(U_s[:, c])
        if ref > 0:
            assert np.linalg.norm(U_d[:, c] - U_s[:, c]) <= 1e-11 * ref


def test_square_workload_symmetry():
    """The c1 mesh and state are symmetric under (x,y)->(y,x) and (x,y)->(1-x,1-y)."""
    wl = I.square_workload(17)
    U, _ = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 2)
    n = 17
    idx = np.arange(n * n).reshape(n, n)  # [j, i]
    sw = idx.T.ravel()
    rot = idx[::-1, ::-1].ravel()
    scale = np.abs(U).max()
    assert np.abs(U - U[sw]).max() <= 1e-10 * scale
    assert np.abs(U - U[rot]).max() <= 1e-10 * scale


# ---------------------------------------------------------------------------
# BSR, ILU(0), RAS and the coarse space (Section 3)
# ---------------------------------------------------------------------------

def test_bsr_spmv_matches_dense():
    rp, col, val = I.random_bsr(40, 35, 6, seed=2)
    x = np.random.default_rng(3).standard_normal(5 * 35)
    A = np.zeros((200, 175))
    for i in range(40):
        for k in range(rp[i], rp[i + 1]):
            A[5 * i:5 * i + 5, 5 * col[k]:5 * col[k] + 5] = val[k]
    assert np.allclose(O.bsr_spmv(rp, col, val, x), A @ x, rtol=1e-14, atol=1e-12)


def _assembled(nside=9, seed=0):
    wl = I.square_workload(nside)
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0)
    return wl, O.to_bsr(J)


def test_block_ilu0_reproduces_matrix_on_its_pattern():
    """Defining property of ILU(0): (L U)_ij = A_ij for every (i, j) in the pattern."""
    wl, (rp, col, val) = _assembled(6)
    Fk = O.block_ilu0(rp, col, val)
    n = len(rp) - 1
    Ld = np.eye(5 * n)
    Ud = np.zeros((5 * n, 5 * n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            j = col[k]
            if j < i:
                Ld[5 * i:5 * i + 5, 5 * j:5 * j + 5] = Fk[k]
            else:
                Ud[5 * i:5 * i + 5, 5 * j:5 * j + 5] = Fk[k]
    P = Ld @ Ud
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            j = col[k]
            blk = P[5 * i:5 * i + 5, 5 * j:5 * j + 5]
            assert np.abs(blk - val[k]).max() <= 1e-11 * np.abs(val).max()
    r = np.random.default_rng(0).standard_normal(5 * n)
    z = O.block_ilu0_solve(rp, col, Fk, r)
    assert np.allclose(Ld @ (Ud @ z), r, atol=1e-9)


def _dense_factors(rp, col, Fk):
    n = len(rp) - 1
    Ld = np.eye(5 * n)
    Ud = np.zeros((5 * n, 5 * n))
    for i in range(n):
        for k in range(rp[i], rp[i + 1]):
            j = col[k]
            (Ld if j < i else Ud)[5 * i:5 * i + 5, 5 * j:5 * j + 5] = Fk[k]
    return Ld, Ud


def _fill_path_levels(rp, col):
    """Level of every (i, j) from its fill paths (Hysom and Pothen, SIAM J. Sci.
    Comput. 22 (2001)): a path i = v_0, ..., v_l = j of the matrix graph whose
    interior vertices are all numbered below min(i, j) gives (i, j) the level
    l - 1; the least such level wins.  Brute force: one breadth-first search per
    (i, j) through the vertices below min(i, j)."""
    n = len(rp) - 1
    adj = [set(int(c) for c in col[rp[i]:rp[i + 1]]) - {i} for i in range(n)]
    lev = {}
    for i in range(n):
        for j in range(n):
            if i == j:
                lev[i, j] = 0
                continue
            lo = min(i, j)
            dist = {i: 0}
            front = [i]
            best = None
            while front and best is None:
                nxt = []
                for v in front:
                    for w in adj[v]:
                        if w == j:
                            best = dist[v] + 1
                        elif w < lo and w not in dist:
                            dist[w] = dist[v] + 1
                            nxt.append(w)
                front = nxt
            if best is not None:
                lev[i, j] = best - 1
    return lev


@pytest.mark.parametrize("k", [1, 2, 3])
def test_iluk_levels_are_the_fill_path_levels(k):
    """The symbolic ILU(k) pattern and levels equal the fill-path characterisation
    (an independent, graph-theoretic definition) on an irregular 5x5-block pattern."""
    wl, (rp, col, val) = _assembled(6)
    # a non-geometric row order, so that fill is not confined to a band
    perm = np.random.default_rng(3).permutation(len(rp) - 1)
    A = sp.bsr_matrix((val, col, rp), shape=(5 * (len(rp) - 1),) * 2).tocsr()
    idx = (5 * perm[:, None] + np.arange(5)).ravel()
    rp2, col2, val2 = O.to_bsr(A[idx][:, idx])
    lev = O.iluk_levels(rp2, col2, k)
    ref = _fill_path_levels(rp2, col2)
    n = len(rp2) - 1
    for i in range(n):
        want = {j: ref[i, j] for j in range(n) if (i, j) in ref and ref[i, j] <= k}
        assert lev[i] == want, i
    # the pattern grows with k and ILU(0) is the matrix's own pattern
    lev0 = O.iluk_levels(rp2, col2, 0)
    assert all(set(lev0[i]) == set(int(c) for c in col2[rp2[i]:rp2[i + 1]]) for i in range(n))
    assert sum(len(r) for r in lev) > sum(len(r) for r in lev0)


@pytest.mark.parametrize("k", [1, 2])
def test_block_iluk_reproduces_matrix_on_its_pattern(k):
    """Defining property of an incomplete factorisation on a pattern: (L U)_ij = A_ij for
    every (i, j) the pattern holds (fill blocks included, where A_ij = 0); off the pattern
    L U differs from A."""
    wl, (rp, col, val) = _assembled(6)
    n = len(rp) - 1
    A = sp.bsr_matrix((val, col, rp), shape=(5 * n, 5 * n)).toarray()
    frp, fcol, Fk = O.block_iluk(rp, col, val, k)
    assert len(fcol) > len(col)
    Ld, Ud = _dense_factors(frp, fcol, Fk)
    P = Ld @ Ud
    scale = np.abs(val).max()
    on = np.zeros((n, n), dtype=bool)
    for i in range(n):
        for q in range(frp[i], frp[i + 1]):
            j = fcol[q]
            on[i, j] = True
            assert np.abs(P[5 * i:5 * i + 5, 5 * j:5 * j + 5] - A[5 * i:5 * i + 5, 5 * j:5 * j + 5]).max() <= 1e-11 * scale
    off = max(np.abs(P - A)[5 * i:5 * i + 5, 5 * j:5 * j + 5].max() for i in range(n) for j in range(n) if not on[i, j])
    assert off > 1e-8 * scale
    r = np.random.default_rng(0).standard_normal(5 * n)
    z = O.block_ilu0_solve(frp, fcol, Fk, r)
    assert np.allclose(Ld @ (Ud @ z), r, atol=1e-9)


def test_block_iluk_limits():
    """k = 0 is block ILU(0) (the same operations, bit for bit); with every level
    allowed nothing is dropped and the factors are the exact block LU: L U = A and
    the solve is A^{-1}, so RAS with one subdomain and ILU(n) is the exact inverse."""
    wl, (rp, col, val) = _assembled(5)
    n = len(rp) - 1
    frp, fcol, F0 = O.block_iluk(rp, col, val, 0)
    assert np.array_equal(frp, rp) and np.array_equal(fcol, col)
    assert np.array_equal(F0, O.block_ilu0(rp, col, val))
    A = sp.bsr_matrix((val, col, rp), shape=(5 * n, 5 * n)).toarray()
    frp, fcol, Fn = O.block_iluk(rp, col, val, n)
    Ld, Ud = _dense_factors(frp, fcol, Fn)
    assert np.abs(Ld @ Ud - A).max() <= 1e-11 * np.abs(A).max()
    r = np.random.default_rng(2).standard_normal(5 * n)
    x = np.linalg.solve(A, r)
    assert np.allclose(O.block_ilu0_solve(frp, fcol, Fn, r), x, rtol=1e-9, atol=1e-12 * np.abs(x).max())
    owner = np.zeros(n, dtype=np.int32)
    z = O.ras_apply(rp, col, val, owner, 0, r, coarse=False, ilu_fill=n)
    assert np.allclose(z, x, rtol=1e-9, atol=1e-12 * np.abs(x).max())


def _chain_bsr(n, seed=0):
    rng = np.random.default_rng(seed)
    rp = [0]
    col = []
    val = []
    for i in range(n):
        for j in (i - 1, i, i + 1):
            if 0 <= j < n:
                col.append(j)
                b = rng.standard_normal((5, 5))
                if j == i:
                    b += 12 * np.eye(5)
                val.append(b)
        rp.append(len(col))
    return np.array(rp, dtype=np.int32), np.array(col, dtype=np.int32), np.array(val)


def test_ilu0_exact_on_block_tridiagonal_and_single_subdomain_ras_is_inverse():
    rp, col, val = _chain_bsr(12)
    A = sp.bsr_matrix((val, col, rp), shape=(60, 60)).toarray()
    r = np.random.default_rng(1).standard_normal(60)
    Fk = O.block_ilu0(rp, col, val)
    assert np.allclose(O.block_ilu0_solve(rp, col, Fk, r), np.linalg.solve(A, r), rtol=1e-10, atol=1e-12)
    owner = np.zeros(12, dtype=np.int32)
    z = O.ras_apply(rp, col, val, owner, 1, r, coarse=False)
    assert np.allclose(z, np.linalg.solve(A, r), rtol=1e-10, atol=1e-12)
    # with an exact subdomain solve both two-level forms are the inverse too: the smoother
    # after the coarse correction removes whatever residual the correction leaves
    owner2 = np.repeat(np.arange(2, dtype=np.int32), 6)
    for mode in (True, "hybrid"):
        zz = O.ras_apply(rp, col, val, owner, 1, r, multiplicative=mode, coarse_owner=owner2)
        assert np.allclose(zz, np.linalg.solve(A, r), rtol=1e-10, atol=1e-12), mode


def test_overlap_layers_and_partition_of_unity():
    rp, col, val = _chain_bsr(10)
    owner = np.array([0] * 5 + [1] * 5, dtype=np.int32)
    owned, over = O.overlap_sets(rp, col, owner, 2)
    assert list(over[0]) == list(range(7)) and list(over[1]) == list(range(3, 10))
    # RAS with identity "subdomain solves" sums to the identity: every node owned once
    counts = np.zeros(10, dtype=int)
    for q in range(2):
        counts[owned[q]] += 1
    assert (counts == 1).all()


def test_coarse_space_projection_and_galerkin_matrix():
    rp, col, val = _chain_bsr(9)
    owner = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2], dtype=np.int32)
    Ac, Z = O.coarse_matrix(rp, col, val, owner)
    r = np.random.default_rng(5).standard_normal(45)
    zr = Z.T @ r
    for q in range(3):
        for c in range(5):
            assert abs(zr[5 * q + c] - r.reshape(9, 5)[owner == q, c].sum()) < 1e-13
    # Galerkin entries are sums of the owned block entries
    A = sp.bsr_matrix((val, col, rp), shape=(45, 45)).toarray()
    for (pq, qq) in [(0, 0), (0, 1), (1, 2)]:
        for c in range(5):
            for c2 in range(5):
                ref = sum(A[5 * i + c, 5 * j + c2] for i in np.nonzero(owner == pq)[0] for j in np.nonzero(owner == qq)[0])
                assert abs(Ac[5 * pq + c, 5 * qq + c2] - ref) < 1e-12
    assert np.all(Ac[0:5, 10:15] == 0)  # subdomains 0 and 2 do not touch


def test_ras_is_a_good_preconditioner_for_the_step_jacobian():
    """Sanity: on the c1 Jacobian, RAS+coarse reduces the residual of a GMRES
    iteration count well below the unpreconditioned one (iterations only, the
    root never depends on it)."""
    import scipy.sparse.linalg as spla
    wl, (rp, col, val) = _assembled(9)
    n = len(rp) - 1
    A = sp.bsr_matrix((val, col, rp), shape=(5 * n, 5 * n)).tocsr()
    b = np.random.default_rng(0).standard_normal(5 * n)
    owner = wl.owner
    M = spla.LinearOperator(A.shape, lambda r: O.ras_apply(rp, col, val, owner, 1, r, coarse=True))
    its = {"pc": 0, "none": 0}

    def cb_pc(_):
        its["pc"] += 1

    def cb_none(_):
        its["none"] += 1

    spla.gmres(A, b, M=M, rtol=1e-10, restart=60, maxiter=5, callback=cb_pc, callback_type="pr_norm")
    spla.gmres(A, b, rtol=1e-10, restart=60, maxiter=5, callback=cb_none, callback_type="pr_norm")
    assert its["pc"] < its["none"]


def test_table1_parameters_golden():
    g = _gold("table1_parameters.json")
    ps = I.params_square()
    assert ps.A == g["square"]["A"] and ps.beta_i == g["square"]["beta_i"]
    assert ps.nu == (g["square"]["nu_S"], g["square"]["nu_E"], g["square"]["nu_I"], g["square"]["nu_R"])
    assert abs(ps.gamma_r - g["square"]["gamma_r"]) < 1e-17 and abs(ps.sigma - g["square"]["sigma"]) < 1e-17
    po = I.params_ontario(2.0)
    assert po.A == g["ontario"]["A"] and po.nu[2] == g["ontario"]["nu_I"]
    assert abs(po.gamma_d - g["ontario"]["gamma_d"]) < 1e-17


def test_multiplicative_two_grid_matches_the_expanded_operator():
    """Eq. RAS_2L: the three-step correction equals P5 = P1 + P2 + P3 - P2 A P1
    - P3 A P1 - P3 A P2 + P3 A P2 A P1 with P1 = P3 = M_RAS^{-1}, P2 = Q."""
    wl, (rp, col, val) = _assembled(7)
    n = len(rp) - 1
    A = sp.bsr_matrix((val, col, rp), shape=(5 * n, 5 * n)).toarray()
    owner = I.box_partition(wl.xy, 2, 2)
    r = np.random.default_rng(2).standard_normal(5 * n)
    Mras = np.column_stack([O.ras_apply(rp, col, val, owner, 1, e, coarse=False) for e in np.eye(5 * n)])
    Ac, Z = O.coarse_matrix(rp, col, val, owner)
    Q = Z.toarray() @ np.linalg.solve(Ac, Z.T.toarray())
    P1 = P3 = Mras
    P2 = Q
    P5 = P1 + P2 + P3 - P2 @ A @ P1 - P3 @ A @ P1 - P3 @ A @ P2 + P3 @ A @ P2 @ A @ P1
    z = O.ras_apply(rp, col, val, owner, 1, r, multiplicative=True)
    assert np.allclose(z, P5 @ r, rtol=1e-10, atol=1e-12 * np.abs(P5 @ r).max())


# ---------------------------------------------------------------------------
# sampled residual and the restricted prolongation of Eq. RAS
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("rule", ["deg5", "vertex"])
def test_residual_at_nodes_equals_the_whole_mesh_residual(rule):
    """F at a node list from only the triangles incident to those nodes equals the
    whole-mesh F at the same nodes (Eq. weakform: row i of F integrates over the
    support of phi_i only).  Nodes include boundary nodes, corners of the
    structured square, interior nodes and unsorted, repeated entries."""
    rng = np.random.default_rng(11)
    xy, tri, _ = I.irregular_mesh(5, 900)
    sq_xy, sq_tri = I.structured_mesh(9)
    p = I.params_ontario(40.0)
    for xyv, triv in ((xy, tri), (sq_xy, sq_tri)):
        n = len(xyv)
        U = 1.0 + rng.random((n, 5)) * np.array([30.0, 2.0, 2.0, 1.0, 0.5])
        Un = U * (1.0 + 0.05 * rng.standard_normal((n, 5)))
        bf = 0.5 + rng.random(n)
        # boundary nodes: endpoints of edges used by exactly one triangle
        e = np.sort(np.concatenate([triv[:, [0, 1]], triv[:, [1, 2]], triv[:, [2, 0]]]), axis=1)
        ue, cnt = np.unique(e, axis=0, return_counts=True)
        bnd = np.unique(ue[cnt == 1])
        inner = np.setdiff1d(np.arange(n), bnd)
        corners = [int(np.argmin(xyv[:, 0] + xyv[:, 1])), int(np.argmax(xyv[:, 0] + xyv[:, 1])),
                   int(np.argmin(xyv[:, 0] - xyv[:, 1])), int(np.argmax(xyv[:, 0] - xyv[:, 1]))]
        nodes = np.concatenate([rng.choice(bnd, 12, replace=False), corners, rng.choice(inner, 12, replace=False),
                                [corners[0], int(inner[0])]])
        full = O.residual(xyv, triv, p, 0.5, U, Un, bf, rule)
        part = O.residual_at_nodes(xyv, triv, p, 0.5, U, Un, nodes, bfield=bf, rule=rule)
        scale = np.abs(full).max()
        assert part.shape == (len(nodes), 5)
        assert np.abs(part - full[nodes]).max() <= 1e-14 * scale
        # a wrong triangle selection is visible: dropping one incident triangle changes the row
        k = int(inner[len(inner) // 2])
        drop = np.nonzero((triv == k).any(axis=1))[0][0]
        keep = np.delete(np.arange(len(triv)), drop)
        other = O.residual(xyv, triv[keep], p, 0.5, U, Un, bf, rule)
        assert np.abs(other[k] - full[k]).max() > 1e-6 * scale


def _chain_parts(nblk, sizes):
    """Owner array of a chain split into consecutive parts of the given sizes."""
    assert sum(sizes) == nblk
    return np.repeat(np.arange(len(sizes), dtype=np.int32), sizes)


def _dense_schwarz(A, owner, delta, restricted):
    """sum_p R_p^T D_p (R_p A R_p^T)^{-1} R_p for a chain of 5x5 blocks, written
    out densely (Eq. ASM, Eq. RAS): subdomain p covers its owned blocks and
    delta neighbours on either side; D_p keeps its owned rows (RAS) or all of
    them (ASM, restricted=False)."""
    nb = len(owner)
    M = np.zeros_like(A)
    for q in range(int(owner.max()) + 1):
        own = np.nonzero(owner == q)[0]
        lo, hi = max(0, own.min() - delta), min(nb, own.max() + 1 + delta)
        blocks = np.arange(lo, hi)
        idx = (5 * blocks[:, None] + np.arange(5)).ravel()
        inv = np.linalg.inv(A[np.ix_(idx, idx)])
        keep = np.isin(blocks, own) if restricted else np.ones(len(blocks), dtype=bool)
        rows = (5 * blocks[keep][:, None] + np.arange(5)).ravel()
        sel = np.repeat(keep, 5)
        M[np.ix_(rows, idx)] += inv[sel]
    return M


@pytest.mark.parametrize("sizes,delta", [((4, 5, 3), 1), ((3, 3, 4, 2), 2), ((6, 6), 2)])
def test_multi_subdomain_ras_against_dense_restricted_schwarz(sizes, delta):
    """Eq. RAS with several overlapping subdomains: on a block-tridiagonal chain
    (block ILU(0) of a block-tridiagonal matrix has no dropped fill, so each
    subdomain solve is exact) the oracle's RAS apply equals the dense
    sum_p R_p^T D_p (R_p A R_p^T)^{-1} R_p r with D_p the owned rows, the ASM
    form (every overlap row written) differs from it, and the additive and
    multiplicative two-level forms (Section 3.1, Eq. RAS_2L) equal their dense
    counterparts with a hand-built constant coarse space."""
    nb = sum(sizes)
    rp, col, val = _chain_bsr(nb, seed=len(sizes) + delta)
    A = sp.bsr_matrix((val, col, rp), shape=(5 * nb, 5 * nb)).toarray()
    owner = _chain_parts(nb, sizes)
    r = np.random.default_rng(7).standard_normal(5 * nb)
    Mras = _dense_schwarz(A, owner, delta, True)
    Masm = _dense_schwarz(A, owner, delta, False)
    z = O.ras_apply(rp, col, val, owner, delta, r, coarse=False)
    ref = Mras @ r
    assert np.abs(z - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(Masm @ r - ref).max() > 1e-3 * np.abs(ref).max()
    # constant coarse space by hand: Z[5 i + c, 5 q + c] = 1 for the blocks i that q owns
    P = len(sizes)
    Z = np.zeros((5 * nb, 5 * P))
    for i in range(nb):
        Z[5 * i:5 * i + 5, 5 * owner[i]:5 * owner[i] + 5] = np.eye(5)
    Q = Z @ np.linalg.solve(Z.T @ A @ Z, Z.T)
    z2 = O.ras_apply(rp, col, val, owner, delta, r, coarse=True)
    ref2 = (Mras + Q) @ r
    assert np.abs(z2 - ref2).max() <= 1e-11 * np.abs(ref2).max()
    u = Mras @ r
    u = u + Q @ (r - A @ u)
    u = u + Mras @ (r - A @ u)
    z3 = O.ras_apply(rp, col, val, owner, delta, r, multiplicative=True)
    assert np.abs(z3 - u).max() <= 1e-11 * np.abs(u).max()
