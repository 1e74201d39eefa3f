"""CPU oracle for one backward-Euler step of the SEIRD reaction-diffusion system.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline legs of ``bench.py`` may import this module.  The product path
(the CUDA library and its binding) never calls it, and it shares no code with
that path: every formula here is restated from the paper in plain FP64
NumPy/SciPy, slowly and without blocking or fusion.

What it computes (the discrete system both sides solve):

  PDE, Eq. seird1-5 with N = s+e+i+r+d (Eq. N); vector form Eq.
  vec_component1/2; backward Euler, Eq. timediscrete; weak form with
  homogeneous Neumann data, Eq. weakform; P1 triangles (Section 2.2).  For node
  i and compartment c, with u_h = sum_j U_j phi_j and U^n the previous step:

    F_ic(U) = (u_c - u_c^n, phi_i)
              + dt * nubar_c * (N_h grad u_c, grad phi_i)
              - dt * (R_c(u_h), phi_i)                       = 0

  where R_c is the reaction part of Eq. seird1-5 (= the rows of B(u)u) and
  nubar_D = 0.  Readings of points the paper leaves open:
    * the mass term is integrated exactly (consistent mass);
    * the diffusion term is integrated exactly: N_h is linear and the
      gradients are constant on a triangle, so it equals
      |T| * mean_T(N) * grad u_c . grad phi_i;
    * the reaction term uses Radon's degree-5 seven-point rule (the default
      triangle rule of FreeFEM, which the paper ran, Section 3.2), or the
      three-vertex rule when asked;
    * the per-node transmission multiplier b (default 1) scales beta_I and
      beta_E and is interpolated with P1 (Eq. beta_ie with a time-frozen
      beta(t)).
  Newton's method on this system (Section 2.2 names it as the coupled
  alternative to the Picard iteration; both have this system's root as fixed
  point) with an exact Jacobian, a sparse direct solve (SuperLU) and
  backtracking on ||F||_2.

Component functions used for kernel parity: the 5x5-block BSR form of the
Jacobian and its product with a vector, the restricted additive Schwarz
preconditioner of Eq. RAS with block ILU(0) or ILU(k) subdomain solves (the
paper leaves the subdomain solver open; ILU(k) by levels of fill as in Saad,
Iterative Methods for Sparse Linear Systems, Section 10.3.3), and the additive
coarse correction Q = Z A_c^{-1} Z^T of Section 3.1 with the per-subdomain,
per-compartment constant coarse space Z.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

NC = 5
S, E, I, R, D = range(5)


# ---------------------------------------------------------------------------
# quadrature and geometry
# ---------------------------------------------------------------------------

def quad_rule(rule: str = "deg5"):
    """Barycentric points [q, 3] and weights [q] (weights sum to 1).

    deg5: Radon's seven-point rule, exact for polynomials of degree <= 5
    (centroid; two orbits of three points at distances set by sqrt(15)).
    vertex: the three vertices, weight 1/3 each (exact for degree 1).
    """
    if rule == "deg5":
        r = np.sqrt(15.0)
        a1, b1 = (6.0 - r) / 21.0, (9.0 + 2.0 * r) / 21.0
        a2, b2 = (6.0 + r) / 21.0, (9.0 - 2.0 * r) / 21.0
        w1, w2 = (155.0 - r) / 1200.0, (155.0 + r) / 1200.0
        L = np.array([[1 / 3, 1 / 3, 1 / 3],
                      [b1, a1, a1], [a1, b1, a1], [a1, a1, b1],
                      [b2, a2, a2], [a2, b2, a2], [a2, a2, b2]])
        W = np.array([9.0 / 40.0, w1, w1, w1, w2, w2, w2])
        return L, W
    if rule == "vertex":
        return np.eye(3), np.full(3, 1.0 / 3.0)
    raise ValueError(rule)


def geometry(xy, tri):
    """Triangle areas [m] and P1 basis gradients [m, 3, 2] (constant per triangle)."""
    p = xy[tri]  # [m, 3, 2]
    x0, y0 = p[:, 0, 0], p[:, 0, 1]
    x1, y1 = p[:, 1, 0], p[:, 1, 1]
    x2, y2 = p[:, 2, 0], p[:, 2, 1]
    twoA = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)
    if np.any(twoA <= 0):
        raise ValueError("triangles must be counter-clockwise and non-degenerate")
    g = np.empty((len(tri), 3, 2))
    g[:, 0, 0] = (y1 - y2) / twoA
    g[:, 0, 1] = (x2 - x1) / twoA
    g[:, 1, 0] = (y2 - y0) / twoA
    g[:, 1, 1] = (x0 - x2) / twoA
    g[:, 2, 0] = (y0 - y1) / twoA
    g[:, 2, 1] = (x1 - x0) / twoA
    return 0.5 * twoA, g


# ---------------------------------------------------------------------------
# the model's reaction terms (Eq. seird1-5, rows of Eq. vec_component2)
# ---------------------------------------------------------------------------

def reaction(u, p, b=1.0):
    """R(u) [..., 5] for states u [..., 5]; b multiplies beta_I and beta_E."""
    s, e, i, r, d = (u[..., k] for k in range(5))
    N = s + e + i + r + d
    kappa = 1.0 - p.A / N  # Allee factor (1 - A/N)
    bi = p.beta_i * b
    be = p.beta_e * b
    out = np.empty(u.shape)
    out[..., S] = p.alpha * N - kappa * bi * s * i - kappa * be * s * e - p.mu * s
    out[..., E] = kappa * bi * s * i + kappa * be * s * e - p.sigma * e - p.gamma_e * e - p.mu * e
    out[..., I] = p.sigma * e - p.gamma_r * i - p.gamma_d * i - p.mu * i
    out[..., R] = p.gamma_e * e + p.gamma_r * i - p.mu * r
    out[..., D] = p.gamma_d * i
    return out


def reaction_jacobian(u, p, b=1.0):
    """dR_c/du_c' [..., 5, 5], differentiated by hand from ``reaction``."""
    s, e, i, r, d = (u[..., k] for k in range(5))
    N = s + e + i + r + d
    kappa = 1.0 - p.A / N
    dkappa = p.A / (N * N)  # d kappa / d u_c for every c (dN/du_c = 1)
    bi = p.beta_i * b
    be = p.beta_e * b
    lam = bi * i + be * e  # force of infection per susceptible
    dT = np.empty(u.shape)
    for c in range(5):
        dT[..., c] = dkappa * s * lam
    dT[..., S] += kappa * lam
    dT[..., E] += kappa * s * be
    dT[..., I] += kappa * s * bi
    Jr = np.zeros(u.shape + (5,))
    for c in range(5):
        Jr[..., S, c] = p.alpha - dT[..., c]
        Jr[..., E, c] = dT[..., c]
    Jr[..., S, S] -= p.mu
    Jr[..., E, E] -= p.sigma + p.gamma_e + p.mu
    Jr[..., I, E] = p.sigma
    Jr[..., I, I] = -(p.gamma_r + p.gamma_d + p.mu)
    Jr[..., R, E] = p.gamma_e
    Jr[..., R, I] = p.gamma_r
    Jr[..., R, R] = -p.mu
    Jr[..., D, I] = p.gamma_d
    return Jr


# ---------------------------------------------------------------------------
# residual and Jacobian of the discrete system (Eq. weakform)
# ---------------------------------------------------------------------------

def _nu5(p):
    return np.array([p.nu[0], p.nu[1], p.nu[2], p.nu[3], 0.0])


def residual(xy, tri, p, dt, U, Un, bfield=None, rule="deg5", forcing=None):
    """F [n, 5] of the discrete system.

    ``forcing`` (manufactured-solution tests only) is an optional callable
    ``forcing(xy, tri) -> G [n, 5]``; its result is subtracted (G holds the
    already dt-scaled load integrals).
    """
    n = len(xy)
    area, g = geometry(xy, tri)
    nu = _nu5(p)
    F = np.zeros((n, NC))
    Ue = U[tri]     # [m, 3, 5]
    dUe = Ue - Un[tri]
    # consistent mass: (phi_a, phi_b)_T = |T| (1 + delta_ab) / 12
    Me = area[:, None, None] * (np.ones((3, 3)) + np.eye(3))[None] / 12.0
    np.add.at(F, tri, np.einsum("tab,tbc->tac", Me, dUe))
    # diffusion: dt nubar_c |T| mean_T(N) grad u_c . grad phi_a
    Nbar = Ue.sum(axis=2).mean(axis=1)  # [m]
    gu = np.einsum("tbc,tbx->tcx", Ue, g)  # grad u_c [m, 5, 2]
    diff = np.einsum("tcx,tax->tac", gu, g) * (area * Nbar)[:, None, None] * nu[None, None, :]
    np.add.at(F, tri, dt * diff)
    # reaction: - dt |T| sum_q w_q R_c(u(x_q)) phi_a(x_q)
    L, W = quad_rule(rule)
    for q in range(len(W)):
        uq = np.einsum("a,tac->tc", L[q], Ue)
        bq = 1.0 if bfield is None else bfield[tri] @ L[q]
        Rq = reaction(uq, p, bq)
        contrib = (dt * W[q] * area)[:, None, None] * L[q][None, :, None] * Rq[:, None, :]
        np.add.at(F, tri, -contrib)
    if forcing is not None:
        F -= forcing(xy, tri)
    return F


def jacobian(xy, tri, p, dt, U, bfield=None, rule="deg5"):
    """Exact dF/dU as a scipy CSR matrix on the node-major index 5*node + c."""
    n = len(xy)
    m = len(tri)
    area, g = geometry(xy, tri)
    nu = _nu5(p)
    Ue = U[tri]
    Nbar = Ue.sum(axis=2).mean(axis=1)
    gu = np.einsum("tbc,tbx->tcx", Ue, g)
    blocks = np.zeros((m, 3, 3, 5, 5))  # [t, a, b, c, c']
    eye5 = np.eye(5)
    Me = (np.ones((3, 3)) + np.eye(3)) / 12.0
    blocks += (area[:, None, None] * Me[None])[:, :, :, None, None] * eye5
    # diffusion, part 1: d/dU_{b,c'} of N_h (mean over T is 1/3 per vertex, any c')
    gdot = np.einsum("tcx,tax->tac", gu, g)  # grad u_c . grad phi_a
    d1 = dt * nu[None, None, :] * gdot * (area / 3.0)[:, None, None]  # [t, a, c]
    blocks += d1[:, :, None, :, None]
    # diffusion, part 2: mean(N) grad phi_b . grad phi_a on the diagonal c = c'
    K = np.einsum("tax,tbx->tab", g, g) * (area * Nbar)[:, None, None]
    blocks += dt * K[:, :, :, None, None] * np.diag(nu)[None, None, None]
    # reaction
    L, W = quad_rule(rule)
    for q in range(len(W)):
        uq = np.einsum("a,tac->tc", L[q], Ue)
        bq = 1.0 if bfield is None else bfield[tri] @ L[q]
        Jr = reaction_jacobian(uq, p, bq)  # [t, 5, 5]
        wab = np.outer(L[q], L[q])  # phi_a phi_b at x_q
        blocks -= (dt * W[q] * area)[:, None, None, None, None] * wab[None, :, :, None, None] * Jr[:, None, None]
    rows = (5 * tri[:, :, None, None, None] + np.arange(5)[None, None, None, :, None])
    cols = (5 * tri[:, None, :, None, None] + np.arange(5)[None, None, None, None, :])
    rows = np.broadcast_to(rows, blocks.shape).ravel()
    cols = np.broadcast_to(cols, blocks.shape).ravel()
    J = sp.coo_matrix((blocks.ravel(), (rows, cols)), shape=(5 * n, 5 * n)).tocsr()
    J.sum_duplicates()
    return J


# ---------------------------------------------------------------------------
# Newton step and time loop
# ---------------------------------------------------------------------------

class StepInfo(dict):
    pass


def newton_step(xy, tri, p, dt, Un, rtol=1e-12, atol=0.0, maxit=30, ls_maxit=10,
                bfield=None, rule="deg5", forcing=None, linear_solver="splu", U_guess=None):
    """Root of F(.; U^n) = 0 from the guess U^n (Section 2.2): exact-Jacobian
    Newton with a sparse direct solve and backtracking (halving) on ||F||_2.

    Converged when ||F(U^k)||_2 <= rtol * ||F(U^n)||_2 + atol.  Also records the
    paper's update measure eps = ||U^{k+1} - U^k||_2 / ||U^n||_2 (Eq. picardtol).
    """
    U = (Un if U_guess is None else U_guess).copy()
    F = residual(xy, tri, p, dt, U, Un, bfield, rule, forcing)
    f0 = np.linalg.norm(F)
    fn = f0
    info = StepInfo(newton_its=0, ls_halvings=0, f0=f0, hist=[f0], eps=[])
    unorm = np.linalg.norm(Un)
    for it in range(maxit):
        if fn <= rtol * f0 + atol:
            break
        J = jacobian(xy, tri, p, dt, U, bfield, rule)
        if linear_solver == "splu":
            delta = spla.splu(J.tocsc()).solve(-F.ravel())
        else:
            delta = np.linalg.solve(J.toarray(), -F.ravel())
        delta = delta.reshape(U.shape)
        lam = 1.0
        for ls in range(ls_maxit + 1):
            Ut = U + lam * delta
            Ft = residual(xy, tri, p, dt, Ut, Un, bfield, rule, forcing)
            ft = np.linalg.norm(Ft)
            if np.isfinite(ft) and (ft <= (1.0 - 1e-4 * lam) * fn or ls == ls_maxit):
                break
            lam *= 0.5
            info["ls_halvings"] += 1
        info["eps"].append(np.linalg.norm(Ut - U) / unorm)
        U, F, fn = Ut, Ft, ft
        info["hist"].append(fn)
        info["newton_its"] = it + 1
    info["converged"] = bool(fn <= rtol * f0 + atol)
    info["fn"] = fn
    return U, info


def run(xy, tri, p, dt, U0, n_steps, **kw):
    U = U0.copy()
    infos = []
    for _ in range(n_steps):
        U, info = newton_step(xy, tri, p, dt, U, **kw)
        infos.append(info)
    return U, infos


def dense_fd_newton_step(xy, tri, p, dt, Un, rtol=1e-12, maxit=30, h_rel=1e-6, bfield=None, rule="deg5"):
    """Brute force: Newton with a dense central-difference Jacobian and a dense
    LU solve (numpy), for meshes of a few hundred nodes."""
    U = Un.copy()
    n = len(xy)

    def Fv(v):
        return residual(xy, tri, p, dt, v.reshape(n, NC), Un, bfield, rule).ravel()

    F = Fv(U.ravel())
    f0 = np.linalg.norm(F)
    for _ in range(maxit):
        if np.linalg.norm(F) <= rtol * f0:
            break
        x = U.ravel()
        Jd = np.empty((x.size, x.size))
        for k in range(x.size):
            hk = h_rel * max(1.0, abs(x[k]))
            xp = x.copy()
            xm = x.copy()
            xp[k] += hk
            xm[k] -= hk
            Jd[:, k] = (Fv(xp) - Fv(xm)) / (2.0 * hk)
        delta = np.linalg.solve(Jd, -F)
        lam = 1.0
        fn = np.linalg.norm(F)
        for _ in range(11):
            xt = x + lam * delta
            Ft = Fv(xt)
            if np.linalg.norm(Ft) <= (1.0 - 1e-4 * lam) * fn:
                break
            lam *= 0.5
        U = xt.reshape(n, NC)
        F = Ft
    return U


# ---------------------------------------------------------------------------
# sampled residual (for meshes too large for the whole-mesh oracle)
# ---------------------------------------------------------------------------

def residual_at_nodes(xy, tri, p, dt, U, Un, nodes, bfield=None, rule="deg5"):
    """F at the listed nodes only, from the triangles incident to them."""
    nodes = np.asarray(nodes)
    mark = np.zeros(len(xy), dtype=bool)
    mark[nodes] = True
    tsel = np.nonzero(mark[tri].any(axis=1))[0]
    sub = tri[tsel]
    used, inv = np.unique(sub.ravel(), return_inverse=True)
    lt = inv.reshape(sub.shape).astype(np.int64)
    bf = None if bfield is None else bfield[used]
    Fl = residual(xy[used], lt, p, dt, U[used], Un[used], bf, rule)
    pos = np.searchsorted(used, nodes)
    return Fl[pos]


# ---------------------------------------------------------------------------
# 5x5-block views and the preconditioner (Section 3, Eq. RAS)
# ---------------------------------------------------------------------------

def to_bsr(J):
    """(row_ptr, col, val[nnzb, 5, 5]) of a CSR matrix on the 5*node + c index,
    columns sorted within each block row."""
    B = sp.bsr_matrix(J, blocksize=(5, 5))
    B.sort_indices()
    return B.indptr.astype(np.int32), B.indices.astype(np.int32), np.array(B.data)


def bsr_spmv(row_ptr, col, val, x):
    """y = A x for a 5x5-block BSR matrix (x, y flat, 5 entries per block row/col)."""
    nrow = len(row_ptr) - 1
    ncol = (x.size // 5)
    A = sp.bsr_matrix((val, col, row_ptr), shape=(5 * nrow, 5 * ncol))
    return A @ x


def node_graph(row_ptr, col):
    """Adjacency lists (excluding self) of the block pattern."""
    nrow = len(row_ptr) - 1
    return [[int(c) for c in col[row_ptr[i]:row_ptr[i + 1]] if c != i] for i in range(nrow)]


def internal_order(owner):
    """Nodes sorted by (owner, node index): the order in which subdomain-local
    unknowns are numbered (and hence the ILU(0) elimination order)."""
    return np.argsort(owner, kind="stable")


def overlap_sets(row_ptr, col, owner, delta):
    """Owned node lists and overlapping node lists (owned plus delta graph layers)."""
    nparts = int(owner.max()) + 1 if len(owner) else 0
    adj = node_graph(row_ptr, col)
    owned = [np.nonzero(owner == q)[0] for q in range(nparts)]
    over = []
    for q in range(nparts):
        cur = set(int(i) for i in owned[q])
        front = set(cur)
        for _ in range(delta):
            nxt = set()
            for i in front:
                for j in adj[i]:
                    if j not in cur:
                        nxt.add(j)
            cur |= nxt
            front = nxt
        over.append(np.array(sorted(cur), dtype=np.int64))
    return owned, over


def block_ilu0(row_ptr, col, val):
    """Block ILU(0) of a 5x5-block BSR matrix in its own row order (IKJ form).

    Returns factor blocks in the same pattern: strictly lower blocks hold L
    (unit block diagonal implied), the diagonal and upper blocks hold U.
    """
    nrow = len(row_ptr) - 1
    F = val.copy()
    pos = [dict((int(col[k]), k) for k in range(row_ptr[i], row_ptr[i + 1])) for i in range(nrow)]
    for i in range(nrow):
        lower = sorted(c for c in pos[i] if c < i)
        for k in lower:
            kk = pos[i][k]
            F[kk] = F[kk] @ np.linalg.inv(F[pos[k][k]])
            for j, kj in pos[k].items():
                if j > k and j in pos[i]:
                    F[pos[i][j]] = F[pos[i][j]] - F[kk] @ F[kj]
    return F


def block_ilu0_solve(row_ptr, col, F, r):
    """Solve (L U) z = r with the factors of ``block_ilu0``."""
    nrow = len(row_ptr) - 1
    y = r.reshape(nrow, 5).copy()
    for i in range(nrow):
        for k in range(row_ptr[i], row_ptr[i + 1]):
            if col[k] < i:
                y[i] -= F[k] @ y[col[k]]
    z = np.zeros_like(y)
    for i in range(nrow - 1, -1, -1):
        acc = y[i].copy()
        dk = None
        for k in range(row_ptr[i], row_ptr[i + 1]):
            if col[k] > i:
                acc -= F[k] @ z[col[k]]
            elif col[k] == i:
                dk = k
        z[i] = np.linalg.solve(F[dk], acc)
    return z.ravel()


def iluk_levels(row_ptr, col, k):
    """Pattern of block ILU(k) by levels of fill (Saad, Iterative Methods for Sparse
    Linear Systems, Section 10.3.3), in the matrix's own row order: for every row a
    dict column -> level.  The row's own blocks have level 0; eliminating with pivot
    row m < i (in increasing m, fill included) gives each block (m, j), j > m, of row
    m's upper part the level lev(i, m) + lev(m, j) + 1, and a block belongs to row i
    when its least level is at most k."""
    n = len(row_ptr) - 1
    lev = []
    for i in range(n):
        row = {int(c): 0 for c in col[row_ptr[i]:row_ptr[i + 1]]}
        done = set()
        while True:
            pending = [c for c in row if c < i and c not in done]
            if not pending:
                break
            m = min(pending)
            done.add(m)
            for j, lmj in lev[m].items():
                if j > m:
                    lv = row[m] + lmj + 1
                    if lv <= k and lv < row.get(j, k + 1):
                        row[j] = lv
        lev.append(row)
    return lev


def block_iluk(row_ptr, col, val, k):
    """Block ILU(k) of a 5x5-block BSR matrix in its own row order (IKJ form on the
    pattern of ``iluk_levels``; fill blocks start at zero).  Returns (row_ptr, col, F)
    of the factors with sorted columns: strictly lower blocks hold L (unit block
    diagonal implied), the diagonal and upper blocks hold U.  k = 0 is ``block_ilu0``."""
    n = len(row_ptr) - 1
    lev = iluk_levels(row_ptr, col, k)
    F = []
    for i in range(n):
        own = {int(col[q]): q for q in range(row_ptr[i], row_ptr[i + 1])}
        F.append({j: (val[own[j]].copy() if j in own else np.zeros((5, 5))) for j in sorted(lev[i])})
    for i in range(n):
        for m in sorted(c for c in F[i] if c < i):
            F[i][m] = F[i][m] @ np.linalg.inv(F[m][m])
            for j, b in F[m].items():
                if j > m and j in F[i]:
                    F[i][j] = F[i][j] - F[i][m] @ b
    rp = np.zeros(n + 1, dtype=np.int64)
    cc, vv = [], []
    for i in range(n):
        cc.extend(F[i].keys())
        vv.extend(F[i].values())
        rp[i + 1] = len(cc)
    return rp, np.array(cc, dtype=np.int64), np.array(vv).reshape(-1, 5, 5)


def submatrix_bsr(row_ptr, col, val, nodes):
    """R_p A R_p^T in BSR form for the ordered node list ``nodes``."""
    loc = {int(g): l for l, g in enumerate(nodes)}
    rp = [0]
    cc = []
    vv = []
    for g in nodes:
        ent = [(loc[int(col[k])], k) for k in range(row_ptr[g], row_ptr[g + 1]) if int(col[k]) in loc]
        ent.sort()
        cc.extend(e[0] for e in ent)
        vv.extend(val[e[1]] for e in ent)
        rp.append(len(cc))
    return (np.array(rp, dtype=np.int64), np.array(cc, dtype=np.int64),
            np.array(vv).reshape(-1, 5, 5))


def coarse_matrix(row_ptr, col, val, owner):
    """A_c = Z^T A Z with Z's column (p, c) the indicator of nodes owned by p in
    compartment c (Section 3.1 Galerkin projection, constant coarse space)."""
    nparts = int(owner.max()) + 1
    n = len(row_ptr) - 1
    Z = sp.coo_matrix((np.ones(5 * n), (np.arange(5 * n), 5 * np.repeat(owner, 5) + np.tile(np.arange(5), n))),
                      shape=(5 * n, 5 * nparts)).tocsr()
    A = sp.bsr_matrix((val, col, row_ptr), shape=(5 * n, 5 * n)).tocsr()
    return (Z.T @ A @ Z).toarray(), Z


def ras_apply(row_ptr, col, val, owner, delta, r, coarse=True, multiplicative=False, coarse_owner=None,
              ilu_fill=0):
    """z = M^{-1} r for the restricted additive Schwarz preconditioner (Eq. RAS)
    with block-ILU(k) subdomain solves (k = ``ilu_fill``; 0 is ILU(0)) on
    R_p A R_p^T (local unknowns numbered by (owner, node index)), plus, if
    ``coarse``, the additive coarse term
    Z A_c^{-1} Z^T r (M_2^{-1} = M_RAS^{-1} + Q, Section 3.1).  ``coarse_owner``
    (default: ``owner``) assigns the nodes to the coarse space's units when
    several subdomains share one unit.

    With ``multiplicative`` the two-grid preconditioner of Eq. RAS_2L instead:
    the three corrections of Eqs. presmoother, coarsecorrection, postsmoother
    with P1 = P3 = M_RAS^{-1} and P2 = Q, each applied to the residual left by
    the previous one (u^0 = 0, f = r).  ``multiplicative="hybrid"`` drops the
    pre-smoother: Q r, then M_RAS^{-1} on the residual it leaves."""
    cown = owner if coarse_owner is None else coarse_owner
    if multiplicative == "hybrid":
        # coarse correction first, then RAS on the residual it leaves: Q r + M_RAS^{-1} (r - A Q r)
        n = len(row_ptr) - 1
        A = sp.bsr_matrix((val, col, row_ptr), shape=(5 * n, 5 * n)).tocsr()
        Ac, Z = coarse_matrix(row_ptr, col, val, cown)
        u = Z @ np.linalg.solve(Ac, Z.T @ r)
        return u + ras_apply(row_ptr, col, val, owner, delta, r - A @ u, coarse=False, ilu_fill=ilu_fill)
    if multiplicative:
        n = len(row_ptr) - 1
        A = sp.bsr_matrix((val, col, row_ptr), shape=(5 * n, 5 * n)).tocsr()
        Ac, Z = coarse_matrix(row_ptr, col, val, cown)
        u = ras_apply(row_ptr, col, val, owner, delta, r, coarse=False, ilu_fill=ilu_fill)  # u^{1/3} = P1 f
        u = u + Z @ np.linalg.solve(Ac, Z.T @ (r - A @ u))                        # u^{2/3} = u + P2 (f - A u)
        u = u + ras_apply(row_ptr, col, val, owner, delta, r - A @ u, coarse=False,
                          ilu_fill=ilu_fill)                                      # u^1 = u + P3 (f - A u)
        return u
    n = len(row_ptr) - 1
    rank = np.empty(n, dtype=np.int64)
    rank[internal_order(owner)] = np.arange(n)
    owned, over = overlap_sets(row_ptr, col, owner, delta)
    z = np.zeros(5 * n)
    rr = r.reshape(n, 5)
    zz = z.reshape(n, 5)
    for q in range(len(owned)):
        nodes = over[q][np.argsort(rank[over[q]], kind="stable")]
        rp, cc, vv = submatrix_bsr(row_ptr, col, val, nodes)
        if ilu_fill:
            rp, cc, Fq = block_iluk(rp, cc, vv, ilu_fill)
        else:
            Fq = block_ilu0(rp, cc, vv)
        zq = block_ilu0_solve(rp, cc, Fq, rr[nodes].ravel()).reshape(-1, 5)
        mine = owner[nodes] == q
        zz[nodes[mine]] = zq[mine]
    if coarse:
        Ac, Z = coarse_matrix(row_ptr, col, val, cown)
        yc = np.linalg.solve(Ac, Z.T @ r)
        z += Z @ yc
    return z
