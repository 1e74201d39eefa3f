"""Manufactured-solution loads for the oracle (Appendix B.1/B.3).

The manufactured solution is the paper's 2-D one, u_c = B sin(10xy + 0.2t) + A_c
(Appendix B.3).  The load is derived symbolically (sympy) from the PDE in its
divergence form (Eq. seird1-5), for ONE backward-Euler step from t0 to t1: with

    f_c = (u_c(t1) - u_c(t0)) / dt - div(nubar_c N grad u_c)(t1) - R_c(u(t1))

and boundary flux g_c = nubar_c N grad u_c . n at t1, the time-discrete problem
started from u(t0) has u(t1) as its exact solution, so the discrete error is the
spatial error alone.  The reaction terms here are written out from Eq. seird1-5
in sympy, independently of the oracle's NumPy code.
"""
import numpy as np
import sympy as sy

from oracle import seird_oracle as O


def mms_solution(B=25.0, offsets=(500.0, 300.0, 200.0, 100.0, 80.0)):
    x, y, t = sy.symbols("x y t", real=True)
    us = [B * sy.sin(10 * x * y + sy.Rational(1, 5) * t) + a for a in offsets]
    return (x, y, t), us


def build_load(p, dt, t0, B=25.0, offsets=(500.0, 300.0, 200.0, 100.0, 80.0)):
    (x, y, t), us = mms_solution(B, offsets)
    s, e, i, r, d = us
    N = s + e + i + r + d
    kap = 1 - sy.Float(p.A) / N
    bi, be = sy.Float(p.beta_i), sy.Float(p.beta_e)
    al, mu = sy.Float(p.alpha), sy.Float(p.mu)
    sig, ge, gr, gd = sy.Float(p.sigma), sy.Float(p.gamma_e), sy.Float(p.gamma_r), sy.Float(p.gamma_d)
    react = [
        al * N - kap * bi * s * i - kap * be * s * e - mu * s,          # Eq. seird1
        kap * bi * s * i + kap * be * s * e - sig * e - ge * e - mu * e,  # Eq. seird2
        sig * e - gr * i - gd * i - mu * i,                               # Eq. seird3
        ge * e + gr * i - mu * r,                                         # Eq. seird4
        gd * i,                                                           # Eq. seird5
    ]
    nus = [sy.Float(v) for v in p.nu] + [sy.Float(0.0)]
    t1 = t0 + dt
    f_exprs, fx_exprs, fy_exprs = [], [], []
    for c in range(5):
        flux_x = nus[c] * N * sy.diff(us[c], x)
        flux_y = nus[c] * N * sy.diff(us[c], y)
        div = sy.diff(flux_x, x) + sy.diff(flux_y, y)
        f = (us[c].subs(t, t1) - us[c].subs(t, t0)) / dt - div.subs(t, t1) - react[c].subs(t, t1)
        f_exprs.append(f)
        fx_exprs.append(flux_x.subs(t, t1))
        fy_exprs.append(flux_y.subs(t, t1))
    f_fun = sy.lambdify((x, y), f_exprs, "numpy")
    fx_fun = sy.lambdify((x, y), fx_exprs, "numpy")
    fy_fun = sy.lambdify((x, y), fy_exprs, "numpy")
    u_fun = sy.lambdify((x, y, t), us, "numpy")

    def exact(xy, tt):
        v = u_fun(xy[:, 0], xy[:, 1], tt)
        return np.stack([np.broadcast_to(np.asarray(vc, dtype=float), (len(xy),)) for vc in v], axis=1)

    def forcing(xy, tri):
        n = len(xy)
        G = np.zeros((n, 5))
        area, _ = O.geometry(xy, tri)
        L, W = O.quad_rule("deg5")
        P = xy[tri]
        for q in range(len(W)):
            xq = np.einsum("a,tax->tx", L[q], P)
            fv = np.stack([np.broadcast_to(np.asarray(v, dtype=float), (len(tri),))
                           for v in f_fun(xq[:, 0], xq[:, 1])], axis=1)
            np.add.at(G, tri, (dt * W[q] * area)[:, None, None] * L[q][None, :, None] * fv[:, None, :])
        # boundary edges (used by one triangle), oriented as in their CCW triangle
        e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
        key = np.sort(e, axis=1)
        k = key[:, 0].astype(np.int64) * n + key[:, 1]
        uniq, inv, cnt = np.unique(k, return_inverse=True, return_counts=True)
        be_ = e[cnt[inv] == 1]
        gl_x, gl_w = np.polynomial.legendre.leggauss(5)
        tq = 0.5 * (gl_x + 1.0)
        wq = 0.5 * gl_w
        a, b = be_[:, 0], be_[:, 1]
        xa, xb = xy[a], xy[b]
        d = xb - xa
        length = np.hypot(d[:, 0], d[:, 1])
        nrm = np.stack([d[:, 1], -d[:, 0]], axis=1) / length[:, None]  # outward for CCW
        for tk, wk in zip(tq, wq):
            pt = xa + tk * d
            fxv = np.stack([np.broadcast_to(np.asarray(v, dtype=float), (len(pt),)) for v in fx_fun(pt[:, 0], pt[:, 1])], axis=1)
            fyv = np.stack([np.broadcast_to(np.asarray(v, dtype=float), (len(pt),)) for v in fy_fun(pt[:, 0], pt[:, 1])], axis=1)
            g = fxv * nrm[:, 0:1] + fyv * nrm[:, 1:2]
            np.add.at(G, a, dt * wk * length[:, None] * (1.0 - tk) * g)
            np.add.at(G, b, dt * wk * length[:, None] * tk * g)
        return G

    return exact, forcing


def l2_error(xy, tri, Uh, exact_fn, tt):
    """Per-compartment L2 norms of u_h - u and of u (7-point rule)."""
    area, _ = O.geometry(xy, tri)
    L, W = O.quad_rule("deg5")
    P = xy[tri]
    err = np.zeros(5)
    ref = np.zeros(5)
    for q in range(len(W)):
        xq = np.einsum("a,tax->tx", L[q], P)
        uh = np.einsum("a,tac->tc", L[q], Uh[tri])
        ue = exact_fn(xq, tt)
        err += ((uh - ue) ** 2 * (W[q] * area)[:, None]).sum(axis=0)
        ref += (ue ** 2 * (W[q] * area)[:, None]).sum(axis=0)
    return np.sqrt(err), np.sqrt(ref)
