"""Seeded synthetic inputs for the SEIRD backward-Euler step.

This module produces meshes, initial states, parameter sets and subdomain
partitions.  It is shared by the CUDA path's tests/bench and by the CPU oracle,
and it deliberately contains none of the method's arithmetic (no residual,
Jacobian, quadrature, solver or preconditioner): only geometry generation and
random draws.

Workloads (the paper's own Ontario mesh, shapefile and case data are not
available, so seeded stand-ins with the same structure are generated):

* ``square``: unit square, structured P1 triangulation, uniform total density
  with a Gaussian infected bump at the centre (Section 4.1, Table 1 "square
  domain" column).
* ``ontario``: a seeded random star-shaped 24-gon, meshed by clipping a
  structured background triangulation, with a log-normal "urban Gaussians on a
  rural floor" density and a handful of infection seeds (Section 4.2, Table 1
  "Southern Ontario" column for the rates).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Compartment order used everywhere: s, e, i, r, d (Eq. seird1-5).
NC = 5


@dataclass
class Params:
    """Scalar rates of Eq. seird1-5 (names follow the paper)."""

    A: float
    beta_i: float
    beta_e: float
    sigma: float
    gamma_e: float
    gamma_r: float
    gamma_d: float
    alpha: float = 0.0
    mu: float = 0.0
    nu: tuple = (0.0, 0.0, 0.0, 0.0)  # nu_S, nu_E, nu_I, nu_R ; nu_D == 0

    def as_dict(self):
        return dict(A=self.A, beta_i=self.beta_i, beta_e=self.beta_e, sigma=self.sigma,
                    gamma_e=self.gamma_e, gamma_r=self.gamma_r, gamma_d=self.gamma_d,
                    alpha=self.alpha, mu=self.mu, nu=tuple(self.nu))


def params_square(**over) -> Params:
    """Table 1, "Square domain" column (Section 4.1)."""
    p = Params(A=500.0, beta_i=3.78e-4, beta_e=3.78e-4, sigma=1.0 / 7.0, gamma_e=1.0 / 6.0,
               gamma_r=1.0 / 24.0, gamma_d=1.0 / 160.0, alpha=0.0, mu=0.0,
               nu=(3.94e-6, 3.94e-6, 1e-8, 3.94e-6))
    for k, v in over.items():
        setattr(p, k, v)
    return p


def params_ontario(max_density: float, **over) -> Params:
    """Table 1, "Southern Ontario" column; beta is chosen so that beta*max(N) = 0.756/day.

    The paper fits the Ontario betas (Eq. beta_ie/beta_x) to case data it does not
    publish; 0.756/day is the square case's beta*N (3.78e-4 * 2000).  Scaling by
    the densest city makes that city grow at the square case's rate and every
    less dense place slower (transmission is density dependent).
    """
    beta = 0.756 / max_density
    p = Params(A=8.9e-3, beta_i=beta, beta_e=beta, sigma=1.0 / 5.0, gamma_e=1.0 / 15.0,
               gamma_r=1.0 / 11.0, gamma_d=1.0 / 750.0, alpha=0.0, mu=0.0,
               nu=(4.5e-7, 4.5e-7, 1e-9, 4.5e-7))
    for k, v in over.items():
        setattr(p, k, v)
    return p


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------

RATE_NAMES = ("beta_i", "beta_e", "sigma", "gamma_e", "gamma_r", "gamma_d")


def rate_samples(base: Params, n_samples: int, seed: int, spread: float = 0.5) -> list:
    """Ensemble members: each of the ten calibrated rates (beta_I, beta_E, sigma,
    gamma_E, gamma_R, gamma_D, nubar_S..R) drawn log-uniformly within a factor
    (1 +- spread) of its base value, independently per sample (seeded)."""
    rng = np.random.default_rng(seed)
    lo, hi = np.log(1.0 - spread), np.log(1.0 + spread)
    out = []
    for _ in range(n_samples):
        f = np.exp(rng.uniform(lo, hi, 10))
        q = Params(**base.as_dict())
        for k, name in enumerate(RATE_NAMES):
            setattr(q, name, float(getattr(base, name) * f[k]))
        q.nu = tuple(float(base.nu[c] * f[6 + c]) for c in range(4))
        out.append(q)
    return out


def structured_mesh(nx: int, ny: int | None = None, x0=0.0, x1=1.0, y0=0.0, y1=1.0):
    """Structured P1 triangulation of a rectangle with nx*ny vertices.

    Node (i, j) (i along x) has index j*nx + i.  Each cell is split along its
    (i, j)-(i+1, j+1) diagonal; both triangles are counter-clockwise.
    Returns ``xy`` float64 [n, 2] and ``tri`` int32 [m, 3].
    """
    ny = nx if ny is None else ny
    if nx < 2 or ny < 2:
        raise ValueError("need at least 2x2 vertices")
    xs = np.linspace(x0, x1, nx)
    ys = np.linspace(y0, y1, ny)
    X, Y = np.meshgrid(xs, ys)  # [ny, nx]
    xy = np.stack([X.ravel(), Y.ravel()], axis=1).astype(np.float64)
    j, i = np.meshgrid(np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
    v00 = (j * nx + i).ravel()
    v10 = v00 + 1
    v11 = v00 + nx + 1
    v01 = v00 + nx
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    tri = np.empty((2 * t1.shape[0], 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2
    return xy, tri


def random_polygon(seed: int, n_vertices: int = 24):
    """Star-shaped simple polygon: sorted U(0, 2pi) angles, radii U(0.6, 1.0),
    mapped into the unit square (centre 0.5, 0.5, scale 0.5)."""
    rng = np.random.default_rng(seed)
    ang = np.sort(rng.uniform(0.0, 2.0 * np.pi, n_vertices))
    rad = rng.uniform(0.6, 1.0, n_vertices)
    px = 0.5 + 0.5 * rad * np.cos(ang)
    py = 0.5 + 0.5 * rad * np.sin(ang)
    return np.stack([px, py], axis=1)


def _points_in_polygon(pts, poly):
    """Even-odd ray casting, vectorised over points."""
    x = pts[:, 0]
    y = pts[:, 1]
    inside = np.zeros(len(pts), dtype=bool)
    nv = len(poly)
    for k in range(nv):
        xa, ya = poly[k]
        xb, yb = poly[(k + 1) % nv]
        cond = (ya > y) != (yb > y)
        with np.errstate(divide="ignore", invalid="ignore"):
            xint = xa + (y - ya) * (xb - xa) / (yb - ya)
        inside ^= cond & (x < xint)
    return inside


def _polygon_area(poly):
    x, y = poly[:, 0], poly[:, 1]
    return 0.5 * abs(np.dot(x, np.roll(y, -1)) - np.dot(y, np.roll(x, -1)))


def irregular_mesh(seed: int, n_target: int, n_vertices: int = 24, jitter: float = 0.2):
    """P1 mesh of a seeded random polygon with about ``n_target`` nodes.

    A structured background triangulation of the unit square is clipped by
    triangle centroid, the largest edge-connected component is kept, interior
    nodes are jittered by at most ``jitter*h`` (a move that would invert a
    triangle is undone) and nodes keep the background's row-major order.
    Returns ``xy`` [n, 2] float64, ``tri`` [m, 3] int32 (CCW), and the polygon.
    """
    poly = random_polygon(seed, n_vertices)
    area = _polygon_area(poly)
    nside = max(4, int(round(math.sqrt(n_target / area))))
    for _ in range(3):
        xy, tri, keep_nodes = _clip(poly, nside)
        n = len(xy)
        if abs(n - n_target) <= 0.01 * n_target:
            break
        nside = max(4, int(round(nside * math.sqrt(n_target / n))))
    h = 1.0 / (nside - 1)
    rng = np.random.default_rng(seed + 7919)
    # boundary nodes: endpoints of edges used by exactly one triangle
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    e = np.sort(e, axis=1)
    key = e[:, 0].astype(np.int64) * len(xy) + e[:, 1]
    uniq, cnt = np.unique(key, return_counts=True)
    bkeys = uniq[cnt == 1]
    bnodes = np.unique(np.concatenate([bkeys // len(xy), bkeys % len(xy)]))
    interior = np.ones(len(xy), dtype=bool)
    interior[bnodes] = False
    disp = rng.uniform(-jitter * h, jitter * h, size=xy.shape)
    disp[~interior] = 0.0
    moved = xy + disp
    # undo moves of nodes touching a triangle whose orientation is not positive
    for _ in range(4):
        p = moved[tri]
        d = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1])
        bad = d <= 0.25 * h * h * 0.5
        if not bad.any():
            break
        nodes = np.unique(tri[bad].ravel())
        moved[nodes] = xy[nodes]
    return moved, tri, poly


def _clip(poly, nside):
    bxy, btri = structured_mesh(nside, nside)
    cen = bxy[btri].mean(axis=1)
    inside = _points_in_polygon(cen, poly)
    tri = btri[inside]
    # largest edge-connected component
    import scipy.sparse as sp
    from scipy.sparse.csgraph import connected_components
    m = len(tri)
    e = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    e = np.sort(e, axis=1)
    key = e[:, 0].astype(np.int64) * len(bxy) + e[:, 1]
    tid = np.tile(np.arange(m), 3)
    order = np.argsort(key, kind="stable")
    ks = key[order]
    same = ks[1:] == ks[:-1]
    a = tid[order][:-1][same]
    b = tid[order][1:][same]
    g = sp.coo_matrix((np.ones(len(a)), (a, b)), shape=(m, m))
    ncomp, lab = connected_components(g, directed=False)
    big = np.argmax(np.bincount(lab))
    tri = tri[lab == big]
    used = np.unique(tri.ravel())
    remap = -np.ones(len(bxy), dtype=np.int64)
    remap[used] = np.arange(len(used))
    return bxy[used].copy(), remap[tri].astype(np.int32), used


# ---------------------------------------------------------------------------
# initial states
# ---------------------------------------------------------------------------

def square_ic(xy, N0: float = 1e4, sigma: float = 0.05, amp: float = 0.1):
    """Uniform total density N0, infected Gaussian bump amp*N0 at (0.5, 0.5) of
    width sigma; e = r = d = 0 and s = N0 - i (Section 4.1)."""
    r2 = (xy[:, 0] - 0.5) ** 2 + (xy[:, 1] - 0.5) ** 2
    U = np.zeros((len(xy), NC))
    i0 = amp * N0 * np.exp(-r2 / (2.0 * sigma * sigma))
    U[:, 2] = i0
    U[:, 0] = N0 - i0
    return U


def uniform_ic(n: int, total: float, frac_i: float = 0.1):
    """Spatially uniform state: a fraction frac_i infected, the rest susceptible
    (Appendix B.4 homogeneous start)."""
    U = np.zeros((n, NC))
    U[:, 2] = frac_i * total
    U[:, 0] = total - U[:, 2]
    return U


@dataclass
class UrbanDensity:
    floor: float
    centres: np.ndarray
    amps: np.ndarray
    widths: np.ndarray

    def __call__(self, xy):
        N = np.full(len(xy), self.floor)
        for c, a, w in zip(self.centres, self.amps, self.widths):
            r2 = (xy[:, 0] - c[0]) ** 2 + (xy[:, 1] - c[1]) ** 2
            m = r2 < (8.0 * w) ** 2
            N[m] += a * np.exp(-r2[m] / (2.0 * w * w))
        return N


def urban_density(seed: int, poly=None, n_urban: int = 40, floor: float = 1.0):
    """Rural floor plus n_urban Gaussians: log-normal amplitudes (median 10*floor,
    sigma_log 0.75), widths U(0.005, 0.03), centres uniform in the polygon (or the
    unit square)."""
    rng = np.random.default_rng(seed + 104729)
    cs = []
    while len(cs) < n_urban:
        c = rng.uniform(0.02, 0.98, size=(4 * n_urban, 2))
        if poly is not None:
            c = c[_points_in_polygon(c, poly)]
        cs.extend(list(c))
    centres = np.array(cs[:n_urban])
    amps = 10.0 * floor * np.exp(0.75 * rng.standard_normal(n_urban))
    widths = rng.uniform(0.005, 0.03, n_urban)
    return UrbanDensity(floor, centres, amps, widths)


def urban_ic(xy, dens: UrbanDensity, seed: int, n_seeds: int = 5, width: float = 0.01, frac: float = 0.01):
    """Infection seeds at n_seeds of the urban centres: i0 = frac*N*Gaussian(width),
    e0 = i0 (the 1:1 exposed:infected ratio of Section 4), s0 = N - i0 - e0."""
    rng = np.random.default_rng(seed + 15485863)
    N = dens(xy)
    pick = rng.choice(len(dens.centres), size=n_seeds, replace=False)
    g = np.zeros(len(xy))
    for c in dens.centres[pick]:
        r2 = (xy[:, 0] - c[0]) ** 2 + (xy[:, 1] - c[1]) ** 2
        g += np.exp(-r2 / (2.0 * width * width))
    g = np.minimum(g, 1.0)
    U = np.zeros((len(xy), NC))
    U[:, 2] = frac * N * g
    U[:, 1] = U[:, 2]
    U[:, 0] = N - U[:, 1] - U[:, 2]
    return U


def smooth_field(xy, seed: int, lo: float = 0.5, hi: float = 1.5, modes: int = 4):
    """Smooth positive per-node multiplier (used as a transmission field b(x))."""
    rng = np.random.default_rng(seed + 31337)
    f = np.zeros(len(xy))
    for _ in range(modes):
        kx, ky = rng.uniform(1, 6, 2)
        ph = rng.uniform(0, 2 * np.pi)
        f += np.sin(kx * xy[:, 0] + ky * xy[:, 1] + ph)
    f = (f - f.min()) / max(f.max() - f.min(), 1e-30)
    return lo + (hi - lo) * f


# ---------------------------------------------------------------------------
# partitions and random sparse inputs
# ---------------------------------------------------------------------------

def box_partition(xy, px: int, py: int):
    """Owner of each node for a px-by-py grid of equal boxes over the bounding box."""
    lo = xy.min(axis=0)
    hi = xy.max(axis=0)
    span = np.maximum(hi - lo, 1e-300)
    bx = np.minimum((px * (xy[:, 0] - lo[0]) / span[0]).astype(np.int64), px - 1)
    by = np.minimum((py * (xy[:, 1] - lo[1]) / span[1]).astype(np.int64), py - 1)
    return (by * px + bx).astype(np.int32)


def random_partition(n: int, n_parts: int, seed: int):
    """Owner array with random (non-geometric) parts, every part non-empty."""
    rng = np.random.default_rng(seed)
    owner = rng.integers(0, n_parts, n).astype(np.int32)
    owner[:n_parts] = np.arange(n_parts, dtype=np.int32)
    return owner


def random_bsr(n_rows: int, n_cols: int, blocks_per_row_max: int, seed: int, empty_row_frac: float = 0.1):
    """Random 5x5-block BSR matrix: row_ptr int32 [n_rows+1], col int32 (sorted,
    unique per row), val float64 [nnzb, 5, 5]; some rows are empty."""
    rng = np.random.default_rng(seed)
    row_ptr = [0]
    cols = []
    for _ in range(n_rows):
        if n_cols == 0 or rng.random() < empty_row_frac:
            k = 0
        else:
            k = int(rng.integers(1, min(blocks_per_row_max, n_cols) + 1))
        c = np.sort(rng.choice(n_cols, size=k, replace=False)) if k else np.zeros(0, dtype=np.int64)
        cols.append(c)
        row_ptr.append(row_ptr[-1] + k)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    val = rng.standard_normal((len(col), 5, 5))
    return np.array(row_ptr, dtype=np.int32), col, val


# ---------------------------------------------------------------------------
# named workloads
# ---------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    xy: np.ndarray
    tri: np.ndarray
    params: Params
    U0: np.ndarray
    dt: float
    n_steps: int
    n_subdomains: int
    overlap: int
    coarse: bool
    owner: np.ndarray | None = None
    beta_field: np.ndarray | None = None
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def n(self):
        return len(self.xy)

    @property
    def dof(self):
        return NC * len(self.xy)


def square_workload(nside: int = 33, seed: int = 0, N0: float = 1e4) -> Workload:
    """Unit square, nside^2 vertices, uniform density N0 (1e4 by default; the
    paper's Section 4.1 uses 2000), infected bump sigma = 0.05, dt = 1 day,
    10 steps, 2x2 box subdomains with overlap 1 (Section 4.1)."""
    xy, tri = structured_mesh(nside)
    U0 = square_ic(xy, N0=N0, sigma=0.05, amp=0.1)
    return Workload("square%dx%d" % (nside, nside), xy, tri, params_square(), U0, dt=1.0, n_steps=10,
                    n_subdomains=4, overlap=1, coarse=False, owner=box_partition(xy, 2, 2), seed=seed)


def ontario_workload(n_target: int = 2_000_000, seed: int = 0, n_subdomains: int = 512, overlap: int = 2,
                     structured: bool = False, nside: int | None = None) -> Workload:
    """Southern-Ontario-like workload: seeded 24-gon meshed to about n_target nodes
    (or, with ``structured``, the unit square at nside^2 nodes), urban density,
    5 infection seeds, dt = 0.5 day, 180 steps (90 days), RAS with the given number
    of subdomains and overlap plus the constant coarse space (Section 4.2)."""
    if structured:
        nside = nside or int(round(math.sqrt(n_target)))
        xy, tri = structured_mesh(nside)
        poly = None
        name = "urban_square%dx%d" % (nside, nside)
    else:
        xy, tri, poly = irregular_mesh(seed, n_target)
        name = "ontario_like_%dk" % (len(xy) // 1000)
    dens = urban_density(seed, poly)
    U0 = urban_ic(xy, dens, seed)
    p = params_ontario(float(U0.sum(axis=1).max()))
    return Workload(name, xy, tri, p, U0, dt=0.5, n_steps=180, n_subdomains=n_subdomains, overlap=overlap,
                    coarse=True, owner=None, seed=seed, extra=dict(polygon=poly))
