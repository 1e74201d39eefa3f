"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances (FP64 on both sides, different summation orders):
  * assembly, SpMV: |diff| <= 1e-12 x (magnitude of the summed terms);
  * preconditioner apply: 1e-10 relative (triangular solves amplify rounding);
  * Newton roots: <= 1e-9 relative L2 per compartment (the target stated for
    the FP64 path), both sides solving to ||F|| <= 1e-12 ||F(u^n)||.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import seird_oracle as O
from paper_2208_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2208_01839_gb300 import build as _b  # noqa: E402

_b.build()
from paper_2208_01839_gb300 import seird as S  # noqa: E402

DEV = "cuda"


def rel_l2_per_comp(a, b):
    return [float(np.linalg.norm(a[:, c] - b[:, c]) / max(np.linalg.norm(b[:, c]), 1e-300)) for c in range(5)]


def newton_floor(wl):
    """Absolute Newton tolerance at the FP64 rounding floor: 1e-14 ||M |u^0|||.
    Where ||F(u^n)|| is small next to ||M u|| (slowly changing states), the
    relative test alone would ask for a residual below what FP64 can resolve."""
    return 1e-14 * np.linalg.norm(O.residual(wl.xy, wl.tri, wl.params, 0.0, np.abs(wl.U0), np.zeros_like(wl.U0)))


def solver(wl, owner=None, **kw):
    opts = dict(dt=wl.dt, overlap=wl.overlap, newton_rtol=1e-12, newton_atol=newton_floor(wl), gmres_rtol=1e-12,
                gmres_restart=30, gmres_maxit=2000)
    opts.update(kw)
    return S.Solver(wl.xy, wl.tri, wl.params, owner=wl.owner if owner is None else owner,
                    beta_field=wl.beta_field, **opts)


# ---------------------------------------------------------------------------
# SpMV
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n_rows,n_cols,bmax,seed", [(0, 0, 1, 0), (1, 1, 1, 1), (7, 5, 4, 2), (1000, 900, 9, 3),
                                                     (20011, 20011, 8, 4)])
def test_bsr_spmv_matches_oracle(n_rows, n_cols, bmax, seed):
    rp, col, val = I.random_bsr(n_rows, n_cols, bmax, seed)
    x = np.random.default_rng(seed + 1).standard_normal(5 * n_cols)
    ref = O.bsr_spmv(rp, col, val, x) if n_rows else np.zeros(0)
    t = lambda a: torch.tensor(a, device=DEV)
    y = torch.full((5 * n_rows,), np.nan, dtype=torch.float64, device=DEV)
    S.bsr_spmv(t(rp), t(col), t(val), t(x), y)
    torch.cuda.synchronize()
    got = y.cpu().numpy()
    A = sp.bsr_matrix((np.abs(val), col, rp), shape=(5 * n_rows, 5 * n_cols)) if n_rows else None
    bound = (A @ np.abs(x)) if n_rows else np.zeros(0)
    assert np.all(np.abs(got - ref) <= 1e-13 * bound + 1e-300)


def test_bsr_spmv_float32_values():
    rp, col, val = I.random_bsr(3001, 2999, 7, 9)
    val32 = val.astype(np.float32)
    x = np.random.default_rng(10).standard_normal(5 * 2999)
    ref = O.bsr_spmv(rp, col, val32.astype(np.float64), x)
    t = lambda a: torch.tensor(a, device=DEV)
    y = torch.empty(5 * 3001, dtype=torch.float64, device=DEV)
    S.bsr_spmv(t(rp), t(col), t(val32), t(x), y)
    torch.cuda.synchronize()
    A = sp.bsr_matrix((np.abs(val), col, rp), shape=(5 * 3001, 5 * 2999))
    assert np.all(np.abs(y.cpu().numpy() - ref) <= 1e-13 * (A @ np.abs(x)))


# ---------------------------------------------------------------------------
# assembly
# ---------------------------------------------------------------------------

def _mass_scale(wl, U):
    """max_i (M |U|)_i: the magnitude of the terms each residual entry sums."""
    Mabs = O.residual(wl.xy, wl.tri, wl.params, 0.0, np.abs(U), np.zeros_like(U))
    return np.abs(Mabs).max()


def _workloads():
    sq = I.square_workload(33)
    irr_xy, irr_tri, _ = I.irregular_mesh(3, 3000)
    dens = I.urban_density(3)
    U0 = I.urban_ic(irr_xy, dens, 3)
    p = I.params_ontario(float(U0.sum(axis=1).max()))
    irr = I.Workload("irregular3k", irr_xy, irr_tri, p, U0, dt=0.5, n_steps=3, n_subdomains=6, overlap=2,
                     coarse=True, owner=I.box_partition(irr_xy, 3, 2), beta_field=I.smooth_field(irr_xy, 3))
    return {"square33": sq, "irregular3k": irr}


WL = _workloads()


@pytest.mark.parametrize("name", list(WL))
@pytest.mark.parametrize("rule", [0, 1])
def test_residual_matches_oracle(name, rule):
    wl = WL[name]
    rng = np.random.default_rng(5)
    U = wl.U0 * (1.0 + 0.05 * rng.standard_normal(wl.U0.shape)) + 1.0
    ref = O.residual(wl.xy, wl.tri, wl.params, wl.dt, U, wl.U0, bfield=wl.beta_field,
                     rule="deg5" if rule == 0 else "vertex")
    with solver(wl, quadrature=rule) as sv:
        got = sv.residual(U, wl.U0)
        # device pointers give the same result as host pointers
        gt = sv.residual(torch.tensor(U, device=DEV), torch.tensor(wl.U0, device=DEV)).cpu().numpy()
    scale = _mass_scale(wl, U) * (1.0 + wl.dt)
    assert np.abs(got - ref).max() <= 1e-12 * scale
    assert np.array_equal(got, gt)


@pytest.mark.parametrize("name", list(WL))
@pytest.mark.parametrize("rule", [0, 1])
def test_jacobian_matches_oracle(name, rule):
    wl = WL[name]
    rng = np.random.default_rng(6)
    U = wl.U0 * (1.0 + 0.05 * rng.standard_normal(wl.U0.shape)) + 1.0
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, U, bfield=wl.beta_field, rule="deg5" if rule == 0 else "vertex")
    rp, col, val = O.to_bsr(J)
    with solver(wl, quadrature=rule) as sv:
        sv.jacobian(U)
        grp, gcol, gval = sv.get_jacobian()
        x = rng.standard_normal(U.shape)
        y = sv.apply_jacobian(x)
    assert np.array_equal(grp, rp) and np.array_equal(gcol, col)
    scale = np.abs(val).max()
    assert np.abs(gval - val).max() <= 1e-12 * scale
    ref = (J @ x.ravel()).reshape(U.shape)
    Jabs = abs(J)
    assert np.all(np.abs(y - ref).ravel() <= 1e-12 * (Jabs @ np.abs(x).ravel()) + 1e-300)


# ---------------------------------------------------------------------------
# preconditioner and linear solve
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("overlap,coarse", [(0, 0), (1, 0), (2, 1), (1, 1)])
def test_ras_apply_matches_oracle(overlap, coarse):
    wl = I.square_workload(17)
    owner = I.box_partition(wl.xy, 3, 2)
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0)
    rp, col, val = O.to_bsr(J)
    r = np.random.default_rng(7).standard_normal(5 * wl.n)
    ref = O.ras_apply(rp, col, val, owner, overlap, r, coarse=bool(coarse))
    with solver(wl, owner=owner, overlap=overlap, coarse=coarse) as sv:
        sv.jacobian(wl.U0)
        sv.precond_setup()
        got = sv.precond_apply(r.reshape(-1, 5)).ravel()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_ras_apply_irregular_partition_with_coarse():
    wl = WL["irregular3k"]
    owner = I.random_partition(wl.n, 5, 3)  # non-geometric parts: many neighbours, wide coarse band
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, bfield=wl.beta_field)
    rp, col, val = O.to_bsr(J)
    r = np.random.default_rng(8).standard_normal(5 * wl.n)
    ref = O.ras_apply(rp, col, val, owner, 1, r, coarse=True)
    with solver(wl, owner=owner, overlap=1, coarse=1) as sv:
        sv.jacobian(wl.U0)
        sv.precond_setup()
        got = sv.precond_apply(r.reshape(-1, 5)).ravel()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_linear_solve_matches_direct_solve():
    wl = WL["irregular3k"]
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, bfield=wl.beta_field)
    b = np.random.default_rng(9).standard_normal(5 * wl.n)
    ref = spla.spsolve(J.tocsc(), b)
    with solver(wl, coarse=1, gmres_restart=20) as sv:
        sv.jacobian(wl.U0)
        sv.precond_setup()
        x, its = sv.linear_solve(b.reshape(-1, 5))
    assert its > 0
    assert np.linalg.norm(x.ravel() - ref) <= 1e-9 * np.linalg.norm(ref)


def test_single_subdomain_without_overlap_is_ilu0():
    """P = 1, overlap 0: the preconditioner is block ILU(0) of J itself."""
    wl = I.square_workload(9)
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0)
    rp, col, val = O.to_bsr(J)
    r = np.random.default_rng(3).standard_normal(5 * wl.n)
    Fk = O.block_ilu0(rp, col, val)
    ref = O.block_ilu0_solve(rp, col, Fk, r)
    with solver(wl, owner=np.zeros(wl.n, dtype=np.int32), overlap=0) as sv:
        sv.jacobian(wl.U0)
        sv.precond_setup()
        got = sv.precond_apply(r.reshape(-1, 5)).ravel()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


# ---------------------------------------------------------------------------
# Newton steps
# ---------------------------------------------------------------------------

def test_square_steps_match_oracle_step_by_step():
    """Config-1 workload (33x33, N = 1e4, dt = 1, 4 box subdomains, overlap 1):
    every step from the same u^n, and the 10-step trajectory."""
    wl = I.square_workload(33)
    U = wl.U0.copy()
    with solver(wl) as sv:
        for k in range(wl.n_steps):
            ref, info = O.newton_step(wl.xy, wl.tri, wl.params, wl.dt, U, rtol=1e-12)
            sv.set_state(U, t=k * wl.dt)
            st = sv.step()
            got = sv.get_state()
            assert max(rel_l2_per_comp(got, ref)) <= 1e-9, (k, rel_l2_per_comp(got, ref), st)
            U = ref
        # whole trajectory from u^0 on the device
        sv.set_state(wl.U0)
        sv.run(wl.n_steps)
        traj = sv.get_state()
    assert max(rel_l2_per_comp(traj, U)) <= 1e-9


@pytest.mark.parametrize("one_pass", [0, 1])
def test_paper_density_irregular_with_coarse_and_field(one_pass):
    """Also with a single classical Gram-Schmidt pass (PETSc's GMRES default): the
    orthogonalisation changes iteration counts, not the root."""
    wl = WL["irregular3k"]
    U_ref, _ = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 3, rtol=1e-12, atol=newton_floor(wl),
                     bfield=wl.beta_field)
    with solver(wl, coarse=1, gmres_one_pass=one_pass) as sv:
        sv.set_state(torch.tensor(wl.U0, device=DEV))
        sv.run(3)
        got = sv.get_state(torch.empty((wl.n, 5), dtype=torch.float64, device=DEV)).cpu().numpy()
    assert max(rel_l2_per_comp(got, U_ref)) <= 1e-9


def test_default_partitioner_and_vertex_rule():
    """Built-in seeded bisection (no owner array) and the three-vertex rule."""
    wl = I.square_workload(33, N0=2000.0)
    U_ref, _ = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 2, rtol=1e-12, rule="vertex")
    with S.Solver(wl.xy, wl.tri, wl.params, dt=wl.dt, n_subdomains=7, overlap=2, coarse=1, quadrature=1,
                  newton_rtol=1e-12, newton_atol=newton_floor(wl), gmres_rtol=1e-12, gmres_maxit=2000) as sv:
        sv.set_state(wl.U0)
        sv.run(2)
        got = sv.get_state()
        inf = sv.info()
    assert inf["n_subdomains"] == 7 and inf["coarse_band"] >= 1
    assert max(rel_l2_per_comp(got, U_ref)) <= 1e-9


def test_smallest_mesh_one_triangle():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    p = I.params_square()
    U0 = np.array([[1800.0, 10.0, 100.0, 0.0, 0.0], [1900.0, 0.0, 50.0, 0.0, 0.0], [2000.0, 0.0, 0.0, 0.0, 0.0]])
    ref, _ = O.newton_step(xy, tri, p, 0.5, U0, rtol=1e-12)
    with S.Solver(xy, tri, p, dt=0.5, n_subdomains=1, newton_rtol=1e-12, gmres_rtol=1e-13) as sv:
        sv.set_state(U0)
        sv.step()
        got = sv.get_state()
    assert np.abs(got - ref).max() <= 1e-9 * np.abs(ref).max()


def test_nonpositive_density_is_reported_not_trapped():
    """Host-prepared state with N < 0: the assembly flags it and the call
    returns ENONFINITE; the context stays usable."""
    wl = I.square_workload(9)
    with solver(wl) as sv:
        bad = -np.ones_like(wl.U0)
        with pytest.raises(S.SeirdError) as e:
            sv.residual(bad, bad)
        assert e.value.code == -7
        ok = sv.residual(wl.U0, wl.U0)
        assert np.isfinite(ok).all()


# ---------------------------------------------------------------------------
# mixed precision: FP32 matrix copy and FP32 subdomain factors inside FP64 FGMRES
# ---------------------------------------------------------------------------

def test_mixed_precision_preconditioner_matches_oracle_to_fp32():
    wl = I.square_workload(17)
    owner = I.box_partition(wl.xy, 3, 2)
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0)
    rp, col, val = O.to_bsr(J)
    r = np.random.default_rng(17).standard_normal(5 * wl.n)
    ref = O.ras_apply(rp, col, val, owner, 1, r, coarse=True)
    with solver(wl, owner=owner, overlap=1, coarse=1, precision=1) as sv:
        sv.jacobian(wl.U0)
        sv.precond_setup()
        got = sv.precond_apply(r.reshape(-1, 5)).ravel()
    assert np.linalg.norm(got - ref) <= 1e-4 * np.linalg.norm(ref)


@pytest.mark.parametrize("rtol,bar", [(1e-12, 1e-9), (1e-8, 1e-6)])
def test_mixed_precision_root_matches_fp64_oracle(rtol, bar):
    """The Newton residual stays FP64, so the FP32 inner solves only change the
    iteration counts: at a tight tolerance the root matches the FP64 oracle to
    the FP64 bar; at the metric's 1e-8 it meets the mixed-precision 1e-6 bar."""
    wl = WL["irregular3k"]
    atol = newton_floor(wl) if rtol < 1e-9 else 0.0
    U_ref, _ = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 3, rtol=1e-12, atol=newton_floor(wl),
                     bfield=wl.beta_field)
    with solver(wl, coarse=1, precision=1, newton_rtol=rtol, newton_atol=atol, gmres_rtol=1e-5) as sv:
        sv.set_state(wl.U0)
        stats = sv.run(3)
        got = sv.get_state()
    assert max(rel_l2_per_comp(got, U_ref)) <= bar, (rel_l2_per_comp(got, U_ref), stats[-1])


def test_mixed_precision_square_step_by_step():
    wl = I.square_workload(33)
    U = wl.U0.copy()
    with solver(wl, precision=1, gmres_rtol=1e-6) as sv:
        for k in range(3):
            ref, _ = O.newton_step(wl.xy, wl.tri, wl.params, wl.dt, U, rtol=1e-12)
            sv.set_state(U)
            sv.step()
            assert max(rel_l2_per_comp(sv.get_state(), ref)) <= 1e-9
            U = ref


# ---------------------------------------------------------------------------
# block ILU(k) subdomain factors (options.ilu_fill)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("fill", [1, 2])
@pytest.mark.parametrize("coarse,precision", [(0, 0), (2, 0), (1, 1)])
def test_iluk_preconditioner_matches_oracle(fill, coarse, precision):
    """RAS with block ILU(k) subdomain solves, one-level, the multiplicative two-grid and the
    FP32 factors, against the oracle's ILU(k) (FP64: 1e-10; FP32 factors: 1e-4)."""
    wl = I.square_workload(17)
    owner = I.box_partition(wl.xy, 3, 2)
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0)
    rp, col, val = O.to_bsr(J)
    r = np.random.default_rng(31 + fill).standard_normal(5 * wl.n)
    ref = O.ras_apply(rp, col, val, owner, 2, r, coarse=coarse == 1, multiplicative=coarse == 2, ilu_fill=fill)
    ref0 = O.ras_apply(rp, col, val, owner, 2, r, coarse=coarse == 1, multiplicative=coarse == 2)
    with solver(wl, owner=owner, overlap=2, coarse=coarse, precision=precision, ilu_fill=fill) as sv:
        sv.jacobian(wl.U0)
        sv.precond_setup()
        got = sv.precond_apply(r.reshape(-1, 5)).ravel()
        assert sv.info()["subdomain_blocks"] > 0
    tol = 1e-4 if precision else 1e-10
    assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
    assert np.linalg.norm(ref - ref0) > 100 * tol * np.linalg.norm(ref)  # the fill changes the result


def test_iluk_on_a_non_geometric_partition_matches_oracle():
    """ILU(1) where the subdomains are scattered node sets (long fill chains, deep level
    schedules) on the irregular mesh with the transmission field."""
    wl = WL["irregular3k"]
    owner = I.random_partition(wl.n, 4, 5)
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, bfield=wl.beta_field)
    rp, col, val = O.to_bsr(J)
    r = np.random.default_rng(33).standard_normal(5 * wl.n)
    ref = O.ras_apply(rp, col, val, owner, 1, r, coarse=True, ilu_fill=1)
    with solver(wl, owner=owner, overlap=1, coarse=1, ilu_fill=1) as sv:
        sv.jacobian(wl.U0)
        sv.precond_setup()
        got = sv.precond_apply(r.reshape(-1, 5)).ravel()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", [0, 1])
def test_iluk_steps_match_oracle(precision):
    """Three steps with ILU(2) subdomain factors and the two-grid reach the oracle's roots."""
    wl = WL["irregular3k"]
    U_ref, _ = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 3, rtol=1e-12, atol=newton_floor(wl),
                     bfield=wl.beta_field)
    with solver(wl, coarse=2, precision=precision, ilu_fill=2) as sv:
        sv.set_state(wl.U0)
        sv.run(3)
        got = sv.get_state()
    assert max(rel_l2_per_comp(got, U_ref)) <= 1e-9


# ---------------------------------------------------------------------------
# the paper's multiplicative two-grid preconditioner (Eq. RAS_2L), coarse = 2
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("overlap", [1, 2])
@pytest.mark.parametrize("mode", [True, "hybrid"])
def test_multiplicative_two_grid_apply_matches_oracle(overlap, mode):
    wl = I.square_workload(17)
    owner = I.box_partition(wl.xy, 3, 2)
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0)
    rp, col, val = O.to_bsr(J)
    r = np.random.default_rng(21).standard_normal(5 * wl.n)
    ref = O.ras_apply(rp, col, val, owner, overlap, r, multiplicative=mode)
    with solver(wl, owner=owner, overlap=overlap, coarse=2 if mode is True else 3) as sv:
        sv.jacobian(wl.U0)
        sv.precond_setup()
        got = sv.precond_apply(r.reshape(-1, 5)).ravel()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("coarse", [2, 3])
def test_multiplicative_two_grid_steps_match_oracle(precision, coarse):
    wl = WL["irregular3k"]
    U_ref, _ = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 3, rtol=1e-12, atol=newton_floor(wl),
                     bfield=wl.beta_field)
    with solver(wl, coarse=coarse, precision=precision) as sv:
        sv.set_state(wl.U0)
        sv.run(3)
        got = sv.get_state()
    assert max(rel_l2_per_comp(got, U_ref)) <= 1e-9


def test_preconditioner_carried_over_steps():
    """options.pc_keep_steps: a preconditioner built in one step serves the next
    ones (iteration counts change, the roots do not); an unconverged solve with a
    carried-over preconditioner is retried with a fresh one."""
    wl = WL["irregular3k"]
    U_ref, _ = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 3, rtol=1e-12, atol=newton_floor(wl),
                     bfield=wl.beta_field)
    with solver(wl, coarse=1, pc_keep_steps=2, pc_lag=20) as sv:
        sv.set_state(wl.U0)
        stats = sv.run(3)
        got = sv.get_state()
    assert max(rel_l2_per_comp(got, U_ref)) <= 1e-9
    assert stats[0]["pc_setups"] >= 1 and stats[1]["pc_setups"] == 0 and stats[2]["pc_setups"] == 0, stats


@pytest.mark.parametrize("group,multiplicative", [(2, False), (3, False), (2, True)])
def test_grouped_coarse_units_match_oracle(group, multiplicative):
    """options.coarse_group: one coarse unit per group of consecutive subdomains
    (here 6 box subdomains in groups of 2 or 3); the oracle's coarse space takes
    the unit of each node as owner // group."""
    wl = WL["irregular3k"]
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, bfield=wl.beta_field)
    rp, col, val = O.to_bsr(J)
    r = np.random.default_rng(9).standard_normal(5 * wl.n)
    ref = O.ras_apply(rp, col, val, wl.owner, 2, r, coarse=True, multiplicative=multiplicative,
                      coarse_owner=wl.owner // group)
    with solver(wl, overlap=2, coarse=2 if multiplicative else 1, coarse_group=group) as sv:
        sv.jacobian(wl.U0)
        sv.precond_setup()
        got = sv.precond_apply(r.reshape(-1, 5)).ravel()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_automatic_coarse_groups_beyond_the_explicit_inverse_limit():
    """1200 subdomains exceed the 1160 units whose explicit inverse is built five
    columns per CTA: the context groups them in pairs (600 units), and the
    preconditioner is the oracle's with the unit of each node = owner // 2."""
    xy, tri = I.structured_mesh(120)
    dens = I.urban_density(11)
    U0 = I.urban_ic(xy, dens, 11)
    p = I.params_ontario(float(U0.sum(axis=1).max()))
    owner = I.box_partition(xy, 40, 30)
    assert owner.max() + 1 == 1200
    J = O.jacobian(xy, tri, p, 0.5, U0)
    rp, col, val = O.to_bsr(J)
    r = np.random.default_rng(12).standard_normal(5 * len(xy))
    ref = O.ras_apply(rp, col, val, owner, 1, r, coarse=True, coarse_owner=owner // 2)
    with S.Solver(xy, tri, p, owner=owner, dt=0.5, overlap=1, coarse=1) as sv:
        assert sv.info()["coarse_units"] == 600
        sv.jacobian(U0)
        sv.precond_setup()
        got = sv.precond_apply(r.reshape(-1, 5)).ravel()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


def test_coarse_space_of_4096_ungrouped_units_matches_oracle():
    """4096 box subdomains, one coarse unit each (coarse_group = 1): 20,480 coarse
    unknowns, beyond the explicit inverse, so every coarse solve runs through the
    banded block-LU factors.  The preconditioner equals the oracle's RAS with the
    additive coarse correction of Section 3.1 (dense A_c of 20,480 unknowns)."""
    xy, tri = I.structured_mesh(128)
    dens = I.urban_density(11)
    U0 = I.urban_ic(xy, dens, 11)
    p = I.params_ontario(float(U0.sum(axis=1).max()))
    owner = I.box_partition(xy, 64, 64)
    assert owner.max() + 1 == 4096
    J = O.jacobian(xy, tri, p, 0.5, U0)
    rp, col, val = O.to_bsr(J)
    r = np.random.default_rng(13).standard_normal(5 * len(xy))
    ref = O.ras_apply(rp, col, val, owner, 1, r, coarse=True)
    with S.Solver(xy, tri, p, owner=owner, dt=0.5, overlap=1, coarse=1, coarse_group=1) as sv:
        assert sv.info()["coarse_units"] == 4096
        sv.jacobian(U0)
        sv.precond_setup()
        got = sv.precond_apply(r.reshape(-1, 5)).ravel()
    assert np.linalg.norm(got - ref) <= 1e-10 * np.linalg.norm(ref)


@pytest.mark.parametrize("predictor", [1, 2, 3, 4, 6])
def test_extrapolation_predictor_reaches_the_same_roots(predictor):
    """options.predictor = p starts Newton from the degree-p extrapolation through u^n
    and the p previous states (2 u^n - u^{n-1}, 3 u^n - 3 u^{n-1} + u^{n-2},
    4 u^n - 6 u^{n-1} + 4 u^{n-2} - u^{n-3}, ...; lower degrees while fewer are known):
    the iterates change, the roots (and the stopping test, relative to ||F(u^n)||)
    do not, and set_state drops the history (the next step starts from u^n again)."""
    wl = WL["irregular3k"]
    U_ref, _ = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 6, rtol=1e-12, atol=newton_floor(wl),
                     bfield=wl.beta_field)
    with solver(wl, coarse=1, predictor=predictor) as sv:
        sv.set_state(wl.U0)
        stats = sv.run(6)
        got = sv.get_state()
        # history dropped by set_state: the same 6 steps again give the same roots
        sv.set_state(wl.U0)
        sv.run(6)
        again = sv.get_state()
    assert max(rel_l2_per_comp(got, U_ref)) <= 1e-9
    assert max(rel_l2_per_comp(again, U_ref)) <= 1e-9
    # from the second step on the first iterate is the extrapolation, closer to the root: the later
    # steps need no more Newton iterations on average than the first one (which starts from u^n)
    assert sum(s["newton_its"] for s in stats[1:]) <= len(stats[1:]) * stats[0]["newton_its"], stats


def test_round_trip_of_the_state_keeps_the_step_history():
    """set_state with the state the context holds, at its own time (the result of the
    previous step read out and written back, as a host-coupled loop does), keeps the
    history the predictor uses: the steps are bitwise those of a loop that never leaves
    the device.  A different state drops it: the steps are bitwise those of a fresh
    context started from that state."""
    wl = WL["irregular3k"]
    kw = dict(coarse=2, predictor=2)
    with solver(wl, **kw) as a:
        a.set_state(wl.U0)
        sa = a.run(4)
        ua = a.get_state()
    with solver(wl, **kw) as b:
        b.set_state(wl.U0)
        sb = []
        for _ in range(4):
            sb += b.run(1)
            u = b.get_state()
            b.set_state(u, t=b.t)
        ub = b.get_state()
        assert np.array_equal(ua, ub)
        assert [x["newton_its"] for x in sa] == [x["newton_its"] for x in sb]
        assert [x["gmres_its"] for x in sa] == [x["gmres_its"] for x in sb]
        # a perturbed state at the same time starts afresh
        up = ub * (1.0 + 1e-6)
        b.set_state(up, t=b.t)
        b.run(2)
        uc = b.get_state()
    with solver(wl, **kw) as c:
        c.set_state(up, t=4 * wl.dt)
        c.run(2)
        assert np.array_equal(uc, c.get_state())


def test_autotuned_launch_shapes():
    """options.autotune picks the SpMV and Gram-Schmidt launch shapes by timing them on
    the context's vectors; the roots are those of the fixed shapes."""
    wl = WL["irregular3k"]
    U_ref, _ = O.run(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, 3, rtol=1e-12, atol=newton_floor(wl),
                     bfield=wl.beta_field)
    for precision in (0, 1):
        with solver(wl, coarse=1, autotune=1, precision=precision) as sv:
            sv.set_state(wl.U0)
            sv.run(3)
            got = sv.get_state()
            inf = sv.info()
        assert inf["spmv_threads"] in (128, 256, 512) and inf["cgs_tile"] in (128, 256), inf
        assert inf["cgs_ctas"] > 0 and inf["ilu_batch"] in (1, 2, 3, 4) and inf["ilu_warps"] in (3, 7), inf
        assert inf["ilu_ring"] in (118, 236), inf
        assert max(rel_l2_per_comp(got, U_ref)) <= (1e-9 if precision == 0 else 1e-6), precision


@pytest.mark.parametrize("precision,fill", [(0, 0), (1, 0), (0, 2), (1, 3)])
def test_subdomain_solve_batches_give_identical_results(precision, fill):
    """The subdomain solve's dependency-load batch (1-4 blocks), consumer warps per
    CTA (7 or 3) and factor-ring size (two stages or one), all autotuner choices,
    change only when a row's loads are issued, which warp takes it and how far the
    copies run ahead: every choice forms the same sums in the same order, so the
    preconditioner apply is bitwise the same for all sixteen.  With ILU(2) and ILU(3)
    factors a row spans several batches of every size."""
    wl = WL["irregular3k"]
    r = np.random.default_rng(31).standard_normal(5 * wl.n)
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, bfield=wl.beta_field)
    rp, col, val = O.to_bsr(J)
    ref = O.ras_apply(rp, col, val, wl.owner, 2, r, coarse=True, multiplicative=True, ilu_fill=fill)
    outs = []
    with solver(wl, overlap=2, coarse=2, precision=precision, autotune=1, ilu_fill=fill) as sv:
        sv.jacobian(wl.U0)
        sv.precond_setup()
        sv.set_state(wl.U0)
        sv.linear_solve(r.reshape(-1, 5))  # runs the autotuner (the chosen batch is one of the four)
        with pytest.raises(S.SeirdError):
            sv.set_launch_shapes(ilu_batch=5)
        for ring in (236, 118):
            for nw in (7, 3):
                for ch in (1, 2, 3, 4):
                    sv.set_launch_shapes(ilu_batch=ch, ilu_warps=nw, ilu_ring=ring)
                    inf = sv.info()
                    assert inf["ilu_batch"] == ch and inf["ilu_warps"] == nw and inf["ilu_ring"] == ring
                    outs.append(sv.precond_apply(r.reshape(-1, 5)).ravel())
        with pytest.raises(S.SeirdError):
            sv.set_launch_shapes(ilu_warps=5)
        with pytest.raises(S.SeirdError):
            sv.set_launch_shapes(ilu_ring=100)
    for k in range(1, len(outs)):
        assert np.array_equal(outs[0], outs[k]), k
    tol = 1e-10 if precision == 0 else 1e-4
    assert np.linalg.norm(outs[0] - ref) <= tol * np.linalg.norm(ref)
