"""Failure detection of the bounded device waits, with no GPU fault.

The subdomain solves of the RAS apply stream each stage's factor blocks through
shared memory and wait on mbarriers for them; every such wait polls a bounded
number of times.  seird_set_wait_limit(-1) makes every one of those waits give
up at once: the call must then return SEIRD_ETIMEOUT (no hang, no trap), a
failed step must leave the state at u^n, and once the limit is restored the
same context must give the oracle's results again.  The wait for issued copies
to land before a CTA exits keeps its own bound, so nothing is in flight when
the kernel returns.
"""
import numpy as np
import pytest

from oracle import seird_oracle as O
from paper_2208_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2208_01839_gb300 import build as _b  # noqa: E402

_b.build()
from paper_2208_01839_gb300 import seird as S  # noqa: E402

ETIMEOUT = -8


def _floor(wl):
    return 1e-14 * np.linalg.norm(O.residual(wl.xy, wl.tri, wl.params, 0.0, np.abs(wl.U0), np.zeros_like(wl.U0)))


@pytest.mark.parametrize("precision,coarse", [(0, 2), (1, 2), (0, 1)])
def test_wait_timeout_is_reported_and_the_context_recovers(precision, coarse):
    wl = I.square_workload(17)
    owner = I.box_partition(wl.xy, 3, 2)
    J = O.jacobian(wl.xy, wl.tri, wl.params, wl.dt, wl.U0)
    rp, col, val = O.to_bsr(J)
    r = np.random.default_rng(21).standard_normal(5 * wl.n)
    ref = O.ras_apply(rp, col, val, owner, 1, r, coarse=True, multiplicative=coarse == 2)
    tol = 1e-10 if precision == 0 else 1e-4
    with S.Solver(wl.xy, wl.tri, wl.params, owner=owner, dt=wl.dt, overlap=1, coarse=coarse, precision=precision,
                  newton_rtol=1e-12, newton_atol=_floor(wl), gmres_rtol=1e-12, gmres_restart=30,
                  gmres_maxit=2000) as sv:
        u0 = torch.tensor(wl.U0, device="cuda")
        sv.set_state(u0)
        sv.jacobian(wl.U0)
        sv.precond_setup()
        # every wait of the subdomain solves gives up at once
        sv.set_wait_limit(-1)
        with pytest.raises(S.SeirdError) as ei:
            sv.precond_apply(r.reshape(-1, 5))
        assert ei.value.code == ETIMEOUT, ei.value
        with pytest.raises(S.SeirdError) as ei:
            sv.step()
        assert ei.value.code == ETIMEOUT, ei.value
        after = sv.get_state()
        assert np.array_equal(after, wl.U0)  # a failed step leaves u^n
        # the default limit again: the same context applies and steps correctly
        sv.set_wait_limit(0)
        got = sv.precond_apply(r.reshape(-1, 5)).ravel()
        assert np.linalg.norm(got - ref) <= tol * np.linalg.norm(ref)
        sv.step()
        U1 = sv.get_state()
    if precision == 0:
        U_ref, _ = O.newton_step(wl.xy, wl.tri, wl.params, wl.dt, wl.U0, rtol=1e-12)
        for c in range(5):
            assert np.linalg.norm(U1[:, c] - U_ref[:, c]) <= 1e-9 * np.linalg.norm(U_ref[:, c]), c


def test_wait_timeout_inside_a_captured_gmres_cycle():
    """With options.graph the restart cycle replays a captured graph; changing the
    limit drops the captured cycle, so the shortened waits take effect there too
    and the restored limit gives the eager loop's result again."""
    wl = I.square_workload(17)
    owner = I.box_partition(wl.xy, 3, 2)
    opts = dict(owner=owner, dt=wl.dt, overlap=1, coarse=2, newton_rtol=1e-12, newton_atol=_floor(wl),
                gmres_rtol=1e-12, gmres_restart=30, gmres_maxit=2000)
    with S.Solver(wl.xy, wl.tri, wl.params, **opts) as eager:
        eager.set_state(wl.U0)
        eager.step()
        ref = eager.get_state()
    with S.Solver(wl.xy, wl.tri, wl.params, graph=1, **opts) as sv:
        sv.set_state(wl.U0)
        sv.set_wait_limit(-1)
        with pytest.raises(S.SeirdError) as ei:
            sv.step()
        assert ei.value.code == ETIMEOUT, ei.value
        assert np.array_equal(sv.get_state(), wl.U0)
        sv.set_wait_limit(0)
        sv.step()
        assert np.array_equal(sv.get_state(), ref)
