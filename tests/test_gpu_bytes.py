"""The library's per-class algorithmic byte counts (seird_stats.alg_bytes), which
the bench divides by device time for its whole-step roofline: after one step,
each single-kernel class has counted its formula once per timed launch."""
import numpy as np
import pytest

from paper_2208_01839_gb300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a GPU", allow_module_level=True)

from paper_2208_01839_gb300 import build as _b  # noqa: E402

_b.build()
from paper_2208_01839_gb300 import seird as S  # noqa: E402


@pytest.mark.parametrize("precision", [0, 1])
def test_algorithmic_bytes_follow_their_formulas(precision):
    wl = I.square_workload(17)
    owner = I.box_partition(wl.xy, 3, 2)
    with S.Solver(wl.xy, wl.tri, wl.params, owner=owner, dt=wl.dt, overlap=1, coarse=2, precision=precision,
                  timing=1, newton_rtol=1e-10, gmres_rtol=1e-10) as sv:
        sv.set_state(wl.U0)
        st = sv.step()
        info = sv.info()
    n, m, nnzb = info["n_nodes"], info["n_tris"], info["nnzb"]
    nl, nlb = info["subdomain_rows"], info["subdomain_blocks"]
    w = 4.0 if precision else 8.0
    calls, b = st["kernel_calls"], st["alg_bytes"]
    assert calls["residual"] > 0 and calls["ilu_solve"] > 0 and calls["spmv"] > 0
    assert b["residual"] == pytest.approx(calls["residual"] * (136.0 * n + 12.0 * m))
    assert b["jacobian"] == pytest.approx(calls["jacobian"] * (56.0 * n + 48.0 * m + 25.0 * w * nnzb))
    assert b["ilu_solve"] == pytest.approx(calls["ilu_solve"] * (nlb * (25.0 * w + 4.0) + 72.0 * nl + 5.0 * n * w))
    # every SpMV reads its values, indices, x and writes y; the two-grid's launches also read r.
    # x is FP64 (8 bytes), or FP32 for the mixed path's products with the preconditioned basis
    plain = lambda wx: nnzb * (25.0 * w + 4.0) + 4.0 * (n + 1) + 5.0 * n * wx + 40.0 * n
    if precision == 0:
        extra = (b["spmv"] - calls["spmv"] * plain(8.0)) / (40.0 * n)
        assert 0 <= extra <= calls["spmv"] and abs(extra - round(extra)) < 1e-6
    else:
        assert calls["spmv"] * plain(4.0) <= b["spmv"] <= calls["spmv"] * (plain(8.0) + 40.0 * n)
    assert b["krylov"] > 0 and b["coarse_apply"] > 0 and b["ilu_factor"] > 0 and b["coarse_setup"] > 0
    assert all(np.isfinite(v) for v in b.values())
