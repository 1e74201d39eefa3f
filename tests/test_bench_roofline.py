"""bench.py's roofline arithmetic on recorded per-kernel timings (no GPU):
the dominant single-kernel class, achieved = algorithmic bytes per launch /
mean launch time, traffic scaled from the small-case capture by the units
processed, and the SpMV's bytes counting the r that the two-grid's fused
r - J z launches also read."""
import pytest

import bench


class _S:
    KERNEL_CLASSES = ("residual", "jacobian", "ilu_factor", "coarse_setup", "spmv", "ilu_solve", "coarse_apply",
                      "krylov")


def _res(spmv_ms=5.8, ilu_ms=17.0, spmv_calls=10, coarse_calls=5):
    kms = {k: 0.0 for k in _S.KERNEL_CLASSES}
    kcalls = {k: 0 for k in _S.KERNEL_CLASSES}
    kms.update(spmv=spmv_ms, ilu_solve=ilu_ms, ilu_factor=1.0)
    kcalls.update(spmv=spmv_calls, ilu_solve=10, ilu_factor=1, coarse_apply=coarse_calls)
    info = {"n_nodes": 2_000_000, "nnzb": 14_000_000, "subdomain_rows": 2_600_000, "subdomain_blocks": 18_000_000}
    return {"stats": [{"kernel_ms": kms, "kernel_calls": kcalls}], "info": info}


def test_dominant_kernel_and_achieved_bandwidth():
    res = _res()
    roof, spmv, kms, kcalls = bench.roofline(_S, res, "fp64", coarse=2)
    assert roof["kernel"] == "ilu_solve"
    ab = bench.algorithmic_bytes("ilu_solve", res["info"], "fp64")
    assert roof["avg_launch_ms"] == pytest.approx(1.7)
    assert roof["achieved"] == pytest.approx(ab / 1.7e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    b_small, units_small, key = bench.NCU_TRAFFIC[("ilu_solve", "fp64")]
    assert roof["traffic"] == pytest.approx(b_small * res["info"][key] / units_small)
    assert roof["fp64_alu"]["fma_per_launch"] == 25 * res["info"]["subdomain_blocks"]


def test_spmv_bytes_count_the_fused_residual_reads():
    res = _res()
    plain = bench.algorithmic_bytes("spmv", res["info"], "fp64")
    _, sp2, _, _ = bench.roofline(_S, res, "fp64", coarse=2)
    _, sp1, _, _ = bench.roofline(_S, res, "fp64", coarse=1)
    assert sp1["algorithmic_bytes"] == plain  # no fused launches without the two-grid
    # half of the launches (5 of 10) also read r: 5n doubles
    assert sp2["algorithmic_bytes"] == pytest.approx(plain + 0.5 * 5 * 2_000_000 * 8)
    assert sp2["gbs"] == pytest.approx(sp2["algorithmic_bytes"] / 0.58e-3 / 1e9)
