"""bench.py's roofline arithmetic on recorded per-kernel timings (no GPU): the
dominant single-kernel class, achieved = the library's algorithmic bytes per
launch / mean launch time, traffic scaled from the small-case capture by the
units processed, the SpMV's average over its launches, and the whole-step
fraction (all classes' bytes over the timed steps / their device time)."""
import pytest

import bench


class _S:
    KERNEL_CLASSES = ("residual", "jacobian", "ilu_factor", "coarse_setup", "spmv", "ilu_solve", "coarse_apply",
                      "krylov")


def _res(spmv_ms=5.8, ilu_ms=17.0, spmv_calls=10, steps=2, ms_per_step=40.0):
    stats = []
    for _ in range(steps):
        kms = {k: 0.0 for k in _S.KERNEL_CLASSES}
        kcalls = {k: 0 for k in _S.KERNEL_CLASSES}
        kbytes = {k: 0.0 for k in _S.KERNEL_CLASSES}
        kms.update(spmv=spmv_ms, ilu_solve=ilu_ms, ilu_factor=1.0, krylov=3.0)
        kcalls.update(spmv=spmv_calls, ilu_solve=10, ilu_factor=1, krylov=10)
        kbytes.update(spmv=spmv_calls * 3.0e9, ilu_solve=10 * 3.5e9, ilu_factor=2.0e9, krylov=5.0e9)
        stats.append({"kernel_ms": kms, "kernel_calls": kcalls, "alg_bytes": kbytes})
    info = {"n_nodes": 2_000_000, "nnzb": 14_000_000, "subdomain_rows": 2_600_000, "subdomain_blocks": 18_000_000}
    return {"stats": stats, "info": info, "ms_per_step": ms_per_step}


def test_dominant_kernel_and_achieved_bandwidth():
    res = _res()
    roof, spmv, step, kms, kcalls = bench.roofline(_S, res, "fp64")
    assert roof["kernel"] == "ilu_solve"
    assert roof["avg_launch_ms"] == pytest.approx(1.7)
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx(3.5e9)
    assert roof["achieved"] == pytest.approx(3.5e9 / 1.7e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    b_small, units_small, key = bench.NCU_TRAFFIC[("ilu_solve", "fp64")]
    assert roof["traffic"] == pytest.approx(b_small * res["info"][key] / units_small)
    roof32, _, _, _, _ = bench.roofline(_S, res, "mixed")
    b32, u32, k32 = bench.NCU_TRAFFIC[("ilu_solve", "mixed")]
    assert roof32["traffic"] == pytest.approx(b32 * res["info"][k32] / u32)
    assert roof32["fp64_alu"] is None  # the FP64 rate applies to the FP64 path only
    assert roof["fp64_alu"]["fma_per_launch"] == 25 * res["info"]["subdomain_blocks"]
    assert spmv["gbs"] == pytest.approx(3.0e9 / 0.58e-3 / 1e9)


def test_spmv_dominant_takes_the_scaled_capture():
    res = _res(spmv_ms=30.0)
    roof, _, _, _, _ = bench.roofline(_S, res, "fp64")
    assert roof["kernel"] == "spmv"
    b_small, units_small, key = bench.NCU_TRAFFIC[("spmv", "fp64")]
    assert roof["traffic"] == pytest.approx(b_small * res["info"][key] / units_small)


def test_whole_step_fraction():
    res = _res()
    _, _, step, _, _ = bench.roofline(_S, res, "fp64")
    per_step = 10 * 3.0e9 + 10 * 3.5e9 + 2.0e9 + 5.0e9
    assert step["bytes_per_step"] == pytest.approx(per_step)
    assert step["achieved"] == pytest.approx(per_step / 40e-3 / 1e9)
    assert step["frac"] == pytest.approx(step["achieved"] / step["peak"])
