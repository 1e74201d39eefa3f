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
    roof, spmv, step, kms, kcalls = bench.roofline(_S, res, "mixed")
    assert roof["kernel"] == "ilu_solve"
    assert roof["bound"] == "hbm"  # FP32 work: the HBM roofline
    assert roof["avg_launch_ms"] == pytest.approx(1.7)
    assert roof["algorithmic_bytes_per_launch"] == pytest.approx(3.5e9)
    assert roof["achieved"] == pytest.approx(3.5e9 / 1.7e-3 / 1e9)
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    b32, u32, k32 = bench.NCU_TRAFFIC[("ilu_solve", "mixed")]
    assert roof["traffic"] == pytest.approx(b32 * res["info"][k32] / u32)
    assert roof["fp64_alu"] is None  # the FP64 rate applies to the FP64 path only
    assert spmv["gbs"] == pytest.approx(3.0e9 / 0.58e-3 / 1e9)
    assert spmv["frac_of_fp64"] is None


def test_fp64_work_takes_the_longer_of_the_hbm_and_fp64_bounds():
    res = _res()
    roof, spmv, _, _, _ = bench.roofline(_S, res, "fp64")
    fma = 25 * res["info"]["subdomain_blocks"]
    peak_tf = 152 * 2 * 2 * 2.070e9 / 1e12  # 152 SMs, 2 FP64 FMA per clock, 2.07 GHz
    assert bench.FP64_PEAK_TFLOPS == pytest.approx(peak_tf)
    # 2 x 4.5e8 flop at 1.259 TFLOP/s (0.71 ms) outlasts 3.5e9 bytes at the HBM peak (0.52 ms)
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s"
    assert roof["fma_per_launch"] == fma
    assert roof["achieved"] == pytest.approx(2 * fma / 1.7e-3 / 1e12)
    assert roof["frac"] == pytest.approx(roof["achieved"] / peak_tf)
    assert roof["hbm"]["achieved"] == pytest.approx(3.5e9 / 1.7e-3 / 1e9)
    b_small, units_small, key = bench.NCU_TRAFFIC[("ilu_solve", "fp64")]
    assert roof["traffic"] == pytest.approx(b_small * res["info"][key] / units_small)
    assert spmv["frac_of_fp64"] == pytest.approx(2 * 25 * res["info"]["nnzb"] / 0.58e-3 / 1e12 / peak_tf)
    # with more bytes per FMA the same launch is bound by HBM instead
    res["info"]["subdomain_blocks"] = 1_000_000
    roof, _, _, _, _ = bench.roofline(_S, res, "fp64")
    assert roof["bound"] == "hbm" and roof["fp64_alu"]["fma_per_launch"] == 25_000_000


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
