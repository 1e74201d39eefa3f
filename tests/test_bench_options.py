"""bench.py's solver options (no GPU): the subdomain fill each measured context gets and
what its config reports."""
import argparse

import bench


def test_fill_per_workload_and_precision():
    args = bench.parse([])
    assert bench.solver_options(args, "fp64", 4096)["ilu_fill"] == args.ilu_fill == 2
    assert bench.solver_options(args, "mixed", 4096)["ilu_fill"] == args.ilu_fill_mixed == 3
    assert bench.solver_options(args, "fp64", 16, ilu_fill=0)["ilu_fill"] == 0  # ensemble and adjoint
    # the 2.0M-node object's copy of the arguments gives both precisions its own fill
    args2 = argparse.Namespace(**vars(args))
    args2.ilu_fill = args2.ilu_fill_mixed = args.ilu_fill_2m
    assert args.ilu_fill_2m == 1
    for prec in ("fp64", "mixed"):
        assert bench.solver_options(args2, prec, 512)["ilu_fill"] == 1
    opts = bench.solver_options(args, "mixed", 4096)
    assert opts["precision"] == 1 and opts["n_subdomains"] == 4096 and opts["overlap"] == 2
    assert opts["coarse"] == 2 and opts["predictor"] == 5 and opts["gmres_one_pass"] == 0


def test_fill_flags_and_reported_solver():
    args = bench.parse(["--ilu-fill", "1", "--ilu-fill-mixed", "0", "--ilu-fill-2m", "2"])
    assert bench.solver_options(args, "fp64", 64)["ilu_fill"] == 1
    assert bench.solver_options(args, "mixed", 64)["ilu_fill"] == 0

    class _WL:
        name, n, dt = "ontario_like_test", 10, 0.5
        tri = [[0, 1, 2]]

    assert bench.workload_config(_WL, args, 64)["subdomain_solver"] == "block ILU(1)"
