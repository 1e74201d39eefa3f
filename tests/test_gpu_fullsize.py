"""Full-size workloads in the benchmark's launch configuration (bench.py's solver
options and autotuner, its workload sizes).

The whole-mesh oracle cannot run at these sizes, so the GPU states are checked
through quantities the oracle can compute one by one and through properties
that hold at any size:
  * the oracle's residual F(u^{n+1}; u^n) at sampled nodes, from the incident
    triangles only, is at the Newton tolerance (relative to the mass-term scale);
  * total population is conserved (alpha = mu = 0, no-flux boundary, Section 2.1);
  * d^{n+1} = d^n + dt gamma_D i^{n+1} node by node (degree-5 rule, Eq. seird5);
  * every compartment stays nonnegative;
  * the mixed-precision path agrees with the FP64 path to 1e-6 relative L2 per
    compartment at the 1e-8 Newton tolerance (config 3 and the paper-scale mesh).
"""
import math

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

import bench  # noqa: E402

_ARGS = bench.parse([])


def bench_opts(precision, subdomains, ilu_fill=None):
    """The options bench.py times: solver_options of its default arguments, autotuner on."""
    return dict(bench.solver_options(_ARGS, "mixed" if precision else "fp64", subdomains, ilu_fill), autotune=1)


def _node_mass(xy, tri):
    area, _ = O.geometry(xy, tri)
    w = np.zeros(len(xy))
    np.add.at(w, tri, np.repeat(area[:, None] / 3.0, 3, axis=1))  # int phi_i
    return w


def _check_step_properties(wl, Un, U, n_samples=300, seed=0, res_final=None):
    rng = np.random.default_rng(seed)
    # sampled residual from the oracle, near the infection seeds and anywhere
    hot = np.argsort(-Un[:, 2])[:n_samples // 2]
    nodes = np.unique(np.concatenate([hot, rng.choice(wl.n, n_samples // 2, replace=False)]))
    F = O.residual_at_nodes(wl.xy, wl.tri, wl.params, wl.dt, U, Un, nodes, bfield=wl.beta_field)
    Ms = O.residual_at_nodes(wl.xy, wl.tri, wl.params, 0.0, np.abs(U), np.zeros_like(U), nodes)
    # ||F|| <= 1e-8 ||F(u^n)||, and ||F(u^n)|| is at most a few percent of ||M u|| here,
    # so a node's residual is far below 1e-7 of the mass-term scale; a wrong term
    # in the discrete system would leave O(dt * rate) = O(1e-2) of it
    assert np.abs(F).max() <= 1e-7 * np.abs(Ms).max(), (np.abs(F).max(), np.abs(Ms).max())
    w = _node_mass(wl.xy, wl.tri)
    tot0, tot1 = w @ Un.sum(axis=1), w @ U.sum(axis=1)
    if res_final is None:
        assert abs(tot1 - tot0) <= 1e-8 * tot0
    else:
        # sum_{i,c} F_ic = tot1 - tot0 exactly (sum_i phi_i = 1, the reaction terms sum to
        # zero over the compartments), so |tot1 - tot0| <= sqrt(5 n) ||F||
        assert abs(tot1 - tot0) <= math.sqrt(5 * wl.n) * res_final * 1.01 + 1e-13 * tot0, (tot1 - tot0, res_final)
    # d - d^n - dt gamma_D i = M^{-1} F_D: small at the Newton tolerance, O(1) for a wrong term
    drow = U[:, 4] - Un[:, 4] - wl.dt * wl.params.gamma_d * U[:, 2]
    assert np.abs(drow).max() <= 1e-3 * np.abs(U[:, 4] - Un[:, 4]).max()
    assert U.min() >= -1e-10 * np.abs(U).max()


@pytest.mark.parametrize("precision", [0, 1])
def test_ontario_2m_steps(precision):
    """Config 2: 2.0M-node Ontario-like mesh, 512 subdomains, overlap 2, coarse on."""
    wl = I.ontario_workload(2_000_000)
    with S.Solver(wl.xy, wl.tri, wl.params, dt=wl.dt, **bench_opts(precision, 512, _ARGS.ilu_fill_2m)) as sv:
        sv.set_state(wl.U0)
        sv.run(2)
        U1 = sv.get_state()
        sv.step()
        U2 = sv.get_state()
    _check_step_properties(wl, U1, U2)


def test_mixed_vs_fp64_on_the_1024_square():
    """Config 3: the urban generator on a 1024x1024 structured mesh (5.2M unknowns);
    mixed precision against the FP64 GPU path, and both against the oracle's
    sampled residual."""
    wl = I.ontario_workload(1024 * 1024, structured=True, nside=1024, n_subdomains=512)
    out = {}
    for precision in (0, 1):
        with S.Solver(wl.xy, wl.tri, wl.params, dt=wl.dt, **bench_opts(precision, 512)) as sv:
            sv.set_state(wl.U0)
            sv.run(3)
            Un = sv.get_state()
            sv.step()
            out[precision] = (Un, sv.get_state())
    for precision in (0, 1):
        _check_step_properties(wl, *out[precision], seed=precision)
    a, b = out[1][1], out[0][1]
    rel = [np.linalg.norm(a[:, c] - b[:, c]) / np.linalg.norm(b[:, c]) for c in range(5)]
    assert max(rel) <= 1e-6, rel


def test_paper_scale_steps_fp64_and_mixed():
    """The headline workload: 18.4M nodes (92M unknowns), 4096 subdomains, the bench's
    options, FP64 and mixed precision from the same start; each step's properties,
    and the two paths' states against each other."""
    wl = I.ontario_workload(bench.PAPER_SCALE_NODES, seed=_ARGS.seed, n_subdomains=bench.PAPER_SCALE_SUBDOMAINS)
    out = {}
    for precision in (0, 1):
        with S.Solver(wl.xy, wl.tri, wl.params, dt=wl.dt,
                      **bench_opts(precision, bench.PAPER_SCALE_SUBDOMAINS)) as sv:
            assert sv.info()["n_subdomains"] == bench.PAPER_SCALE_SUBDOMAINS
            sv.set_state(wl.U0)
            sv.run(2)
            Un = sv.get_state()
            st = sv.step()
            out[precision] = (Un, sv.get_state(), st["res_final"])
    for precision in (0, 1):
        Un, U, res = out[precision]
        _check_step_properties(wl, Un, U, seed=precision, res_final=res)
    a, b = out[1][1], out[0][1]
    rel = [np.linalg.norm(a[:, c] - b[:, c]) / np.linalg.norm(b[:, c]) for c in range(5)]
    assert max(rel) <= 1e-6, rel
