"""Host-side set-up invariants (seird_setup_check; no GPU).

The subdomain kernels trust the set-up without checking it: the ILU(k) solve
streams each stage into fixed shared-memory rings, reads a row's dependencies
from earlier stages with no synchronisation beyond the stage barrier, and
writes every owned row of z exactly once.  These tests build the set-up on the
CPU for the workload generators, geometric and non-geometric partitions, every
overlap and several levels of fill, and require every invariant to hold.
"""
import numpy as np
import pytest

from paper_2208_01839_gb300 import inputs as I

from paper_2208_01839_gb300 import build as _b  # noqa: E402

_b.build()
from paper_2208_01839_gb300 import seird as S  # noqa: E402


def _check(xy, tri, owner=None, **opts):
    st = S.setup_check(xy, tri, owner=owner, **opts)
    assert st["violations"] == 0
    assert st["n_nodes"] == len(xy) and st["n_tris"] == len(tri)
    # every subdomain has at least one forward and one backward stage
    assert st["forward_stages"] >= st["n_subdomains"] and st["backward_stages"] >= st["n_subdomains"]
    return st


@pytest.mark.parametrize("overlap", [0, 1, 2])
def test_square_default_partition(overlap):
    wl = I.square_workload(33)
    st = _check(wl.xy, wl.tri, n_subdomains=4, overlap=overlap)
    assert st["n_subdomains"] == 4
    # overlap adds rows: the subdomains hold at least every node once
    assert st["subdomain_rows"] >= st["n_nodes"]
    if overlap == 0:
        assert st["subdomain_rows"] == st["n_nodes"]


@pytest.mark.parametrize("overlap", [1, 2])
def test_irregular_mesh_box_partition(overlap):
    xy, tri, _ = I.irregular_mesh(3, 3000)
    _check(xy, tri, owner=I.box_partition(xy, 3, 2), overlap=overlap)


def test_random_partition_is_not_geometric():
    """Subdomains scattered over the mesh (every node's owner drawn at random):
    the level schedules and records must still hold."""
    xy, tri, _ = I.irregular_mesh(5, 1500)
    owner = np.random.default_rng(5).integers(0, 7, len(xy)).astype(np.int32)
    owner[:7] = np.arange(7)  # every subdomain owns a node
    _check(xy, tri, owner=owner, overlap=1)


def test_ontario_like_uneven_bisection():
    wl = I.ontario_workload(20_000, n_subdomains=16)
    st = _check(wl.xy, wl.tri, n_subdomains=16, overlap=2, seed=3, coarse=2)  # with the J Z segments
    assert st["n_subdomains"] == 16
    # a 5x5 block per node pair of the P1 graph: about 7 blocks per row
    assert 5 * st["n_nodes"] < st["nnzb"] < 9 * st["n_nodes"]


def test_single_subdomain_and_one_triangle():
    wl = I.square_workload(9)
    st = _check(wl.xy, wl.tri, n_subdomains=1, overlap=0)
    assert st["subdomain_rows"] == st["n_nodes"]
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2]], dtype=np.int32)
    st = _check(xy, tri, n_subdomains=1, overlap=0)
    assert st["nnzb"] == 9


def test_bad_mesh_is_reported_not_checked():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 2, 1]], dtype=np.int32)  # clockwise
    with pytest.raises(S.SeirdError, match="counter-clockwise"):
        S.setup_check(xy, tri)


@pytest.mark.parametrize("fill", [0, 2])
def test_ensemble_union_mesh(fill):
    """The union mesh an ensemble is solved on: sample k's copy of the mesh with its
    nodes offset by k n and the per-sample partition shifted by k P (block-diagonal
    system, no block couples two samples); with fill, no fill block couples two
    samples either (every sample's schedule is its own)."""
    xy, tri, _ = I.irregular_mesh(4, 800)
    owner = I.box_partition(xy, 2, 2).astype(np.int32)
    n, P, B = len(xy), int(owner.max()) + 1, 3
    uxy = np.concatenate([xy] * B)
    utri = np.concatenate([tri + k * n for k in range(B)]).astype(np.int32)
    uown = np.concatenate([owner + k * P for k in range(B)]).astype(np.int32)
    st = _check(uxy, utri, owner=uown, overlap=2, coarse=2, ilu_fill=fill)
    one = _check(xy, tri, owner=owner, overlap=2, coarse=2, ilu_fill=fill)
    assert st["n_subdomains"] == B * P and st["nnzb"] == B * one["nnzb"]
    assert st["subdomain_rows"] == B * one["subdomain_rows"]
    assert st["forward_stages"] == B * one["forward_stages"] and st["backward_stages"] == B * one["backward_stages"]


@pytest.mark.parametrize("group", [2, 3, 4, 16])
def test_coarse_units_spanning_several_subdomains(group):
    """Coarse units of `group` consecutive subdomains (the grouping the paper-scale
    partition uses): units tile the nodes and every J Z segment stays in one unit."""
    wl = I.ontario_workload(20_000, n_subdomains=16)
    st = _check(wl.xy, wl.tri, n_subdomains=16, overlap=2, seed=3, coarse=2, coarse_group=group)
    assert st["n_subdomains"] == 16


@pytest.mark.parametrize("fill", [1, 2, 3])
def test_iluk_factor_patterns(fill):
    """Block ILU(k) patterns: symmetric, holding R_p J R_p^T, fill naming no J block,
    and every invariant of the solve plans on the larger pattern; the level schedules
    deepen with k.  A fill level outside 0-8 is refused."""
    wl = I.ontario_workload(20_000, seed=1, n_subdomains=16)
    st0 = _check(wl.xy, wl.tri, n_subdomains=16, overlap=2, coarse=2)
    st = _check(wl.xy, wl.tri, n_subdomains=16, overlap=2, coarse=2, ilu_fill=fill)
    assert st["subdomain_rows"] == st0["subdomain_rows"]
    assert st["forward_stages"] > st0["forward_stages"] and st["backward_stages"] > st0["backward_stages"]
    # an owner array that is not geometric makes long fill chains
    owner = np.random.default_rng(fill).integers(0, 4, size=len(wl.xy)).astype(np.int32)
    _check(wl.xy, wl.tri, owner=owner, n_subdomains=4, overlap=1, ilu_fill=fill)
    for bad in (-1, 9):
        with pytest.raises(S.SeirdError):
            S.setup_check(wl.xy, wl.tri, n_subdomains=16, ilu_fill=bad)
