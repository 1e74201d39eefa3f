"""The seeded input generators (no GPU): the structure the tests and the bench
rely on -- counter-clockwise, non-degenerate meshes near the requested size,
positive densities and states, partitions that cover every node, rate samples
inside their log-uniform band -- and reproducibility from the seed."""
import numpy as np
import pytest

from paper_2208_01839_gb300 import inputs as I


def _areas(xy, tri):
    p0, p1, p2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    return 0.5 * ((p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1]))


@pytest.mark.parametrize("nside", [2, 9, 33])
def test_structured_mesh(nside):
    xy, tri = I.structured_mesh(nside)
    assert xy.shape == (nside * nside, 2) and tri.shape == (2 * (nside - 1) ** 2, 3)
    a = _areas(xy, tri)
    assert np.all(a > 0) and abs(a.sum() - 1.0) < 1e-12  # tiles the unit square


@pytest.mark.parametrize("seed,n_target", [(0, 500), (3, 3000), (7, 20000)])
def test_irregular_mesh(seed, n_target):
    xy, tri, poly = I.irregular_mesh(seed, n_target)
    assert 0.8 * n_target <= len(xy) <= 1.2 * n_target
    assert np.all(_areas(xy, tri) > 0)
    assert np.all((xy >= 0) & (xy <= 1))
    used = np.zeros(len(xy), bool)
    used[tri.ravel()] = True
    assert used.all()  # no orphan nodes
    xy2, tri2, _ = I.irregular_mesh(seed, n_target)
    assert np.array_equal(xy, xy2) and np.array_equal(tri, tri2)


def test_ontario_workload_state_and_partition():
    wl = I.ontario_workload(20_000, n_subdomains=16)
    assert wl.U0.shape == (len(wl.xy), 5) and np.all(wl.U0 >= 0)
    N = wl.U0.sum(axis=1)
    assert N.min() > 0 and N.max() / N.min() > 5  # urban peaks over a rural floor
    assert wl.U0[:, 2].sum() > 0 and wl.U0[:, 3].sum() == 0 and wl.U0[:, 4].sum() == 0  # seeds infected only
    assert wl.dt == 0.5 and wl.overlap == 2


@pytest.mark.parametrize("px,py", [(1, 1), (2, 2), (3, 2)])
def test_box_partition_covers_every_node(px, py):
    xy, tri, _ = I.irregular_mesh(2, 2000)
    owner = I.box_partition(xy, px, py)
    assert owner.shape == (len(xy),) and owner.min() == 0
    assert set(np.unique(owner)) <= set(range(px * py))


def test_rate_samples_band_and_seed():
    base = I.params_ontario(1e4)
    s = I.rate_samples(base, 64, seed=5)
    again = I.rate_samples(base, 64, seed=5)
    other = I.rate_samples(base, 64, seed=6)
    names = ("beta_i", "beta_e", "sigma", "gamma_e", "gamma_r", "gamma_d")
    f = np.array([[getattr(q, k) / getattr(base, k) for k in names] + [q.nu[c] / base.nu[c] for c in range(4)]
                  for q in s])
    assert np.all(f >= 0.5) and np.all(f <= 1.5)
    lf = np.log(f)  # log-uniform on [log 0.5, log 1.5]: spread over the band, not clustered
    assert lf.min() < np.log(0.6) and lf.max() > np.log(1.35)
    assert [q.as_dict() for q in s] == [q.as_dict() for q in again]
    assert [q.as_dict() for q in s] != [q.as_dict() for q in other]
    # the rates outside the sampled ten stay at their base values
    assert all(q.A == base.A and q.alpha == base.alpha and q.mu == base.mu for q in s)
