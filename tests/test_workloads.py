"""The seeded input generators: the SplitMix64 reference vector, counter-mode
slicing, and the distributions the workloads state."""
import numpy as np

from paper_2602_05179_gb300 import workloads as wl


def test_splitmix64_reference_vector():
    # first outputs of SplitMix64 started from state 0 (published reference
    # implementation): state += G; return mix(state)
    assert wl._mix_int(wl.G) == 0xE220A8397B1DCDAF
    assert wl._mix_int(2 * wl.G & wl.MASK) == 0x6E789E6AA1B965F4
    z = np.array([wl.G, 2 * wl.G & wl.MASK], dtype=np.uint64)
    assert [int(v) for v in wl._mix(z)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4]


def test_counter_mode_slices_agree():
    a = wl.draws(5, 3, 0, 1000)
    b = wl.draws(5, 3, 400, 100)
    np.testing.assert_array_equal(a[400:500], b)
    spec = wl.SPLIT_C1
    full = wl.split_demands(spec, 0, 40)
    np.testing.assert_array_equal(full[17:29], wl.split_demands(spec, 17, 29))


def test_distributions():
    u = wl.uniform_int(1, 3, 0, 200_000, 1, 30)
    assert u.min() == 1 and u.max() == 30 and abs(u.mean() - 15.5) < 0.05
    q = wl.poisson_clip(0, 3, 0, 200_000, 10.0, 1, 100)
    assert q.min() >= 1 and abs(q.mean() - 10.0) < 0.05 and abs(q.var() - 10.0) < 0.2
    cdf = wl.poisson_cdf(8.0)
    assert np.all(np.diff(cdf) >= 0) and cdf[-1] >= 1 - 2 ** -52
    f = wl.uniform_f32(2, 5, 0, 100_000, 5.0, 50.0)
    assert f.dtype == np.float32 and f.min() >= 5.0 and f.max() < 50.0
    xy = wl.coords_f32(0, 1, 500)
    assert tuple(xy[0]) == (50.0, 50.0) and xy[1:].min() >= 0 and xy[1:].max() < 100
    t = wl.permutation(0, 2, 1000)
    assert sorted(t.tolist()) == list(range(1, 1001))


def test_workload_shapes():
    tour, xy, dist = wl.split_tour(wl.ADJOINT_C5)
    assert dist.shape == (301, 301) and dist.dtype == np.float32
    assert np.allclose(dist, dist.T) and np.all(np.diag(dist) == 0)
    nb = wl.batch_sizes(wl.BATCH_C4)
    assert nb.min() >= 20 and nb.max() <= 1000 and len(nb) == 4096
    cons = wl.reinsert_consumption(wl.REINSERT_C3, 0, 100)
    assert cons.shape == (100, 60) and abs(cons.mean() - 8.0) < 0.3
