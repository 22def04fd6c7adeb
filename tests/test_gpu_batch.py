"""Independent point sets of uneven size multiplied with one CUDA graph
launch (hodlr2d_batch_*): equal bit for bit to the per-set products, with 1
to 8 right-hand sides per set, across replays and when x changes in place.
The leaf-size autotuner returns one of its candidates with its timings."""
import numpy as np
import pytest

from paper_2204_05536_gb300 import inputs

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_05536_gb300 as p
    p.load()
    return p


@pytest.mark.parametrize("mode", ["f64", "f32"])
def test_batch_equals_individual_products(pkg, mode):
    sets = inputs.point_sets(12, seed=4, nmin=300, nmax=6000)
    rng = np.random.default_rng(1)
    mats, xs, ys = [], [], []
    for i, p in enumerate(sets):
        g = pkg.HODLR2D(p, pkg.kernel("imq", 1.0 / np.sqrt(len(p))), 32, 1e-8)
        if mode != "f64":
            g.prepare(mode)
        mats.append(g)
        nr = int(rng.integers(1, 9))
        xs.append(torch.from_numpy(rng.standard_normal((nr, len(p)))).cuda())
        ys.append(torch.zeros_like(xs[-1]))
    b = pkg.Batch(mats)
    for rep in range(3):
        if rep == 2:  # new data in the same buffers: the recorded graph sees it
            for x in xs:
                x.mul_(-0.5)
        b.matvec(xs, ys, mode=mode)
        torch.cuda.synchronize()
        for g, x, y in zip(mats, xs, ys):
            ref = g.matvec(x.t().contiguous(), mode=mode).t()
            assert torch.equal(y, ref)


def test_autotune_leaf(pkg):
    p = inputs.uniform(20000, seed=2)
    best, times = pkg.autotune_leaf(p, pkg.kernel("imq", 0.01), 1e-8, candidates=(16, 32, 64))
    assert best in (16, 32, 64) and set(times) == {16, 32, 64}
    assert all(t > 0 for t in times.values())
