"""Independent point sets of uneven size multiplied as one unit
(hodlr2d_batch_*): the graph form equal bit for bit to the per-set products,
the persistent form within rounding of them (its sums run in another
order), with 1 to 8 right-hand sides per set, across replays, when x changes
in place and when a handle's working memory moves between calls.  The
shape autotuner keeps one of its candidates; the leaf-size autotuner returns
one of its candidates with its timings."""
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


TOL = {"f64": 1e-13, "f32": 1e-5}


@pytest.mark.parametrize("form", ["graph", "persistent"])
@pytest.mark.parametrize("mode", ["f64", "f32"])
def test_batch_equals_individual_products(pkg, mode, form):
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
    b = pkg.Batch(mats, form=form)
    for rep in range(4):
        if rep == 2:  # new data in the same buffers: the recorded launch sees it
            for x in xs:
                x.mul_(-0.5)
        if rep == 3:  # a handle's working memory moves: the batch is set up again
            big = torch.zeros((9, mats[0].n), dtype=torch.float64, device="cuda")
            mats[0].matvec(big.t(), mode=mode)
        b.matvec(xs, ys, mode=mode)
        b.check()
        assert b.last_form == form
        for g, x, y in zip(mats, xs, ys):
            ref = g.matvec(x.t().contiguous(), mode=mode).t()
            if form == "graph":
                assert torch.equal(y, ref)
            else:
                err = float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref))
                assert err <= TOL[mode], err
    b.close()


def test_batch_shape_autotuner(pkg):
    sets = inputs.point_sets(6, seed=6, nmin=2000, nmax=20000)
    mats = [pkg.HODLR2D(p, pkg.kernel("imq", 1.0 / np.sqrt(len(p))), 32, 1e-8) for p in sets]
    for g in mats:
        g.prepare("f32")
    rng = np.random.default_rng(2)
    xs = [torch.from_numpy(rng.standard_normal((2, g.n))).cuda() for g in mats]
    ys = [torch.empty_like(x) for x in xs]
    b = pkg.Batch(mats, form="persistent")
    (pr, wr), ms = b.autotune(xs, ys, mode="f32", reps=2)
    assert pr in (0, 128, 256, 512, 1024, 2048) and wr in (0, 48, 64) and wr <= pr and ms > 0
    table = b.tune_table()
    assert table[-1][:4] == (-1, -1, -1, -1)  # the graph form, timed last
    b.set_form("auto")
    b.matvec(xs, ys, mode="f32")
    want = "graph" if table[-1][4] < ms else "persistent"
    assert b.last_form == want
    b.set_form("persistent")
    b.matvec(xs, ys, mode="f32")
    b.check()
    assert len(b.phase_ms()) == 5 and all(t >= 0 for t in b.phase_ms())
    for g, x, y in zip(mats, xs, ys):
        ref = g.matvec(x.t().contiguous(), mode="f32").t()
        assert float(torch.linalg.norm(y - ref) / torch.linalg.norm(ref)) <= TOL["f32"]
    b.close()


def test_autotune_leaf(pkg):
    p = inputs.uniform(20000, seed=2)
    best, times = pkg.autotune_leaf(p, pkg.kernel("imq", 0.01), 1e-8, candidates=(16, 32, 64))
    assert best in (16, 32, 64) and set(times) == {16, 32, 64}
    assert all(t > 0 for t in times.values())


def test_batch_rejects_a_repeated_handle(pkg):
    from paper_2204_05536_gb300 import _lib
    p = inputs.uniform(2000, seed=7)
    g = pkg.HODLR2D(p, pkg.kernel("imq", 0.02), 32, 1e-8)
    h = pkg.HODLR2D(p, pkg.kernel("imq", 0.02), 32, 1e-8)
    with pytest.raises(_lib.HodlrError) as ei:
        pkg.Batch([g, h, g])
    assert ei.value.code == _lib.ERR_ARG
    pkg.Batch([g, h]).close()
