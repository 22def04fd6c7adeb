"""Same-factor parity (P1) at the sizes and in the launch forms the benchmark
runs, through the C ABI (needs a GB300).

The GPU handle is built with compress=False (tree and lists only) and takes
the oracle's factors through hodlr2d_import_factors, so both sides multiply
with identical U and V (Alg. 2) and differ only by rounding order:
  - N = 2^18 of the benchmark recipe (uniform points, multiquadric
    a = 1/sqrt(N), leaf 64, eps 1e-8, root [-1,1]^2; kappa = 7): levels 1-3
    hold boxes of more than 2048 points, which the binary64 product runs in
    two passes (projection over row chunks, chunk sums, expansion), the
    float-float product partly in two passes and partly with the 512-thread
    register pair kernel; every mode against the oracle, one and three
    right-hand sides;
  - N = 2^17, 32 right-hand sides: the many-RHS forms (tensor-core bfloat16
    coarse levels, the binary32 tiled projection, the multi-RHS pair
    kernel) against the oracle's 32-column product;
  - N = 2^20 (marked slow): the benchmark's own workload, binary64 and
    float-float, one right-hand side;
  - a batch of independent point sets multiplied with one graph launch or
    one persistent kernel, each set against its own oracle, and the
    persistent kernel's bounded barrier wait giving up on request.
Bounds: 1e-12 (relative 2-norm) for binary64 and float-float, 5e-6 for
binary32 factors and sums, 2e-2 for bfloat16 factors (the factors' own
rounding, 2^-9 relative per value, sets it).
"""
import numpy as np
import pytest

from paper_2204_05536_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = (-1.0, -1.0, 2.0)
BOUND = {"f64": 1e-12, "df32": 1e-12, "f32": 5e-6, "bf16": 2e-2}


@pytest.fixture(scope="module")
def h2d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_05536_gb300 as pkg
    pkg.load()
    return pkg


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def same_factors(h2d, oracle, n, nrhs, seed_x=1):
    """Oracle build of the benchmark recipe at n points, a GPU handle holding
    its factors, x (n x nrhs) and the oracle's product."""
    pts = inputs.uniform(n, seed=0)
    a = 1.0 / np.sqrt(n)
    o = oracle.Oracle(pts, oracle.kernel("mq", a), 64, 1e-8, root=ROOT)
    g = h2d.HODLR2D(pts, h2d.kernel("mq", a), 64, 1e-8, root=ROOT, compress=False)
    g.import_factors(*o.export_factors())
    x = inputs.rhs(n, nrhs, seed=seed_x)
    if nrhs == 1:
        x = x[:, None]
    return o, g, x, o.matvec(x)


@pytest.fixture(scope="module")
def bench_recipe_2e18(h2d, oracle):
    o, g, x, y_o = same_factors(h2d, oracle, 1 << 18, 3)
    assert o.kappa == 7
    for mode in ("df32", "f32", "bf16"):
        g.prepare(mode)
    return g, x, y_o


def gpu_product(g, x, mode):
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    return g.matvec(xd if x.shape[1] > 1 else xd[:, 0], mode=mode).cpu().numpy().reshape(x.shape)


@pytest.mark.parametrize("mode", ["f64", "df32", "f32", "bf16"])
def test_p1_bench_recipe_2e18_one_rhs(h2d, bench_recipe_2e18, mode):
    g, x, y_o = bench_recipe_2e18
    g.profile(True)
    y = gpu_product(g, x[:, :1], mode)
    prof = g.get_profile()
    g.profile(False)
    if mode == "f64":  # levels 1-3 (boxes of 4096+ points) run in two passes
        assert prof["proj"]["launches"] == 1 and prof["exp"]["launches"] == 1
    assert rel(y, y_o[:, :1]) <= BOUND[mode], mode


@pytest.mark.parametrize("mode", ["f64", "df32", "f32", "bf16"])
def test_p1_bench_recipe_2e18_three_rhs(h2d, bench_recipe_2e18, mode):
    g, x, y_o = bench_recipe_2e18
    y = gpu_product(g, x, mode)
    for c in range(3):
        assert rel(y[:, c], y_o[:, c]) <= BOUND[mode], (mode, c)


def test_p1_32_rhs_2e17(h2d, oracle):
    """32 right-hand sides at N = 2^17 in every mode against the oracle's
    32-column Alg. 2 product on the same factors: the bfloat16 coarse levels
    on the tensor cores, binary32 with the tiled projection, the multi-RHS
    register pair kernel for boxes of <= 256 points."""
    o, g, x, y_o = same_factors(h2d, oracle, 1 << 17, 32, seed_x=3)
    for mode in ("f64", "df32", "f32", "bf16"):
        if mode != "f64":
            g.prepare(mode)
        y = gpu_product(g, x, mode)
        assert rel(y, y_o) <= BOUND[mode], mode
        worst = max(rel(y[:, c], y_o[:, c]) for c in range(32))
        assert worst <= BOUND[mode], (mode, worst)


@pytest.mark.slow
def test_p1_bench_workload_2e20(h2d, oracle):
    """The benchmark's workload itself (N = 2^20, kappa = 8): the binary64
    and float-float products on the oracle's factors."""
    o, g, x, y_o = same_factors(h2d, oracle, 1 << 20, 1)
    assert o.kappa == 8
    g.prepare("df32")
    for mode in ("f64", "df32"):
        y = gpu_product(g, x, mode)
        assert rel(y, y_o) <= BOUND[mode], mode


@pytest.fixture(scope="module")
def batch_sets(h2d, oracle):
    """Five independent point sets of 1500-6000 points (leaves 32-64), IMQ,
    GPU handles on the oracle's factors, 1-4 right-hand sides each, and each
    set's oracle product."""
    sets = inputs.point_sets(5, seed=3, nmin=1500, nmax=6000)
    rng = np.random.default_rng(4)
    mats, orcs, xs = [], [], []
    for i, p in enumerate(sets):
        a = 1.0 / np.sqrt(len(p))
        leaf = (32, 64, 48, 64, 32)[i]
        o = oracle.Oracle(p, oracle.kernel("imq", a), leaf, 1e-8)
        g = h2d.HODLR2D(p, h2d.kernel("imq", a), leaf, 1e-8, compress=False)
        g.import_factors(*o.export_factors())
        g.prepare("f32")
        r = int(rng.integers(1, 5))
        xs.append(rng.standard_normal((r, len(p))))
        mats.append(g)
        orcs.append(o)
    want = [o.matvec(np.ascontiguousarray(x.T)) for o, x in zip(orcs, xs)]
    return mats, xs, want


@pytest.mark.parametrize("form,shapes,blocks,place", [("graph", None, None, None),
                                                      ("persistent", None, None, None),
                                                      ("persistent", (0, 0), 2, 0),
                                                      ("persistent", (128, 0), 4, 1),
                                                      ("persistent", (512, 48), 3, 3),
                                                      ("persistent", (2048, 64), 3, 2)])
def test_batch_against_oracle(h2d, batch_sets, form, shapes, blocks, place):
    """hodlr2d_batch_matvec over independent handles of uneven size against
    each set's own oracle product on the same factors, in binary64 and
    binary32: one graph launch (recorded on the first call, replayed on the
    second), or one persistent cooperative kernel (five phases behind
    bounded grid barriers) with its default shapes, with every level in two
    passes (0, 0), with pairs up to 128 points four per 256-thread unit
    (128, 0), and with pairs up to 512 points, those of <= 48 one per warp
    (512, 48), and with pairs up to 2048 points (binary64: 1024), at most
    8 rows a thread (2048, 64); at 2, 4 and 3 resident blocks per SM; with
    the near field in
    the first phase or beside the expansions, the one-warp pairs beside the
    chunk sums."""
    mats, xs, want = batch_sets
    b = h2d.Batch(mats, stream=torch.cuda.current_stream(), form=form)
    if shapes is not None:
        b.set_shapes(*shapes)
        b.set_blocks_per_sm(blocks)
        b.set_placement(place)
    xd = [torch.from_numpy(x).cuda() for x in xs]
    for mode in ("f64", "f32"):
        ys = [torch.empty_like(x) for x in xd]
        for _ in range(2):
            b.matvec(xd, ys, mode=mode)
            b.check()
            assert b.last_form == form
            if form == "persistent":  # one cooperative launch, replayed from a CUDA graph
                assert b.persistent_recorded is True
            for y, w in zip(ys, want):
                assert rel(y.cpu().numpy().T, w) <= BOUND[mode], mode
    b.close()


def test_batch_persistent_wait_gives_up(h2d, batch_sets):
    """The persistent form's grid-barrier waits are bounded: with a wait
    limit of 0 polls every block gives up at the first barrier, the launch
    ends without writing y, hodlr2d_batch_check reports HODLR2D_ERR_TIMEOUT,
    and the context stays usable (the next product with the default limit is
    right)."""
    from paper_2204_05536_gb300 import _lib
    mats, xs, want = batch_sets
    b = h2d.Batch(mats, stream=torch.cuda.current_stream(), form="persistent")
    xd = [torch.from_numpy(x).cuda() for x in xs]
    ys = [torch.full_like(x, 123.0) for x in xd]
    b.set_wait_limit(0)
    b.matvec(xd, ys, mode="f64")
    with pytest.raises(_lib.HodlrError) as ei:
        b.check()
    assert ei.value.code == _lib.ERR_TIMEOUT
    assert all(bool((y == 123.0).all()) for y in ys)  # the combine never ran
    b.check()  # the record was cleared
    b.set_wait_limit(1 << 22)
    b.matvec(xd, ys, mode="f64")
    b.check()
    for y, w in zip(ys, want):
        assert rel(y.cpu().numpy().T, w) <= BOUND["f64"]
    b.close()


def test_df32_rank_near_200_blocks(h2d, oracle):
    """Long float-float sums: 1/r on N = 2^15 points, leaf 64 (kappa = 5),
    eps = 1e-15, so the vertex-sharing pairs of the 8192-point boxes (level
    1, two passes) and of the 2048-point boxes (level 2, register pair
    kernel) carry ranks of about 150-200 and their projections sum 8192 or
    2048 terms.  The float-float accumulator folds its error terms back
    every 16 terms.  Bounds, on the oracle's factors: binary64 1e-12;
    float-float 1e-11, derived as its rounding per multiply-add (about
    2^-46: the low-times-low product is dropped and the cross terms are
    rounded in binary32) times the cancellation of an 8192-term dot product
    with random x (about sqrt(8192) = 90), times the two passes and the
    handful of levels that add up: 1.4e-14 x 90 x 8 = 1e-11.  Measured:
    4.0e-12 (the workloads of eps >= 1e-10 stay below 1e-12)."""
    n = 1 << 15
    pts = inputs.uniform(n, seed=3)
    o = oracle.Oracle(pts, oracle.kernel("inv_r"), 64, 1e-15)
    ranks = [d["rank"] for d, _, _ in o.pairs()]
    assert max(ranks) >= 150
    g = h2d.HODLR2D(pts, h2d.kernel("inv_r"), 64, 1e-15, compress=False)
    g.import_factors(*o.export_factors())
    g.prepare("df32")
    x = inputs.rhs(n, 1, seed=5)[:, None]
    y_o = o.matvec(x)
    for mode, bound in (("f64", 1e-12), ("df32", 1e-11)):
        y = gpu_product(g, x, mode)
        assert rel(y, y_o) <= bound, mode


@pytest.mark.parametrize("form", ["graph", "persistent"])
def test_batch_degenerate_sets(h2d, oracle, form):
    """Batches that mix degenerate sets with ordinary ones, each against its
    own oracle product on the same factors: a single point, a set no larger
    than one leaf (kappa = 0: the whole matrix is the dense self block, no
    stored pairs), a set of exactly one leaf plus one point (kappa = 1), a
    set whose points all sit in one corner (deep, lopsided tree with empty
    boxes), and an ordinary set; one and five right-hand sides."""
    rng = np.random.default_rng(11)
    corner = 0.9 + 0.1 * rng.uniform(0.0, 1.0, (700, 2))
    corner = np.concatenate([corner, rng.uniform(-1.0, 1.0, (60, 2))])
    sets = [rng.uniform(-1.0, 1.0, (1, 2)), inputs.uniform(32, seed=12),
            inputs.uniform(33, seed=13), corner, inputs.uniform(3000, seed=14)]
    mats, orcs, xs = [], [], []
    for i, p in enumerate(sets):
        a = 0.05
        o = oracle.Oracle(p, oracle.kernel("imq", a), 32, 1e-10)
        g = h2d.HODLR2D(p, h2d.kernel("imq", a), 32, 1e-10, compress=False)
        g.import_factors(*o.export_factors())
        g.prepare("f32")
        xs.append(rng.standard_normal(((1, 5)[i % 2], len(p))))
        mats.append(g)
        orcs.append(o)
    assert [o.kappa for o in orcs[:3]] == [0, 0, 1]
    want = [o.matvec(np.ascontiguousarray(x.T)) for o, x in zip(orcs, xs)]
    b = h2d.Batch(mats, stream=torch.cuda.current_stream(), form=form)
    xd = [torch.from_numpy(x).cuda() for x in xs]
    for mode in ("f64", "f32"):
        ys = [torch.empty_like(x) for x in xd]
        b.matvec(xd, ys, mode=mode)
        b.check()
        assert b.last_form == form
        for y, w in zip(ys, want):
            assert rel(y.cpu().numpy().T, w) <= BOUND[mode], mode
    b.close()
