"""GPU path against the CPU oracle, through the C ABI (needs a GB300).

P1  same factors: the GPU product on factors imported from the oracle equals
    the oracle's Alg. 2 product to relative 2-norm <= 1e-12.
P2  independent builds: identical tree, lists and pair set; ranks equal on
    >= 99.9% of pairs; each block within 10 eps of the dense block; the GPU
    product within 10 eps of the direct product.
Plus determinism, edge cases (tiny, ragged, empty boxes, kappa = 0, deep
trees), several right-hand sides, and argument errors.
"""
import numpy as np
import pytest

from paper_2204_05536_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def h2d():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2204_05536_gb300 as pkg
    pkg.load()
    return pkg


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def both(h2d, oracle, pts, kind, a, leaf, eps, diag=None, root=None, levels=-1, compress=True):
    g = h2d.HODLR2D(pts, h2d.kernel(kind, a, diag), leaf, eps, root=root, levels=levels,
                    compress=compress)
    o = oracle.Oracle(pts, oracle.kernel(kind, a, diag), leaf, eps, root=root, levels=levels)
    return g, o


CASES = [
    # (name, n, kind, a, leaf, eps)
    ("imq4096", 4096, "imq", 1 / 64, 64, 1e-10),
    ("mq3000", 3000, "mq", 0.02, 40, 1e-8),
    ("log2500", 2500, "log", 0.0, 32, 1e-10),
    ("invr1800", 1800, "inv_r", 0.0, 16, 1e-9),
    ("phi1_2000", 2000, "phi1", 0.001, 50, 1e-10),
    ("phi2_2000", 2000, "phi2", 0.001, 50, 1e-10),
]


@pytest.mark.parametrize("name,n,kind,a,leaf,eps", CASES)
def test_tree_lists_and_pairs_match_oracle(h2d, oracle, name, n, kind, a, leaf, eps):
    pts = inputs.uniform(n, seed=0)
    g, o = both(h2d, oracle, pts, kind, a, leaf, eps)
    st = g.stats()
    assert st["kappa"] == o.kappa
    assert np.allclose(st["root"], o.root, rtol=0, atol=0)
    # every leaf holds the same points, in ascending original index
    perm = g.perm()
    k = o.kappa
    pos = 0
    # tree order: leaves in Morton order; compare each leaf's point set
    m = 2 ** k
    for key in range(4 ** k):
        ix = int(sum(((key >> (2 * s)) & 1) << s for s in range(k)))
        iy = int(sum(((key >> (2 * s + 1)) & 1) << s for s in range(k)))
        want = o.box_points(k, oracle.paper_index(k, ix, iy))
        got = perm[pos: pos + len(want)]
        np.testing.assert_array_equal(got, want)
        pos += len(want)
    assert pos == n
    # same stored pairs (level, row box, column box)
    gp = g.pairs()
    op = np.array([[d["level"], *d["x"], *d["y"], d["rank"]] for d, _, _ in o.pairs()])
    gs = sorted(map(tuple, gp[:, :5].tolist()))
    os_ = sorted(map(tuple, op[:, :5].tolist()))
    assert gs == os_
    # ranks agree on >= 99.9% of pairs (near-ties in a pivot may flip)
    rk_g = {tuple(r[:5]): r[5] for r in gp.tolist()}
    same = sum(rk_g[tuple(r[:5])] == r[5] for r in op.tolist())
    assert same >= 0.999 * len(op)
    assert st["unconverged"] == 0


@pytest.mark.parametrize("name,n,kind,a,leaf,eps", CASES)
@pytest.mark.parametrize("nrhs", [1, 3])
def test_p1_same_factors_matches_oracle_matvec(h2d, oracle, name, n, kind, a, leaf, eps, nrhs):
    pts = inputs.uniform(n, seed=0)
    o = oracle.Oracle(pts, oracle.kernel(kind, a), leaf, eps)
    g = h2d.HODLR2D(pts, h2d.kernel(kind, a), leaf, eps, compress=False)
    g.import_factors(*o.export_factors())
    x = inputs.rhs(n, nrhs, seed=1)
    y_o = o.matvec(x)
    y_g = g.matvec(torch.from_numpy(np.ascontiguousarray(x)).cuda()).cpu().numpy()
    assert rel(y_g, y_o) <= 1e-12
    # host buffers through the same entry point
    y_h = g.matvec(np.ascontiguousarray(x))
    np.testing.assert_array_equal(y_h, y_g)


@pytest.mark.parametrize("name,n,kind,a,leaf,eps", CASES)
def test_p2_gpu_build_vs_direct(h2d, oracle, name, n, kind, a, leaf, eps):
    pts = inputs.uniform(n, seed=0)
    g = h2d.HODLR2D(pts, h2d.kernel(kind, a), leaf, eps)
    x = inputs.rhs(n, seed=2)
    yd = oracle.direct_matvec(pts, oracle.kernel(kind, a), x)
    y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, yd) <= 10 * eps


def test_block_errors_of_gpu_factors(h2d, oracle):
    n, eps = 3000, 1e-10
    pts = inputs.uniform(n, seed=4)
    k_o = oracle.kernel("imq", 0.02)
    g = h2d.HODLR2D(pts, h2d.kernel("imq", 0.02), 48, eps)
    o = oracle.Oracle(pts, k_o, 48, eps, compress=False)
    info, offs, vals = g.export_factors()
    worst = 0.0
    for p in range(0, len(info), max(1, len(info) // 200)):
        lv, ax, ay, bx, by, k = info[p]
        I = o.box_points(lv, oracle.paper_index(lv, ax, ay))
        J = o.box_points(lv, oracle.paper_index(lv, bx, by))
        U = vals[offs[p]: offs[p] + len(I) * k].reshape(k, len(I)).T
        V = vals[offs[p] + len(I) * k: offs[p + 1]].reshape(k, len(J)).T
        A = np.array([[oracle.entry(pts, k_o, i, j) for j in J] for i in I])
        worst = max(worst, rel(U @ V.T, A))
    assert worst <= 10 * eps


def test_deterministic(h2d):
    pts = inputs.uniform(5000, seed=3)
    g = h2d.HODLR2D(pts, h2d.kernel("mq", 0.01), 32, 1e-8)
    x = torch.from_numpy(inputs.rhs(5000, 2, seed=5)).cuda()
    a = g.matvec(x)
    b = g.matvec(x)
    assert torch.equal(a, b)
    g2 = h2d.HODLR2D(pts, h2d.kernel("mq", 0.01), 32, 1e-8)
    assert np.array_equal(g.export_factors()[2], g2.export_factors()[2])


def test_kappa0_and_tiny(h2d, oracle):
    for n in (1, 2, 7, 300):
        pts = inputs.uniform(n, seed=n)
        g = h2d.HODLR2D(pts, h2d.kernel("imq", 0.05), 1000, 1e-10)
        assert g.stats()["kappa"] == 0
        x = inputs.rhs(n, 2, seed=1)
        yd = oracle.direct_matvec(pts, oracle.kernel("imq", 0.05), x)
        y = g.matvec(np.ascontiguousarray(x))
        assert rel(y, yd) <= 1e-14


def test_ragged_empty_boxes_and_deep_tree(h2d, oracle):
    rng = np.random.default_rng(8)
    pts = np.concatenate([rng.normal(0.3, 0.01, (700, 2)), rng.normal(-0.5, 0.05, (500, 2)),
                          rng.uniform(-1, 1, (300, 2))])
    cases = [(pts, 6), (pts, 33), (inputs.uniform(1500, seed=12), 1)]
    for pts, leaf in cases:
        g, o = both(h2d, oracle, pts, "imq", 0.001, leaf, 1e-10)
        assert g.stats()["kappa"] == o.kappa
        x = inputs.rhs(len(pts), seed=3)
        g2 = h2d.HODLR2D(pts, h2d.kernel("imq", 0.001), leaf, 1e-10, compress=False)
        g2.import_factors(*o.export_factors())
        assert rel(g2.matvec(x), o.matvec(x)) <= 1e-12
        yd = oracle.direct_matvec(pts, oracle.kernel("imq", 0.001), x)
        assert rel(g.matvec(x), yd) <= 1e-9


def test_forced_levels_and_root(h2d, oracle):
    pts = inputs.uniform(2000, seed=6)
    for levels in (0, 1, 2, 5):
        g, o = both(h2d, oracle, pts, "log", 0.0, 10, 1e-10, root=(-1.0, -1.0, 2.0),
                    levels=levels)
        assert g.stats()["kappa"] == levels
        x = inputs.rhs(2000, seed=1)
        yd = oracle.direct_matvec(pts, oracle.kernel("log"), x)
        assert rel(g.matvec(x), yd) <= 1e-9


def test_errors(h2d):
    pts = inputs.uniform(100, seed=1)
    bad = pts.copy()
    bad[5, 0] = np.nan
    with pytest.raises(h2d.HodlrError) as e:
        h2d.HODLR2D(bad, h2d.kernel("imq", 0.1), 8, 1e-8)
    assert e.value.code == -1
    g = h2d.HODLR2D(pts, h2d.kernel("imq", 0.1), 8, 1e-8, compress=False)
    with pytest.raises(h2d.HodlrError) as e:
        g.matvec(np.zeros(100))
    assert e.value.code == -7  # no factors yet


def test_gmres_solves_rbf_system(h2d, oracle):
    """Eq. ker: beta lambda_i + sum_{j != i} phi(r_ij) lambda_j = f_i with
    beta = N (Sec. 5.2)."""
    n = 2500
    pts = inputs.uniform(n, seed=2)
    lam = inputs.rhs(n, seed=9)
    ko = oracle.kernel("phi2", 0.001, diag=float(n))
    f = oracle.direct_matvec(pts, ko, lam)
    g = h2d.HODLR2D(pts, h2d.kernel("phi2", 0.001, diag=float(n)), 50, 1e-12)
    x, it, rr, code = g.gmres(torch.from_numpy(f).cuda(), tol=1e-10)
    assert code == 0 and rr <= 1e-10
    assert rel(x.cpu().numpy(), lam) <= 1e-8
    # host buffers
    xh, it2, rr2, code2 = g.gmres(f, tol=1e-10)
    assert code2 == 0 and np.array_equal(xh, x.cpu().numpy())


def test_independent_builds_agree_at_2e16(h2d, oracle):
    """N = 2^16 of the headline recipe (uniform, MQ a = 1/sqrt(N), leaf 64,
    eps = 1e-8): GPU and oracle build independently; the same pivots give the
    same factors, so the two products agree far below eps (a rare pivot flip
    on a near-tie would show up as an eps-sized difference)."""
    n, eps = 1 << 16, 1e-8
    pts = inputs.uniform(n, seed=0)
    a = 1.0 / np.sqrt(n)
    g = h2d.HODLR2D(pts, h2d.kernel("mq", a), 64, eps, root=(-1.0, -1.0, 2.0))
    o = oracle.Oracle(pts, oracle.kernel("mq", a), 64, eps, root=(-1.0, -1.0, 2.0))
    gp = {tuple(r[:5]): r[5] for r in g.pairs().tolist()}
    op = {(d["level"], *d["x"], *d["y"]): d["rank"] for d, _, _ in o.pairs()}
    assert gp.keys() == op.keys()
    assert sum(gp[k] == op[k] for k in op) >= 0.999 * len(op)
    x = inputs.rhs(n, seed=1)
    y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel(y, o.matvec(x)) <= 1e-10


def test_full_size_sampled_rows(h2d, oracle):
    """N = 2^20 uniform points, MQ a = 2^-10, leaf 64, eps = 1e-8, one
    right-hand side, 256 seeded rows against the direct product.

    ACA's stopping rule |u||v| <= eps |S_k|_F bounds each block's error
    relative to the block, not relative to |A x|: for MQ the blocks carry a
    large constant component that a zero-mean x cancels, so the product's
    relative error exceeds eps on the coarse levels.  The oracle itself gives
    2.5e-7 (25 eps) at N = 2^18 on these rows.  Bounds: relative 2-norm
    <= 50 eps, and per row |dy_i| <= eps * sum_j |A_ij| |x_j|."""
    n, eps = 1 << 20, 1e-8
    pts = inputs.uniform(n, seed=0)
    a = 2.0 ** -10
    g = h2d.HODLR2D(pts, h2d.kernel("mq", a), 64, eps, root=(-1.0, -1.0, 2.0))
    st = g.stats()
    assert st["kappa"] == 8 and st["unconverged"] == 0
    x = inputs.rhs(n, seed=1)
    y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    rows = np.random.default_rng(7).choice(n, 256, replace=False)
    ko = oracle.kernel("mq", a)
    yd = oracle.direct_rows(pts, ko, x, rows)
    assert rel(y[rows], yd) <= 50 * eps
    scale = oracle.direct_rows(pts, ko, np.abs(x), rows)  # MQ > 0: sum |A_ij||x_j|
    assert np.max(np.abs(y[rows] - yd) / scale) <= eps


@pytest.mark.parametrize("name,n,kind,a,leaf,eps", CASES)
@pytest.mark.parametrize("nrhs", [1, 2])
def test_p1_df32_same_factors(h2d, oracle, name, n, kind, a, leaf, eps, nrhs):
    """The float-float product on the oracle's factors equals the oracle's
    Alg. 2 product to <= 1e-12 (binary64-level accuracy).  One right-hand
    side runs the register pair kernel, two the two-read pair kernel."""
    pts = inputs.uniform(n, seed=0)
    o = oracle.Oracle(pts, oracle.kernel(kind, a), leaf, eps)
    g = h2d.HODLR2D(pts, h2d.kernel(kind, a), leaf, eps, compress=False)
    g.import_factors(*o.export_factors())
    g.prepare("df32")
    x = inputs.rhs(n, nrhs, seed=1)
    y_o = o.matvec(x)
    y_g = g.matvec(torch.from_numpy(np.ascontiguousarray(x)).cuda(), mode="df32").cpu().numpy()
    assert rel(y_g, y_o) <= 1e-12


def test_df32_f64_agree_and_deterministic(h2d):
    n = 20000
    pts = inputs.uniform(n, seed=5)
    g = h2d.HODLR2D(pts, h2d.kernel("imq", 1.0 / np.sqrt(n)), 32, 1e-10)
    g.prepare("df32")
    x = torch.from_numpy(inputs.rhs(n, 3, seed=2)).cuda()
    a = g.matvec(x, mode="df32")
    b = g.matvec(x, mode="df32")
    assert torch.equal(a, b)
    c = g.matvec(x, mode="f64")
    assert rel(a.cpu().numpy(), c.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("n", [6000, 20000, 65536])
def test_register_pair_kernel_block_sizes(h2d, oracle, n):
    """One right-hand side in the float-float, binary32 and bfloat16 modes
    runs the register pair kernel; these sizes give pair-mode levels whose
    largest boxes select its 512-, 256-, 128- and 32-thread forms.  Checked
    against the oracle's product on the same factors (P1) and against the
    same mode with two equal right-hand sides, which takes the two-read
    pair kernel."""
    pts = inputs.uniform(n, seed=3)
    kind, a, leaf, eps = "imq", 1.0 / np.sqrt(n), 64, 1e-10
    o = oracle.Oracle(pts, oracle.kernel(kind, a), leaf, eps)
    g = h2d.HODLR2D(pts, h2d.kernel(kind, a), leaf, eps, compress=False)
    g.import_factors(*o.export_factors())
    x = inputs.rhs(n, seed=4)
    y_o = o.matvec(x)
    xd = torch.from_numpy(x).cuda()
    x2 = torch.stack([xd, xd], dim=1)
    # bound2: the two forms sum in different orders; float-float rounds each
    # operation to about 2^-44, binary32 to 2^-24; the bound of bfloat16
    # also covers its tensor-core form (more than four right-hand sides),
    # which rounds x and t to two bfloat16 terms (about 2^-17)
    for mode, bound, bound2 in (("df32", 1e-12, 1e-12), ("f32", 5e-6, 1e-6), ("bf16", 2e-2, 1e-4)):
        g.prepare(mode)
        y1 = g.matvec(xd, mode=mode)
        y2 = g.matvec(x2, mode=mode)
        assert rel(y1.cpu().numpy(), y_o) <= bound, mode
        assert torch.equal(y2[:, 0], y2[:, 1])
        assert rel(y1.cpu().numpy(), y2[:, 0].cpu().numpy()) <= bound2, mode
        assert torch.equal(y1, g.matvec(xd, mode=mode))  # deterministic


def test_many_rhs_equal_columnwise(h2d):
    """11 right-hand sides (not a multiple of the kernels' 8 or 4 per pass):
    coarse boxes in two passes, boxes of <= 256 points with the multi-RHS
    register kernel; each column agrees with the one-RHS product."""
    n = 30000
    pts = inputs.uniform(n, seed=8)
    g = h2d.HODLR2D(pts, h2d.kernel("imq", 1.0 / np.sqrt(n)), 64, 1e-10)
    X = torch.from_numpy(inputs.rhs(n, 11, seed=9)).cuda()
    # bfloat16: tensor-core products with x and t in two bfloat16 terms (2^-17)
    for mode, bound in (("f64", 1e-15), ("df32", 1e-12), ("f32", 1e-6), ("bf16", 1e-4)):
        if mode != "f64":
            g.prepare(mode)
        Y = g.matvec(X, mode=mode)
        assert torch.equal(Y, g.matvec(X, mode=mode))
        for c in (0, 7, 8, 10):
            y1 = g.matvec(X[:, c].contiguous(), mode=mode)
            assert rel(Y[:, c].cpu().numpy(), y1.cpu().numpy()) <= bound, (mode, c)


@pytest.mark.parametrize("kind,a", [("mq", 0.01), ("log", 0.0), ("phi1", 0.001)])
def test_large_leaves_near_field(h2d, oracle, kind, a):
    """Leaves of several hundred points (depth forced to 2), so the near field
    carries most of the product: the float-float and binary32 near fields
    (32-target work items; float-float logarithm for log r and phi_1)
    against the oracle on the same factors."""
    n = 5000
    pts = inputs.chebyshev_grid(71)[:n]
    leaf, eps = 64, 1e-10
    o = oracle.Oracle(pts, oracle.kernel(kind, a), leaf, eps, levels=2)
    g = h2d.HODLR2D(pts, h2d.kernel(kind, a), leaf, eps, levels=2, compress=False)
    g.import_factors(*o.export_factors())
    assert g.stats()["kappa"] == 2
    x = inputs.rhs(n, seed=6)
    y_o = o.matvec(x)
    xd = torch.from_numpy(x).cuda()
    for mode, bound in (("df32", 1e-12), ("f32", 5e-6)):
        g.prepare(mode)
        assert rel(g.matvec(xd, mode=mode).cpu().numpy(), y_o) <= bound, mode


def test_df32_full_size_sampled_rows(h2d, oracle):
    n, eps = 1 << 20, 1e-8
    pts = inputs.uniform(n, seed=0)
    a = 2.0 ** -10
    g = h2d.HODLR2D(pts, h2d.kernel("mq", a), 64, eps, root=(-1.0, -1.0, 2.0))
    g.prepare("df32")
    x = torch.from_numpy(inputs.rhs(n, seed=1)).cuda()
    y64 = g.matvec(x, mode="f64").cpu().numpy()
    y = g.matvec(x, mode="df32").cpu().numpy()
    assert rel(y, y64) <= 1e-12
    rows = np.random.default_rng(7).choice(n, 256, replace=False)
    yd = oracle.direct_rows(pts, oracle.kernel("mq", a), x.cpu().numpy(), rows)
    assert rel(y[rows], yd) <= 50 * eps


def test_gmres_df32(h2d, oracle):
    """GMRES with float-float products (binary64-level accuracy, no
    refinement loop); restarting from the solution costs one product."""
    n = 3000
    pts = inputs.uniform(n, seed=2)
    lam = inputs.rhs(n, seed=9)
    ko = oracle.kernel("phi2", 0.001, diag=float(n))
    f = oracle.direct_matvec(pts, ko, lam)
    g = h2d.HODLR2D(pts, h2d.kernel("phi2", 0.001, diag=float(n)), 50, 1e-12)
    g.prepare("df32")
    x, it, rr, code = g.gmres(torch.from_numpy(f).cuda(), tol=1e-10, inner_mode="df32")
    assert code == 0 and rr <= 1e-10
    assert rel(x.cpu().numpy(), lam) <= 1e-8
    x2, it2, rr2, code2 = g.gmres(torch.from_numpy(f).cuda(), x0=x, tol=1e-10, inner_mode="df32")
    assert code2 == 0 and it2 == 1 and torch.equal(x2, x)


@pytest.mark.parametrize("mode,bound", [("f32", 5e-6), ("bf16", 2e-2)])
def test_mixed_modes_error(h2d, oracle, mode, bound):
    """Binary32 and bfloat16 factor storage with binary32 sums: error against
    the F64 product (same factors) and against the direct product."""
    n = 20000
    pts = inputs.uniform(n, seed=5)
    a = 1.0 / np.sqrt(n)
    g = h2d.HODLR2D(pts, h2d.kernel("mq", a), 32, 1e-8, root=(-1.0, -1.0, 2.0))
    g.prepare(mode)
    x = torch.from_numpy(inputs.rhs(n, 2, seed=3)).cuda()
    y64 = g.matvec(x, mode="f64").cpu().numpy()
    y = g.matvec(x, mode=mode).cpu().numpy()
    assert rel(y, y64) <= bound
    assert torch.equal(g.matvec(x, mode=mode), g.matvec(x, mode=mode))


@pytest.mark.parametrize("mode", ["f32", "bf16"])
def test_gmres_mixed_refinement(h2d, oracle, mode):
    """Iterative refinement reaches the F64 tolerance with low-precision inner
    products (Eq. ker system, beta = N)."""
    n = 3000
    pts = inputs.uniform(n, seed=2)
    lam = inputs.rhs(n, seed=9)
    ko = oracle.kernel("phi2", 0.001, diag=float(n))
    f = oracle.direct_matvec(pts, ko, lam)
    g = h2d.HODLR2D(pts, h2d.kernel("phi2", 0.001, diag=float(n)), 50, 1e-12)
    g.prepare(mode)
    x, it, rr, code = g.gmres(torch.from_numpy(f).cuda(), tol=1e-10, inner_mode=mode)
    assert code == 0 and rr <= 1e-10
    assert rel(x.cpu().numpy(), lam) <= 1e-8


@pytest.mark.parametrize("mode", ["f64", "df32"])
def test_box_pairs_larger_than_a_slice(h2d, oracle, mode):
    """Box-mode levels (boxes of <= 64 points in binary64, <= 48 in
    float-float) whose pairs hold more values than one shared-memory slice of
    the box kernel (960) are read from global memory instead of staged; with
    eps = 1e-12 the finest pairs have ranks that force that path.  Checked
    against the oracle's product on the same factors (P1)."""
    if mode == "f64":  # exactly 64 points per leaf
        pts, _ = inputs.jittered_grid(64, seed=0)
        kind, a, leaf = "log", 0.0, 64
    else:
        pts = inputs.uniform(4096, seed=7)
        kind, a, leaf = "imq", 1.0 / 64, 48
    eps = 1e-12
    o = oracle.Oracle(pts, oracle.kernel(kind, a), leaf, eps)
    kappa = o.kappa
    big = [d for d, U, V in o.pairs()
           if d["level"] == kappa
           and (U.shape[0] + U.shape[0] % 2 + V.shape[0] + V.shape[0] % 2) * d["rank"] > 960]
    assert big, "no finest-level pair exceeds a slice: the case does not test the path"
    g = h2d.HODLR2D(pts, h2d.kernel(kind, a), leaf, eps, compress=False)
    g.import_factors(*o.export_factors())
    if mode == "df32":
        g.prepare("df32")
    for nrhs in (1, 2):
        x = inputs.rhs(len(pts), nrhs, seed=2)
        y_o = o.matvec(x)
        y_g = g.matvec(torch.from_numpy(np.ascontiguousarray(x)).cuda(), mode=mode).cpu().numpy()
        assert rel(y_g, y_o) <= 1e-12


def test_rank_one_blocks_exact(h2d, oracle):
    """Four clusters of coincident points, one per quadrant: every stored
    pair (the two diagonal pairs of level 1) couples two clusters, a block
    with identical columns, so the GPU ACA returns rank 1 exactly (the
    residual after one term is exactly zero) and the product equals the
    direct one to rounding."""
    centres = np.array([[-0.5, -0.5], [0.5, -0.5], [0.5, 0.5], [-0.5, 0.5]])
    pts = np.repeat(centres, 50, axis=0)
    n = len(pts)
    g = h2d.HODLR2D(pts, h2d.kernel("mq", 0.01), 64, 1e-12, root=(-1.0, -1.0, 2.0))
    st = g.stats()
    assert st["kappa"] == 1
    gp = g.pairs()
    assert len(gp) == 2
    assert np.all(gp[:, 5] == 1)
    x = inputs.rhs(n, seed=3)
    y = g.matvec(torch.from_numpy(x).cuda()).cpu().numpy()
    yd = oracle.direct_matvec(pts, oracle.kernel("mq", 0.01), x)
    assert rel(y, yd) <= 1e-13


def test_gmres_tiny_system_breakdown(h2d, oracle):
    """A 7-point system (kappa = 0: one dense block): the Krylov space is
    exhausted after at most 7 steps, so the Arnoldi process breaks down
    (|v_{j+1}| = 0 up to rounding) inside the first cycle; the solution must
    still equal the dense solve of the oracle's matrix."""
    n = 7
    pts = inputs.uniform(n, seed=21)
    k = oracle.kernel("imq", 0.3)
    A = oracle.dense_matrix(pts, k)
    b = inputs.rhs(n, seed=22)
    want = np.linalg.solve(A, b)
    g = h2d.HODLR2D(pts, h2d.kernel("imq", 0.3), 64, 1e-12)
    for mode in ("f64", "df32"):
        if mode != "f64":
            g.prepare(mode)
        x, it, rr, code = g.gmres(b, tol=1e-13, restart=50, inner_mode=mode)
        assert code == 0 and rr <= 1e-13, (mode, it, rr)
        assert rel(x, want) <= 1e-10, mode


def test_release_f64_keeps_df32(h2d):
    """A float-float-only handle: after hodlr2d_release(F64) the float-float
    product is unchanged bit for bit, and every call that needs the binary64
    factors reports HODLR2D_ERR_STATE."""
    n = 6000
    pts = inputs.uniform(n, seed=13)
    g = h2d.HODLR2D(pts, h2d.kernel("imq", 1.0 / np.sqrt(n)), 32, 1e-10)
    g.prepare("df32")
    x = torch.from_numpy(inputs.rhs(n, seed=14)).cuda()
    want = g.matvec(x, mode="df32")
    g.release("f64")
    assert torch.equal(g.matvec(x, mode="df32"), want)
    for call in (lambda: g.matvec(x, mode="f64"), lambda: g.prepare("f32"),
                 lambda: g.export_factors(), lambda: g.prepare("f64")):
        with pytest.raises(h2d.HodlrError) as e:
            call()
        assert e.value.code == -7
    g.release("df32")
    with pytest.raises(h2d.HodlrError):
        g.matvec(x, mode="df32")
