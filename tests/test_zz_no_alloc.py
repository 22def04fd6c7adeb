"""hodlr2d_matvec_noalloc: the F64 product whose working memory is a static
device array, for callers that must not allocate device memory while they run.

Checked through the C ABI: two calls in a row against hodlr2d_matvec (the
entry point that allocates its own scratch), a size beyond the array's limit
rejected with HODLR2D_ERR_ARG, and host pointers rejected.  Collected last
(file name) so that a failure here leaves every other test already run; it
also passes alone in a fresh process, where its first call does the one-time
per-device set-up.
"""
import ctypes as C

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


def _rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _noalloc(lib, g, x, y, nrhs):
    return lib.hodlr2d_matvec_noalloc(g.handle, C.c_void_p(x.data_ptr()),
                                      C.c_void_p(y.data_ptr()), nrhs)


@pytest.mark.parametrize("nrhs", [1, 3])
def test_noalloc_matches_matvec_twice(pkg, nrhs):
    """Two calls on the same handle against hodlr2d_matvec, with a call on
    another handle (more points, another x scaled by 1e6) in between, so the
    second call starts from scratch words that hold another problem's
    values: a scratch word the product reads without writing it first would
    show up as a mismatch."""
    lib = pkg._lib.load()
    n = 4096
    pts = inputs.uniform(n, seed=0)
    g = pkg.HODLR2D(pts, pkg.kernel("imq", 1.0 / 64), 64, 1e-10, root=(-1.0, -1.0, 2.0))
    x = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n, nrhs, seed=1).T)).cuda()
    y_ref = torch.empty_like(x)
    rc = lib.hodlr2d_matvec(g.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y_ref.data_ptr()),
                            nrhs)
    assert rc == 0
    n2 = 9000
    g2 = pkg.HODLR2D(inputs.uniform(n2, seed=4), pkg.kernel("mq", 0.01), 32, 1e-8)
    x2 = torch.from_numpy(np.ascontiguousarray(1e6 * inputs.rhs(n2, nrhs, seed=6).T)).cuda()
    y2_ref = torch.empty_like(x2)
    assert lib.hodlr2d_matvec(g2.handle, C.c_void_p(x2.data_ptr()),
                              C.c_void_p(y2_ref.data_ptr()), nrhs) == 0
    for step in range(2):  # the shared array keeps the previous call's contents
        y = torch.full_like(x, float("nan"))
        assert _noalloc(lib, g, x, y, nrhs) == 0
        torch.cuda.synchronize()
        assert _rel(y, y_ref) <= 1e-12, step
        if step == 0:  # fill the array with another problem's values
            y2 = torch.full_like(x2, float("nan"))
            assert _noalloc(lib, g2, x2, y2, nrhs) == 0
            torch.cuda.synchronize()
            assert _rel(y2, y2_ref) <= 1e-12


def test_noalloc_rejects_oversized_and_host_buffers(pkg):
    """n = 2^18 with four right-hand sides: the tree-order copy of x and the
    per-level slabs alone take 8 n nrhs (kappa + 2) = 75 MB, whatever the
    ranks, beyond the 32 MiB array; the call returns HODLR2D_ERR_ARG and
    leaves y as it was.  Host pointers are rejected too."""
    lib = pkg._lib.load()
    n, nrhs = 1 << 18, 4
    pts = inputs.uniform(n, seed=0)
    g = pkg.HODLR2D(pts, pkg.kernel("mq", 1.0 / 512), 64, 1e-8, root=(-1.0, -1.0, 2.0))
    assert 8 * n * nrhs * (g.stats()["kappa"] + 2) > (32 << 20)
    x = torch.ones(nrhs, n, dtype=torch.float64, device="cuda")
    y = torch.full_like(x, 123.0)
    assert _noalloc(lib, g, x, y, nrhs) == -1  # needs more than HODLR2D_NOALLOC_SCRATCH_BYTES
    torch.cuda.synchronize()
    assert bool(torch.all(y == 123.0))
    small = pkg.HODLR2D(inputs.uniform(500, seed=2), pkg.kernel("imq", 0.05), 32, 1e-8)
    xh = np.zeros(500)
    yh = np.zeros(500)
    rc = lib.hodlr2d_matvec_noalloc(small.handle, C.c_void_p(xh.ctypes.data),
                                    C.c_void_p(yh.ctypes.data), 1)
    assert rc == -1  # host pointers are not accepted
