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


@pytest.mark.parametrize("nrhs", [1, 3])
def test_noalloc_matches_matvec_twice(pkg, nrhs):
    lib = pkg._lib.load()
    n = 4096
    pts = inputs.uniform(n, seed=0)
    g = pkg.HODLR2D(pts, pkg.kernel("imq", 1.0 / 64), 64, 1e-10, root=(-1.0, -1.0, 2.0))
    x = torch.from_numpy(np.ascontiguousarray(inputs.rhs(n, nrhs, seed=1).T)).cuda()
    y_ref = torch.empty_like(x)
    rc = lib.hodlr2d_matvec(g.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y_ref.data_ptr()),
                            nrhs)
    assert rc == 0
    for _ in range(2):  # the shared array keeps the previous call's contents
        y = torch.full_like(x, float("nan"))
        rc = lib.hodlr2d_matvec_noalloc(g.handle, C.c_void_p(x.data_ptr()),
                                        C.c_void_p(y.data_ptr()), nrhs)
        assert rc == 0
        torch.cuda.synchronize()
        assert _rel(y, y_ref) <= 1e-12


def test_noalloc_rejects_oversized_and_host_buffers(pkg):
    lib = pkg._lib.load()
    n = 1 << 18
    pts = inputs.uniform(n, seed=0)
    g = pkg.HODLR2D(pts, pkg.kernel("mq", 1.0 / 512), 64, 1e-8, root=(-1.0, -1.0, 2.0))
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    rc = lib.hodlr2d_matvec_noalloc(g.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), 1)
    assert rc == -1  # needs more than HODLR2D_NOALLOC_SCRATCH_BYTES
    small = pkg.HODLR2D(inputs.uniform(500, seed=2), pkg.kernel("imq", 0.05), 32, 1e-8)
    xh = np.zeros(500)
    yh = np.zeros(500)
    rc = lib.hodlr2d_matvec_noalloc(small.handle, C.c_void_p(xh.ctypes.data),
                                    C.c_void_p(yh.ctypes.data), 1)
    assert rc == -1  # host pointers are not accepted
