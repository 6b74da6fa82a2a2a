"""The memory-bound calibration kernels (BabelStream ops and the seven-point
stencil) against their numpy oracle: exact for element-wise ops, FP64 dot
to rounding, stencil exact on a quadratic and to FP rounding elsewhere."""
import numpy as np
import pytest
import torch

from oracle import stream_oracle as so
from paper_2509_21039_gb300 import bude

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2509_21039_gb300 import build
    build.build()
    bude.load()


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n", [1, 3, 1000, 4097, 1 << 20, (1 << 22) + 5])
def test_stream_ops_match_oracle(dtype, n):
    g = torch.Generator().manual_seed(n)
    a0 = torch.rand(n, generator=g, dtype=dtype)
    b0 = torch.rand(n, generator=g, dtype=dtype)
    c0 = torch.rand(n, generator=g, dtype=dtype)
    s = 0.4
    A, B, C = a0.numpy(), b0.numpy(), c0.numpy()
    a, b, c = a0.to(DEV), b0.to(DEV), c0.to(DEV)
    bude.stream_op("copy", a=a, c=c)
    assert np.array_equal(c.cpu().numpy(), so.copy(A))
    bude.stream_op("mul", b=b, c=c, scalar=s)
    assert np.array_equal(b.cpu().numpy(), so.mul(A, s))
    bude.stream_op("add", a=a, b=b, c=c)
    ref_c = so.add(A, so.mul(A, s))
    assert np.array_equal(c.cpu().numpy(), ref_c)
    bude.stream_op("triad", a=a, b=b, c=c, scalar=s)
    ref_a = so.triad(so.mul(A, s), ref_c, s)
    np.testing.assert_allclose(a.cpu().numpy(), ref_a, rtol=2e-7 if dtype == torch.float32 else 1e-15)
    d = bude.stream_op("dot", a=a, b=b).item()
    # FP32: products rounded to FP32, compensated FP32 sums per thread, FP64 after
    tol = 1e-6 if dtype == torch.float32 else 1e-12
    assert d == pytest.approx(so.dot(a.cpu().numpy(), b.cpu().numpy()), rel=tol)


def test_dot_is_exact_on_small_integers():
    n = (1 << 20) + 3
    a = (torch.arange(n) % 7).to(torch.float32).to(DEV)
    b = torch.full((n,), 2.0, device=DEV)
    assert bude.stream_op("dot", a=a, b=b).item() == 2.0 * float((np.arange(n) % 7).sum())


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_laplacian_of_quadratic_is_exact(dtype):
    nx, ny, nz = 7, 19, 45          # ragged tiles in j and k
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    u = torch.from_numpy((i ** 2 + 2 * j ** 2 + 3 * k ** 2).astype(np.float64)).to(dtype).to(DEV)
    f = torch.full_like(u, -1.0)
    bude.laplacian(u, f, 1.0, 1.0, 1.0, -6.0)
    F = f.cpu().numpy()
    assert np.all(F[1:-1, 1:-1, 1:-1] == 12.0)
    # boundary untouched
    assert np.all(F[0] == -1) and np.all(F[-1] == -1) and np.all(F[:, 0] == -1)
    assert np.all(F[:, :, -1] == -1)


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("shape", [(3, 3, 3), (5, 40, 33), (33, 9, 130), (64, 64, 64)])
def test_laplacian_matches_oracle(dtype, shape):
    g = torch.Generator().manual_seed(sum(shape))
    u0 = torch.rand(shape, generator=g, dtype=dtype)
    f0 = torch.zeros(shape, dtype=dtype)
    coef = (0.7, 1.3, 2.1, -8.2)
    ref = so.laplacian(u0.numpy(), *coef, f=f0.numpy())
    f = f0.to(DEV)
    bude.laplacian(u0.to(DEV), f, *coef)
    tol = 1e-6 if dtype == torch.float32 else 1e-14
    np.testing.assert_allclose(f.cpu().numpy(), ref, rtol=tol, atol=tol)


def test_calibration_edge_cases():
    x = torch.zeros(8, device=DEV)
    assert bude.stream_op("dot", a=x[:0], b=x[:0]).item() == 0.0
    with pytest.raises(bude.BudeError):
        bude.stream_op("copy", a=x[1:5], c=x[:4])        # misaligned start
    u = torch.zeros((2, 5, 5), device=DEV)
    bude.laplacian(u, torch.zeros_like(u))              # no interior: no-op
