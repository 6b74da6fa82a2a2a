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


def test_stream_ops_beyond_the_cta_cap():
    # 2^29 floats: 2^17 one-chunk CTAs for the element-wise ops, and a dot
    # whose grid-stride loop runs many rounds; exact results by construction
    n = (1 << 29) + 12345
    a = (torch.arange(n, device=DEV, dtype=torch.int64) % 7).to(torch.float32)
    b = torch.full((n,), 2.0, device=DEV)
    expect = 2.0 * ((n // 7) * 21 + sum(range(n % 7)))
    assert bude.stream_op("dot", a=a, b=b).item() == expect
    c = torch.empty_like(a)
    bude.stream_op("copy", a=a, c=c)
    assert torch.equal(c, a)
    bude.stream_op("triad", a=c, b=b, c=a, scalar=3.0)   # c = b + 3 a
    assert torch.equal(c, b + 3.0 * a)


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


def _stencil_atol(dtype, coef):
    """Rounding bound of the stencil on u in [0, 1): four operations (three
    sums and the fused multiply-adds), each off by at most one unit of
    roundoff of a partial sum no larger than S = |c0| + 2 (|cx| + |cy| + |cz|);
    twice that for margin.  The result itself may cancel to far below S, so a
    relative tolerance on it does not apply."""
    eps = np.finfo(np.float32 if dtype == torch.float32 else np.float64).eps
    cx, cy, cz, c0 = coef
    return 8 * eps * (abs(c0) + 2 * (abs(cx) + abs(cy) + abs(cz)))


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
    np.testing.assert_allclose(f.cpu().numpy(), ref, rtol=0, atol=_stencil_atol(dtype, coef))


def test_calibration_edge_cases():
    x = torch.zeros(8, device=DEV)
    assert bude.stream_op("dot", a=x[:0], b=x[:0]).item() == 0.0
    with pytest.raises(bude.BudeError):
        bude.stream_op("copy", a=x[1:5], c=x[:4])        # misaligned start
    u = torch.zeros((2, 5, 5), device=DEV)
    bude.laplacian(u, torch.zeros_like(u))              # no interior: no-op
    # the dot's output: one float64 on the arrays' device, else refused
    for bad in (torch.empty((), device=DEV), torch.empty(2, dtype=torch.float64, device=DEV),
                torch.empty((), dtype=torch.float64)):
        with pytest.raises(ValueError, match="dot_out"):
            bude.stream_op("dot", a=x, b=x, dot_out=bad)
    d = torch.full((1,), 7.0, dtype=torch.float64, device=DEV)
    assert bude.stream_op("dot", a=x + 1, b=x + 2, dot_out=d) is d and d.item() == 16.0


def _misaligned_copy(u):
    """The same values in a buffer whose base is 4 bytes past a 16-byte
    boundary, so that bude_laplacian takes the register kernel."""
    base = torch.empty(u.numel() + 1, dtype=u.dtype, device=u.device)
    v = base[1:].view(u.shape)
    v.copy_(u)
    return v


@pytest.mark.parametrize("shape", [(3, 3, 4), (3, 17, 8), (7, 19, 44), (131, 33, 260),
                                   (40, 300, 132), (20, 1000, 8), (300, 20, 36)])
def test_tma_stencil_matches_oracle_and_register_kernel(shape):
    g = torch.Generator().manual_seed(7 + sum(shape))
    u0 = torch.rand(shape, generator=g, dtype=torch.float32)
    coef = (0.7, 1.3, 2.1, -8.2)
    ref = so.laplacian(u0.numpy(), *coef, f=np.full(shape, -3.0, np.float32))
    u = u0.to(DEV)
    assert bude.laplacian_path(u) == "tma"
    f = torch.full(shape, -3.0, device=DEV)
    bude.laplacian(u, f, *coef)
    um = _misaligned_copy(u)
    assert bude.laplacian_path(um) == "register"
    fr = torch.full(shape, -3.0, device=DEV)
    bude.laplacian(um, fr, *coef)
    assert bude.wait_timeouts() == 0
    # the same expression in the same order: identical bits, boundary untouched
    assert torch.equal(f, fr)
    np.testing.assert_allclose(f.cpu().numpy(), ref, rtol=0, atol=_stencil_atol(torch.float32, coef))


def test_tma_stencil_quadratic_is_exact():
    nx, ny, nz = 9, 21, 148
    i, j, k = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    u = torch.from_numpy((i ** 2 + 2 * j ** 2 + 3 * k ** 2).astype(np.float32)).to(DEV)
    assert bude.laplacian_path(u) == "tma"
    f = torch.full_like(u, -1.0)
    bude.laplacian(u, f, 1.0, 1.0, 1.0, -6.0)
    F = f.cpu().numpy()
    assert np.all(F[1:-1, 1:-1, 1:-1] == 12.0)
    inner = np.zeros(F.shape, bool)
    inner[1:-1, 1:-1, 1:-1] = True
    assert np.all(F[~inner] == -1.0)


def test_tma_stencil_full_size_sampled():
    # the bench grid, 1024^3 float32 (4 GiB per array): equal to the register
    # kernel everywhere, and to the oracle on sampled 4^3 blocks
    L = 1024
    g = torch.Generator(device=DEV).manual_seed(11)
    u = torch.rand((L, L, L), generator=g, device=DEV)
    f = torch.zeros_like(u)
    bude.laplacian(u, f)
    assert bude.laplacian_path(u) == "tma"
    rng = np.random.default_rng(3)
    for _ in range(24):
        i0, j0, k0 = (int(x) for x in rng.integers(1, L - 5, 3))
        blk = u[i0 - 1:i0 + 5, j0 - 1:j0 + 5, k0 - 1:k0 + 5].cpu().numpy()
        ref = so.laplacian(blk, 1.0, 1.0, 1.0, -6.0, f=np.zeros_like(blk))[1:-1, 1:-1, 1:-1]
        got = f[i0:i0 + 4, j0:j0 + 4, k0:k0 + 4].cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=0, atol=_stencil_atol(torch.float32, (1, 1, 1, -6)))
    um = _misaligned_copy(u)
    del u
    fr = torch.zeros_like(f)
    bude.laplacian(um, fr)
    assert torch.equal(f, fr)
    assert bude.wait_timeouts() == 0


def test_tma_stencil_bounded_wait_gives_up_and_recovers():
    # a CTA whose staged plane never arrives (its copy is skipped) gives up
    # after its wait limit, leaves its tile unwritten, and the context and the
    # next call are unaffected
    shape = (40, 40, 256)
    g = torch.Generator().manual_seed(5)
    u0 = torch.rand(shape, generator=g, dtype=torch.float32)
    ref = so.laplacian(u0.numpy(), 1.0, 1.0, 1.0, -6.0, f=np.full(shape, -5.0, np.float32))
    u = u0.to(DEV)
    assert bude.wait_timeouts() == 0
    f = torch.full(shape, -5.0, device=DEV)
    bude.debug_stall_next_stencil()
    bude.laplacian(u, f)
    assert bude.wait_timeouts() == 1
    F = f.cpu().numpy()
    tol = _stencil_atol(torch.float32, (1, 1, 1, -6))
    bad = ~np.isclose(F, ref, rtol=0, atol=tol)
    assert bad.any()
    assert np.all(F[bad] == -5.0)                       # unwritten, not wrong
    ii, jj, kk = np.nonzero(bad)
    assert jj.max() < 16 and kk.max() < 128 and ii.min() == 1   # inside the first CTA's tile
    assert bad[1, 1:16, 1:128].all()
    f2 = torch.full(shape, -5.0, device=DEV)
    bude.laplacian(u, f2)
    assert bude.wait_timeouts() == 0
    np.testing.assert_allclose(f2.cpu().numpy(), ref, rtol=0, atol=tol)
