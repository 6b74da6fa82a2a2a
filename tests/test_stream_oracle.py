"""Pins for the memory-bound-kernel oracle: closed forms and exact cases."""
import numpy as np
import pytest

from oracle import stream_oracle as so


def test_laplacian_of_a_quadratic_is_exact():
    # with unit spacing (invh = 1, invhxyz2 = -6) the discrete Laplacian of
    # x^2 + 2 y^2 + 3 z^2 is 2 + 4 + 6 = 12 at every interior point
    L = 9
    i, j, k = np.meshgrid(np.arange(L), np.arange(L), np.arange(L), indexing="ij")
    u = (i ** 2 + 2 * j ** 2 + 3 * k ** 2).astype(np.float64)
    f = so.laplacian(u, 1.0, 1.0, 1.0, -6.0)
    assert np.all(f[1:-1, 1:-1, 1:-1] == 12.0)
    assert np.all(f[0] == 0) and np.all(f[:, -1] == 0) and np.all(f[:, :, 0] == 0)


def test_laplacian_axis_roles():
    # a function of the slowest index only feels invhx2
    L = 6
    u = np.zeros((L, L, L))
    u[:] = (np.arange(L) ** 2)[:, None, None]
    f = so.laplacian(u, 1.0, 0.0, 0.0, -2.0)
    assert np.all(f[1:-1, 1:-1, 1:-1] == 2.0)
    f = so.laplacian(u, 0.0, 5.0, 7.0, 0.0)
    expect = 10.0 * u[1:-1, 1:-1, 1:-1] + 14.0 * u[1:-1, 1:-1, 1:-1]
    np.testing.assert_array_equal(f[1:-1, 1:-1, 1:-1], expect)


def test_stream_ops_small_integers_are_exact():
    a = (np.arange(1000) % 7).astype(np.float32)
    b = np.full(1000, 2.0, np.float32)
    c = np.arange(1000, dtype=np.float32)
    assert np.array_equal(so.copy(a), a)
    assert np.array_equal(so.mul(c, 3.0), 3 * c)
    assert np.array_equal(so.add(a, b), a + 2)
    assert np.array_equal(so.triad(b, c, 0.5), 2 + 0.5 * c)
    assert so.dot(a, b) == 2.0 * sum(i % 7 for i in range(1000))


def test_bandwidth_formulas():
    # Eq. 1: all points but the 8 corners and the 12 edges are read once,
    # the (L-2)^3 interior written once; Eq. 2: arrays touched per op
    assert so.stencil_bytes(4, 8) == (64 - 8 - 24 + 8) * 8
    L = 5
    touched = np.zeros((L, L, L), bool)
    for i in range(1, L - 1):
        for j in range(1, L - 1):
            for k in range(1, L - 1):
                for di, dj, dk in ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                                   (0, 0, 1), (0, 0, -1)):
                    touched[i + di, j + dj, k + dk] = True
    assert so.stencil_bytes(L, 1) == touched.sum() + (L - 2) ** 3
    assert so.stream_bytes("triad", 10, 4) == 120 and so.stream_bytes("copy", 10, 8) == 160
