"""Plain numpy oracle for the paper's memory-bound kernels (arxiv 2509.21039,
Sec. 2.2, Listings 2 and 3; bandwidth metrics Eq. 1 and Eq. 2) -- TEST
INFRASTRUCTURE ONLY, used by the test suite and nothing in the product.

BabelStream (Listing 3):  copy  c = a;  mul  b = s c;  add  c = a + b;
triad  a = b + s c;  dot  sum_i a_i b_i (accumulated in float64 here).
Seven-point stencil (Listing 2), on the interior points of an L x L x L grid:
  f[i,j,k] = u[i,j,k] invhxyz2 + (u[i-1,j,k] + u[i+1,j,k]) invhx2
           + (u[i,j-1,k] + u[i,j+1,k]) invhy2 + (u[i,j,k-1] + u[i,j,k+1]) invhz2
with i the slowest index; boundary points of f are left untouched.
"""
import numpy as np


def copy(a):
    return a.copy()


def mul(c, s):
    return (np.asarray(s, c.dtype) * c).astype(c.dtype)


def add(a, b):
    return (a + b).astype(a.dtype)


def triad(b, c, s):
    return (b + np.asarray(s, c.dtype) * c).astype(b.dtype)


def dot(a, b):
    return float(np.dot(a.astype(np.float64), b.astype(np.float64)))


def laplacian(u, invhx2, invhy2, invhz2, invhxyz2, f=None):
    """Interior update of Listing 2; returns f (a copy of the given f, or zeros)."""
    u = np.asarray(u)
    out = np.zeros_like(u) if f is None else np.array(f, copy=True)
    c = u[1:-1, 1:-1, 1:-1]
    dt = u.dtype.type
    out[1:-1, 1:-1, 1:-1] = (c * dt(invhxyz2)
                             + (u[:-2, 1:-1, 1:-1] + u[2:, 1:-1, 1:-1]) * dt(invhx2)
                             + (u[1:-1, :-2, 1:-1] + u[1:-1, 2:, 1:-1]) * dt(invhy2)
                             + (u[1:-1, 1:-1, :-2] + u[1:-1, 1:-1, 2:]) * dt(invhz2))
    return out


def stencil_bytes(L, itemsize):
    """Eq. 1: bytes moved per stencil application on an L^3 grid."""
    fetch = L ** 3 - 8 - 12 * (L - 2)
    write = (L - 2) ** 3
    return (fetch + write) * itemsize


def stream_bytes(op, n, itemsize):
    """Eq. 2: bytes per BabelStream operation on n elements."""
    arrays = {"copy": 2, "mul": 2, "add": 3, "triad": 3, "dot": 2}[op]
    return arrays * n * itemsize
