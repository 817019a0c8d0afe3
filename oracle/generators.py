"""Entry functions A(I, J): every entry computable in O(1) (abstract; Sec. 1;
Sec. 5 list of kernels).  Each generator object maps global row and column
index arrays to the dense submatrix A(I, J) in float64 or complex128.

TEST INFRASTRUCTURE ONLY (see the package docstring).
"""
import numpy as np


class Gaussian:
    """Gaussian kernel exp(-||x_i - y_j||^2 / (2 h^2)) (Sec. 5, kernel 1)."""
    dtype = np.float64

    def __init__(self, x, y, h):
        self.x = np.asarray(x, np.float64)
        self.y = np.asarray(y, np.float64)
        self.h = float(h)
        self.m, self.n = self.x.shape[0], self.y.shape[0]

    def __call__(self, I, J):
        diff = self.x[np.asarray(I)][:, None, :] - self.y[np.asarray(J)][None, :, :]
        return np.exp(-(diff * diff).sum(axis=2) / (2.0 * self.h * self.h))


class Helmholtz:
    """3-D Helmholtz point kernel exp(i k r) / r, r = ||x_i - y_j||: a stand-in
    for the oscillatory, complex-valued EFIE kernels of Sec. 5 (kernels 2, 3)."""
    dtype = np.complex128

    def __init__(self, x, y, k):
        self.x = np.asarray(x, np.float64)
        self.y = np.asarray(y, np.float64)
        self.k = float(k)
        self.m, self.n = self.x.shape[0], self.y.shape[0]

    def __call__(self, I, J):
        diff = self.x[np.asarray(I)][:, None, :] - self.y[np.asarray(J)][None, :, :]
        r = np.sqrt((diff * diff).sum(axis=2))
        return np.exp(1j * self.k * r) / r


class Polynomial:
    """Polynomial kernel (x_i^t y_j + h)^2 (Sec. 5, kernel 5)."""
    dtype = np.float64

    def __init__(self, x, y, h):
        self.x = np.asarray(x, np.float64)
        self.y = np.asarray(y, np.float64)
        self.h = float(h)
        self.m, self.n = self.x.shape[0], self.y.shape[0]

    def __call__(self, I, J):
        return (self.x[np.asarray(I)] @ self.y[np.asarray(J)].T + self.h) ** 2


class Hankel2D:
    """EFIE2D kernel H0^(2)(k ||x_i - y_j||) (Sec. 5, kernel 2): the Hankel
    function of the second kind of order 0 (scipy.special.hankel2)."""
    dtype = np.complex128

    def __init__(self, x, y, k):
        self.x = np.asarray(x, np.float64)
        self.y = np.asarray(y, np.float64)
        self.k = float(k)
        self.m, self.n = self.x.shape[0], self.y.shape[0]

    def __call__(self, I, J):
        import scipy.special
        diff = self.x[np.asarray(I)][:, None, :] - self.y[np.asarray(J)][None, :, :]
        return scipy.special.hankel2(0, self.k * np.sqrt((diff * diff).sum(axis=2)))


class SparseProduct:
    """A = P Q + P2 Q2 with sparse P (m x K), Q (K x n) and a dense low-rank
    term: a coherent, non-smooth matrix of the kind on which ACA terminates
    prematurely (Sec. 1; Sec. 3.1).  P and Q are given densely here; the entry
    is the plain inner product over k."""
    dtype = np.float64

    def __init__(self, P, Q, P2, Q2):
        self.P = np.asarray(P, np.float64)
        self.Q = np.asarray(Q, np.float64)
        self.P2 = np.asarray(P2, np.float64)
        self.Q2 = np.asarray(Q2, np.float64)
        self.m, self.n = self.P.shape[0], self.Q.shape[1]

    def __call__(self, I, J):
        I = np.asarray(I); J = np.asarray(J)
        return self.P[I] @ self.Q[:, J] + self.P2[I] @ self.Q2[:, J]


class LowRank:
    """Product-of-random kernel A = U V (Sec. 5, kernel 6)."""

    def __init__(self, U, V):
        self.U = np.asarray(U)
        self.V = np.asarray(V)
        self.dtype = np.result_type(self.U, self.V)
        self.m, self.n = self.U.shape[0], self.V.shape[1]

    def __call__(self, I, J):
        return self.U[np.asarray(I)] @ self.V[:, np.asarray(J)]


class Dense:
    """An explicit matrix held in memory (tests only)."""

    def __init__(self, A):
        self.A = np.asarray(A)
        self.dtype = self.A.dtype
        self.m, self.n = self.A.shape

    def __call__(self, I, J):
        return self.A[np.ix_(np.asarray(I), np.asarray(J))]


class Window:
    """Restriction of a generator to the index window rows [r0, r0+m) x cols
    [c0, c0+n), addressed with local indices (a leaf A(I_tau, J_nu) of Alg. 3)."""

    def __init__(self, gen, r0, m, c0, n):
        self.gen, self.r0, self.c0 = gen, r0, c0
        self.m, self.n = m, n
        self.dtype = gen.dtype

    def __call__(self, I, J):
        return self.gen(np.asarray(I) + self.r0, np.asarray(J) + self.c0)
