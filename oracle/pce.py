"""FP64 reference of the paper's own UQ surrogate (test infrastructure only).

Section 2.7 expands an output in orthogonal polynomials of the standardised
stochastic inputs (generalised polynomial chaos, Eq. 27, truncated), fits the
coefficients by least squares on the outputs of deterministic runs at
collocation points (the Vandermonde system of Eq. 28), picks the points as
roots of the basis polynomials, combined by a tensor product or by
Smolyak's sparse rule, and reads sensitivities off the coefficients (total
Sobol indices, Section 5).  Hermite polynomials serve normal inputs (the
paper's case); Legendre polynomials serve uniform ones (the Askey scheme the
paper cites for choosing the family).

Only the tests, the smoke entry point and the benchmark's CPU leg use this
file; the CUDA library has its own implementation.  Library primitives used
as steps: numpy's Gauss quadrature rules for the 1-D roots, numpy's
least-squares solver.
"""
from __future__ import annotations

import itertools
import math

import numpy as np
from numpy.polynomial.hermite_e import hermegauss
from numpy.polynomial.legendre import leggauss

NORMAL = 0    # parameters (mean, standard deviation); xi = (x - mean)/sd ~ N(0, 1)
UNIFORM = 1   # parameters (lo, hi); xi = (2x - lo - hi)/(hi - lo) ~ U(-1, 1)


def basis_1d(family, xi, nmax):
    """Orthonormal 1-D polynomials psi_0..psi_nmax at xi: probabilists'
    Hermite He_n/sqrt(n!) (He_{n+1} = xi He_n - n He_{n-1}) or Legendre
    sqrt(2n+1) P_n ((n+1) P_{n+1} = (2n+1) xi P_n - n P_{n-1}), both
    normalised to unit variance under their distribution.
    Eq. 27."""
    xi = np.asarray(xi, dtype=np.float64)
    P = np.zeros((nmax + 1,) + xi.shape)
    P[0] = 1.0
    if nmax >= 1:
        P[1] = xi
    for n in range(1, nmax):
        if family == NORMAL:
            P[n + 1] = xi * P[n] - n * P[n - 1]
        else:
            P[n + 1] = ((2 * n + 1) * xi * P[n] - n * P[n - 1]) / (n + 1)
    for n in range(nmax + 1):
        P[n] *= 1.0 / math.sqrt(math.factorial(n)) if family == NORMAL else math.sqrt(2 * n + 1)
    return P


def multi_indices(d, p):
    """All alpha in N^d with |alpha| <= p, graded by total degree (alpha = 0 first).
    The total-degree truncation of Eq. 27."""
    out = []
    for deg in range(p + 1):
        for a in itertools.product(range(deg + 1), repeat=d):
            if sum(a) == deg:
                out.append(a)
    return np.array(out, dtype=np.int64)


class PCE:
    """Polynomial chaos expansion of n_out outputs in d inputs, total degree p.
    Eq. 27-28."""

    def __init__(self, families, params, degree):
        """Eq. 27-28."""
        self.fam = list(families)
        self.par = [tuple(map(float, q)) for q in params]
        self.d = len(self.fam)
        self.p = int(degree)
        self.alpha = multi_indices(self.d, self.p)
        self.coef = None

    def standardise(self, X):
        """Section 2.7: inputs mapped to the standard variables of Eq. 27."""
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        xi = np.empty_like(X)
        for j, (f, (a, b)) in enumerate(zip(self.fam, self.par)):
            xi[:, j] = (X[:, j] - a) / b if f == NORMAL else (2.0 * X[:, j] - a - b) / (b - a)
        return xi

    def vandermonde(self, X):
        """Psi[m, k] = prod_j psi_{alpha_kj}(xi_mj) (the matrix of Eq. 28)."""
        xi = self.standardise(X)
        B = [basis_1d(self.fam[j], xi[:, j], self.p) for j in range(self.d)]
        V = np.ones((len(xi), len(self.alpha)))
        for k, a in enumerate(self.alpha):
            for j in range(self.d):
                V[:, k] *= B[j][a[j]]
        return V

    def fit(self, X, Y):
        """Least-squares coefficients of Eq. 28 for each output column of Y."""
        V = self.vandermonde(X)
        Y = np.asarray(Y, dtype=np.float64).reshape(len(V), -1)
        self.coef, *_ = np.linalg.lstsq(V, Y, rcond=None)
        return self

    def __call__(self, X):
        """Eq. 27 evaluated at new inputs."""
        return self.vandermonde(X) @ self.coef

    def mean(self):
        """Mean of the expansion of Eq. 27 (its constant term)."""
        return self.coef[0]

    def variance(self):
        """Variance of the expansion of Eq. 27 (sum of squared non-constant terms)."""
        return (self.coef[1:] ** 2).sum(axis=0)

    def sobol_total(self):
        """Total index of input j: the variance share of every term with
        alpha_j > 0.  Returns [n_out, d].
        Section 5, Fig. 13."""
        v = self.variance()
        c2 = self.coef ** 2
        return np.stack([c2[self.alpha[:, j] > 0].sum(axis=0) / v for j in range(self.d)], axis=1)

    def sobol_first(self):
        """First-order index of input j: terms in alpha_j alone.  [n_out, d].
        Section 5, Fig. 13."""
        v = self.variance()
        c2 = self.coef ** 2
        only = [(self.alpha[:, j] > 0) & (self.alpha.sum(axis=1) == self.alpha[:, j]) for j in range(self.d)]
        return np.stack([c2[o].sum(axis=0) / v for o in only], axis=1)


def rule_1d(family, n):
    """n roots of the degree-n basis polynomial (Gauss points) and weights
    summing to 1, in the standardised variable.
    Section 2.7: the Gauss points the collocation samples."""
    if family == NORMAL:
        x, w = hermegauss(n)
    else:
        x, w = leggauss(n)
    return x, w / w.sum()


def tensor_nodes(families, level):
    """Tensor product of level-point Gauss rules: level^d points.
    Section 2.7, Table 2 (27 and 216 points)."""
    rules = [rule_1d(f, level)[0] for f in families]
    return np.array(list(itertools.product(*rules)))


def smolyak_nodes(families, level):
    """Smolyak's sparse grid on the level-i Gauss rules with i points: the
    union of the tensor grids X_i1 x ... x X_id over the multi-indices with
    i_j >= 1 and max(d, level) <= |i| <= level + d - 1 (Smolyak 1963; the
    non-nested Gaussian form of Heiss and Winschel).
    Section 2.7, Table 1."""
    d = len(families)
    pts = {}
    for idx in itertools.product(range(1, level + 1), repeat=d):
        if not (max(d, level) <= sum(idx) <= level + d - 1):
            continue
        for p in itertools.product(*[rule_1d(f, i)[0] for f, i in zip(families, idx)]):
            pts[tuple(np.round(p, 12))] = p
    return np.array(list(pts.values()))


def from_standard(families, params, xi):
    """Map standardised points back to the inputs' own units.
    Section 2.7."""
    xi = np.atleast_2d(xi)
    X = np.empty_like(xi)
    for j, (f, (a, b)) in enumerate(zip(families, params)):
        X[:, j] = a + b * xi[:, j] if f == NORMAL else 0.5 * (a + b) + 0.5 * (b - a) * xi[:, j]
    return X


def latin_hypercube(families, params, n, seed):
    """n Latin-hypercube samples of the inputs (one point per equal-probability
    stratum of every marginal, strata paired by random permutations).
    Sections 3 and 5: the Latin-hypercube test sets."""
    from scipy.stats import norm
    rng = np.random.default_rng(seed)
    d = len(families)
    U = (np.stack([rng.permutation(n) for _ in range(d)], axis=1) + rng.uniform(size=(n, d))) / n
    xi = np.empty_like(U)
    for j, f in enumerate(families):
        xi[:, j] = norm.ppf(U[:, j]) if f == NORMAL else 2.0 * U[:, j] - 1.0
    return from_standard(families, params, xi)
