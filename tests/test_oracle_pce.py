"""Pins of the polynomial-chaos oracle (Section 2.7, Eq. 27-28; Section 5).

* The basis: the recurrences reproduce the closed forms He_2..He_4 and
  P_2, P_3; the Gauss rules integrate the normal moments (2k-1)!! and the
  uniform moments 1/(2k+1); the basis is orthonormal under them.
* The collocation grids: a tensor grid of level l has l^3 points in three
  dimensions, the paper's 27 and 216 (Table 2); Smolyak's sparse grid on
  Gaussian rules in four dimensions has 137, 385 and 953 points at levels
  4, 5 and 6, the counts of Table 1.
* The fit: polynomials of the truncation degree are recovered exactly, on
  tensor and on sparse grids.
* Total Sobol indices: closed forms for a quadratic in normal inputs and for
  the Ishigami function (uniform inputs), whose indices follow from
  E[sin^2] = 1/2, E[sin^4] = 3/8, E[x^4] = pi^4/5, E[x^8] = pi^8/9 on
  [-pi, pi].
"""
import math

import numpy as np

from oracle.pce import (NORMAL, UNIFORM, PCE, basis_1d, from_standard, latin_hypercube, multi_indices, rule_1d,
                        smolyak_nodes, tensor_nodes)


def test_recurrences_match_closed_forms():
    x = np.linspace(-3, 3, 13)
    H = basis_1d(NORMAL, x, 4)
    np.testing.assert_allclose(H[2] * math.sqrt(2), x ** 2 - 1, atol=1e-13)
    np.testing.assert_allclose(H[3] * math.sqrt(6), x ** 3 - 3 * x, atol=1e-12)
    np.testing.assert_allclose(H[4] * math.sqrt(24), x ** 4 - 6 * x ** 2 + 3, atol=1e-11)
    y = np.linspace(-1, 1, 11)
    P = basis_1d(UNIFORM, y, 3)
    np.testing.assert_allclose(P[2] / math.sqrt(5), (3 * y ** 2 - 1) / 2, atol=1e-14)
    np.testing.assert_allclose(P[3] / math.sqrt(7), (5 * y ** 3 - 3 * y) / 2, atol=1e-14)


def test_gauss_rules_and_orthonormality():
    for n in (3, 6, 9):
        x, w = rule_1d(NORMAL, n)
        for k in range(n):     # exact up to degree 2n - 1
            dfact = np.prod(np.arange(2 * k - 1, 0, -2)) if k > 0 else 1.0
            assert abs((w * x ** (2 * k)).sum() - dfact) <= 1e-11 * dfact
        x, w = rule_1d(UNIFORM, n)
        for k in range(n):
            assert abs((w * x ** (2 * k)).sum() - 1.0 / (2 * k + 1)) <= 1e-14
        for fam in (NORMAL, UNIFORM):
            x, w = rule_1d(fam, n)
            B = basis_1d(fam, x, n - 1)
            np.testing.assert_allclose((B * w) @ B.T, np.eye(n), atol=1e-12)


def test_collocation_node_counts_match_the_paper():
    fam3 = [NORMAL] * 3
    assert len(tensor_nodes(fam3, 3)) == 27 and len(tensor_nodes(fam3, 6)) == 216     # Table 2
    fam4 = [NORMAL] * 4
    assert [len(smolyak_nodes(fam4, l)) for l in (4, 5, 6)] == [137, 385, 953]        # Table 1
    # a two-dimensional sparse grid (the table's caption) would be far smaller
    assert len(smolyak_nodes([NORMAL] * 2, 6)) < 137


def test_polynomials_are_recovered_exactly():
    fams = [NORMAL, UNIFORM, NORMAL]
    pars = [(1000.0, 10.0), (650.0, 750.0), (10.0, 0.2)]
    rng = np.random.default_rng(0)
    for p in (2, 4):
        truth = PCE(fams, pars, p)
        truth.coef = rng.normal(size=(len(truth.alpha), 2))
        for xi in (tensor_nodes(fams, p + 1), smolyak_nodes(fams, p + 2)):
            X = from_standard(fams, pars, xi)
            fit = PCE(fams, pars, p).fit(X, truth(X))
            np.testing.assert_allclose(fit.coef, truth.coef, atol=1e-10)
    assert len(multi_indices(3, 4)) == math.comb(3 + 4, 4)


def test_sobol_indices_of_a_quadratic_in_normal_inputs():
    """f = a xi1 + b (xi2^2 - 1) + c xi1 xi3 + 5: mean 5, variance
    a^2 + 2 b^2 + c^2, S_T1 = (a^2 + c^2)/V, S_T2 = 2 b^2/V, S_T3 = c^2/V;
    first-order S_1 = a^2/V, S_3 = 0."""
    fams = [NORMAL] * 3
    pars = [(1000.0, 10.0), (500.0, 5.0), (10.0, 0.2)]
    a, b, c = 1.3, -0.7, 0.4
    X = from_standard(fams, pars, tensor_nodes(fams, 3))
    xi = (X - np.array([p[0] for p in pars])) / np.array([p[1] for p in pars])
    f = a * xi[:, 0] + b * (xi[:, 1] ** 2 - 1) + c * xi[:, 0] * xi[:, 2] + 5.0
    pce = PCE(fams, pars, 2).fit(X, f)
    V = a * a + 2 * b * b + c * c
    assert abs(pce.mean()[0] - 5.0) < 1e-12 and abs(pce.variance()[0] - V) < 1e-12
    np.testing.assert_allclose(pce.sobol_total()[0], [(a * a + c * c) / V, 2 * b * b / V, c * c / V], atol=1e-12)
    np.testing.assert_allclose(pce.sobol_first()[0], [a * a / V, 2 * b * b / V, 0.0], atol=1e-12)


def test_ishigami_total_indices():
    a, b = 7.0, 0.1
    pi = math.pi
    V1 = 0.5 * (1 + b * pi ** 4 / 5) ** 2
    V2 = a * a / 8
    V13 = b * b * pi ** 8 * (1 / 18 - 1 / 50)
    V = V1 + V2 + V13
    fams = [UNIFORM] * 3
    pars = [(-pi, pi)] * 3
    X = from_standard(fams, pars, tensor_nodes(fams, 16))
    f = np.sin(X[:, 0]) + a * np.sin(X[:, 1]) ** 2 + b * X[:, 2] ** 4 * np.sin(X[:, 0])
    pce = PCE(fams, pars, 14).fit(X, f)
    assert abs(pce.variance()[0] - V) <= 1e-4 * V
    np.testing.assert_allclose(pce.sobol_total()[0], [(V1 + V13) / V, V2 / V, V13 / V], atol=1e-4)
    # held-out Latin-hypercube points: the expansion interpolates the function
    Xt = latin_hypercube(fams, pars, 60, seed=1)
    ft = np.sin(Xt[:, 0]) + a * np.sin(Xt[:, 1]) ** 2 + b * Xt[:, 2] ** 4 * np.sin(Xt[:, 0])
    assert np.sqrt(np.mean((pce(Xt)[:, 0] - ft) ** 2)) <= 1e-3 * np.abs(ft).max()
