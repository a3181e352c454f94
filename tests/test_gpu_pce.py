"""The polynomial chaos surrogate on the GPU (Section 2.7, Eq. 27-28;
Section 5) against the FP64 oracle of the same expansion: collocation
points, multi-index order, least-squares coefficients, evaluation on Latin
hypercube samples and the Sobol indices."""
import numpy as np
import pytest

from oracle import pce as ref

pytestmark = [pytest.mark.gpu]

FAMS = [ref.NORMAL, ref.UNIFORM, ref.NORMAL]
PARS = [(1000.0, 10.0), (650.0, 750.0), (10.0, 0.2)]


@pytest.fixture(scope="module")
def fvs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import os
    from paper_1810_08572_gb300 import LIB_PATH, build
    if not os.path.exists(LIB_PATH):
        build()
    from paper_1810_08572_gb300 import fvs as f
    return f


def _sorted(X):
    return X[np.lexsort(X.T[::-1])]


def test_nodes_and_terms_match_the_oracle(fvs):
    P = fvs.Pce(FAMS, PARS, 4, 2)
    assert P.num_terms() == 35
    np.testing.assert_array_equal(P.multi_indices(), ref.multi_indices(3, 4))
    for level, sparse in ((3, False), (6, False), (4, True), (5, True)):
        X = P.nodes(level, sparse)
        xi = ref.smolyak_nodes(FAMS, level) if sparse else ref.tensor_nodes(FAMS, level)
        Xr = ref.from_standard(FAMS, PARS, xi)
        assert X.shape == Xr.shape
        np.testing.assert_allclose(_sorted(X), _sorted(Xr), rtol=1e-12, atol=1e-12)
    assert len(P.nodes(3)) == 27 and len(P.nodes(6)) == 216          # Table 2
    P4 = fvs.Pce([ref.NORMAL] * 4, [(0.0, 1.0)] * 4, 2, 1)
    assert [len(P4.nodes(l, True)) for l in (4, 5, 6)] == [137, 385, 953]   # Table 1


@pytest.mark.parametrize("degree,level,sparse", [(3, 5, False), (6, 8, False), (4, 7, True)])
def test_fit_eval_and_sobol_match_the_oracle(fvs, degree, level, sparse):
    """A smooth two-output map of the three UQ inputs (not a polynomial):
    coefficients, predictions at 60 Latin-hypercube points and the Sobol
    indices agree with the oracle's least-squares fit."""
    P = fvs.Pce(FAMS, PARS, degree, 2)
    X = P.nodes(level, sparse)

    def f(X):
        a = (X[:, 0] - 1000.0) / 10.0
        b = (X[:, 1] - 700.0) / 50.0
        c = (X[:, 2] - 10.0) / 0.2
        return np.stack([np.exp(0.3 * a) + np.sin(b) * c, 1.0 / (2.5 + np.tanh(a * b)) + 0.1 * c * c], axis=1)

    Y = f(X)
    P.fit(X, Y)
    o = ref.PCE(FAMS, PARS, degree).fit(X, Y)
    scale = np.abs(o.coef).max(axis=0)
    assert np.all(np.abs(P.coefficients() - o.coef).max(axis=0) <= 1e-9 * scale)
    Xt = ref.latin_hypercube(FAMS, PARS, 60, seed=3)
    np.testing.assert_allclose(P(Xt), o(Xt), rtol=1e-9, atol=1e-9 * np.abs(o(Xt)).max())
    m, v, t, fi = P.sensitivity()
    np.testing.assert_allclose(m, o.mean(), rtol=1e-10)
    np.testing.assert_allclose(v, o.variance(), rtol=1e-9)
    np.testing.assert_allclose(t, o.sobol_total(), atol=1e-9)
    np.testing.assert_allclose(fi, o.sobol_first(), atol=1e-9)


def test_exact_polynomial_and_device_evaluation(fvs):
    """A polynomial of the truncation degree is recovered exactly, and
    evaluation from device buffers equals evaluation from host ones."""
    import torch
    P = fvs.Pce(FAMS, PARS, 3, 1)
    truth = ref.PCE(FAMS, PARS, 3)
    truth.coef = np.random.default_rng(2).normal(size=(len(truth.alpha), 1))
    X = P.nodes(4)
    P.fit(X, truth(X))
    np.testing.assert_allclose(P.coefficients(), truth.coef, atol=1e-10)
    Xt = ref.latin_hypercube(FAMS, PARS, 1000, seed=4)
    Yd = torch.empty((1000, 1), dtype=torch.float64, device="cuda")
    P(torch.tensor(Xt, device="cuda"), Yd)
    np.testing.assert_array_equal(Yd.cpu().numpy(), P(Xt))
