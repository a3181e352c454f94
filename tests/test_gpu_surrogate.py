"""The BF16 tensor-core surrogate against the FP64 reference network, and
what it gains over plain solves in a Monte Carlo loop."""
import time

import numpy as np
import pytest

from fvs_inputs import box_mesh, cases
from oracle import mlp as ref

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

SIZES = [3, 128, 128, 128, 128, 4]


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


def test_forward_and_gradients_match_fp64_reference(fvs):
    """Same parameters on both sides: BF16 operands with FP32 accumulation
    stay within BF16 rounding of the FP64 forward pass and gradients."""
    S = fvs.Surrogate(3, 128, 4, 4, seed=11)
    p = S.get_params()
    params = ref.unflatten(p, SIZES)
    rng = np.random.default_rng(0)
    X = rng.normal(size=(300, 3))
    T = rng.normal(size=(300, 4))
    Y = S.predict(X)
    Yr, _ = ref.forward(params, X)
    assert np.abs(Y - Yr).max() <= 3e-2 * np.abs(Yr).max()
    g, loss = S.gradients(X, T)
    gr = ref.flatten(ref.backward(params, X, T))
    assert abs(loss - ref.loss(params, X, T)) <= 1e-2 * ref.loss(params, X, T)
    cos = g @ gr / (np.linalg.norm(g) * np.linalg.norm(gr))
    assert cos > 0.999 and np.linalg.norm(g - gr) <= 5e-2 * np.linalg.norm(gr), (cos, np.linalg.norm(g - gr) / np.linalg.norm(gr))
    # parameters round-trip through the flat layout
    S.set_params(p * 0.5)
    np.testing.assert_allclose(S.get_params(), p * 0.5, rtol=1e-7)


def test_adam_steps_match_oracle(fvs):
    """Two full-batch Adam steps on the GPU (FP32 master weights) against the
    FP64 Adam of the oracle fed with the GPU's own gradients at the same
    weights, so that only the optimiser is compared: the first step is
    -lr g/(|g| + eps) in closed form, the second one mixes both gradients."""
    S = fvs.Surrogate(3, 128, 4, 4, seed=21)
    rng = np.random.default_rng(3)
    X = rng.normal(size=(200, 3))
    T = rng.normal(size=(200, 4))
    lr = 1e-3
    st = ref.adam_init(S.num_params())
    th = S.get_params()
    for _ in range(2):
        g, _ = S.gradients(X, T)
        th_ref = ref.adam_step(st, th, g, lr)
        S.train(X, T, 1, lr)
        th_gpu = S.get_params()
        # FP32 weights and moments: a few ulps of the weight plus a few ulps
        # of the step where |g| is near eps
        tol = 4e-7 * np.abs(th) + 1e-6 * lr
        bad = np.abs(th_gpu - th_ref) > tol
        assert not bad.any(), (bad.sum(), np.abs(th_gpu - th_ref)[bad][:5])
        th = th_gpu


def test_training_fits_a_smooth_map(fvs):
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, size=(512, 3))
    f = lambda x: np.stack([np.sin(2 * x[:, 0]) + x[:, 1] ** 2, x[:, 0] * x[:, 2], np.exp(0.5 * x[:, 1]),
                            x[:, 0] + x[:, 1] - x[:, 2]], axis=1)
    T = f(X)
    S = fvs.Surrogate(3, 128, 4, 4, seed=2)
    S.set_scaling(X.mean(0), X.std(0), T.mean(0), T.std(0))
    loss = S.train(X, T, 1500, 1e-3)
    assert loss < 2e-3
    Xh = rng.uniform(-1, 1, size=(256, 3))
    err = np.abs(S.predict(Xh) - f(Xh)).max(axis=0) / T.std(0)
    assert np.all(err < 0.1), err


def test_surrogate_gain_over_plain_solves(fvs):
    """Train on plain batched UQ solves of a small cooled cavity, judge on
    held-out solves, and compare Monte Carlo statistics and throughput."""
    m = box_mesh(8, 8, 2, (0.01, 0.01, 0.0025))
    M = fvs.Mesh(m)
    props = cases.props(p_rtol=1e-8, mom_rtol=1e-10, e_rtol=1e-10, e_tol_T=1e-6)
    Xtr = cases.uq_inputs(96, seed=1)
    Xte = cases.uq_inputs(24, seed=2)
    t0 = time.perf_counter()
    Ytr, _ = fvs.uq_batch(M, props, Xtr, 2e-3, 600, n_streams=8)
    plain_rate = len(Xtr) / (time.perf_counter() - t0)
    Yte, _ = fvs.uq_batch(M, props, Xte, 2e-3, 600, n_streams=8)
    assert np.isfinite(Ytr).all() and np.isfinite(Yte).all()
    S = fvs.Surrogate(3, 128, 4, 4, seed=3)
    S.set_scaling(Xtr.mean(0), Xtr.std(0), Ytr.mean(0), Ytr.std(0))
    S.train(Xtr, Ytr, 3000, 1e-3)
    rel = np.abs(S.predict(Xte) - Yte) / np.abs(Yte)
    assert rel.mean() < 0.02, rel.mean(axis=0)
    # paired Monte Carlo means on the held-out inputs
    assert np.all(np.abs(S.predict(Xte).mean(0) - Yte.mean(0)) <= 0.01 * np.abs(Yte.mean(0)))
    Xmc = cases.uq_inputs(200000, seed=4)
    S.predict(Xmc[:1000])
    t0 = time.perf_counter()
    S.predict(Xmc)
    sur_rate = len(Xmc) / (time.perf_counter() - t0)
    assert sur_rate > 1000 * plain_rate, (sur_rate, plain_rate)
