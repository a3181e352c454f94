"""fvs_uq_batch beyond the per-sample means: each sample's final fields
against the oracle (lockstep and independent solves), the paper's own UQ
study (Section 5: Al-Si with the smeared Scheil law, its input
distributions, convection off, grain growth, the four domain outputs), and
the surrogate mode with its fallback to plain solves."""
import numpy as np
import pytest

from fvs_inputs import box_mesh, cases
from oracle.fv import Oracle

pytestmark = [pytest.mark.gpu, pytest.mark.filterwarnings("ignore::RuntimeWarning")]

TIGHT = dict(p_rtol=1e-13, mom_rtol=1e-12, e_rtol=1e-13, e_tol_T=1e-11, max_krylov_iters=2000)
GRAIN = dict(kp=cases.AL_SI_PAPER["kp"], D_s=3e-9, r0=1e-6)


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


def rel(a, b):
    s = np.abs(b).max()
    return np.abs(a - b).max() / (s if s > 0 else 1.0)


@pytest.mark.parametrize("mode", [0, 1])
def test_sample_fields_match_oracle(fvs, mode):
    """Three samples on a jittered, permuted 10x10x2 mesh for 25 steps
    (cells freeze at the walls meanwhile): every sample's temperature,
    velocity and pressure equal an oracle run with that sample's melt
    temperature, wall temperature and liquidus, cell by cell."""
    m = box_mesh(10, 10, 2, (0.012, 0.012, 0.003), jitter=0.2, jitter_seed=91, permute_seed=92)
    inputs = np.array([[930.0, 700.0, 4.0], [955.0, 680.0, 3.2], [942.0, 735.0, 4.8]])
    props = cases.props(**TIGHT)
    M = fvs.Mesh(m)
    nsteps = 25
    q, steps, ex = fvs.uq_run(M, props, inputs, 2e-3, nsteps, n_streams=2, mode=mode, fields=True)
    assert (steps == nsteps).all() and ex["used_plain"].all()
    for s, (Tm, Tw, C0) in enumerate(inputs):
        mat = dict(props["material"], T_liq=float(cases.liquidus_of(C0)))
        o = Oracle(m, cases.props(material=mat, walls=cases.all_walls(Tw), T_init=Tm, **TIGHT))
        o.run(2e-3, nsteps)
        assert (~o.lm).any()
        assert np.abs(ex["T"][s] - o.T).max() <= 1e-8, s
        assert rel(ex["U"][s], o.u) <= 1e-8, s
        assert rel(ex["P"][s], o.p) <= 1e-8, s


@pytest.mark.parametrize("mode", [0, 1])
def test_paper_uq_study_outputs(fvs, mode):
    """Section 5's study on a small box: Al-Si (smeared Scheil law, liquidus
    line T_f + m_l C0), inputs drawn from its distributions (melt N(1000, 10)
    K, walls N(500, 5) K, C0 N(10, 0.2) wt%), natural convection off, grain
    growth on, run to full solidification.  The four outputs -- total
    solidification time, maximum SDAS, minimum yield strength, maximum grain
    size -- equal the oracle's per sample."""
    m = box_mesh(8, 8, 2, (0.03, 0.03, 0.0075))
    inputs = cases.paper_uq_inputs(3, seed=5)
    props = cases.props(material=cases.AL_SI_PAPER, no_flow=True, **TIGHT)
    M = fvs.Mesh(m)
    q, steps, ex = fvs.uq_run(M, props, inputs, 2e-3, 2000, n_streams=2, mode=mode, qoi_kind=fvs.QOI_EXTREMES,
                              liquidus=(cases.AL_SI_T_F, cases.AL_SI_SLOPE), grain=GRAIN)
    assert np.isfinite(q).all()
    for s, (Tm, Tw, C0) in enumerate(inputs):
        mat = dict(cases.AL_SI_PAPER, T_liq=float(cases.paper_liquidus_of(C0)))
        o = Oracle(m, cases.props(material=mat, walls=cases.all_walls(Tw), T_init=Tm, no_flow=True, grain=GRAIN,
                                  **TIGHT))
        k = 0
        while k < 2000:
            k += 1
            if o.step(2e-3)["n_active"] == 0:
                break
        assert steps[s] == k
        np.testing.assert_allclose(q[s], o.qoi_extremes(), rtol=1e-8, err_msg=str(s))
    # the grains grew, and the yield strength follows from the largest SDAS (Eq. 23)
    assert (q[:, 3] > GRAIN["r0"]).all()
    np.testing.assert_allclose(q[:, 2], 59.0 / np.sqrt(q[:, 1]) + 120.3, rtol=1e-12)


def test_surrogate_mode_and_fallback(fvs):
    """Two networks trained on plain solves answer the samples inside their
    training box (the ensemble mean, steps 0); samples outside it fall back
    to plain solves equal to a direct plain run; with a spread limit no
    ensemble can meet, every sample falls back."""
    m = box_mesh(6, 6, 2, (0.008, 0.008, 0.002))
    M = fvs.Mesh(m)
    props = cases.props(p_rtol=1e-10, mom_rtol=1e-12, e_rtol=1e-12, e_tol_T=1e-9, max_krylov_iters=1000)
    Xtr = cases.uq_inputs(48, seed=1)
    Ytr, _ = fvs.uq_batch(M, props, Xtr, 2e-3, 1000)
    models = []
    for k in range(2):
        S = fvs.Surrogate(3, 32, 2, 4, seed=10 + k)
        S.set_scaling(Xtr.mean(0), Xtr.std(0), Ytr.mean(0), Ytr.std(0))
        S.train(Xtr, Ytr, 300, 3e-3)
        models.append(S)
    lo, hi = Xtr.min(0), Xtr.max(0)
    X = cases.uq_inputs(8, seed=2)
    X = np.clip(X, lo, hi)
    X[5, 1] = lo[1] - 30.0           # wall colder than any training sample
    X[6, 0] = hi[0] + 15.0           # hotter melt
    outside = np.zeros(8, bool)
    outside[[5, 6]] = True
    q, steps, ex = fvs.uq_run(M, props, X, 2e-3, 1000, mode=fvs.UQ_SURROGATE, models=models, box=(lo, hi),
                              plain_mode=fvs.UQ_LOCKSTEP)
    assert np.array_equal(ex["used_plain"], outside)
    assert (steps[~outside] == 0).all() and (steps[outside] > 0).all()
    ens = np.mean([S.predict(X[~outside]) for S in models], axis=0)
    np.testing.assert_allclose(q[~outside], ens, rtol=1e-12)
    qp, sp = fvs.uq_batch(M, props, X[outside], 2e-3, 1000)
    np.testing.assert_allclose(q[outside], qp, rtol=1e-10)
    assert np.array_equal(steps[outside], sp)
    # a spread limit the ensemble cannot meet: everything is solved plainly
    q2, s2, ex2 = fvs.uq_run(M, props, X, 2e-3, 1000, mode=fvs.UQ_SURROGATE, models=models, box=(lo, hi),
                             max_spread=1e-12, plain_mode=fvs.UQ_STREAMS, n_streams=4)
    assert ex2["used_plain"].all()
    qa, sa = fvs.uq_batch(M, props, X, 2e-3, 1000)
    np.testing.assert_allclose(q2, qa, rtol=1e-9)
    assert np.array_equal(s2, sa)
