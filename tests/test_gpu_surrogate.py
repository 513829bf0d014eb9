"""Surrogate-assisted APO on the GPU: with one candidate per protozoon it is
the plain method draw for draw (bit-identical curve and best), and its
bookkeeping (true evaluations, retrains) matches its parameters."""
import numpy as np
import pytest

from paper_2510_14982_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14982_gb300 import apo as m
    return m


@pytest.mark.parametrize("mk,ps,T", [(lambda: inputs.single_rastrigin(0), 20, 80),
                                     (lambda: inputs.composition(D=20, seed=2), 64, 40)])
def test_one_candidate_is_the_plain_method(apo, mk, ps, T):
    spec = mk()
    prob = apo.problem_from_spec(spec)
    prm = apo.apo_params_make(ps, 1, 0.1, T, 7)
    xp, fp, cp = apo.apo_run(prob, prm)
    xs, fs, cs, st = apo.apo_run_surrogate(prob, prm, apo.surrogate_params(k=1, retrain_every=10, train_steps=5))
    assert fs == fp
    np.testing.assert_array_equal(cs, cp)
    np.testing.assert_array_equal(xs, xp)
    assert st["true_evals"] == ps * (T + 1)
    assert st["screened"] == ps * T


def test_screening_bookkeeping(apo):
    spec = inputs.composition(D=20, seed=3)
    prob = apo.problem_from_spec(spec)
    ps, T, k = 64, 45, 4
    _, f, c, st = apo.apo_run_surrogate(prob, apo.apo_params_make(ps, 1, 0.1, T, 1),
                                        apo.surrogate_params(k=k, retrain_every=10, train_steps=20, batch=256))
    assert st["true_evals"] == ps * (T + 1)
    assert st["retrains"] == 4
    assert st["screening_iters"] + 10 + st["fallback_iters"] == T
    assert st["screened"] == ps * (T - st["screening_iters"]) + ps * k * st["screening_iters"]
    assert np.all(np.diff(c) <= 0) and c[-1] == np.float32(f)


@pytest.mark.parametrize("mk,ps,t,T,k", [
    (lambda: inputs.scale_forms(0, 20)[2], 48, 9, 60, 6),          # Rastrigin D 20, several ranks per chunk
    (lambda: inputs.scale_forms(1, 37)[3], 300, 150, 300, 3),      # hybrid, ragged D 37, ragged ps
    (lambda: inputs.composition(D=200, seed=0), 256, 40, 300, 8),  # the surrogate workload's problem
])
def test_surrogate_candidates_match_oracle(apo, orc, mk, ps, t, T, k):
    """The k candidates of every protozoon as the surrogate path generates them
    (slots | (c << 8)) against the oracle's, element by element: the modes,
    masks and indices are the same integer decisions on both sides, the
    positions agree within the one-iteration tolerance."""
    import torch
    from parity_helpers import close
    spec = mk()
    gprob = apo.problem_from_spec(spec)
    oprob = orc.OracleProblem.from_spec(spec)
    oprm = orc.params(ps, 1, 0.1, T, 5)
    gprm = apo.apo_params_make(ps, 1, 0.1, T, 5)
    X0, _ = orc.init_population(oprob, oprm)
    X32 = X0.astype(np.float32)
    F32 = orc.objective(oprob, X32.astype(np.float64)).astype(np.float32)
    d_X = torch.tensor(X32, device="cuda")
    d_F = torch.tensor(F32, device="cuda")
    d_Xc = torch.empty((ps, k, spec.D), device="cuda")
    apo.apo_surrogate_candidates(gprob, gprm, t, k, d_X, d_F, d_Xc)
    Xc_o, _ = orc.candidates(oprob, oprm, t, k, X32.astype(np.float64), F32.astype(np.float64))
    ok = close(d_Xc.cpu().numpy(), Xc_o)
    assert ok.all(), np.argwhere(~ok)[:10]


def test_trained_network_gains_over_the_plain_method(apo):
    """What the online-trained network adds: on the expensive composition
    objective (D 200, ps 256, 300 iterations), the surrogate-assisted form and
    the plain method spend the same number of true evaluations (ps per
    iteration plus the initial ps), and over 15 seeds the surrogate form's
    median best fitness is lower.  Its screening must actually have run (the
    rank correlation of predicted and true fitness kept it on)."""
    spec = inputs.composition(D=200, seed=0)
    prob = apo.problem_from_spec(spec)
    ps, T = 256, 300
    sp = apo.surrogate_params(k=8, retrain_every=10, archive_cap=50000, train_steps=50, batch=512, lr=1e-3,
                              train_window=1280)
    plain, surr, screening = [], [], []
    for seed in range(15):
        prm = apo.apo_params_make(ps, 1, 0.1, T, seed)
        plain.append(apo.apo_run(prob, prm, want_curve=False)[1])
        _, f, _, st = apo.apo_run_surrogate(prob, prm, sp, want_curve=False)
        assert st["true_evals"] == ps * (T + 1)
        surr.append(f)
        screening.append(st["screening_iters"])
    print("median best: plain %.6g, surrogate %.6g; screening iterations %s"
          % (np.median(plain), np.median(surr), screening))
    assert np.median(surr) < np.median(plain)
    assert np.median(screening) > T / 2
