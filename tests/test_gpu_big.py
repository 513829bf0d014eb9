"""GPU parity of the large-dimension path (256 < D <= 1024; the paper's Table 2
shapes at D = 1000): the TMA-fed tcgen05 rotation GEMM with the objective in
its epilogue, the chunked sort and rank, and the warp-per-row generation,
against the FP64 oracle.  Tolerance |gpu - oracle| <= 1e-4 + 1e-5 |oracle|;
acceptance decisions may differ only at near-ties, at most 1% of ps."""
import numpy as np
import pytest

from paper_2510_14982_gb300 import inputs
from parity_helpers import assert_step_ok, close, compare_step, gpu_eval

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14982_gb300 import apo as m
    return m


FORMS = [inputs.OBJ_BENTCIGAR, inputs.OBJ_ELLIPTIC, inputs.OBJ_HGBAT, inputs.OBJ_ROSENBROCK, inputs.OBJ_GRIEWANK,
         inputs.OBJ_RASTRIGIN, inputs.OBJ_HYBRID]


@pytest.mark.parametrize("D", [300, 1000])
@pytest.mark.parametrize("kind", FORMS, ids=[inputs.FORM_NAMES[k] for k in FORMS])
def test_objective_parity_large_dimension(apo, orc, kind, D):
    """Rows spanning several 128-row GEMM tiles with a ragged tail; the shift
    itself (f(o) = 0 where the form has it there)."""
    spec = inputs.shifted_rotated(kind, D, 21 + D, run=kind)
    X = inputs.random_state(spec, 300, seed=5)
    if kind not in (inputs.OBJ_ROSENBROCK, inputs.OBJ_HYBRID):
        X[7] = spec.shift
    Fg = gpu_eval(apo, apo.problem_from_spec(spec), X)
    Fo = orc.objective(orc.OracleProblem.from_spec(spec), X.astype(np.float64))
    worst = np.max(np.abs(Fg - Fo) / (1e-4 + 1e-5 * np.abs(Fo)))
    assert np.all(close(Fg, Fo)), worst


def test_unrotated_large_dimension(apo, orc):
    spec = inputs.ProblemSpec(kind=inputs.OBJ_ELLIPTIC, D=513, lb=np.full(513, -50.0), ub=np.full(513, 50.0),
                              shift=inputs.shift(513, 3))
    X = inputs.random_state(spec, 129, seed=2)
    Fg = gpu_eval(apo, apo.problem_from_spec(spec), X)
    Fo = orc.objective(orc.OracleProblem.from_spec(spec), X.astype(np.float64))
    assert np.all(close(Fg, Fo))


BIG_STEPS = [
    # (name, spec factory, ps, t, T, kwargs)
    ("hybrid300_ps300", lambda: inputs.shifted_rotated(inputs.OBJ_HYBRID, 300, 1), 300, 3, 100, {}),
    ("rosenbrock1000_ps1000", lambda: inputs.shifted_rotated(inputs.OBJ_ROSENBROCK, 1000, 2), 1000, 2, 1000, {}),
    ("bent1000_ps1100_two_chunks", lambda: inputs.shifted_rotated(inputs.OBJ_BENTCIGAR, 1000, 3), 1100, 5, 1000, {}),
    ("griewank1000_ps512", lambda: inputs.shifted_rotated(inputs.OBJ_GRIEWANK, 1000, 4), 512, 7, 1000, {}),
    ("hgbat1000_ps512", lambda: inputs.shifted_rotated(inputs.OBJ_HGBAT, 1000, 5), 512, 9, 1000, {}),
    ("elliptic777_pfmax1_pdr1", lambda: inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 777, 6), 256, 4, 100,
     dict(pf_max=1.0, pdr_form=1)),
    ("rastrigin1024_np3_policy1", lambda: inputs.shifted_rotated(inputs.OBJ_RASTRIGIN, 1024, 7), 256, 6, 100,
     dict(np_=3, pair_policy=1)),
    ("elliptic300_last_iteration", lambda: inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 300, 8), 200, 50, 50,
     dict(pf_max=0.5)),
]


@pytest.mark.parametrize("name,mk,ps,t,T,kw", BIG_STEPS, ids=[c[0] for c in BIG_STEPS])
def test_step_parity_large_dimension(apo, orc, name, mk, ps, t, T, kw):
    r = compare_step(apo, orc, mk(), ps, t, T, **kw)
    assert_step_ok(r)


def test_initial_population_large_dimension(apo, orc):
    import torch
    spec = inputs.shifted_rotated(inputs.OBJ_BENTCIGAR, 1000, 9)
    prob = apo.problem_from_spec(spec)
    prm = apo.apo_params_make(257, 1, 0.1, 10, 3)
    X = torch.empty((257, 1000), device="cuda")
    F = torch.empty(257, device="cuda")
    apo.apo_init_state(prob, prm, X, F)
    torch.cuda.synchronize()
    oprob = orc.OracleProblem.from_spec(spec)
    Xo, Fo = orc.init_population(oprob, orc.params(257, 1, 0.1, 10, 3))
    assert close(X.cpu().numpy(), Xo).all()
    assert close(F.cpu().numpy(), orc.objective(oprob, X.cpu().numpy().astype(np.float64))).all()


def test_run_invariants_and_resume_large_dimension(apo):
    """A whole run at D 1000 (ps 300, 40 iterations): monotone curve, best inside
    the bounds with f(best_x) = best_f; the run split into two segments
    (apo_init_state, apo_run_from_state) gives the same curve bit for bit."""
    import torch
    spec = inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 1000, 10)
    prob = apo.problem_from_spec(spec)
    T = 40
    prm = apo.apo_params_make(300, 1, 0.1, T, 4)
    bx, bf, curve = apo.apo_run(prob, prm)
    assert np.all(np.diff(curve) <= 0) and curve[-1] == np.float32(bf) and bf < curve[0]
    assert np.all(bx >= spec.lb) and np.all(bx <= spec.ub)
    assert close(gpu_eval(apo, prob, bx[None]), [bf]).all()
    X = torch.empty((300, 1000), device="cuda")
    F = torch.empty(300, device="cuda")
    apo.apo_init_state(prob, prm, X, F)
    c1 = torch.empty(18, device="cuda")
    c2 = torch.empty(T - 18 + 2, device="cuda")
    bx2 = torch.empty(1000, device="cuda")
    bf2 = torch.empty(1, dtype=torch.float64, device="cuda")
    apo.apo_run_from_state(prob, prm, 1, 17, X, F, None, None, c1)
    apo.apo_run_from_state(prob, prm, 18, T, X, F, bx2, bf2, c2)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(np.concatenate([c1.cpu().numpy(), c2.cpu().numpy()[1:]]), curve)
    assert bf2.item() == bf
    np.testing.assert_array_equal(bx2.cpu().numpy(), bx)


def test_batch_of_large_runs_equals_single_runs(apo):
    import torch
    specs = [inputs.shifted_rotated(k, 600, 11, run=k) for k in (inputs.OBJ_GRIEWANK, inputs.OBJ_HGBAT)]
    probs = [apo.problem_from_spec(s) for s in specs]
    T = 15
    prms = [apo.apo_params_make(200, 1, 0.1, T, 6, k) for k in range(2)]
    bx = torch.zeros((2, 600), device="cuda")
    bf = torch.zeros(2, dtype=torch.float64, device="cuda")
    cv = torch.zeros((2, T + 1), device="cuda")
    apo.apo_run_batch(probs, prms, bx, 600, bf, cv, T + 1)
    torch.cuda.synchronize()
    for k in range(2):
        x, f, c = apo.apo_run(probs[k], prms[k])
        assert bf[k].item() == f
        np.testing.assert_array_equal(cv[k].cpu().numpy(), c)
        np.testing.assert_array_equal(bx[k].cpu().numpy(), x)
