"""GPU: the initial population (S0) element by element against the oracle,
resumable runs (apo_init_state / apo_run_from_state) against uninterrupted
runs, the evaluation budget, and the pair-policy variant of Eq. 6-7 against
the oracle's step."""
import numpy as np
import pytest

from paper_2510_14982_gb300 import inputs
from parity_helpers import assert_step_ok, close, compare_step

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14982_gb300 import apo as m
    return m


INIT_CASES = [
    ("rastrigin10_ps20", lambda: inputs.single_rastrigin(0), 20),           # work-queue kernel, resident
    ("hybrid37_ps300", lambda: inputs.shifted_rotated(inputs.OBJ_HYBRID, 37, 2), 300),   # grid kernel
    ("elliptic100_ps4096", lambda: inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 100, 1), 4096),
    ("composition200_ps64", lambda: inputs.composition(D=200, seed=1), 64),
]


@pytest.mark.parametrize("name,mk,ps", INIT_CASES, ids=[c[0] for c in INIT_CASES])
def test_initial_population_matches_oracle(apo, orc, name, mk, ps):
    """Algorithm 1 initialisation: X_p = Xmin + U (Xmax - Xmin) from the INIT
    draws, F_p = f(X_p), element by element within the tolerance."""
    import torch
    spec = mk()
    prob = apo.problem_from_spec(spec)
    prm = apo.apo_params_make(ps, 1, 0.1, 100, 7, 3)
    X = torch.empty((ps, spec.D), device="cuda")
    F = torch.empty(ps, device="cuda")
    apo.apo_init_state(prob, prm, X, F)
    torch.cuda.synchronize()
    oprob = orc.OracleProblem.from_spec(spec)
    Xo, Fo = orc.init_population(oprob, orc.params(ps, 1, 0.1, 100, 7, 3))
    assert close(X.cpu().numpy(), Xo).all()
    # fitness of the float32 positions (the state the GPU keeps)
    Fo32 = orc.objective(oprob, X.cpu().numpy().astype(np.float64))
    assert close(F.cpu().numpy(), Fo32).all()
    assert close(F.cpu().numpy(), Fo).all()


def test_initial_population_otsu(apo, orc):
    hist = np.bincount(inputs.gmm_image(3, 1 << 16), minlength=256)
    spec = inputs.otsu_problem(hist, 4)
    prob = apo.problem_from_spec(spec)
    import torch
    X = torch.empty((100, 4), device="cuda")
    F = torch.empty(100, dtype=torch.float64, device="cuda")
    apo.apo_init_state(prob, apo.apo_params_make(100, 1, 0.1, 50, 2), X, F)
    torch.cuda.synchronize()
    oprob = orc.OracleProblem.from_spec(spec)
    Xo, _ = orc.init_population(oprob, orc.params(100, 1, 0.1, 50, 2))
    assert close(X.cpu().numpy(), Xo).all()
    assert np.array_equal(F.cpu().numpy(), orc.objective(oprob, X.cpu().numpy().astype(np.float64)))


RESUME_CASES = [
    ("rastrigin10_ps20", lambda: inputs.single_rastrigin(0), 20, 120, (1, 37, 38, 120)),
    ("hybrid50_ps1500", lambda: inputs.shifted_rotated(inputs.OBJ_HYBRID, 50, 2), 1500, 60, (1, 20, 45, 60)),
    ("elliptic100_ps4096", lambda: inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 100, 1), 4096, 40, (1, 13, 40)),
]


@pytest.mark.parametrize("name,mk,ps,T,cuts", RESUME_CASES, ids=[c[0] for c in RESUME_CASES])
def test_segmented_run_equals_uninterrupted_run(apo, name, mk, ps, T, cuts):
    """apo_init_state, then apo_run_from_state over segments [1, c1), [c1, c2),
    ..., gives the uninterrupted run's curve and best, bit for bit."""
    import torch
    spec = mk()
    prob = apo.problem_from_spec(spec)
    prm = apo.apo_params_make(ps, 1, 0.1, T, 11)
    bx_ref, bf_ref, c_ref = apo.apo_run(prob, prm)
    X = torch.empty((ps, spec.D), device="cuda")
    F = torch.empty(ps, device="cuda")
    apo.apo_init_state(prob, prm, X, F)
    curve = np.empty(T + 1, np.float32)
    bx = torch.empty(spec.D, device="cuda")
    bf = torch.empty(1, dtype=torch.float64, device="cuda")
    edges = list(cuts)
    if edges[-1] != T + 1:
        edges.append(T + 1)
    for a, b in zip(edges[:-1], edges[1:]):
        seg = torch.full((b - a + 1,), float("nan"), device="cuda")
        apo.apo_run_from_state(prob, prm, a, b - 1, X, F, bx, bf, seg)
        torch.cuda.synchronize()
        s = seg.cpu().numpy()
        if a > 1:
            assert s[0] == curve[a - 1]          # the segment starts from the previous one's end
        curve[a - 1:b] = s
    np.testing.assert_array_equal(curve, c_ref)
    assert bf.item() == bf_ref
    np.testing.assert_array_equal(bx.cpu().numpy(), bx_ref)
    # the returned state holds the best at rank 0 of its order, with the run's best value
    assert F.cpu().numpy().min() == np.float32(bf_ref)


def test_zero_iteration_segment_returns_its_input(apo):
    import torch
    spec = inputs.single_rastrigin(1)
    prob = apo.problem_from_spec(spec)
    prm = apo.apo_params_make(20, 1, 0.1, 50, 1)
    X = torch.empty((20, 10), device="cuda")
    F = torch.empty(20, device="cuda")
    apo.apo_init_state(prob, prm, X, F)
    X0, F0 = X.clone(), F.clone()
    c = torch.empty(1, device="cuda")
    apo.apo_run_from_state(prob, prm, 5, 4, X, F, None, None, c)
    torch.cuda.synchronize()
    assert torch.equal(X, X0) and torch.equal(F, F0)
    assert c.item() == F0.min().item()


def test_evaluation_budget(apo, orc):
    """max_fes = ps (T + 1) + r (r < ps) runs T iterations with iter_max = T:
    the same results as max_iter = T, and the same number of iterations as
    the oracle's budget reading; the first iterations follow the oracle."""
    spec = inputs.single_rastrigin(0)
    prob = apo.problem_from_spec(spec)
    p_budget = apo.apo_params_make(20, 1, 0.1, 999999, 3, 0, 0, 0, 20 * 301 + 13)
    assert apo.apo_effective_iterations(p_budget) == 300
    bx1, bf1, c1 = apo.apo_run(prob, p_budget)
    bx2, bf2, c2 = apo.apo_run(prob, apo.apo_params_make(20, 1, 0.1, 300, 3))
    assert len(c1) == 301 and bf1 == bf2
    np.testing.assert_array_equal(c1, c2)
    np.testing.assert_array_equal(bx1, bx2)
    oprob = orc.OracleProblem.from_spec(spec)
    _, _, co = orc.apo_run(oprob, orc.params(20, 1, 0.1, 999999, 3, 0, 0, 0, 20 * 301 + 13))
    assert len(co) == len(c1)
    assert close(c1[:20], co[:20]).all()
    with pytest.raises(apo.ApoError) as e:
        apo.apo_run(prob, apo.apo_params_make(20, 1, 0.1, 10, 3, 0, 0, 0, 39))
    assert e.value.status == apo.APO_ERR_INVALID_ARG


PAIR_CASES = [
    ("rastrigin10_ps20", lambda: inputs.single_rastrigin(0), 20, 2, 1),
    ("hybrid37_ps300_np3", lambda: inputs.shifted_rotated(inputs.OBJ_HYBRID, 37, 2), 300, 5, 3),
    ("rosenbrock100_ps4096", lambda: inputs.shifted_rotated(inputs.OBJ_ROSENBROCK, 100, 2), 4096, 3, 1),
]


@pytest.mark.parametrize("name,mk,ps,t,np_", PAIR_CASES, ids=[c[0] for c in PAIR_CASES])
def test_pair_policy_step_matches_oracle(apo, orc, name, mk, ps, t, np_):
    r = compare_step(apo, orc, mk(), ps, t, 50, seed=4, np_=np_, pair_policy=1)
    assert r["modes"][2] > 0, r
    assert_step_ok(r)
