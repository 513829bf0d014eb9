"""GPU parity: the CUDA path (called through the C ABI) against the FP64 oracle
on the same seeded inputs.

* Philox4x32-10 on the device: bit-exact against the oracle's generator.
* Objectives: every form within the tolerance; Otsu bit-exact.
* One iteration of Algorithm 1 from identical state, at sizes the oracle
  finishes in seconds (several chunks and a ragged tail), at the full
  population 4096 x D = 100 of the scale workload in the same grid launch the
  benchmark times, and at the edge cases (odd D, pf_max 0 and 1, t = T,
  pdr_form 1, np > 1, D = 200, Otsu).  Tolerance |gpu - oracle| <= 1e-4 +
  1e-5 |oracle|; acceptance decisions may differ only at near-ties, at most
  1% of ps.
"""
import json
import os

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


def test_philox_device_matches_oracle(apo, orc, golden_dir):
    import torch
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2 ** 32, (20000, 4), dtype=np.uint64).astype(np.uint32)
    with open(os.path.join(golden_dir, "philox4x32_10_kat.json")) as f:
        kat = json.load(f)
    for v in kat["vectors"]:
        c = np.array([int(x, 16) for x in v["ctr"]], np.uint32)[None]
        k = [int(x, 16) for x in v["key"]]
        dc = torch.tensor(c.view(np.int32), device="cuda")
        do = torch.empty_like(dc)
        apo.apo_philox4x32_10(dc, k[0], k[1], do)
        assert do.cpu().numpy().view(np.uint32)[0].tolist() == [int(x, 16) for x in v["out"]]
    dc = torch.tensor(ctr.view(np.int32), device="cuda")
    do = torch.empty_like(dc)
    apo.apo_philox4x32_10(dc, 12345, 678, do)
    got = do.cpu().numpy().view(np.uint32)
    for i in range(0, 20000, 97):
        assert got[i].tolist() == orc.philox(ctr[i].tolist(), [12345, 678])


SPECS = [
    ("sphere3", lambda: inputs.sphere(3, 0, 10)),
    ("rastrigin10", lambda: inputs.shifted_rotated(inputs.OBJ_RASTRIGIN, 10, 0)),
    ("elliptic100", lambda: inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 100, 1)),
    ("rosenbrock100", lambda: inputs.shifted_rotated(inputs.OBJ_ROSENBROCK, 100, 2)),
    ("rastrigin100", lambda: inputs.shifted_rotated(inputs.OBJ_RASTRIGIN, 100, 3)),
    ("hybrid100", lambda: inputs.shifted_rotated(inputs.OBJ_HYBRID, 100, 4)),
    ("hybrid37", lambda: inputs.shifted_rotated(inputs.OBJ_HYBRID, 37, 5)),
    ("elliptic200", lambda: inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 200, 6)),
    ("composition20", lambda: inputs.composition(D=20, seed=7)),
    ("composition200", lambda: inputs.composition(D=200, seed=8)),
    # the further forms of the paper's Table 2 at the sizes of the fused kernels
    ("bent_cigar50", lambda: inputs.shifted_rotated(inputs.OBJ_BENTCIGAR, 50, 12)),
    ("hgbat100", lambda: inputs.shifted_rotated(inputs.OBJ_HGBAT, 100, 13)),
    ("griewank100", lambda: inputs.shifted_rotated(inputs.OBJ_GRIEWANK, 100, 14)),
    ("griewank7_unrotated", lambda: inputs.ProblemSpec(kind=inputs.OBJ_GRIEWANK, D=7, lb=np.full(7, -100.0),
                                                       ub=np.full(7, 100.0), shift=inputs.shift(7, 15))),
]


@pytest.mark.parametrize("name,mk", SPECS, ids=[s[0] for s in SPECS])
def test_objective_parity(apo, orc, name, mk):
    spec = mk()
    X = inputs.random_state(spec, 77, seed=3)
    # include the shift itself (f(o) = 0 for the zero-at-shift forms)
    if spec.shift is not None and spec.kind in (inputs.OBJ_ELLIPTIC, inputs.OBJ_RASTRIGIN, inputs.OBJ_BENTCIGAR,
                                                inputs.OBJ_HGBAT, inputs.OBJ_GRIEWANK):
        X[0] = spec.shift
    Fg = gpu_eval(apo, apo.problem_from_spec(spec), X)
    Fo = orc.objective(orc.OracleProblem.from_spec(spec), X.astype(np.float64))
    assert np.all(close(Fg, Fo)), (np.max(np.abs(Fg - Fo) / (1e-4 + 1e-5 * np.abs(Fo))))


def test_otsu_objective_bit_exact(apo, orc):
    px = inputs.gmm_image(2, 100_000)
    hist = np.bincount(px, minlength=256)
    for T in (1, 2, 4, 8, 16, 31):
        spec = inputs.otsu_problem(hist, T)
        X = inputs.random_state(spec, 200, seed=T)
        X[0, :] = 0.0
        X[1, :] = 255.0
        Fg = gpu_eval(apo, apo.problem_from_spec(spec), X)
        Fo = orc.objective(orc.OracleProblem.from_spec(spec), X.astype(np.float64))
        np.testing.assert_array_equal(Fg, Fo)


def test_worked_example_clamp_eval_select(apo, golden_dir):
    import torch
    with open(os.path.join(golden_dir, "worked_example.json")) as f:
        ex = json.load(f)
    spec = inputs.sphere(ex["dim"], ex["xmin"], ex["xmax"])
    prob = apo.problem_from_spec(spec)
    X = torch.tensor(ex["step2_sorted_X"], dtype=torch.float32, device="cuda")
    F = (X.double() ** 2).sum(1).float()
    Xn = torch.tensor(ex["step5_Xnew"], dtype=torch.float32, device="cuda")
    Fn = torch.empty(4, dtype=torch.float32, device="cuda")
    apo.apo_clamp_eval_select(prob, X, F, Xn, Fn)
    torch.cuda.synchronize()
    np.testing.assert_allclose(Xn.cpu().numpy(), ex["step6_Xnew_clamped"], atol=1e-6)
    tol = 0.5 * 10 ** -ex["printed_decimals"]
    ftol = tol + 2 * tol * np.abs(np.array(ex["step6_Xnew_clamped"])).sum(1)
    assert np.all(np.abs(Fn.cpu().numpy() - ex["step6_fnew"]) <= ftol)
    np.testing.assert_allclose(X.cpu().numpy(), ex["step6_final_X"], atol=1e-6)


STEP_CASES = [
    # (name, spec factory, ps, t, T, kwargs)
    ("single_rastrigin_t1", lambda: inputs.single_rastrigin(0), 20, 1, 1000, {}),
    ("single_rastrigin_t500", lambda: inputs.single_rastrigin(0), 20, 500, 1000, {}),
    ("sphere_worked_shape", lambda: inputs.sphere(3, 0, 10), 4, 1, 10, {}),
    ("ragged_hybrid37_ps300", lambda: inputs.shifted_rotated(inputs.OBJ_HYBRID, 37, 1), 300, 7, 50, {}),
    ("elliptic100_ps1500_grid", lambda: inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 100, 2), 1500, 3, 2000, {}),
    ("pfmax1_pdr1", lambda: inputs.shifted_rotated(inputs.OBJ_RASTRIGIN, 20, 3), 200, 5, 100,
     dict(pf_max=1.0, pdr_form=1)),
    ("pfmax0", lambda: inputs.shifted_rotated(inputs.OBJ_ROSENBROCK, 20, 3), 200, 5, 100, dict(pf_max=0.0)),
    ("last_iteration", lambda: inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 50, 4), 128, 100, 100, dict(pf_max=0.5)),
    ("np3", lambda: inputs.shifted_rotated(inputs.OBJ_HYBRID, 50, 5), 256, 9, 100, dict(np_=3)),
    ("d200_ps256", lambda: inputs.shifted_rotated(inputs.OBJ_RASTRIGIN, 200, 6), 256, 2, 300, {}),
    ("composition20_ps64", lambda: inputs.composition(D=20, seed=9), 64, 4, 300, {}),
    ("odd_d1", lambda: inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 1, 7), 40, 2, 10, {}),
    # placement of the per-protozoon draws: a call of their own when fewer
    # than three lanes of the last per-dimension call are free (D 64, D 126),
    # a last call with no pair at all (D 150), pair draws past lane 31 (np 16)
    ("d64_own_scalar_call", lambda: inputs.shifted_rotated(inputs.OBJ_RASTRIGIN, 64, 8), 128, 3, 100, {}),
    ("d126_np3_own_scalar_call", lambda: inputs.shifted_rotated(inputs.OBJ_HYBRID, 126, 9), 200, 4, 100,
     dict(np_=3)),
    ("d150_free_last_call", lambda: inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 150, 10), 128, 2, 100, {}),
    ("d100_np16", lambda: inputs.shifted_rotated(inputs.OBJ_RASTRIGIN, 100, 11), 256, 3, 100, dict(np_=16)),
    ("bent_cigar50_ps200", lambda: inputs.shifted_rotated(inputs.OBJ_BENTCIGAR, 50, 16), 200, 3, 100, {}),
    ("hgbat100_ps4096_grid", lambda: inputs.shifted_rotated(inputs.OBJ_HGBAT, 100, 17), 4096, 5, 1000, {}),
    ("griewank30_ps64", lambda: inputs.shifted_rotated(inputs.OBJ_GRIEWANK, 30, 18), 64, 2, 100, {}),
]


@pytest.mark.parametrize("name,mk,ps,t,T,kw", STEP_CASES, ids=[c[0] for c in STEP_CASES])
def test_step_parity(apo, orc, name, mk, ps, t, T, kw):
    r = compare_step(apo, orc, mk(), ps, t, T, **kw)
    assert_step_ok(r)


@pytest.mark.parametrize("form", inputs.SCALE_FORMS)
def test_step_parity_full_scale(apo, orc, form):
    """ps = 4096, D = 100: the full scale workload, in the cooperative grid launch."""
    spec = inputs.shifted_rotated(form, 100, 0, run=form)
    r = compare_step(apo, orc, spec, 4096, 17, 2000, seed=5)
    assert_step_ok(r)


@pytest.mark.parametrize("T", [2, 4, 16])
def test_step_parity_otsu(apo, orc, T):
    px = inputs.gmm_image(T, 200_000)
    spec = inputs.otsu_problem(np.bincount(px, minlength=256), T)
    r = compare_step(apo, orc, spec, 100, 3, 500, exact_f=True)
    assert r["ambiguous"] <= 5, r
    assert_step_ok(r)
