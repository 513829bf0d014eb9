"""Oracle pins of the two variant switches and of the evaluation budget
(TEST INFRASTRUCTURE).

* Pair policy 1, the alternative reading of Eq. 6-7 (k- among the ranks at
  least as good as i, k+ among the ranks at most as good): read off
  unit-vector populations, k- is uniform over 1..i and k+ over i..ps; policy 0
  keeps the reading R2 (uniform over all ranks), which its own test pins.
* The evaluation budget (MaxFEs counted in objective evaluations): ps at
  initialisation and ps per iteration, so floor(max_fes / ps) - 1 whole
  iterations, which also set iter_max of Eq. 4, 9 and 12; the run equals the
  run with that max_iter.
"""
import numpy as np
import pytest

from paper_2510_14982_gb300 import inputs


def test_pair_policy_one_draws_better_and_worse_ranks(orc):
    """With rows X_q = e_q, X_i = 0, equal fitness (w = e^-1, Eq. 7) and a mask
    of half the dimensions, the autotrophic candidate is f e_j + f w (e_a - e_b)
    on the mask.  Over many seeds a (k-) lies in ranks 0..r and b (k+) in
    r..ps-1, each uniform there (chi-square), while policy 0 reaches beyond."""
    chi2 = pytest.importorskip("scipy.stats").chi2
    ps = D = 32
    r = 15                                     # i = 16: mask ceil(D i / ps) = 16 dimensions
    prob = orc.OracleProblem(inputs.OBJ_SPHERE, D, -10.0, 10.0)
    X = np.eye(ps)
    X[r] = 0.0
    F = np.ones(ps)
    w = np.exp(-1.0)
    got = {0: ([], []), 1: ([], [])}
    for policy in (0, 1):
        for seed in range(3000):
            prm = orc.params(ps, 1, 0.0, 1000, seed, 0, 0, policy)
            _, _, info = orc.apo_step(prob, prm, 1, X, F, with_info=True)
            if info["mode"][r] != 2:
                continue
            delta = info["xnew_raw"][r]
            f = delta.max()
            if f <= 0:
                continue
            ratio = delta / f
            a = np.flatnonzero(np.abs(ratio - w) < 1e-9)
            b = np.flatnonzero(np.abs(ratio + w) < 1e-9)
            j = np.flatnonzero(np.abs(ratio - 1.0) < 1e-9)
            if len(a) == 1 and len(j) == 1:
                got[policy][0].append(int(a[0]))
            if len(b) == 1 and len(j) == 1:
                got[policy][1].append(int(b[0]))
    a1, b1 = map(np.asarray, got[1])
    assert len(a1) > 300 and len(b1) > 300
    assert np.all(a1 <= r) and np.all(b1 >= r)
    # uniform over the ranks 0..r-1 (rank r itself has the zero row: invisible)
    ca = np.bincount(a1, minlength=r)[:r]
    cb = np.bincount(b1 - (r + 1), minlength=ps - r - 1)[:ps - r - 1]
    for c in (ca, cb):
        e = c.sum() / len(c)
        assert ((c - e) ** 2 / e).sum() < chi2.ppf(1 - 1e-6, len(c) - 1)
    a0, b0 = map(np.asarray, got[0])
    assert np.any(a0 > r) and np.any(b0 < r)    # policy 0 is not restricted


@pytest.mark.parametrize("ps,max_fes,T", [(20, 20 * 51, 50), (20, 20 * 51 + 19, 50), (7, 15, 1), (64, 6400, 99)])
def test_budget_counts_whole_iterations(orc, ps, max_fes, T):
    assert orc.iterations(orc.params(ps, 1, 0.1, 5, 0, 0, 0, 0, max_fes)) == T


def test_budget_too_small_is_rejected(orc):
    assert orc.iterations(orc.params(20, 1, 0.1, 5, 0, 0, 0, 0, 39)) == -1
    spec = inputs.single_rastrigin(0)
    with pytest.raises(ValueError):
        orc.apo_run(orc.OracleProblem.from_spec(spec), orc.params(20, 1, 0.1, 5, 0, 0, 0, 0, 39))


def test_budget_run_equals_the_run_of_that_many_iterations(orc):
    spec = inputs.single_rastrigin(0)
    p = orc.OracleProblem.from_spec(spec)
    bx1, bf1, c1 = orc.apo_run(p, orc.params(20, 1, 0.1, 1, 4, 0, 0, 0, 20 * 61 + 7))
    bx2, bf2, c2 = orc.apo_run(p, orc.params(20, 1, 0.1, 60, 4))
    assert len(c1) == 61
    assert bf1 == bf2 and np.array_equal(bx1, bx2) and np.array_equal(c1, c2)
