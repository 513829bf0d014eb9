"""The oracle's surrogate-assisted candidates (TEST INFRASTRUCTURE pins).

Candidate c of rank r draws from the plain method's Philox slots | (c << 8);
candidate 0 is therefore the plain method's own candidate, and every candidate
obeys the same structural rules as the plain one: the iteration's Dr_index set
(Eq. 11) is shared, a foraging candidate changes at most ceil(D i / ps)
coordinates (Eq. 5), every candidate lies in the box (clamp), and candidates
c >= 1 are new draws (they differ from candidate 0)."""
import numpy as np
import pytest

from paper_2510_14982_gb300 import inputs


@pytest.fixture(scope="module")
def case(orc):
    spec = inputs.scale_forms(0, 20)[2]          # Rastrigin, D 20
    prob = orc.OracleProblem.from_spec(spec)
    prm = orc.params(48, 1, 0.1, 50, 11)
    X, F = orc.init_population(prob, prm)
    return prob, prm, X, F


def test_candidate_zero_is_the_plain_candidate(orc, case):
    prob, prm, X, F = case
    for t in (1, 17, 50):
        Xc, order = orc.candidates(prob, prm, t, 4, X, F)
        _, _, info = orc.apo_step(prob, prm, t, X, F, with_info=True)
        assert np.array_equal(order, info["order"])
        assert np.array_equal(Xc[:, 0, :], info["xnew"])


def test_candidates_follow_the_plain_rules(orc, case):
    prob, prm, X, F = case
    ps, D = prm.ps, prob.D
    lb, ub = np.full(D, -100.0), np.full(D, 100.0)
    t = 9
    Xc, order = orc.candidates(prob, prm, t, 6, X, F)
    _, _, info = orc.apo_step(prob, prm, t, X, F, with_info=True)
    Xs = X[order]
    assert np.all(Xc >= lb) and np.all(Xc <= ub)
    for r in range(ps):
        if info["in_dr"][r]:
            continue                                  # dormancy / reproduction rows
        kf = (D * (r + 1) + ps - 1) // ps             # ceil(D i / ps), i = r + 1
        for c in range(6):
            assert np.count_nonzero(Xc[r, c] != Xs[r]) <= kf
    # candidates c >= 1 are fresh draws, not copies of candidate 0
    moved = [not np.array_equal(Xc[r, c], Xc[r, 0]) for r in range(ps) for c in range(1, 6)]
    assert np.mean(moved) > 0.9
