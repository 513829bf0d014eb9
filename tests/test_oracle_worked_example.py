"""Pins the oracle to the worked example the paper prints (Sec. 4.1, steps 1-6).

The example's random draws are not printed, so only its deterministic parts
are pinned: the sphere fitness values (Eq. 14), the sort of Algorithm 1, the
size of Dr_index, the mask sizes of Eq. 5, the bound clamp, the evaluation and
the greedy replacement.
"""
import json
import os

import numpy as np
import pytest

from paper_2510_14982_gb300 import inputs


@pytest.fixture(scope="module")
def ex(golden_dir):
    with open(os.path.join(golden_dir, "worked_example.json")) as f:
        return json.load(f)


@pytest.fixture(scope="module")
def prob(orc, ex):
    spec = inputs.sphere(ex["dim"], ex["xmin"], ex["xmax"])
    return orc.OracleProblem.from_spec(spec)


def test_step1_sphere_fitness(orc, ex, prob):
    F = orc.objective(prob, np.array(ex["step1_X"]))
    np.testing.assert_allclose(F, ex["step1_f"], atol=0.5 * 10 ** -ex["printed_decimals"])


def test_step2_sort_order(orc, ex, prob):
    X = np.array(ex["step1_X"])
    F = orc.objective(prob, X)
    prm = orc.params(ps=ex["ps"], pf_max=ex["pf_max"], max_iter=10, seed=3)
    _, _, info = orc.apo_step(prob, prm, 1, X, F, with_info=True)
    sorted_X = X[info["order"]]
    np.testing.assert_allclose(sorted_X, ex["step2_sorted_X"])
    np.testing.assert_allclose(F[info["order"]], ex["step2_sorted_f"], atol=0.005)


def test_step3_dr_size_is_one_for_every_draw(orc, ex, prob):
    """ceil(ps * pf) with ps = 4 and pf = pf_max * rand <= 0.1 is always 1."""
    X = np.array(ex["step1_X"])
    F = orc.objective(prob, X)
    for seed in range(5):
        prm = orc.params(ps=ex["ps"], pf_max=ex["pf_max"], max_iter=20, seed=seed)
        for t in range(1, 21):
            _, _, info = orc.apo_step(prob, prm, t, X, F, with_info=True)
            assert info["m"] == ex["step3_dr_size"]
            assert info["in_dr"].sum() == ex["step3_dr_size"]


def test_step5_mask_sizes_match_the_example(orc, ex, prob):
    """Eq. 5: ceil(dim * i / ps) with 1-based ranks gives 1 changed coordinate for
    rank 1 and 3 for ranks 3 and 4, as the printed candidates show."""
    old = np.array(ex["step2_sorted_X"])
    new = np.array(ex["step5_Xnew"])
    changed = (np.abs(new - old) > 1e-12).sum(axis=1)
    D, ps = ex["dim"], ex["ps"]
    for rank, mode in enumerate(ex["step4_modes"], start=1):
        if mode in ("autotrophic", "heterotrophic"):
            assert changed[rank - 1] == -(-D * rank // ps)
    # and the oracle's own foraging masks have exactly that many ones
    X = np.array(ex["step1_X"])
    F = orc.objective(prob, X)
    seen = set()
    for seed in range(40):
        prm = orc.params(ps=ps, pf_max=ex["pf_max"], max_iter=50, seed=seed)
        _, _, info = orc.apo_step(prob, prm, 1, X, F, with_info=True)
        for r in range(ps):
            if info["mode"][r] in (orc.MODE_AUTOTROPHIC, orc.MODE_HETEROTROPHIC):
                want = -(-D * (r + 1) // ps)
                assert info["mask_count"][r] == want
                assert info["mask"][r].sum() == want
                seen.add(r)
    assert len(seen) == ps


def test_step6_clamp_eval_select(orc, ex, prob):
    old = np.array(ex["step2_sorted_X"])
    Fold = orc.objective(prob, old)
    Xout, Fout, Xnew_clamped, Fnew = orc.clamp_eval_select(prob, old, Fold, np.array(ex["step5_Xnew"]))
    tol = 0.5 * 10 ** -ex["printed_decimals"]
    np.testing.assert_allclose(Xnew_clamped, ex["step6_Xnew_clamped"], atol=1e-12)
    # the printed candidates are themselves rounded to 2 decimals, so their
    # sphere value carries up to 2 * tol * sum|x| of propagated rounding, plus
    # the rounding of the printed fitness
    ftol = tol + 2 * tol * np.abs(Xnew_clamped).sum(axis=1)
    assert np.all(np.abs(Fnew - np.array(ex["step6_fnew"])) <= ftol)
    np.testing.assert_allclose(Xout, ex["step6_final_X"], atol=1e-12)
