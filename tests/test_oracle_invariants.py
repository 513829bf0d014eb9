"""Invariants and special cases of the oracle's APO step and run (Eq. 1-13,
Algorithm 1).  These pin behaviour the paper fixes without printing numbers:
bounds, the monotone best, |Dr| = ceil(ps pf), the mask sizes, unmasked
coordinates unchanged, strict-improvement acceptance, the sort being a
permutation, and the mode probabilities of Eq. 12-13."""
import numpy as np
import pytest

from paper_2510_14982_gb300 import inputs


def _setup(orc, kind=inputs.OBJ_RASTRIGIN, D=7, ps=24, seed=0, T=50, pf_max=0.1, np_=1, pdr_form=0):
    spec = inputs.shifted_rotated(kind, D, seed=seed)
    p = orc.OracleProblem.from_spec(spec)
    prm = orc.params(ps=ps, np_=np_, pf_max=pf_max, max_iter=T, seed=seed, pdr_form=pdr_form)
    X, F = orc.init_population(p, prm)
    return spec, p, prm, X, F


def test_init_inside_bounds_and_evaluated(orc):
    spec, p, prm, X, F = _setup(orc)
    assert (X >= spec.lb).all() and (X <= spec.ub).all()
    np.testing.assert_allclose(F, orc.objective(p, X))


@pytest.mark.parametrize("np_", [1, 3])
def test_step_invariants(orc, np_):
    spec, p, prm, X, F = _setup(orc, np_=np_, ps=30, D=9, pf_max=0.5)
    D, ps = spec.D, prm.ps
    for t in range(1, prm.max_iter + 1):
        Xo, Fo, info = orc.apo_step(p, prm, t, X, F, with_info=True)
        order = info["order"]
        # the sort is a permutation and orders the old fitness (stable)
        assert sorted(order.tolist()) == list(range(ps))
        Fs = F[order]
        assert np.all(np.diff(Fs) >= 0)
        Xs = X[order]
        # |Dr| = ceil(ps * pf), pf <= pf_max
        m = info["m"]
        assert 1 <= m <= int(np.ceil(ps * prm.pf_max))
        assert info["in_dr"].sum() == m
        modes = info["mode"]
        assert np.all(np.isin(modes[info["in_dr"] == 1], [0, 1]))
        assert np.all(np.isin(modes[info["in_dr"] == 0], [2, 3]))
        for r in range(ps):
            mk = info["mask"][r].astype(bool)
            if modes[r] == 0:
                continue
            k = info["mask_count"][r]
            assert mk.sum() == k
            if modes[r] in (2, 3):
                assert k == -(-D * (r + 1) // ps)
            else:
                assert 1 <= k <= D
            # unmasked coordinates are unchanged before the clamp
            np.testing.assert_array_equal(info["xnew_raw"][r][~mk], Xs[r][~mk])
        # clamp
        assert (info["xnew"] >= spec.lb).all() and (info["xnew"] <= spec.ub).all()
        np.testing.assert_array_equal(info["xnew"], np.clip(info["xnew_raw"], spec.lb, spec.ub))
        # strict-improvement acceptance
        acc = info["accepted"].astype(bool)
        assert np.all(info["fnew"][acc] < Fs[acc])
        assert np.all(info["fnew"][~acc] >= Fs[~acc])
        np.testing.assert_array_equal(Xo[acc], info["xnew"][acc])
        np.testing.assert_array_equal(Xo[~acc], Xs[~acc])
        assert np.all(Fo <= Fs)
        X, F = Xo, Fo


def test_run_curve_monotone_and_best_consistent(orc):
    spec, p, prm, _, _ = _setup(orc, T=120)
    bx, bf, curve = orc.apo_run(p, prm)
    assert np.all(np.diff(curve) <= 0)
    assert curve[-1] == bf
    assert orc.objective(p, bx)[0] == pytest.approx(bf, rel=1e-12)
    assert (bx >= spec.lb).all() and (bx <= spec.ub).all()
    assert bf < curve[0]


def test_no_dr_when_pf_max_is_zero(orc):
    spec, p, prm, X, F = _setup(orc, pf_max=0.0)
    for t in (1, 5, 17):
        _, _, info = orc.apo_step(p, prm, t, X, F, with_info=True)
        assert info["m"] == 0 and info["in_dr"].sum() == 0


def test_last_iteration_foraging_is_identity(orc):
    """At t = T, f = rand (1 + cos(pi)) = 0 (Eq. 4): foraging leaves X unchanged."""
    spec, p, prm, X, F = _setup(orc, pf_max=0.3)
    _, _, info = orc.apo_step(p, prm, prm.max_iter, X, F, with_info=True)
    Xs = X[info["order"]]
    forage = info["mode"] >= 2
    assert forage.any()
    np.testing.assert_array_equal(info["xnew_raw"][forage], Xs[forage])


def test_identical_population_autotrophic_is_identity_heterotrophic_scales(orc):
    """With every protozoon equal, the autotrophic update (Eq. 6) only sees zero
    differences, and the heterotrophic one (Eq. 8-9) reduces to
    X (1 + f s Rand (1 - t/T)) on the mask: one sign per protozoon and a
    magnitude of at most (1 + cos(pi t / T)) (1 - t / T)."""
    spec = inputs.sphere(6, 1.0, 10.0)
    p = orc.OracleProblem.from_spec(spec)
    ps, T = 40, 10
    X = np.full((ps, 6), 5.0)
    F = orc.objective(p, X)
    seen_h = 0
    for t in (2, 3, 4, 6):
        prm = orc.params(ps=ps, pf_max=0.0, max_iter=T, seed=t)
        _, _, info = orc.apo_step(p, prm, t, X, F, with_info=True)
        bound = (1 + np.cos(np.pi * t / T)) * (1 - t / T)
        for r in range(ps):
            raw = info["xnew_raw"][r]
            if info["mode"][r] == 2:
                np.testing.assert_array_equal(raw, X[0])
            else:
                mk = info["mask"][r].astype(bool)
                rel = raw[mk] / 5.0 - 1.0
                assert np.all(np.abs(rel) <= bound + 1e-12)
                assert np.all(rel >= 0) or np.all(rel <= 0)
                seen_h += 1
    assert seen_h > 0


def test_dormancy_ignores_the_old_position(orc):
    spec, p, prm, X, F = _setup(orc, pf_max=1.0, ps=40)
    X2 = X[::-1].copy()   # a different population with the same fitness ranks reversed
    F2 = orc.objective(p, X2)
    _, _, a = orc.apo_step(p, prm, 3, X, F, with_info=True)
    _, _, b = orc.apo_step(p, prm, 3, X2, F2, with_info=True)
    for r in range(prm.ps):
        if a["mode"][r] == 0 and b["mode"][r] == 0:
            np.testing.assert_array_equal(a["xnew_raw"][r], b["xnew_raw"][r])
            assert (a["xnew_raw"][r] >= spec.lb).all() and (a["xnew_raw"][r] <= spec.ub).all()


@pytest.mark.parametrize("form", [0, 1])
def test_dormancy_probability_follows_eq13(orc, form):
    """Among Dr members, dormancy happens with probability p_dr(i) (Eq. 13)."""
    ps, T = 16, 400
    spec, p, prm, X, F = _setup(orc, ps=ps, D=3, pf_max=1.0, T=T, pdr_form=form)
    dorm = np.zeros(ps)
    cnt = np.zeros(ps)
    for t in range(1, T + 1):
        _, _, info = orc.apo_step(p, prm, t, X, F, with_info=True)
        inr = info["in_dr"] == 1
        cnt[inr] += 1
        dorm[inr & (info["mode"] == 0)] += 1
    i = np.arange(1, ps + 1)
    c = np.cos((1 - i / ps) * np.pi)
    pdr = 0.5 * (1 - c) if form == 0 else 0.5 * (1 + c)
    freq = dorm / np.maximum(cnt, 1)
    sd = np.sqrt(pdr * (1 - pdr) / np.maximum(cnt, 1)) + 1e-3
    assert np.all(np.abs(freq - pdr) <= 5 * sd + 0.02)


def test_autotrophic_probability_follows_eq12(orc):
    ps, T = 64, 8
    for t in (1, 2, 4, 6, 8):
        auto = tot = 0
        for seed in range(12):
            spec, p, prm, X, F = _setup(orc, ps=ps, D=3, pf_max=0.0, T=T, seed=seed)
            _, _, info = orc.apo_step(p, prm, t, X, F, with_info=True)
            auto += int((info["mode"] == 2).sum())
            tot += ps
        pah = 0.5 * (1 + np.cos(np.pi * t / T))
        sd = np.sqrt(max(pah * (1 - pah), 1e-4) / tot)
        assert abs(auto / tot - pah) <= 5 * sd + 0.01


def test_masks_and_dr_are_uniform_subsets(orc):
    """randperm: every index is drawn with probability k / n."""
    D, ps, T = 8, 16, 300
    spec, p, prm, X, F = _setup(orc, ps=ps, D=D, pf_max=0.5, T=T)
    hits = np.zeros(D)
    expect = np.zeros(D)
    dr_hits = np.zeros(ps)
    dr_expect = np.zeros(ps)
    for t in range(1, T + 1):
        _, _, info = orc.apo_step(p, prm, t, X, F, with_info=True)
        r = ps - 1   # last rank: foraging mask of size ceil(D * ps / ps) = D? use a middle rank
        for r in range(ps):
            if info["mode"][r] >= 2 and info["mask_count"][r] < D:
                hits += info["mask"][r]
                expect += info["mask_count"][r] / D
        dr_hits += info["in_dr"]
        dr_expect += info["m"] / ps
    assert np.all(np.abs(hits - expect) <= 5 * np.sqrt(expect) + 5)
    assert np.all(np.abs(dr_hits - dr_expect) <= 5 * np.sqrt(dr_expect) + 5)


def test_apo_minimises_the_sphere(orc):
    spec = inputs.sphere(5, -10.0, 10.0)
    p = orc.OracleProblem.from_spec(spec)
    prm = orc.params(ps=30, pf_max=0.1, max_iter=300, seed=1)
    _, bf, curve = orc.apo_run(p, prm)
    assert bf < 1e-3 * curve[0]


def test_autotrophic_partners_are_independent_uniform_ranks(orc):
    """Reading R2: in the autotrophic mode (Eq. 6-7) j and the pair k-, k+ are
    independent uniform ranks over the whole population.  With rows X_r = e_r
    (D = ps), equal fitness (w = exp(-1) for every pair, Eq. 7) and every
    dimension of the last-ranked protozoon masked (ceil(D ps / ps) = D, Eq. 5),
    its candidate minus X_i is f (e_j - e_i) + f w (e_a - e_b), so j, a, b can be
    read off.  Over many seeds they must be uniform and independent (a mistake
    such as taking rank neighbours, or one draw for two of them, fails)."""
    chi2 = pytest.importorskip("scipy.stats").chi2
    ps = D = 32
    prob = orc.OracleProblem(inputs.OBJ_SPHERE, D, -10.0, 10.0)
    X = np.eye(ps)
    F = np.ones(ps)
    w = np.exp(-1.0)
    i = ps - 1
    js, as_, bs = [], [], []
    n_two_f = n_two_fw = 0
    N = 3000
    for seed in range(N):
        prm = orc.params(ps, 1, 0.0, 100000, seed)
        _, _, info = orc.apo_step(prob, prm, 1, X, F, with_info=True)
        assert np.array_equal(info["order"], np.arange(ps))
        assert info["mode"][i] == 2 and info["mask"][i].all()
        delta = info["xnew_raw"][i] - X[i]
        nz = np.flatnonzero(np.abs(delta) > 1e-12)
        f = -delta[i]
        if len(nz) == 4 and f > 0:
            rest = [d for d in nz if d != i]
            vals = {d: delta[d] / f for d in rest}
            j = [d for d in rest if abs(vals[d] - 1.0) < 1e-9]
            a = [d for d in rest if abs(vals[d] - w) < 1e-9]
            b = [d for d in rest if abs(vals[d] + w) < 1e-9]
            assert len(j) == len(a) == len(b) == 1, (seed, vals)
            js.append(j[0]); as_.append(a[0]); bs.append(b[0])
        elif len(nz) == 2:
            ratio = delta[nz].max() / -delta[nz].min()
            assert abs(ratio - 1.0) < 1e-9, (seed, delta[nz])
            if i in nz:
                n_two_f += 1      # a == b: only f (e_j - e_i) remains
            else:
                n_two_fw += 1     # j == i: only f w (e_a - e_b) remains
    clean = len(js)
    # all four distinct with probability (31/32)(30/32)(29/32)
    assert abs(clean / N - 31 * 30 * 29 / 32 ** 3) < 0.03, clean
    # a == b and j == i each happen with probability about 1/ps
    for n in (n_two_f, n_two_fw):
        assert 0.5 * N / ps < n < 1.6 * N / ps, (n_two_f, n_two_fw)
    # in the clean samples each of j, a, b is uniform over the 31 ranks other than i
    crit = chi2.ppf(1.0 - 1e-6, ps - 2)
    for v in (js, as_, bs):
        counts = np.bincount(v, minlength=ps)[:ps - 1]
        expected = clean / (ps - 1)
        assert ((counts - expected) ** 2 / expected).sum() < crit
    # and j, a are independent: (j mod 4, a mod 4) over 16 cells, up to the
    # small dependence that distinctness induces (same-cell pairs are 1/30 rarer)
    cells = np.zeros((4, 4))
    for j, a in zip(js, as_):
        cells[j % 4, a % 4] += 1
    expected = np.outer(cells.sum(1), cells.sum(0)) / clean
    assert ((cells - expected) ** 2 / expected).sum() < chi2.ppf(1.0 - 1e-6, 9)


def test_heterotrophic_neighbours_clamp_at_the_last_rank(orc):
    """Reading R3: X_{i-k}, X_{i+k} (Eq. 8, 10) clamp to ranks 1..ps.  With rows
    X_r = e_r (D = ps), equal fitness and the last rank fully masked (Eq. 5),
    its heterotrophic candidate minus X_i is f (x_near - x_i) + f w (e_{ps-2} -
    e_{ps-1}): x_near (Eq. 9) moves only dimension ps-1, and the clamped k+ is
    the protozoon itself.  So only dimensions ps-2 and ps-1 change, dimension
    ps-2 by +f w.  Wrapping k+ around to rank 1 would move dimension 0;
    reflecting it to rank ps-1 would cancel the e_{ps-2} term."""
    ps = D = 16
    prob = orc.OracleProblem(inputs.OBJ_SPHERE, D, -10.0, 10.0)
    X = np.eye(ps)
    F = np.ones(ps)
    i = ps - 1
    seen = 0
    for seed in range(200):
        # t = T - 1: heterotrophic with probability 1 - p_ah(t) close to 1 (Eq. 12),
        # and the foraging factor f (Eq. 4) is small but not zero
        prm = orc.params(ps, 1, 0.0, 100, seed)
        _, _, info = orc.apo_step(prob, prm, 99, X, F, with_info=True)
        if info["mode"][i] != 3:
            continue
        seen += 1
        assert info["mask"][i].all()
        delta = info["xnew_raw"][i] - X[i]
        assert np.all(delta[:ps - 2] == 0.0), (seed, delta)
        assert delta[ps - 2] > 0.0, (seed, delta)
    assert seen > 150
