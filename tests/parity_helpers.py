"""Shared helpers of the GPU parity tests: the tolerance, the near-tie rule,
and side-by-side calls of the CUDA path (through the C ABI) and the oracle."""
import numpy as np

# Tolerance of one iteration from identical state: |gpu - oracle| <= ATOL + RTOL |oracle|
# (positions and fitness), element-wise.
ATOL, RTOL = 1e-4, 1e-5


def close(g, o):
    g = np.asarray(g, np.float64)
    o = np.asarray(o, np.float64)
    return np.abs(g - o) <= ATOL + RTOL * np.abs(o)


def tol(o):
    return ATOL + RTOL * np.abs(np.asarray(o, np.float64))


def gpu_step(apo, prob, prm, t, X32, F):
    import torch
    dX = torch.tensor(X32, dtype=torch.float32, device="cuda")
    dF = torch.tensor(F, dtype=prob.fit_dtype, device="cuda")
    apo.apo_step(prob, prm, t, dX, dF)
    torch.cuda.synchronize()
    return dX.cpu().numpy(), dF.cpu().numpy()


def gpu_eval(apo, prob, X32):
    import torch
    dX = torch.tensor(np.asarray(X32, np.float32), device="cuda")
    dF = torch.empty(dX.shape[0], dtype=prob.fit_dtype, device="cuda")
    apo.apo_evaluate(prob, dX, dF)
    torch.cuda.synchronize()
    return dF.cpu().numpy()


def compare_step(apo, orc, spec, ps, t, T, seed=0, np_=1, pf_max=0.1, pdr_form=0, state_seed=1,
                 max_flip_frac=0.01, exact_f=False, pair_policy=0):
    """One iteration from the same float32 state on both sides; returns a dict of
    counts.  Rows whose acceptance decision differs must be near-ties
    (|f_new - f_old| within tolerance); they are compared on the branch the GPU
    took and counted."""
    gprob = apo.problem_from_spec(spec)
    oprob = orc.OracleProblem.from_spec(spec)
    X32 = _state(spec, ps, state_seed)
    F = orc.objective(oprob, X32.astype(np.float64))
    if spec.kind != 6:
        F = F.astype(np.float32)
    gprm = apo.apo_params_make(ps, np_, pf_max, T, seed, 0, pdr_form, pair_policy)
    oprm = orc.params(ps, np_, pf_max, T, seed, 0, pdr_form, pair_policy)
    Xg, Fg = gpu_step(apo, gprob, gprm, t, X32, F)
    Xo, Fo, info = orc.apo_step(oprob, oprm, t, X32.astype(np.float64), np.asarray(F, np.float64),
                                with_info=True)
    Xs = X32.astype(np.float64)[info["order"]]
    Fs = np.asarray(F, np.float64)[info["order"]]
    acc_o = info["accepted"].astype(bool)
    # the GPU accepted iff its fitness changed (acceptance needs a strict decrease)
    Fs_stored = np.asarray(F)[info["order"]]
    took_new = Fg != Fs_stored
    # a candidate identical to the old position (e.g. foraging at t = T) is a
    # tie whatever the decision: it changes no position
    same = np.all(info["xnew"] == Xs.astype(np.float32).astype(np.float64), axis=1)
    flips = (took_new != acc_o) & ~same
    near = np.abs(info["fnew"] - Fs) <= tol(Fs) + tol(info["fnew"])
    bad_flip = flips & ~near
    # compare on the GPU's branch
    want_X = np.where(took_new[:, None], info["xnew"], Xs)
    want_F = np.where(took_new, info["fnew"], Fs)
    ok_x = close(Xg, want_X)
    ok_f = close(Fg, want_F)
    amb = np.zeros(ps, bool)
    if exact_f:
        # Otsu: thresholds are floor() of float32 positions, so a candidate
        # coordinate within rounding of an integer may land in either bin; those
        # rows are ambiguous.  Every other row must match bit for bit.
        raw = info["xnew"]
        dist = np.abs(raw - np.rint(raw))
        amb = np.any((dist > 0) & (dist < 1e-4), axis=1)
        ok_f = (Fg == want_F) | amb
        ok_x = ok_x | amb[:, None]
        bad_flip = bad_flip & ~amb
        flips = flips & ~amb
    return dict(ps=ps, flips=int(flips.sum()), bad_flips=int(bad_flip.sum()), ambiguous=int(amb.sum()),
                bad_x=int((~ok_x).sum()), bad_f=int((~ok_f).sum()),
                max_flip=int(np.ceil(max_flip_frac * ps)), accepted=int(acc_o.sum()),
                modes=np.bincount(info["mode"], minlength=4), m=info["m"],
                worst_x=float(np.max(np.abs(Xg - want_X) / tol(want_X))),
                worst_f=float(np.max(np.abs(Fg - want_F) / tol(want_F))))


def _state(spec, ps, seed):
    from paper_2510_14982_gb300 import inputs
    return inputs.random_state(spec, ps, seed)


def assert_step_ok(r):
    assert r["bad_flips"] == 0, r
    assert r["flips"] <= r["max_flip"], r
    assert r["bad_x"] == 0, r
    assert r["bad_f"] == 0, r
