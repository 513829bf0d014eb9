"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle checks.

This module only draws problem data (shifts, rotations, permutations,
composition parameters, run sizes, Gaussian-mixture images); it holds none of
the optimiser's arithmetic.  Random numbers come from numpy's PCG64 streams
keyed by (seed, stream id), so every input is reproducible.

Workloads (the paper's CEC2022 data and its photograph are not available, so
these synthetic stand-ins of the same shapes replace them):
  * ``single_rastrigin``   D=10 cosine-sum form, o ~ U[-80,80]^D, M = Q of QR(N(0,1)).
  * ``scale_forms``        D=100: ill-conditioned elliptic, chained Rosenbrock,
                           cosine-sum, and a 30/30/40 hybrid over a seeded permutation.
  * ``batched_runs``       1024 runs with ps ~ U{20..512}, D in {10,20,50}, form ~ U{4 forms}.
  * ``gmm_images``         8-bit images from a K in [3,8] Gaussian mixture
                           (means U[20,235], sigma U[5,30], weights U[0.5,1.5]).
  * ``composition``        10 shifted-rotated components, sigma ~ U[10,50], bias 100 k.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Optional

import numpy as np

(OBJ_SPHERE, OBJ_ELLIPTIC, OBJ_ROSENBROCK, OBJ_RASTRIGIN, OBJ_HYBRID, OBJ_COMPOSITION, OBJ_OTSU,
 OBJ_BENTCIGAR, OBJ_HGBAT, OBJ_GRIEWANK) = range(10)
FORM_NAMES = {OBJ_SPHERE: "sphere", OBJ_ELLIPTIC: "elliptic", OBJ_ROSENBROCK: "rosenbrock",
              OBJ_RASTRIGIN: "rastrigin", OBJ_HYBRID: "hybrid", OBJ_COMPOSITION: "composition",
              OBJ_OTSU: "otsu", OBJ_BENTCIGAR: "bent_cigar", OBJ_HGBAT: "hgbat", OBJ_GRIEWANK: "griewank"}

# stream ids keep unrelated draws independent of one another
_S_SHIFT, _S_ROT, _S_PERM, _S_COMP, _S_SIZES, _S_IMAGE, _S_STATE = range(1, 8)


def _rng(seed: int, run: int, stream: int) -> np.random.Generator:
    return np.random.default_rng(np.random.SeedSequence([int(seed) & 0xFFFFFFFF,
                                                         int(run) & 0xFFFFFFFF, stream]))


@dataclass
class ProblemSpec:
    kind: int
    D: int
    lb: np.ndarray
    ub: np.ndarray
    shift: Optional[np.ndarray] = None      # float32 [D] or [n_comp, D]
    rot: Optional[np.ndarray] = None        # float32 [D, D] or [n_comp, D, D]
    perm: Optional[np.ndarray] = None       # int32 [D] or [n_comp, D]
    comp_sigma: Optional[np.ndarray] = None  # float64 [n_comp]
    comp_bias: Optional[np.ndarray] = None   # float64 [n_comp]
    hist: Optional[np.ndarray] = None        # int64/int32 [256]
    name: str = ""
    meta: dict = field(default_factory=dict)


def rotation(D: int, seed: int, run: int = 0, comp: int = 0) -> np.ndarray:
    """Q factor of the QR factorisation of a seeded N(0,1) D x D matrix.

    Householder QR in FP64 (LAPACK via numpy); columns are sign-fixed so that
    diag(R) > 0, which makes Q unique.  Returned as float32 (both the oracle
    and the GPU consume this same float32 matrix)."""
    g = _rng(seed, run, _S_ROT * 1000 + comp)
    A = g.standard_normal((D, D))
    Q, R = np.linalg.qr(A)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    Q = Q * s[None, :]
    return Q.astype(np.float32)


def shift(D: int, seed: int, run: int = 0, comp: int = 0, lo=-80.0, hi=80.0) -> np.ndarray:
    return _rng(seed, run, _S_SHIFT * 1000 + comp).uniform(lo, hi, D).astype(np.float32)


def permutation(D: int, seed: int, run: int = 0, comp: int = 0) -> np.ndarray:
    return _rng(seed, run, _S_PERM * 1000 + comp).permutation(D).astype(np.int32)


def shifted_rotated(kind: int, D: int, seed: int, run: int = 0, lb=-100.0, ub=100.0) -> ProblemSpec:
    """One of the basic seeded forms (elliptic, Rosenbrock, Rastrigin, hybrid)."""
    perm = permutation(D, seed, run) if kind == OBJ_HYBRID else None
    return ProblemSpec(kind=kind, D=D, lb=np.full(D, lb), ub=np.full(D, ub),
                       shift=shift(D, seed, run), rot=rotation(D, seed, run), perm=perm,
                       name=FORM_NAMES[kind])


# The five forms of the paper's Table 2 (D = 1000): Bent Cigar, the
# high-conditioned elliptic, HGBat, Rosenbrock and Griewank, each shifted and
# rotated with its own seeded o and M.
TABLE2_FORMS = (OBJ_BENTCIGAR, OBJ_ELLIPTIC, OBJ_HGBAT, OBJ_ROSENBROCK, OBJ_GRIEWANK)


def table2_forms(seed: int = 0, D: int = 1000):
    return [shifted_rotated(k, D, seed, run=k) for k in TABLE2_FORMS]


def sphere(D: int, lb=0.0, ub=10.0) -> ProblemSpec:
    return ProblemSpec(kind=OBJ_SPHERE, D=D, lb=np.full(D, float(lb)), ub=np.full(D, float(ub)),
                       name="sphere")


def single_rastrigin(seed: int = 0) -> ProblemSpec:
    """Single run, D = 10 cosine-sum form on [-100, 100]."""
    return shifted_rotated(OBJ_RASTRIGIN, 10, seed)


SCALE_FORMS = (OBJ_ELLIPTIC, OBJ_ROSENBROCK, OBJ_RASTRIGIN, OBJ_HYBRID)


def scale_forms(seed: int = 0, D: int = 100):
    """The four D = 100 shifted-rotated forms used at population 4096."""
    return [shifted_rotated(k, D, seed, run=k) for k in SCALE_FORMS]


def composition(D: int = 200, seed: int = 0, run: int = 0, n_comp: int = 10,
                lb=-100.0, ub=100.0) -> ProblemSpec:
    """n_comp shifted-rotated components; component k uses form 1 + (k mod 4)."""
    g = _rng(seed, run, _S_COMP)
    shifts = np.stack([shift(D, seed, run, comp=k) for k in range(n_comp)])
    rots = np.stack([rotation(D, seed, run, comp=k) for k in range(n_comp)])
    perms = np.stack([permutation(D, seed, run, comp=k) for k in range(n_comp)])
    sigma = g.uniform(10.0, 50.0, n_comp)
    bias = 100.0 * np.arange(n_comp, dtype=np.float64)
    return ProblemSpec(kind=OBJ_COMPOSITION, D=D, lb=np.full(D, lb), ub=np.full(D, ub),
                       shift=shifts, rot=rots, perm=perms, comp_sigma=sigma, comp_bias=bias,
                       name="composition")


def batched_runs(n_runs: int = 1024, seed: int = 0, ps_lo=20, ps_hi=512, dims=(10, 20, 50)):
    """Per-run sizes and forms of the batched workload: list of (ProblemSpec, ps)."""
    g = _rng(seed, 0, _S_SIZES)
    ps = g.integers(ps_lo, ps_hi + 1, n_runs)
    Ds = g.choice(np.asarray(dims), n_runs)
    forms = g.choice(np.asarray(SCALE_FORMS), n_runs)
    out = []
    for r in range(n_runs):
        spec = shifted_rotated(int(forms[r]), int(Ds[r]), seed, run=r)
        out.append((spec, int(ps[r])))
    return out


def gmm_image_params(image_id: int, seed: int = 0):
    g = _rng(seed, image_id, _S_IMAGE)
    K = int(g.integers(3, 9))
    means = g.uniform(20.0, 235.0, K)
    sig = g.uniform(5.0, 30.0, K)
    w = g.uniform(0.5, 1.5, K)
    return means, sig, w / w.sum()


def gmm_image(image_id: int, n_pixels: int, seed: int = 0) -> np.ndarray:
    """uint8 pixels of one Gaussian-mixture image (numpy; for small images)."""
    means, sig, w = gmm_image_params(image_id, seed)
    g = _rng(seed, image_id, _S_IMAGE * 1000 + 1)
    comp = g.choice(len(w), size=n_pixels, p=w)
    v = np.rint(g.standard_normal(n_pixels) * sig[comp] + means[comp])
    return np.clip(v, 0, 255).astype(np.uint8)


def gmm_images_torch(n_images: int, side: int, seed: int = 0, device="cuda"):
    """[n_images, side*side] uint8 images drawn with torch's device RNG (large inputs)."""
    import torch
    n = side * side
    out = torch.empty((n_images, n), dtype=torch.uint8, device=device)
    gen = torch.Generator(device=device)
    for i in range(n_images):
        means, sig, w = gmm_image_params(i, seed)
        gen.manual_seed((int(seed) * 1_000_003 + i) & 0x7FFFFFFF)
        comp = torch.multinomial(torch.tensor(w, device=device, dtype=torch.float32), n,
                                 replacement=True, generator=gen)
        mu = torch.tensor(means, device=device, dtype=torch.float32)[comp]
        sd = torch.tensor(sig, device=device, dtype=torch.float32)[comp]
        v = torch.randn(n, device=device, generator=gen) * sd + mu
        out[i] = torch.clamp(torch.round(v), 0, 255).to(torch.uint8)
    return out


def otsu_problem(hist, T: int) -> ProblemSpec:
    return ProblemSpec(kind=OBJ_OTSU, D=int(T), lb=np.zeros(T), ub=np.full(T, 255.0),
                       hist=np.asarray(hist, np.int64), name="otsu")


def random_state(spec: ProblemSpec, ps: int, seed: int = 0):
    """A seeded float32 population inside the bounds (for single-step parity)."""
    g = _rng(seed, 0, _S_STATE)
    lb, ub = np.asarray(spec.lb), np.asarray(spec.ub)
    X = lb[None, :] + g.random((ps, spec.D)) * (ub - lb)[None, :]
    return X.astype(np.float32)

