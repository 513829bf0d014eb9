"""Pins the oracle's objectives to closed forms and special cases.

Each check is chosen so that a plausible slip in the oracle -- a transposed
rotation, a wrong exponent base, a reversed Rosenbrock chain, a wrong hybrid
split, a dropped composition weight -- fails it.
"""
import numpy as np
import pytest

from paper_2510_14982_gb300 import inputs


def _prob(orc, spec):
    return orc.OracleProblem.from_spec(spec)


def test_rotation_is_orthogonal_and_unique():
    for D in (3, 10, 100):
        M = inputs.rotation(D, seed=7).astype(np.float64)
        np.testing.assert_allclose(M.T @ M, np.eye(D), atol=2e-6)
        # deterministic in the seed, different across seeds
        assert np.array_equal(inputs.rotation(D, seed=7), inputs.rotation(D, seed=7))
        assert not np.array_equal(inputs.rotation(D, seed=7), inputs.rotation(D, seed=8))


@pytest.mark.parametrize("kind", [inputs.OBJ_ELLIPTIC, inputs.OBJ_RASTRIGIN])
def test_zero_at_the_shift(orc, kind):
    spec = inputs.shifted_rotated(kind, 10, seed=1)
    f = orc.objective(_prob(orc, spec), spec.shift.astype(np.float64))
    assert abs(f[0]) < 1e-9


def _x_for_z(spec, z):
    """x with M (x - o) = z, using M^-1 = M^T of the float32 rotation in FP64."""
    M = spec.rot.astype(np.float64)
    return spec.shift.astype(np.float64) + np.linalg.solve(M, z)


def test_elliptic_unit_vectors_give_the_conditioning_weights(orc):
    D = 10
    spec = inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, D, seed=2)
    p = _prob(orc, spec)
    for i in range(D):
        z = np.zeros(D)
        z[i] = 1.0
        f = orc.objective(p, _x_for_z(spec, z))[0]
        assert f == pytest.approx(10.0 ** (6.0 * i / (D - 1)), rel=1e-9)


def test_rosenbrock_closed_forms(orc):
    D = 6
    spec = inputs.shifted_rotated(inputs.OBJ_ROSENBROCK, D, seed=3)
    p = _prob(orc, spec)
    # minimum at z = 1 (x = o + M^T 1)
    assert orc.objective(p, _x_for_z(spec, np.ones(D)))[0] == pytest.approx(0.0, abs=1e-9)
    # z = 0 gives D - 1
    assert orc.objective(p, _x_for_z(spec, np.zeros(D)))[0] == pytest.approx(D - 1, rel=1e-9)
    # chain direction: z = (2, 1, 1, ...) -> 100 (1 - 4)^2 + 1 = 901
    z = np.ones(D)
    z[0] = 2.0
    assert orc.objective(p, _x_for_z(spec, z))[0] == pytest.approx(901.0, rel=1e-9)


def test_rastrigin_integer_and_half_points(orc):
    D = 10
    spec = inputs.shifted_rotated(inputs.OBJ_RASTRIGIN, D, seed=4)
    p = _prob(orc, spec)
    z = np.arange(D, dtype=np.float64) - 4.0   # integers: cos term is 1
    assert orc.objective(p, _x_for_z(spec, z))[0] == pytest.approx(float((z * z).sum()), rel=1e-9)
    z = np.full(D, 0.5)                         # cos(pi) = -1: 0.25 + 10 + 10 per dim
    assert orc.objective(p, _x_for_z(spec, z))[0] == pytest.approx(20.25 * D, rel=1e-9)


@pytest.mark.parametrize("D,sizes", [(100, (30, 30, 40)), (10, (3, 3, 4)), (20, (6, 6, 8)), (50, (15, 15, 20))])
def test_hybrid_split_and_zero(orc, D, sizes):
    spec = inputs.shifted_rotated(inputs.OBJ_HYBRID, D, seed=5)
    p = _prob(orc, spec)
    n1, n2, n3 = sizes
    perm = spec.perm
    # zero: w = z[perm] is 1 on the Rosenbrock group and 0 elsewhere
    w = np.zeros(D)
    w[n1:n1 + n2] = 1.0
    z = np.zeros(D)
    z[perm] = w
    assert orc.objective(p, _x_for_z(spec, z))[0] == pytest.approx(0.0, abs=1e-8)
    # a unit bump at the last elliptic slot costs 10^6 (and nothing else moves)
    w2 = w.copy()
    w2[n1 - 1] = 1.0
    z[perm] = w2
    assert orc.objective(p, _x_for_z(spec, z))[0] == pytest.approx(1e6, rel=1e-9)
    # a 0.5 at the first Rastrigin slot costs 20.25
    w3 = w.copy()
    w3[n1 + n2] = 0.5
    z[perm] = w3
    assert orc.objective(p, _x_for_z(spec, z))[0] == pytest.approx(20.25, rel=1e-9)
    assert n3 == D - n1 - n2


def test_composition_special_cases(orc):
    D = 8
    full = inputs.composition(D=D, seed=6, n_comp=4)
    # one component: exactly g_0 + bias_0 (the weight cancels)
    one = inputs.ProblemSpec(kind=inputs.OBJ_COMPOSITION, D=D, lb=full.lb, ub=full.ub,
                             shift=full.shift[:1], rot=full.rot[:1], perm=full.perm[:1],
                             comp_sigma=full.comp_sigma[:1], comp_bias=np.array([37.0]))
    ell = inputs.ProblemSpec(kind=inputs.OBJ_ELLIPTIC, D=D, lb=full.lb, ub=full.ub,
                             shift=full.shift[0], rot=full.rot[0])
    x = np.linspace(-50, 50, D)
    assert orc.objective(_prob(orc, one), x)[0] == pytest.approx(orc.objective(_prob(orc, ell), x)[0] + 37.0, rel=1e-12)
    # two components with the same centre and sigma: equal weights, plain mean
    two = inputs.ProblemSpec(kind=inputs.OBJ_COMPOSITION, D=D, lb=full.lb, ub=full.ub,
                             shift=np.stack([full.shift[0], full.shift[0]]), rot=full.rot[:2],
                             perm=full.perm[:2], comp_sigma=np.array([20.0, 20.0]),
                             comp_bias=np.array([0.0, 100.0]))
    ros = inputs.ProblemSpec(kind=inputs.OBJ_ROSENBROCK, D=D, lb=full.lb, ub=full.ub,
                             shift=full.shift[0], rot=full.rot[1])
    g0 = orc.objective(_prob(orc, ell), x)[0]
    g1 = orc.objective(_prob(orc, ros), x)[0]
    assert orc.objective(_prob(orc, two), x)[0] == pytest.approx((g0 + g1 + 100.0) / 2, rel=1e-12)
    # far from component 1 and at the centre of component 0: component 0 dominates
    far = inputs.ProblemSpec(kind=inputs.OBJ_COMPOSITION, D=D, lb=full.lb, ub=full.ub,
                             shift=np.stack([full.shift[0], full.shift[0] + 90.0]), rot=full.rot[:2],
                             perm=full.perm[:2], comp_sigma=np.array([1.0, 1.0]),
                             comp_bias=np.array([0.0, 100.0]))
    x0 = full.shift[0].astype(np.float64)
    assert orc.objective(_prob(orc, far), x0)[0] == pytest.approx(0.0, abs=1e-9)


def test_sphere_is_sum_of_squares(orc):
    spec = inputs.sphere(5, -10, 10)
    x = np.array([1.0, -2.0, 3.0, 0.5, 0.0])
    assert orc.objective(_prob(orc, spec), x)[0] == pytest.approx(14.25)


@pytest.mark.parametrize("kind", [inputs.OBJ_BENTCIGAR, inputs.OBJ_HGBAT, inputs.OBJ_GRIEWANK])
@pytest.mark.parametrize("D", [7, 1000])
def test_table2_forms_vanish_at_the_shift(orc, kind, D):
    """Bent Cigar, HGBat (y = z / 20 - 1 is -1 at z = 0) and Griewank are 0 at o."""
    spec = inputs.shifted_rotated(kind, D, seed=3)
    f = orc.objective(_prob(orc, spec), spec.shift.astype(np.float64))[0]
    assert abs(f) < 1e-9


def test_bent_cigar_weights_one_axis_by_one_and_the_rest_by_a_million(orc):
    D = 9
    spec = inputs.shifted_rotated(inputs.OBJ_BENTCIGAR, D, seed=4)
    p = _prob(orc, spec)
    for i in range(D):
        z = np.zeros(D)
        z[i] = 2.0
        f = orc.objective(p, _x_for_z(spec, z))[0]
        assert f == pytest.approx(4.0 if i == 0 else 4e6, rel=1e-9)


@pytest.mark.parametrize("c", [2.0, -0.5, 3.0])
def test_hgbat_on_a_constant_vector(orc, c):
    """y_i = c for all i: Sum y^2 = D c^2, Sum y = D c, so
    f = D |c| sqrt(|c^2 - 1|) + c^2 / 2 + c + 1/2 (z = 20 (1 + c))."""
    D = 12
    spec = inputs.shifted_rotated(inputs.OBJ_HGBAT, D, seed=5)
    z = np.full(D, 20.0 * (1.0 + c))
    f = orc.objective(_prob(orc, spec), _x_for_z(spec, z))[0]
    want = D * abs(c) * np.sqrt(abs(c * c - 1.0)) + c * c / 2 + c + 0.5
    assert f == pytest.approx(want, rel=1e-9)


def test_griewank_product_takes_the_square_root_of_the_index(orc):
    """y = 6 z with y_k / sqrt(k) = pi in coordinate k (1-based) and 0 elsewhere:
    the product is cos(pi) = -1, so f = 1 + y_k^2 / 4000 + 1; the cosine period
    pins sqrt(k) (an index without the root, or 0-based, gives another value)."""
    D = 10
    spec = inputs.shifted_rotated(inputs.OBJ_GRIEWANK, D, seed=6)
    p = _prob(orc, spec)
    for k in (1, 4, 9):
        y = np.pi * np.sqrt(k)
        z = np.zeros(D)
        z[k - 1] = y / 6.0
        f = orc.objective(p, _x_for_z(spec, z))[0]
        assert f == pytest.approx(2.0 + y * y / 4000.0, rel=1e-9)
