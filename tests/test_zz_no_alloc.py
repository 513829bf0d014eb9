"""apo_run_device_noalloc, the entry point for callers that cannot allocate
device memory (their memory belongs to their own pool, or they cannot afford
the synchronisation of cudaFree), must give the same results as
apo_run_device.  Two calls in a row check that the shared static scratch is
reset correctly between calls.  Collected last so that a first failure here
leaves every other test already run."""
import numpy as np
import pytest

from paper_2510_14982_gb300 import inputs
from parity_helpers import close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def apo():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_14982_gb300 import apo as m
    return m


def _otsu_spec():
    hist = np.bincount(inputs.gmm_image(5, 1 << 16), minlength=256)
    return inputs.otsu_problem(hist, 4)


CASES = [
    # resident single run (population in shared memory)
    ("rastrigin10_ps20", lambda: inputs.single_rastrigin(0), 20, 300),
    # cooperative grid run (population in the scratch array)
    ("hybrid50_ps1500", lambda: inputs.shifted_rotated(inputs.OBJ_HYBRID, 50, 2), 1500, 40),
    # float64 fitness (Otsu): 8-byte fitness buffers and 16-byte ranking keys in the scratch
    ("otsu4_ps256", _otsu_spec, 256, 60),
    # work-queue run whose resident layout does not fit shared memory (population in the scratch)
    ("sphere256_ps120", lambda: inputs.sphere(256, -5.0, 5.0), 120, 30),
]


@pytest.mark.parametrize("name,mk,ps,T", CASES, ids=[c[0] for c in CASES])
def test_noalloc_matches_allocating_entry_point(apo, name, mk, ps, T):
    import torch
    spec = mk()
    prob = apo.problem_from_spec(spec)
    D = spec.D
    for seed in (3, 4):   # two calls in a row on the shared scratch
        prm = apo.apo_params_make(ps, 1, 0.1, T, seed)
        ref_x = torch.zeros(D, device="cuda")
        ref_f = torch.zeros(1, dtype=torch.float64, device="cuda")
        ref_c = torch.zeros(T + 1, device="cuda")
        apo.apo_run_device(prob, prm, ref_x, ref_f, ref_c)
        torch.cuda.synchronize()
        x = torch.full((D,), float("nan"), device="cuda")
        f = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        c = torch.full((T + 1,), float("nan"), device="cuda")
        apo.apo_run_device_noalloc(prob, prm, x, f, c)
        # the same kernels on the same inputs: identical bits (well within the
        # parity tolerance of the other tests)
        assert close(x.cpu().numpy(), ref_x.cpu().numpy()).all()
        assert torch.equal(x, ref_x) and torch.equal(f, ref_f) and torch.equal(c, ref_c)
        assert np.all(np.diff(c.cpu().numpy()) <= 0)


def test_noalloc_rejects_oversized_runs(apo):
    import torch
    spec = inputs.shifted_rotated(inputs.OBJ_ELLIPTIC, 100, 1)
    prob = apo.problem_from_spec(spec)
    x = torch.zeros(100, device="cuda")
    f = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(apo.ApoError) as e:
        apo.apo_run_device_noalloc(prob, apo.apo_params_make(4096, 1, 0.1, 20000, 0), x, f)
    assert e.value.status == apo.APO_ERR_UNSUPPORTED
    assert "scratch" in str(e.value)
