"""The split-BF16 line operators on the 5th-generation tensor cores
(tcgen05.mma, accumulators in tensor memory, bulk-copy staging) that serve
lines of N = 4096 samples with q = 1: against the dense oracle for both
boundary kinds and several filter lengths, batch 2 (line addressing across
instances), against the earlier tensor-core kernels, and the bounded waits
(a wait that gives up is reported, nothing hangs, the next call is right)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, wavelets as W
from paper_2106_00554_gb300 import F32, F32_SPLIT_BF16, PERIODIC, VMP, Plan, _lib, build, inputs

pytestmark = pytest.mark.gpu
R, Q = 11, 1
N = 2 ** (R + Q)


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def names(plan):
    return [e["name"] for e in _lib.uw_plan_profile_read(plan._h)]


def products(plan, x, y, prec):
    xd = torch.tensor(x, dtype=torch.float32, device="cuda")
    yd = torch.tensor(y, dtype=torch.float32, device="cuda")
    _lib.uw_plan_profile(plan._h, True)
    got_y = plan.forward(xd, precision=prec)
    got_x = plan.adjoint(yd, precision=prec)
    torch.cuda.synchronize()
    used = names(plan)
    _lib.uw_plan_profile(plan._h, False)
    return got_y.double().cpu().numpy(), got_x.double().cpu().numpy(), used


@pytest.mark.parametrize("p,bd", [(8, VMP), (8, PERIODIC), (2, VMP), (5, VMP), (1, VMP)])
def test_tcgen05_lines_against_dense_oracle(p, bd):
    """All four line passes of the pair run on the tcgen05 kernels and match
    the dense oracle at 1e-5 (a 25% radial mask: m is a multiple of 4, which
    the batched scatter's aligned copies need)."""
    rng = np.random.default_rng(500 + 10 * p + bd)
    omega = inputs.mask_2d(rng, N, 0.25)
    plan = Plan(2, R, Q, p, bd, omega=omega, max_batch=2)
    J0 = plan.J0
    G = dense.G1d(R, Q, p, bd)
    x = np.stack([inputs.coeffs_2d(rng, R, J0, a) for a in (1.0, 1.5)])
    y = rng.standard_normal((2, omega.size))
    got_y, got_x, used = products(plan, x, y, F32_SPLIT_BF16)
    assert sum(n.endswith("_umma") for n in used) == 4, used
    assert rel(got_y, dense.forward2d(x, R, Q, p, bd, J0, omega, G=G)) < 1e-5
    assert rel(got_x, dense.adjoint2d(y, R, Q, p, bd, J0, omega, G=G)) < 1e-5
    plan.close()


def test_tcgen05_lines_agree_with_the_earlier_tensor_core_kernels(monkeypatch):
    """The same pair through the tcgen05 kernels and through the mma.sync
    kernels (UW_NO_UMMA=1): both within FP32 rounding of each other."""
    rng = np.random.default_rng(77)
    p = 8
    omega = inputs.mask_2d(rng, N, 0.12)
    plan = Plan(2, R, Q, p, VMP, omega=omega)
    x = inputs.coeffs_2d(rng, R, plan.J0, 1.5)
    y = rng.standard_normal(omega.size)
    y5, x5, used5 = products(plan, x, y, F32_SPLIT_BF16)
    monkeypatch.setenv("UW_NO_UMMA", "1")
    y4, x4, used4 = products(plan, x, y, F32_SPLIT_BF16)
    monkeypatch.delenv("UW_NO_UMMA")
    assert sum(n.endswith("_umma") for n in used5) == 4
    assert sum(n.endswith("_tc") for n in used4) == 4
    assert rel(y5, y4) < 1e-5 and rel(x5, x4) < 1e-5
    yf, xf, _ = products(plan, x, y, F32)
    assert rel(y5, yf) < 1e-5 and rel(x5, xf) < 1e-5
    plan.close()


def test_tcgen05_wait_gives_up_and_reports(monkeypatch):
    """With a spin limit of zero every wait of the tcgen05 kernels gives up at
    once: the call returns, uw_plan_device_status reports UW_ERR_TIMEOUT, the
    kernels drained their copies and freed their tensor memory (the next
    launch allocates it again), and the next call with the default limit is
    right."""
    UW_OK, UW_ERR_TIMEOUT = 0, 5
    rng = np.random.default_rng(12)
    omega = inputs.mask_2d(rng, N, 0.25)
    plan = Plan(2, R, Q, 4, VMP, omega=omega)
    x = inputs.coeffs_2d(rng, R, plan.J0, 1.0)
    y = rng.standard_normal(omega.size)
    assert _lib.uw_plan_device_status(plan._h) == UW_OK
    monkeypatch.setenv("UW_TC_SPIN_LIMIT", "0")
    products(plan, x, y, F32_SPLIT_BF16)
    assert _lib.uw_plan_device_status(plan._h) == UW_ERR_TIMEOUT
    monkeypatch.delenv("UW_TC_SPIN_LIMIT")
    G = dense.G1d(R, Q, 4, VMP)
    got_y, got_x, used = products(plan, x, y, F32_SPLIT_BF16)
    assert sum(n.endswith("_umma") for n in used) == 4
    assert rel(got_y, dense.forward2d(x, R, Q, 4, VMP, plan.J0, omega, G=G)) < 1e-5
    assert rel(got_x, dense.adjoint2d(y, R, Q, 4, VMP, plan.J0, omega, G=G)) < 1e-5
    assert _lib.uw_plan_device_status(plan._h) == UW_OK
    plan.close()
