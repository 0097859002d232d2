"""uw_forward_noalloc: the 2D forward product with the library's fixed device
scratch in place of the plan's workspace.  Its results must equal those of
uw_forward bit for bit (same kernels, same launch shapes), call after call.
The file name sorts last so that the GPU test also runs after every other
test in the same process, when the device already holds the other tests'
plans and modules."""
import numpy as np
import pytest

from paper_2106_00554_gb300 import F32, F32_SPLIT_BF16, F64, VMP, Plan, UWError, _lib, build, inputs

UW_ERR_INVALID_ARG = 1
UW_ERR_UNSUPPORTED = 2


def test_null_plan_rejected_without_gpu():
    build.build()
    L = _lib.lib()
    assert L.uw_forward_noalloc(None, F32, None, None, 1, None) == UW_ERR_INVALID_ARG


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [F32, F64])
def test_noalloc_matches_uw_forward_on_consecutive_calls(prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    rng = np.random.default_rng(11)
    R, q, p, batch = 8, 1, 4, 2
    plan = Plan(2, R, q, p, VMP)
    plan.set_mask(inputs.mask_2d(rng, 2 ** (R + q), 0.25))
    plan.reserve(batch)
    dt = torch.float64 if prec == F64 else torch.float32
    xs = [torch.tensor(inputs.coeffs_2d(rng, R, plan.J0, 1.5, batch=batch), dtype=dt, device="cuda")
          for _ in range(2)]
    refs = [plan.forward(x, precision=prec) for x in xs]
    outs = [torch.full_like(r, float("nan")) for r in refs]
    for x, y in zip(xs, outs):
        plan.forward_noalloc(x, y, precision=prec)
    torch.cuda.synchronize()
    for r, y in zip(refs, outs):
        assert torch.equal(r, y)
    # the same array again, after the scratch holds the second call's data
    again = plan.forward_noalloc(xs[0], torch.empty_like(refs[0]), precision=prec)
    torch.cuda.synchronize()
    assert torch.equal(again, refs[0])
    plan.close()


@pytest.mark.gpu
def test_noalloc_rejects_what_does_not_fit():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    big = Plan(2, 10, 1, 2, VMP)       # FP32 needs 4 (2 512^2 + 1024^2 + 2 1024 2048) bytes > 8 MiB
    x = torch.zeros((1024, 1024), dtype=torch.float32, device="cuda")
    y = torch.zeros(big.m, dtype=torch.float32, device="cuda")
    with pytest.raises(UWError) as e:
        big.forward_noalloc(x, y)
    assert e.value.status == UW_ERR_INVALID_ARG
    big.close()
    one = Plan(1, 8, 1, 2, VMP)
    x1 = torch.zeros(256, dtype=torch.float32, device="cuda")
    y1 = torch.zeros(one.m, dtype=torch.float32, device="cuda")
    with pytest.raises(UWError) as e:
        one.forward_noalloc(x1, y1)
    assert e.value.status == UW_ERR_UNSUPPORTED
    small = Plan(2, 6, 1, 2, VMP)
    xs = torch.zeros((64, 64), dtype=torch.float32, device="cuda")
    ys = torch.zeros(small.m, dtype=torch.float32, device="cuda")
    with pytest.raises(UWError) as e:
        small.forward_noalloc(xs, ys, precision=F32_SPLIT_BF16)
    assert e.value.status == UW_ERR_UNSUPPORTED
    one.close()
    small.close()
