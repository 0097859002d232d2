"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Tolerances (relative L2 error against the FP64 oracle):
1e-12 for UW_F64, 1e-5 for UW_F32 and UW_F32_SPLIT_BF16."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, fast, tables, wavelets as W
from paper_2106_00554_gb300 import F32, F32_SPLIT_BF16, F64, PERIODIC, VMP, Plan, UWError, build, inputs

pytestmark = pytest.mark.gpu
TOL = {F64: 1e-12, F32: 1e-5, F32_SPLIT_BF16: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def dev(a, prec):
    dt = torch.float64 if prec == F64 else torch.float32
    return torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def run_fwd(plan, x, prec):
    y = plan.forward(dev(x, prec), precision=prec)
    torch.cuda.synchronize()
    return y.double().cpu().numpy()


def run_adj(plan, y, prec):
    x = plan.adjoint(dev(y, prec), precision=prec)
    torch.cuda.synchronize()
    return x.double().cpu().numpy()


# ----------------------------------------------------------------------------
# 1D
# ----------------------------------------------------------------------------
def test_config1_fp64_dense():
    """p = 2 VMP, M = 2^10, q = 1, all Walsh rows, one x (level decay 1.0) and
    one y ~ N(0,1), seed 0: against the dense 2048 x 1024 oracle."""
    rng = np.random.default_rng(0)
    R, q, p = 10, 1, 2
    plan = Plan(1, R, q, p, VMP)
    assert plan.J0 == 3
    x = inputs.coeffs_1d(rng, R, plan.J0, 1.0)
    y = inputs.gaussian(rng, 2 ** (R + q))
    U = dense.U1d(R, q, p, VMP, plan.J0)
    for prec in (F64, F32):
        assert rel(run_fwd(plan, x, prec), U @ x) < TOL[prec]
        assert rel(run_adj(plan, y, prec), U.T @ y) < TOL[prec]


CASES_1D = [(p, bd, dR, q) for p in (1, 2, 3, 4, 6, 8) for bd in (PERIODIC, VMP)
            for dR, q in ((0, 1), (1, 0), (1, 2), (3, 1))]


@pytest.mark.parametrize("p,bd,dR,q", CASES_1D)
def test_1d_sweep_against_dense(p, bd, dR, q):
    rng = np.random.default_rng(100 * p + 10 * bd + dR + q)
    J0 = W.default_J0(p)
    R = J0 + dR
    M, N = 2 ** R, 2 ** (R + q)
    omega = np.sort(rng.choice(N, size=max(1, (2 * N) // 5), replace=False))
    plan = Plan(1, R, q, p, bd, omega=omega, max_batch=3)
    U = dense.U1d(R, q, p, bd, J0)[omega]
    x = rng.standard_normal((3, M))
    y = rng.standard_normal((3, omega.size))
    for prec in (F64, F32):
        assert rel(run_fwd(plan, x, prec), x @ U.T) < TOL[prec]
        assert rel(run_adj(plan, y, prec), y @ U) < TOL[prec]


@pytest.mark.parametrize("prec,R,q,p,bd", [(F64, 13, 2, 3, VMP), (F32, 14, 2, 2, VMP), (F64, 12, 4, 4, VMP),
                                            (F32, 14, 2, 3, PERIODIC), (F64, 14, 1, 5, PERIODIC),
                                            (F32, 15, 1, 8, VMP), (F32, 14, 1, 10, VMP), (F32, 13, 2, 9, PERIODIC),
                                            (F32, 17, 2, 4, VMP)])
def test_1d_large_lines_against_algorithm1(prec, R, q, p, bd):
    """Lines longer than one CTA's shared memory take the multi-kernel path:
    the coarse levels of each line in one CTA's shared memory (as many as
    fit), the levels above them one launch each, T, the two-pass FWHT.  At
    N = 2^19 (FP32) the stages across segments exceed one CTA's columns and
    the separate gather / scatter run."""
    rng = np.random.default_rng(R + q + 10 * bd)
    J0 = W.default_J0(p)
    N = 2 ** (R + q)
    omega = inputs.mask_1d(rng, N, 0.2)
    plan = Plan(1, R, q, p, bd, omega=omega, max_batch=2)
    x = inputs.coeffs_1d(rng, R, J0, 1.5, batch=2)
    y = rng.standard_normal((2, omega.size))
    assert rel(run_fwd(plan, x, prec), fast.forward1d(x, R, q, p, bd, J0, omega)) < TOL[prec]
    assert rel(run_adj(plan, y, prec), fast.adjoint1d(y, R, q, p, bd, J0, omega)) < TOL[prec]


@pytest.mark.parametrize("bd", [VMP, PERIODIC])
def test_1d_large_lines_unaligned_buffers(bd):
    """FP32 lines longer than shared memory with x and y buffers 4 bytes off
    a 16-byte boundary (views one element into larger tensors): the kernels
    that move 16 bytes at a time fall back to their scalar forms.  The
    forward matches the aligned call bit for bit (same arithmetic); the
    adjoint's levels take the generic per-pair kernels, so it matches to
    rounding; both match Algorithm 1."""
    import torch
    rng = np.random.default_rng(77 + bd)
    R, q, p = 14, 2, 4
    J0 = W.default_J0(p)
    M, N = 2 ** R, 2 ** (R + q)
    omega = inputs.mask_1d(rng, N, 0.2)
    plan = Plan(1, R, q, p, bd, omega=omega, max_batch=2)
    x = inputs.coeffs_1d(rng, R, J0, 1.5, batch=2)
    y = rng.standard_normal((2, omega.size))
    xa, ya = dev(x, F32), dev(y, F32)
    bx = torch.zeros(2 * M + 1, dtype=torch.float32, device="cuda")
    by = torch.zeros(2 * omega.size + 1, dtype=torch.float32, device="cuda")
    xu, yu = bx[1:].view(2, M), by[1:].view(2, omega.size)
    xu.copy_(xa)
    yu.copy_(ya)
    assert xu.data_ptr() % 16 and yu.data_ptr() % 16
    got_y = torch.zeros(2 * omega.size + 1, dtype=torch.float32, device="cuda")[1:].view(2, omega.size)
    got_x = torch.zeros(2 * M + 1, dtype=torch.float32, device="cuda")[1:].view(2, M)
    plan.forward(xu, got_y, precision=F32)
    plan.adjoint(yu, got_x, precision=F32)
    want_y = plan.forward(xa, precision=F32)
    want_x = plan.adjoint(ya, precision=F32)
    torch.cuda.synchronize()
    assert torch.equal(got_y, want_y)
    assert rel(got_x.double().cpu().numpy(), want_x.double().cpu().numpy()) < 1e-6
    assert rel(got_y.double().cpu().numpy(), fast.forward1d(x, R, q, p, bd, J0, omega)) < TOL[F32]
    assert rel(got_x.double().cpu().numpy(), fast.adjoint1d(y, R, q, p, bd, J0, omega)) < TOL[F32]


@pytest.mark.parametrize("prec", [F32, F64])
def test_config2_full_size(prec):
    """p = 4, M = 2^16, q = 2 (N = 2^18), multilevel 15% mask, batch 64 with
    level decay 1.5, seed 1; two sampled instances against Algorithm 1 and the
    whole batch through the dot-product test."""
    rng = np.random.default_rng(1)
    R, q, p = 16, 2, 4
    N = 2 ** (R + q)
    omega = inputs.mask_1d(rng, N, 0.15)
    assert omega.size == 39322
    plan = Plan(1, R, q, p, VMP, omega=omega, max_batch=64)
    J0 = plan.J0
    x = inputs.coeffs_1d(rng, R, J0, 1.5, batch=64)
    y = rng.standard_normal((64, omega.size))
    yg = run_fwd(plan, x, prec)
    xg = run_adj(plan, y, prec)
    for b in (0, 63):
        assert rel(yg[b], fast.forward1d(x[b], R, q, p, VMP, J0, omega)) < TOL[prec]
        assert rel(xg[b], fast.adjoint1d(y[b], R, q, p, VMP, J0, omega)) < TOL[prec]
    lhs = np.sum(yg * y)
    rhs = np.sum(x * xg)
    assert abs(lhs - rhs) <= 10 * TOL[prec] * (abs(lhs) + np.linalg.norm(yg) * np.linalg.norm(y))


# ----------------------------------------------------------------------------
# 2D
# ----------------------------------------------------------------------------
CASES_2D = [(p, bd, dR, q) for p in (1, 2, 4) for bd in (PERIODIC, VMP)
            for dR, q in ((0, 1), (1, 1), (2, 0), (2, 2))]


@pytest.mark.parametrize("p,bd,dR,q", CASES_2D)
def test_2d_sweep_against_dense(p, bd, dR, q):
    rng = np.random.default_rng(1000 + 100 * p + 10 * bd + dR + q)
    J0 = W.default_J0(p)
    R = J0 + dR
    M, N = 2 ** R, 2 ** (R + q)
    omega = np.sort(rng.choice(N * N, size=max(1, (N * N) // 3), replace=False))
    plan = Plan(2, R, q, p, bd, omega=omega, max_batch=2)
    G = dense.G1d(R, q, p, bd)
    x = rng.standard_normal((2, M, M))
    y = rng.standard_normal((2, omega.size))
    want_y = dense.forward2d(x, R, q, p, bd, J0, omega, G=G)
    want_x = dense.adjoint2d(y, R, q, p, bd, J0, omega, G=G)
    for prec in (F64, F32):
        assert rel(run_fwd(plan, x, prec), want_y) < TOL[prec]
        assert rel(run_adj(plan, y, prec), want_x) < TOL[prec]


COARSE_PATHS = {"fused": None, "separate_transposes": "UW_COARSE_SEPARATE_TRANSPOSE",
                "generic_tiles": "UW_COARSE_GENERIC", "per_level": "UW_COARSE_PER_LEVEL"}


@pytest.mark.parametrize("path", list(COARSE_PATHS))
@pytest.mark.parametrize("p,bd,R,q", [(5, VMP, 8, 1), (6, PERIODIC, 8, 1), (7, VMP, 7, 2), (8, VMP, 9, 1),
                                       (9, PERIODIC, 9, 1), (10, VMP, 9, 1), (10, PERIODIC, 8, 1)])
def test_2d_coarse_levels_long_filters(monkeypatch, path, p, bd, R, q):
    """Several coarse 2D levels with long filters, through each coarse-level
    path: one cooperative launch that also moves the coefficient array into
    (forward) and out of (adjoint) the transposed layout of the line passes,
    the same launch with separate transpose kernels, the generic tiles, and
    one launch per level.  Tiles of 8 to 32 samples meet the boundary blocks
    of both edges."""
    from paper_2106_00554_gb300 import _lib
    if COARSE_PATHS[path]:
        monkeypatch.setenv(COARSE_PATHS[path], "1")
    rng = np.random.default_rng(2000 + 10 * p + bd)
    J0 = W.default_J0(p)
    M, N = 2 ** R, 2 ** (R + q)
    omega = np.sort(rng.choice(N * N, size=(N * N) // 5, replace=False))
    plan = Plan(2, R, q, p, bd, omega=omega)
    G = dense.G1d(R, q, p, bd)
    x = inputs.coeffs_2d(rng, R, J0, 1.0)
    y = rng.standard_normal(omega.size)
    want_y = dense.forward2d(x, R, q, p, bd, J0, omega, G=G)
    want_x = dense.adjoint2d(y, R, q, p, bd, J0, omega, G=G)
    _lib.uw_plan_profile(plan._h, True)
    for prec in (F64, F32):
        assert rel(run_fwd(plan, x, prec), want_y) < TOL[prec]
        assert rel(run_adj(plan, y, prec), want_x) < TOL[prec]
    names = _kernel_names(plan)
    _lib.uw_plan_profile(plan._h, False)
    moved_in_levels = path == "fused" and R - 1 - J0 >= 2
    assert ("transpose_in" in names) == (not moved_in_levels), names
    assert ("transpose_out" in names) == (not moved_in_levels), names


@pytest.mark.parametrize("generic", [False, True])
@pytest.mark.parametrize("p,bd,dR,q", [(2, VMP, 2, 1), (4, PERIODIC, 3, 2), (8, VMP, 4, 1), (3, VMP, 4, 1)])
def test_fp32_line_kernels_both_implementations(monkeypatch, generic, p, bd, dR, q):
    """The register-blocked FP32 line kernels and the generic ones (selected
    with UW_GENERIC_LINES=1) both match the oracle, 1D and 2D."""
    if generic:
        monkeypatch.setenv("UW_GENERIC_LINES", "1")
    rng = np.random.default_rng(7 * p + q)
    J0 = W.default_J0(p)
    R = J0 + dR
    M, N = 2 ** R, 2 ** (R + q)
    om1 = inputs.mask_1d(rng, N, 0.3)
    plan1 = Plan(1, R, q, p, bd, omega=om1, max_batch=2)
    x1 = inputs.coeffs_1d(rng, R, J0, 1.0, batch=2)
    y1 = rng.standard_normal((2, om1.size))
    assert rel(run_fwd(plan1, x1, F32), fast.forward1d(x1, R, q, p, bd, J0, om1)) < 1e-5
    assert rel(run_adj(plan1, y1, F32), fast.adjoint1d(y1, R, q, p, bd, J0, om1)) < 1e-5
    if R > 9:
        return
    om2 = inputs.mask_2d(rng, N, 0.2)
    plan2 = Plan(2, R, q, p, bd, omega=om2)
    x2 = inputs.coeffs_2d(rng, R, J0, 1.5)
    y2 = rng.standard_normal(om2.size)
    G = dense.G1d(R, q, p, bd)
    assert rel(run_fwd(plan2, x2, F32), dense.forward2d(x2, R, q, p, bd, J0, om2, G=G)) < 1e-5
    assert rel(run_adj(plan2, y2, F32), dense.adjoint2d(y2, R, q, p, bd, J0, om2, G=G)) < 1e-5


@pytest.mark.parametrize("prec", [F64, F32, F32_SPLIT_BF16])
def test_config3(prec):
    """p = 4, M = 256^2, q = 1, radial 25% mask, level decay 1.5, seed 2."""
    rng = np.random.default_rng(2)
    R, q, p = 8, 1, 4
    N = 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, 0.25)
    assert omega.size == 65536
    plan = Plan(2, R, q, p, VMP, omega=omega)
    x = inputs.coeffs_2d(rng, R, plan.J0, 1.5)
    y = rng.standard_normal(omega.size)
    G = dense.G1d(R, q, p, VMP)
    assert rel(run_fwd(plan, x, prec), dense.forward2d(x, R, q, p, VMP, plan.J0, omega, G=G)) < TOL[prec]
    assert rel(run_adj(plan, y, prec), dense.adjoint2d(y, R, q, p, VMP, plan.J0, omega, G=G)) < TOL[prec]


SPLIT_CASES = [(1, PERIODIC, 8, 1), (2, VMP, 8, 1), (3, VMP, 8, 2), (4, PERIODIC, 9, 1), (5, VMP, 9, 1),
               (6, VMP, 8, 2), (8, VMP, 9, 1), (8, PERIODIC, 9, 2), (9, PERIODIC, 9, 2), (10, VMP, 9, 1),
               (10, VMP, 8, 2)]


def _kernel_names(plan):
    from paper_2106_00554_gb300 import _lib
    return [e["name"] for e in _lib.uw_plan_profile_read(plan._h)]


@pytest.mark.parametrize("p,bd,R,q", SPLIT_CASES)
def test_split_bf16_tensor_core_lines(p, bd, R, q):
    """UW_F32_SPLIT_BF16: the tensor-core line operators (block GEMM of the
    last level, T and bits 0-3; exact +-1 MMA for bits 4-7) against the dense
    oracle, both boundary types, q = 1 and 2, batch 2."""
    from paper_2106_00554_gb300 import _lib
    rng = np.random.default_rng(3000 + 10 * p + bd + q)
    J0 = W.default_J0(p)
    M, N = 2 ** R, 2 ** (R + q)
    omega = np.sort(rng.choice(N * N, size=(N * N) // 4, replace=False))
    plan = Plan(2, R, q, p, bd, omega=omega, max_batch=2)
    G = dense.G1d(R, q, p, bd)
    x = np.stack([inputs.coeffs_2d(rng, R, J0, 1.0) for _ in range(2)])
    y = rng.standard_normal((2, omega.size))
    want_y = dense.forward2d(x, R, q, p, bd, J0, omega, G=G)
    want_x = dense.adjoint2d(y, R, q, p, bd, J0, omega, G=G)
    _lib.uw_plan_profile(plan._h, True)
    got_y = run_fwd(plan, x, F32_SPLIT_BF16)
    got_x = run_adj(plan, y, F32_SPLIT_BF16)
    names = _kernel_names(plan)
    _lib.uw_plan_profile(plan._h, False)
    assert rel(got_y, want_y) < TOL[F32_SPLIT_BF16]
    assert rel(got_x, want_x) < TOL[F32_SPLIT_BF16]
    assert sum(n.endswith("_tc") for n in names) == 4, names


def test_split_bf16_small_lines_use_fp32_kernels():
    """Lines shorter than 512 samples are not served by the tensor-core
    kernels; the split precision then runs the FP32 line kernels."""
    from paper_2106_00554_gb300 import _lib
    rng = np.random.default_rng(7)
    R, q, p = 6, 1, 2
    N = 2 ** (R + q)
    omega = np.sort(rng.choice(N * N, size=N * N // 3, replace=False))
    plan = Plan(2, R, q, p, VMP, omega=omega)
    x = rng.standard_normal((2 ** R, 2 ** R))
    _lib.uw_plan_profile(plan._h, True)
    got = run_fwd(plan, x, F32_SPLIT_BF16)
    names = _kernel_names(plan)
    assert not any(n.endswith("_tc") for n in names)
    want = dense.forward2d(x, R, q, p, VMP, plan.J0, omega)
    assert rel(got, want) < 1e-5


def test_config5_full_size_split_bf16():
    """The benchmark workload (p = 8, M = 2048^2, q = 1, 12% radial mask,
    seed 4) on the split-BF16 tensor-core path against the oracle."""
    rng = np.random.default_rng(4)
    R, q, p = 11, 1, 8
    N = 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, 0.12)
    plan = Plan(2, R, q, p, VMP, omega=omega)
    x = inputs.coeffs_2d(rng, R, plan.J0, 1.5)
    y = rng.standard_normal(omega.size)
    G = dense.G1d(R, q, p, VMP)
    from paper_2106_00554_gb300 import _lib
    _lib.uw_plan_profile(plan._h, True)
    assert rel(run_fwd(plan, x, F32_SPLIT_BF16), dense.forward2d(x, R, q, p, VMP, plan.J0, omega, G=G)) < 1e-5
    assert rel(run_adj(plan, y, F32_SPLIT_BF16), dense.adjoint2d(y, R, q, p, VMP, plan.J0, omega, G=G)) < 1e-5
    # all four line passes of the benchmark workload run on the tcgen05 kernels
    assert sum(n.endswith("_umma") for n in _kernel_names(plan)) == 4


def test_config5_full_size_fp32():
    """p = 8, M = 2048^2, q = 1 (N = 4096^2), radial 12% mask, seed 4: the
    workload the benchmark times, against the dense-per-dimension oracle."""
    rng = np.random.default_rng(4)
    R, q, p = 11, 1, 8
    N = 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, 0.12)
    plan = Plan(2, R, q, p, VMP, omega=omega)
    x = inputs.coeffs_2d(rng, R, plan.J0, 1.5)
    y = rng.standard_normal(omega.size)
    G = dense.G1d(R, q, p, VMP)
    assert rel(run_fwd(plan, x, F32), dense.forward2d(x, R, q, p, VMP, plan.J0, omega, G=G)) < 1e-5
    assert rel(run_adj(plan, y, F32), dense.adjoint2d(y, R, q, p, VMP, plan.J0, omega, G=G)) < 1e-5


# ----------------------------------------------------------------------------
# edge cases and API behaviour
# ----------------------------------------------------------------------------
def test_empty_and_single_sample_masks():
    R, q, p = 4, 1, 2
    plan = Plan(2, R, q, p, VMP, omega=np.zeros(0, dtype=np.int64))
    assert plan.m == 0
    x = np.random.default_rng(0).standard_normal((16, 16))
    xa = run_adj(plan, np.zeros(0), F64)
    assert np.all(xa == 0)
    plan.set_mask(np.array([5]))
    G = dense.G1d(R, q, p, VMP)
    assert rel(run_fwd(plan, x, F64), dense.forward2d(x, R, q, p, VMP, plan.J0, [5], G=G)) < 1e-12


def test_invalid_calls_raise():
    plan = Plan(1, 6, 1, 2, VMP)
    x = torch.zeros((2, 64), dtype=torch.float64, device="cuda")
    with pytest.raises(UWError):
        plan.forward(x, precision=F64)           # batch 2 > reserved 1
    with pytest.raises(UWError):
        plan.set_mask(np.array([3, 2]))          # unsorted
    with pytest.raises(UWError):
        plan.set_mask(np.array([0, 128]))        # out of range
    plan.reserve(2)
    plan.forward(x, precision=F64)


def test_host_buffer_api_matches_device():
    rng = np.random.default_rng(5)
    R, q, p = 7, 1, 3
    N = 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, 0.3)
    plan = Plan(2, R, q, p, VMP, omega=omega)
    x = np.ascontiguousarray(rng.standard_normal((2 ** R, 2 ** R)).astype(np.float32))
    y = np.zeros(plan.m, dtype=np.float32)
    plan.forward_host(x.ctypes.data, y.ctypes.data, F32, 1)
    assert rel(y, run_fwd(plan, x, F32)) < 1e-6
    xb = np.zeros_like(x)
    plan.adjoint_host(y.ctypes.data, xb.ctypes.data, F32, 1)
    assert rel(xb, run_adj(plan, y, F32)) < 1e-6


@pytest.mark.parametrize("prec,batch", [(F32, 1), (F64, 2)])
def test_host_async_pipeline_matches_device(prec, batch):
    """uw_forward_host_async / uw_adjoint_host_async: five forward and five
    adjoint calls with different inputs in flight at once (two staging slots,
    copies on the plan's own streams), then uw_host_wait; every result equals
    the device API's.  A synchronous host call afterwards still agrees."""
    rng = np.random.default_rng(7)
    R, q, p = 8, 1, 4
    N = 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, 0.2)
    plan = Plan(2, R, q, p, VMP, omega=omega, max_batch=batch)
    dt = torch.float64 if prec == F64 else torch.float32
    shape = (batch, 2 ** R, 2 ** R) if batch > 1 else (2 ** R, 2 ** R)
    xs = [torch.tensor(rng.standard_normal(shape), dtype=dt).pin_memory() for _ in range(5)]
    ys = [torch.tensor(rng.standard_normal((batch, plan.m) if batch > 1 else plan.m), dtype=dt).pin_memory()
          for _ in range(5)]
    yo = [torch.empty_like(y).pin_memory() for y in ys]
    xo = [torch.empty_like(x).pin_memory() for x in xs]
    for k in range(5):
        plan.forward_host_async(xs[k].data_ptr(), yo[k].data_ptr(), prec, batch)
        plan.adjoint_host_async(ys[k].data_ptr(), xo[k].data_ptr(), prec, batch)
    plan.host_wait()
    tol = 1e-12 if prec == F64 else 1e-6
    for k in range(5):
        assert rel(yo[k].numpy(), run_fwd(plan, xs[k].numpy(), prec)) < tol
        assert rel(xo[k].numpy(), run_adj(plan, ys[k].numpy(), prec)) < tol
    ysync = torch.empty_like(yo[0]).pin_memory()
    plan.forward_host(xs[3].data_ptr(), ysync.data_ptr(), prec, batch)
    assert rel(ysync.numpy(), yo[3].numpy()) < tol


def test_host_async_graphs_follow_plan_changes(monkeypatch):
    """The asynchronous host calls replay their products as CUDA graphs
    captured at first use; a change of anything a graph was built from
    (mask, reserved buffers, coarsest level, launch switches) must capture
    anew.  After each change the asynchronous result equals the device API's
    for the changed plan (and the FP64 oracle's)."""
    rng = np.random.default_rng(11)
    R, q, p = 7, 1, 4
    N = 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, 0.2)
    plan = Plan(2, R, q, p, VMP, omega=omega)
    x = torch.tensor(rng.standard_normal((2 ** R, 2 ** R)), dtype=torch.float32).pin_memory()

    def check(batch=1, xin=None):
        xin = x if xin is None else xin
        out = torch.empty((batch, plan.m) if batch > 1 else plan.m, dtype=torch.float32).pin_memory()
        for _ in range(3):                       # first call captures, the next ones replay
            plan.forward_host_async(xin.data_ptr(), out.data_ptr(), F32, batch)
        plan.host_wait()
        want = dense.forward2d(xin.double().numpy(), R, q, p, VMP, plan.J0, plan_omega[0])
        assert rel(out.numpy(), run_fwd(plan, xin.numpy(), F32)) < 1e-6
        assert rel(out.numpy(), want) < 1e-5

    plan_omega = [omega]
    check()
    omega2 = inputs.mask_2d(rng, N, 0.35)        # another mask: another m, positions, prefix
    plan.set_mask(omega2)
    plan_omega[0] = omega2
    check()
    plan.reserve(2)                              # new workspace and staging buffers
    xb = torch.tensor(rng.standard_normal((2, 2 ** R, 2 ** R)), dtype=torch.float32).pin_memory()
    check(batch=2, xin=xb)
    check()
    from paper_2106_00554_gb300 import _lib
    _lib.uw_plan_set_coarsest(plan._h, plan.J0 + 1)   # one coarse level fewer
    check()
    monkeypatch.setenv("UW_GENERIC_LINES", "1")        # other line kernels
    check()


def test_dot_product_2d_fp64():
    rng = np.random.default_rng(6)
    R, q, p = 7, 2, 4
    N = 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, 0.2)
    plan = Plan(2, R, q, p, VMP, omega=omega)
    x = rng.standard_normal((2 ** R, 2 ** R))
    y = rng.standard_normal(omega.size)
    a = np.dot(run_fwd(plan, x, F64), y)
    b = np.sum(x * run_adj(plan, y, F64))
    assert abs(a - b) < 1e-12 * abs(a)


F32_LINE_CASES = [(1, PERIODIC, 10, 1), (2, VMP, 10, 1), (3, VMP, 9, 2), (5, PERIODIC, 9, 2), (8, VMP, 10, 1),
                  (9, VMP, 9, 2), (10, PERIODIC, 10, 1), (10, VMP, 10, 1), (4, VMP, 10, 2), (7, PERIODIC, 10, 2),
                  (8, VMP, 10, 2), (6, VMP, 10, 2)]


@pytest.mark.parametrize("p,bd,R,q", F32_LINE_CASES)
def test_fp32_persistent_line_kernels(p, bd, R, q):
    """UW_F32 on lines of N = 2048 and 4096 samples: the persistent FP32 line
    operators (interior formulas with zero or wrapped halos, VMP edges as
    small corrections) against the dense oracle, both boundary types, q = 1
    and 2, batch 2, natural-order and sampled passes.  The VMP cases take
    both ways of applying the edge corrections: weights held in registers
    (p <= 4 at N = 2048; p <= 8 at N = 4096) and weights read per line
    (p >= 5 at N = 2048, p = 9, 10)."""
    from paper_2106_00554_gb300 import _lib
    rng = np.random.default_rng(4000 + 10 * p + bd + q)
    J0 = W.default_J0(p)
    M, N = 2 ** R, 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, 0.2)
    plan = Plan(2, R, q, p, bd, omega=omega, max_batch=2)
    G = dense.G1d(R, q, p, bd)
    x = np.stack([inputs.coeffs_2d(rng, R, J0, 1.0) for _ in range(2)])
    y = rng.standard_normal((2, omega.size))
    want_y = dense.forward2d(x, R, q, p, bd, J0, omega, G=G)
    want_x = dense.adjoint2d(y, R, q, p, bd, J0, omega, G=G)
    _lib.uw_plan_profile(plan._h, True)
    got_y = run_fwd(plan, x, F32)
    got_x = run_adj(plan, y, F32)
    names = _kernel_names(plan)
    _lib.uw_plan_profile(plan._h, False)
    assert rel(got_y, want_y) < TOL[F32]
    assert rel(got_x, want_x) < TOL[F32]
    assert sum(n.endswith("_f32") for n in names) == 4, names


SYM_CASES = [(2, 4, VMP, 7, 1), (2, 6, PERIODIC, 7, 2), (2, 5, VMP, 8, 1), (2, 8, VMP, 10, 1),
             (1, 4, VMP, 10, 2), (1, 7, PERIODIC, 11, 1)]


@pytest.mark.parametrize("d,p,bd,R,q", SYM_CASES)
def test_symlets_against_dense_oracle(d, p, bd, R, q):
    """Least-asymmetric filters (UW_FILTER_SYMLET; Table 1's sym rows) through
    every kernel family: coarse 2D levels and line operators (the persistent
    FP32 kernels at N = 2048), 1D lines; FP64 and FP32 against the dense
    oracle built on the oracle's own symlet tables."""
    Sp = tables.Sym(p)
    rng = np.random.default_rng(6000 + 10 * p + bd + d)
    J0 = W.default_J0(p)
    M, N = 2 ** R, 2 ** (R + q)
    if d == 2:
        omega = inputs.mask_2d(rng, N, 0.2)
        x = inputs.coeffs_2d(rng, R, J0, 1.0)
    else:
        omega = inputs.mask_1d(rng, N, 0.3)
        x = inputs.coeffs_1d(rng, R, J0, 1.0)
    plan = Plan(d, R, q, p, bd, omega=omega, symlet=True)
    y = rng.standard_normal(omega.size)
    if d == 2:
        G = dense.G1d(R, q, Sp, bd)
        want_y = dense.forward2d(x, R, q, Sp, bd, J0, omega, G=G)
        want_x = dense.adjoint2d(y, R, q, Sp, bd, J0, omega, G=G)
    else:
        want_y = dense.forward1d(x, R, q, Sp, bd, J0, omega)
        want_x = dense.adjoint1d(y, R, q, Sp, bd, J0, omega)
    for prec in (F64, F32):
        assert rel(run_fwd(plan, x, prec), want_y) < TOL[prec]
        assert rel(run_adj(plan, y, prec), want_x) < TOL[prec]
    # the extremal-phase plan of the same p gives a different product
    db = Plan(d, R, q, p, bd, omega=omega)
    assert rel(run_fwd(db, x, F64), want_y) > 1e-3


def test_coarse_barrier_gives_up_and_reports(monkeypatch):
    """The coarse 2D levels run as one cooperative launch whose CTAs meet at
    bounded grid barriers.  With a spin limit of zero every wait gives up at
    once: the call returns (no hang), uw_plan_device_status reports
    UW_ERR_TIMEOUT and resets the barrier, and the next call with the default
    limit is correct again."""
    from paper_2106_00554_gb300 import _lib
    UW_OK, UW_ERR_TIMEOUT = 0, 5
    rng = np.random.default_rng(11)
    R, q, p = 8, 1, 2
    N = 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, 0.3)
    plan = Plan(2, R, q, p, VMP, omega=omega)
    assert R - 1 - plan.J0 >= 2
    x = inputs.coeffs_2d(rng, R, plan.J0, 1.0)
    want = dense.forward2d(x, R, q, p, VMP, plan.J0, omega)
    assert _lib.uw_plan_device_status(plan._h) == UW_OK
    monkeypatch.setenv("UW_BARRIER_SPIN_LIMIT", "0")
    run_fwd(plan, x, F32)
    assert _lib.uw_plan_device_status(plan._h) == UW_ERR_TIMEOUT
    monkeypatch.delenv("UW_BARRIER_SPIN_LIMIT")
    assert rel(run_fwd(plan, x, F32), want) < TOL[F32]
    assert _lib.uw_plan_device_status(plan._h) == UW_OK


@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2,
                    reason="needs two visible CUDA devices")
def test_call_with_another_device_current_is_rejected():
    """A plan's tables and workspace live on its own device.  A call made with
    another device current is refused before any lookup or launch (only the
    argument checks run), for the device products and the no-allocation one."""
    from paper_2106_00554_gb300 import UWError
    torch.cuda.set_device(0)
    plan = Plan(2, 6, 1, 2, VMP)
    x = torch.zeros((64, 64), dtype=torch.float32, device="cuda:0")
    y = torch.zeros(plan.m, dtype=torch.float32, device="cuda:0")
    try:
        torch.cuda.set_device(1)
        for call in (lambda: plan.forward(x, y, precision=F32), lambda: plan.adjoint(y, x, precision=F32),
                     lambda: plan.forward_noalloc(x, y, precision=F32)):
            with pytest.raises(UWError) as e:
                call()
            assert e.value.status == 1
    finally:
        torch.cuda.set_device(0)
    plan.close()
