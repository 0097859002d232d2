"""Differentiable products and the unrolled FISTA solve (GPU): autograd
against the dense oracle's transpose, finite differences (step 1e-3, FP64),
the dot-product identity, FISTA against a plain CPU FISTA on the dense oracle
matrices, and gradients of a loss through the iterations with respect to lam
and y (finite differences, with and without per-iteration checkpointing)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import dense, wavelets as W
from paper_2106_00554_gb300 import F32, F32_SPLIT_BF16, F64, PERIODIC, VMP, Plan, build, inputs
from paper_2106_00554_gb300 import solvers as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()


def _case(R=6, q=1, p=2, bd=VMP, frac=0.3, seed=0):
    rng = np.random.default_rng(seed)
    N = 2 ** (R + q)
    omega = np.sort(rng.choice(N * N, size=int(frac * N * N), replace=False))
    plan = Plan(2, R, q, p, bd, omega=omega)
    G = dense.G1d(R, q, p, bd)
    return rng, plan, omega, G


def test_backward_is_the_oracle_transpose():
    rng, plan, omega, G = _case()
    x = torch.tensor(rng.standard_normal((plan.M, plan.M)), device="cuda", requires_grad=True)
    w = rng.standard_normal(omega.size)
    f = (S.forward_op(plan, x) * torch.tensor(w, device="cuda")).sum()
    f.backward()
    want = dense.adjoint2d(w, plan.R, plan.q, plan.p, VMP, plan.J0, omega, G=G)
    got = x.grad.cpu().numpy()
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-12
    y = torch.tensor(w, device="cuda", requires_grad=True)
    v = rng.standard_normal((plan.M, plan.M))
    (S.adjoint_op(plan, y) * torch.tensor(v, device="cuda")).sum().backward()
    want2 = dense.forward2d(v, plan.R, plan.q, plan.p, VMP, plan.J0, omega, G=G)
    assert np.linalg.norm(y.grad.cpu().numpy() - want2) / np.linalg.norm(want2) < 1e-12


def test_finite_differences_fp64_step_1e_3():
    rng, plan, omega, _ = _case(R=5, p=2, bd=PERIODIC, seed=1)
    x = torch.tensor(rng.standard_normal((plan.M, plan.M)), device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: S.forward_op(plan, t), (x,), eps=1e-3, atol=1e-8, rtol=1e-7,
                                    fast_mode=True)
    y = torch.tensor(rng.standard_normal(omega.size), device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(lambda t: S.adjoint_op(plan, t), (y,), eps=1e-3, atol=1e-8, rtol=1e-7,
                                    fast_mode=True)


@pytest.mark.parametrize("prec,tol", [(F64, 1e-12), (F32, 1e-5), (F32_SPLIT_BF16, 1e-5)])
def test_dot_product_identity(prec, tol):
    rng, plan, omega, _ = _case(R=8, p=4, seed=2)       # the config-3 sizes: 256^2 -> 512^2
    dt = torch.float64 if prec == F64 else torch.float32
    x = torch.tensor(rng.standard_normal((plan.M, plan.M)), dtype=dt, device="cuda")
    y = torch.tensor(rng.standard_normal(omega.size), dtype=dt, device="cuda")
    lhs = float(S.dot64(S.forward_op(plan, x, prec), y))
    rhs = float(S.dot64(x, S.adjoint_op(plan, y, prec)))
    scale = float(torch.linalg.vector_norm(x.double())) * float(torch.linalg.vector_norm(y.double()))
    assert abs(lhs - rhs) / scale < tol


def _cpu_fista(G, omega, J0, R, q, p, bd, y, lam, iters, tau=1.0):
    """Plain FISTA on the dense-per-dimension oracle (FP64, CPU)."""
    x = np.zeros((2 ** R, 2 ** R))
    z = x.copy()
    B = dense.adjoint2d(y, R, q, p, bd, J0, omega, G=G)
    t = 1.0
    for _ in range(iters):
        Gz = dense.adjoint2d(dense.forward2d(z, R, q, p, bd, J0, omega, G=G), R, q, p, bd, J0, omega, G=G)
        v = z - tau * (Gz - B)
        x1 = np.sign(v) * np.maximum(np.abs(v) - tau * lam, 0.0)
        t1 = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        z = x1 + (t - 1.0) / t1 * (x1 - x)
        x, t = x1, t1
    return x


def test_fista_matches_a_plain_cpu_fista():
    rng, plan, omega, G = _case(R=6, p=2, seed=3)
    xt = inputs.sparse_coeffs_2d(rng, plan.R, plan.J0, 1.5, 0.05)
    y = dense.forward2d(xt, plan.R, plan.q, plan.p, VMP, plan.J0, omega, G=G) + 1e-3 * rng.standard_normal(omega.size)
    lam, iters = 1e-3, 30
    got = S.fista(plan, torch.tensor(y, device="cuda"), lam, iters=iters, checkpoint=False).cpu().numpy()
    want = _cpu_fista(G, omega, plan.J0, plan.R, plan.q, plan.p, VMP, y, lam, iters)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-10


def _torch_cpu_fista_loss(A, y, lam, xt, iters, tau=1.0):
    """The same unrolled FISTA and loss in plain CPU torch with the dense
    matrix A of x -> P_Omega U x (autograd gives the exact derivative for
    the same active sets)."""
    M2 = A.shape[1]
    x = torch.zeros(M2, dtype=torch.float64)
    z = x
    Bv = A.T @ y
    t = 1.0
    for _ in range(iters):
        v = z - tau * (A.T @ (A @ z) - Bv)
        x1 = torch.sign(v) * torch.relu(v.abs() - tau * lam)
        t1 = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        z = x1 + (t - 1.0) / t1 * (x1 - x)
        x, t = x1, t1
    return 0.5 * ((x - xt.reshape(-1)) ** 2).sum()


def _dense_matrix(plan, omega, G):
    """m x M^2 matrix of the 2D product, column by column from the oracle."""
    M = plan.M
    cols = []
    for i in range(M * M):
        e = np.zeros(M * M)
        e[i] = 1.0
        cols.append(dense.forward2d(e.reshape(M, M), plan.R, plan.q, plan.p, VMP, plan.J0, omega, G=G))
    return torch.tensor(np.stack(cols, axis=1))


@pytest.mark.parametrize("checkpoint", [True, False])
def test_gradients_through_fista(checkpoint):
    """d/dlam and d/dy of 1/2 ||x_K - x_true||^2 through K FISTA iterations
    equal the derivatives autograd finds for the same iterations written in
    plain CPU torch on the dense oracle."""
    rng, plan, omega, G = _case(R=5, p=2, seed=4)
    xt = inputs.sparse_coeffs_2d(rng, plan.R, plan.J0, 1.0, 0.2)
    y0 = dense.forward2d(xt, plan.R, plan.q, plan.p, VMP, plan.J0, omega, G=G)
    y0 = y0 + 1e-2 * rng.standard_normal(omega.size)
    iters, lam = 15, 2e-2
    yv = torch.tensor(y0, device="cuda", requires_grad=True)
    lt = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    L = S.half_sq_dist(S.fista(plan, yv, lt, iters=iters, checkpoint=checkpoint), torch.tensor(xt, device="cuda"))
    L.backward()
    yc = torch.tensor(y0, requires_grad=True)
    lc = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    Lc = _torch_cpu_fista_loss(_dense_matrix(plan, omega, G), yc, lc, torch.tensor(xt), iters)
    Lc.backward()
    assert abs(float(L.detach()) - float(Lc.detach())) <= 1e-10 * float(Lc.detach())
    assert abs(float(lt.grad) - float(lc.grad)) <= 1e-8 * max(1.0, abs(float(lc.grad)))
    gy, gyc = yv.grad.cpu().numpy(), yc.grad.numpy()
    assert np.linalg.norm(gy - gyc) <= 1e-8 * np.linalg.norm(gyc)


def test_fista_reduces_the_objective_on_the_benchmark_shape_split_bf16():
    """100 iterations at p = 8, 2048^2 -> 4096^2, 12% radial mask, x_true
    level-decaying with 5% nonzeros, noise 1e-3, lam = 1e-3 (seed 4), on the
    split-BF16 products, with gradients of 1/2 ||x_100 - x_true||^2 with
    respect to lam and y through checkpointed iterations."""
    rng = np.random.default_rng(4)
    R, q, p = 11, 1, 8
    N = 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, 0.12)
    plan = Plan(2, R, q, p, VMP, omega=omega)
    xt = inputs.sparse_coeffs_2d(rng, R, plan.J0, 1.5, 0.05)
    xt_d = torch.tensor(xt, dtype=torch.float32, device="cuda")
    y = plan.forward(xt_d, precision=F32) + 1e-3 * torch.tensor(rng.standard_normal(omega.size),
                                                                dtype=torch.float32, device="cuda")
    yv = y.clone().requires_grad_(True)
    lam = 1e-3
    lt = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    x = S.fista(plan, yv, lt, iters=100, precision=F32_SPLIT_BF16, checkpoint=True)
    L = S.half_sq_dist(x, xt_d)
    L.backward()
    torch.cuda.synchronize()

    def objective(v):   # 1/2 ||P U v - y||^2 + lam ||v||_1, in FP64 on the CPU copies
        r = plan.forward(v.detach().contiguous(), precision=F32).double().cpu() - y.double().cpu()
        return 0.5 * float(r @ r) + lam * float(v.detach().double().abs().sum())

    assert objective(x) < objective(torch.zeros_like(xt_d))
    assert torch.isfinite(yv.grad).all() and float(yv.grad.abs().max()) > 0
    assert np.isfinite(float(lt.grad))


@pytest.mark.parametrize("bd_name", ["periodic", "vmp"])
def test_periodic_vs_vmp_reconstructions_fig4(bd_name):
    """The periodic-versus-boundary comparison of Sec. 3.2 (Fig. 4) on the
    GPU: f(t) = cos(2 pi t) and g(t) = cos(2 pi t) + t from their first 32
    Walsh samples, generalised sampling in M = 16 DB4 functions (R = 4, q = 1)
    with the plan's boundary extension, solved by CG on the normal equations
    through the library's 1D products.  Each solution matches the oracle's
    least-squares fit, and the errors of the GPU solutions show what the
    figure's caption states (the oracle pins the same in
    tests/test_oracle_fig4.py): periodic wavelets fit the periodic f and leave
    boundary artefacts on g; VMP wavelets fit g, with the same error as f
    since g - f = t lies in their span."""
    from oracle import dense, wavelets as W
    from paper_2106_00554_gb300 import F64, PERIODIC, VMP, Plan, solvers
    import test_oracle_fig4 as fig4

    bd = PERIODIC if bd_name == "periodic" else VMP
    R, q, p = fig4.R, fig4.Q, fig4.P
    plan = Plan(1, R, q, p, bd)
    A = dense.U1d_scaling(R, q, p, bd)
    out = {}
    for name in ("f", "g"):
        c = fig4.samples(name)
        x, iters, res = solvers.cg_normal(plan, torch.tensor(c, dtype=torch.float64, device="cuda"), iters=100,
                                          tol=1e-14)
        x = x.cpu().numpy()
        want = W.dwt1d(np.linalg.lstsq(A, c, rcond=None)[0], plan.J0, p, bd)   # wavelet-basis coefficients
        assert np.linalg.norm(x - want) < 1e-10 * np.linalg.norm(want), (name, iters, res)
        z = W.idwt1d(x, plan.J0, p, bd)                                           # scaling-basis coefficients
        out[name] = fig4.errors(name, z, bd)
    (rel_f, d_f, eb_f, ei_f), (rel_g, d_g, eb_g, ei_g) = out["f"], out["g"]
    if bd == PERIODIC:
        assert rel_f < 2e-3 and eb_f < 2 * ei_f, (rel_f, eb_f, ei_f)
        assert rel_g > 2e-2 and eb_g > 5 * ei_g, (rel_g, eb_g, ei_g)
    else:
        assert rel_g < 5e-3 and eb_g < 3 * ei_g, (rel_g, eb_g, ei_g)
        assert np.max(np.abs(d_g - d_f)) < 1e-9, np.max(np.abs(d_g - d_f))


def test_generalised_sampling_example2_db2():
    """Generalised sampling of the paper's Example 2 (Sec. 6) on the GPU:
    f(t1, t2) = cos(3 pi t1 / 2) sin(3 pi t2) from its 32 x 32 first Walsh
    samples, DB2 with VMP boundaries at M = 16 x 16 (R = 4, q = 1), solved by
    CG on the normal equations through the library's products.  The solution
    matches the oracle's least-squares fit, and its relative L2 error matches
    the 0.0518 the paper prints (the oracle pins the same number on the CPU)."""
    scipy_integrate = pytest.importorskip("scipy.integrate")
    from oracle import dense, walsh, wavelets as W
    from paper_2106_00554_gb300 import F64, VMP, Plan, solvers

    quad = scipy_integrate.quad
    f1 = lambda t: np.cos(1.5 * np.pi * t)
    f2 = lambda t: np.sin(3.0 * np.pi * t)

    def cells(f, n):
        return np.array([quad(f, k / n, (k + 1) / n)[0] for k in range(n)])

    R, q, p = 4, 1, 2
    N = 2 ** (R + q)
    c1 = walsh.hadamard(N) @ cells(f1, N)
    c2 = walsh.hadamard(N) @ cells(f2, N)
    y = np.outer(c1, c2).reshape(-1)                  # all 32 x 32 samples, row-major sequency order
    plan = Plan(2, R, q, p, VMP)
    yd = torch.tensor(y, dtype=torch.float64, device="cuda")
    x, iters, res = solvers.cg_normal(plan, yd, iters=200, tol=1e-13)
    x = x.cpu().numpy()
    # the oracle's least-squares fit in the Mallat wavelet basis
    A = dense.U1d_scaling(R, q, p, VMP)
    z1 = np.linalg.lstsq(A, c1, rcond=None)[0]
    z2 = np.linalg.lstsq(A, c2, rcond=None)[0]
    want = W.dwt2d(np.outer(z1, z2), plan.J0, p, VMP)
    assert np.linalg.norm(x - want) < 1e-9 * np.linalg.norm(want), (iters, res)
    # relative L2 error of the reconstruction: <f, r> from Parseval on 2^12 Walsh functions
    Af = dense.U1d_scaling(R, 12 - R, p, VMP)
    fr1 = (walsh.hadamard(4096) @ cells(f1, 4096)) @ Af
    fr2 = (walsh.hadamard(4096) @ cells(f2, 4096)) @ Af
    S = W.idwt2d(x, plan.J0, p, VMP)                 # scaling-basis coefficients of the fit
    n2 = quad(lambda t: f1(t) ** 2, 0, 1)[0] * quad(lambda t: f2(t) ** 2, 0, 1)[0]
    err = np.sqrt((n2 - 2 * fr1 @ S @ fr2 + np.sum(S ** 2)) / n2)
    assert abs(err - 0.0518) < 5e-4, err


@pytest.mark.parametrize("prec", [F32_SPLIT_BF16, F32])
def test_fista_iterate_against_the_fp64_gpu_solve(prec):
    """The 100-iteration solve in split-BF16 (and FP32) against the same solve
    with the FP64 products, at the size of config 3 (p = 4, 256^2 -> 512^2,
    25% radial mask, x_true level-decaying with 5% nonzeros, noise 1e-3,
    lam = 1e-3).  Bound: each iteration's proximal-gradient map is
    nonexpansive, so the per-iteration product errors (<= 1e-5 of ||x||)
    add up to at most 100 * 1e-5 = 1e-3 of ||x_100||; the difference is
    printed (pytest -s) and is far below that in practice."""
    rng = np.random.default_rng(2)
    R, q, p = 8, 1, 4
    N = 2 ** (R + q)
    omega = inputs.mask_2d(rng, N, 0.25)
    plan = Plan(2, R, q, p, VMP, omega=omega)
    xt = inputs.sparse_coeffs_2d(rng, R, plan.J0, 1.5, 0.05)
    xt64 = torch.tensor(xt, dtype=torch.float64, device="cuda")
    y64 = plan.forward(xt64, precision=F64) + 1e-3 * torch.tensor(rng.standard_normal(omega.size),
                                                                  dtype=torch.float64, device="cuda")
    with torch.no_grad():
        ref = S.fista(plan, y64, 1e-3, iters=100, precision=F64, checkpoint=False)
        got = S.fista(plan, y64.float(), 1e-3, iters=100, precision=prec, checkpoint=False)
    torch.cuda.synchronize()
    d = float(torch.linalg.norm(got.double() - ref) / torch.linalg.norm(ref))
    print(f"FISTA x_100, precision {prec} against FP64: relative difference {d:.2e}")
    assert d < 1e-3
    # and the FP64 solve itself reduced the objective
    r = plan.forward(ref, precision=F64) - y64
    obj = 0.5 * float(r @ r) + 1e-3 * float(ref.abs().sum())
    assert obj < 0.5 * float(y64 @ y64)
