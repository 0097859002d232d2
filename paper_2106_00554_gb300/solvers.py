"""Differentiable products and an unrolled FISTA reconstruction.

* ``forward_op(plan, x)`` / ``adjoint_op(plan, y)``: y = P_Omega U x and
  x = U^* P_Omega^* y as torch.autograd.Functions whose backward passes are
  the library's adjoint and forward products (U and U^* are each other's
  transposes).
* ``fista(plan, y, lam, iters)``: FISTA for the l1-regularised recovery
  min_x 1/2 ||P_Omega U x - y||^2 + lam ||x||_1 (the compressive-sensing use
  of the products, Sec. 1.2 and Remark 4.2 of the paper), step tau <= 1 since
  ||P_Omega U|| <= 1.  Each iteration is one fused library kernel for the
  proximal step with momentum (and its vector-Jacobian product), so the
  solve can be differentiated with respect to lam and y; with
  ``checkpoint=True`` every iteration is recomputed during the backward pass
  instead of storing its products.
* ``half_sq_dist(a, b)``: 1/2 ||a - b||^2 accumulated in FP64 (a loss).
* ``cg_normal(plan, y, iters)``: generalised sampling (Sec. 1.2), the
  least-squares fit min_x ||P_Omega U x - y||^2, by conjugate gradients on
  the normal equations U^* P_Omega^* P_Omega U x = U^* P_Omega^* y (the paper
  solves its least-squares problems with CG), inner products in FP64.

Every arithmetic step runs in libuw's kernels; torch supplies tensors,
streams and the autograd tape.
"""
import math

import torch
from torch.utils.checkpoint import checkpoint as _checkpoint

from . import F32, F64, _lib


def _prec(t):
    return F64 if t.dtype == torch.float64 else F32


def _stream():
    return torch.cuda.current_stream().cuda_stream


class _Forward(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, plan, precision):
        ctx.plan, ctx.precision = plan, precision
        return plan.forward(x.contiguous(), precision=precision)

    @staticmethod
    def backward(ctx, gy):
        return ctx.plan.adjoint(gy.contiguous(), precision=ctx.precision), None, None


class _Adjoint(torch.autograd.Function):
    @staticmethod
    def forward(ctx, y, plan, precision):
        ctx.plan, ctx.precision = plan, precision
        return plan.adjoint(y.contiguous(), precision=precision)

    @staticmethod
    def backward(ctx, gx):
        return ctx.plan.forward(gx.contiguous(), precision=ctx.precision), None, None


def forward_op(plan, x, precision=None):
    """Differentiable y = P_Omega U x (backward: U^* P_Omega^*)."""
    return _Forward.apply(x, plan, precision)


def adjoint_op(plan, y, precision=None):
    """Differentiable x = U^* P_Omega^* y (backward: P_Omega U)."""
    return _Adjoint.apply(y, plan, precision)


class _FistaStep(torch.autograd.Function):
    """x1 = soft(z - tau (G - B), tau lam), z1 = x1 + beta (x1 - x0)."""

    @staticmethod
    def forward(ctx, z, G, B, x0, lam, tau, beta):
        z, G, B, x0 = (t.contiguous() for t in (z, G, B, x0))
        x1, z1 = torch.empty_like(z), torch.empty_like(z)
        lam_v = float(lam)
        _lib.uw_fista_step(_prec(z), z.numel(), z.data_ptr(), G.data_ptr(), B.data_ptr(), x0.data_ptr(), tau, lam_v,
                           beta, x1.data_ptr(), z1.data_ptr(), _stream())
        ctx.save_for_backward(z, G, B)
        ctx.lam, ctx.tau, ctx.beta = lam_v, tau, beta
        ctx.lam_like = lam if torch.is_tensor(lam) else None
        return x1, z1

    @staticmethod
    def backward(ctx, gx1, gz1):
        z, G, B = ctx.saved_tensors
        gz, gG, gB, gx0 = (torch.empty_like(z) for _ in range(4))
        glam = torch.zeros(1, dtype=torch.float64, device=z.device)
        gx1 = gx1.contiguous() if gx1 is not None else None
        gz1 = gz1.contiguous() if gz1 is not None else None
        _lib.uw_fista_step_backward(_prec(z), z.numel(), z.data_ptr(), G.data_ptr(), B.data_ptr(), ctx.tau, ctx.lam,
                                    ctx.beta, gx1.data_ptr() if gx1 is not None else None,
                                    gz1.data_ptr() if gz1 is not None else None, gz.data_ptr(), gG.data_ptr(),
                                    gB.data_ptr(), gx0.data_ptr(), glam.data_ptr(), _stream())
        lt = ctx.lam_like
        g_lam = glam.reshape(lt.shape).to(device=lt.device, dtype=lt.dtype) if lt is not None else None
        return gz, gG, gB, gx0, g_lam, None, None


class _HalfSqDist(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a, b):
        a, b = a.contiguous(), b.contiguous()
        d = torch.empty_like(a)
        _lib.uw_axpby(_prec(a), a.numel(), 1.0, a.data_ptr(), -1.0, b.data_ptr(), d.data_ptr(), _stream())
        out = torch.empty(1, dtype=torch.float64, device=a.device)
        _lib.uw_dot(_prec(a), a.numel(), d.data_ptr(), d.data_ptr(), out.data_ptr(), _stream())
        ctx.save_for_backward(d)
        return (0.5 * out).reshape(())

    @staticmethod
    def backward(ctx, g):
        (d,) = ctx.saved_tensors
        s = float(g)
        ga, gb = torch.empty_like(d), torch.empty_like(d)
        _lib.uw_axpby(_prec(d), d.numel(), s, d.data_ptr(), 0.0, None, ga.data_ptr(), _stream())
        _lib.uw_axpby(_prec(d), d.numel(), -s, d.data_ptr(), 0.0, None, gb.data_ptr(), _stream())
        return ga, gb


def half_sq_dist(a, b):
    """1/2 ||a - b||^2 as an FP64 scalar tensor (differentiable in a and b)."""
    return _HalfSqDist.apply(a, b)


def dot64(a, b):
    """sum a_i b_i accumulated in FP64 on the device (not differentiable)."""
    a, b = a.contiguous(), b.contiguous()
    out = torch.empty(1, dtype=torch.float64, device=a.device)
    _lib.uw_dot(_prec(a), a.numel(), a.data_ptr(), b.data_ptr(), out.data_ptr(), _stream())
    return out.reshape(())


def momentum_schedule(iters):
    """FISTA's beta_k = (t_k - 1) / t_{k+1}, t_0 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2)) / 2."""
    t, betas = 1.0, []
    for _ in range(iters):
        t1 = 0.5 * (1.0 + math.sqrt(1.0 + 4.0 * t * t))
        betas.append((t - 1.0) / t1)
        t = t1
    return betas


def fista(plan, y, lam, iters=100, tau=1.0, precision=None, checkpoint=True, x0=None):
    """Unrolled FISTA for min_x 1/2 ||P_Omega U x - y||^2 + lam ||x||_1.

    y: samples (m,) on the device; lam: float or 0-d tensor (then the result
    is differentiable in lam); returns x after `iters` iterations (shape
    M^d).  Differentiable in y and lam through every iteration; with
    `checkpoint` the backward pass recomputes each iteration's two products
    instead of storing them."""
    shape = (plan.M,) * plan.d
    B = adjoint_op(plan, y, precision)                      # U^* P^* y
    x = torch.zeros(shape, dtype=y.dtype, device=y.device) if x0 is None else x0
    z = x
    for beta in momentum_schedule(iters):
        def body(z, x, B, lam, beta=beta):
            G = adjoint_op(plan, forward_op(plan, z, precision), precision)
            return _FistaStep.apply(z, G, B, x, lam, tau, beta)
        if checkpoint and torch.is_grad_enabled():
            x, z = _checkpoint(body, z, x, B, lam, use_reentrant=False)
        else:
            x, z = body(z, x, B, lam)
    return x


def _axpby(alpha, a, beta, b, out):
    _lib.uw_axpby(_prec(a), a.numel(), float(alpha), a.data_ptr(), float(beta),
                  b.data_ptr() if b is not None else None, out.data_ptr(), _stream())


def cg_normal(plan, y, iters=50, tol=0.0, precision=None, x0=None):
    """Conjugate gradients for min_x ||P_Omega U x - y||^2 (generalised
    sampling, Sec. 1.2): the operator A = U^* P_Omega^* P_Omega U is
    symmetric positive semi-definite, so CG on A x = U^* P_Omega^* y converges
    to the least-squares solution (on the range of A^*).  Every product is a
    library call; the inner products are FP64 device reductions (uw_dot) and
    the vector updates uw_axpby.  Stops after `iters` iterations or when
    ||r|| <= tol ||b||.  Returns (x, number of iterations, ||r|| / ||b||)."""
    shape = (plan.M,) * plan.d
    b = plan.adjoint(y.contiguous(), precision=precision)
    x = torch.zeros(shape, dtype=y.dtype, device=y.device) if x0 is None else x0.clone()
    if x0 is None:
        r = b.clone()
    else:
        r = torch.empty_like(b)
        _axpby(1.0, b, -1.0, plan.adjoint(plan.forward(x, precision=precision), precision=precision), r)
    bb = float(dot64(b, b))
    rr = float(dot64(r, r))
    p = r.clone()
    k = 0
    while k < iters and bb > 0 and rr > (tol * tol) * bb:
        Ap = plan.adjoint(plan.forward(p, precision=precision), precision=precision)
        pAp = float(dot64(p, Ap))
        if pAp <= 0:
            break
        alpha = rr / pAp
        x1, r1, p1 = torch.empty_like(x), torch.empty_like(r), torch.empty_like(p)
        _axpby(1.0, x, alpha, p, x1)
        _axpby(1.0, r, -alpha, Ap, r1)
        rr_new = float(dot64(r1, r1))
        _axpby(1.0, r1, rr_new / rr, p, p1)
        x, r, p, rr = x1, r1, p1, rr_new
        k += 1
    return x, k, (rr / bb) ** 0.5 if bb > 0 else 0.0
