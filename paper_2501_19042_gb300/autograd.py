"""``torch.autograd.Function`` over the unrolled safety filter.

Forward: ``sf_project_train`` (K iterations, checkpoints every
``checkpoint_every``); backward: ``sf_project_backward`` (hand-written adjoint
kernel). Outputs are the K-th iterate (xi, lambda), the fixed-point residual
sum per sample (first term of Eq. NN_loss) and the final primal residual
(not differentiable).
"""
from __future__ import annotations

import torch


class _SFUnroll(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xi_bar, xi0, lam0, sf, start, goal, K, n_robots, n_samples):
        out, fp, ckpt = sf.project_train(xi_bar.detach().contiguous(), start, goal, K, n_robots=n_robots,
                                         n_samples=n_samples,
                                         xi0=None if xi0 is None else xi0.detach().contiguous(),
                                         lam0=None if lam0 is None else lam0.detach().contiguous())
        ctx.sf, ctx.K, ctx.nr, ctx.ns = sf, K, n_robots, n_samples
        ctx.init_from_xi_bar = xi0 is None
        ctx.has_xi0, ctx.has_lam0 = xi0 is not None, lam0 is not None
        ctx.save_for_backward(xi_bar.detach().contiguous(), start, goal, ckpt)
        ctx.mark_non_differentiable(out.residual)
        return out.xi, out.lam, fp, out.residual

    @staticmethod
    def backward(ctx, g_xi, g_lam, g_fp, _g_res):
        xi_bar, start, goal, ckpt = ctx.saved_tensors
        f = lambda t: None if t is None else t.contiguous().float()
        gx0, gl0, gxb = ctx.sf.project_backward(xi_bar, start, goal, ctx.K, ckpt, grad_xi=f(g_xi),
                                                grad_lam=f(g_lam), grad_fp=f(g_fp),
                                                init_from_xi_bar=ctx.init_from_xi_bar, n_robots=ctx.nr,
                                                n_samples=ctx.ns)
        return (gxb, gx0 if ctx.has_xi0 else None, gl0 if ctx.has_lam0 else None,
                None, None, None, None, None, None)


def sf_unroll(sf, xi_bar, start, goal, K: int, xi0=None, lam0=None, n_robots=None, n_samples=None):
    """Differentiable K-iteration safety filter. ``sf`` is a ``SafetyFilter``
    created with ``checkpoint_every > 0``. Returns (xi^K, lambda^K,
    fixed-point residual sum per sample, final ||r_p|| per sample)."""
    return _SFUnroll.apply(xi_bar, xi0, lam0, sf, start, goal, K, n_robots, n_samples)


class _EqProject(torch.autograd.Function):
    """The decoders' QP layer as a differentiable op: forward
    ``sf_eq_project``, backward ``sf_eq_project_backward`` (dL/dxi' = Pi g).
    The boundary values (start / goal) are conditioning inputs and get no
    gradient here; ``SafetyFilter.eq_project_backward`` returns dL/db per row."""

    @staticmethod
    def forward(ctx, xi_prime, sf, start, goal, n_robots, n_samples):
        out = sf.eq_project(xi_prime.detach().contiguous(), start, goal, n_robots=n_robots, n_samples=n_samples)
        ctx.sf, ctx.nr, ctx.ns = sf, n_robots, n_samples
        ctx.save_for_backward(start, goal)
        return out

    @staticmethod
    def backward(ctx, g):
        start, goal = ctx.saved_tensors
        gin, _ = ctx.sf.eq_project_backward(g.contiguous().float(), start, goal, n_robots=ctx.nr, n_samples=ctx.ns)
        return gin, None, None, None, None, None


def eq_project(sf, xi_prime, start, goal, n_robots=None, n_samples=None):
    """Differentiable projection of decoder outputs xi' onto the boundary
    conditions (Sec. III-A / B); the layout is that of xi_bar."""
    return _EqProject.apply(xi_prime, sf, start, goal, n_robots, n_samples)
