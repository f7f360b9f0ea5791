"""Test-only plain-PyTorch FP64 unroll of the SF iteration, for autograd
checks of the hand-written adjoint.

It is written from the paper's steps (Appendix): positions from the basis,
the closed-form projection of every pair / velocity / acceleration row, the
lambda step (minus-sign reading) and the KKT solve of the xi step, with the
dense per-axis KKT inverse built here from F^T F = (N I - 1 1^T) (x) P^T P +
I (x) (Pd^T Pd + Pdd^T Pdd). Its own forward is checked against the oracle in
the tests before its gradients are used.
"""
from __future__ import annotations

import numpy as np
import torch


class TorchSF:
    def __init__(self, P, Pd, Pdd, start, goal, rho, a, b, v_max, a_max, workspace=None):
        dt = torch.float64
        self.P, self.Pd, self.Pdd = (torch.as_tensor(m, dtype=dt) for m in (P, Pd, Pdd))
        self.T, self.nv = self.P.shape
        start = np.asarray(start, np.float64)
        goal = np.asarray(goal, np.float64)
        self.N, self.dim = start.shape
        self.rho, self.a, self.b = rho, a, b
        self.v_max, self.a_max = v_max, a_max
        self.ws = workspace          # None or (centre, a_w, b_w)
        N, nv = self.N, self.nv
        pairs = [(i, j) for i in range(N) for j in range(i + 1, N)]
        self.pi = torch.tensor([p[0] for p in pairs], dtype=torch.long)
        self.pj = torch.tensor([p[1] for p in pairs], dtype=torch.long)
        Q = self.P.T @ self.P
        G = torch.zeros_like(Q)
        if v_max > 0:
            G = G + self.Pd.T @ self.Pd
        if a_max > 0:
            G = G + self.Pdd.T @ self.Pdd
        if workspace is not None:
            G = G + Q                 # workspace rows I (x) P
        L = N * torch.eye(N, dtype=dt) - torch.ones((N, N), dtype=dt)
        H = torch.kron(L, Q) + torch.kron(torch.eye(N, dtype=dt), G)
        A1 = torch.stack([self.P[0], self.Pd[0], self.Pdd[0], self.P[-1], self.Pd[-1], self.Pdd[-1]])
        A = torch.kron(torch.eye(N, dtype=dt), A1)
        nc = N * nv
        Kmat = torch.zeros((nc + 6 * N, nc + 6 * N), dtype=dt)
        Kmat[:nc, :nc] = torch.eye(nc, dtype=dt) + rho * H
        Kmat[:nc, nc:] = A.T
        Kmat[nc:, :nc] = A
        Kinv = torch.linalg.inv(Kmat)
        self.Sx, self.Rx = Kinv[:nc, :nc], Kinv[:nc, nc:]
        self.H = H
        bvec = np.zeros((self.dim, N, 6))
        for ax in range(self.dim):
            bvec[ax, :, 0] = start[:, ax]
            bvec[ax, :, 3] = goal[:, ax]
        self.bvec = torch.as_tensor(bvec.reshape(self.dim, N * 6), dtype=dt)

    def _states(self, xi, M):
        return torch.einsum("tk,sdnk->sdnt", M, xi)

    def project_q(self, xi):
        """q = e - F xi for every block, as time-domain tensors. e is built
        explicitly so that autograd sees de/ddelta = 0 at delta = 0 (the
        tie-break point) and I on inactive rows."""
        p = self._states(xi, self.P)
        D = p[:, :, self.pi, :] - p[:, :, self.pj, :]               # [S, dim, npair, T]
        scale = torch.tensor([1 / self.a] * 2 + [1 / self.b], dtype=torch.float64)[: self.dim]
        s2 = ((D * scale[None, :, None, None]) ** 2).sum(1, keepdim=True)
        zero = s2 == 0
        inv = torch.where(zero, torch.ones_like(s2), s2).rsqrt()
        inside = (s2 < 1) & ~zero
        e = torch.where(inside, D * inv, D)
        tie = torch.zeros_like(D)
        tie[:, -1 if self.dim == 3 else 0] = self.b if self.dim == 3 else self.a
        e = torch.where(zero.expand_as(D), tie, e)
        out = {"pair": e - D}
        for name, M, r in (("vel", self.Pd, self.v_max), ("acc", self.Pdd, self.a_max)):
            if r > 0:
                v = self._states(xi, M)
                n2 = (v ** 2).sum(1, keepdim=True)
                outside = n2 > r * r
                nrm = torch.where(outside, n2, torch.ones_like(n2)).sqrt()
                ev = torch.where(outside, r * v / nrm, v)
                out[name] = ev - v
        if self.ws is not None:
            c = torch.tensor(np.asarray(self.ws[0], np.float64)[: self.dim], dtype=torch.float64)
            wax = torch.tensor([self.ws[1]] * 2 + [self.ws[2]], dtype=torch.float64)[: self.dim]
            d = p - c[None, :, None, None]
            s2 = ((d / wax[None, :, None, None]) ** 2).sum(1, keepdim=True)
            outside = s2 > 1
            sc = torch.where(outside, s2, torch.ones_like(s2)).rsqrt()
            out["ws"] = torch.where(outside, d * sc - d, torch.zeros_like(d))
        return out

    def Ft(self, q):
        S = q["pair"].shape[0]
        E = torch.zeros((S, self.dim, self.N, self.T), dtype=torch.float64)
        E = E.index_add(2, self.pi, q["pair"]).index_add(2, self.pj, -q["pair"])
        g = torch.einsum("tk,sdnt->sdnk", self.P, E)
        if "vel" in q:
            g = g + torch.einsum("tk,sdnt->sdnk", self.Pd, q["vel"])
        if "acc" in q:
            g = g + torch.einsum("tk,sdnt->sdnk", self.Pdd, q["acc"])
        if "ws" in q:
            g = g + torch.einsum("tk,sdnt->sdnk", self.P, q["ws"])
        return g

    def step(self, xi, lam, xi_bar):
        """One f_FP step (Appendix): e from xi, lambda step, xi step."""
        S = xi.shape[0]
        q = self.project_q(xi)
        g = self.Ft(q)                                   # F^T (e - F xi)
        lam2 = lam + self.rho * g
        Hx = torch.einsum("ij,sdj->sdi", self.H, xi.reshape(S, self.dim, -1))
        u = self.rho * (Hx + g.reshape(S, self.dim, -1)) + lam2.reshape(S, self.dim, -1) \
            + xi_bar.reshape(S, self.dim, -1)
        xi2 = torch.einsum("ij,sdj->sdi", self.Sx, u) + (self.Rx @ self.bvec.T).T[None]
        return xi2.reshape(xi.shape), lam2

    def unroll(self, xi0, lam0, xi_bar, K, fp_weight=0.0):
        xi, lam = xi0, lam0
        fp = torch.zeros(xi0.shape[0], dtype=torch.float64)
        for _ in range(K):
            xn, ln = self.step(xi, lam, xi_bar)
            if fp_weight:
                fp = fp + ((xn - xi) ** 2).flatten(1).sum(1) + ((ln - lam) ** 2).flatten(1).sum(1)
            xi, lam = xn, ln
        return xi, lam, fp
