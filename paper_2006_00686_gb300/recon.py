"""Reconstruction loops on top of the projector: SIRT, ordered-subset SIRT, Tikhonov-regularised
least squares by CGLS, and gradient-descent least squares through autograd.

All of them only compose the CUDA forward and adjoint (through the C ABI) with elementwise
torch operations on the device -- the reconstruction use the paper's method is built for
(Section 1: iterative methods need the transform and its adjoint many times).  The SIRT
iteration can be captured once in a CUDA graph and replayed.
"""
from __future__ import annotations

import numpy as np
import torch

from .xray import Projector, project


class SIRT:
    """x <- x + relax * C A^T R (b - A x), R = 1/(A 1), C = 1/(A^T 1) (zero where the row or
    column sum vanishes).  For 0 < relax < 2 the R-weighted residual ||b - A x||_R never
    increases."""

    def __init__(self, proj: Projector, b: torch.Tensor, relax: float = 1.0):
        self.P, self.b, self.relax = proj, b.contiguous(), float(relax)
        g = proj.geom
        batch = b.shape[0] if b.dim() == len(g.sino_shape()) + 1 else None
        dev = b.device
        ones_img = torch.ones(g.image_shape(batch), device=dev)
        ones_sino = torch.ones(g.sino_shape(batch), device=dev)
        row = proj.forward(ones_img)
        col = proj.adjoint(ones_sino)
        self.R = torch.where(row > 0, 1.0 / row.clamp_min(1e-30), torch.zeros_like(row))
        self.C = torch.where(col > 0, 1.0 / col.clamp_min(1e-30), torch.zeros_like(col))
        self.x = torch.zeros(g.image_shape(batch), device=dev)
        self.r = torch.empty_like(b)  # residual b - A x
        self.Ax = torch.empty_like(b)
        self.upd = torch.empty_like(self.x)
        self._graph = None

    def step(self):
        self.P.forward(self.x, out=self.Ax)
        torch.sub(self.b, self.Ax, out=self.r)
        self.r.mul_(self.R)
        self.P.adjoint(self.r, out=self.upd)
        self.x.addcmul_(self.C, self.upd, value=self.relax)

    def residual_norm(self) -> float:
        """||b - A x||_R for the current x (float64 reduction)."""
        self.P.forward(self.x, out=self.Ax)
        d = (self.b - self.Ax).double()
        return float((d * d * self.R.double()).sum().sqrt())

    def capture(self):
        """Capture one iteration in a CUDA graph (replayed by run(graph=True))."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.step()  # warm-up outside the capture
        torch.cuda.current_stream().wait_stream(s)
        self.x.zero_()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step()
        self._graph = g
        return g

    def run(self, n_iter: int, graph: bool = False, track: bool = False):
        res = [self.residual_norm()] if track else []
        if graph and self._graph is None:
            self.capture()
        for _ in range(n_iter):
            if graph:
                self._graph.replay()
            else:
                self.step()
            if track:
                res.append(self.residual_norm())
        return self.x, res


def lsq_gradient_descent(proj: Projector, b: torch.Tensor, n_iter: int, step: float,
                         x0: torch.Tensor | None = None):
    """Minimise 0.5 ||A x - b||^2 by gradient descent with autograd (backward = adjoint)."""
    g = proj.geom
    x = (torch.zeros(g.image_shape(), device=b.device) if x0 is None else x0.clone()).requires_grad_(True)
    losses = []
    for _ in range(n_iter):
        loss = 0.5 * ((project(x, proj) - b) ** 2).sum()
        x.grad = None
        loss.backward()
        losses.append(float(loss.detach()))
        with torch.no_grad():
            x -= step * x.grad
    return x.detach(), losses


def subset_views(n_views: int, n_subsets: int) -> list:
    """Interleaved view subsets: subset s holds views s, s + S, s + 2S, ... (each subset spans
    the whole angular range)."""
    return [np.arange(s, n_views, n_subsets, dtype=np.int64) for s in range(n_subsets)]


class OSSIRT:
    """Ordered-subset SIRT: one sweep applies, subset by subset,
    x <- x + relax * C_s A_s^T R_s (b_s - A_s x), with A_s the transform restricted to the
    views of subset s and R_s, C_s its inverse row and column sums.  Each subset is a
    Projector of its own (a view subset of the scan), so every update runs the CUDA kernels."""

    def __init__(self, geom, b: torch.Tensor, n_subsets: int, relax: float = 1.0):
        self.geom, self.relax = geom, float(relax)
        self.subsets = subset_views(geom.n_views, n_subsets)
        dev = b.device
        sino = b.reshape(geom.n_views, -1)
        self.P, self.b, self.R, self.C = [], [], [], []
        for idx in self.subsets:
            g = geom.subset_views(idx)
            P = Projector(g)
            bs = sino[torch.from_numpy(idx).to(dev)].reshape(g.sino_shape()).contiguous()
            row = P.forward(torch.ones(g.image_shape(), device=dev))
            col = P.adjoint(torch.ones(g.sino_shape(), device=dev))
            self.P.append(P)
            self.b.append(bs)
            self.R.append(torch.where(row > 0, 1.0 / row.clamp_min(1e-30), torch.zeros_like(row)))
            self.C.append(torch.where(col > 0, 1.0 / col.clamp_min(1e-30), torch.zeros_like(col)))
        self.x = torch.zeros(geom.image_shape(), device=dev)

    def sweep(self):
        for P, b, R, C in zip(self.P, self.b, self.R, self.C):
            r = (b - P.forward(self.x)) * R
            self.x.addcmul_(C, P.adjoint(r), value=self.relax)

    def run(self, n_sweeps: int):
        for _ in range(n_sweeps):
            self.sweep()
        return self.x

    def close(self):
        for P in self.P:
            P.close()


def cgls(proj: Projector, b: torch.Tensor, n_iter: int, lam: float = 0.0, x0: torch.Tensor | None = None):
    """Tikhonov-regularised least squares, min ||A x - b||^2 + lam ||x||^2, by CGLS (conjugate
    gradients on (A^T A + lam I) x = A^T b without forming A^T A).  Returns x and the norms
    ||A^T (b - A x) - lam x|| of the normal-equation residual per iteration (float64
    reductions)."""
    g = proj.geom
    x = torch.zeros(g.image_shape(), device=b.device) if x0 is None else x0.clone()
    r = b - proj.forward(x)
    s = proj.adjoint(r) - lam * x
    p = s.clone()
    gamma = float((s.double() ** 2).sum())
    norms = [gamma ** 0.5]
    for _ in range(n_iter):
        if gamma == 0.0:
            break
        q = proj.forward(p)
        delta = float((q.double() ** 2).sum()) + lam * float((p.double() ** 2).sum())
        if delta <= 0.0:
            break
        alpha = gamma / delta
        x.add_(p, alpha=alpha)
        r.sub_(q, alpha=alpha)
        s = proj.adjoint(r) - lam * x
        gamma_new = float((s.double() ** 2).sum())
        p.mul_(gamma_new / gamma).add_(s)
        gamma = gamma_new
        norms.append(gamma ** 0.5)
    return x, norms

