"""Reconstruction loops on top of the projector: SIRT and gradient-descent least squares.

Both only compose the CUDA forward and adjoint (through the C ABI) with elementwise torch
operations on the device.  The SIRT iteration can be captured once in a CUDA graph and
replayed.
"""
from __future__ import annotations

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
