"""Training and use of the start-vector network on a parametric family.

Orchestration only: every computation runs in the library (rks_solve for the
training targets, rks_sketch_qr for their orthonormal bases, rks_ws_* for the
network's forward and backward passes, Adam and the start vector).

Family: the 2D upwind convection-diffusion operators of
``inputs.grf_convdiff2d_problem`` (diffusivity exp(GRF), correlation length
0.1; convection uniform in [0, 50]^2); the network reads the coefficient
planes of ``inputs.grf_member_fields``.
"""
from __future__ import annotations

import time

import numpy as np

from . import inputs as I
from . import rks


def solve_member(P, u1=None, prec: str = "df", want_basis: bool = False):
    """rKS on problem P to ||A x - l x|| / (||A||_1 ||x||) <= P.tol (thick
    restart keep = k).  Returns (info, wall seconds, n x k Schur basis or None)."""
    with rks.Solver.from_csr(P.A, P.k, P.p, P.d, which=P.which, zeta=P.zeta, seed=P.omega_seed, u1=u1,
                             keep=P.k, maxit=4000, prec=prec, **P.solver_opts()) as s:
        t0 = time.perf_counter()
        info = s.solve(allow_noconv=False)
        wall = time.perf_counter() - t0
        U = s.schur()[1][:, :P.k] if want_basis else None
    return info, wall, U


def target_basis(U, d: int = 64):
    """Euclidean-orthonormal basis (CUDA float32, rows = columns of Q) of the
    span of the Schur vectors U (n x k host FP64), by randomized Cholesky QR."""
    import torch
    K = torch.from_numpy(np.ascontiguousarray(U.T)).cuda()
    Q, _, _ = rks.sketch_qr(K, max(d, 2 * U.shape[1]), method="rcholqr")
    return Q.float().contiguous()


def make_samples(indices, seed0: int, N: int):
    """(fields on the device, target basis, solve info) for members seed0 + i."""
    import torch
    out = []
    for i in indices:
        P = I.grf_convdiff2d_problem(i, seed0=seed0, N=N)
        info, wall, U = solve_member(P, want_basis=True)
        x = torch.from_numpy(I.grf_member_fields(i, seed0=seed0, N=N)).cuda()
        out.append((x, target_basis(U), info, wall))
    return out


def train(net, samples, epochs: int, lr: float = 1e-3, batch: int = 8, seed: int = 0):
    """Minibatch Adam on the subspace-capture loss; returns the mean loss per epoch."""
    hist = []
    rng = np.random.default_rng(seed)
    for _ in range(epochs):
        order = rng.permutation(len(samples))
        losses = []
        for j, idx in enumerate(order):
            x, Q = samples[idx][0], samples[idx][1]
            losses.append(net.accumulate(x, Q))
            if (j + 1) % batch == 0 or j == len(order) - 1:
                net.step(lr)
        hist.append(float(np.mean(losses)))
    return hist


def capture(net, x, Q) -> float:
    """||Q^T u||^2 / ||u||^2 of the network's output u (1 - the loss)."""
    u = net.forward(x).double().ravel()
    return float(((Q.double() @ u) ** 2).sum() / (u @ u))
