"""Learned start vector for rKS on a parametric operator family: FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring): the product path never
imports this module.

The paper draws the start vector of Algorithm 1 at random (Sec. 2.1: any
vector with components along the wanted eigenvectors).  For a family of
operators A(theta) whose coefficient fields are known, a small convolutional
network can map the fields to a start vector u_1 that already lies close to
the wanted invariant subspace of A(theta).  This module is the plain FP64
reference of that network, its loss and its gradients, written in the order
of the definitions below; the library's CUDA kernels must reproduce it.

Network (a 4-level U-Net, 32 channels, 3x3 convolutions with zero padding,
ReLU, 2x2 average pooling, 2x nearest upsampling, additive skips):

  e0 = R(C2(R(C1(x))))                       H x W      (C1: 3 -> 32)
  e1 = R(C4(R(C3(P(e0)))))                   H/2
  e2 = R(C6(R(C5(P(e1)))))                   H/4
  e3 = R(C8(R(C7(P(e2)))))                   H/8        (the fourth level)
  d2 = R(C10(R(C9(U(e3) + e2))))             H/4
  d1 = R(C12(R(C11(U(d2) + e1))))            H/2
  d0 = R(C14(R(C13(U(d1) + e0))))            H
  u  = C15(d0)                               H x W      (C15: 32 -> 1)

with R = max(0, .), P = 2x2 mean, U = 2x nearest copy, and C_l(z)[o] =
b_l[o] + sum_{c, dy, dx} W_l[o, c, dy, dx] z[c, y + dy - 1, x + dx - 1]
(zero outside the grid).  Input channels: log nu, bx / 50, by / 50.

Loss (subspace capture): with Q (n x q) an orthonormal basis of the span of
the wanted Schur vectors rKS computed for this operator and u flattened in
the solver's order (x fastest),

  L(u) = 1 - ||Q^T u||^2 / ||u||^2,      0 <= L <= 1,

dL/du = -2 Q Q^T u / ||u||^2 + 2 ||Q^T u||^2 u / ||u||^4.

The library computes with FP16 weights (FP32 masters) and FP32 activations
and accumulation; this oracle takes the same FP16-rounded weights as FP64
numbers, so the two differ by FP32 rounding only.
"""
from __future__ import annotations

import numpy as np

CH = 32
NCONV = 15
# (input channels, output channels) of C1 .. C15
SHAPES = [(3, CH)] + [(CH, CH)] * 13 + [(CH, 1)]


def param_sizes():
    """Sizes of (W_l, b_l) for l = 1..15, in storage order W_1, b_1, W_2, ..."""
    out = []
    for ci, co in SHAPES:
        out += [co * ci * 9, co]
    return out


def unpack(theta: np.ndarray):
    """Flat parameter vector -> list of (W (co, ci, 3, 3), b (co,))."""
    layers, o = [], 0
    for ci, co in SHAPES:
        W = theta[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = theta[o:o + co]
        o += co
        layers.append((W, b))
    return layers


def conv3x3(z, W, b):
    """C(z)[o, y, x] = b[o] + sum_{c,dy,dx} W[o,c,dy,dx] z[c, y+dy-1, x+dx-1]."""
    c, H, Wd = z.shape
    zp = np.zeros((c, H + 2, Wd + 2))
    zp[:, 1:-1, 1:-1] = z
    out = np.repeat(b[:, None, None], H, axis=1).repeat(Wd, axis=2).astype(np.float64)
    for dy in range(3):
        for dx in range(3):
            out += np.einsum("oc,chw->ohw", W[:, :, dy, dx], zp[:, dy:dy + H, dx:dx + Wd])
    return out


def conv3x3_backward(z, W, g):
    """Gradients of sum(g * C(z)) w.r.t. z, W and b."""
    c, H, Wd = z.shape
    zp = np.zeros((c, H + 2, Wd + 2))
    zp[:, 1:-1, 1:-1] = z
    gz = np.zeros((c, H + 2, Wd + 2))
    gW = np.zeros_like(W)
    for dy in range(3):
        for dx in range(3):
            gW[:, :, dy, dx] = np.einsum("ohw,chw->oc", g, zp[:, dy:dy + H, dx:dx + Wd])
            gz[:, dy:dy + H, dx:dx + Wd] += np.einsum("oc,ohw->chw", W[:, :, dy, dx], g)
    return gz[:, 1:-1, 1:-1], gW, g.sum(axis=(1, 2))


def pool(z):
    c, H, Wd = z.shape
    return z.reshape(c, H // 2, 2, Wd // 2, 2).mean(axis=(2, 4))


def pool_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) / 4.0


def up(z):
    return np.repeat(np.repeat(z, 2, axis=1), 2, axis=2)


def up_backward(g):
    c, H, Wd = g.shape
    return g.reshape(c, H // 2, 2, Wd // 2, 2).sum(axis=(2, 4))


def relu(z):
    return np.maximum(z, 0.0)


def forward(theta: np.ndarray, x: np.ndarray):
    """u (H x W) and the activations the backward pass needs."""
    L = unpack(theta)
    acts = {}

    def block(z, l, tag):               # R(C_{l+1}(R(C_l(z))))
        a = relu(conv3x3(z, *L[l - 1]))
        o = relu(conv3x3(a, *L[l]))
        acts[tag] = (z, a, o)
        return o

    e0 = block(x, 1, "e0")
    e1 = block(pool(e0), 3, "e1")
    e2 = block(pool(e1), 5, "e2")
    e3 = block(pool(e2), 7, "e3")
    d2 = block(up(e3) + e2, 9, "d2")
    d1 = block(up(d2) + e1, 11, "d1")
    d0 = block(up(d1) + e0, 13, "d0")
    u = conv3x3(d0, *L[14])[0]
    return u, acts


def loss(u: np.ndarray, Q: np.ndarray):
    """L = 1 - ||Q^T u||^2 / ||u||^2 and dL/du (u as H x W, Q as n x q)."""
    v = u.ravel()
    uu = v @ v
    c = Q.T @ v
    cc = c @ c
    L = 1.0 - cc / uu
    g = -2.0 * (Q @ c) / uu + 2.0 * cc * v / uu ** 2
    return L, g.reshape(u.shape)


def backward(theta: np.ndarray, acts, g_u: np.ndarray) -> np.ndarray:
    """dL/dtheta (flat, storage order) from dL/du."""
    L = unpack(theta)
    grads = [None] * NCONV

    def conv_back(z, l, g):             # through C_l: returns dL/dz
        gz, gW, gb = conv3x3_backward(z, L[l - 1][0], g)
        grads[l - 1] = (gW, gb)
        return gz

    def block_back(tag, l, g):          # through R(C_{l+1}(R(C_l(z)))): returns dL/dz
        z, a, o = acts[tag]
        g = g * (o > 0)
        g = conv_back(a, l + 1, g)
        g = g * (a > 0)
        return conv_back(z, l, g)

    d0 = acts["d0"][2]
    g = conv_back(d0, 15, g_u[None])
    g = block_back("d0", 13, g)              # g = dL/d(U(d1) + e0)
    g_e0 = g.copy()
    g = block_back("d1", 11, up_backward(g))
    g_e1 = g.copy()
    g = block_back("d2", 9, up_backward(g))
    g_e2 = g.copy()
    g = block_back("e3", 7, up_backward(g))  # dL/dP(e2)
    g_e2 += pool_backward(g)
    g = block_back("e2", 5, g_e2)
    g_e1 += pool_backward(g)
    g = block_back("e1", 3, g_e1)
    g_e0 += pool_backward(g)
    block_back("e0", 1, g_e0)
    return np.concatenate([np.concatenate([gW.ravel(), gb]) for gW, gb in grads])


def loss_and_grad(theta: np.ndarray, x: np.ndarray, Q: np.ndarray):
    u, acts = forward(theta, x)
    L, gu = loss(u, Q)
    return L, backward(theta, acts, gu), u


def adam(theta, m, v, grad, t: int, lr: float, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015), bias-corrected, in place; t >= 1."""
    m[:] = b1 * m + (1 - b1) * grad
    v[:] = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    theta[:] = theta - lr * mh / (np.sqrt(vh) + eps)
