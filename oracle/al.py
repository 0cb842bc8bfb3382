"""FP64 CPU oracle of the augmented-Lagrangian loop (include/opf_al.h).

TEST INFRASTRUCTURE ONLY: it judges libopf's AL kernels and shares no code
with them. It takes the loop's steps in order with the C oracle's
callbacks (f, grad f, g and the sparse Jacobian, whose transpose-product is
a scipy sparse matvec):

    s = g(x) + lambda / rho,  d = s - clip(s, gl, gu),  mu = rho d
    L(x; lambda) = f(x) + sum(rho / 2 d^2 - lambda^2 / (2 rho))
    G = grad f(x) + J(x)^T mu
    Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on x, then
    x = clip(x, xl, xu);  outer update lambda = mu(x).

Adam's scale 1 / (sqrt(v_hat) + eps) is formed in FP32 (v_hat rounded to
FP32, then the correctly rounded square root, sum and reciprocal of IEEE
single precision), as the library defines it; the rest is FP64.

Pinned by tests/test_al_oracle.py: G against Richardson central differences
of L; L = f and mu = 0 at a point strictly inside every row's bounds with
lambda = 0; the update's fixed point (lambda = mu) at such a point.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


class AugLagOracle:
    def __init__(self, O, rho: float, lr: float):
        self.O, self.rho, self.lr = O, float(rho), float(lr)
        self.xl, self.xu, self.gl, self.gu = O.bounds()
        self.rows, self.cols = O.jac_pattern()
        self.m1 = np.zeros(len(self.xl))
        self.m2 = np.zeros(len(self.xl))
        self.k = 0

    def mu(self, x, lam):
        c = self.O.cons(x)
        s = c + lam / self.rho
        return self.rho * (s - np.clip(s, self.gl, self.gu)), c

    def value(self, x, lam):
        mu, _ = self.mu(x, lam)
        return self.O.obj(x) + float(np.sum(mu * mu) - np.sum(lam * lam)) / (2.0 * self.rho)

    def gradient(self, x, lam):
        mu, _ = self.mu(x, lam)
        J = sp.csr_matrix((self.O.jac(x), (self.rows, self.cols)), shape=(len(self.gl), len(x)))
        return self.O.grad(x) + J.T @ mu

    def stats(self, x, lam):
        mu, c = self.mu(x, lam)
        viol = float(np.max(np.maximum(np.maximum(self.gl - c, c - self.gu), 0.0)))
        f = self.O.obj(x)
        return np.array([f, viol, f + float(np.sum(mu * mu) - np.sum(lam * lam)) / (2.0 * self.rho)])

    def iterate(self, x, lam, iters):
        """`iters` Adam steps; returns the final x and its statistics."""
        x = np.array(x, dtype=np.float64, copy=True)
        for _ in range(iters):
            G = self.gradient(x, lam)
            self.k += 1
            self.m1 = 0.9 * self.m1 + 0.1 * G
            self.m2 = 0.999 * self.m2 + 0.001 * G * G
            v32 = (self.m2 / (1 - 0.999 ** self.k)).astype(np.float32)
            r = (np.float32(1.0) / (np.sqrt(v32) + np.float32(1e-8))).astype(np.float64)
            step = self.lr * (self.m1 / (1 - 0.9 ** self.k)) * r
            x = np.clip(x - step, self.xl, self.xu)
        return x, self.stats(x, lam)

    def update(self, x, lam):
        mu, _ = self.mu(x, lam)
        return mu, self.stats(x, lam)
