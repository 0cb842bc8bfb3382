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


class NewtonOracle(AugLagOracle):
    """The projected Newton-CG step of include/opf_al.h (opf_al_newton), in
    the steps' order, with the C oracle's callbacks and scipy's sparse
    products (TEST INFRASTRUCTURE ONLY, as above):

        x = clip(x, xl, xu),
        c = g(x), s = c + lambda / rho, d = s - clip(s, gl, gu), mu = rho d,
        D_i = 1 where s_i lies outside [gl_i, gu_i] (else 0),
        G = grad f(x) + J^T mu,
        K = H(x; mu, sigma = 1) + rho J^T diag(D) J   (H: Lagrangian Hessian),
        free F_j unless (x_j <= xl_j and G_j > 0) or (x_j >= xu_j and G_j < 0),
        Jacobi diagonal M_j = K_jj (1 where K_jj <= 1e-12);
    preconditioned conjugate gradients (diagonal M (1 + delta)) on
    (K + delta diag(M)) p = -G over the free entries, at most `cg_iters`
    iterations, stopping at non-positive curvature (the first direction
    itself is taken if that happens at once) or when r^T z falls below 1e-24
    of its first value; p scaled by 1 / max|p_j| where that is above 1 (no
    entry moves by more than 1 in one step); then x_t = clip(x + a_t p) for
    a_t = 1, 1/2, ...,
    1/128 and the largest a_t with L(x_t) <= L(x) + 1e-4 a_t G^T p is taken,
    else the a_t of least L(x_t) if it is below L(x), else no move. The
    Levenberg-Marquardt weight delta (1e-2 at first) is divided by 4 after a
    full step and multiplied by 10 after a step of 1/8 or less (or none),
    kept within [1e-8, 1e4].
    """

    NLS = 8
    DELTA0 = 1e-2

    def __init__(self, O, rho: float, lr: float):
        super().__init__(O, rho, lr)
        self.delta = self.DELTA0

    def system(self, x, lam):
        """(G, K, D, free mask, Jacobi diagonal M) of the step at x."""
        O, rho = self.O, self.rho
        c = O.cons(x)
        s = c + lam / rho
        mu = rho * (s - np.clip(s, self.gl, self.gu))
        D = ((s < self.gl) | (s > self.gu)).astype(np.float64)
        m, n = len(self.gl), len(x)
        J = sp.csr_matrix((O.jac(x), (self.rows, self.cols)), shape=(m, n))
        G = O.grad(x) + J.T @ mu
        hr, hc = O.hess_pattern()
        Hl = sp.csr_matrix((O.hess(x, mu, 1.0), (hr, hc)), shape=(n, n))
        K = (Hl + sp.tril(Hl, -1).T + rho * (J.T @ sp.diags(D) @ J)).tocsr()
        F = ~(((x <= self.xl) & (G > 0)) | ((x >= self.xu) & (G < 0)))
        Mj = K.diagonal().copy()
        Mj[Mj <= 1e-12] = 1.0
        return G, K, D, F, Mj

    def newton_step(self, x, lam, cg_iters):
        x = np.clip(np.array(x, dtype=np.float64), self.xl, self.xu)
        G, K, _, F, Mj = self.system(x, lam)
        dl = self.delta
        Kd = K + sp.diags(dl * Mj)
        p = pcg(lambda v: Kd @ v, G, F, Mj * (1.0 + dl), cg_iters)
        pm = float(np.max(np.abs(p))) if len(p) else 0.0
        if pm > 1.0:  # no entry moves by more than 1 (per-unit) in one step
            p = p * (1.0 / pm)
        L0 = self.value(x, lam)
        gp = float(G @ p)
        trials = [self.value(np.clip(x + 0.5 ** t * p, self.xl, self.xu), lam) for t in range(self.NLS)]
        pick = next((t for t in range(self.NLS) if trials[t] <= L0 + 1e-4 * 0.5 ** t * gp), None)
        if pick is None:
            best = int(np.argmin(trials))
            pick = best if trials[best] < L0 else None
        # Levenberg-Marquardt weight of the next step
        if pick == 0:
            self.delta = dl / 4.0
        elif pick is None or pick > 2:
            self.delta = dl * 10.0
        self.delta = min(max(self.delta, 1e-8), 1e4)
        xn = x if pick is None else np.clip(x + 0.5 ** pick * p, self.xl, self.xu)
        return xn, self.stats(xn, lam), p


def pcg(Kmul, G, F, Mj, iters):
    """Jacobi-preconditioned conjugate gradients on K p = -G over the entries
    where F holds (the others stay 0), from p = 0: at most `iters`
    iterations; stops at d^T K d <= 0 (returning the first direction itself
    if that happens at once) or when r^T z falls below 1e-24 of its first
    value."""
    r = np.where(F, -G, 0.0)
    z = r / Mj
    d = z.copy()
    rz = float(r @ z)
    rz0 = rz
    p = np.zeros(len(G))
    if rz == 0.0:
        return p
    for k in range(iters):
        q = np.where(F, Kmul(d), 0.0)
        dq = float(d @ q)
        if dq <= 0.0:
            return d.copy() if k == 0 else p
        a = rz / dq
        p = p + a * d
        r = r - a * q
        z = r / Mj
        rz_new = float(r @ z)
        if rz_new <= 1e-24 * rz0:
            return p
        d = z + (rz_new / rz) * d
        rz = rz_new
    return p
