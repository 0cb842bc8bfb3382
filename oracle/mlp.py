"""FP64 CPU oracle of the warm-start network and of its training loss.

TEST INFRASTRUCTURE ONLY (tests, bench CPU baseline): it judges the BF16
kernels of libopf's warm start and shares no code with them.

Network (the three-layer MLP with GELU of the warm start):
    h1 = gelu(W1 u + b1), h2 = gelu(W2 h1 + b2), y = W3 h2 + b3,
    gelu(z) = 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3)))   (tanh form)
Backward pass by the chain rule, written out layer by layer.
Output map: y = [ya | yv | yp | yq] (blocks padded to multiples of 128)
    gives x: va = s ya (0 at the reference bus), vm = (vmin + vmax)/2 + yv,
    pg = (pmin + pmax)/2 + (pmax - pmin)/2 yp, qg likewise, p, q = the
    flows at (va, vm).
Loss of one profile (with the C oracle for f, g and the bounds):
    L = f(x) + w (sum_i (g_i - clip(g_i, gl_i, gu_i))^2
                  + sum_j (x_j - clip(x_j, xl_j, xu_j))^2)
Parity status: forward/backward pinned by central differences and by the
erf form of GELU (the tanh form is within 1e-3 of it). point() pinned on a
two-bus lossless line: bounds mid-points and half ranges, the reference
angle, the padded block offsets, and p, q equal to the textbook lossless
flows. loss() pinned on the same line with every row, bound violation and
the quadratic cost written out by hand (tests/test_mlp_oracle.py); f and g
are the C oracle's, pinned in test_oracle_pins.
"""
from __future__ import annotations

import math

import numpy as np

K0 = math.sqrt(2.0 / math.pi)
K1 = 0.044715


def gelu(z):
    return 0.5 * z * (1.0 + np.tanh(K0 * (z + K1 * z ** 3)))


def gelu_grad(z):
    t = np.tanh(K0 * (z + K1 * z ** 3))
    return 0.5 * (1.0 + t) + 0.5 * z * (1.0 - t * t) * K0 * (1.0 + 3.0 * K1 * z * z)


def unpack(flat, n_in, hidden, n_out):
    o = 0
    out = []
    for shape in ((hidden, n_in), (hidden,), (hidden, hidden), (hidden,), (n_out, hidden), (n_out,)):
        k = int(np.prod(shape))
        out.append(np.asarray(flat[o:o + k], np.float64).reshape(shape))
        o += k
    return out


def forward(flat, U, n_in, hidden, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(flat, n_in, hidden, n_out)
    Z1 = U @ W1.T + b1
    H1 = gelu(Z1)
    Z2 = H1 @ W2.T + b2
    H2 = gelu(Z2)
    Y = H2 @ W3.T + b3
    return Y, (U, Z1, H1, Z2, H2)


def backward(flat, cache, dY, n_in, hidden, n_out):
    W1, b1, W2, b2, W3, b3 = unpack(flat, n_in, hidden, n_out)
    U, Z1, H1, Z2, H2 = cache
    dW3 = dY.T @ H2
    db3 = dY.sum(0)
    dZ2 = (dY @ W3) * gelu_grad(Z2)
    dW2 = dZ2.T @ H1
    db2 = dZ2.sum(0)
    dZ1 = (dZ2 @ W2) * gelu_grad(Z1)
    dW1 = dZ1.T @ U
    db1 = dZ1.sum(0)
    return np.concatenate([a.ravel() for a in (dW1, db1, dW2, db2, dW3, db3)])


def inputs(pd, qd, pd0, qd0, n_in):
    """u of each profile: (load / base load - 1) / 0.2 for Pd then Qd, zero
    where the base load is zero, zero-padded to n_in."""
    count, nload = pd.shape
    U = np.zeros((count, n_in))
    with np.errstate(divide="ignore", invalid="ignore"):
        up = np.where(pd0 > 0, (pd / np.where(pd0 > 0, pd0, 1.0) - 1.0) / 0.2, 0.0)
        uq = np.where(qd0 > 0, (qd / np.where(qd0 > 0, qd0, 1.0) - 1.0) / 0.2, 0.0)
    U[:, :nload] = up
    U[:, nload:2 * nload] = uq
    return U


def pad(v, q=128):
    return (v + q - 1) // q * q


def point(grid, y, va_scale, oracle_ctx):
    """x of one profile (single-period layout) from its network output y."""
    nb, ng, nl = grid.nbus, grid.ngen, grid.nbranch
    nbp, ngp = pad(nb), pad(ng)
    y = np.asarray(y, np.float64)
    va = va_scale * y[:nb]
    va[grid.ref_bus] = 0.0
    vm = 0.5 * (grid.bus_vmin + grid.bus_vmax) + y[nbp:nbp + nb]
    pg = 0.5 * (grid.gen_pmin + grid.gen_pmax) + 0.5 * (grid.gen_pmax - grid.gen_pmin) * y[2 * nbp:2 * nbp + ng]
    qg = 0.5 * (grid.gen_qmin + grid.gen_qmax) + 0.5 * (grid.gen_qmax - grid.gen_qmin) * \
        y[2 * nbp + ngp:2 * nbp + ngp + ng]
    x = np.concatenate([va, vm, pg, qg, np.zeros(4 * nl)])
    c = oracle_ctx.cons(x)
    # flow rows are p - P(v): at p = q = 0 they are -P(v)
    x[2 * nb + 2 * ng:2 * nb + 2 * ng + 2 * nl] = -np.concatenate([c[1:1 + nl], c[1 + 2 * nl:1 + 3 * nl]])
    x[2 * nb + 2 * ng + 2 * nl:] = -np.concatenate([c[1 + nl:1 + 2 * nl], c[1 + 3 * nl:1 + 4 * nl]])
    return x


def loss(grid, y, va_scale, penalty, oracle_ctx, bounds):
    """Loss of one profile at network output y (oracle_ctx built on that
    profile's loads; bounds = its (xl, xu, gl, gu))."""
    x = point(grid, y, va_scale, oracle_ctx)
    c = oracle_ctx.cons(x)
    xl, xu, gl, gu = bounds
    rho = c - np.clip(c, gl, gu)
    r = x - np.clip(x, xl, xu)
    return oracle_ctx.obj(x) + penalty * (float(rho @ rho) + float(r @ r))
