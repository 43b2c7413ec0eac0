"""HoT surrogate network: features, forward, backward, Adam, in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper extracts the higher-order terms (Eq. hot_constitutive) from the
noisy DSMC moments.  This extension (not in the paper) learns them from
local, dimensionless quantities, so that the synthetic equations can use a
smooth estimate where Kn_GLL >= Kn_ref.

Inputs (12 per cell): the gradients of rho, u_x, u_y, T_t, T_r along x and y
(cell-centred differences as for the HoT), each made dimensionless with the
local mean free path lambda = mu(T)/(rho T) sqrt(pi T / 2):
    lambda d(rho)/rho,  lambda d(u)/sqrt(T),  lambda d(T_t)/T,  lambda d(T_r)/T
in the order (rho_x, rho_y, ux_x, ux_y, uy_x, uy_y, Tt_x, Tt_y, Tr_x, Tr_y),
then Kn_GLL and T_r / T_t.
Outputs (5 per cell): HoT_sigma_xx / p, HoT_sigma_xy / p, HoT_sigma_yy / p,
and the components of HoT_q_t and HoT_q_r along e = grad T / |grad T| (e = x
where grad T = 0), divided by p sqrt(T); p = rho T with T the total
temperature.
Network: 12 -> 64 -> 64 -> 64 -> 5, tanh on the hidden layers, linear
output; loss: mean over the training cells of the mean squared error of the
5 outputs; Adam (beta1 0.9, beta2 0.999, eps 1e-8).  Weights used by the
network may be rounded to bfloat16 (round to nearest even), as the GPU does.
"""
from __future__ import annotations

import math

import numpy as np

from .fields import F_RHO, F_TR, F_TT, F_U, gradient_of, mu_ref_of

SIZES = (12, 64, 64, 64, 5)
NPARAM = sum(SIZES[k] * SIZES[k + 1] + SIZES[k + 1] for k in range(4))


def unpack(theta: np.ndarray):
    """[(W1, b1), ..., (W4, b4)] with W_k of shape (out, in), views of theta."""
    out, o = [], 0
    for k in range(4):
        n_in, n_out = SIZES[k], SIZES[k + 1]
        W = theta[o:o + n_in * n_out].reshape(n_out, n_in)
        o += n_in * n_out
        b = theta[o:o + n_out]
        o += n_out
        out.append((W, b))
    return out


def init_params(seed: int = 0) -> np.ndarray:
    """Glorot-uniform weights, zero biases (numpy generator)."""
    rng = np.random.default_rng(seed)
    theta = np.zeros(NPARAM)
    for W, b in unpack(theta):
        lim = math.sqrt(6.0 / (W.shape[0] + W.shape[1]))
        W[...] = rng.uniform(-lim, lim, W.shape)
    return theta


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round FP32 values to the nearest bfloat16 (ties to even), returned as
    float64."""
    f = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (f >> 16) & 1
    r = ((f + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _geometry(cfg):
    dim, nx = int(cfg["dim"]), int(cfg["nx"])
    ny = int(cfg.get("ny", 1)) if dim == 2 else 1
    dx = float(cfg["lx"]) / nx
    dy = float(cfg.get("ly", 1.0)) / ny if dim == 2 else 1.0
    return dim, nx, ny, dx, dy


def features(fields: np.ndarray, kngll: np.ndarray, cfg: dict):
    """Returns (X [n x 12], scale [n x 4]) with scale = (p, p sqrt(T), e_x, e_y).
    Gradients as for the HoT (fields.gradient_of: uniform box, annulus or
    wall-refined box)."""
    grad = gradient_of(cfg)
    d_r, omega = float(cfg["d_r"]), float(cfg["omega"])
    mu_ref = mu_ref_of(float(cfg["kn"]))
    rho = fields[:, F_RHO]
    tt, tr = fields[:, F_TT], fields[:, F_TR]
    T = (3.0 * tt + d_r * tr) / (3.0 + d_r)
    mu = mu_ref * T ** omega
    lam = mu / (rho * T) * np.sqrt(math.pi * T / 2.0)
    sq = np.sqrt(T)
    cols = []
    for f, norm in ((rho, rho), (fields[:, F_U], sq), (fields[:, F_U + 1], sq), (tt, T), (tr, T)):
        gx, gy = grad(f)
        cols += [lam * gx / norm, lam * gy / norm]
    X = np.stack(cols + [kngll, tr / tt], axis=1)
    gTx, gTy = grad(T)
    gn = np.sqrt(gTx * gTx + gTy * gTy)
    ex = np.where(gn > 0, gTx / np.where(gn > 0, gn, 1.0), 1.0)
    ey = np.where(gn > 0, gTy / np.where(gn > 0, gn, 1.0), 0.0)
    p = rho * T
    scale = np.stack([p, p * sq, ex, ey], axis=1)
    return X, scale


def targets(hot: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """Normalised HoT (5 per cell) from the 12 HoT components."""
    p, ps, ex, ey = scale.T
    return np.stack([hot[:, 0] / p, hot[:, 3] / p, hot[:, 1] / p,
                     (hot[:, 6] * ex + hot[:, 7] * ey) / ps,
                     (hot[:, 9] * ex + hot[:, 10] * ey) / ps], axis=1)


def to_hot(Y: np.ndarray, scale: np.ndarray, hot_dsmc: np.ndarray) -> np.ndarray:
    """12 HoT components from the network's 5: sigma_xx, sigma_xy, sigma_yy
    and the components of q_t, q_r along e from the network, every other
    component (and the part of q_t, q_r across e) from the DSMC HoT."""
    p, ps, ex, ey = scale.T
    h = hot_dsmc.copy()
    h[:, 0] = Y[:, 0] * p
    h[:, 3] = Y[:, 1] * p
    h[:, 1] = Y[:, 2] * p
    for base, k in ((6, 3), (9, 4)):
        along = h[:, base] * ex + h[:, base + 1] * ey
        new = Y[:, k] * ps
        h[:, base] += (new - along) * ex
        h[:, base + 1] += (new - along) * ey
    return h


def forward(theta: np.ndarray, X: np.ndarray, bf16: bool = False, bf16_act: bool = False):
    """Returns (Y, cache).  bf16: the weights (not the biases) rounded to
    bfloat16.  bf16_act: each layer's input (the features, then the tanh
    activations) rounded to bfloat16 as well, the inference form that feeds
    bfloat16 tensor-core products with FP32 sums."""
    layers = unpack(theta)
    a = X
    cache = [X]
    for k, (W, b) in enumerate(layers):
        Wk = bf16_round(W) if bf16 else W
        if bf16_act:
            a = bf16_round(a)
        z = a @ Wk.T + b
        a = np.tanh(z) if k < 3 else z
        cache.append(a)
    return a, cache


def loss_and_grad(theta: np.ndarray, X: np.ndarray, Y: np.ndarray, bf16: bool = False):
    """Mean over cells of the mean squared error of the 5 outputs, and its
    gradient with respect to theta (backpropagation, same weights as the
    forward pass)."""
    n = X.shape[0]
    out, cache = forward(theta, X, bf16)
    r = out - Y
    loss = float(np.sum(r * r) / (n * SIZES[-1]))
    grad = np.zeros_like(theta)
    glayers = unpack(grad)
    layers = unpack(theta)
    d = 2.0 * r / (n * SIZES[-1])  # dL/d(output)
    for k in range(3, -1, -1):
        W = bf16_round(layers[k][0]) if bf16 else layers[k][0]
        a_in = cache[k]
        gW, gb = glayers[k]
        gW[...] = d.T @ a_in
        gb[...] = d.sum(0)
        if k > 0:
            d = (d @ W) * (1.0 - cache[k] ** 2)  # tanh' = 1 - tanh^2
    return loss, grad


class Adam:
    def __init__(self, n: int, lr: float, b1: float = 0.9, b2: float = 0.999, eps: float = 1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, theta: np.ndarray, g: np.ndarray) -> np.ndarray:
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)
