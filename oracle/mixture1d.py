"""FP64 oracle of the 1D mixture-fitting study (Sec. 3.2 "Assessing 1D GEF Mixtures"; App. A) --
TEST INFRASTRUCTURE ONLY, like the rest of this package.

Models, N components, parameters per component (weight w, mean mu, scale sigma (gamma for the LoG),
shape beta for the GEF), with eps = 1e-8 (App. A, Eq. gaussianmixture onward):
    Gaussian  g(x) = sum_i w_i exp(-(x - mu_i)^2 / (2 sigma_i^2 + eps))
    DoG       d(x) = sum_i w_i [exp(-(x - mu_i)^2 / (2 sigma_i^2 + eps)) - exp(-(x - mu_i)^2 / (2 sigma_i^2 / nu + eps))],
              nu = 4
    LoG       l(x) = sum_i w_i (1 - (x - mu_i)^2 / gamma_i^2) exp(-(x - mu_i)^2 / (2 gamma_i^2 + eps))
    GEF       h(x) = sum_i w_i exp(-|x - mu_i|^beta_i / (2 sigma_i^2 + eps))          (Eq. genmixture)
Positive weights: w = |omega| of the optimised omega (unrestricted: w = omega).
Signals of width s on (-s/2, s/2), zero outside (App. A, Data Generation): square 1; triangle
s/2 - |x|; parabolic (s/2)^2 - x^2; half sinusoid sin((x + s/2) pi / s); exponential exp(-|x|);
and the Gaussian exp(-x^2 / (2 s^2)) everywhere.
Training: full-batch Adam on the mean squared error over the sample points, for a fixed number of
epochs (torch.optim.Adam, FP64, on the CPU); the gradient is torch.autograd's.

Readings where the paper is silent (the kernels implement the same): beta is one parameter per
component; positivity by |omega|; the final loss is the MSE at the parameters after the last step;
a run whose loss is not finite is unstable and its later losses are NaN.
"""
from __future__ import annotations

import math

import numpy as np

MODELS = ("gaussian", "dog", "log", "gef")
SIGNALS = ("square", "triangle", "parabolic", "half_sinusoid", "exponential", "gaussian")
MIX_EPS = 1e-8
DOG_NU = 4.0


def n_rows(model: str) -> int:
    """Parameter rows per component: omega, mu, sigma (gamma), and beta for the GEF."""
    return 4 if model == "gef" else 3


def signal(kind: str, x, width: float = 1.0):
    x = np.asarray(x, np.float64)
    h = width / 2.0
    inside = (x > -h) & (x < h)
    if kind == "square":
        v = np.ones_like(x)
    elif kind == "triangle":
        v = h - np.abs(x)
    elif kind == "parabolic":
        v = h * h - x * x
    elif kind == "half_sinusoid":
        v = np.sin((x + h) * math.pi / width)
    elif kind == "exponential":
        v = np.exp(-np.abs(x))
    elif kind == "gaussian":
        return np.exp(-x * x / (2.0 * width * width))
    else:
        raise ValueError(kind)
    return np.where(inside, v, 0.0)


def model_eval(model: str, params, x, positive: bool = True, nu: float = DOG_NU, eps: float = MIX_EPS):
    """The mixture at x for params [rows, N] (torch tensors or numpy arrays, FP64)."""
    import torch
    p = torch.as_tensor(params, dtype=torch.float64)
    xs = torch.as_tensor(np.asarray(x, np.float64))[:, None]
    w = p[0].abs() if positive else p[0]
    d = xs - p[1]
    s = p[2]
    if model == "gaussian":
        comp = torch.exp(-d * d / (2 * s * s + eps))
    elif model == "dog":
        comp = torch.exp(-d * d / (2 * s * s + eps)) - torch.exp(-d * d / (2 * (s * s / nu) + eps))
    elif model == "log":
        comp = (-(d * d) / (s * s) + 1.0) * torch.exp(-d * d / (2 * s * s + eps))
    elif model == "gef":
        comp = torch.exp(-d.abs().pow(p[3]) / (2 * s * s + eps))
    else:
        raise ValueError(model)
    return (w * comp).sum(1)


def fit(model: str, params0, x, y, epochs: int, positive: bool = True, lr: float = 0.01, betas=(0.9, 0.999),
        adam_eps: float = 1e-8, nu: float = DOG_NU, eps: float = MIX_EPS):
    """Adam on MSE from params0 [rows, N].  Returns (final params [rows, N], loss history [epochs + 1]
    (the MSE before each step, then after the last), gradient of the MSE at the final params)."""
    import torch
    p = torch.tensor(np.asarray(params0, np.float64), requires_grad=True)
    yt = torch.as_tensor(np.asarray(y, np.float64))
    opt = torch.optim.Adam([p], lr=lr, betas=betas, eps=adam_eps)
    hist = []
    for _ in range(epochs):
        opt.zero_grad()
        loss = ((model_eval(model, p, x, positive, nu, eps) - yt) ** 2).mean()
        loss.backward()
        hist.append(float(loss.detach()))
        opt.step()
    opt.zero_grad()
    loss = ((model_eval(model, p, x, positive, nu, eps) - yt) ** 2).mean()
    loss.backward()
    hist.append(float(loss.detach()))
    return p.detach().numpy(), np.array(hist), p.grad.detach().numpy()
