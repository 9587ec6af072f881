"""Exponential-sum form of the inverse Laplacian preconditioner — oracle, test infrastructure only.

The paper applies the Laplacian preconditioner P^-1 (Sec. 2.3) in low-rank form as an element-wise
product that raises the rank (Sec. 3.2, Table "operations"), but it does not print a low-rank form of
1/(k.k), which is not low-rank itself.  Our reading: approximate 1/x on x in [1, X], X = sum_a ((N_a-1)/2)^2,
by an exponential sum

    1/x ~= sum_m w_m exp(-t_m x),     so   1/(k.k) ~= sum_m w_m prod_a exp(-t_m k_a^2),

a CP/TT tensor of rank R.  The nodes come from the trapezoidal (sinc) rule applied to
1/x = int_R exp(tau - x e^tau) d tau (Stenger, "Numerical Methods Based on Sinc and Analytic
Functions", 1993; Braess & Hackbusch, IMA J. Numer. Anal. 25 (2005) 685-697): t_m = e^{tau_m},
w_m = h e^{tau_m}, tau_m = tau_min + m h, with

    h = pi^2 / ln(32/eps)           (discretisation error ~ exp(-pi^2/h), strip |Im tau| < pi/2)
    tau_min = ln(eps / (2 X))        (lower tail  <= e^{tau_min} <= eps/(2X) relative at x <= X)
    tau_max = ln(ln(2/eps))          (upper tail  = e^{-x e^{tau_max}}/x <= eps/2 relative at x >= 1)

Because P^-1 only preconditions, replacing it with this P~^-1 leaves the solution of the untruncated
system unchanged; eps trades rank for convergence speed.  The value at k = 0 is immaterial: the
divergence output it multiplies vanishes there.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = ["expsum_inverse", "expsum_eval"]


def expsum_inverse(xmax: float, eps: float):
    """Nodes t (ascending) and weights w with max_{1<=x<=xmax} |x sum_m w_m e^{-t_m x} - 1| ~<= eps."""
    if not (0.0 < eps < 1.0) or xmax < 1.0:
        raise ValueError("need 0 < eps < 1 and xmax >= 1")
    h = math.pi ** 2 / math.log(32.0 / eps)
    tau_min = math.log(eps / (2.0 * xmax))
    tau_max = math.log(math.log(2.0 / eps))
    R = int(math.ceil((tau_max - tau_min) / h)) + 1
    tau = tau_min + h * np.arange(R, dtype=np.float64)
    t = np.exp(tau)
    w = h * np.exp(tau)
    return t, w


def expsum_eval(x, t, w):
    """sum_m w_m exp(-t_m x) at the points x."""
    x = np.asarray(x, dtype=np.float64)
    return np.sum(w[:, None] * np.exp(-np.outer(t, x.ravel())), axis=0).reshape(x.shape)
