"""Gradient of an observation misfit through the TPFA pressure solve -- oracle.

Not in the paper.  For A(theta) p = f(theta) with A SPD and a loss
L = sum_o (p_o - p_obs,o)^2 over observation cells o, the adjoint is

    A lambda = g,   g_o = 2 (p_o - p_obs,o)            (A symmetric)
    dL/dtheta = lambda^T (df/dtheta - (dA/dtheta) p).

With the TPFA assembly A = sum_faces T_kl (e_k - e_l)(e_k - e_l)^T + sum_b T_b e_k e_k^T
and f = sum_b T_b p_bc e_k this gives

    dL/dT_kl = -(lambda_k - lambda_l)(p_k - p_l)        interior face
    dL/dT_b  =  lambda_k (p_bc - p_k)                    Dirichlet half-face
    T_kl = 2 K_k K_l / (K_k + K_l):  dT_kl/d ln K_k = T_kl K_l / (K_k + K_l)
    T_b  = 2 K_k:                    dT_b / d ln K_k = T_b

(an anisotropy factor on T multiplies both K's and cancels in the ratio).
`solve(A, rhs)` is any exact SPD solve supplied by the caller.
"""
from __future__ import annotations

import numpy as np


def misfit(p, obs, p_obs):
    d = p[obs] - p_obs
    return float(d @ d)


def grad_lnK(A, f, faces, lnK_flat, obs, p_obs, solve):
    """Return (L, dL/dlnK, p, lambda) for one permeability sample."""
    p = solve(A, f)
    g = np.zeros_like(p)
    d = p[obs] - p_obs
    np.add.at(g, obs, 2.0 * d)
    lam = solve(A, g)
    K = np.exp(lnK_flat)
    k, l, T = faces["k"], faces["l"], faces["T"]
    dT = -(lam[k] - lam[l]) * (p[k] - p[l])
    grad = np.zeros_like(p)
    np.add.at(grad, k, dT * T * K[l] / (K[k] + K[l]))
    np.add.at(grad, l, dT * T * K[k] / (K[k] + K[l]))
    c, Tb, pb = faces["bc_cell"], faces["bc_T"], faces["bc_p"]
    np.add.at(grad, c, lam[c] * (pb - p[c]) * Tb)
    return float(d @ d), grad, p, lam
