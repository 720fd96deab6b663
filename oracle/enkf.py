"""Diffusion ensemble Kalman filter of the hierarchical mesoscale data
assimilation -- oracle (TEST INFRASTRUCTURE ONLY; see the package docstring).

Follows Supplementary Algorithm 3 step by step in FP64 with plain numpy:

  step 4  ensemble mean mu and covariance C = sum (x - mu)(x - mu)^T / (N - 1)
  step 5  per observer l: S_l = H_l C H_l^T + Gamma_o, K_l = C H_l^T S_l^{-1}
  step 6  per observer l and member n: x^{n,l} = x^n + K_l (y - eps^{n,l} - H_l x^n)
  step 7  fusion: x^n = diag(x_half^n Upsilon(gamma)), Upsilon_ij = gamma on the
          diagonal and (1 - gamma)/(L - 1) off it

and the random walk of the hyperparameters (Supplementary Sec. 6,
theta(t) = theta(t-1) + eps_theta).

Readings (the paper is silent or garbled here):
  * the state of member n is, per region r, the block
      [log g_AMPA scale, log g_GABA_A scale, s, f, v, q, y]  (7 values),
    the two log scales being the region's hyperparameters; for a scale
    family cdf^{-1}(cdf(theta; old); new) is theta * new / old, so the scales
    are simply replaced;
  * in "diffusion" mode observer l sees the BOLD signal of region l (L = R)
    and "diag" of the (7R x L) product keeps, for every component, the column
    of the observer that owns the component's region;
  * with a single observer there is nothing to fuse (x^n = x^{n,1});
  * in "global" mode one observer sees all R signals (the textbook
    stochastic EnKF);
  * Gamma_o = obs_var * I; eps^{n,l} = sqrt(obs_var) * (a standard normal
    passed in by the caller).
"""
from __future__ import annotations

import numpy as np

BLOCK = 7          # values per region in the state vector
Y_INDEX = 6        # position of the BOLD signal inside a block
THETA = (0, 1)     # positions of the two log scales


def diffusion_enkf(X: np.ndarray, y_obs: np.ndarray, obs_var: float, gamma: float,
                   eps_obs: np.ndarray, mode: str = "diffusion") -> np.ndarray:
    """Analysis of forecast ensemble X [M, 7R] against y_obs [R]."""
    X = np.asarray(X, dtype=np.float64)
    M, n = X.shape
    R = n // BLOCK
    assert n == BLOCK * R and y_obs.shape == (R,)
    mu = X.sum(axis=0) / M
    A = X - mu
    C = A.T @ A / (M - 1)
    sd = np.sqrt(obs_var)
    Xa = np.empty_like(X)
    if mode == "global":
        H = np.zeros((R, n))
        for r in range(R):
            H[r, BLOCK * r + Y_INDEX] = 1.0
        S = H @ C @ H.T + obs_var * np.eye(R)
        K = C @ H.T @ np.linalg.inv(S)
        for m in range(M):
            Xa[m] = X[m] + K @ (y_obs - sd * eps_obs[m] - H @ X[m])
        return Xa
    assert mode == "diffusion"
    L = R
    Xl = np.empty((L, M, n))
    for l in range(L):
        h = BLOCK * l + Y_INDEX
        S = C[h, h] + obs_var
        K = C[:, h] / S
        for m in range(M):
            Xl[l, m] = X[m] + K * (y_obs[l] - sd * eps_obs[m, l] - X[m, h])
    if L == 1:
        return Xl[0].copy()
    U = np.full((L, L), (1.0 - gamma) / (L - 1))
    np.fill_diagonal(U, gamma)
    for m in range(M):
        P = Xl[:, m, :].T @ U          # [n, L]
        for c in range(n):
            Xa[m, c] = P[c, c // BLOCK]
    return Xa


def constrain(X: np.ndarray, theta_lo: float, theta_hi: float, floor: float = 1e-2) -> np.ndarray:
    """Keep hyperparameters inside the prior support and the hemodynamic
    flow, volume and deoxyhemoglobin positive."""
    X = X.copy()
    R = X.shape[1] // BLOCK
    for r in range(R):
        b = BLOCK * r
        for t in THETA:
            X[:, b + t] = np.clip(X[:, b + t], theta_lo, theta_hi)
        for k in (3, 4, 5):
            X[:, b + k] = np.maximum(X[:, b + k], floor)
    return X


def random_walk(X: np.ndarray, rw_sigma: float, xi: np.ndarray, theta_lo: float,
                theta_hi: float) -> np.ndarray:
    """theta <- clip(theta + rw_sigma * xi); xi [M, R, 2] standard normals."""
    X = X.copy()
    R = X.shape[1] // BLOCK
    for r in range(R):
        for t_i, t in enumerate(THETA):
            c = BLOCK * r + t
            X[:, c] = np.clip(X[:, c] + rw_sigma * xi[:, r, t_i], theta_lo, theta_hi)
    return X


def pack_state(theta: np.ndarray, bw: np.ndarray, y: np.ndarray) -> np.ndarray:
    """theta [M, R, 2], bw [M, R, 4], y [M, R] -> X [M, 7R]."""
    M, R, _ = theta.shape
    X = np.empty((M, R, BLOCK))
    X[:, :, 0:2] = theta
    X[:, :, 2:6] = bw
    X[:, :, 6] = y
    return X.reshape(M, R * BLOCK)


def unpack_state(X: np.ndarray):
    M = X.shape[0]
    R = X.shape[1] // BLOCK
    B = X.reshape(M, R, BLOCK)
    return B[:, :, 0:2].copy(), B[:, :, 2:6].copy(), B[:, :, 6].copy()
