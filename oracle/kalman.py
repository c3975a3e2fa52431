"""Exact log-likelihood of the linear-Gaussian constant-velocity model.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

With Gaussian observation noise the model of Sec. 5.1.1 is linear-Gaussian,
so p(y_0, ..., y_{T-1}) is available in closed form.  Two independent
evaluations are given:
* ``kalman_loglik``: the standard Kalman filter prediction-error
  decomposition, sum_t log N(y_t; B m_{t|t-1}, B P_{t|t-1} B' + s^2 I);
* ``stacked_loglik``: the joint normal law of the stacked observations,
  Cov(y_s, y_t) = B Cov(x_s, x_t) B' + s^2 I [s == t], with
  Cov(x_s, x_t) = A^s P0 (A^t)' + sum_{k=1}^{min(s,t)} A^{s-k} Q (A^{t-k})',
  evaluated by scipy's multivariate normal density (pins the Kalman filter).

The Kalman value pins the particle filter's evidence estimate, whose
exponential is unbiased for p(y_{0:T-1}).
"""
import math

import numpy as np

from .cv import transition_matrix

B = np.array([[1, 0, 0, 0], [0, 1, 0, 0]], dtype=np.float64)


def _mats(p):
    A = transition_matrix(p.delta)
    Q = np.diag([p.sd_pos ** 2, p.sd_pos ** 2, p.sd_vel ** 2, p.sd_vel ** 2])
    P0 = np.diag([p.sd_pos0 ** 2, p.sd_pos0 ** 2, p.sd_vel0 ** 2, p.sd_vel0 ** 2])
    R = np.eye(2) * p.obs_scale ** 2
    return A, Q, P0, R


def kalman_loglik(y, p):
    A, Q, P0, R = _mats(p)
    m = np.zeros(4)
    P = P0.copy()
    ll = 0.0
    for t in range(y.shape[0]):
        if t > 0:
            m = A @ m
            P = A @ P @ A.T + Q
        S = B @ P @ B.T + R
        r = y[t] - B @ m
        Si = np.linalg.inv(S)
        ll += -math.log(2 * math.pi) - 0.5 * math.log(np.linalg.det(S)) - 0.5 * r @ Si @ r
        K = P @ B.T @ Si
        m = m + K @ r
        P = (np.eye(4) - K @ B) @ P
    return float(ll)


def kalman_means(y, p):
    """Filtered means E[x_t | y_{0:t}] of the positions, (T, 2)."""
    A, Q, P0, R = _mats(p)
    m = np.zeros(4)
    P = P0.copy()
    out = []
    for t in range(y.shape[0]):
        if t > 0:
            m = A @ m
            P = A @ P @ A.T + Q
        S = B @ P @ B.T + R
        K = P @ B.T @ np.linalg.inv(S)
        m = m + K @ (y[t] - B @ m)
        P = (np.eye(4) - K @ B) @ P
        out.append(m[:2].copy())
    return np.array(out)


def stacked_loglik(y, p):
    from scipy.stats import multivariate_normal
    A, Q, P0, R = _mats(p)
    T = y.shape[0]
    Ap = [np.linalg.matrix_power(A, k) for k in range(T)]
    C = np.zeros((2 * T, 2 * T))
    for s in range(T):
        for t in range(T):
            cx = Ap[s] @ P0 @ Ap[t].T
            for k in range(1, min(s, t) + 1):
                cx = cx + Ap[s - k] @ Q @ Ap[t - k].T
            blk = B @ cx @ B.T
            if s == t:
                blk = blk + R
            C[2 * s:2 * s + 2, 2 * t:2 * t + 2] = blk
    return float(multivariate_normal(mean=np.zeros(2 * T), cov=C).logpdf(y.reshape(-1)))
