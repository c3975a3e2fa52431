"""Pins of the oracle's constant-velocity model and particle filter (Sec. 5.1)."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import cv, kalman
from paper_1306_5583_b300 import workloads


def test_student_t_loglik_matches_scipy():
    p = cv.CVParams()
    g = np.random.default_rng(0)
    x = g.normal(size=(4, 200)) * 3
    y = np.array([0.7, -1.2])
    ref = (stats.t.logpdf(y[0], p.obs_df, loc=x[0], scale=p.obs_scale)
           + stats.t.logpdf(y[1], p.obs_df, loc=x[1], scale=p.obs_scale))
    assert np.max(np.abs(cv.loglik(x, y, p) - ref)) < 1e-12


def test_gaussian_loglik_matches_scipy():
    p = cv.CVParams(gaussian_obs=True, obs_scale=0.3)
    g = np.random.default_rng(1)
    x = g.normal(size=(4, 50))
    y = np.array([0.1, 0.4])
    ref = stats.norm.logpdf(y[0], x[0], 0.3) + stats.norm.logpdf(y[1], x[1], 0.3)
    assert np.max(np.abs(cv.loglik(x, y, p) - ref)) < 1e-12


def test_zero_noise_move_is_multiplication_by_A():
    p = cv.CVParams(sd_pos=0.0, sd_vel=0.0, delta=0.25)
    g = np.random.default_rng(2)
    x = g.normal(size=(4, 30))
    assert np.allclose(cv.move(x, 5, 1, p), cv.transition_matrix(0.25) @ x, atol=0, rtol=1e-15)


def test_move_noise_scales():
    p = cv.CVParams(sd_pos=0.3, sd_vel=2.0)
    x = np.zeros((4, 40000))
    d = cv.move(x, 1, 3, p)
    assert abs(d[0].std() - 0.3) < 0.01 and abs(d[1].std() - 0.3) < 0.01
    assert abs(d[2].std() - 2.0) < 0.05 and abs(d[3].std() - 2.0) < 0.05


def test_kalman_matches_stacked_normal():
    p = cv.CVParams(gaussian_obs=True)
    _, y = workloads.cv_data(7, seed=3, gaussian_obs=True)
    assert abs(kalman.kalman_loglik(y, p) - kalman.stacked_loglik(y, p)) < 1e-9


def test_kalman_matches_stacked_normal_paper_constants():
    kw = dict(workloads.CV_PAPER)
    p = cv.CVParams(gaussian_obs=True, **kw)
    _, y = workloads.cv_data(6, seed=4, gaussian_obs=True, **kw)
    assert abs(kalman.kalman_loglik(y, p) - kalman.stacked_loglik(y, p)) < 1e-9


def test_particle_filter_evidence_matches_kalman():
    """exp(log Z-hat) is unbiased for the Kalman likelihood: over R
    independent runs, the mean of Z-hat / Z is 1 within Monte Carlo error."""
    p = cv.CVParams(gaussian_obs=True)
    T, n, R = 15, 2048, 16
    _, y = workloads.cv_data(T, seed=5, gaussian_obs=True)
    logz = kalman.kalman_loglik(y, p)
    est = []
    for r in range(R):
        recs, _ = cv.run(y, n, seed=100 + r, p=p, scheme="systematic", threshold=0.5)
        est.append(recs[-1]["logZ"])
    est = np.array(est)
    ratio = np.exp(est - logz)
    assert abs(ratio.mean() - 1) < 5 * ratio.std(ddof=1) / math.sqrt(R) + 0.01
    assert abs(est.mean() - logz) < 0.1


def test_particle_filter_means_track_kalman():
    p = cv.CVParams(gaussian_obs=True)
    T, n = 12, 4096
    _, y = workloads.cv_data(T, seed=6, gaussian_obs=True)
    km = kalman.kalman_means(y, p)
    recs, _ = cv.run(y, n, seed=7, p=p)
    pm = np.array([[r["mean_x"], r["mean_y"]] for r in recs])
    assert np.max(np.abs(pm - km)) < 0.05


def test_first_step_is_importance_sampling_from_the_prior():
    """At t = 0 the estimate is log mean_i g(y_0 | x_i) (Sec. 2.1, phi-hat-1)."""
    p = cv.CVParams()
    y0 = np.array([0.3, -0.2])
    r = cv.init_step(500, y0, 9, p, 0.5)
    x = cv.init_state(500, 9, p)
    ll = cv.loglik(x, y0, p)
    assert abs(r.L - (np.log(np.mean(np.exp(ll - ll.max()))) + ll.max())) < 1e-12


def test_post_resampling_mean_is_the_mean_of_the_copies():
    """The post-resampling monitor: without resampling it is the weighted
    mean; with it, the plain mean of the selected copies, whose expectation
    over the resampling draws is the weighted mean (unbiased resampling)."""
    import math as _m
    from oracle import cv as _cv, resample as _rs
    p = _cv.CVParams()
    y = np.array([[0.3, -0.2], [0.5, 0.1]])
    r = _cv.init_step(400, y[0], 3, p, 0.5)
    assert _cv.post_resampling_mean(r, None) == (r.mean_x, r.mean_y)
    a = _rs.resample("multinomial", r.lw, 3, 0)
    mx, my = _cv.post_resampling_mean(r, a)
    assert mx == float(np.mean(r.x[0][a])) and my == float(np.mean(r.x[1][a]))
    vals = [_cv.post_resampling_mean(r, _rs.resample("multinomial", r.lw, 3, t))[0] for t in range(300)]
    W = np.exp(r.lw - r.L)
    sd = _m.sqrt(float(np.sum(W * (r.x[0] - r.mean_x) ** 2)) / 400)
    assert abs(np.mean(vals) - r.mean_x) < 5 * sd / _m.sqrt(300)
    recs, _ = _cv.run(np.array([[0.1, 0.0]] * 6), 300, 2, p, threshold=1.0)
    assert all(rr["resampled"] for rr in recs)
