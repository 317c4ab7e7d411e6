"""Pins of the oracle's map-making loop (the adjoint application of the
normalised gridding operator, Eq. 3): gradient descent on
L(m) = 1/2 ||G^T m - D||^2 with step 1 / (largest column sum of G).

* the dense operator built by gridding the identity equals the oracle's
  gridder (G x) and its degridder (G^T y) -- two independent code paths;
* unit row sums where W_p > 0 (the normalisation of Eq. 3);
* the loss sequence equals the closed form of the iteration,
  L_k = 1/2 sum_i (1 - alpha lambda_i)^(2k) (q_i . D)^2 over the eigenpairs of
  G^T G (numpy eigh), so a wrong sign, step or operator fails;
* the step rule keeps alpha lambda_max <= 1, hence a non-increasing loss.
"""
import math

import numpy as np

import oracle
import workloads

ARCMIN = 1.0 / 60.0


def _case(seed=301, n=150, side=10, weights=True):
    wl = workloads.random_field(seed, n, side, 2, 200.0, -20.0, 0.5, 1.5 * ARCMIN,
                                weights=weights)
    return wl, oracle.gauss1d(1.5 * ARCMIN, 4.5 * ARCMIN)


def test_operator_matrix_is_grid_and_degrid():
    wl, k = _case()
    G = oracle.operator_matrix(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, k, wl.omega)
    rng = np.random.Generator(np.random.PCG64(302))
    x = rng.normal(0, 1, (wl.n_samples, 3))
    y = rng.normal(0, 1, (wl.n_targets, 3))
    gx = oracle.grid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, x, k, wl.omega)
    on = gx.wsum > 0
    assert np.allclose((G @ x)[on], gx.out[on], rtol=0, atol=1e-12)
    assert np.all(G[~on] == 0.0)
    xhat = oracle.degrid_bruteforce(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, y, k, wl.omega)
    assert np.allclose(G.T @ y, xhat, rtol=0, atol=1e-12)
    assert np.allclose(G[on].sum(axis=1), 1.0, rtol=0, atol=1e-12)


def test_gd_losses_match_closed_form():
    wl, k = _case(seed=303)
    G = oracle.operator_matrix(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, k, wl.omega)
    D = np.asarray(wl.data, dtype=np.float64)
    steps = 50
    m, losses, alpha = oracle.mapmaking_gd(G, D, steps)
    assert math.isclose(alpha, 1.0 / G.sum(axis=0).max(), rel_tol=1e-15)
    lam, Q = np.linalg.eigh(G.T @ G)
    proj = Q.T @ D                                   # [N, C]
    ref = np.array([0.5 * float(np.sum(((1.0 - alpha * lam) ** (2 * kk))[:, None] * proj ** 2))
                    for kk in range(steps + 1)])
    assert np.allclose(losses, ref, rtol=1e-9, atol=0)
    # the returned map is the last iterate: its residual gives the last loss
    r = G.T @ m - D
    assert math.isclose(0.5 * float(np.sum(r * r)), losses[-1], rel_tol=1e-12)


def test_gd_step_rule_monotone():
    for seed in (304, 305, 306):
        wl, k = _case(seed=seed, n=200)
        G = oracle.operator_matrix(wl.lon_t, wl.lat_t, wl.lon_s, wl.lat_s, k, wl.omega)
        _, losses, alpha = oracle.mapmaking_gd(G, wl.data, 50)
        lam_max = np.linalg.eigvalsh(G @ G.T).max()
        assert alpha * lam_max <= 1.0 + 1e-12
        assert np.all(np.diff(losses) <= 1e-12 * losses[0])
        assert losses[-1] < losses[0]
