"""Pins of the learned-screening oracle (oracle/learned_scs.py) against closed forms,
invariances and central differences.  CPU only."""
import numpy as np
import pytest

from oracle import learned_scs as L


def params(seed=0):
    rng = np.random.default_rng(seed)
    return [(rng.normal(0, 1 / np.sqrt(i), (i, o)), rng.normal(0, 0.1, o)) for i, o in L.LAYERS]


def test_two_atom_features_closed_form():
    R = np.array([[0.0, 0.0, 0.0], [0.0, 3.3, 4.4]])          # d = 5.5
    a0, om, rv, v = np.array([7.0, 9.0]), np.array([0.4, 0.6]), np.array([3.1, 3.6]), np.array([0.8, 0.9])
    X = L.features(R, a0, om, rv, v)
    mu = (np.arange(64) + 0.5) * 0.375
    fc = 0.5 * (1 + np.cos(np.pi * 5.5 / 24))
    assert np.allclose(X[0, :64], 9.0 * fc * np.exp(-(5.5 - mu) ** 2 / (2 * 0.375 ** 2)), rtol=1e-14, atol=0)
    assert np.allclose(X[1, :64], 7.0 * fc * np.exp(-(5.5 - mu) ** 2 / (2 * 0.375 ** 2)), rtol=1e-14, atol=0)
    assert np.allclose(X[0, 64:68], [7.0, 0.4, 3.1, 0.8]) and np.allclose(X[1, 64:68], [9.0, 0.6, 3.6, 0.9])
    assert np.argmax(X[0, :64]) == 14                          # mu_14 = 5.4375 is the nearest centre
    # screening moments of one pair: M_0 = a0_1 B, M_1 = a0_0 B with B = (1 - f) T^GG (even in r)
    from oracle import oracle as orc
    s = np.hypot(*np.cbrt(np.sqrt(2 / np.pi) * a0 / 3))
    Bm = (1 - orc.fermi(5.5, 3.1 + 3.6, 0.83, 6.0)) * orc.T_gg(R[1] - R[0], s)
    tr, tr2 = np.trace(Bm), np.trace(Bm @ Bm)
    # two hops: alpha0_j B (alpha0_i B) = 63 B^2 for either atom
    assert np.allclose(X[0, 68:74], [9 * tr / 3, 63 * tr2 / 3, 81 * tr2 / 3, 7 * 9 * tr / 3,
                                   49 * 63 * tr2 / 3, 49 * 81 * tr2 / 3], rtol=1e-12)
    assert np.allclose(X[1, 68:71], [7 * tr / 3, 63 * tr2 / 3, 49 * tr2 / 3], rtol=1e-12)
    # per-frequency Dyson block, feature 74 + 3 k + q - 1: at u_k the widths and couplings of
    # alpha(u_k) = a0 / (1 + u_k^2 / om^2); one pair gives H^(q)_0 = a_1^ceil(q/2) a_0^floor(q/2) B^q
    import oracle as o
    u, _ = o.freq_grid(15)
    assert X.shape == (2, 122) and u[0] == 0.0
    for k, uk in enumerate(u):
        al = a0 / (1 + uk ** 2 / om ** 2)
        Bk = (1 - orc.fermi(5.5, 6.7, 0.83, 6.0)) * orc.T_gg(R[1] - R[0], np.hypot(*L.orc_sigma(al)))
        t = [np.trace(np.linalg.matrix_power(Bk, q)) / 3 for q in (1, 2, 3)]
        assert np.allclose(X[0, 74 + 3 * k:77 + 3 * k], [al[1] * t[0], al[0] * al[1] * t[1], al[1] ** 2 * al[0] * t[2]],
                           rtol=1e-12)
        assert np.allclose(X[1, 74 + 3 * k:77 + 3 * k], [al[0] * t[0], al[0] * al[1] * t[1], al[0] ** 2 * al[1] * t[2]],
                           rtol=1e-12)


def test_features_vanish_beyond_cutoff_and_are_continuous_there():
    a0, om, rv, v = np.ones(2) * 6, np.ones(2) * 0.5, np.ones(2) * 3.5, np.ones(2)
    far = L.features(np.array([[0, 0, 0], [0, 0, 24.0]]), a0, om, rv, v)
    assert np.all(far[:, :64] == 0) and np.all(far[:, 68:74] == 0)   # the Dyson block has no cutoff
    near = L.features(np.array([[0, 0, 0], [0, 0, 24.0 - 1e-6]]), a0, om, rv, v)
    assert np.abs(near[:, :64]).max() < 1e-10                  # smooth cutoff: fc(24) = fc'(24) = 0


def test_features_invariances():
    rng = np.random.default_rng(3)
    R = rng.uniform(0, 12, (7, 3))
    a0, om, rv, v = rng.uniform(4, 12, 7), rng.uniform(0.3, 0.9, 7), rng.uniform(3, 4, 7), rng.uniform(0.7, 1, 7)
    X = L.features(R, a0, om, rv, v)
    Qm, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    assert np.allclose(L.features(R @ Qm.T + [1.0, -2.0, 3.0], a0, om, rv, v), X, rtol=1e-12, atol=1e-13)
    p = rng.permutation(7)
    assert np.allclose(L.features(R[p], a0[p], om[p], rv[p], v[p]), X[p], rtol=1e-13, atol=1e-14)


def test_feature_jacobian_vs_fd():
    rng = np.random.default_rng(4)
    R = rng.uniform(0, 10, (5, 3))
    a0, om, rv, v = rng.uniform(4, 12, 5), rng.uniform(0.3, 0.9, 5), rng.uniform(3, 4, 5), rng.uniform(0.7, 1, 5)
    J = L.feature_position_jacobian(R, a0)
    h = 1e-6
    for k in range(5):
        for c in range(3):
            Rp, Rm = R.copy(), R.copy()
            Rp[k, c] += h; Rm[k, c] -= h
            fd = (L.static_features(Rp, a0, om, rv, v) - L.static_features(Rm, a0, om, rv, v))[:, :64] / (2 * h)
            assert np.abs(fd - J[:, :, k, c]).max() < 1e-7 * max(1.0, np.abs(J).max())


def test_silu_derivative():
    z = np.linspace(-6, 6, 41)
    h = 1e-6
    assert np.allclose((L.silu(z + h) - L.silu(z - h)) / (2 * h), L.dsilu(z), atol=1e-9)
    assert L.silu(np.array([0.0]))[0] == 0.0 and abs(L.silu(np.array([30.0]))[0] - 30.0) < 1e-9


def test_mlp_backward_vs_fd():
    P = params(1)
    rng = np.random.default_rng(5)
    X = rng.normal(size=(6, L.N_FEAT))
    dy = rng.normal(size=(6, L.N_OUT))
    y, cache = L.forward(X, P)
    grads, dX = L.backward(dy, P, cache)
    f = lambda P_, X_: float((L.forward(X_, P_)[0] * dy).sum())
    h = 1e-6
    for li, (W, b) in enumerate(P):
        for (a, c) in [(0, 0), (W.shape[0] - 1, W.shape[1] - 1), (W.shape[0] // 2, W.shape[1] // 3)]:
            Wp = [(w.copy(), bb.copy()) for w, bb in P]
            Wm = [(w.copy(), bb.copy()) for w, bb in P]
            Wp[li][0][a, c] += h; Wm[li][0][a, c] -= h
            assert (f(Wp, X) - f(Wm, X)) / (2 * h) == pytest.approx(grads[li][0][a, c], rel=1e-6, abs=1e-9)
        Bp = [(w.copy(), bb.copy()) for w, bb in P]
        Bm = [(w.copy(), bb.copy()) for w, bb in P]
        Bp[li][1][1] += h; Bm[li][1][1] -= h
        assert (f(Bp, X) - f(Bm, X)) / (2 * h) == pytest.approx(grads[li][1][1], rel=1e-6, abs=1e-9)
    for (a, c) in [(0, 0), (3, 73), (5, 20)]:
        Xp, Xm = X.copy(), X.copy()
        Xp[a, c] += h; Xm[a, c] -= h
        assert (f(P, Xp) - f(P, Xm)) / (2 * h) == pytest.approx(dX[a, c], rel=1e-6, abs=1e-9)


def test_mse_and_adam_first_step():
    y, t = np.array([[1.0, 2.0], [3.0, 5.0]]), np.array([[0.0, 2.0], [1.0, 1.0]])
    loss, g = L.mse_loss_grad(y, t)
    assert loss == pytest.approx((1 + 0 + 4 + 16) / 4)
    assert np.allclose(g, 2 * (y - t) / 4)
    p, gg = np.array([1.0, -2.0, 0.5]), np.array([0.3, -4.0, 0.0])
    m, v = np.zeros(3), np.zeros(3)
    L.adam_step(p, gg, m, v, 1, lr=0.01)
    # first step: m_hat = g, v_hat = g^2, so the update is -lr g / (|g| + eps)
    assert np.allclose(p, [1.0 - 0.01 * 0.3 / (0.3 + 1e-8), -2.0 + 0.01 * 4.0 / (4.0 + 1e-8), 0.5])


def test_ensemble_prediction_and_estimate():
    P = params(2)
    rng = np.random.default_rng(6)
    X = rng.normal(size=(5, L.N_FEAT))
    alpha_u = rng.uniform(1, 10, (16, 5))
    ab, s = L.predict_alpha_bar(X, [P, P, P], alpha_u)
    assert np.all(s < 1e-12 * ab.max())                         # identical members: no spread
    y = L.forward(X, P)[0]
    assert np.allclose(ab, alpha_u * np.exp(y.T), rtol=1e-14)
    zero = [(W * 0, b * 0) for W, b in P]
    ab0, _ = L.predict_alpha_bar(X, [zero], alpha_u)
    assert np.allclose(ab0, alpha_u)                            # y = 0: no screening
    h = rng.normal(size=(16, 5))
    ys = np.stack([L.forward(X, P)[0]] * 3)
    assert L.estimated_error_per_atom(h, alpha_u, ys) < 1e-14   # identical members: no spread (rounding only)
    # two members apart in one entry (u = 3, atom 2) by delta: D = -+ h alpha (e^delta - 1) / 2
    y2 = np.zeros((2, 5, 16))
    y2[1, 2, 3] = 0.3
    ref = abs(h[3, 2] * alpha_u[3, 2] * (np.exp(0.3) - 1.0)) / 2.0 / 5
    assert L.estimated_error_per_atom(h, alpha_u, y2) == pytest.approx(ref, rel=1e-13)
    assert L.estimated_error_per_atom(h, alpha_u, y2, scale=0.2) == pytest.approx(0.2 * ref, rel=1e-13)


def test_fp16_rounding_is_round_to_nearest():
    P = [(np.array([[1.0 + 2 ** -12]]), np.array([0.1]))]
    W, b = L.round_fp16(P)[0]
    assert W[0, 0] == 1.0 and b[0] == np.float16(0.1).astype(np.float64)


def test_dyson_moments_two_atoms_closed_form():
    # one pair: B_01 = B_10 = B (even in r), so H^(1)_0 = a_1 B, H^(2)_0 = a_1 a_0 B^2,
    # H^(3)_0 = a_1^2 a_0 B^3 at each frequency
    from oracle import oracle as orc
    R = np.array([[0.0, 0.0, 0.0], [0.0, 3.3, 4.4]])
    a0, om, rv = np.array([7.0, 9.0]), np.array([0.4, 0.6]), np.array([3.1, 3.6])
    u = np.array([0.0, 0.3, 2.0])
    m = L.dyson_moments(R, a0, om, rv, u)
    for k, uk in enumerate(u):
        al = a0 / (1 + uk ** 2 / om ** 2)
        s = np.hypot(*L.orc_sigma(al))
        Bm = (1 - orc.fermi(5.5, 6.7, 0.83, 6.0)) * orc.T_gg(R[1] - R[0], s)
        t1, t2, t3 = (np.trace(np.linalg.matrix_power(Bm, p)) / 3 for p in (1, 2, 3))
        assert np.allclose(m[k, :, 0], [al[1] * t1, al[0] * t1], rtol=1e-13)
        assert np.allclose(m[k, :, 1], [al[0] * al[1] * t2] * 2, rtol=1e-13)
        assert np.allclose(m[k, :, 2], [al[1] ** 2 * al[0] * t3, al[0] ** 2 * al[1] * t3], rtol=1e-13)


def test_dyson_series_converges_to_the_screening():
    # a dilute cluster (weak coupling): from the first order on, the partial sums
    # 1 - m1 + m2 - m3 + m4 approach the exact screened alpha_bar / alpha of the oracle, each
    # order closer than the one before (here 2.6e-2, 3.3e-3, 8.9e-4, 1.7e-4)
    import oracle as o
    rng = np.random.default_rng(8)
    R = rng.uniform(0, 16, (6, 3))
    a0, om, rv = rng.uniform(3, 6, 6), rng.uniform(0.4, 0.9, 6), rng.uniform(3, 4, 6)
    u, _ = o.freq_grid(15)
    ab = o.scs(R, a0, om, rv)                                    # [16, N], exact screening
    m = L.dyson_moments(R, a0, om, rv, u, orders=4)
    al = a0[None] / (1 + u[:, None] ** 2 / om[None] ** 2)
    exact = ab / al
    errs = [np.abs(exact - (1 + sum((-1) ** (q + 1) * m[..., q] for q in range(Q)))).max() for Q in range(1, 5)]
    assert errs[0] > errs[1] > errs[2] > errs[3] and errs[3] < 1e-2 * errs[0]


def test_dyson_moments_invariances():
    rng = np.random.default_rng(9)
    R = rng.uniform(0, 9, (4, 3))
    a0, om, rv = rng.uniform(4, 12, 4), rng.uniform(0.3, 1.2, 4), rng.uniform(3, 4, 4)
    u = np.array([0.0, 0.6, 5.0])
    m = L.dyson_moments(R, a0, om, rv, u)
    th = 0.7
    Rot = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    assert np.allclose(L.dyson_moments(R @ Rot.T + 3.0, a0, om, rv, u), m, rtol=1e-11, atol=1e-15)
    p = np.array([2, 0, 3, 1])
    assert np.allclose(L.dyson_moments(R[p], a0[p], om[p], rv[p], u), m[:, p], rtol=1e-12, atol=1e-15)
