"""Plain FP64 oracle of the learned screening model (NumPy, explicit definitions).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: used by the tests and the benchmark's
CPU leg, never by the product path; it shares no code with the CUDA kernels.

The paper has no learned part; the model below is this project's reading of the task it
stands in for (the screening of Eqs. scs and contraction, Sec. 2.3):
- features of atom i (122): for every other atom j of the same system at distance d < 24 bohr,
  alpha0_j fc(d) G_m(d) summed over j, for 64 Gaussians G_m(d) = exp(-(d - mu_m)^2 / (2 w^2)),
  mu_m = (m + 1/2) w, w = 0.375 bohr (4 radial shells of 6 bohr x 16 Gaussians, width =
  spacing), fc(d) = (1 + cos(pi d / 24)) / 2 (smooth cutoff); then the atom's own TS-scaled
  alpha0, omega, R_vdW and its volume ratio; then the screening moments of the static
  Dyson series (Eqs. scs, contraction at u = 0): with M_i = sum_{j, d<24} alpha0_j
  (1 - f_ij) T^GG_ij (the SCS coupling of Eq. scs-sr-dipole, widths of Eq. mayer),
  m1 = Tr M_i / 3 (first order), m2 = Tr(sum_j alpha0_j (1 - f_ij) T^GG_ij M_j) / 3 (second
  order, two hops), m3 = Tr(M_i M_i) / 3, each also times alpha0_i (m1) or alpha0_i^2 (m2, m3);
  then the Dyson moments at every grid point (48 more): m_q,i(u_k) of dyson_moments below for
  q = 1, 2, 3 and the 16 points u_0 = 0, u_1..u_15 of Eq. (casimir-polder)'s grid, stored
  as feature 74 + 3 k + q - 1 (no distance cutoff);
- standardisation x' = (x - mean) / std with stored mean and std;
- MLP 122 -> 128 -> 128 -> 16, SiLU activations, FP16 weights (rounded; the oracle evaluates
  them exactly in FP64);
- output y_k = log(alpha_bar_i(u_k) / alpha_i(u_k)) at the 16 grid points (u_0 = 0);
- ensemble of members: the prediction is the mean of y over members; the energy error
  estimate is the members' spread of their first-order energies, std_m of
  sum_{i,u} dE/d alpha_bar_i(u) (alpha_bar_m,i(u) - mean over members) with
  alpha_bar_m = alpha exp(y_m) (the adjoints of the screened-parameter chain), per atom and
  times a scale fitted on held-out systems.
"""
from __future__ import annotations

import numpy as np

N_SHELL, N_GAUSS = 4, 16
SHELL = 6.0
CUTOFF = N_SHELL * SHELL
WIDTH = SHELL / N_GAUSS
N_FREQ_POINTS, N_HOPS = 16, 3
N_FEAT_STATIC = N_SHELL * N_GAUSS + 4 + 6
N_FEAT = N_FEAT_STATIC + N_FREQ_POINTS * N_HOPS
HIDDEN = 128
N_OUT = 16
LAYERS = ((N_FEAT, HIDDEN), (HIDDEN, HIDDEN), (HIDDEN, N_OUT))


def centers():
    return (np.arange(N_SHELL * N_GAUSS) + 0.5) * WIDTH


def cutoff_fn(d):
    """fc(d) = (1 + cos(pi d / 24)) / 2 for d < 24, else 0."""
    return np.where(d < CUTOFF, 0.5 * (1.0 + np.cos(np.pi * d / CUTOFF)), 0.0)


def scs_coupling(r, a0_i, a0_j, rv_i, rv_j, beta=0.83, a=6.0):
    """(1 - f) T^GG of one pair at u = 0 (Eqs. scs-sr-dipole, tgg, mayer, fermi-damping), by the
    finite oracle's own tensor and damping routines."""
    from oracle import oracle as orc
    s = np.hypot(orc_sigma(a0_i), orc_sigma(a0_j))
    d = np.linalg.norm(r)
    return (1.0 - orc.fermi(d, rv_i + rv_j, beta, a)) * orc.T_gg(r, s)


def orc_sigma(alpha):
    """Mayer width of Eq. (mayer): (sqrt(2/pi) alpha / 3)^(1/3)."""
    return np.cbrt(np.sqrt(2.0 / np.pi) * alpha / 3.0)


def grid_points():
    """The 16 frequencies of the moments: u_0 = 0 and the 15 nodes of the Casimir-Polder grid."""
    import oracle as o
    return o.freq_grid(N_FREQ_POINTS - 1)[0]


def features(R, a0, om, rv, ratio):
    """Raw features [N, 122] of one system (TS-scaled a0, om, rv), by the definition above,
    one atom pair at a time."""
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
    N = R.shape[0]
    X = np.zeros((N, N_FEAT))
    X[:, :N_FEAT_STATIC] = static_features(R, a0, om, rv, ratio)
    m = dyson_moments(R, a0, om, rv, grid_points(), orders=N_HOPS)   # [16, N, 3]
    X[:, N_FEAT_STATIC:] = m.transpose(1, 0, 2).reshape(N, N_FREQ_POINTS * N_HOPS)
    return X


def static_features(R, a0, om, rv, ratio):
    """The first 74 features (radial Gaussians, own parameters, static moments)."""
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
    N = R.shape[0]
    mu = centers()
    X = np.zeros((N, N_FEAT_STATIC))
    M = np.zeros((N, 3, 3))
    B = {}
    for i in range(N):
        for j in range(N):
            if j == i:
                continue
            d = np.linalg.norm(R[j] - R[i])
            if d >= CUTOFF:
                continue
            X[i, :64] += a0[j] * cutoff_fn(d) * np.exp(-(d - mu) ** 2 / (2.0 * WIDTH ** 2))
            B[i, j] = scs_coupling(R[j] - R[i], a0[i], a0[j], rv[i], rv[j])
            M[i] += a0[j] * B[i, j]
        X[i, 64:68] = (a0[i], om[i], rv[i], ratio[i])
    for i in range(N):
        two_hop = np.zeros((3, 3))
        for j in range(N):
            if (i, j) in B:
                two_hop += a0[j] * B[i, j] @ M[j]
        m1, m2, m3 = np.trace(M[i]) / 3.0, np.trace(two_hop) / 3.0, np.trace(M[i] @ M[i]) / 3.0
        X[i, 68:] = (m1, m2, m3, a0[i] * m1, a0[i] ** 2 * m2, a0[i] ** 2 * m3)
    return X


def feature_position_jacobian(R, a0):
    """dX[i, m] / dR[k, c] for the 64 radial features: [N, 64, N, 3]."""
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
    N = R.shape[0]
    mu = centers()
    J = np.zeros((N, 64, N, 3))
    for i in range(N):
        for j in range(N):
            if j == i:
                continue
            r = R[j] - R[i]
            d = np.linalg.norm(r)
            if d >= CUTOFF:
                continue
            g = np.exp(-(d - mu) ** 2 / (2.0 * WIDTH ** 2))
            fc = cutoff_fn(d)
            dfc = -0.5 * np.pi / CUTOFF * np.sin(np.pi * d / CUTOFF)
            dval = a0[j] * (dfc * g + fc * g * (-(d - mu) / WIDTH ** 2))   # d/dd
            for c in range(3):
                J[i, :, j, c] += dval * r[c] / d
                J[i, :, i, c] -= dval * r[c] / d
    return J


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def round_fp16(params):
    """Weights and biases as the GPU stores them (FP16), returned in FP64."""
    return [(np.asarray(W, np.float16).astype(np.float64), np.asarray(b, np.float16).astype(np.float64))
            for W, b in params]


def forward(Xs, params):
    """MLP on standardised features Xs [B, 122]; params [(W [in, out], b [out])] x 3.
    Returns y [B, 16] and the cache for backward."""
    z1 = Xs @ params[0][0] + params[0][1]
    h1 = silu(z1)
    z2 = h1 @ params[1][0] + params[1][1]
    h2 = silu(z2)
    y = h2 @ params[2][0] + params[2][1]
    return y, (Xs, z1, h1, z2, h2)


def backward(dy, params, cache):
    """Gradients of sum(dy * y) with respect to the weights, biases and the inputs."""
    Xs, z1, h1, z2, h2 = cache
    gW3, gb3 = h2.T @ dy, dy.sum(0)
    dz2 = (dy @ params[2][0].T) * dsilu(z2)
    gW2, gb2 = h1.T @ dz2, dz2.sum(0)
    dz1 = (dz2 @ params[1][0].T) * dsilu(z1)
    gW1, gb1 = Xs.T @ dz1, dz1.sum(0)
    dX = dz1 @ params[0][0].T
    return [(gW1, gb1), (gW2, gb2), (gW3, gb3)], dX


def mse_loss_grad(y, t):
    """Loss mean((y - t)^2) over all entries and its gradient with respect to y."""
    diff = y - t
    return float(np.mean(diff ** 2)), 2.0 * diff / diff.size


def adam_step(p, g, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba), in place; step counts from 1."""
    m[...] = b1 * m + (1 - b1) * g
    v[...] = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    p[...] = p - lr * mh / (np.sqrt(vh) + eps)


def predict_alpha_bar(Xs, members, alpha_u):
    """Ensemble prediction: alpha_bar [16, N] = alpha(u) exp(mean_m y_m) and the spread
    s [16, N] of alpha(u) exp(y_m) over the members (population standard deviation)."""
    ys = np.stack([forward(Xs, p)[0] for p in members])          # [M, N, 16]
    ab_m = alpha_u.T[None, :, :] * np.exp(ys)                   # [M, N, 16]
    ab = alpha_u.T * np.exp(ys.mean(0))
    return ab.T, ab_m.std(0).T


def estimated_error_per_atom(h, alpha_u, ys, scale=1.0):
    """|dE| estimate per atom: scale * std over members m of
    D_m = sum_{u,i} h[u, i] alpha_u[u, i] (exp(y_m[i, u]) - mean_m' exp(y_m'[i, u])), over N.
    h, alpha_u [16, N]; ys [M, N, 16]."""
    v = np.exp(np.transpose(ys, (0, 2, 1)))                      # [M, 16, N]
    D = (h[None] * alpha_u[None] * (v - v.mean(0))).sum(axis=(1, 2))
    return float(scale * np.sqrt(np.mean(D ** 2)) / h.shape[1])


# ---- per-frequency Dyson moments (the inputs a second feature set adds) -----------------
def dyson_moments(R, a0, om, rv, u, orders=3, beta=0.83, a=6.0):
    """Terms of the Dyson series of Eq. scs at each frequency u_k.  With A(u) = alpha(u)^-1 +
    B(u), B_ij = (1 - f_ij) T^GG_ij at the widths of alpha(u) (Eqs. scs-sr-dipole, tgg,
    mayer), A^-1 = sum_q (-alpha B)^q alpha, so the contraction of Eq. contraction reads
        alpha_bar_i(u) / alpha_i(u) = sum_q (-1)^q m_q,i(u),   m_q,i = Tr H^(q)_i / 3,
        H^(0)_i = I,   H^(q)_i = sum_{j != i} alpha_j(u) B_ij(u) H^(q-1)_j   (q-hop sums).
    Returns m [len(u), N, orders] for q = 1..orders, one pair at a time (no cutoff)."""
    from oracle import oracle as orc
    R = np.asarray(R, dtype=np.float64).reshape(-1, 3)
    N = R.shape[0]
    out = np.zeros((len(u), N, orders))
    for k, uk in enumerate(u):
        al = a0 / (1.0 + uk * uk / om ** 2)
        sig = orc_sigma(al)
        B = {}
        for i in range(N):
            for j in range(N):
                if j != i:
                    r = R[j] - R[i]
                    d = np.linalg.norm(r)
                    B[i, j] = (1.0 - orc.fermi(d, rv[i] + rv[j], beta, a)) * orc.T_gg(r, np.hypot(sig[i], sig[j]))
        H = [np.eye(3) for _ in range(N)]
        for q in range(orders):
            Hn = [sum((al[j] * B[i, j] @ H[j] for j in range(N) if j != i), np.zeros((3, 3))) for i in range(N)]
            H = Hn
            out[k, :, q] = [np.trace(h) / 3.0 for h in H]
    return out
