"""TS pairwise dispersion, CPU oracle (test infrastructure only; nothing in the product path
imports it).

Finite systems (Secs. 2.6 and 2.7, Eq. pairwise with the TS parametrization, Eqs. ts-scaling and
fermi-damping):
    E = -1/2 sum_{i != j} C6_ij f_ij / R_ij^6,   C6_ij = 3/2 a_i a_j / (1/w_i + 1/w_j),
    a_i = alpha0_ref,i v_i, w_i = 4 C6_ref,i / (3 alpha0_ref,i^2), R_i = R_ref,i v_i^(1/3),
    f_ij = 1 / (1 + exp(-d (R_ij / (s_R (R_i + R_j)) - 1))),  d = 20.
Periodic systems (Eq. ts-ewald, readings in the notes of ewald_inverse_r6):
    E (per cell) = -1/2 sum_{i,j in cell} C6_ij sum'_n f(R_nij) / R_nij^6,
with sum'_n f/R^6 = [Ewald sum of 1/R^6] - [real-space sum of (1 - f)/R^6].
Plain numpy with explicit loops over image vectors; written for clarity, not speed.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

D_TS = 20.0   # steepness of the TS Fermi damping (Sec. 2.7, paragraph TS)


def ts_params(a0ref, c6ref, rref, ratio):
    """Eq. (ts-scaling): alpha0 = alpha0_ref v, omega = 4 C6_ref / (3 alpha0_ref^2),
    R_vdW = R_ref v^(1/3)."""
    a0ref, c6ref, rref, v = (np.asarray(x, float) for x in (a0ref, c6ref, rref, ratio))
    return a0ref * v, 4.0 * c6ref / (3.0 * a0ref ** 2), rref * np.cbrt(v)


def c6_matrix(a0, om):
    """Eq. (pairwise): C6_ij = 3/2 a_i a_j / (1/w_i + 1/w_j)."""
    return 1.5 * np.outer(a0, a0) / (1.0 / om[:, None] + 1.0 / om[None, :])


def fermi(r, rsum, s_r, d=D_TS):
    """Eq. (fermi-damping) and its derivatives d f/d r, d f/d rsum."""
    eta = r / (s_r * rsum)
    f = 1.0 / (1.0 + np.exp(-d * (eta - 1.0)))
    dfe = d * f * (1.0 - f)
    return f, dfe / (s_r * rsum), -dfe * eta / rsum


def ts_energy(R, a0ref, c6ref, rref, ratio, s_r=0.94, d=D_TS, grad=False):
    """Finite TS energy; with grad also dE/dR [N,3] and dE/d(alpha0_ref, C6_ref, R_ref, v) [4,N]."""
    R = np.asarray(R, float).reshape(-1, 3)
    N = len(R)
    a0, om, rv = ts_params(a0ref, c6ref, rref, ratio)
    C6 = c6_matrix(a0, om)
    E = 0.0
    gR = np.zeros((N, 3))
    gC6 = np.zeros((N, N))      # dE/dC6_ij (ordered pairs)
    grv = np.zeros(N)
    for i in range(N):
        for j in range(N):
            if i == j:
                continue
            r = R[j] - R[i]
            rr = math.sqrt(r @ r)
            f, dfr, dfs = fermi(rr, rv[i] + rv[j], s_r, d)
            e = -0.5 * C6[i, j] * f / rr ** 6
            E += e
            if grad:
                de_dr = -0.5 * C6[i, j] * (dfr / rr ** 6 - 6.0 * f / rr ** 7)
                gR[j] += de_dr * r / rr
                gR[i] -= de_dr * r / rr
                gC6[i, j] += -0.5 * f / rr ** 6
                grv[i] += -0.5 * C6[i, j] * dfs / rr ** 6
                grv[j] += -0.5 * C6[i, j] * dfs / rr ** 6
    if not grad:
        return E
    ga0, gom = _c6_chain(a0, om, gC6)
    return E, gR, _ts_chain(a0ref, c6ref, rref, ratio, ga0, gom, grv)


def _c6_chain(a0, om, gC6):
    """dE/d a_i and dE/d w_i from dE/dC6_ij through C6_ij = 3/2 a_i a_j w_i w_j / (w_i + w_j)
    (for i = j the two factors of each kind give C6_ii' = 2 C6_ii/a_i and C6_ii/w_i)."""
    N = len(a0)
    ga0, gom = np.zeros(N), np.zeros(N)
    for i in range(N):
        for j in range(N):
            if gC6[i, j] == 0.0:         # finite systems: no i = j term; periodic: the images
                continue
            c = 1.5 * a0[i] * a0[j] * om[i] * om[j] / (om[i] + om[j])
            ga0[i] += gC6[i, j] * c / a0[i]
            ga0[j] += gC6[i, j] * c / a0[j]
            gom[i] += gC6[i, j] * c * (1.0 / om[i] - 1.0 / (om[i] + om[j]))
            gom[j] += gC6[i, j] * c * (1.0 / om[j] - 1.0 / (om[i] + om[j]))
    return ga0, gom


def _ts_chain(a0ref, c6ref, rref, ratio, ga0, gom, grv):
    """Chain through Eq. (ts-scaling) to (alpha0_ref, C6_ref, R_ref, v)."""
    a0ref, c6ref, rref, v = (np.asarray(x, float) for x in (a0ref, c6ref, rref, ratio))
    om = 4.0 * c6ref / (3.0 * a0ref ** 2)
    return np.array([ga0 * v - gom * 2.0 * om / a0ref,
                     gom * om / c6ref,
                     grv * np.cbrt(v),
                     ga0 * a0ref + grv * rref / (3.0 * np.cbrt(v) ** 2)])


# ---- periodic ---------------------------------------------------------------------------
def phi_r(x):
    """Real-space kernel of Eq. (ts-ewald): (1/x^6 + 1/x^4 + 1/(2 x^2)) exp(-x^2)."""
    return (1.0 / x ** 6 + 1.0 / x ** 4 + 0.5 / x ** 2) * np.exp(-x * x)


def phi_k(k):
    """Reciprocal kernel of Eq. (ts-ewald): pi^(3/2)/12 ((4 - 2k^2) e^{-k^2/4} + k^3 sqrt(pi) erfc(k/2))."""
    return math.pi ** 1.5 / 12.0 * ((4.0 - 2.0 * k * k) * np.exp(-k * k / 4.0) + k ** 3 * math.sqrt(math.pi) * erfc(k / 2.0))


def _images(A, rc):
    """Integer image vectors n (as n A) with |n A| possibly below rc + the cell diameter."""
    A = np.asarray(A, float)
    B = np.linalg.inv(A).T   # rows: reciprocal vectors / (2 pi)
    diam = np.linalg.norm(A.sum(0)) + sum(np.linalg.norm(a) for a in A)
    m = [int(math.ceil((rc + diam) * np.linalg.norm(B[c]))) for c in range(3)]
    ns = np.array(np.meshgrid(*[np.arange(-mc, mc + 1) for mc in m], indexing="ij")).reshape(3, -1).T
    return ns @ A


def ewald_inverse_r6(R, A, gamma, rc, kc):
    """S[i, j] = sum'_n 1/|R_j + n A - R_i|^6 by Eq. (ts-ewald), with these readings of the
    printed formula: the phase factor is cos(G . (R_j - R_i)); the G = 0 term, gamma^3
    phi_k(0)/Omega = pi^(3/2) gamma^3/(3 Omega), belongs to the sum (the split
    1/r^6 = gamma^6 phi_r(gamma r) + 1/2 int_0^{gamma^2} t^2 e^{-r^2 t} dt makes the
    long-range part smooth at G = 0); the self correction for i = j is -gamma^6/6 (the
    long-range part at r = 0, which the reciprocal sum contains and the primed sum excludes)."""
    R = np.asarray(R, float).reshape(-1, 3)
    A = np.asarray(A, float)
    N = len(R)
    Om = abs(np.linalg.det(A))
    Bm = 2.0 * math.pi * np.linalg.inv(A).T
    shifts = _images(A, rc)
    # G = m B with |G| < kc: |m_c| = |G . A_c| / (2 pi) <= kc |A_c| / (2 pi)
    mg = [int(math.ceil(kc * np.linalg.norm(A[c]) / (2.0 * math.pi))) + 1 for c in range(3)]
    ms = np.array(np.meshgrid(*[np.arange(-m, m + 1) for m in mg], indexing="ij")).reshape(3, -1).T
    G = ms @ Bm
    G = G[np.linalg.norm(G, axis=1) < kc]
    Gn = np.linalg.norm(G, axis=1)
    S = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            d = R[j] + shifts - R[i]
            rn = np.linalg.norm(d, axis=1)
            sel = (rn > 1e-12) & (rn < rc)
            real = np.sum(gamma ** 6 * phi_r(gamma * rn[sel]))
            rec = np.sum(gamma ** 3 * phi_k(Gn / gamma) * np.cos(G @ (R[j] - R[i]))) / Om
            S[i, j] = real + rec - (gamma ** 6 / 6.0 if i == j else 0.0)
    return S


def damped_away_sum(R, A, rv, s_r, rc, d=D_TS):
    """Dm[i, j] = sum'_{|R_nij| < rc} (1 - f(R_nij)) / R_nij^6 (short range: 1 - f decays as
    exp(-d (eta - 1)))."""
    R = np.asarray(R, float).reshape(-1, 3)
    N = len(R)
    shifts = _images(A, rc)
    Dm = np.zeros((N, N))
    for i in range(N):
        for j in range(N):
            rn = np.linalg.norm(R[j] + shifts - R[i], axis=1)
            rn = rn[(rn > 1e-12) & (rn < rc)]
            f, _, _ = fermi(rn, rv[i] + rv[j], s_r, d)
            Dm[i, j] = np.sum((1.0 - f) / rn ** 6)
    return Dm


def ts_energy_periodic(R, A, a0ref, c6ref, rref, ratio, gamma, rc, kc, s_r=0.94, d=D_TS, grad=False):
    """Periodic TS energy per cell by Eq. (ts-ewald) for the bare sum minus the damped-away
    real-space part.  With grad also dE/dR [N,3], dE/dA [3,3] (rows of A are the lattice
    vectors; Cartesian positions, gamma and the cutoffs held fixed) and
    dE/d(alpha0_ref, C6_ref, R_ref, v) [4,N]."""
    a0, om, rv = ts_params(a0ref, c6ref, rref, ratio)
    C6 = c6_matrix(a0, om)
    S = ewald_inverse_r6(R, A, gamma, rc, kc)
    Dm = damped_away_sum(R, A, rv, s_r, rc, d)
    E = -0.5 * float(np.sum(C6 * (S - Dm)))
    if not grad:
        return E
    gR, gA, grv = _periodic_geometry_grad(R, A, C6, rv, gamma, rc, kc, s_r, d)
    ga0, gom = _c6_chain(a0, om, -0.5 * (S - Dm))
    return E, gR, gA, _ts_chain(a0ref, c6ref, rref, ratio, ga0, gom, grv)


def _phi_r_prime(x):
    """d phi_r / dx."""
    e = np.exp(-x * x)
    return (-6.0 / x ** 7 - 4.0 / x ** 5 - 1.0 / x ** 3) * e - 2.0 * x * phi_r(x)


def _phi_k_prime(k):
    """d phi_k / dk; the erfc term's derivative cancels against part of the Gaussian's."""
    return math.pi ** 1.5 / 12.0 * (-4.0 * k * np.exp(-k * k / 4.0) - 0.5 * k * (4.0 - 2.0 * k * k) * np.exp(-k * k / 4.0)
                                    + 3.0 * k * k * math.sqrt(math.pi) * erfc(k / 2.0) - k ** 3 * np.exp(-k * k / 4.0))


def _periodic_geometry_grad(R, A, C6, rv, gamma, rc, kc, s_r, d):
    """dE/dR, dE/dA and dE/dR_vdW of E = -1/2 sum_ij C6_ij (S_ij - Dm_ij), term by term:
    real-space images h(r) = gamma^6 phi_r(gamma r) - (1 - f(r))/r^6 with R_nij = R_j + n A - R_i,
    and reciprocal terms gamma^3 phi_k(|G|/gamma) cos(G . (R_j - R_i)) / Omega with
    G = m B, B = 2 pi A^-T, Omega = |det A| (dB = -B dA^T B / (2 pi), dOmega = Omega A^-T dA)."""
    R = np.asarray(R, float).reshape(-1, 3)
    A = np.asarray(A, float)
    N = len(R)
    Om = abs(np.linalg.det(A))
    AinvT = np.linalg.inv(A).T
    Bm = 2.0 * math.pi * AinvT
    nvec = _images_int(A, rc)
    shifts = nvec @ A
    mg = [int(math.ceil(kc * np.linalg.norm(A[c]) / (2.0 * math.pi))) + 1 for c in range(3)]
    ms = np.array(np.meshgrid(*[np.arange(-m, m + 1) for m in mg], indexing="ij")).reshape(3, -1).T
    G = ms @ Bm
    G = G[np.linalg.norm(G, axis=1) < kc]
    Gn = np.linalg.norm(G, axis=1)
    gR = np.zeros((N, 3))
    gA = np.zeros((3, 3))
    grv = np.zeros(N)
    for i in range(N):
        for j in range(N):
            c = -0.5 * C6[i, j]
            # real space
            rvec = R[j] + shifts - R[i]
            rn = np.linalg.norm(rvec, axis=1)
            sel = (rn > 1e-12) & (rn < rc)
            r, v, n = rn[sel], rvec[sel], nvec[sel]
            f, dfr, dfs = fermi(r, rv[i] + rv[j], s_r, d)
            dh = gamma ** 7 * _phi_r_prime(gamma * r) + dfr / r ** 6 + 6.0 * (1.0 - f) / r ** 7
            w = (c * dh / r)[:, None] * v            # dE/d(R_nij)
            gR[j] += w.sum(0)
            gR[i] -= w.sum(0)
            gA += n.T @ w                            # d R_nij / d A_cd = n_c
            gsum = c * np.sum(dfs / r ** 6)          # -(1 - f) term: d/d rsum of -(1-f) = +df/drsum
            grv[i] += gsum
            grv[j] += gsum
            # reciprocal space
            dij = R[j] - R[i]
            ph = G @ dij
            t = gamma ** 3 * phi_k(Gn / gamma) / Om
            gk = np.zeros_like(G)
            nz = Gn > 0
            gk[nz] = (gamma ** 2 * _phi_k_prime(Gn[nz] / gamma) / Om * np.cos(ph[nz]) / Gn[nz])[:, None] * G[nz]
            gk -= (t * np.sin(ph))[:, None] * dij[None, :]    # d term / d G
            wsin = c * t * np.sin(ph)
            gR[j] -= wsin @ G
            gR[i] += wsin @ G
            # d/dA_fc through G: dG_e = -sum G_c B_fe dA_fc / (2 pi); through Omega: -t/Omega dOmega
            gA += -c * (Bm @ (gk.T @ G)) / (2.0 * math.pi)
            gA += -c * np.sum(t * np.cos(ph)) * AinvT
    return gR, gA, grv


def _images_int(A, rc):
    """Integer image vectors n with |n A| possibly below rc + the cell diameter (as _images)."""
    A = np.asarray(A, float)
    B = np.linalg.inv(A).T
    diam = np.linalg.norm(A.sum(0)) + sum(np.linalg.norm(a) for a in A)
    m = [int(math.ceil((rc + diam) * np.linalg.norm(B[c]))) for c in range(3)]
    return np.array(np.meshgrid(*[np.arange(-mc, mc + 1) for mc in m], indexing="ij")).reshape(3, -1).T.astype(float)


def ts_energy_periodic_direct(R, A, a0ref, c6ref, rref, ratio, r_big, s_r=0.94, d=D_TS):
    """The same energy by the plain (absolutely convergent) lattice sum of f/R^6 up to r_big,
    plus the continuum estimate of the tail, -1/2 sum_ij C6_ij 4 pi / (3 Omega r_big^3)."""
    R = np.asarray(R, float).reshape(-1, 3)
    N = len(R)
    a0, om, rv = ts_params(a0ref, c6ref, rref, ratio)
    C6 = c6_matrix(a0, om)
    Om = abs(np.linalg.det(np.asarray(A, float)))
    shifts = _images(A, r_big)
    E = 0.0
    for i in range(N):
        for j in range(N):
            rn = np.linalg.norm(R[j] + shifts - R[i], axis=1)
            rn = rn[(rn > 1e-12) & (rn < r_big)]
            f, _, _ = fermi(rn, rv[i] + rv[j], s_r, d)
            E += -0.5 * C6[i, j] * (np.sum(f / rn ** 6) + 4.0 * math.pi / (3.0 * Om * r_big ** 3))
    return E
