"""ctypes binding of the plain FP64 C oracle (mbd_oracle.c: finite systems, mbd_periodic.c:
periodic systems) -- test infrastructure only.

`build()` compiles the oracle's C files with gcc into oracle/_build/libmbd_oracle.so for the
host it runs on (x86_64 here, aarch64 on the GPU host); `lib()` loads it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(HERE, f) for f in ("mbd_oracle.c", "mbd_periodic.c")]
DEPS = SRCS + [os.path.join(HERE, "mbd_oracle_internal.h")]
OUT_DIR = os.path.join(HERE, "_build")
SO = os.path.join(OUT_DIR, "libmbd_oracle.so")

OK, ERR_INPUT, ERR_NEG_EIGENVALUE, ERR_SCS_NEG_ALPHA, ERR_SINGULAR, ERR_NOT_CONVERGED = range(6)

_lock = threading.Lock()
_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle if the shared object is missing or older than its source."""
    os.makedirs(OUT_DIR, exist_ok=True)
    if force or not os.path.exists(SO) or os.path.getmtime(SO) < max(map(os.path.getmtime, DEPS)):
        tmp = SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", tmp, *SRCS, "-lm"])
        os.replace(tmp, SO)
    return SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            i, d = C.c_int, C.c_double
            P = C.POINTER(C.c_double)
            L.orc_gauss_legendre.argtypes = [i, _dp, _dp]
            L.orc_freq_grid.argtypes = [i, _dp, _dp]
            L.orc_T_bare.argtypes = [_dp, _dp]
            L.orc_T_gg.argtypes = [_dp, d, _dp]
            L.orc_T_erfc.argtypes = [_dp, d, _dp]
            L.orc_T_gg_deriv.argtypes = [_dp, d, _dp, _dp]
            L.orc_T_bare_deriv.argtypes = [_dp, _dp]
            L.orc_fermi.argtypes = [d, d, d, d]
            L.orc_fermi.restype = d
            L.orc_gauss_jordan_inverse.argtypes = [i, _dp, _dp]
            L.orc_jacobi_eigh.argtypes = [i, _dp, _dp, _dp]
            L.orc_ts_scaling.argtypes = [i, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_scs_matrix.argtypes = [i, _dp, _dp, _dp, d, d, _dp]
            L.orc_scs.argtypes = [i, _dp, _dp, _dp, _dp, d, d, i, _dp, _dp, P]
            L.orc_screened_params.argtypes = [i, i, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_mbd_q.argtypes = [i, _dp, _dp, _dp, _dp, d, d, _dp]
            L.orc_energy_from_q.argtypes = [i, _dp, _dp, P, P]
            L.orc_mbd_energy.argtypes = [i, _dp, _dp, _dp, _dp, d, d, P]
            L.orc_mbd_rsscs_energy.argtypes = [i, _dp, _dp, _dp, _dp, _dp, d, d, i, P, P]
            L.orc_mbd_rsscs_gradient.argtypes = [i, _dp, _dp, _dp, _dp, _dp, d, d, i, i, P, _dp, _dp]
            L.orc_mbd_nl.argtypes = [i, _dp, _dp, _dp, _dp, _dp, d, d, P, P, P, P]
            L.orc_mbd_log_energy.argtypes = [i, _dp, _dp, _dp, _dp, d, d, i, i, P, _dp]
            L.orc_mbd_chain.argtypes = [i, i, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, d, d,
                                        _dp, _dp, _dp, _dp]
            L.orc_mbd_chain.restype = None
            L.orc_scs_adjoint_pass.argtypes = [i, i, _dp, _dp, _dp, _dp, _dp, d, d, _dp, _dp, _dp, _dp, _dp, _dp]
            L.orc_scs_adjoint_pass.restype = None
            L.ts_chain.argtypes = [i, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            L.ts_chain.restype = None
            L.alpha_iu.argtypes = [d, d, d]
            L.alpha_iu.restype = d
            # periodic
            L.orc_cell_reciprocal.argtypes = [_dp, _dp, P]
            L.orc_monkhorst_pack.argtypes = [C.POINTER(C.c_int), _dp]
            L.orc_T_erfc_deriv.argtypes = [_dp, d, _dp]
            L.orc_tlr_block.argtypes = [_dp, _dp, i, _dp, d, d, d, d, d, d, i, _dp, P, P, P]
            L.orc_tlr_block.restype = None
            L.orc_ewald_T.argtypes = [i, _dp, _dp, _dp, d, d, d, _dp]
            L.orc_periodic_q.argtypes = [i, _dp, _dp, _dp, _dp, _dp, _dp, d, d, d, d, d, _dp]
            L.orc_hermitian_sqrt.argtypes = [i, _dp, P, P, P]
            L.orc_periodic_scs_matrix.argtypes = [i, _dp, _dp, _dp, _dp, d, d, d, _dp]
            L.orc_periodic_rsscs_energy.argtypes = [i, _dp, _dp, i, _dp, _dp, _dp, _dp, _dp, d, d, i,
                                                    d, d, d, P, P]
            L.orc_periodic_rsscs_gradient.argtypes = [i, _dp, _dp, i, _dp, _dp, _dp, _dp, _dp, d, d, i,
                                                      d, d, d, P, _dp, _dp, _dp]
            _lib = L
    return _lib


def _a(x, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    return a.reshape(shape) if shape is not None else a


class OracleError(RuntimeError):
    def __init__(self, code, where):
        super().__init__(f"oracle {where} failed with code {code}")
        self.code = code


def _check(rc, where):
    if rc != OK:
        raise OracleError(rc, where)


# ---- elementary pieces -------------------------------------------------------------
def gauss_legendre(n):
    x, w = np.zeros(n), np.zeros(n)
    _check(lib().orc_gauss_legendre(n, x, w), "gauss_legendre")
    return x, w


def freq_grid(n_freq=15):
    u, w = np.zeros(n_freq + 1), np.zeros(n_freq + 1)
    _check(lib().orc_freq_grid(n_freq, u, w), "freq_grid")
    return u, w


def T_bare(r):
    T = np.zeros(9); lib().orc_T_bare(_a(r), T); return T.reshape(3, 3)


def T_gg(r, s):
    T = np.zeros(9); lib().orc_T_gg(_a(r), float(s), T); return T.reshape(3, 3)


def T_erfc(r, gamma):
    T = np.zeros(9); lib().orc_T_erfc(_a(r), float(gamma), T); return T.reshape(3, 3)


def T_gg_deriv(r, s):
    dr, ds = np.zeros(27), np.zeros(9)
    lib().orc_T_gg_deriv(_a(r), float(s), dr, ds)
    return dr.reshape(3, 3, 3), ds.reshape(3, 3)


def T_bare_deriv(r):
    dr = np.zeros(27); lib().orc_T_bare_deriv(_a(r), dr); return dr.reshape(3, 3, 3)


def fermi(rho, rsum, sr, a):
    return lib().orc_fermi(float(rho), float(rsum), float(sr), float(a))


def inverse(A):
    A = _a(A); n = A.shape[0]; out = np.zeros_like(A)
    _check(lib().orc_gauss_jordan_inverse(n, A, out), "gauss_jordan_inverse")
    return out


def eigh(A):
    A = _a(A); n = A.shape[0]; lam = np.zeros(n); V = np.zeros_like(A)
    _check(lib().orc_jacobi_eigh(n, A, lam, V), "jacobi_eigh")
    return lam, V


def ts_scaling(a0ref, c6ref, rref, ratio):
    N = len(a0ref); a0, om, rv = np.zeros(N), np.zeros(N), np.zeros(N)
    lib().orc_ts_scaling(N, _a(a0ref), _a(c6ref), _a(rref), _a(ratio), a0, om, rv)
    return a0, om, rv


def dyn_alpha(alpha0, omega, u):
    """alpha_i(iu), Eq. (dyn-pol), per atom."""
    return np.array([lib().alpha_iu(float(a0), float(w), float(u)) for a0, w in zip(alpha0, omega)])


def scs_matrix(R, alpha, rvdw, beta=0.83, a=6.0):
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    M = np.zeros((3 * N, 3 * N))
    lib().orc_scs_matrix(N, R, _a(alpha), _a(rvdw), beta, a, M)
    return M


def scs(R, alpha0, omega, rvdw, beta=0.83, a=6.0, n_freq=15):
    """alpha_bar[k, i] for k = 0..n_freq (u_0 = 0)."""
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    u, _ = freq_grid(n_freq)
    ab = np.zeros((n_freq + 1, N))
    _check(lib().orc_scs(N, R, _a(alpha0), _a(omega), _a(rvdw), beta, a, n_freq, u, ab, None), "scs")
    return ab


def screened_params(alpha_bar, alpha0, rvdw, n_freq=15):
    N = alpha_bar.shape[1]; _, wu = freq_grid(n_freq)
    outs = [np.zeros(N) for _ in range(4)]
    rc = lib().orc_screened_params(N, n_freq, _a(alpha_bar), wu, _a(alpha0), _a(rvdw), *outs)
    return rc, tuple(outs)  # abar0, c6bar, ombar, rbar


def mbd_q(R, alpha0, omega, rdamp, beta=0.83, a=6.0):
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    Q = np.zeros((3 * N, 3 * N))
    lib().orc_mbd_q(N, R, _a(alpha0), _a(omega), _a(rdamp), beta, a, Q)
    return Q


def energy_from_q(Q, omega, want_z=False):
    Q = _a(Q); N = Q.shape[0] // 3
    E = C.c_double()
    Z = np.zeros_like(Q) if want_z else None
    _check(lib().orc_energy_from_q(N, Q, _a(omega), C.byref(E),
                                   Z.ctypes.data_as(C.POINTER(C.c_double)) if want_z else None),
           "energy_from_q")
    return (E.value, Z) if want_z else E.value


def mbd_energy(R, alpha0, omega, rdamp, beta=0.83, a=6.0):
    """Unscreened MBD energy of given oscillators (damping radii rdamp)."""
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    E = C.c_double()
    _check(lib().orc_mbd_energy(N, R, _a(alpha0), _a(omega), _a(rdamp), beta, a, C.byref(E)),
           "mbd_energy")
    return E.value


def mbd_rsscs_energy(R, a0ref, c6ref, rref, ratio, beta=0.83, a=6.0, n_freq=15, detail=False):
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    E = C.c_double()
    det = np.zeros((n_freq + 4) * N)
    rc = lib().orc_mbd_rsscs_energy(N, R, _a(a0ref), _a(c6ref), _a(rref), _a(ratio), beta, a,
                                    n_freq, C.byref(E), det.ctypes.data_as(C.POINTER(C.c_double)))
    _check(rc, "mbd_rsscs_energy")
    if not detail:
        return E.value
    return E.value, dict(alpha_bar=det[:(n_freq + 1) * N].reshape(n_freq + 1, N),
                         c6=det[(n_freq + 1) * N:(n_freq + 2) * N],
                         omega=det[(n_freq + 2) * N:(n_freq + 3) * N],
                         rvdw=det[(n_freq + 3) * N:])


def mbd_rsscs_gradient(R, a0ref, c6ref, rref, ratio, beta=0.83, a=6.0, n_freq=15, mode="adjoint"):
    """Energy, dE/dR [N,3], dE/d(alpha0_ref, C6_ref, R_ref, ratio) [4,N].
    mode: "forward" (per-input forward mode with the paper's fused SCS formula) or
    "adjoint"."""
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    E = C.c_double()
    gR, gp = np.zeros((N, 3)), np.zeros((4, N))
    rc = lib().orc_mbd_rsscs_gradient(N, R, _a(a0ref), _a(c6ref), _a(rref), _a(ratio), beta, a,
                                      n_freq, 0 if mode == "forward" else 1, C.byref(E), gR, gp)
    _check(rc, "mbd_rsscs_gradient")
    return E.value, gR, gp


def gradient_from_dense_steps(R, a0ref, c6ref, rref, ratio, alpha_bar, X, Z, solve, beta=0.83, a=6.0, n_freq=15):
    """The oracle's adjoint gradient (Eqs. mbd-gradient, scs-gradient) with its two dense steps
    supplied by the caller: X [nf+1, n, 3] = M(u_k)^{-1} E and Z = Q^{-1/2} (n x n), and
    solve(k, H) -> M(u_k)^{-1} H for the adjoint right-hand sides.  Every other step (TS
    scaling, screened parameters, the MBD pair pass and chain, the SCS pair pass, the TS
    chain) is the oracle's.  Returns dE/dR [N,3], dE/d(alpha0_ref, C6_ref, R_ref, ratio) [4,N]."""
    R = _a(R).reshape(-1, 3); N = R.shape[0]; n = 3 * N; nf = n_freq
    a0, om, rv = ts_scaling(a0ref, c6ref, rref, ratio)
    u, wu = freq_grid(nf)
    rc, (abar0, c6bar, ombar, rbar) = screened_params(alpha_bar, a0, rv, nf)
    _check(rc, "gradient_from_dense_steps")
    h = np.zeros((nf + 1) * N); g_a0, g_om, g_rv, gR = np.zeros(N), np.zeros(N), np.zeros(N), np.zeros(3 * N)
    lib().orc_mbd_chain(N, nf, R, a0, rv, _a(alpha_bar), abar0, c6bar, ombar, rbar, wu, _a(Z), beta, a, h, g_a0,
                        g_rv, gR)
    h = h.reshape(nf + 1, N)
    V = np.zeros((nf + 1, n, 3))
    for k in range(nf + 1):
        H = np.zeros((n, 3))
        for c in range(3):
            H[c::3, c] = h[k]
        V[k] = solve(k, H)
    lib().orc_scs_adjoint_pass(N, nf, R, a0, om, rv, u, beta, a, _a(X), _a(V), g_a0, g_om, g_rv, gR)
    gp = np.zeros(4 * N)
    lib().ts_chain(N, _a(a0ref), _a(c6ref), _a(rref), _a(ratio), g_a0, g_om, g_rv, gp)
    return gR.reshape(N, 3), gp.reshape(4, N)


def mbd_log_energy(R, alpha0, omega, rdamp, beta=0.83, a=6.0, n_freq=15, max_order=2):
    """MBD energy of given oscillators by the log formula (Eq. log-formula) on the n_freq-point
    frequency grid, and its many-body orders E^(2..max_order) (Eq. rpa).  Returns
    (E, orders [max_order - 1])."""
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    E = C.c_double()
    orders = np.zeros(max(max_order - 1, 1))
    _check(lib().orc_mbd_log_energy(N, R, _a(alpha0), _a(omega), _a(rdamp), beta, a, n_freq, max_order,
                                    C.byref(E), orders), "mbd_log_energy")
    return E.value, orders[:max_order - 1]


def mbd_nl(R, a0ref, c6ref, ra, rw, beta=0.83, a=6.0, grad=False, detail=False):
    """MBD-NL energy (Sec. 2.7, Eqs. mbd-nl-scaling, mbd-nl-rvdw): no screening, oscillators
    from the free-atom reference (alpha0_ref, C6_ref) and the density-functional ratios
    ra = alpha0_df/alpha0_df,ref, rw = omega_df/omega_df,ref.  grad: also dE/dR [N,3] and
    dE/d(alpha0_ref, C6_ref, ra, rw) [4,N].  detail: also the oscillators (alpha0, omega,
    R_damp) [3,N]."""
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    E = C.c_double()
    gR, gp, par = np.zeros((N, 3)), np.zeros((4, N)), np.zeros((3, N))
    ptr = lambda x: x.ctypes.data_as(C.POINTER(C.c_double))
    rc = lib().orc_mbd_nl(N, R, _a(a0ref), _a(c6ref), _a(ra), _a(rw), beta, a, C.byref(E),
                          ptr(gR) if grad else None, ptr(gp) if grad else None, ptr(par))
    _check(rc, "mbd_nl")
    out = (E.value, gR, gp) if grad else (E.value,)
    if detail:
        out = out + (par,)
    return out if len(out) > 1 else out[0]


def system_args(sys):
    """(R, alpha0_ref, c6_ref, rvdw_ref, ratio) of a synthetic.System."""
    return sys.coords, sys.alpha0_ref, sys.c6_ref, sys.rvdw_ref, sys.ratio


# ---- periodic systems (mbd_periodic.c) ---------------------------------------------
def _ptr(x):
    return None if x is None else x.ctypes.data_as(C.POINTER(C.c_double))


def _cplx(buf, shape):
    return buf.view(np.complex128).reshape(shape)


def cell_reciprocal(A):
    """(B, volume): rows of B are the reciprocal vectors, a_c . b_d = 2 pi delta_cd."""
    B, vol = np.zeros(9), C.c_double()
    _check(lib().orc_cell_reciprocal(_a(A).reshape(9), B, C.byref(vol)), "cell_reciprocal")
    return B.reshape(3, 3), vol.value


def monkhorst_pack(grid):
    g = (C.c_int * 3)(*[int(x) for x in grid])
    out = np.zeros(3 * int(np.prod(grid)))
    lib().orc_monkhorst_pack(g, out)
    return out.reshape(-1, 3)


def T_erfc_deriv(r, gamma):
    dr = np.zeros(27); lib().orc_T_erfc_deriv(_a(r), float(gamma), dr); return dr.reshape(3, 3, 3)


def tlr_block(A, x, same, kappa, gamma, rc, kc, rsum=1.0, beta=0.83, a=6.0, damp=True, derivs=False):
    """T^lr(q) block (3x3 complex) for separation x; with derivs also d/dx [3,3,3],
    d/dS [3,3] and d/dA [3,3,3,3] (indices c, d, a, b)."""
    T = np.zeros(18)
    dx, dS, dA = (np.zeros(54), np.zeros(18), np.zeros(162)) if derivs else (None, None, None)
    lib().orc_tlr_block(_a(A).reshape(9), _a(x), int(same), _a(kappa), float(gamma), float(rc), float(kc),
                        float(rsum), float(beta), float(a), int(bool(damp)), T, _ptr(dx), _ptr(dS), _ptr(dA))
    if not derivs:
        return _cplx(T, (3, 3))
    return _cplx(T, (3, 3)), _cplx(dx, (3, 3, 3)), _cplx(dS, (3, 3)), _cplx(dA, (3, 3, 3, 3))


def ewald_T(R, A, kappa, gamma, rc, kc):
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    out = np.zeros(2 * (3 * N) ** 2)
    lib().orc_ewald_T(N, R, _a(A).reshape(9), _a(kappa), float(gamma), float(rc), float(kc), out)
    return _cplx(out, (3 * N, 3 * N))


def periodic_q(R, A, kappa, alpha0, omega, rdamp, gamma, rc, kc, beta=0.83, a=6.0):
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    out = np.zeros(2 * (3 * N) ** 2)
    lib().orc_periodic_q(N, R, _a(A).reshape(9), _a(kappa), _a(alpha0), _a(omega), _a(rdamp), beta, a,
                         float(gamma), float(rc), float(kc), out)
    return _cplx(out, (3 * N, 3 * N))


def hermitian_sqrt(Q, want_z=False):
    """(1/2 Tr Q^{1/2}, eigenvalues ascending[, Q^{-1/2}]) of a Hermitian matrix."""
    Q = np.ascontiguousarray(np.asarray(Q, dtype=np.complex128))
    n = Q.shape[0]
    h, lam = C.c_double(), np.zeros(n)
    Z = np.zeros(2 * n * n) if want_z else None
    _check(lib().orc_hermitian_sqrt(n, Q.view(np.float64).reshape(-1), C.byref(h), _ptr(Z), _ptr(lam)),
           "hermitian_sqrt")
    return (h.value, lam, _cplx(Z, (n, n))) if want_z else (h.value, lam)


def periodic_scs_matrix(R, A, alpha, rvdw, rc, beta=0.83, a=6.0):
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    M = np.zeros((3 * N, 3 * N))
    _check(lib().orc_periodic_scs_matrix(N, R, _a(A).reshape(9), _a(alpha), _a(rvdw), beta, a, float(rc), M),
           "periodic_scs_matrix")
    return M


def periodic_rsscs_energy(R, A, kappa, a0ref, c6ref, rref, ratio, gamma, rc, kc, beta=0.83, a=6.0,
                          n_freq=15, detail=False):
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    kappa = _a(kappa).reshape(-1, 3); nk = kappa.shape[0]
    E = C.c_double()
    det = np.zeros((n_freq + 4) * N + nk)
    rc0 = lib().orc_periodic_rsscs_energy(N, R, _a(A).reshape(9), nk, kappa, _a(a0ref), _a(c6ref), _a(rref),
                                          _a(ratio), beta, a, n_freq, float(gamma), float(rc), float(kc),
                                          C.byref(E), _ptr(det))
    _check(rc0, "periodic_rsscs_energy")
    if not detail:
        return E.value
    o = (n_freq + 1) * N
    return E.value, dict(alpha_bar=det[:o].reshape(n_freq + 1, N), c6=det[o:o + N], omega=det[o + N:o + 2 * N],
                         rvdw=det[o + 2 * N:o + 3 * N], e_q=det[o + 3 * N:])


def periodic_rsscs_gradient(R, A, kappa, a0ref, c6ref, rref, ratio, gamma, rc, kc, beta=0.83, a=6.0,
                            n_freq=15):
    """Energy, dE/dR [N,3], dE/dA [3,3] (Cartesian positions fixed), dE/dparams [4,N]."""
    R = _a(R).reshape(-1, 3); N = R.shape[0]
    kappa = _a(kappa).reshape(-1, 3); nk = kappa.shape[0]
    E = C.c_double()
    gR, gA, gp = np.zeros((N, 3)), np.zeros((3, 3)), np.zeros((4, N))
    rc0 = lib().orc_periodic_rsscs_gradient(N, R, _a(A).reshape(9), nk, kappa, _a(a0ref), _a(c6ref), _a(rref),
                                            _a(ratio), beta, a, n_freq, float(gamma), float(rc), float(kc),
                                            C.byref(E), gR, gA, gp)
    _check(rc0, "periodic_rsscs_gradient")
    return E.value, gR, gA, gp
