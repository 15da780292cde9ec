"""Thin ctypes binding of libmbdgb.so (C ABI in include/mbd_gb300.h).

Argument marshalling only: every step of the computation runs in the library's CUDA
kernels.  The functions keep the C names (mbd_create, mbd_set_geometry, ...); the
class `MBD` bundles them for convenience.  There is no CPU fallback: if the library
is missing, `load()` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_PATH = _build.LIB

MBD_OK = 0
ERRORS = {1: "MBD_ERR_INPUT", 2: "MBD_ERR_NEG_EIGENVALUE", 3: "MBD_ERR_SCS_NEG_ALPHA",
          4: "MBD_ERR_SCS_NOT_PD", 5: "MBD_ERR_NOT_CONVERGED", 6: "MBD_ERR_CUDA",
          7: "MBD_ERR_STATE", 8: "MBD_ERR_UNSUPPORTED", 9: "MBD_ERR_SCRATCH_LIMIT"}
MBD_PREC_FP64, MBD_PREC_TF32, MBD_PREC_BF16X3, MBD_PREC_TF32X3, MBD_PREC_FP64_SPLIT = 0, 1, 2, 3, 4

# Every symbol declared in include/mbd_gb300.h.
EXPORTS = ("mbd_default_options", "mbd_create", "mbd_destroy", "mbd_set_geometry",
           "mbd_set_free_atom_params", "mbd_evaluate", "mbd_evaluate_dev", "mbd_backward_dev",
           "mbd_get_evaluation_count",
           "mbd_get_lattice_gradient", "mbd_set_scs_model", "mbd_get_learned_stats", "mbd_screen",
           "mbd_get_scs_detail", "mbd_log_energy", "mbd_ts_energy",
           "mbd_get_stats", "mbd_get_exception", "mbd_set_profiling", "mbd_get_profile",
           "mbdk_gemm_f64", "mbdk_gemm_tc", "mbdk_tc_wait_check", "mbdk_gemm_f64_split", "mbdk_gemm_f64_split_work_bytes", "mbdk_cholesky_f64", "mbdk_chol_solve3_f64",
           "mbdk_cholesky_solve3_f64_noalloc", "mbdk_scs_features", "mbdk_mlp_forward", "mbdk_mlp_backward",
           "mbdk_mse_grad", "mbdk_adam_step", "mbdk_learned_targets", "mbdk_gather_rows")
LEARNED_FEATURES, LEARNED_OUTPUTS, LEARNED_PARAMS, LEARNED_WORK = 122, 16, 34320, 144


class mbd_options(C.Structure):
    _fields_ = [("n_freq", C.c_int), ("beta", C.c_double), ("a", C.c_double),
                ("precision", C.c_int), ("ns_tol", C.c_double), ("ns_max_iter", C.c_int),
                ("tc_chunk_stages", C.c_int), ("ewald_gamma", C.c_double), ("real_cutoff", C.c_double),
                ("recip_cutoff", C.c_double), ("scs_mode", C.c_int), ("learned_max_error", C.c_double),
                ("mixed_max_error", C.c_double), ("learned_estimate_scale", C.c_double)]
MBD_SCS_PLAIN, MBD_SCS_LEARNED, MBD_SCS_NL = 0, 1, 2


class mbd_profile(C.Structure):
    _fields_ = [("launches", C.c_int), ("gemm_launches", C.c_int), ("gemm_ms", C.c_double),
                ("gemm_flops", C.c_double), ("screening_ms", C.c_double),
                ("screening_flops", C.c_double), ("newton_schulz_ms", C.c_double),
                ("gradient_ms", C.c_double), ("total_ms", C.c_double), ("tc_launches", C.c_int),
                ("tc_ms", C.c_double), ("tc_flops", C.c_double), ("correction_ms", C.c_double)]


class MBDError(RuntimeError):
    def __init__(self, code, origin, msg):
        super().__init__(f"{ERRORS.get(code, code)} in {origin}: {msg}")
        self.code, self.origin, self.msg = code, origin, msg


_lib = None
_P = C.POINTER(C.c_double)


def load(path: str | None = None):
    """Loads the CUDA library (built by `build.build()`); raises if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"libmbdgb.so not built ({path}); run paper_2308_03140_gb300.build.build()")
    L = C.CDLL(path)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    L.mbd_default_options.argtypes = [C.POINTER(mbd_options)]
    L.mbd_create.argtypes = [C.POINTER(vp), i, C.POINTER(mbd_options)]
    L.mbd_destroy.argtypes = [vp]
    L.mbd_set_geometry.argtypes = [vp, i, _P, _P, C.POINTER(C.c_int)]
    L.mbd_set_free_atom_params.argtypes = [vp, _P, _P, _P, _P]
    L.mbd_evaluate.argtypes = [vp, _P, _P, _P, _P, _P]
    L.mbd_evaluate_dev.argtypes = [vp, vp, i, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.mbd_backward_dev.argtypes = [vp, vp, C.c_longlong, i, vp, vp, vp, vp, vp, vp, vp, vp]
    L.mbd_get_evaluation_count.argtypes = [vp, C.POINTER(C.c_longlong)]
    L.mbd_get_scs_detail.argtypes = [vp, _P, _P, _P, _P]
    L.mbd_get_lattice_gradient.argtypes = [vp, _P]
    L.mbd_set_scs_model.argtypes = [vp, i, vp, vp, vp]
    L.mbd_get_learned_stats.argtypes = [vp, _P, C.POINTER(C.c_int)]
    L.mbd_screen.argtypes = [vp, _P, _P, _P, _P, _P]
    L.mbd_get_stats.argtypes = [vp, C.POINTER(C.c_int), _P, _P, _P]
    L.mbd_log_energy.argtypes = [vp, C.c_int, _P, _P]
    L.mbd_ts_energy.argtypes = [vp, C.c_double, _P, _P, _P, _P]
    L.mbd_get_exception.argtypes = [vp, C.POINTER(C.c_int), C.c_char_p, C.c_char_p, sz]
    L.mbd_set_profiling.argtypes = [vp, i]
    L.mbd_get_profile.argtypes = [vp, C.POINTER(mbd_profile)]
    ll = C.c_longlong
    L.mbdk_gemm_f64.argtypes = [vp, i, i, i, i, i, d, vp, ll, vp, ll, d, vp, ll, vp, ll]
    L.mbdk_cholesky_f64.argtypes = [vp, vp, ll, i, vp, vp]
    f = C.c_float
    L.mbdk_gemm_tc.argtypes = [vp, i, i, i, i, i, f, vp, vp, ll, vp, vp, ll, f, vp, vp, vp, vp, vp, ll, i, vp]
    L.mbdk_tc_wait_check.argtypes = [vp, ll, vp]
    L.mbdk_chol_solve3_f64.argtypes = [vp, vp, ll, i, vp, vp, vp]
    L.mbdk_cholesky_solve3_f64_noalloc.argtypes = [vp, vp, ll, i, vp, vp]
    L.mbdk_scs_features.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp, vp, vp]
    L.mbdk_mlp_forward.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp]
    L.mbdk_mlp_backward.argtypes = [vp, i, i, vp, vp, vp, vp, vp, vp, vp, vp]
    L.mbdk_mse_grad.argtypes = [vp, ll, vp, vp, vp, vp]
    L.mbdk_adam_step.argtypes = [vp, ll, vp, vp, vp, vp, i, f, vp]
    L.mbdk_gather_rows.argtypes = [vp, ll, i, vp, vp, vp]
    L.mbdk_learned_targets.argtypes = [vp, i, vp, vp, vp]
    L.mbdk_gemm_f64_split.argtypes = [vp, i, i, i, i, d, vp, ll, vp, ll, d, vp, ll, vp, ll, vp, vp]
    L.mbdk_gemm_f64_split_work_bytes.argtypes = [i, i, i]
    for name in EXPORTS:
        getattr(L, name).restype = C.c_int
    L.mbdk_gemm_f64_split_work_bytes.restype = C.c_size_t
    _lib = L
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


def _f64(x, shape=None):
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape is not None:
        a = a.reshape(shape)
    return a


def _tptr(t):
    """Device pointer of a torch tensor; the library reads every array densely in row-major
    order, so strided views are refused."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensor passed to the library must be contiguous")
    return C.c_void_p(t.data_ptr())


class MBD:
    """One library context on one CUDA device (mirrors mbd_calc_t of the paper's API)."""

    def __init__(self, device: int = 0, n_freq: int = 15, beta: float = 0.83, a: float = 6.0,
                 ns_tol: float = 1e-8, ns_max_iter: int = 100, precision: int = MBD_PREC_FP64,
                 tc_chunk_stages: int | None = None, ewald_gamma: float = 0.0, real_cutoff: float = 0.0,
                 recip_cutoff: float = 0.0, scs_mode: int = MBD_SCS_PLAIN, learned_max_error: float = 1e-6,
                 mixed_max_error: float = 1e-7, learned_estimate_scale: float = 1.0):
        self.lib = load()
        opt = mbd_options()
        self.lib.mbd_default_options(C.byref(opt))
        opt.n_freq, opt.beta, opt.a, opt.ns_tol, opt.ns_max_iter = n_freq, beta, a, ns_tol, ns_max_iter
        opt.precision = precision
        if tc_chunk_stages is not None:
            opt.tc_chunk_stages = tc_chunk_stages
        opt.ewald_gamma, opt.real_cutoff, opt.recip_cutoff = ewald_gamma, real_cutoff, recip_cutoff
        opt.scs_mode, opt.learned_max_error = scs_mode, learned_max_error
        opt.mixed_max_error = mixed_max_error
        opt.learned_estimate_scale = learned_estimate_scale
        h = C.c_void_p()
        rc = self.lib.mbd_create(C.byref(h), device, C.byref(opt))
        if rc:
            raise MBDError(rc, "mbd_create", "cannot create context")
        self.h, self.n_freq, self.device = h, n_freq, device
        self.n_atoms = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.mbd_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def exception(self):
        code = C.c_int()
        o, m = C.create_string_buffer(256), C.create_string_buffer(256)
        self.lib.mbd_get_exception(self.h, C.byref(code), o, m, 256)
        return code.value, o.value.decode(), m.value.decode()

    def _check(self, rc):
        if rc:
            code, origin, msg = self.exception()
            raise MBDError(rc, origin, msg)

    def set_geometry(self, coords, lattice=None, k_grid=None):
        R = _f64(coords, (-1, 3))
        lat = None if lattice is None else _f64(lattice, (3, 3))
        kg = None if k_grid is None else (C.c_int * 3)(*[int(k) for k in k_grid])
        self._check(self.lib.mbd_set_geometry(self.h, R.shape[0], _ptr(R), _ptr(lat), kg))
        self.n_atoms = R.shape[0]
        self.periodic = lattice is not None

    def set_free_atom_params(self, alpha0_ref, c6_ref, rvdw_ref, volume_ratio):
        arrs = [_f64(x) for x in (alpha0_ref, c6_ref, rvdw_ref, volume_ratio)]
        self._check(self.lib.mbd_set_free_atom_params(self.h, *[_ptr(x) for x in arrs]))

    def set_nl_params(self, alpha0_ref, c6_ref, alpha_ratio, omega_ratio):
        """MBD-NL inputs (contexts created with scs_mode=MBD_SCS_NL): the free-atom reference
        alpha0_ref, c6_ref and the density-functional ratios alpha0_df/alpha0_df,ref and
        omega_df/omega_df,ref, passed in the third and fourth parameter slots of
        mbd_set_free_atom_params."""
        self.set_free_atom_params(alpha0_ref, c6_ref, alpha_ratio, omega_ratio)

    def evaluate(self, gradients: bool = True, param_gradients: bool = True):
        """Host-memory evaluation.  Returns (energy, grad_coords [N,3] | None,
        grad_params [4,N] | None, alpha_scs [N]); for a periodic system the lattice
        gradient [3,3] is available afterwards from lattice_gradient()."""
        N = self.n_atoms
        E = C.c_double()
        gR = np.zeros((N, 3)) if gradients else None
        gp = np.zeros((4, N)) if gradients and param_gradients else None
        gA = np.zeros((3, 3)) if gradients and getattr(self, "periodic", False) else None
        al = np.zeros(N)
        self._check(self.lib.mbd_evaluate(self.h, C.byref(E), _ptr(gR), _ptr(gA), _ptr(gp), _ptr(al)))
        self._last_gA = gA
        return E.value, gR, gp, al

    def set_scs_model(self, params16, mean, std):
        """Learned screening model: params16 [members, LEARNED_PARAMS] (float16 values), feature
        mean and std [LEARNED_FEATURES]."""
        p = np.ascontiguousarray(np.asarray(params16, dtype=np.float16).reshape(-1, LEARNED_PARAMS))
        mean = np.ascontiguousarray(np.asarray(mean, dtype=np.float32))
        std = np.ascontiguousarray(np.asarray(std, dtype=np.float32))
        self._check(self.lib.mbd_set_scs_model(self.h, p.shape[0], p.ctypes.data_as(C.c_void_p),
                                               mean.ctypes.data_as(C.c_void_p), std.ctypes.data_as(C.c_void_p)))

    def learned_stats(self):
        est, fb = C.c_double(), C.c_int()
        self._check(self.lib.mbd_get_learned_stats(self.h, C.byref(est), C.byref(fb)))
        return dict(estimated_error_per_atom=est.value, fell_back=bool(fb.value))

    def screen(self):
        """Plain screening only: dict(alpha_bar, alpha_free [n_freq+1, N], c6, omega, rvdw)."""
        N = self.n_atoms
        ab, af = np.zeros((self.n_freq + 1, N)), np.zeros((self.n_freq + 1, N))
        c6, om, rv = np.zeros(N), np.zeros(N), np.zeros(N)
        self._check(self.lib.mbd_screen(self.h, _ptr(ab), _ptr(af), _ptr(c6), _ptr(om), _ptr(rv)))
        return dict(alpha_bar=ab, alpha_free=af, c6=c6, omega=om, rvdw=rv)

    def lattice_gradient(self):
        """dE/dA [3,3] (rows: lattice vectors) of the last gradient evaluation of a periodic
        system, with the Cartesian positions held fixed."""
        gA = np.zeros((3, 3))
        self._check(self.lib.mbd_get_lattice_gradient(self.h, _ptr(gA)))
        return gA

    def evaluate_dev(self, coords, alpha0_ref, c6_ref, rvdw_ref, volume_ratio, energy,
                     grad_coords=None, grad_params=None, alpha_scs=None, stream=None):
        """Device-memory evaluation on torch CUDA float64 tensors (outputs preallocated).
        `stream` is a torch.cuda.Stream or None for the current stream."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(coords.device)
        for t in (coords, alpha0_ref, c6_ref, rvdw_ref, volume_ratio, energy, grad_coords,
                  grad_params, alpha_scs):
            if t is not None and (not t.is_cuda or t.dtype != torch.float64 or not t.is_contiguous()):
                raise ValueError("device evaluation needs contiguous float64 CUDA tensors")
        rc = self.lib.mbd_evaluate_dev(self.h, C.c_void_p(stream.cuda_stream), int(coords.shape[0]),
                                       _tptr(coords), _tptr(alpha0_ref), _tptr(c6_ref), _tptr(rvdw_ref),
                                       _tptr(volume_ratio), _tptr(energy), _tptr(grad_coords),
                                       _tptr(grad_params), _tptr(alpha_scs))
        self._check(rc)

    def evaluation_count(self):
        """Number of successful evaluations of this context (the last one's number)."""
        c = C.c_longlong()
        self._check(self.lib.mbd_get_evaluation_count(self.h, C.byref(c)))
        return c.value

    def backward_dev(self, coords, alpha0_ref, c6_ref, rvdw_ref, volume_ratio, grad_energy=None,
                     grad_coords=None, grad_params=None, stream=None, evaluation=0):
        """Hand-written backward of the last evaluation (device tensors, outputs
        preallocated): grad_energy * dE/dX for coordinates and parameters.  `evaluation`:
        the number of the evaluation to differentiate (evaluation_count() after it; 0: the
        last, unchecked)."""
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(coords.device)
        rc = self.lib.mbd_backward_dev(self.h, C.c_void_p(stream.cuda_stream), int(evaluation),
                                       int(coords.shape[0]),
                                       _tptr(coords), _tptr(alpha0_ref), _tptr(c6_ref), _tptr(rvdw_ref),
                                       _tptr(volume_ratio), _tptr(grad_energy), _tptr(grad_coords),
                                       _tptr(grad_params))
        self._check(rc)

    def scs_detail(self):
        N, nf1 = self.n_atoms, self.n_freq + 1
        a, c6, om, rv = np.zeros((nf1, N)), np.zeros(N), np.zeros(N), np.zeros(N)
        self._check(self.lib.mbd_get_scs_detail(self.h, _ptr(a), _ptr(c6), _ptr(om), _ptr(rv)))
        return dict(alpha_bar=a, c6=c6, omega=om, rvdw=rv)

    def set_profiling(self, enable: bool = True):
        self._check(self.lib.mbd_set_profiling(self.h, int(bool(enable))))

    def profile(self):
        p = mbd_profile()
        self._check(self.lib.mbd_get_profile(self.h, C.byref(p)))
        return {k: getattr(p, k) for k, _ in mbd_profile._fields_}

    def log_energy(self, max_order: int = 2):
        """MBD energy by the log formula and its many-body orders for the oscillators of the
        last evaluation (mbd_log_energy): returns (energy, orders [max_order - 1] = E^(2..))."""
        E = C.c_double()
        orders = np.zeros(max(max_order - 1, 1))
        self._check(self.lib.mbd_log_energy(self.h, max_order, C.byref(E), _ptr(orders) if max_order > 1 else None))
        return E.value, orders[:max_order - 1]

    def ts_energy(self, s_r: float = 0.94, gradients: bool = True, lattice: bool = False):
        """TS pairwise energy (mbd_ts_energy) of the system set above, per cell for a periodic
        system: (energy, grad_coords [N,3] | None, grad_params [4,N] | None), and with
        lattice=True (cells only) also grad_lattice [3,3] as a fourth item."""
        N = self.n_atoms
        E = C.c_double()
        gR = np.zeros((N, 3)) if gradients else None
        gp = np.zeros((4, N)) if gradients else None
        gA = np.zeros((3, 3)) if lattice else None
        self._check(self.lib.mbd_ts_energy(self.h, s_r, C.byref(E), _ptr(gR), _ptr(gA), _ptr(gp)))
        return (E.value, gR, gp, gA) if lattice else (E.value, gR, gp)

    def stats(self):
        it, sc, res, cr = C.c_int(), C.c_double(), C.c_double(), C.c_double()
        self._check(self.lib.mbd_get_stats(self.h, C.byref(it), C.byref(sc), C.byref(res), C.byref(cr)))
        return dict(ns_iterations=it.value, ns_scale=sc.value, ns_residual=res.value,
                    correction_residual=cr.value)


def _stream(t, stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream(t.device)
    return C.c_void_p(s.cuda_stream)


def mbdk_gemm_f64(A, B, C_out, alpha=1.0, beta=0.0, D=None, mode=0, trans_b=True, stream=None):
    """C_out = alpha A op(B) + beta D on torch float64 CUDA tensors (dims multiples of 64);
    op(B) = B^T if trans_b else B."""
    L = load()
    M, K = A.shape
    N = B.shape[0] if trans_b else B.shape[1]
    rc = L.mbdk_gemm_f64(_stream(A, stream), int(bool(trans_b)), mode, M, N, K, alpha, _tptr(A), A.stride(0),
                         _tptr(B), B.stride(0), beta, _tptr(D), D.stride(0) if D is not None else 0,
                         _tptr(C_out), C_out.stride(0))
    if rc:
        raise MBDError(rc, "mbdk_gemm_f64", "launch rejected")


def mbdk_gemm_tc(kind, A0, B0, C_out=None, A1=None, B1=None, alpha=1.0, beta=0.0, D=None, C_hi=None,
                 C_lo=None, CT=None, mode=0, err=None, chunk_stages=0, stream=None):
    """Tensor-core GEMM C = alpha sum A_p B_p^T + beta D (see mbdk_gemm_tc in the header);
    torch CUDA tensors; returns the C return code."""
    L = load()
    M, K = A0.shape
    N = B0.shape[0]
    ref = C_out if C_out is not None else (CT if CT is not None else C_hi)
    return L.mbdk_gemm_tc(_stream(A0, stream), kind, mode, M, N, K, alpha, _tptr(A0), _tptr(A1), A0.stride(0),
                          _tptr(B0), _tptr(B1), B0.stride(0), beta, _tptr(D), _tptr(C_out), _tptr(C_hi),
                          _tptr(C_lo), _tptr(CT), ref.stride(0), chunk_stages, _tptr(err))


def mbdk_tc_wait_check(err, spin_cycles, stream=None):
    """The tensor-core GEMM's bounded wait on a barrier nothing arrives at (see the header):
    err is an int32 CUDA tensor; returns the C return code."""
    L = load()
    return L.mbdk_tc_wait_check(_stream(err, stream), int(spin_cycles), _tptr(err))


def mbdk_gemm_f64_split(A, B, C_out, alpha=1.0, beta=0.0, D=None, trans_b=True, work=None, err=None,
                        stream=None):
    """C_out = alpha A op(B) + beta D, FP64-accurate on the TF32 tensor cores by error-free
    splitting (see mbdk_gemm_f64_split in the header); torch float64 CUDA tensors, M and N
    multiples of 128, K of 64.  work (uint8 CUDA tensor of mbdk_gemm_f64_split_work_bytes)
    and err (int32 CUDA tensor) are allocated here when not given."""
    import torch
    L = load()
    M, K = A.shape
    N = B.shape[0] if trans_b else B.shape[1]
    if work is None:
        work = torch.empty(int(L.mbdk_gemm_f64_split_work_bytes(M, N, K)), dtype=torch.uint8, device=A.device)
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device=A.device)
    rc = L.mbdk_gemm_f64_split(_stream(A, stream), int(bool(trans_b)), M, N, K, alpha, _tptr(A), A.stride(0),
                               _tptr(B), B.stride(0), beta, _tptr(D), D.stride(0) if D is not None else 0,
                               _tptr(C_out), C_out.stride(0), _tptr(work), _tptr(err))
    if rc:
        raise MBDError(rc, "mbdk_gemm_f64_split", "launch rejected")
    return err


def mbdk_cholesky_f64(A, dinv, status, stream=None):
    """In-place batched Cholesky of A [batch, ld, ld] (float64 CUDA)."""
    L = load()
    rc = L.mbdk_cholesky_f64(_stream(A, stream), _tptr(A), A.shape[-1], A.shape[0], _tptr(dinv), _tptr(status))
    if rc:
        raise MBDError(rc, "mbdk_cholesky_f64", "launch rejected")


def mbdk_chol_solve3_f64(Lf, dinv, X, work=None, stream=None):
    """Solves in place with the factors of mbdk_cholesky_f64; work: same shape as X
    (allocated here with torch when not given)."""
    import torch
    L = load()
    if work is None:
        work = torch.empty_like(X)
    rc = L.mbdk_chol_solve3_f64(_stream(Lf, stream), _tptr(Lf), Lf.shape[-1], Lf.shape[0], _tptr(dinv), _tptr(X),
                                _tptr(work))
    if rc:
        raise MBDError(rc, "mbdk_chol_solve3_f64", "launch rejected")


def mbdk_cholesky_solve3_f64_noalloc(A, X, status, stream=None):
    """Factor A [batch, ld, ld] in place and solve A X = B in place (X [batch, ld, 3]),
    with the factorisation's scratch in the library's static device array; returns the
    C return code (0, or MBD_ERR_SCRATCH_LIMIT = 9 for requests beyond 2^21 doubles)."""
    L = load()
    return L.mbdk_cholesky_solve3_f64_noalloc(_stream(A, stream), _tptr(A), A.shape[-1], A.shape[0],
                                              _tptr(X), _tptr(status))


def _chk(rc, name):
    if rc:
        raise MBDError(rc, name, "launch rejected")


def mbdk_scs_features(offsets, coords, alpha0_ref, c6_ref, rvdw_ref, volume_ratio, X, work=None, stream=None):
    """Learned-model features X [n_atoms, LEARNED_FEATURES] (float32 CUDA) of systems stored
    back to back (offsets int32 [n_systems + 1]); inputs float64 CUDA tensors; work
    [n_atoms, LEARNED_WORK] float64 scratch (allocated here with torch when not given)."""
    import torch
    L = load()
    if work is None:
        work = torch.empty(X.shape[0], LEARNED_WORK, dtype=torch.float64, device=X.device)
    _chk(L.mbdk_scs_features(_stream(X, stream), X.shape[0], offsets.shape[0] - 1, _tptr(offsets), _tptr(coords),
                             _tptr(alpha0_ref), _tptr(c6_ref), _tptr(rvdw_ref), _tptr(volume_ratio), _tptr(X),
                             _tptr(work)), "mbdk_scs_features")


def mbdk_mlp_forward(X, mean, std, params16, Y, zcache=None, stream=None):
    """Y [members, B, 16] = MLP(X [B, LEARNED_FEATURES]) for params16 [members, LEARNED_PARAMS] (float16)."""
    L = load()
    _chk(L.mbdk_mlp_forward(_stream(X, stream), X.shape[0], params16.shape[0], _tptr(X), _tptr(mean), _tptr(std),
                            _tptr(params16), _tptr(Y), _tptr(zcache)), "mbdk_mlp_forward")


def mbdk_mlp_backward(X, mean, std, params16, zcache, dY, dX=None, grad=None, stream=None):
    """Backward of sum(dY * Y): dX [members, B, LEARNED_FEATURES] and/or grad [members, LEARNED_PARAMS]
    (float32, accumulated)."""
    L = load()
    _chk(L.mbdk_mlp_backward(_stream(X, stream), X.shape[0], params16.shape[0], _tptr(X), _tptr(mean), _tptr(std),
                             _tptr(params16), _tptr(zcache), _tptr(dY), _tptr(dX), _tptr(grad)), "mbdk_mlp_backward")


def mbdk_mse_grad(y, t, dy, loss=None, stream=None):
    L = load()
    _chk(L.mbdk_mse_grad(_stream(y, stream), y.numel(), _tptr(y), _tptr(t), _tptr(dy), _tptr(loss)), "mbdk_mse_grad")


def mbdk_adam_step(params, grad, m, v, step, lr, params16=None, stream=None):
    L = load()
    _chk(L.mbdk_adam_step(_stream(params, stream), params.numel(), _tptr(params), _tptr(grad), _tptr(m), _tptr(v),
                          int(step), float(lr), _tptr(params16)), "mbdk_adam_step")


def mbdk_learned_targets(alpha_bar, alpha_free, Y, stream=None):
    """Y [n_atoms, 16] (float32 CUDA) = log(alpha_bar / alpha_free) of [16, n_atoms] float64 CUDA tensors."""
    L = load()
    _chk(L.mbdk_learned_targets(_stream(Y, stream), Y.shape[0], _tptr(alpha_bar), _tptr(alpha_free), _tptr(Y)),
         "mbdk_learned_targets")


def mbdk_gather_rows(idx, src, dst, stream=None):
    L = load()
    _chk(L.mbdk_gather_rows(_stream(src, stream), idx.shape[0], src.shape[1], _tptr(idx), _tptr(src), _tptr(dst)),
         "mbdk_gather_rows")


def evaluate_system(sys, device: int = 0, gradients: bool = True, **opts):
    """One-shot host evaluation of a synthetic.System."""
    with MBD(device, **opts) as m:
        m.set_geometry(sys.coords, sys.lattice, sys.k_grid)
        m.set_free_atom_params(sys.alpha0_ref, sys.c6_ref, sys.rvdw_ref, sys.ratio)
        E, gR, gp, al = m.evaluate(gradients)
        return E, gR, gp, al, m.stats()
