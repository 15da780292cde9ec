"""Pins of the oracle's per-atom formulas with hand-computed values, CPU only.

- TS volume scaling, Eq. (ts-scaling): alpha0 = alpha0_ref v, omega = 4 C6_ref/(3 alpha0_ref^2),
  R_vdW = R_ref v^(1/3).  Inputs are chosen so that every value is exact in a few digits
  (v = 0.9^3, 0.8^3, 0.7^3; C6_ref/alpha0_ref^2 = 3/4 or 3/8).
- Screened parameters, Eqs. (casimir-polder), (osc-param), (scale-rvdw-scs): for a screened
  polarizability of one-oscillator shape A/(1 + u^2/w^2) the Casimir-Polder integral is
  3/4 w A^2 in closed form, so C6bar, omega_bar = 4 C6bar/(3 alpha_bar0^2) and
  R_bar = R_vdW (alpha_bar0/alpha0)^(1/3) have known values; alpha_bar0/alpha0 = 0.8^3 makes the
  cube root exact.
- Two atoms: the screened polarizabilities of the pair follow from the per-axis 2x2 inverse
  (Eqs. scs, contraction); the oracle's whole pipeline (TS scaling, screening, screened
  parameters, Q and its energy) must reproduce the screened parameters and the two-oscillator
  energy built from them.
Each pin is also run against copies of the oracle with one plausible slip planted in its
source (the scaled alpha0 in place of alpha0_ref, a wrong root, a wrong prefactor): every slip
must fail it.
"""
import ctypes as C
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle as o

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_DIR = os.path.join(os.path.dirname(HERE), "oracle")
BETA, A_DAMP = 0.83, 6.0
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")

# (alpha0_ref, C6_ref, R_ref, v) -> (alpha0, omega, R_vdW), worked by hand
TS_CASES = [
    ((8.0, 48.0, 3.5, 0.729), (5.832, 1.0, 3.15)),
    ((6.0, 27.0, 3.0, 0.512), (3.072, 1.0, 2.4)),
    ((10.0, 150.0, 4.0, 1.0), (10.0, 2.0, 4.0)),
    ((4.0, 6.0, 3.2, 0.343), (1.372, 0.5, 2.24)),
]


class _Lib:
    """The two per-atom entry points of an oracle build (the real one or a mutant)."""

    def __init__(self, cdll):
        i = C.c_int
        self.L = cdll
        cdll.orc_ts_scaling.argtypes = [i, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        cdll.orc_screened_params.argtypes = [i, i, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
        cdll.orc_freq_grid.argtypes = [i, _dp, _dp]

    def ts_scaling(self, a0ref, c6ref, rref, ratio):
        N = len(a0ref)
        out = [np.zeros(N) for _ in range(3)]
        self.L.orc_ts_scaling(N, *(np.ascontiguousarray(x, dtype=float) for x in (a0ref, c6ref, rref, ratio)), *out)
        return out

    def screened_params(self, alpha_bar, alpha0, rvdw, n_freq=15):
        N = alpha_bar.shape[1]
        u, wu = np.zeros(n_freq + 1), np.zeros(n_freq + 1)
        self.L.orc_freq_grid(n_freq, u, wu)
        outs = [np.zeros(N) for _ in range(4)]
        rc = self.L.orc_screened_params(N, n_freq, np.ascontiguousarray(alpha_bar), wu,
                                        np.ascontiguousarray(alpha0, dtype=float),
                                        np.ascontiguousarray(rvdw, dtype=float), *outs)
        return rc, outs


def ts_pin_failures(lib):
    """Names of the hand-computed TS values the build misses (empty: pinned)."""
    inp = np.array([c[0] for c in TS_CASES]).T
    ref = np.array([c[1] for c in TS_CASES]).T
    got = lib.ts_scaling(*inp)
    names = ("alpha0", "omega", "R_vdW")
    return [names[k] for k in range(3) if not np.allclose(got[k], ref[k], rtol=1.6e-15, atol=0)]


def screened_pin_failures(lib):
    """Screened parameters of one-oscillator-shaped alpha_bar(u) rows against their closed forms.
    Atom i: alpha_bar(0) = B_i, alpha_bar(u_k > 0) = A_i/(1 + u_k^2/w_i^2), free alpha0_i, R_vdW,i.
    Then C6bar = 3/4 w A^2 (to the quadrature error of the 15-point grid, 1e-9 relative at
    w = 0.6), omega_bar = 4 C6bar/(3 B^2) = w A^2/B^2, R_bar = R_vdW (B/alpha0)^(1/3)."""
    u, _ = o.freq_grid(15)
    # (A, w, B, alpha0, R_vdW): B/alpha0 = 0.512 = 0.8^3, 0.729 = 0.9^3, 1.0; A != B in two atoms
    atoms = [(5.12, 0.6, 5.12, 10.0, 3.5), (6.0, 0.6, 7.29, 10.0, 4.0), (9.0, 0.6, 4.5, 4.5, 3.0)]
    A, w, B, a0, rv = (np.array(x) for x in zip(*atoms))
    ab = A[None, :] / (1.0 + u[:, None] ** 2 / w[None, :] ** 2)
    ab[0] = B
    rc, (abar0, c6, ombar, rbar) = lib.screened_params(ab, a0, rv)
    bad = []
    if rc != o.OK:
        bad.append("status")
    if not np.allclose(abar0, B, rtol=0, atol=0):
        bad.append("alpha_bar0")
    if not np.allclose(c6, 0.75 * w * A ** 2, rtol=2e-9):
        bad.append("C6bar")
    # worked by hand: w A^2/B^2 = 0.6, 0.6 (36/53.1441), 0.6 * 4
    if not np.allclose(ombar, [0.6, 0.6 * 36.0 / 53.1441, 2.4], rtol=2e-9):
        bad.append("omega_bar")
    if not np.allclose(rbar, [2.8, 3.6, 3.0], rtol=1e-15):
        bad.append("R_bar")
    return bad


def test_ts_scaling_hand_values():
    assert ts_pin_failures(_Lib(o.lib())) == []


def test_screened_params_hand_values():
    assert screened_pin_failures(_Lib(o.lib())) == []


def test_screened_params_flags_non_positive_alpha():
    lib = _Lib(o.lib())
    u, _ = o.freq_grid(15)
    ab = np.ones((16, 2)) / (1.0 + u[:, None] ** 2)
    ab[0, 1] = -0.5
    rc, _ = lib.screened_params(ab, np.array([1.0, 1.0]), np.array([3.0, 3.0]))
    assert rc == o.ERR_SCS_NEG_ALPHA


def two_atom_closed_form(R, a0ref, c6ref, rref, ratio):
    """Screened parameters and MBD energy of two atoms a distance R apart along z, written out:
    TS scaling by hand, the screened alpha_bar_i(u) of each axis from the 2x2 inverse of
    [[1/a1, t], [t, 1/a2]] with t the diagonal of (1 - f) T^GG, then Eqs. (casimir-polder),
    (scale-rvdw-scs), and the two-oscillator modes of Q with the damping g(R_bar)."""
    a0 = a0ref * ratio
    om = 4.0 * c6ref / (3.0 * a0ref ** 2)
    rv = rref * np.cbrt(ratio)
    u, wu = o.freq_grid(15)
    f = o.fermi(R, rv.sum(), BETA, A_DAMP)
    ab = np.zeros((16, 2))
    for k in range(16):
        al = a0 / (1 + u[k] ** 2 / om ** 2)
        s = math.hypot(*[(math.sqrt(2 / math.pi) * x / 3) ** (1 / 3) for x in al])
        t = np.diag((1 - f) * o.T_gg([0, 0, R], s))
        det = 1 / (al[0] * al[1]) - t ** 2
        ab[k, 0] = np.mean((1 / al[1] - t) / det)
        ab[k, 1] = np.mean((1 / al[0] - t) / det)
    abar0 = ab[0]
    c6 = 3 / math.pi * (wu[1:, None] * ab[1:] ** 2).sum(0)
    ombar = 4 * c6 / (3 * abar0 ** 2)
    rbar = rv * np.cbrt(abar0 / a0)
    g = o.fermi(R, rbar.sum(), BETA, A_DAMP)
    E = -1.5 * ombar.sum()
    for tz in (g / R ** 3, g / R ** 3, -2 * g / R ** 3):
        m = 0.5 * (ombar[0] ** 2 + ombar[1] ** 2)
        d = math.sqrt((0.5 * (ombar[0] ** 2 - ombar[1] ** 2)) ** 2
                      + ombar[0] ** 2 * ombar[1] ** 2 * abar0[0] * abar0[1] * tz * tz)
        E += 0.5 * (math.sqrt(m + d) + math.sqrt(m - d))
    return dict(alpha_bar=ab, c6=c6, omega=ombar, rvdw=rbar, energy=E, alpha0=a0)


@pytest.mark.parametrize("R", [3.4, 3.8])
def test_two_atom_pipeline_closed_form(R):
    a0ref, c6ref = np.array([8.0, 10.0]), np.array([48.0, 150.0])
    rref, ratio = np.array([3.5, 4.0]), np.array([0.729, 0.9])
    pos = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, R]])
    ref = two_atom_closed_form(R, a0ref, c6ref, rref, ratio)
    # the pair screens strongly enough that alpha_bar0 differs from alpha0 by more than 1 %
    assert np.all(np.abs(ref["alpha_bar"][0] / ref["alpha0"] - 1) > 0.01)
    E, det = o.mbd_rsscs_energy(pos, a0ref, c6ref, rref, ratio, BETA, A_DAMP, 15, detail=True)
    assert np.allclose(det["alpha_bar"], ref["alpha_bar"], rtol=1e-13)
    assert np.allclose(det["c6"], ref["c6"], rtol=1e-13)
    assert np.allclose(det["omega"], ref["omega"], rtol=1e-13)
    assert np.allclose(det["rvdw"], ref["rvdw"], rtol=1e-13)
    # osc-param: the screened oscillator reproduces its own C6 (C6 = 3/4 omega alpha0^2)
    assert np.allclose(det["c6"], 0.75 * det["omega"] * det["alpha_bar"][0] ** 2, rtol=1e-14)
    assert abs(E - ref["energy"]) < 50 * 2.2e-16 * 1.5 * ref["omega"].sum()


# ---- planted slips: each copy of the oracle with one mistake fails a pin --------------------
MUTANTS = {
    "omega from the scaled alpha0": ("om[i] = 4.0 * c6ref[i] / (3.0 * a0ref[i] * a0ref[i]);",
                                     "om[i] = 4.0 * c6ref[i] / (3.0 * a0[i] * a0[i]);", "ts"),
    "R_vdW root 1/7": ("rv[i] = rref[i] * cbrt(ratio[i]);", "rv[i] = rref[i] * pow(ratio[i], 1.0 / 7.0);", "ts"),
    "alpha0 times v^2": ("a0[i] = a0ref[i] * ratio[i];", "a0[i] = a0ref[i] * ratio[i] * ratio[i];", "ts"),
    "omega_bar from the free alpha0": ("ombar[i] = 4.0 * c6bar[i] / (3.0 * abar0[i] * abar0[i]);",
                                       "ombar[i] = 4.0 * c6bar[i] / (3.0 * a0[i] * a0[i]);", "scs"),
    "R_bar root 1/7": ("rbar[i] = rv[i] * cbrt(abar0[i] / a0[i]);",
                       "rbar[i] = rv[i] * pow(abar0[i] / a0[i], 1.0 / 7.0);", "scs"),
    "C6bar prefactor 3/(2 pi)": ("c6bar[i] = 3.0 / ORC_PI * ksum_get(&s);",
                                 "c6bar[i] = 1.5 / ORC_PI * ksum_get(&s);", "scs"),
    "C6bar from alpha_bar, not its square": ("ksum_add(&s, wu[k] * ab * ab);", "ksum_add(&s, wu[k] * ab);", "scs"),
}


@pytest.fixture(scope="module")
def mutant_libs(tmp_path_factory):
    src = open(os.path.join(ORACLE_DIR, "mbd_oracle.c")).read()
    out = {}
    for name, (old, new, _) in MUTANTS.items():
        assert src.count(old) == 1, f"planted slip '{name}': its source line is not unique"
        d = tmp_path_factory.mktemp("mutant")
        open(d / "mbd_oracle.c", "w").write(src.replace(old, new))
        shutil.copy(os.path.join(ORACLE_DIR, "mbd_oracle_internal.h"), d / "mbd_oracle_internal.h")
        so = d / "libmutant.so"
        subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-fopenmp", "-o", str(so), str(d / "mbd_oracle.c"),
                               "-lm"])
        out[name] = _Lib(C.CDLL(str(so)))
    return out


@pytest.mark.parametrize("name", list(MUTANTS))
def test_planted_slip_fails_a_pin(mutant_libs, name):
    lib = mutant_libs[name]
    which = MUTANTS[name][2]
    failures = ts_pin_failures(lib) if which == "ts" else screened_pin_failures(lib)
    assert failures, f"the slip '{name}' passes the {which} pin"
