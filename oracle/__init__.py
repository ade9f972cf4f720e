"""FP64 CPU oracle for the SFHK high-harmonic path (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only ``tests/``, the package smoke
check and the CPU-baseline leg of ``bench.py`` may import it; the product
library never does.  It wraps ``sfhk_oracle.c`` (plain C, double precision,
written step by step from the paper's equations) with ctypes and numpy.

Functions that are pinned only by the paper's own figures (the spectra
themselves) are "parity unpinned": the figures are placeholders in the
source, the fitted GTO coefficients are not printed and there is no TDSE
data.  Every other function is pinned by the tests in ``tests/test_oracle_*``.
"""
from __future__ import annotations

import contextlib
import ctypes as C
import os
import shutil
import subprocess
import tempfile
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfhk_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

NFIELDS = 12      # n0 | q0[3] | p0[3] | nhat[3] | w_re w_im
NFINAL = 47       # q[3] p[3] M[36] S C_re C_im theta status
NY = 43

POT_MOLECULE = 0
POT_HARMONIC = 1
POT_POLY = 2
ALIGN_FIXED, ALIGN_ISO, ALIGN_COS2, ALIGN_QUAD = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (no fast-math, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-std=gnu11", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


class PulseIn(C.Structure):
    _fields_ = [("lambda_nm", C.c_double), ("intensity", C.c_double),
                ("n_cycles", C.c_double), ("cep", C.c_double), ("dt", C.c_double),
                ("t_center", C.c_double)]


class TargetIn(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_prim", C.c_int), ("R", C.c_double),
                ("Zinf", C.c_double), ("Z0", C.c_double), ("alpha", C.c_double),
                ("soft_a", C.c_double), ("Ip", C.c_double), ("ho_omega", C.c_double),
                ("pexp", C.c_double * 8), ("pcoef", C.c_double * 8), ("ionization", C.c_int),
                ("sampling", C.c_int), ("sampling_factor", C.c_double),
                ("pkind", C.c_int * 8), ("pi_azimuth", C.c_double),
                ("n_centres", C.c_int), ("cpos", (C.c_double * 3) * 8),
                ("cZinf", C.c_double * 8), ("cZ0", C.c_double * 8), ("calpha", C.c_double * 8),
                ("pcentre", C.c_int * 8), ("pdir", (C.c_double * 3) * 8),
                ("proposal_mix", C.c_double), ("proposal_floor", C.c_double),
                ("origin", C.c_double * 3)]


_dp = C.POINTER(C.c_double)


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def lib():
    global _lib
    if _lib is None:
        build()
        _lib = _configure(C.CDLL(_LIB))
    return _lib


def _configure(L):
    """Declare the argument and result types of the oracle's exports."""
    u32p = C.POINTER(C.c_uint32)
    L.or_philox4x32_10.argtypes = [u32p, u32p, u32p]
    L.or_uniforms.argtypes = [C.c_uint64, C.c_uint32, C.c_uint64, _dp]
    L.or_pulse_derive.argtypes = [C.POINTER(PulseIn), _dp, C.POINTER(C.c_int)]
    L.or_pulse_A_real.argtypes = [C.POINTER(PulseIn), C.c_double]
    L.or_pulse_A_real.restype = C.c_double
    L.or_pulse_E_real.argtypes = [C.POINTER(PulseIn), C.c_double]
    L.or_pulse_E_real.restype = C.c_double
    L.or_pulse_E_complex.argtypes = [C.POINTER(PulseIn), C.c_double, C.c_double, _dp]
    L.or_pulse_A_complex.argtypes = [C.POINTER(PulseIn), C.c_double, C.c_double, _dp]
    L.or_potential.argtypes = [C.POINTER(TargetIn), _dp, _dp, _dp]
    L.or_trajectory.argtypes = [C.POINTER(TargetIn), C.POINTER(PulseIn), _dp, _dp,
                                C.c_double, C.c_double, C.c_int, _dp]
    L.or_hk_det.argtypes = [_dp, C.c_double, _dp]
    L.or_pi_direction.argtypes = [_dp, C.c_double, _dp]
    L.or_orbital_norm.argtypes = [C.POINTER(TargetIn)]
    L.or_orbital_norm.restype = C.c_double
    L.or_orbital_value.argtypes = [C.POINTER(TargetIn), _dp, _dp]
    L.or_orbital_value.restype = C.c_double
    L.or_recomb.argtypes = [C.POINTER(TargetIn), _dp, _dp, _dp, C.c_double, _dp]
    L.or_dipole_matrix_element.argtypes = [C.POINTER(TargetIn), _dp, _dp, _dp, _dp]
    L.or_saddle.argtypes = [C.POINTER(PulseIn), C.c_double, C.c_double, C.c_double, _dp]
    L.or_saddle.restype = C.c_int
    L.or_tunnel.argtypes = [C.POINTER(PulseIn), C.c_double, C.c_double, C.c_double,
                            _dp, _dp]
    L.or_adk_table.argtypes = [C.POINTER(PulseIn), C.c_double, _dp, _dp]
    L.or_sample.argtypes = [C.POINTER(TargetIn), C.POINTER(PulseIn), C.c_int, C.c_double,
                            C.c_double, C.c_double, C.c_int, C.c_int, C.c_uint64, C.c_uint32,
                            C.c_uint64, C.c_uint64, _dp, _dp]
    L.or_quad_nodes.argtypes = [C.c_int, _dp, _dp]
    L.or_propagate_returns.argtypes = [C.POINTER(TargetIn), C.POINTER(PulseIn), C.c_double,
                                       C.c_double, C.c_double, _dp, C.c_uint64, C.c_double,
                                       _dp, C.c_double, C.c_double, _dp, C.c_int]
    L.or_propagate_returns.restype = C.c_int
    L.or_abs_sampling_constants.argtypes = [C.POINTER(TargetIn), C.POINTER(PulseIn), C.c_int,
                                            C.c_double, C.c_double, C.c_double, C.c_int,
                                            C.c_uint64, C.c_uint32, _dp]
    L.or_euler_rotation.argtypes = [C.c_double, C.c_double, C.c_double, _dp]
    L.or_orbital_values.argtypes = [C.POINTER(TargetIn), _dp, _dp, C.c_int64, _dp]
    L.or_saddle_modified.argtypes = [C.POINTER(PulseIn), C.c_double, C.c_double, C.c_double,
                                     C.c_double, _dp]
    L.or_saddle_modified.restype = C.c_int
    L.or_pulse_Edot_complex.argtypes = [C.POINTER(PulseIn), C.c_double, C.c_double, _dp]
    L.or_sample.restype = C.c_int
    L.or_propagate.argtypes = [C.POINTER(TargetIn), C.POINTER(PulseIn), C.c_double,
                               C.c_double, C.c_double, C.c_double, _dp, C.c_uint64,
                               C.c_double, _dp, _dp, C.c_int]
    L.or_stab_taper_weight.argtypes = [C.c_double, C.c_double, C.c_double]
    L.or_stab_taper_weight.restype = C.c_double
    L.or_propagate.restype = C.c_int
    L.or_spectrum.argtypes = [_dp, C.c_int, C.c_double, C.c_double, C.c_double, C.c_int,
                              _dp, _dp, _dp, _dp, _dp]
    L.or_ionization_step.argtypes = [C.POINTER(TargetIn), C.POINTER(PulseIn), _dp,
                                     C.c_double, C.c_double, C.c_double, C.c_int, _dp]
    L.or_ionization_step.restype = C.c_int
    return L


@contextlib.contextmanager
def mutated(edits):
    """Build a copy of the oracle with a planted mistake and make every
    function of this module use it inside the ``with`` block.

    edits: (old, new) source replacements; each ``old`` must occur exactly
    once in sfhk_oracle.c.  Tests use this to show that a pin fails when the
    term it guards is changed.  The copy is compiled like the oracle itself,
    in a temporary directory that is removed afterwards."""
    global _lib
    src = open(_SRC).read()
    for old, new in edits:
        if src.count(old) != 1:
            raise ValueError(f"mutation site not found exactly once: {old!r}")
        src = src.replace(old, new)
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    try:
        c_path, so_path = os.path.join(d, "mut.c"), os.path.join(d, "libmut.so")
        with open(c_path, "w") as f:
            f.write(src)
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                        "-std=gnu11", "-o", so_path, c_path, "-lm"], check=True)
        with _lock:
            saved = lib()
            _lib = _configure(C.CDLL(so_path))
        try:
            yield
        finally:
            with _lock:
                _lib = saved
    finally:
        shutil.rmtree(d, ignore_errors=True)


# ---------------------------------------------------------------- inputs
def pulse_in(p) -> PulseIn:
    """p: mapping with lambda_nm, intensity, n_cycles, cep, dt (+ t_center, the
    time of the pulse centre, 0 by default)."""
    return PulseIn(p["lambda_nm"], p["intensity"], p["n_cycles"], p.get("cep", 0.0), p["dt"],
                   p.get("t_center", 0.0))


def target_in(t) -> TargetIn:
    """t: mapping with R, Zinf, Z0, alpha, soft_a, Ip, pexp, pcoef (+ kind, ho_omega,
    ionization, sampling, sampling_factor, pkind, pi_azimuth)."""
    T = TargetIn()
    T.kind = int(t.get("kind", POT_MOLECULE))
    T.ionization = int(t.get("ionization", 0))
    T.sampling = int(t.get("sampling", 0))
    T.sampling_factor = float(t.get("sampling_factor", 0.0))
    T.n_prim = len(t.get("pexp", ()))
    for name in ("R", "Zinf", "Z0", "alpha", "soft_a", "Ip", "ho_omega"):
        setattr(T, name, float(t.get(name, 0.0)))
    kinds = list(t.get("pkind", [0] * len(t.get("pexp", ()))))
    for i, (e, c) in enumerate(zip(t.get("pexp", ()), t.get("pcoef", ()))):
        T.pexp[i] = e
        T.pcoef[i] = c
        T.pkind[i] = int(kinds[i]) if i < len(kinds) else 0
    T.pi_azimuth = float(t.get("pi_azimuth", 0.0))
    cen = t.get("centres", ())
    T.n_centres = len(cen)
    for i, c in enumerate(cen):          # (x, y, z, Zinf, Z0, alpha)
        for a in range(3):
            T.cpos[i][a] = c[a]
        T.cZinf[i], T.cZ0[i], T.calpha[i] = c[3], c[4], c[5]
    for i, c in enumerate(t.get("pcentre", ())):
        T.pcentre[i] = int(c)
    for i, d in enumerate(t.get("pdir", ())):
        for a in range(3):
            T.pdir[i][a] = d[a]
    T.proposal_mix = float(t.get("proposal_mix", 0.0))
    T.proposal_floor = float(t.get("proposal_floor", 0.0))
    for a, x in enumerate(t.get("origin", (0.0, 0.0, 0.0))):
        T.origin[a] = float(x)
    return T


# ---------------------------------------------------------------- wrappers
def philox(ctr, key):
    a = (C.c_uint32 * 4)(*ctr)
    k = (C.c_uint32 * 2)(*key)
    o = (C.c_uint32 * 4)()
    lib().or_philox4x32_10(a, k, o)
    return list(o)


def uniforms(seed, instance, j):
    u = np.zeros(6)
    lib().or_uniforms(seed, instance, j, _p(u))
    return u


def pulse_derived(p):
    out = np.zeros(6)
    nt = C.c_int()
    lib().or_pulse_derive(C.byref(pulse_in(p)), _p(out), C.byref(nt))
    return dict(omega=out[0], E0=out[1], Tp=out[2], cep=out[3], dt=out[4],
                t_origin=out[5], nt=nt.value)


def pulse_A(p, t):
    P = pulse_in(p)
    return np.array([lib().or_pulse_A_real(C.byref(P), float(x)) for x in np.atleast_1d(t)])


def pulse_E(p, t):
    P = pulse_in(p)
    return np.array([lib().or_pulse_E_real(C.byref(P), float(x)) for x in np.atleast_1d(t)])


def pulse_A_complex(p, tau):
    out = np.zeros(2)
    lib().or_pulse_A_complex(C.byref(pulse_in(p)), tau.real, tau.imag, _p(out))
    return complex(out[0], out[1])


def pulse_E_complex(p, tau):
    out = np.zeros(2)
    lib().or_pulse_E_complex(C.byref(pulse_in(p)), tau.real, tau.imag, _p(out))
    return complex(out[0], out[1])


def potential(t, nhat, q):
    """Returns V, grad[3], hess[3,3]."""
    out = np.zeros(13)
    lib().or_potential(C.byref(target_in(t)), _p(np.asarray(nhat, float).copy()),
                       _p(np.asarray(q, float).copy()), _p(out))
    return out[0], out[1:4].copy(), out[4:13].reshape(3, 3).copy()


def trajectory(t, p, nhat, y0, t_start, h, n_steps):
    out = np.zeros((n_steps + 1, NY))
    lib().or_trajectory(C.byref(target_in(t)), C.byref(pulse_in(p)),
                        _p(np.asarray(nhat, float).copy()), _p(np.asarray(y0, float).copy()),
                        t_start, h, n_steps, _p(out))
    return out


def initial_state(q0, p0):
    y = np.zeros(NY)
    y[0:3] = q0
    y[3:6] = p0
    y[6:42] = np.eye(6).ravel()
    return y


def hk_det(M, gamma):
    out = np.zeros(2)
    lib().or_hk_det(_p(np.ascontiguousarray(M, dtype=float).ravel().copy()), gamma, _p(out))
    return complex(out[0], out[1])


def orbital_norm(t):
    return lib().or_orbital_norm(C.byref(target_in(t)))


def orbital_value(t, nhat, r):
    return lib().or_orbital_value(C.byref(target_in(t)), _p(np.asarray(nhat, float).copy()),
                                  _p(np.asarray(r, float).copy()))


def recomb(t, nhat, q, p, gamma):
    out = np.zeros(2)
    lib().or_recomb(C.byref(target_in(t)), _p(np.asarray(nhat, float).copy()),
                    _p(np.asarray(q, float).copy()), _p(np.asarray(p, float).copy()),
                    gamma, _p(out))
    return complex(out[0], out[1])


def dipole_matrix_element(t, nhat, kappa):
    kappa = np.asarray(kappa, complex)
    out = np.zeros(2)
    lib().or_dipole_matrix_element(C.byref(target_in(t)), _p(np.asarray(nhat, float).copy()),
                                   _p(kappa.real.copy()), _p(kappa.imag.copy()), _p(out))
    return complex(out[0], out[1])


def saddle(p, Ip, t0, kperp2):
    out = np.zeros(2)
    rc = lib().or_saddle(C.byref(pulse_in(p)), Ip, t0, kperp2, _p(out))
    return rc, out[0], out[1]


def tunnel(p, Ip, t0, tt, k):
    out = np.zeros(3)
    lib().or_tunnel(C.byref(pulse_in(p)), Ip, t0, tt, _p(np.asarray(k, float).copy()), _p(out))
    return out[0], complex(out[1], out[2])


def adk_table(p, Ip):
    nt = pulse_derived(p)["nt"]
    W = np.zeros(nt)
    cdf = np.zeros(nt)
    lib().or_adk_table(C.byref(pulse_in(p)), Ip, _p(W), _p(cdf))
    return W, cdf


def sample(t, p, align=(ALIGN_FIXED, 0.0, 0.0), seed=0, instance=0, j_begin=0, n=1,
           eta_force=0):
    """Initial ensemble as a (12, n) field-major array plus aux (tt, S_down).
    align = (kind, theta, phi[, n_nodes[, psi]]); n_nodes is the K of the
    quadrature kind, psi the third Euler angle of a fixed polyatomic
    orientation.  For a polyatomic target fields 7..9 hold the Euler angles
    (phi, theta, psi) instead of the axis.  eta_force = +-1 fixes the emitting side of the modified saddle
    (target ionization 1) with weight 1 instead of drawing it."""
    soa = np.zeros((NFIELDS, n))
    aux = np.zeros((3, n))
    k = int(align[3]) if len(align) > 3 else 0
    psi = float(align[4]) if len(align) > 4 else 0.0
    bad = lib().or_sample(C.byref(target_in(t)), C.byref(pulse_in(p)), int(align[0]),
                          float(align[1]), float(align[2]), psi, k, int(eta_force), seed,
                          instance, j_begin, n, _p(soa), _p(aux))
    if bad < 0:
        raise ValueError("bad alignment")
    return soa, aux, bad


def quad_nodes(K):
    """The oracle's K-node rule on x = cos(theta) in [0, 1] (descending x,
    weights summing to 1)."""
    x, w = np.zeros(K), np.zeros(K)
    lib().or_quad_nodes(K, _p(x), _p(w))
    return x, w


def propagate(t, p, soa, gamma, cutoff=0.0, n_norm=0.0, want_final=False, n_threads=0,
              stab_cutoff=0.0, stab_taper=0.0):
    """stab_taper = r > 1: the stability filter tapers the contributions
    smoothly between stab_cutoff and r stab_cutoff (hard cut when 0)."""
    soa = np.ascontiguousarray(soa, dtype=np.float64)
    n = soa.shape[1]
    nt = pulse_derived(p)["nt"]
    vz = np.zeros(nt)
    fin = np.zeros((NFINAL, n)) if want_final else None
    bad = lib().or_propagate(C.byref(target_in(t)), C.byref(pulse_in(p)), gamma, cutoff,
                             float(stab_cutoff), float(stab_taper), _p(soa), n, float(n_norm),
                             _p(vz), _p(fin) if fin is not None else None, n_threads)
    return vz, fin, bad


def stab_taper_weight(Mhat, m0, r):
    return lib().or_stab_taper_weight(float(Mhat), float(m0), float(r))


def spectrum(vz, dt, t_origin, tau_H, n_out):
    vz = np.ascontiguousarray(vz, dtype=np.float64)
    om, y, ph, vr, vi = (np.zeros(n_out) for _ in range(5))
    lib().or_spectrum(_p(vz), len(vz), dt, t_origin, tau_H, n_out, _p(om), _p(y), _p(ph),
                      _p(vr), _p(vi))
    return om, y, ph, vr + 1j * vi


def gabor(vz, dt, t_origin, sigma, t_centres, omegas):
    """Gabor time-frequency map of the dipole velocity (the analysis of
    Sec. III.D), straight from its definition on the time grid:

        G(t_m, w_k) = | sum_n v_z(t_n) exp(-(t_n - t_m)^2 / (2 sigma^2))
                                 exp(i w_k t_n) dt |^2,

    t_n = t_origin + n dt, no truncation of the Gaussian.  Returns an
    (len(t_centres), len(omegas)) array."""
    vz = np.asarray(vz, dtype=np.float64)
    t = t_origin + dt * np.arange(len(vz))
    out = np.zeros((len(t_centres), len(omegas)))
    phase = np.exp(1j * np.outer(np.asarray(omegas, dtype=np.float64), t))   # (n_w, nt)
    for m, tm in enumerate(t_centres):
        u = vz * np.exp(-(t - tm) ** 2 / (2.0 * sigma * sigma)) * dt
        out[m] = np.abs(phase @ u) ** 2
    return out


def saddle_modified(p, Ip, t0, kperp2, c):
    """SFHK2 saddle with c = eta (R/2) n_z: (rc, tt, kz), rc = 0 on success."""
    out = np.zeros(2)
    rc = lib().or_saddle_modified(C.byref(pulse_in(p)), Ip, t0, kperp2, c, _p(out))
    return rc, out[0], out[1]


def pulse_Edot_complex(p, tau):
    out = np.zeros(2)
    lib().or_pulse_Edot_complex(C.byref(pulse_in(p)), float(np.real(tau)), float(np.imag(tau)),
                                _p(out))
    return out[0] + 1j * out[1]


def propagate_returns(t, p, soa, gamma, cutoff=0.0, stab_cutoff=0.0, r_out=5.0, r_in=2.0,
                      n_norm=0.0, n_threads=0):
    """propagate() that also records each trajectory's first return: the first
    grid step with |q_z| < r_in (along the polarisation axis, measured from
    the molecular centre) after one with |q_z| > r_out, and |p|^2/2 there.
    Returns (vz, steps, energies); step -1 = no return."""
    soa = np.ascontiguousarray(soa, dtype=np.float64)
    n = soa.shape[1]
    vz = np.zeros(pulse_derived(p)["nt"])
    ret = np.zeros((2, n))
    lib().or_propagate_returns(C.byref(target_in(t)), C.byref(pulse_in(p)), gamma, cutoff,
                               float(stab_cutoff), _p(soa), n, float(n_norm), _p(vz), r_out, r_in,
                               _p(ret), n_threads)
    return vz, ret[0].astype(int), ret[1]


def abs_sampling_constants(t, p, align=(ALIGN_FIXED, 0.0, 0.0), seed=0, instance=0):
    """(M, P) of the |a|-proportional sampler: acceptance min(1, |w|/M),
    accepted weight P w / alpha."""
    out = np.zeros(2)
    k = int(align[3]) if len(align) > 3 else 0
    psi = float(align[4]) if len(align) > 4 else 0.0
    lib().or_abs_sampling_constants(C.byref(target_in(t)), C.byref(pulse_in(p)), int(align[0]),
                                    float(align[1]), float(align[2]), psi, k, seed, instance,
                                    _p(out))
    return out[0], out[1]


def orbital_values(t, nhat, r):
    """psi0 at the points r (n x 3)."""
    r = np.ascontiguousarray(r, dtype=np.float64)
    out = np.zeros(r.shape[0])
    lib().or_orbital_values(C.byref(target_in(t)), _p(np.asarray(nhat, float).copy()), _p(r),
                            r.shape[0], _p(out))
    return out


def pi_direction(nhat, chi):
    """Unit vector m perpendicular to the axis n at azimuth chi (pi p-type primitives)."""
    n = np.ascontiguousarray(nhat, np.float64)
    m = np.zeros(3)
    lib().or_pi_direction(_p(n), float(chi), _p(m))
    return m


def euler_rotation(phi, theta, psi):
    """Rotation Rz(phi) Ry(theta) Rz(psi), molecular frame -> lab (3x3)."""
    R = np.zeros(9)
    lib().or_euler_rotation(float(phi), float(theta), float(psi), _p(R))
    return R.reshape(3, 3)


def ionization_step(t, p, orient, t0, kx, ky, eta=0):
    """The sampler's ionization step for one initial point (t0 on or off the
    grid, k_perp = (kx, ky)): dict with the saddle's tt, kz, the exit qz, the
    tunnelling action Sd, curv = E(t_s) kappa_z (+ c dE/dt for SFHK2), the
    dipole element mz = <kappa|z|psi0> and the amplitude a; None without a
    saddle root.  eta = +-1 picks the emitting centre of an SFHK2 target."""
    out = np.zeros(11)
    rc = lib().or_ionization_step(C.byref(target_in(t)), C.byref(pulse_in(p)),
                                  _p(np.asarray(orient, float).copy()), float(t0), float(kx),
                                  float(ky), int(eta), _p(out))
    if rc < 0:
        raise ValueError("eta must be +-1 for an SFHK2 target")
    if rc:
        return None
    return dict(tt=out[0], kz=out[1], qz=out[2], Sd=complex(out[3], out[4]),
                curv=complex(out[5], out[6]), mz=complex(out[7], out[8]),
                a=complex(out[9], out[10]))
