"""Thin ctypes binding of libsfhk (include/sfhk.h), same names as the C ABI.

Argument marshalling only: every step of the SFHK path runs in the library's
CUDA kernels.  Importing this module loads ``libsfhk.so`` from the package
directory and raises if it is missing (there is no CPU fallback); build it
with ``python -m paper_2608_13686_b300._build``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libsfhk.so")

SFHK_OK = 0
SFHK_E_INVAL, SFHK_E_NOMEM, SFHK_E_CUDA = -1, -2, -3
SFHK_E_TIMEOUT, SFHK_E_NUMERIC, SFHK_E_BUSY, SFHK_E_NOTFOUND = -4, -5, -6, -7
SFHK_MAX_PRIM = 8
SFHK_MAX_CENTRES = 8
SFHK_POT_MOLECULE, SFHK_POT_HARMONIC, SFHK_POT_POLYATOMIC = 0, 1, 2
SFHK_ALIGN_FIXED, SFHK_ALIGN_ISOTROPIC, SFHK_ALIGN_COS2, SFHK_ALIGN_QUADRATURE = 0, 1, 2, 3
SFHK_FP64, SFHK_MIXED = 0, 1
SFHK_PRIM_S, SFHK_PRIM_P_SIGMA, SFHK_PRIM_P_PI, SFHK_PRIM_P_DIR = 0, 1, 2, 3
SOA_FIELDS = 12
FINAL_FIELDS = 47


class SfhkError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class sfhk_target_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("n_prim", C.c_int), ("R", C.c_double),
                ("Z_inf", C.c_double), ("Z0", C.c_double), ("alpha", C.c_double),
                ("soft_a", C.c_double), ("Ip", C.c_double), ("ho_omega", C.c_double),
                ("prim_exp", C.c_double * SFHK_MAX_PRIM), ("prim_coef", C.c_double * SFHK_MAX_PRIM),
                ("ionization", C.c_int), ("sampling", C.c_int), ("sampling_factor", C.c_double),
                ("prim_kind", C.c_int * SFHK_MAX_PRIM), ("pi_azimuth", C.c_double),
                ("n_centres", C.c_int), ("centre_pos", (C.c_double * 3) * SFHK_MAX_CENTRES),
                ("centre_Z_inf", C.c_double * SFHK_MAX_CENTRES),
                ("centre_Z0", C.c_double * SFHK_MAX_CENTRES),
                ("centre_alpha", C.c_double * SFHK_MAX_CENTRES),
                ("prim_centre", C.c_int * SFHK_MAX_PRIM),
                ("prim_dir", (C.c_double * 3) * SFHK_MAX_PRIM)]


class sfhk_pulse_desc(C.Structure):
    _fields_ = [("lambda_nm", C.c_double), ("intensity_Wcm2", C.c_double),
                ("n_cycles", C.c_double), ("cep", C.c_double), ("dt", C.c_double)]


class sfhk_align_desc(C.Structure):
    _fields_ = [("kind", C.c_int), ("theta", C.c_double), ("phi", C.c_double),
                ("n_nodes", C.c_int), ("psi", C.c_double)]


class sfhk_run_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("gamma", C.c_double), ("prefactor_cutoff", C.c_double),
                ("dump_final", C.c_int), ("block_threads", C.c_int), ("blocks_per_sm", C.c_int),
                ("stability_cutoff", C.c_double), ("kernel_variant", C.c_int),
                ("record_returns", C.c_int), ("return_r_out", C.c_double),
                ("return_r_in", C.c_double), ("stability_taper", C.c_double),
                ("check_nonfinite", C.c_int), ("max_nonfinite", C.c_uint64)]


class sfhk_stats(C.Structure):
    _fields_ = [("n_traj", C.c_uint64), ("n_invalid", C.c_uint64), ("n_filtered", C.c_uint64),
                ("n_nonfinite", C.c_uint64), ("n_unstable", C.c_uint64),
                ("traj_steps", C.c_uint64), ("nt", C.c_int),
                ("kernel_ms", C.c_float), ("recomb_evals", C.c_uint64),
                ("fixed_params", C.c_int)]


class sfhk_server_opts(C.Structure):
    _fields_ = [("device_mem_budget", C.c_size_t), ("max_pending", C.c_int),
                ("max_active", C.c_int), ("precision", C.c_int), ("gamma", C.c_double),
                ("prefactor_cutoff", C.c_double), ("stability_cutoff", C.c_double),
                ("slice_ms", C.c_double), ("spectrum", C.c_int), ("fifo", C.c_int),
                ("stability_taper", C.c_double), ("check_nonfinite", C.c_int),
                ("max_nonfinite", C.c_uint64), ("max_reorder_s", C.c_double),
                ("max_queued_s", C.c_double)]


class sfhk_request(C.Structure):
    _fields_ = [("target", sfhk_target_desc), ("pulse", sfhk_pulse_desc),
                ("align", sfhk_align_desc), ("n_traj", C.c_uint64), ("seed", C.c_uint64),
                ("instance", C.c_uint32)]


class sfhk_result(C.Structure):
    _fields_ = [("status", C.c_int), ("nt", C.c_int), ("t_origin", C.c_double),
                ("dt", C.c_double), ("n_out", C.c_size_t), ("vz", C.POINTER(C.c_double)),
                ("vz_capacity", C.c_size_t), ("yield_", C.POINTER(C.c_double)),
                ("phase", C.POINTER(C.c_double)), ("spec_capacity", C.c_size_t),
                ("t_submit", C.c_double), ("t_admit", C.c_double), ("t_done", C.c_double),
                ("traj_steps", C.c_uint64), ("n_filtered", C.c_uint64),
                ("n_unstable", C.c_uint64), ("n_nonfinite", C.c_uint64),
                ("recomb_evals", C.c_uint64)]


class sfhk_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("rejected", C.c_uint64),
                ("cancelled", C.c_uint64), ("failed", C.c_uint64), ("slices", C.c_uint64),
                ("traj_steps", C.c_uint64), ("pending", C.c_int), ("active", C.c_int),
                ("gpu_busy_s", C.c_double), ("uptime_s", C.c_double),
                ("device_bytes", C.c_uint64), ("parked", C.c_uint64)]


SFHK_E_CANCELLED = -8

_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_lib = None


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2608_13686_b300._build` (no CPU fallback exists)")
    L = C.CDLL(LIB_PATH)
    sig = {
        "sfhk_strerror": ([C.c_int], C.c_char_p),
        "sfhk_create": ([C.POINTER(_vp), C.c_int, C.c_size_t], C.c_int),
        "sfhk_destroy": ([_vp], C.c_int),
        "sfhk_mem_used": ([_vp, C.POINTER(C.c_size_t)], C.c_int),
        "sfhk_create_target": ([_vp, C.POINTER(sfhk_target_desc), C.POINTER(_vp)], C.c_int),
        "sfhk_destroy_target": ([_vp], C.c_int),
        "sfhk_set_pulse": ([_vp, C.POINTER(sfhk_pulse_desc), C.POINTER(_vp)], C.c_int),
        "sfhk_destroy_pulse": ([_vp], C.c_int),
        "sfhk_pulse_grid": ([_vp, C.POINTER(C.c_int), _dp, _dp, _dp], C.c_int),
        "sfhk_sample_initial": ([_vp, _vp, _vp, C.POINTER(sfhk_align_desc), C.c_uint64, C.c_uint64,
                                 C.c_uint32, C.POINTER(_vp), _vp], C.c_int),
        "sfhk_sample_into": ([_vp, _vp, C.POINTER(sfhk_align_desc), C.c_uint64, C.c_uint32, _vp],
                             C.c_int),
        "sfhk_launch_count": ([C.POINTER(C.c_uint64)], C.c_int),
        "sfhk_fma_peak": ([C.c_int, C.c_int, C.c_int, _dp, C.POINTER(C.c_float)], C.c_int),
        "sfhk_load_ensemble": ([_vp, _vp, _vp, _dp, C.c_uint64, C.c_double, C.POINTER(_vp)],
                               C.c_int),
        "sfhk_ensemble_read": ([_vp, _dp, C.c_uint64], C.c_int),
        "sfhk_destroy_ensemble": ([_vp], C.c_int),
        "sfhk_propagate": ([_vp, _vp, C.POINTER(sfhk_run_opts), _vp], C.c_int),
        "sfhk_propagate_batch": ([_vp, C.POINTER(_vp), C.c_int, C.POINTER(sfhk_run_opts), _vp],
                                 C.c_int),
        "sfhk_dipole": ([_vp, _vp, _dp, C.c_size_t, _dp, _dp], C.c_int),
        "sfhk_spectrum_noalloc": ([_vp, C.c_size_t, C.c_double, C.c_double, C.c_double, _vp,
                                   _vp, _vp, C.c_size_t, _vp], C.c_int),
        "sfhk_server_create": ([C.c_int, C.POINTER(sfhk_server_opts), C.POINTER(_vp)], C.c_int),
        "sfhk_server_destroy": ([_vp], C.c_int),
        "sfhk_submit": ([_vp, C.POINTER(sfhk_request), C.POINTER(C.c_uint64)], C.c_int),
        "sfhk_poll": ([_vp, C.c_uint64, C.POINTER(sfhk_result)], C.c_int),
        "sfhk_wait": ([_vp, C.c_uint64, C.c_double, C.POINTER(sfhk_result)], C.c_int),
        "sfhk_cancel": ([_vp, C.c_uint64], C.c_int),
        "sfhk_server_stats_get": ([_vp, C.POINTER(sfhk_server_stats)], C.c_int),
        "sfhk_batch_create": ([_vp, C.POINTER(_vp), C.c_int, C.POINTER(sfhk_run_opts),
                               C.POINTER(_vp)], C.c_int),
        "sfhk_batch_launch": ([_vp, _vp], C.c_int),
        "sfhk_batch_destroy": ([_vp], C.c_int),
        "sfhk_autotune": ([_vp, _vp, C.POINTER(sfhk_run_opts), C.c_int, C.POINTER(C.c_int)],
                          C.c_int),
        "sfhk_dipole_device": ([_vp, C.POINTER(_vp), C.POINTER(C.c_size_t)], C.c_int),
        "sfhk_stats_get": ([_vp, C.POINTER(sfhk_stats)], C.c_int),
        "sfhk_final_state": ([_vp, _dp, C.c_uint64], C.c_int),
        "sfhk_returns": ([_vp, _dp, C.c_uint64], C.c_int),
        "sfhk_spectrum": ([_vp, C.c_size_t, C.c_double, C.c_double, C.c_double, _vp, _vp, _vp,
                           C.c_size_t, C.c_int, _vp], C.c_int),
        "sfhk_gabor": ([_vp, C.c_size_t, C.c_double, C.c_double, C.c_double, C.c_double,
                        C.c_double, C.c_size_t, C.c_double, C.c_double, C.c_size_t, _vp, C.c_int,
                        _vp], C.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def lib():
    return _load()


def strerror(code: int) -> str:
    return _load().sfhk_strerror(code).decode()


def _check(rc, where):
    if rc != SFHK_OK:
        raise SfhkError(rc, where)


def _p(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


# ------------------------------------------------------------------ descriptors
def target_desc(t: dict) -> sfhk_target_desc:
    d = sfhk_target_desc()
    d.kind = int(t.get("kind", SFHK_POT_MOLECULE))
    pe, pc = list(t["pexp"]), list(t["pcoef"])
    d.n_prim = len(pe)
    d.R, d.Z_inf, d.Z0 = float(t["R"]), float(t["Zinf"]), float(t["Z0"])
    d.alpha, d.soft_a, d.Ip = float(t["alpha"]), float(t["soft_a"]), float(t["Ip"])
    d.ho_omega = float(t.get("ho_omega", 0.0))
    d.ionization = int(t.get("ionization", 0))
    d.sampling = int(t.get("sampling", 0))
    d.sampling_factor = float(t.get("sampling_factor", 0.0))
    kinds = list(t.get("pkind", [SFHK_PRIM_S] * len(pe)))
    for i, (e, c) in enumerate(zip(pe, pc)):
        d.prim_exp[i] = e
        d.prim_coef[i] = c
        d.prim_kind[i] = int(kinds[i]) if i < len(kinds) else SFHK_PRIM_S
    d.pi_azimuth = float(t.get("pi_azimuth", 0.0))
    cen = t.get("centres", ())
    d.n_centres = len(cen)
    for i, c in enumerate(cen):          # (x, y, z, Z_inf, Z0, alpha)
        for a in range(3):
            d.centre_pos[i][a] = c[a]
        d.centre_Z_inf[i], d.centre_Z0[i], d.centre_alpha[i] = c[3], c[4], c[5]
    for i, c in enumerate(t.get("pcentre", ())):
        d.prim_centre[i] = int(c)
    for i, u in enumerate(t.get("pdir", ())):
        for a in range(3):
            d.prim_dir[i][a] = u[a]
    return d


def pulse_desc(p: dict) -> sfhk_pulse_desc:
    return sfhk_pulse_desc(p["lambda_nm"], p["intensity"], p["n_cycles"], p.get("cep", 0.0),
                           p["dt"])


def align_desc(a) -> sfhk_align_desc:
    """(kind, theta, phi[, n_nodes[, psi]])"""
    return sfhk_align_desc(int(a[0]), float(a[1]), float(a[2]), int(a[3]) if len(a) > 3 else 0,
                           float(a[4]) if len(a) > 4 else 0.0)


def run_opts(precision=SFHK_FP64, gamma=0.5, cutoff=0.0, dump=False, block_threads=0,
             blocks_per_sm=0, stab_cutoff=0.0, kernel_variant=0, returns=None,
             stab_taper=0.0, max_nonfinite=None) -> sfhk_run_opts:
    """returns = (r_out, r_in) records each trajectory's first return;
    stab_taper = r > 1 tapers the stability filter between stab_cutoff and
    r stab_cutoff (0: hard cut); max_nonfinite = n makes sfhk_dipole and
    sfhk_stats_get fail with SFHK_E_NUMERIC above n non-finite trajectories
    (None: no limit)."""
    r_out, r_in = returns if returns else (0.0, 0.0)
    return sfhk_run_opts(precision, gamma, cutoff, int(dump), block_threads, blocks_per_sm,
                         stab_cutoff, kernel_variant, int(bool(returns)), r_out, r_in,
                         stab_taper, int(max_nonfinite is not None),
                         int(max_nonfinite or 0))


# ------------------------------------------------------------------ C-ABI calls
def sfhk_create(device=0, budget=0):
    h = _vp()
    _check(_load().sfhk_create(C.byref(h), device, budget), "sfhk_create")
    return h


def sfhk_destroy(ctx):
    _check(_load().sfhk_destroy(ctx), "sfhk_destroy")


def sfhk_mem_used(ctx):
    v = C.c_size_t()
    _check(_load().sfhk_mem_used(ctx, C.byref(v)), "sfhk_mem_used")
    return v.value


def sfhk_create_target(ctx, t: dict):
    h = _vp()
    d = target_desc(t)
    _check(_load().sfhk_create_target(ctx, C.byref(d), C.byref(h)), "sfhk_create_target")
    return h


def sfhk_destroy_target(h):
    _check(_load().sfhk_destroy_target(h), "sfhk_destroy_target")


def sfhk_set_pulse(ctx, p: dict):
    h = _vp()
    d = pulse_desc(p)
    _check(_load().sfhk_set_pulse(ctx, C.byref(d), C.byref(h)), "sfhk_set_pulse")
    return h


def sfhk_destroy_pulse(h):
    _check(_load().sfhk_destroy_pulse(h), "sfhk_destroy_pulse")


def sfhk_pulse_grid(h):
    nt, t0, dt, tp = C.c_int(), C.c_double(), C.c_double(), C.c_double()
    _check(_load().sfhk_pulse_grid(h, C.byref(nt), C.byref(t0), C.byref(dt), C.byref(tp)),
           "sfhk_pulse_grid")
    return dict(nt=nt.value, t_origin=t0.value, dt=dt.value, Tp=tp.value)


def sfhk_sample_initial(ctx, target, pulse, align, n_traj, seed=0, instance=0, stream=None):
    h = _vp()
    a = align_desc(align)
    _check(_load().sfhk_sample_initial(ctx, target, pulse, C.byref(a), n_traj, seed, instance,
                                       C.byref(h), stream), "sfhk_sample_initial")
    return h


def sfhk_sample_into(ctx, ens, align, seed=0, instance=0, stream=None):
    a = align_desc(align)
    _check(_load().sfhk_sample_into(ctx, ens, C.byref(a), seed, instance, stream),
           "sfhk_sample_into")


def sfhk_launch_count():
    v = C.c_uint64()
    _check(_load().sfhk_launch_count(C.byref(v)), "sfhk_launch_count")
    return v.value


def sfhk_load_ensemble(ctx, target, pulse, soa: np.ndarray, n_norm=0.0):
    soa = np.ascontiguousarray(soa, dtype=np.float64)
    assert soa.shape[0] == SOA_FIELDS
    h = _vp()
    _check(_load().sfhk_load_ensemble(ctx, target, pulse, _p(soa), soa.shape[1], n_norm,
                                      C.byref(h)), "sfhk_load_ensemble")
    return h


def sfhk_ensemble_read(ens, n):
    out = np.zeros((SOA_FIELDS, n))
    _check(_load().sfhk_ensemble_read(ens, _p(out), n), "sfhk_ensemble_read")
    return out


def sfhk_destroy_ensemble(h):
    _check(_load().sfhk_destroy_ensemble(h), "sfhk_destroy_ensemble")


def sfhk_propagate(ctx, ens, opts: sfhk_run_opts, stream=None):
    _check(_load().sfhk_propagate(ctx, ens, C.byref(opts), stream), "sfhk_propagate")


def sfhk_propagate_batch(ctx, ens_list, opts: sfhk_run_opts, stream=None):
    arr = (_vp * len(ens_list))(*[e.value if isinstance(e, _vp) else e for e in ens_list])
    _check(_load().sfhk_propagate_batch(ctx, arr, len(ens_list), C.byref(opts), stream),
           "sfhk_propagate_batch")


def sfhk_batch_create(ctx, ens_list, opts: sfhk_run_opts):
    arr = (_vp * len(ens_list))(*[e.value if isinstance(e, _vp) else e for e in ens_list])
    h = _vp()
    _check(_load().sfhk_batch_create(ctx, arr, len(ens_list), C.byref(opts), C.byref(h)),
           "sfhk_batch_create")
    return h


def sfhk_batch_launch(batch, stream=None):
    _check(_load().sfhk_batch_launch(batch, stream), "sfhk_batch_launch")


def sfhk_batch_destroy(batch):
    _check(_load().sfhk_batch_destroy(batch), "sfhk_batch_destroy")


def sfhk_autotune(ctx, ens, opts: sfhk_run_opts, max_items=0):
    choice = (C.c_int * 3)()
    _check(_load().sfhk_autotune(ctx, ens, C.byref(opts), max_items, choice), "sfhk_autotune")
    return dict(block_threads=choice[0], kernel_variant=choice[1], max_registers=choice[2])


def sfhk_dipole(ctx, ens, nt):
    vz = np.zeros(nt)
    t0, dt = C.c_double(), C.c_double()
    _check(_load().sfhk_dipole(ctx, ens, _p(vz), nt, C.byref(t0), C.byref(dt)), "sfhk_dipole")
    return vz


def sfhk_dipole_device(ens):
    p, nt = _vp(), C.c_size_t()
    _check(_load().sfhk_dipole_device(ens, C.byref(p), C.byref(nt)), "sfhk_dipole_device")
    return p.value, nt.value


def sfhk_stats_get(ens):
    """Counters of the last propagation.  Over the non-finite limit the call
    raises SfhkError(SFHK_E_NUMERIC) whose .stats holds the counters."""
    s = sfhk_stats()
    rc = _load().sfhk_stats_get(ens, C.byref(s))
    d = {f: getattr(s, f) for f, _ in sfhk_stats._fields_}
    if rc == SFHK_E_NUMERIC:
        err = SfhkError(rc, "sfhk_stats_get")
        err.stats = d
        raise err
    _check(rc, "sfhk_stats_get")
    return d


def sfhk_returns(ens, n):
    """(steps, energies) of the first returns; step -1 = none."""
    out = np.zeros((2, n))
    _check(_load().sfhk_returns(ens, _p(out), n), "sfhk_returns")
    return out[0].astype(int), out[1]


def sfhk_final_state(ens, n):
    out = np.zeros((FINAL_FIELDS, n))
    _check(_load().sfhk_final_state(ens, _p(out), n), "sfhk_final_state")
    return out


def sfhk_spectrum(vz, dt, t_origin, tau_H, n_out):
    """Host-buffer form: returns (omega, yield, phase)."""
    vz = np.ascontiguousarray(vz, dtype=np.float64)
    om, y, ph = np.zeros(n_out), np.zeros(n_out), np.zeros(n_out)
    _check(_load().sfhk_spectrum(vz.ctypes.data, len(vz), dt, t_origin, tau_H, om.ctypes.data,
                                 y.ctypes.data, ph.ctypes.data, n_out, 0, None), "sfhk_spectrum")
    return om, y, ph


def sfhk_spectrum_device(vz_ptr, nt, dt, t_origin, tau_H, om_ptr, y_ptr, ph_ptr, n_out,
                         stream=None):
    """Device-buffer form (raw device pointers, asynchronous on `stream`)."""
    _check(_load().sfhk_spectrum(vz_ptr, nt, dt, t_origin, tau_H, om_ptr, y_ptr, ph_ptr, n_out, 1,
                                 stream), "sfhk_spectrum")


SFHK_NOALLOC_MAX_NT = 32768


# ------------------------------------------------------------------ serving
def server_opts(precision=SFHK_MIXED, gamma=0.5, cutoff=0.0, stab_cutoff=0.0, budget=0,
                max_pending=0, max_active=0, slice_ms=0.0, spectrum=True, fifo=False,
                stab_taper=0.0, max_nonfinite=None, max_reorder_s=0.0, max_queued_s=0.0):
    return sfhk_server_opts(budget, max_pending, max_active, precision, gamma, cutoff,
                            stab_cutoff, slice_ms, int(spectrum), int(fifo), stab_taper,
                            int(max_nonfinite is not None), int(max_nonfinite or 0),
                            float(max_reorder_s), float(max_queued_s))


def request(target: dict, pulse: dict, align, n_traj, seed=0, instance=0) -> sfhk_request:
    return sfhk_request(target_desc(target), pulse_desc(pulse), align_desc(align), n_traj, seed,
                        instance)


def sfhk_server_create(device=0, opts: sfhk_server_opts = None):
    h = _vp()
    o = opts if opts is not None else server_opts()
    _check(_load().sfhk_server_create(device, C.byref(o), C.byref(h)), "sfhk_server_create")
    return h


def sfhk_server_destroy(h):
    _check(_load().sfhk_server_destroy(h), "sfhk_server_destroy")


def sfhk_submit(server, req: sfhk_request):
    rid = C.c_uint64()
    _check(_load().sfhk_submit(server, C.byref(req), C.byref(rid)), "sfhk_submit")
    return rid.value


class Result:
    """Host buffers for one server result and the fields sfhk_poll/sfhk_wait fill."""

    def __init__(self, nt_max=1 << 16):
        self.vz = np.zeros(nt_max)
        self.yield_ = np.zeros(nt_max // 2)
        self.phase = np.zeros(nt_max // 2)
        self.c = sfhk_result()
        self.c.vz = _p(self.vz)
        self.c.vz_capacity = nt_max
        self.c.yield_ = _p(self.yield_)
        self.c.phase = _p(self.phase)
        self.c.spec_capacity = nt_max // 2

    def as_dict(self):
        c = self.c
        return dict(status=c.status, nt=c.nt, t_origin=c.t_origin, dt=c.dt,
                    vz=self.vz[:c.nt].copy(), yield_=self.yield_[:c.n_out].copy(),
                    phase=self.phase[:c.n_out].copy(), t_submit=c.t_submit, t_admit=c.t_admit,
                    t_done=c.t_done, traj_steps=c.traj_steps, n_filtered=c.n_filtered,
                    n_unstable=c.n_unstable, n_nonfinite=c.n_nonfinite,
                    recomb_evals=c.recomb_evals)


def sfhk_poll(server, rid, res: Result = None):
    """None while the request is running; its result dict once it has ended."""
    res = res or Result()
    rc = _load().sfhk_poll(server, rid, C.byref(res.c))
    if rc == SFHK_E_BUSY:
        return None
    _check(rc, "sfhk_poll")
    return res.as_dict()


def sfhk_wait(server, rid, timeout_s=60.0, res: Result = None):
    res = res or Result()
    _check(_load().sfhk_wait(server, rid, timeout_s, C.byref(res.c)), "sfhk_wait")
    return res.as_dict()


def sfhk_cancel(server, rid):
    _check(_load().sfhk_cancel(server, rid), "sfhk_cancel")


def sfhk_server_stats_get(server):
    st = sfhk_server_stats()
    _check(_load().sfhk_server_stats_get(server, C.byref(st)), "sfhk_server_stats_get")
    return {f: getattr(st, f) for f, _ in sfhk_server_stats._fields_}


def sfhk_spectrum_noalloc(vz_ptr, nt, dt, t_origin, tau_H, om_ptr, y_ptr, ph_ptr, n_out,
                          stream=None):
    """Device-buffer spectrum that allocates nothing (fixed scratch of
    SFHK_NOALLOC_MAX_NT points shared by all calls; serialise overlapping calls)."""
    _check(_load().sfhk_spectrum_noalloc(vz_ptr, nt, dt, t_origin, tau_H, om_ptr, y_ptr, ph_ptr,
                                         n_out, stream), "sfhk_spectrum_noalloc")


def sfhk_gabor(vz, dt, t_origin, sigma, t_first, t_step, n_t, omega_first, omega_step, n_w):
    """Host-buffer form: returns the (n_t, n_w) Gabor map."""
    vz = np.ascontiguousarray(vz, dtype=np.float64)
    out = np.zeros((n_t, n_w))
    _check(_load().sfhk_gabor(vz.ctypes.data, len(vz), dt, t_origin, sigma, t_first, t_step, n_t,
                              omega_first, omega_step, n_w, out.ctypes.data, 0, None),
           "sfhk_gabor")
    return out


def sfhk_gabor_device(vz_ptr, nt, dt, t_origin, sigma, t_first, t_step, n_t, omega_first,
                      omega_step, n_w, out_ptr, stream=None):
    """Device-buffer form (raw device pointers, asynchronous on `stream`)."""
    _check(_load().sfhk_gabor(vz_ptr, nt, dt, t_origin, sigma, t_first, t_step, n_t, omega_first,
                              omega_step, n_w, out_ptr, 1, stream), "sfhk_gabor")


EXPORTED = [
    "sfhk_create", "sfhk_destroy", "sfhk_mem_used", "sfhk_create_target", "sfhk_destroy_target",
    "sfhk_set_pulse", "sfhk_destroy_pulse", "sfhk_pulse_grid", "sfhk_sample_initial",
    "sfhk_load_ensemble", "sfhk_ensemble_read", "sfhk_destroy_ensemble", "sfhk_propagate",
    "sfhk_propagate_batch", "sfhk_dipole", "sfhk_dipole_device", "sfhk_stats_get",
    "sfhk_final_state", "sfhk_spectrum", "sfhk_strerror", "sfhk_sample_into",
    "sfhk_launch_count", "sfhk_autotune", "sfhk_spectrum_noalloc", "sfhk_server_create",
    "sfhk_server_destroy", "sfhk_submit", "sfhk_poll", "sfhk_wait", "sfhk_cancel",
    "sfhk_server_stats_get", "sfhk_batch_create", "sfhk_batch_launch", "sfhk_batch_destroy",
    "sfhk_gabor", "sfhk_returns", "sfhk_fma_peak",
]


def sfhk_fma_peak(kind, iters, device=0):
    """Measured FMA throughput (TFLOP/s, ms): kind 0 FP32, 1 packed FP32 pairs,
    2 FP64."""
    tf, ms = C.c_double(), C.c_float()
    _check(_load().sfhk_fma_peak(device, kind, iters, C.byref(tf), C.byref(ms)), "sfhk_fma_peak")
    return tf.value, ms.value

