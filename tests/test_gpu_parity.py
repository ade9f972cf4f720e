"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every input is seeded and synthetic; the oracle computes the expected values
from the same inputs (its own sampler for the ionization step, the same
initial points for the propagation).  Tolerances:
  * integer decisions (birth index, filter/non-finite status): exact;
  * ionization step (closed forms on the GPU vs quadrature in the oracle):
    relative 1e-10 (weights) and 1e-12 (phase-space points);
  * FP64 propagation, per trajectory: |dy| <= 1e-10 max(1, |M|) |y|-scale,
    where |M| is the largest stability-matrix element (chaotic trajectories
    amplify last-bit differences of exp/rsqrt by |M|);
  * dipole: relative L2 1e-9 (FP64) and 1e-4 (mixed precision);
  * spectrum: relative 1e-12 of the largest |v(omega)|.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W

pytestmark = pytest.mark.gpu

GAMMA = W.GAMMA
CUT = W.CUTOFF
STAB = W.STAB_CUTOFF


@pytest.fixture(scope="module")
def S():
    from paper_2608_13686_b300 import _build
    _build.build()
    from paper_2608_13686_b300 import sfhk
    return sfhk


@pytest.fixture(scope="module")
def ctx(S):
    c = S.sfhk_create(0, 0)
    yield c
    S.sfhk_destroy(c)


def _rel_l2(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# ------------------------------------------------------------------ pulse grid
def test_pulse_grid_matches_oracle(S, ctx):
    for p in (W.PULSE_800, W.PULSE_1200, W.pulse(1333.0, 1.1e14, 2.5, cep=0.3)):
        h = S.sfhk_set_pulse(ctx, p)
        g = S.sfhk_pulse_grid(h)
        d = O.pulse_derived(p)
        assert g["nt"] == d["nt"]
        assert g["t_origin"] == pytest.approx(d["t_origin"], rel=1e-15)
        assert g["Tp"] == pytest.approx(d["Tp"], rel=1e-15)
        S.sfhk_destroy_pulse(h)


# ------------------------------------------------------------------ ionization step
def _target(name):
    """A workload target by name, with '+'-separated variants: sfhk2 (modified
    saddle), abs (sampling ~ |a|), abs150 (the same at kappa = 150, where
    about a fifth of the trajectories exhaust their attempts), chi90 (the
    other 1 pi_u component), 8prim (SFHK_MAX_PRIM s-type primitives per
    centre)."""
    base, *variants = name.split("+")
    t = W.TARGETS[base]
    if "8prim" in variants:
        t = dict(t, pexp=[3.0, 1.8, 1.3, 0.9, 0.6, 0.4, 0.25, 0.15],
                 pcoef=[0.05, 0.1, 0.2, 0.3, 0.3, 0.2, 0.1, 0.05])
    if "sfhk2" in variants:
        t = W.sfhk2(t)
    if "abs" in variants:
        t = W.abs_sampled(t, 5.0)
    if "abs150" in variants:
        t = W.abs_sampled(t, 150.0)
    if "chi90" in variants:
        t = W.pi_component(t, 0.5 * np.pi)
    return t


@pytest.mark.parametrize("name,pulse,align,n,seed,inst", [
    ("H2", W.PULSE_800, W.fixed(0.0), 1000, 0, 0),
    ("H2", W.PULSE_800, W.fixed(45.0, 30.0), 777, 5, 3),
    ("N2", W.PULSE_1200, W.COS2, 1000, 1, 7),
    ("N2", W.pulse(1500.0, 0.9e14, 2), W.ISO, 333, 2, 1),
    ("H2", W.PULSE_800, W.quadrature(10), 1001, 3, 2),
    ("N2", W.PULSE_1200, W.quadrature(7), 500, 4, 0),
    ("N2+sfhk2", W.PULSE_1200, W.fixed(0.0), 800, 5, 0),
    ("N2+sfhk2", W.PULSE_PAPER, W.fixed(30.0, 10.0), 600, 6, 1),
    ("H2+sfhk2", W.PULSE_800, W.ISO, 700, 7, 2),
    ("H2+abs", W.PULSE_800, W.fixed(0.0), 900, 8, 0),
    ("N2+abs", W.PULSE_1200, W.ISO, 600, 9, 3),
    ("N2+abs+sfhk2", W.PULSE_1200, W.quadrature(5), 500, 10, 1),
    ("N2_sp", W.PULSE_1200, W.ISO, 700, 11, 0),
    ("N2_sp", W.PULSE_1200, W.fixed(20.0, 40.0), 500, 12, 2),
    ("N2_sp+sfhk2", W.PULSE_1200, W.quadrature(4), 500, 13, 1),
    ("N2_sp+abs", W.PULSE_1200, W.fixed(60.0, 0.0), 400, 14, 0),
    ("N2_pi", W.PULSE_1200, W.ISO, 600, 15, 0),
    ("N2_pi+chi90", W.PULSE_1200, W.fixed(60.0, 30.0), 500, 16, 1),
    ("N2_pi+sfhk2", W.PULSE_1200, W.fixed(90.0, 0.0), 500, 17, 2),
    ("N2_pi+abs", W.PULSE_1200, W.quadrature(6), 400, 18, 0),
    ("H2+abs150", W.PULSE_800, W.fixed(0.0), 400, 21, 0),
    # the largest sizes the interface declares: SFHK_MAX_QUAD_NODES nodes,
    # SFHK_MAX_PRIM primitives per centre, and a long pulse (Nt = 26477)
    ("H2", W.PULSE_800, W.quadrature(64), 640, 22, 0),
    ("H2+8prim", W.PULSE_800, W.fixed(20.0), 500, 23, 0),
    ("H2", W.pulse(2400.0, 0.8e14, 4), W.fixed(0.0), 300, 24, 0),
])
def test_sampler_matches_oracle(S, ctx, name, pulse, align, n, seed, inst):
    t = _target(name)
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, pulse)
    e = S.sfhk_sample_initial(ctx, th, ph, align, n, seed, inst)
    g = S.sfhk_ensemble_read(e, n)
    o, _, bad = O.sample(t, pulse, align, seed=seed, instance=inst, n=n)
    assert np.array_equal(g[0], o[0])                      # birth index: exact
    for f in range(1, 10):
        sc = max(1.0, np.abs(o[f]).max())
        assert np.max(np.abs(g[f] - o[f])) <= 1e-12 * sc, f
    w_g, w_o = g[10] + 1j * g[11], o[10] + 1j * o[11]
    assert np.all(np.abs(w_g - w_o) <= 1e-10 * np.abs(w_o) + 1e-300)
    st = S.sfhk_stats_get(e)
    assert st["n_invalid"] == bad
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)


# ------------------------------------------------------------------ propagation
def _run(S, ctx, t, p, soa, precision, cutoff=CUT, dump=True, n_norm=0.0, stab=STAB):
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
    e = S.sfhk_load_ensemble(ctx, th, ph, soa, n_norm)
    S.sfhk_propagate(ctx, e, S.run_opts(precision, GAMMA, cutoff, dump, stab_cutoff=stab))
    nt = S.sfhk_pulse_grid(ph)["nt"]
    vz = S.sfhk_dipole(ctx, e, nt)
    fin = S.sfhk_final_state(e, soa.shape[1]) if dump else None
    st = S.sfhk_stats_get(e)
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)
    return vz, fin, st


def _compare_final(fin_g, fin_o, tol):
    """Per-trajectory comparison scaled by max(1, |M|); returns the fraction
    that also passes without the |M| scaling."""
    st_g, st_o = fin_g[46], fin_o[46]
    assert np.array_equal(st_g, st_o)
    M = np.abs(fin_o[6:42]).max(axis=0)
    scale = np.maximum(1.0, M)
    ysc = np.maximum(1.0, np.abs(fin_o[0:43]).max(axis=0))
    err = np.abs(fin_g[0:43] - fin_o[0:43]).max(axis=0) / ysc
    C_g, C_o = fin_g[43] + 1j * fin_g[44], fin_o[43] + 1j * fin_o[44]
    errC = np.abs(C_g - C_o) / np.maximum(1.0, np.abs(C_o))
    ok = (err <= tol * scale) & (errC <= tol * scale ** 1.5)
    assert ok.all(), (np.flatnonzero(~ok)[:10], err[~ok][:5], M[~ok][:5], errC[~ok][:5])
    return float(np.mean((err <= tol) & (errC <= tol)))


@pytest.mark.parametrize("name,pulse,align,n", [
    ("H2", W.PULSE_800, W.fixed(0.0), 1000),
    ("H2", W.PULSE_800, W.fixed(90.0), 517),
    ("N2", W.PULSE_1200, W.COS2, 700),
    ("N2_sp", W.PULSE_1200, W.ISO, 600),
    ("N2_pi", W.PULSE_1200, W.ISO, 600),
    ("N2_pi+chi90", W.PULSE_1200, W.fixed(70.0, 20.0), 500),
    ("H2+8prim", W.PULSE_800, W.fixed(20.0), 400),
    ("H2", W.pulse(2400.0, 0.8e14, 4), W.fixed(0.0), 200),
])
def test_fp64_propagation_per_trajectory_and_dipole(S, ctx, name, pulse, align, n):
    t = _target(name)
    soa, _, _ = O.sample(t, pulse, align, seed=11, n=n)
    vz_o, fin_o, bad_o = O.propagate(t, pulse, soa, GAMMA, cutoff=CUT, want_final=True,
                                         stab_cutoff=STAB)
    vz_g, fin_g, st = _run(S, ctx, t, pulse, soa, S.SFHK_FP64)
    frac = _compare_final(fin_g, fin_o, 1e-10)
    assert frac > 0.9
    # time index of the stored state: the last grid point for a trajectory
    # that ran to the end, never before its birth
    nt = O.pulse_derived(pulse)["nt"]
    assert np.all(fin_g[45][fin_g[46] == 0] == nt - 1)
    assert np.all((fin_g[45] >= soa[0]) & (fin_g[45] <= nt - 1))
    assert st["n_filtered"] + st["n_nonfinite"] + st["n_unstable"] == bad_o
    assert _rel_l2(vz_g, vz_o) <= 1e-9


@pytest.mark.parametrize("name,pulse,align,n", [
    ("H2", W.PULSE_800, W.fixed(0.0), 1000),
    ("H2", W.PULSE_800, W.fixed(45.0), 1000),
    ("N2", W.PULSE_1200, W.COS2, 600),
    ("N2_sp", W.PULSE_1200, W.ISO, 600),
    ("N2_pi", W.PULSE_1200, W.ISO, 600),
    ("H2+8prim", W.PULSE_800, W.fixed(20.0), 400),
    ("H2", W.pulse(2400.0, 0.8e14, 4), W.fixed(0.0), 200),
])
def test_mixed_precision_dipole(S, ctx, name, pulse, align, n):
    t = _target(name)
    soa, _, _ = O.sample(t, pulse, align, seed=12, n=n)
    vz_o, _, _ = O.propagate(t, pulse, soa, GAMMA, cutoff=CUT, stab_cutoff=STAB)
    vz_g, _, _ = _run(S, ctx, t, pulse, soa, S.SFHK_MIXED, dump=False)
    err = _rel_l2(vz_g, vz_o)
    print(f"mixed rel-L2 {name}: {err:.3e}")
    assert err <= 1e-4


def test_prefactor_filter_off_matches(S, ctx):
    # without the filter (the library default) the FP64 path still agrees;
    # H2 at 45 degrees, a small ensemble
    t = W.TARGETS["H2"]
    soa, _, _ = O.sample(t, W.PULSE_800, W.fixed(45.0), seed=3, n=200)
    vz_o, fin_o, _ = O.propagate(t, W.PULSE_800, soa, GAMMA, cutoff=0.0, want_final=True)
    vz_g, fin_g, _ = _run(S, ctx, t, W.PULSE_800, soa, S.SFHK_FP64, cutoff=0.0, stab=0.0)
    M = np.abs(fin_o[6:42]).max(axis=0)
    tame = M < 1e4
    C_g, C_o = fin_g[43] + 1j * fin_g[44], fin_o[43] + 1j * fin_o[44]
    assert np.all(np.abs(C_g - C_o)[tame] <= 1e-9 * np.maximum(1, np.abs(C_o[tame])))


# ------------------------------------------------------------------ edge cases
def test_single_trajectory_and_last_grid_point(S, ctx):
    t, p = W.TARGETS["H2"], W.PULSE_800
    nt = O.pulse_derived(p)["nt"]
    soa, _, _ = O.sample(t, p, W.fixed(30.0), seed=4, n=3)
    soa[0, 1] = nt - 1          # born at the last grid point: one contribution, no step
    soa[0, 2] = 0               # born at the first grid point: the whole pulse
    for n in (1, 3):
        s = np.ascontiguousarray(soa[:, :n])
        vz_o, fin_o, _ = O.propagate(t, p, s, GAMMA, cutoff=CUT, want_final=True,
                                      stab_cutoff=STAB)
        vz_g, fin_g, st = _run(S, ctx, t, p, s, S.SFHK_FP64)
        assert _rel_l2(vz_g, vz_o) <= 1e-9
        _compare_final(fin_g, fin_o, 1e-10)
    if st["n_filtered"] == 0 and st["n_nonfinite"] == 0 and st["n_unstable"] == 0:
        assert st["traj_steps"] == (nt - 1 - int(soa[0, 0])) + 0 + (nt - 1)


def test_harmonic_prefactor_closed_form_on_gpu(S, ctx):
    # gamma = omega: C = exp(-3 i omega tau / 2) (field off)
    w = 0.5
    t = W.harmonic_target(w)
    p = W.pulse(800.0, 0.0, 3)
    nt = O.pulse_derived(p)["nt"]
    taus = np.array([1.0, 30.0, 200.0])
    soa = np.zeros((12, 3))
    soa[0] = nt - 1 - np.round(taus / 0.05)
    soa[1:4] = np.array([[0.3], [-0.2], [0.5]])
    soa[4:7] = np.array([[0.1], [0.2], [-0.1]])
    soa[9], soa[10] = 1.0, 1.0
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
    e = S.sfhk_load_ensemble(ctx, th, ph, soa)
    for prec, tol in ((S.SFHK_FP64, 1e-6), (S.SFHK_MIXED, 2e-4)):
        S.sfhk_propagate(ctx, e, S.run_opts(prec, w, 0.0, True))
        fin = S.sfhk_final_state(e, 3)
        C = fin[43] + 1j * fin[44]
        assert np.max(np.abs(C - np.exp(-1.5j * w * taus))) < tol, prec
    S.sfhk_destroy_ensemble(e)


def test_invalid_arguments(S, ctx):
    t = W.TARGETS["H2"]
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, W.PULSE_800)
    with pytest.raises(S.SfhkError):
        S.sfhk_sample_initial(ctx, th, ph, W.fixed(0.0), 0)
    bad = np.zeros((12, 2))
    bad[0, 0] = 1e7
    with pytest.raises(S.SfhkError):
        S.sfhk_load_ensemble(ctx, th, ph, bad)
    e = S.sfhk_sample_initial(ctx, th, ph, W.fixed(0.0), 64)
    with pytest.raises(S.SfhkError):
        S.sfhk_propagate(ctx, e, S.run_opts(7, GAMMA))
    with pytest.raises(S.SfhkError):
        S.sfhk_propagate(ctx, e, S.run_opts(S.SFHK_FP64, -1.0))
    with pytest.raises(S.SfhkError):
        S.sfhk_final_state(e, 64)     # no dump taken
    bad_t = dict(t)
    bad_t["pexp"] = [-1.0]
    bad_t["pcoef"] = [1.0]
    with pytest.raises(S.SfhkError):
        S.sfhk_create_target(ctx, bad_t)
    with pytest.raises(S.SfhkError):
        S.sfhk_set_pulse(ctx, W.pulse(800.0, 1e14, 1.0))
    S.sfhk_destroy_ensemble(e)


def test_memory_budget_refusal(S):
    c = S.sfhk_create(0, 1 << 20)          # 1 MiB budget
    t = S.sfhk_create_target(c, W.TARGETS["H2"])
    p = S.sfhk_set_pulse(c, W.PULSE_800)
    with pytest.raises(S.SfhkError) as e:
        S.sfhk_sample_initial(c, t, p, W.fixed(0.0), 100_000)
    assert e.value.code == S.SFHK_E_NOMEM
    S.sfhk_destroy_pulse(p)
    assert S.sfhk_mem_used(c) == 0
    S.sfhk_destroy(c)


# ------------------------------------------------------------------ batch
def test_batch_equals_separate(S, ctx):
    cases = [("H2", W.PULSE_800, W.fixed(20.0), 300, 1),
             ("N2", W.pulse(1000.0, 1.6e14, 2), W.COS2, 257, 2),
             ("H2", W.pulse(1400.0, 1.0e14, 4), W.fixed(70.0), 65, 3)]
    handles, ens, nts = [], [], []
    for name, p, al, n, seed in cases:
        th, ph = S.sfhk_create_target(ctx, W.TARGETS[name]), S.sfhk_set_pulse(ctx, p)
        handles += [th, ph]
        ens.append(S.sfhk_sample_initial(ctx, th, ph, al, n, seed, seed))
        nts.append(S.sfhk_pulse_grid(ph)["nt"])
    for prec in (S.SFHK_FP64, S.SFHK_MIXED):
        opts = S.run_opts(prec, GAMMA, CUT, stab_cutoff=STAB)
        alone = []
        for e, nt in zip(ens, nts):
            S.sfhk_propagate(ctx, e, opts)
            alone.append(S.sfhk_dipole(ctx, e, nt))
        S.sfhk_propagate_batch(ctx, ens, opts)
        for e, nt, a in zip(ens, nts, alone):
            b = S.sfhk_dipole(ctx, e, nt)
            assert _rel_l2(b, a) <= 1e-12, prec
    for e in ens:
        S.sfhk_destroy_ensemble(e)


# ------------------------------------------------------------------ spectrum
def test_spectrum_matches_oracle(S, ctx):
    rng = np.random.default_rng(8)
    for nt in (1000, 6620, 997):
        vz = rng.normal(size=nt) * np.exp(-np.linspace(-3, 3, nt) ** 2)
        dt, t0 = 0.05, -0.5 * (nt - 1) * 0.05
        tau = 0.5 * nt * dt
        n_out = nt // 2
        om_o, y_o, ph_o, v_o = O.spectrum(vz, dt, t0, tau, n_out)
        om_g, y_g, ph_g = S.sfhk_spectrum(vz, dt, t0, tau, n_out)
        assert np.allclose(om_g, om_o, rtol=1e-15)
        assert np.max(np.abs(y_g - y_o)) <= 1e-11 * y_o.max()
        big = np.abs(v_o) > 1e-6 * np.abs(v_o).max()
        dph = np.angle(np.exp(1j * (ph_g - ph_o)))
        assert np.max(np.abs(dph[big])) < 1e-9


def test_autotuner_choice_is_valid_and_result_independent(S, ctx):
    """The launch shape changes only the scheduling: FP64 results agree to
    rounding of the reduction order.  In FP32 the register-cap variants are
    separate ptxas compilations, which may fuse multiplies and adds into FMAs
    differently, so the mixed dipole is compared at 1e-5 (its oracle tolerance
    is 1e-4)."""
    t = W.TARGETS["H2"]
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, W.PULSE_800)
    e = S.sfhk_sample_initial(ctx, th, ph, W.fixed(0.0), 3000, 21, 0)
    nt = S.sfhk_pulse_grid(ph)["nt"]
    for prec, tol in ((S.SFHK_MIXED, 1e-5), (S.SFHK_FP64, 1e-12)):
        ref = None
        for var in range(1, 7):
            for bt in ((32, 64, 128) if prec == S.SFHK_MIXED else (64,)):
                S.sfhk_propagate(ctx, e, S.run_opts(prec, GAMMA, CUT, block_threads=bt,
                                                    stab_cutoff=STAB, kernel_variant=var))
                vz = S.sfhk_dipole(ctx, e, nt)
                if ref is None:
                    ref = vz
                assert _rel_l2(vz, ref) <= tol, (prec, var, bt)
    choice = S.sfhk_autotune(ctx, e, S.run_opts(S.SFHK_MIXED, GAMMA, CUT, stab_cutoff=STAB))
    assert choice["block_threads"] in (32, 64, 128) and 1 <= choice["kernel_variant"] <= 6
    S.sfhk_propagate(ctx, e, S.run_opts(S.SFHK_MIXED, GAMMA, CUT, stab_cutoff=STAB))
    S.sfhk_destroy_ensemble(e)


def test_sfhk2_dipole_end_to_end(S, ctx):
    """SFHK2 (modified saddle, Sec. III.D): each side samples its own ensemble
    (device sampler vs the oracle's) and propagates it; FP64 dipoles agree."""
    t, p = W.sfhk2(W.TARGETS["N2"]), W.PULSE_1200
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
    e = S.sfhk_sample_initial(ctx, th, ph, W.fixed(0.0), 600, 9, 0)
    S.sfhk_propagate(ctx, e, S.run_opts(S.SFHK_FP64, GAMMA, CUT, stab_cutoff=STAB))
    vz = S.sfhk_dipole(ctx, e, S.sfhk_pulse_grid(ph)["nt"])
    soa, _, _ = O.sample(t, p, W.fixed(0.0), seed=9, n=600)
    vz_o, _, _ = O.propagate(t, p, soa, GAMMA, cutoff=CUT, stab_cutoff=STAB)
    assert _rel_l2(vz, vz_o) <= 1e-9
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)


def test_first_returns_match_oracle(S, ctx):
    """First returns (long/short trajectory analysis, Sec. III.D): FP64 steps
    equal the oracle's and energies agree; mixed precision agrees except at
    threshold ties."""
    t, p = W.TARGETS["N2"], W.PULSE_1200
    soa, _, _ = O.sample(t, p, W.fixed(0.0), seed=17, n=700)
    _, st_o, en_o = O.propagate_returns(t, p, soa, GAMMA, cutoff=CUT, stab_cutoff=STAB,
                                        r_out=6.0, r_in=2.0)
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
    e = S.sfhk_load_ensemble(ctx, th, ph, soa, 0.0)
    for prec in (S.SFHK_FP64, S.SFHK_MIXED):
        S.sfhk_propagate(ctx, e, S.run_opts(prec, GAMMA, CUT, stab_cutoff=STAB,
                                            returns=(6.0, 2.0)))
        st, en = S.sfhk_returns(e, soa.shape[1])
        if prec == S.SFHK_FP64:
            assert np.array_equal(st, st_o)
            ok = st_o >= 0
            assert np.allclose(en[ok], en_o[ok], rtol=1e-9, atol=1e-12)
        else:
            assert np.mean(st == st_o) >= 0.99
            both = (st == st_o) & (st_o >= 0)
            assert np.allclose(en[both], en_o[both], rtol=1e-3, atol=1e-6)
    assert (st_o >= 0).sum() >= 50
    # without the option the call is refused
    S.sfhk_propagate(ctx, e, S.run_opts(S.SFHK_MIXED, GAMMA, CUT, stab_cutoff=STAB))
    with pytest.raises(RuntimeError):
        S.sfhk_returns(e, soa.shape[1])
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)


def test_ptype_target_validation(S, ctx):
    """A primitive kind other than s, sigma p or pi p is refused; a target whose
    p-type primitives cancel (R = 0, only p-type) has no normalisable orbital
    and is refused too."""
    t = dict(W.TARGETS["N2_sp"], pkind=[0, 0, 3, 1])
    with pytest.raises(S.SfhkError):
        S.sfhk_create_target(ctx, t)
    t = dict(W.TARGETS["N2_sp"], R=0.0, pexp=[1.2], pcoef=[0.5], pkind=[1])
    with pytest.raises(S.SfhkError):
        S.sfhk_create_target(ctx, t)
    t = dict(W.TARGETS["N2_pi"], pi_azimuth=float("nan"))
    with pytest.raises(S.SfhkError):
        S.sfhk_create_target(ctx, t)
    # a pi_u orbital is normalisable at R = 0 (a single-centre 2p)
    S.sfhk_destroy_target(S.sfhk_create_target(ctx, dict(W.TARGETS["N2_pi"], R=0.0)))


@pytest.mark.parametrize("name,pulse,align,n", [
    ("H2", W.PULSE_800, W.fixed(0.0), 1000),
    ("N2", W.PULSE_1200, W.COS2, 600),
    ("H2O", W.PULSE_800, W.ISO, 500),
])
def test_tapered_stability_filter(S, ctx, name, pulse, align, n):
    """The tapered stability filter (weight 1 -> 0 between the cutoff and twice
    it, in the running maximum of |M|): FP64 and mixed dipoles against the
    oracle's, and the FP64 per-trajectory stop status."""
    t = W.TARGETS[name]
    soa, _, _ = O.sample(t, pulse, align, seed=13, n=n)
    vz_o, fin_o, _ = O.propagate(t, pulse, soa, GAMMA, cutoff=CUT, want_final=True,
                                 stab_cutoff=STAB, stab_taper=2.0)
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, pulse)
    e = S.sfhk_load_ensemble(ctx, th, ph, soa)
    nt = S.sfhk_pulse_grid(ph)["nt"]
    for prec, tol in ((S.SFHK_FP64, 1e-9), (S.SFHK_MIXED, 1e-4)):
        S.sfhk_propagate(ctx, e, S.run_opts(prec, GAMMA, CUT, prec == S.SFHK_FP64,
                                            stab_cutoff=STAB, stab_taper=2.0))
        vz = S.sfhk_dipole(ctx, e, nt)
        err = _rel_l2(vz, vz_o)
        print(f"taper {name} prec {prec}: {err:.3e}")
        assert err <= tol
        if prec == S.SFHK_FP64:
            assert np.array_equal(S.sfhk_final_state(e, n)[46], fin_o[46])
    with pytest.raises(S.SfhkError):
        S.sfhk_propagate(ctx, e, S.run_opts(S.SFHK_MIXED, GAMMA, CUT, stab_cutoff=STAB,
                                            stab_taper=0.5))
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)
