"""Polyatomic targets on the GPU (the N-centre generalisation of Eq. 7, the
full Euler-angle orientation of Eq. 6, primitives on their own centres),
through the C ABI, against the FP64 oracle.  Tolerances as in the diatomic
parity tests: sampler 1e-12 (points) and 1e-10 (weights), FP64 propagation
1e-10 x max(1, |M|) per trajectory and 1e-9 on the dipole, mixed precision
1e-4 on the dipole."""
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


def _target(name):
    if name.endswith("+abs"):
        return W.abs_sampled(_target(name[:-4]), 5.0)
    if name.startswith("asPoly:"):
        return W.diatomic_as_poly(W.TARGETS[name[7:]])
    return W.TARGETS[name]


@pytest.mark.parametrize("name,pulse,align,n,seed,inst", [
    ("H2O", W.PULSE_800, W.ISO, 700, 21, 0),
    ("H2O_3a1", W.PULSE_800, W.fixed(40.0, 20.0, 70.0), 500, 22, 1),
    ("H2O_3a1", W.PULSE_1200, W.COS2, 500, 23, 2),
    ("H2O+abs", W.PULSE_800, W.ISO, 400, 24, 0),
    ("asPoly:N2_sp", W.PULSE_1200, W.ISO, 600, 25, 3),
])
def test_sampler_matches_oracle(S, ctx, name, pulse, align, n, seed, inst):
    t = _target(name)
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, pulse)
    e = S.sfhk_sample_initial(ctx, th, ph, align, n, seed, inst)
    g = S.sfhk_ensemble_read(e, n)
    o, _, bad = O.sample(t, pulse, align, seed=seed, instance=inst, n=n)
    assert np.array_equal(g[0], o[0])
    for f in range(1, 10):
        sc = max(1.0, np.abs(o[f]).max())
        assert np.max(np.abs(g[f] - o[f])) <= 1e-12 * sc, f
    w_g, w_o = g[10] + 1j * g[11], o[10] + 1j * o[11]
    assert np.all(np.abs(w_g - w_o) <= 1e-10 * np.abs(w_o) + 1e-300)
    assert S.sfhk_stats_get(e)["n_invalid"] == bad
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)


def _run(S, ctx, t, p, soa, precision, dump=True):
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
    e = S.sfhk_load_ensemble(ctx, th, ph, soa)
    S.sfhk_propagate(ctx, e, S.run_opts(precision, GAMMA, CUT, dump, stab_cutoff=STAB))
    vz = S.sfhk_dipole(ctx, e, S.sfhk_pulse_grid(ph)["nt"])
    fin = S.sfhk_final_state(e, soa.shape[1]) if dump else None
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)
    return vz, fin


@pytest.mark.parametrize("name,pulse,align,n", [
    ("H2O", W.PULSE_800, W.ISO, 400),
    ("H2O_3a1", W.PULSE_800, W.fixed(60.0, 10.0, 30.0), 300),
    ("asPoly:N2", W.PULSE_1200, W.COS2, 300),
])
def test_fp64_propagation_per_trajectory_and_dipole(S, ctx, name, pulse, align, n):
    t = _target(name)
    soa, _, _ = O.sample(t, pulse, align, seed=31, n=n)
    vz_o, fin_o, _ = O.propagate(t, pulse, soa, GAMMA, cutoff=CUT, want_final=True,
                                 stab_cutoff=STAB)
    vz_g, fin_g = _run(S, ctx, t, pulse, soa, S.SFHK_FP64)
    assert np.array_equal(fin_g[46], fin_o[46])
    M = np.abs(fin_o[6:42]).max(axis=0)
    ysc = np.maximum(1.0, np.abs(fin_o[0:43]).max(axis=0))
    err = np.abs(fin_g[0:43] - fin_o[0:43]).max(axis=0) / ysc
    assert np.all(err <= 1e-10 * np.maximum(1.0, M)), err.max()
    assert _rel_l2(vz_g, vz_o) <= 1e-9


@pytest.mark.parametrize("name,pulse,align,n", [
    ("H2O", W.PULSE_800, W.ISO, 500),
    ("H2O_3a1", W.PULSE_800, W.ISO, 500),
])
def test_mixed_precision_dipole(S, ctx, name, pulse, align, n):
    t = _target(name)
    soa, _, _ = O.sample(t, pulse, align, seed=32, n=n)
    vz_o, _, _ = O.propagate(t, pulse, soa, GAMMA, cutoff=CUT, stab_cutoff=STAB)
    vz_g, _ = _run(S, ctx, t, pulse, soa, S.SFHK_MIXED, dump=False)
    err = _rel_l2(vz_g, vz_o)
    print(f"mixed rel-L2 {name}: {err:.3e}")
    assert err <= 1e-4


def test_diatomic_as_polyatomic_matches_the_diatomic_kernel(S, ctx):
    """The same molecule through both kernels: sampled with the same draws,
    the two-centre polyatomic and the diatomic give the same dipole."""
    t = W.TARGETS["N2"]
    tp = W.diatomic_as_poly(t)
    p = W.PULSE_1200
    out = []
    for tt in (t, tp):
        th, ph = S.sfhk_create_target(ctx, tt), S.sfhk_set_pulse(ctx, p)
        e = S.sfhk_sample_initial(ctx, th, ph, W.ISO, 2000, 7, 0)
        for prec in (S.SFHK_FP64, S.SFHK_MIXED):
            S.sfhk_propagate(ctx, e, S.run_opts(prec, GAMMA, CUT, stab_cutoff=STAB))
            out.append(S.sfhk_dipole(ctx, e, S.sfhk_pulse_grid(ph)["nt"]))
        S.sfhk_destroy_ensemble(e)
        S.sfhk_destroy_pulse(ph)
        S.sfhk_destroy_target(th)
    assert _rel_l2(out[2], out[0]) <= 1e-9
    assert _rel_l2(out[3], out[1]) <= 1e-4


def test_batch_of_polyatomic_ensembles(S, ctx):
    cases = [("H2O", W.PULSE_800, W.ISO, 200, 1), ("H2O_3a1", W.pulse(1000.0, 1.4e14, 2),
                                                   W.COS2, 150, 2)]
    hs, ens, nts = [], [], []
    for name, p, al, n, seed in cases:
        th, ph = S.sfhk_create_target(ctx, W.TARGETS[name]), S.sfhk_set_pulse(ctx, p)
        hs += [th, ph]
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
            assert _rel_l2(S.sfhk_dipole(ctx, e, nt), a) <= 1e-12
    # a batch may not mix polyatomic and diatomic targets
    thd, phd = S.sfhk_create_target(ctx, W.TARGETS["H2"]), S.sfhk_set_pulse(ctx, W.PULSE_800)
    ed = S.sfhk_sample_initial(ctx, thd, phd, W.ISO, 64, 0, 0)
    with pytest.raises(S.SfhkError):
        S.sfhk_propagate_batch(ctx, [ens[0], ed], S.run_opts(S.SFHK_MIXED, GAMMA, CUT))
    for e in ens + [ed]:
        S.sfhk_destroy_ensemble(e)


def test_batch_mixing_centre_counts_uses_the_generic_kernel(S, ctx):
    """H2O (three centres: alone it runs the kernel unrolled for three
    centres) batched with N2 written as a two-centre polyatomic: the batch
    runs the kernel for any number of centres, and each dipole equals the
    one of its ensemble alone (FP64 to the oracle's tolerance, the two
    kernels summing the centres in a different order; mixed precision to
    1e-5)."""
    cases = [(W.TARGETS["H2O"], W.PULSE_800, W.ISO, 300, 1),
             (W.diatomic_as_poly(W.TARGETS["N2"]), W.pulse(1000.0, 1.4e14, 2), W.COS2, 200, 2)]
    hs, ens, nts = [], [], []
    for t, p, al, n, seed in cases:
        th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
        hs += [th, ph]
        ens.append(S.sfhk_sample_initial(ctx, th, ph, al, n, seed, seed))
        nts.append(S.sfhk_pulse_grid(ph)["nt"])
    for prec, tol in ((S.SFHK_FP64, 1e-9), (S.SFHK_MIXED, 1e-5)):
        opts = S.run_opts(prec, GAMMA, CUT, stab_cutoff=STAB, stab_taper=W.STAB_TAPER)
        alone = []
        for e, nt in zip(ens, nts):
            S.sfhk_propagate(ctx, e, opts)
            alone.append(S.sfhk_dipole(ctx, e, nt))
        S.sfhk_propagate_batch(ctx, ens, opts)
        for e, nt, a in zip(ens, nts, alone):
            assert _rel_l2(S.sfhk_dipole(ctx, e, nt), a) <= tol, prec
    for e in ens:
        S.sfhk_destroy_ensemble(e)


def test_polyatomic_validation(S, ctx):
    t = W.TARGETS["H2O_3a1"]
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, W.PULSE_800)
    with pytest.raises(S.SfhkError):          # quadrature rests on the diatomic's symmetry
        S.sfhk_sample_initial(ctx, th, ph, W.quadrature(4), 64, 0, 0)
    for bad in (dict(t, ionization=1),                         # SFHK2 is diatomic only
                dict(t, pcentre=[0, 0, 3, 2]),                  # no centre 3
                dict(t, pdir=[(0.0, 0.0, 0.0)] * 4),            # zero p direction
                dict(t, centres=[]),                            # no centres
                dict(t, pkind=[1, 1, 0, 0])):                   # sigma p-type needs a diatomic
        with pytest.raises(S.SfhkError):
            S.sfhk_create_target(ctx, bad)
    with pytest.raises(S.SfhkError):          # p along a direction needs a polyatomic target
        S.sfhk_create_target(ctx, dict(W.TARGETS["N2"], pkind=[3, 0]))
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)


def _eight_centre_target():
    """Eight centres on a distorted cube, eight p-type primitives (one per
    centre, directions not normalised): the largest table (16 rows per lane)."""
    rng = np.random.default_rng(5)
    cen = []
    for k in range(8):
        x = np.array([(k & 1) * 2.0 - 1.0, ((k >> 1) & 1) * 2.0 - 1.0, ((k >> 2) & 1) * 2.0 - 1.0])
        x = 1.6 * x + 0.1 * rng.normal(size=3)
        cen.append((*x, 1.0 / 8.0, 1.0 + 0.25 * (k % 3), 1.0))
    prims = [(k, 0.6 + 0.1 * k, 0.3 + 0.05 * k, tuple(rng.normal(size=3) * 2.0)) for k in range(8)]
    return W._poly(cen, 0.5, prims)


def test_largest_polyatomic_target(S, ctx):
    """SFHK_MAX_CENTRES centres and SFHK_MAX_PRIM p-type primitives, in
    128-thread blocks: the FP64 kernel then needs more than 48 KB of dynamic
    shared memory (the opt-in path).  Sampler, FP64 and mixed dipoles against
    the oracle."""
    t = _eight_centre_target()
    p = W.PULSE_800
    n = 256
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
    e = S.sfhk_sample_initial(ctx, th, ph, W.ISO, n, 3, 0)
    g = S.sfhk_ensemble_read(e, n)
    o, _, _ = O.sample(t, p, W.ISO, seed=3, n=n)
    assert np.array_equal(g[0], o[0])
    w_g, w_o = g[10] + 1j * g[11], o[10] + 1j * o[11]
    assert np.all(np.abs(w_g - w_o) <= 1e-10 * np.abs(w_o) + 1e-300)
    vz_o, _, _ = O.propagate(t, p, o, GAMMA, cutoff=CUT, stab_cutoff=STAB,
                             stab_taper=W.STAB_TAPER)
    nt = S.sfhk_pulse_grid(ph)["nt"]
    for prec, tol in ((S.SFHK_FP64, 1e-9), (S.SFHK_MIXED, 1e-4)):
        S.sfhk_propagate(ctx, e, S.run_opts(prec, GAMMA, CUT, block_threads=128,
                                            stab_cutoff=STAB, stab_taper=W.STAB_TAPER))
        assert _rel_l2(S.sfhk_dipole(ctx, e, nt), vz_o) <= tol, prec
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)
