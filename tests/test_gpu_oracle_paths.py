"""The CUDA paths that the small parity cases do not reach, against the oracle.

* the small workload itself (H2 at theta = 0, 4096 trajectories, seed 0):
  device sampler end to end, FP64 (dipole 1e-9, per-trajectory state) and
  mixed precision (dipole 1e-4), against the oracle's own sampler and
  propagation of the same draws;
* the persistent work queue with more work items than warps: 10240
  trajectories in 32-thread blocks at one block per SM, so each of the 148
  warps takes two or more items in turn, as every warp does at the
  benchmark's sizes;
* a prepared batch of three uneven mixed-precision ensembles and its CUDA
  graph replay: every ensemble's dipole against the oracle;
* the served requests (continuous batching, the workloads' tapered
  stability filter, one request on another time step so that the slices
  switch between the generic and the fixed-parameter integrator): every
  result against the oracle;
* the benchmark's own workload (1e6 trajectories, autotuned launch shape):
  trajectories drawn at random from the full-size run, their final states
  against the oracle's propagation of each of them alone;
* the non-finite limit (SFHK_E_NUMERIC) on an ensemble in which some
  trajectories overflow, and the dipole of the rest against the oracle;
* the unfiltered FP64 path on an ensemble without prefactor blow-up;
* the integrator compiled with the prescribed dt, gamma and the workloads'
  filters: chosen exactly when every instance has those values, equal to the
  generic integrator on the same ensemble (1e-7) and to the oracle.

Tolerances are those of the other parity tests: relative L2 1e-9 (FP64) and
1e-4 (mixed) for dipoles; |dy| <= 1e-10 max(1, |M|) per FP64 trajectory.
"""
import numpy as np
import pytest

import oracle as O
from paper_2608_13686_b300 import workloads as W

pytestmark = pytest.mark.gpu

GAMMA, CUT, STAB, TAPER = W.GAMMA, W.CUTOFF, W.STAB_CUTOFF, W.STAB_TAPER


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


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _opts(S, prec, **kw):
    return S.run_opts(prec, GAMMA, CUT, stab_cutoff=STAB, stab_taper=TAPER, **kw)


def _compare_final(fin_g, fin_o, tol):
    assert np.array_equal(fin_g[46], fin_o[46])
    M = np.abs(fin_o[6:42]).max(axis=0)
    scale = np.maximum(1.0, M)
    ysc = np.maximum(1.0, np.abs(fin_o[0:43]).max(axis=0))
    err = np.abs(fin_g[0:43] - fin_o[0:43]).max(axis=0) / ysc
    C_g, C_o = fin_g[43] + 1j * fin_g[44], fin_o[43] + 1j * fin_o[44]
    errC = np.abs(C_g - C_o) / np.maximum(1.0, np.abs(C_o))
    ok = (err <= tol * scale) & (errC <= tol * scale ** 1.5)
    assert ok.all(), (np.flatnonzero(~ok)[:10], err[~ok][:5], M[~ok][:5])


# ------------------------------------------------------------------ small workload + queue
N_SMALL, N_QUEUE = 4096, 10240


@pytest.fixture(scope="module")
def h2_oracle():
    """The oracle on H2 theta = 0, seed 0: the first 4096 trajectories (the
    small workload) and the next 6144, each part with its final states.  By
    Philox's per-trajectory counters the first part is also the beginning of
    the 10240-trajectory ensemble."""
    t, p, al = W.TARGETS["H2"], W.PULSE_800, W.fixed(0.0)
    s1, _, _ = O.sample(t, p, al, seed=0, n=N_SMALL)
    s2, _, _ = O.sample(t, p, al, seed=0, j_begin=N_SMALL, n=N_QUEUE - N_SMALL)
    v1, f1, _ = O.propagate(t, p, s1, GAMMA, cutoff=CUT, want_final=True, stab_cutoff=STAB,
                            stab_taper=TAPER)
    v2, f2, _ = O.propagate(t, p, s2, GAMMA, cutoff=CUT, want_final=True, stab_cutoff=STAB,
                            stab_taper=TAPER)
    return dict(soa=np.concatenate([s1, s2], axis=1), vz_small=v1,
                vz_queue=(N_SMALL * v1 + (N_QUEUE - N_SMALL) * v2) / N_QUEUE,
                fin=np.concatenate([f1, f2], axis=1))


def test_small_workload_end_to_end(S, ctx, h2_oracle):
    t, p = W.TARGETS["H2"], W.PULSE_800
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
    nt = S.sfhk_pulse_grid(ph)["nt"]
    e = S.sfhk_sample_initial(ctx, th, ph, W.fixed(0.0), N_SMALL, 0, 0)
    g = S.sfhk_ensemble_read(e, N_SMALL)
    o = h2_oracle["soa"][:, :N_SMALL]
    assert np.array_equal(g[0], o[0])
    assert np.allclose(g[1:10], o[1:10], rtol=0.0, atol=1e-12 * max(1.0, np.abs(o).max()))
    S.sfhk_propagate(ctx, e, _opts(S, S.SFHK_FP64, dump=True))
    vz = S.sfhk_dipole(ctx, e, nt)
    assert _rel(vz, h2_oracle["vz_small"]) <= 1e-9
    _compare_final(S.sfhk_final_state(e, N_SMALL), h2_oracle["fin"][:, :N_SMALL], 1e-10)
    st64 = S.sfhk_stats_get(e)
    S.sfhk_propagate(ctx, e, _opts(S, S.SFHK_MIXED))
    err = _rel(S.sfhk_dipole(ctx, e, nt), h2_oracle["vz_small"])
    print(f"small workload, mixed vs oracle: {err:.3e}")
    assert err <= 1e-4
    # recombination evaluations: at most one per integrated step and birth;
    # FP64 skips an overlap only below e^-200 of its peak, mixed precision
    # below e^-30, so mixed precision evaluates fewer (1 % slack for the
    # trajectories whose paths differ in the last digits)
    st = S.sfhk_stats_get(e)
    for x in (st, st64):
        assert 0 < x["recomb_evals"] <= x["traj_steps"] + N_SMALL
    assert st["recomb_evals"] <= 1.01 * st64["recomb_evals"]
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)


def test_queue_with_several_items_per_warp(S, ctx, h2_oracle):
    """10240 trajectories = 320 work items of 32; one 32-thread block per SM
    is 148 warps, so most warps take a second and third item from the queue."""
    t, p = W.TARGETS["H2"], W.PULSE_800
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
    nt = S.sfhk_pulse_grid(ph)["nt"]
    e = S.sfhk_sample_initial(ctx, th, ph, W.fixed(0.0), N_QUEUE, 0, 0)
    S.sfhk_propagate(ctx, e, _opts(S, S.SFHK_FP64, dump=True, block_threads=32,
                                   blocks_per_sm=1))
    assert _rel(S.sfhk_dipole(ctx, e, nt), h2_oracle["vz_queue"]) <= 1e-9
    _compare_final(S.sfhk_final_state(e, N_QUEUE), h2_oracle["fin"], 1e-10)
    for var in (2, 6):
        S.sfhk_propagate(ctx, e, _opts(S, S.SFHK_MIXED, block_threads=32, blocks_per_sm=1,
                                       kernel_variant=var))
        err = _rel(S.sfhk_dipole(ctx, e, nt), h2_oracle["vz_queue"])
        print(f"queue path, mixed variant {var} vs oracle: {err:.3e}")
        assert err <= 1e-4
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)


# ------------------------------------------------------------------ batch + graph
BATCH = [("H2", W.PULSE_800, W.fixed(20.0), 3000, 1),
         ("N2", W.pulse(1000.0, 1.6e14, 2), W.COS2, 2570, 2),
         ("H2", W.pulse(1400.0, 1.0e14, 4), W.fixed(70.0), 650, 3)]


def test_batch_and_graph_replay_against_oracle(S):
    import torch
    ctx = S.sfhk_create(0, 0)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    handles, ens, grids, ref = [], [], [], []
    for name, p, al, n, seed in BATCH:
        t = W.TARGETS[name]
        th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
        handles += [th, ph]
        ens.append(S.sfhk_sample_initial(ctx, th, ph, al, n, seed, seed, sp))
        grids.append(S.sfhk_pulse_grid(ph))
        soa, _, _ = O.sample(t, p, al, seed=seed, instance=seed, n=n)
        ref.append(O.propagate(t, p, soa, GAMMA, cutoff=CUT, stab_cutoff=STAB,
                               stab_taper=TAPER)[0])
    torch.cuda.synchronize()
    for prec, tol in ((S.SFHK_MIXED, 1e-4), (S.SFHK_FP64, 1e-9)):
        b = S.sfhk_batch_create(ctx, ens, _opts(S, prec))
        S.sfhk_batch_launch(b, sp)
        torch.cuda.synchronize()
        for e, g, r in zip(ens, grids, ref):
            err = _rel(S.sfhk_dipole(ctx, e, g["nt"]), r)
            print(f"batch precision {prec}: {err:.3e}")
            assert err <= tol
        graph = torch.cuda.CUDAGraph()

        def step():
            for (name, p, al, n, seed), e in zip(BATCH, ens):
                S.sfhk_sample_into(ctx, e, al, seed, seed, sp)
            S.sfhk_batch_launch(b, sp)

        with torch.cuda.stream(stream):
            step()                       # warm-up outside the capture
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            step()
        for _ in range(2):
            graph.replay()
            torch.cuda.synchronize()
            for e, g, r in zip(ens, grids, ref):
                assert _rel(S.sfhk_dipole(ctx, e, g["nt"]), r) <= tol
        del graph
        S.sfhk_batch_destroy(b)
    for e in ens:
        S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy(ctx)


# ------------------------------------------------------------------ served requests
MIX = [("H2", W.PULSE_800, W.fixed(10.0), 3000, 1),
       ("N2", W.pulse(1000.0, 1.6e14, 2), W.COS2, 2500, 2),
       ("H2", W.pulse(1400.0, 1.0e14, 4), W.fixed(70.0), 700, 3),
       ("N2", W.PULSE_1200, W.fixed(40.0), 4100, 4),
       ("H2", W.pulse(900.0, 1.9e14, 3), W.COS2, 33, 5),
       ("N2_sp", W.PULSE_1200, W.ISO, 900, 6),
       ("N2_pi", W.pulse(1000.0, 1.4e14, 3), W.fixed(60.0), 600, 7),
       # another time step: while it is served the slices run the generic
       # integrator, the others the one compiled with the fixed parameters
       ("H2", dict(W.PULSE_800, dt=0.04), W.fixed(20.0), 800, 8)]


@pytest.fixture(scope="module")
def mix_oracle():
    out = []
    for name, p, al, n, inst in MIX:
        t = W.TARGETS[name]
        soa, _, _ = O.sample(t, p, al, seed=7, instance=inst, n=n)
        out.append(O.propagate(t, p, soa, GAMMA, cutoff=CUT, stab_cutoff=STAB,
                               stab_taper=TAPER)[0])
    return out


@pytest.mark.parametrize("prec_name,tol", [("FP64", 1e-9), ("MIXED", 1e-4)])
def test_served_requests_against_oracle(S, mix_oracle, prec_name, tol):
    prec = getattr(S, "SFHK_" + prec_name)
    srv = S.sfhk_server_create(0, S.server_opts(prec, GAMMA, CUT, STAB, slice_ms=5.0,
                                                stab_taper=TAPER))
    ids = [S.sfhk_submit(srv, S.request(W.TARGETS[nm], p, al, n, 7, inst))
           for nm, p, al, n, inst in MIX]
    res = [S.sfhk_wait(srv, i, 300.0) for i in ids]
    st = S.sfhk_server_stats_get(srv)
    S.sfhk_server_destroy(srv)
    assert st["completed"] == len(MIX) and st["failed"] == 0
    for (nm, p, al, n, inst), r, ref in zip(MIX, res, mix_oracle):
        assert r["status"] == S.SFHK_OK
        err = _rel(r["vz"], ref)
        print(f"served {nm} n={n} precision {prec_name}: {err:.3e}")
        assert err <= tol, (nm, n)


# ------------------------------------------------------------------ full size, sampled
def test_full_size_run_sampled_trajectories(S, ctx):
    """The benchmark's workload at one angle: 1e6 trajectories sampled on the
    device, the launch shape chosen by the autotuner, final states of all
    trajectories kept.  48 trajectories drawn at random are propagated by the
    oracle one by one from their own draws; their birth, initial point, stop
    status and final state must match (FP64 as in the other parity tests;
    mixed precision: status and a loose state bound, the FP32 state error
    being about 1e-5)."""
    t, p, al, n = W.TARGETS["H2"], W.PULSE_800, W.fixed(45.0), 1_000_000
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
    e = S.sfhk_sample_initial(ctx, th, ph, al, n, 0, 1)
    S.sfhk_autotune(ctx, e, _opts(S, S.SFHK_MIXED))
    soa_g = S.sfhk_ensemble_read(e, n)
    rng = np.random.default_rng(5)
    js = np.sort(rng.choice(n, 48, replace=False))
    o = np.concatenate([O.sample(t, p, al, seed=0, instance=1, j_begin=int(j), n=1)[0]
                        for j in js], axis=1)
    assert np.array_equal(soa_g[0, js], o[0])
    assert np.allclose(soa_g[1:10, js], o[1:10], rtol=0.0, atol=1e-12 * max(1.0, np.abs(o).max()))
    fin_o = np.concatenate([O.propagate(t, p, o[:, k:k + 1], GAMMA, cutoff=CUT,
                                        want_final=True, stab_cutoff=STAB,
                                        stab_taper=TAPER)[1] for k in range(len(js))], axis=1)
    S.sfhk_propagate(ctx, e, _opts(S, S.SFHK_FP64, dump=True))
    _compare_final(S.sfhk_final_state(e, n)[:, js], fin_o, 1e-10)
    S.sfhk_propagate(ctx, e, _opts(S, S.SFHK_MIXED, dump=True))
    fin_m = S.sfhk_final_state(e, n)[:, js]
    same = fin_m[46] == fin_o[46]
    assert same.mean() >= 0.95
    ysc = np.maximum(1.0, np.abs(fin_o[0:6]).max(axis=0))
    M = np.maximum(1.0, np.abs(fin_o[6:42]).max(axis=0))
    err = np.abs(fin_m[0:6] - fin_o[0:6]).max(axis=0) / ysc
    print("mixed final q,p error, sampled: max %.2e median %.2e" % (err[same].max(),
                                                                  np.median(err[same])))
    assert np.all(err[same] <= 1e-3 * M[same])
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)


# ------------------------------------------------------------------ non-finite limit
def _limits(S, ctx, e, nt, prec, n_bad):
    """With the limit at n_bad the calls succeed; one below, sfhk_dipole and
    sfhk_stats_get return SFHK_E_NUMERIC (the stats still carry the count)."""
    S.sfhk_propagate(ctx, e, _opts(S, prec, max_nonfinite=n_bad))
    assert S.sfhk_stats_get(e)["n_nonfinite"] == n_bad
    S.sfhk_dipole(ctx, e, nt)
    if n_bad == 0:
        return
    S.sfhk_propagate(ctx, e, _opts(S, prec, max_nonfinite=n_bad - 1))
    with pytest.raises(S.SfhkError) as err:
        S.sfhk_dipole(ctx, e, nt)
    assert err.value.code == S.SFHK_E_NUMERIC
    with pytest.raises(S.SfhkError) as err:
        S.sfhk_stats_get(e)
    assert err.value.code == S.SFHK_E_NUMERIC and err.value.stats["n_nonfinite"] == n_bad


def test_nonfinite_limit_on_fp32_momentum_overflow(S, ctx):
    """Five trajectories start with p_x = 1e20: finite in both precisions, but
    |p|^2 = 1e40 overflows FP32, so in mixed precision their action becomes
    infinite at the first step and they stop as non-finite, while FP64 runs
    them to the end (the oracle does too; their recombination element is
    zero, e^{-|p|^2/...}).  Both dipoles agree with the oracle's."""
    t, p = W.TARGETS["H2"], W.PULSE_800
    soa, _, _ = O.sample(t, p, W.fixed(30.0), seed=3, n=64)
    bad = [3, 17, 18, 40, 63]
    soa[4, bad] = 1e20
    vz_o, fin_o, _ = O.propagate(t, p, soa, GAMMA, cutoff=CUT, want_final=True,
                                 stab_cutoff=STAB, stab_taper=TAPER)
    assert np.all(fin_o[46, bad] == 0)
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
    nt = S.sfhk_pulse_grid(ph)["nt"]
    e = S.sfhk_load_ensemble(ctx, th, ph, soa)
    for prec, tol, n_bad in ((S.SFHK_FP64, 1e-9, 0), (S.SFHK_MIXED, 1e-4, len(bad))):
        S.sfhk_propagate(ctx, e, _opts(S, prec))
        assert S.sfhk_stats_get(e)["n_nonfinite"] == n_bad
        assert _rel(S.sfhk_dipole(ctx, e, nt), vz_o) <= tol
        _limits(S, ctx, e, nt, prec, n_bad)
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)


def test_nonfinite_limit_on_an_overflowing_potential(S, ctx):
    """A target whose near-nucleus charge is 1e300 drives every trajectory to
    a non-finite state at its first step, in either precision (FP64: |p|^2
    overflows; FP32: the charge itself does).  Each trajectory then
    contributes only at its birth, before any step; that dipole agrees with
    the oracle's, and the limit turns the count into SFHK_E_NUMERIC."""
    wild = dict(W.TARGETS["N2"], Z0=1e300)
    p = W.PULSE_800
    soa, _, _ = O.sample(wild, p, W.fixed(0.0), seed=1, n=32)
    vz_o, fin_o, _ = O.propagate(wild, p, soa, GAMMA, want_final=True)
    assert np.all(fin_o[46] == 2)
    th, ph = S.sfhk_create_target(ctx, wild), S.sfhk_set_pulse(ctx, p)
    nt = S.sfhk_pulse_grid(ph)["nt"]
    e = S.sfhk_load_ensemble(ctx, th, ph, soa)
    for prec, tol in ((S.SFHK_FP64, 1e-9), (S.SFHK_MIXED, 1e-4)):
        S.sfhk_propagate(ctx, e, S.run_opts(prec, GAMMA))
        assert S.sfhk_stats_get(e)["n_nonfinite"] == 32
        assert _rel(S.sfhk_dipole(ctx, e, nt), vz_o) <= tol
        _limits(S, ctx, e, nt, prec, 32)
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)


def test_server_request_over_the_nonfinite_limit(S):
    """A request whose target has a near-nucleus charge of 1e300 overflows in
    every trajectory within its first steps; with a limit the server ends it
    with SFHK_E_NUMERIC, and keeps serving."""
    srv = S.sfhk_server_create(0, S.server_opts(S.SFHK_FP64, GAMMA, 0.0, 0.0, slice_ms=5.0,
                                                max_nonfinite=10))
    wild = dict(W.TARGETS["N2"], Z0=1e300)
    rid = S.sfhk_submit(srv, S.request(wild, W.PULSE_800, W.fixed(0.0), 200, 1, 0))
    r = S.sfhk_wait(srv, rid, 300.0)
    assert r["status"] == S.SFHK_E_NUMERIC and r["n_nonfinite"] > 10
    ok = S.sfhk_submit(srv, S.request(W.TARGETS["H2"], W.PULSE_800, W.fixed(0.0), 200, 1, 1))
    r2 = S.sfhk_wait(srv, ok, 300.0)
    assert r2["status"] == S.SFHK_OK and r2["n_nonfinite"] <= 10
    S.sfhk_server_destroy(srv)


# ------------------------------------------------------------------ unfiltered FP64
def test_unfiltered_fp64_on_an_ensemble_without_blowup(S, ctx):
    """Without any filter (the library default) the FP64 dipole agrees with
    the oracle's at 1e-9 on an ensemble whose trajectories all keep
    max |M| <= 1e3 (picked by the oracle with the hard stability filter: those
    it never stopped).  The filters therefore play no part in this parity;
    they only decide which chaotic trajectories count."""
    t, p = W.TARGETS["H2"], W.PULSE_800
    soa, _, _ = O.sample(t, p, W.fixed(45.0), seed=19, n=1500)
    _, fin, _ = O.propagate(t, p, soa, GAMMA, cutoff=CUT, want_final=True, stab_cutoff=STAB)
    tame = np.ascontiguousarray(soa[:, fin[46] == 0])
    assert tame.shape[1] > 1200
    vz_o, fin_o, bad = O.propagate(t, p, tame, GAMMA, want_final=True)
    assert bad == 0
    th, ph = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p)
    e = S.sfhk_load_ensemble(ctx, th, ph, tame)
    S.sfhk_propagate(ctx, e, S.run_opts(S.SFHK_FP64, GAMMA, 0.0, True))
    vz = S.sfhk_dipole(ctx, e, S.sfhk_pulse_grid(ph)["nt"])
    assert _rel(vz, vz_o) <= 1e-9
    _compare_final(S.sfhk_final_state(e, tame.shape[1]), fin_o, 1e-10)
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)


def test_fixed_parameter_integrator(S, ctx):
    """The mixed integrator compiled with dt = 0.05, gamma = 0.5 and the
    workloads' filters as constants runs exactly when every instance of a
    launch has those values, and gives the generic integrator's dipole: an H2
    ensemble propagated alone (specialised), in a batch with an ensemble on
    another time step (generic for the whole launch), and with the hard
    stability filter (generic), against each other and the oracle."""
    t = W.TARGETS["H2"]
    p, p2 = W.PULSE_800, dict(W.PULSE_800, dt=0.04)
    th, ph, ph2 = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p), S.sfhk_set_pulse(ctx, p2)
    nt = S.sfhk_pulse_grid(ph)["nt"]
    e = S.sfhk_sample_initial(ctx, th, ph, W.fixed(30.0), 3000, 5, 0)
    e2 = S.sfhk_sample_initial(ctx, th, ph2, W.fixed(30.0), 300, 6, 0)
    tapered = S.run_opts(S.SFHK_MIXED, GAMMA, CUT, stab_cutoff=STAB, stab_taper=TAPER)
    S.sfhk_propagate(ctx, e, tapered)
    assert S.sfhk_stats_get(e)["fixed_params"] == 1
    v_fixed = S.sfhk_dipole(ctx, e, nt)
    S.sfhk_propagate_batch(ctx, [e, e2], tapered)
    assert S.sfhk_stats_get(e)["fixed_params"] == 0
    v_generic = S.sfhk_dipole(ctx, e, nt)
    assert _rel(v_fixed, v_generic) <= 1e-7
    S.sfhk_propagate_batch(ctx, [e], tapered)
    assert S.sfhk_stats_get(e)["fixed_params"] == 1
    S.sfhk_propagate(ctx, e, S.run_opts(S.SFHK_MIXED, GAMMA, CUT, stab_cutoff=STAB))
    assert S.sfhk_stats_get(e)["fixed_params"] == 0
    # a launch that records first returns runs the generic integrator
    S.sfhk_propagate(ctx, e, S.run_opts(S.SFHK_MIXED, GAMMA, CUT, stab_cutoff=STAB,
                                        stab_taper=TAPER, returns=(5.0, 2.0)))
    assert S.sfhk_stats_get(e)["fixed_params"] == 0
    S.sfhk_propagate(ctx, e, S.run_opts(S.SFHK_FP64, GAMMA, CUT, stab_cutoff=STAB,
                                        stab_taper=TAPER))
    assert S.sfhk_stats_get(e)["fixed_params"] == 0
    soa, _, _ = O.sample(t, p, W.fixed(30.0), seed=5, n=3000)      # the same draws
    vz_o, _, _ = O.propagate(t, p, soa, GAMMA, cutoff=CUT, stab_cutoff=STAB, stab_taper=TAPER)
    assert _rel(v_fixed, vz_o) <= 1e-4
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_ensemble(e2)


def test_fixed_parameter_three_centre_integrator(S, ctx):
    """The same for the three-centre polyatomic integrator: H2O 1b1 at fixed
    Euler angles, specialised alone, generic in a batch with an ensemble on
    another time step; equal to each other (1e-7) and to the oracle (1e-4)."""
    t = W.TARGETS["H2O"]
    p, p2 = W.PULSE_800, dict(W.PULSE_800, dt=0.04)
    th, ph, ph2 = S.sfhk_create_target(ctx, t), S.sfhk_set_pulse(ctx, p), S.sfhk_set_pulse(ctx, p2)
    nt = S.sfhk_pulse_grid(ph)["nt"]
    al = W.fixed(63.0, 23.0, 40.0)
    e = S.sfhk_sample_initial(ctx, th, ph, al, 2000, 7, 0)
    e2 = S.sfhk_sample_initial(ctx, th, ph2, al, 200, 8, 0)
    tapered = S.run_opts(S.SFHK_MIXED, GAMMA, CUT, stab_cutoff=STAB, stab_taper=TAPER)
    S.sfhk_propagate(ctx, e, tapered)
    assert S.sfhk_stats_get(e)["fixed_params"] == 1
    v_fixed = S.sfhk_dipole(ctx, e, nt)
    S.sfhk_propagate_batch(ctx, [e, e2], tapered)
    assert S.sfhk_stats_get(e)["fixed_params"] == 0
    v_generic = S.sfhk_dipole(ctx, e, nt)
    assert _rel(v_fixed, v_generic) <= 1e-7
    soa, _, _ = O.sample(t, p, al, seed=7, n=2000)
    vz_o, _, _ = O.propagate(t, p, soa, GAMMA, cutoff=CUT, stab_cutoff=STAB, stab_taper=TAPER)
    assert _rel(v_fixed, vz_o) <= 1e-4
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_ensemble(e2)


def test_fixed_parameter_integrator_potential_forms(S, ctx):
    """The fixed-parameter integrator comes in three forms of the two-centre
    potential, chosen from the launch's instances: unscreened (H2 alone),
    screened (N2 alone) and the screening decided per instance (H2 and N2 in
    one batch).  Each gives the generic integrator's dipoles on the same
    ensembles (the generic one forced by an extra ensemble on another time
    step) to 1e-7, and the N2 dipole agrees with the oracle."""
    p, p2 = W.PULSE_800, dict(W.PULSE_800, dt=0.04)
    th2, tn2 = S.sfhk_create_target(ctx, W.TARGETS["H2"]), S.sfhk_create_target(ctx, W.TARGETS["N2"])
    ph, ph2 = S.sfhk_set_pulse(ctx, p), S.sfhk_set_pulse(ctx, p2)
    nt = S.sfhk_pulse_grid(ph)["nt"]
    eh = S.sfhk_sample_initial(ctx, th2, ph, W.fixed(20.0), 2000, 9, 0)
    en = S.sfhk_sample_initial(ctx, tn2, ph, W.COS2, 2000, 10, 0)
    ex = S.sfhk_sample_initial(ctx, th2, ph2, W.fixed(20.0), 200, 11, 0)
    tapered = S.run_opts(S.SFHK_MIXED, GAMMA, CUT, stab_cutoff=STAB, stab_taper=TAPER)

    def dipoles(batch, keep):
        S.sfhk_propagate_batch(ctx, batch, tapered)
        return [S.sfhk_dipole(ctx, e, nt) for e in keep], S.sfhk_stats_get(keep[0])["fixed_params"]

    for batch in ([eh], [en], [eh, en]):
        v_fixed, f1 = dipoles(batch, batch)
        v_gen, f0 = dipoles(batch + [ex], batch)
        assert f1 == 1 and f0 == 0
        for a, b in zip(v_fixed, v_gen):
            assert _rel(a, b) <= 1e-7
    soa, _, _ = O.sample(W.TARGETS["N2"], p, W.COS2, seed=10, n=2000)
    vz_o, _, _ = O.propagate(W.TARGETS["N2"], p, soa, GAMMA, cutoff=CUT, stab_cutoff=STAB,
                             stab_taper=TAPER)
    S.sfhk_propagate(ctx, en, tapered)
    assert _rel(S.sfhk_dipole(ctx, en, nt), vz_o) <= 1e-4
    for e in (eh, en, ex):
        S.sfhk_destroy_ensemble(e)
