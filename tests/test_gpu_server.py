"""The continuous-batching server (sfhk_server_* / sfhk_submit / sfhk_poll).

* every request's result equals the same request run alone through
  sfhk_sample_initial + sfhk_propagate (FP64: to the rounding of the
  reduction order; mixed precision: 1e-5, the slice kernel being a separate
  compilation of the same integrator);
* requests that arrive while another one is running join the running work
  (admitted before the long one ends) and finish first when they are short,
  unless a request admitted earlier has waited longer than the age limit;
* with an admission horizon, a burst waits in the pending queue and is
  admitted as the queued work drains;
* admission follows the device-memory budget; a request larger than the
  budget is refused at submission; cancellation ends a request.
"""
import time

import numpy as np
import pytest

from paper_2608_13686_b300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2608_13686_b300 import _build
    _build.build()
    from paper_2608_13686_b300 import sfhk
    return sfhk


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


MIX = [("H2", W.PULSE_800, W.fixed(10.0), 3000, 1),
       ("N2", W.pulse(1000.0, 1.6e14, 2), W.COS2, 2500, 2),
       ("H2", W.pulse(1400.0, 1.0e14, 4), W.fixed(70.0), 700, 3),
       ("N2", W.PULSE_1200, W.fixed(40.0), 4100, 4),
       ("H2", W.pulse(900.0, 1.9e14, 3), W.COS2, 33, 5),
       ("N2_sp", W.PULSE_1200, W.ISO, 900, 6),
       ("N2_pi", W.pulse(1000.0, 1.4e14, 3), W.fixed(60.0), 600, 7)]


def _alone(S, ctx, name, pulse, align, n, inst, prec):
    th, ph = S.sfhk_create_target(ctx, W.TARGETS[name]), S.sfhk_set_pulse(ctx, pulse)
    e = S.sfhk_sample_initial(ctx, th, ph, align, n, 7, inst)
    S.sfhk_propagate(ctx, e, S.run_opts(prec, W.GAMMA, W.CUTOFF, stab_cutoff=W.STAB_CUTOFF))
    vz = S.sfhk_dipole(ctx, e, S.sfhk_pulse_grid(ph)["nt"])
    st = S.sfhk_stats_get(e)
    S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy_pulse(ph)
    S.sfhk_destroy_target(th)
    return vz, st


@pytest.mark.parametrize("prec_name,tol,slice_ms", [("FP64", 1e-12, 5.0), ("MIXED", 1e-5, 5.0),
                                                    ("FP64", 1e-12, 0.5), ("MIXED", 1e-5, 0.5)])
def test_results_in_the_mix_equal_alone(S, prec_name, tol, slice_ms):
    """With 0.5 ms slices nearly every item is parked at a chunk boundary and
    resumed by the next slice many times over; the results do not change."""
    prec = getattr(S, "SFHK_" + prec_name)
    srv = S.sfhk_server_create(0, S.server_opts(prec, W.GAMMA, W.CUTOFF, W.STAB_CUTOFF,
                                                slice_ms=slice_ms))
    ids = [S.sfhk_submit(srv, S.request(W.TARGETS[nm], p, al, n, 7, inst))
           for nm, p, al, n, inst in MIX]
    res = [S.sfhk_wait(srv, i, 300.0) for i in ids]
    st = S.sfhk_server_stats_get(srv)
    S.sfhk_server_destroy(srv)
    assert st["completed"] == len(MIX) and st["failed"] == 0
    if slice_ms < 1.0:          # more parkings than work items
        assert st["parked"] > sum(-(-n // 32) for _, _, _, n, _ in MIX)
    ctx = S.sfhk_create(0, 0)
    for (nm, p, al, n, inst), r in zip(MIX, res):
        assert r["status"] == S.SFHK_OK
        ref, st_alone = _alone(S, ctx, nm, p, al, n, inst, prec)
        assert r["nt"] == len(ref)
        assert _rel(r["vz"], ref) <= tol, (nm, n)
        # the same trajectory-steps and recombination evaluations as alone
        # (mixed precision: a separately compiled kernel may stop a chaotic
        # trajectory a step apart)
        for key in ("traj_steps", "recomb_evals"):
            if prec == S.SFHK_FP64:
                assert r[key] == st_alone[key], key
            else:
                assert abs(r[key] - st_alone[key]) <= 1e-3 * st_alone[key], key
        # the server's spectrum is the spectrum of its dipole
        om, y, ph = S.sfhk_spectrum(r["vz"], r["dt"], r["t_origin"], -r["t_origin"],
                                    r["nt"] // 2)
        assert np.max(np.abs(r["yield_"] - y)) <= 1e-10 * max(y.max(), 1e-300)
        assert r["t_submit"] <= r["t_admit"] <= r["t_done"]
        assert r["traj_steps"] > 0
    S.sfhk_destroy(ctx)


def test_short_request_joins_a_running_long_one(S):
    """Short-first admission (the default): a short request submitted while a
    long one runs is put in front of the long one's queued work items and
    finishes first; with fifo it waits behind them."""
    srv = S.sfhk_server_create(0, S.server_opts(S.SFHK_MIXED, W.GAMMA, W.CUTOFF, W.STAB_CUTOFF,
                                                slice_ms=10.0))
    long_id = S.sfhk_submit(srv, S.request(W.TARGETS["N2"], W.pulse(1600.0, 1.0e14, 4), W.COS2,
                                           1_000_000, 1, 0))
    t0 = time.time()
    while S.sfhk_server_stats_get(srv)["active"] < 1 and time.time() - t0 < 60:
        time.sleep(0.005)
    short_id = S.sfhk_submit(srv, S.request(W.TARGETS["H2"], W.PULSE_800, W.fixed(0.0), 2000,
                                            1, 1))
    short = S.sfhk_wait(srv, short_id, 300.0)
    long = S.sfhk_wait(srv, long_id, 300.0)
    S.sfhk_server_destroy(srv)
    assert short["status"] == S.SFHK_OK and long["status"] == S.SFHK_OK
    assert short["t_admit"] < long["t_done"]      # admitted while the long one ran
    assert short["t_done"] < long["t_done"]       # and finished first
    assert long["t_done"] - short["t_done"] > 0.3 * (long["t_done"] - long["t_admit"])


def test_age_limit_bounds_reordering(S):
    """With an age limit on short-first, a short request submitted after a long
    one has been admitted for longer than the limit goes to the tail: it no
    longer finishes well before the long one (compare the test above)."""
    srv = S.sfhk_server_create(0, S.server_opts(S.SFHK_MIXED, W.GAMMA, W.CUTOFF, W.STAB_CUTOFF,
                                                slice_ms=10.0, max_reorder_s=0.05))
    long_id = S.sfhk_submit(srv, S.request(W.TARGETS["N2"], W.pulse(1600.0, 1.0e14, 4), W.COS2,
                                           1_000_000, 1, 0))
    t0 = time.time()
    while S.sfhk_server_stats_get(srv)["active"] < 1 and time.time() - t0 < 60:
        time.sleep(0.005)
    time.sleep(0.2)
    short_id = S.sfhk_submit(srv, S.request(W.TARGETS["H2"], W.PULSE_800, W.fixed(0.0), 2000,
                                            1, 1))
    short = S.sfhk_wait(srv, short_id, 300.0)
    long = S.sfhk_wait(srv, long_id, 300.0)
    S.sfhk_server_destroy(srv)
    assert short["status"] == S.SFHK_OK and long["status"] == S.SFHK_OK
    span = long["t_done"] - long["t_admit"]
    assert short["t_done"] > long["t_done"] - 0.15 * span
    with pytest.raises(S.SfhkError):
        S.sfhk_server_create(0, S.server_opts(S.SFHK_MIXED, W.GAMMA, max_reorder_s=-1.0))


def _burst_behind_a_long_request(S, **opts):
    """A long request runs for a few slices; then 30 shorter ones arrive at
    once.  Returns the largest number of requests resident at once after the
    burst and every request's result."""
    srv = S.sfhk_server_create(0, S.server_opts(S.SFHK_MIXED, W.GAMMA, W.CUTOFF, W.STAB_CUTOFF,
                                                slice_ms=10.0, **opts))
    ids = [S.sfhk_submit(srv, S.request(W.TARGETS["N2"], W.pulse(1600.0, 1.0e14, 4), W.COS2,
                                        1_000_000, 1, 0))]
    t0 = time.time()
    while S.sfhk_server_stats_get(srv)["slices"] < 5 and time.time() - t0 < 60:
        time.sleep(0.005)
    ids += [S.sfhk_submit(srv, S.request(W.TARGETS["H2"], W.PULSE_800, W.fixed(0.0), 100_000,
                                         2 + i, 1 + i)) for i in range(30)]
    peak = 0
    t0 = time.time()
    while time.time() - t0 < 300:
        st = S.sfhk_server_stats_get(srv)
        peak = max(peak, st["active"])
        if st["completed"] + st["failed"] + st["cancelled"] >= len(ids):
            break
        time.sleep(0.002)
    res = [S.sfhk_wait(srv, i, 300.0) for i in ids]
    S.sfhk_server_destroy(srv)
    return peak, res


def test_admission_horizon_bounds_resident_work(S):
    """With an admission horizon of 50 ms, a burst of 30 requests arriving
    behind a long one waits in the pending queue and is admitted a few at a
    time as the queued work drains; without it all are admitted at once.
    Every request completes either way."""
    peak, res = _burst_behind_a_long_request(S, max_queued_s=0.05)
    assert all(r["status"] == S.SFHK_OK for r in res)
    assert peak <= 16                 # at most half the burst resident (10 to 13 measured)
    assert max(r["t_admit"] - r["t_submit"] for r in res[1:]) > 0.05
    peak0, res0 = _burst_behind_a_long_request(S)
    assert all(r["status"] == S.SFHK_OK for r in res0)
    assert peak0 >= 25
    with pytest.raises(S.SfhkError):
        S.sfhk_server_create(0, S.server_opts(S.SFHK_MIXED, W.GAMMA, max_queued_s=-1.0))


def test_admission_by_memory_budget_and_refusal(S):
    n = 200_000
    per = n * 110                                   # a request's device state, roughly
    probe = S.sfhk_server_create(0, S.server_opts(S.SFHK_MIXED, W.GAMMA, W.CUTOFF,
                                                  W.STAB_CUTOFF))
    base = S.sfhk_server_stats_get(probe)["device_bytes"]   # the server's own buffers
    S.sfhk_server_destroy(probe)
    # room for one request of 200k trajectories, not two
    budget = base + int(1.5 * per)
    srv = S.sfhk_server_create(0, S.server_opts(S.SFHK_MIXED, W.GAMMA, W.CUTOFF, W.STAB_CUTOFF,
                                                budget=budget, slice_ms=10.0))
    with pytest.raises(S.SfhkError) as e:
        S.sfhk_submit(srv, S.request(W.TARGETS["H2"], W.PULSE_800, W.fixed(0.0), 10 * n, 1, 0))
    assert e.value.code == S.SFHK_E_NOMEM
    ids = [S.sfhk_submit(srv, S.request(W.TARGETS["H2"], W.PULSE_800, W.fixed(a), n, 1, k))
           for k, a in enumerate((0.0, 30.0, 60.0))]
    res = [S.sfhk_wait(srv, i, 300.0) for i in ids]
    st = S.sfhk_server_stats_get(srv)
    S.sfhk_server_destroy(srv)
    assert all(r["status"] == S.SFHK_OK for r in res)
    assert st["rejected"] == 1
    # only one fits at a time: each is admitted after the previous one is done
    assert res[1]["t_admit"] >= res[0]["t_done"] - 1e-6
    assert res[2]["t_admit"] >= res[1]["t_done"] - 1e-6


def test_cancel(S):
    srv = S.sfhk_server_create(0, S.server_opts(S.SFHK_MIXED, W.GAMMA, W.CUTOFF, W.STAB_CUTOFF,
                                                slice_ms=5.0))
    big = S.sfhk_submit(srv, S.request(W.TARGETS["N2"], W.pulse(1600.0, 1.0e14, 4), W.COS2,
                                       1_000_000, 2, 0))
    queued = S.sfhk_submit(srv, S.request(W.TARGETS["H2"], W.PULSE_800, W.fixed(0.0), 1000, 2, 1))
    S.sfhk_cancel(srv, queued)
    S.sfhk_cancel(srv, big)
    r_big = S.sfhk_wait(srv, big, 300.0)
    r_q = S.sfhk_wait(srv, queued, 300.0)
    assert r_big["status"] == S.SFHK_E_CANCELLED and r_q["status"] == S.SFHK_E_CANCELLED
    # the server keeps serving
    ok = S.sfhk_submit(srv, S.request(W.TARGETS["H2"], W.PULSE_800, W.fixed(0.0), 500, 2, 2))
    assert S.sfhk_wait(srv, ok, 300.0)["status"] == S.SFHK_OK
    with pytest.raises(S.SfhkError) as e:
        S.sfhk_poll(srv, 987654321)
    assert e.value.code == S.SFHK_E_NOTFOUND
    S.sfhk_server_destroy(srv)


@pytest.mark.parametrize("slice_ms", [5.0, 0.5])
def test_polyatomic_requests_are_served_with_diatomic_ones(S, slice_ms):
    """Polyatomic requests (their own ring and integrator kernel) served in one
    stream with diatomic ones, each result against the FP64 oracle on the same
    draws: 1e-9 in FP64, 1e-4 in mixed precision; with 0.5 ms slices the
    items of both rings are parked and resumed many times (a resumed
    polyatomic item rebuilds its lanes' centre table).  A polyatomic request
    with a quadrature alignment is refused at submission."""
    import oracle as O
    mix = [(W.TARGETS["H2O"], W.PULSE_800, W.ISO, 700, 1),
           (W.TARGETS["H2"], W.PULSE_800, W.fixed(30.0), 1500, 2),
           (W.TARGETS["H2O_3a1"], W.pulse(1000.0, 1.2e14, 2), W.fixed(50.0, 20.0, 70.0), 400, 3),
           (W.TARGETS["N2"], W.PULSE_1200, W.COS2, 900, 4)]
    ref = []
    for t, p, al, n, inst in mix:
        soa, _, _ = O.sample(t, p, al, seed=7, instance=inst, n=n)
        ref.append(O.propagate(t, p, soa, W.GAMMA, cutoff=W.CUTOFF, stab_cutoff=W.STAB_CUTOFF,
                               stab_taper=W.STAB_TAPER)[0])
    for prec, tol in ((S.SFHK_FP64, 1e-9), (S.SFHK_MIXED, 1e-4)):
        srv = S.sfhk_server_create(0, S.server_opts(prec, W.GAMMA, W.CUTOFF, W.STAB_CUTOFF,
                                                    slice_ms=slice_ms, stab_taper=W.STAB_TAPER))
        with pytest.raises(S.SfhkError):
            S.sfhk_submit(srv, S.request(W.TARGETS["H2O"], W.PULSE_800, W.quadrature(4), 64, 1, 0))
        ids = [S.sfhk_submit(srv, S.request(t, p, al, n, 7, inst)) for t, p, al, n, inst in mix]
        res = [S.sfhk_wait(srv, i, 300.0) for i in ids]
        st = S.sfhk_server_stats_get(srv)
        S.sfhk_server_destroy(srv)
        if slice_ms < 1.0:          # more parkings than work items
            assert st["parked"] > sum(-(-n // 32) for _, _, _, n, _ in mix)
        for (t, p, al, n, inst), r, v in zip(mix, res, ref):
            assert r["status"] == S.SFHK_OK
            err = _rel(r["vz"], v)
            print(f"served kind {t.get('kind', 0)} n={n} precision {prec}: {err:.3e}")
            assert err <= tol, (inst, prec)
