"""Prepared batches (sfhk_batch_*) and a whole step captured in a CUDA graph.

A step = re-sampling every ensemble on the device (sfhk_sample_into), one
prepared batched propagation (sfhk_batch_launch) and the device-buffer
spectra.  Its results must equal those of the uncaptured calls, on the first
replay and on later ones.
"""
import numpy as np
import pytest

from paper_2608_13686_b300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [("H2", W.PULSE_800, W.fixed(20.0), 3000, 1),
         ("N2", W.pulse(1000.0, 1.6e14, 2), W.COS2, 2570, 2),
         ("H2", W.pulse(1400.0, 1.0e14, 4), W.fixed(70.0), 650, 3)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_prepared_batch_and_graph_replay():
    import torch
    from paper_2608_13686_b300 import _build
    _build.build()
    from paper_2608_13686_b300 import sfhk as S

    ctx = S.sfhk_create(0, 0)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    handles, ens, grids = [], [], []
    for name, p, al, n, seed in CASES:
        th, ph = S.sfhk_create_target(ctx, W.TARGETS[name]), S.sfhk_set_pulse(ctx, p)
        handles += [th, ph]
        ens.append(S.sfhk_sample_initial(ctx, th, ph, al, n, seed, seed, sp))
        grids.append(S.sfhk_pulse_grid(ph))
    torch.cuda.synchronize()
    for prec, tol in ((S.SFHK_FP64, 1e-12), (S.SFHK_MIXED, 1e-12)):
        opts = S.run_opts(prec, W.GAMMA, W.CUTOFF, stab_cutoff=W.STAB_CUTOFF)
        S.sfhk_propagate_batch(ctx, ens, opts, sp)
        ref = [S.sfhk_dipole(ctx, e, g["nt"]) for e, g in zip(ens, grids)]
        b = S.sfhk_batch_create(ctx, ens, opts)
        S.sfhk_batch_launch(b, sp)
        torch.cuda.synchronize()
        got = [S.sfhk_dipole(ctx, e, g["nt"]) for e, g in zip(ens, grids)]
        for a, r in zip(got, ref):
            assert _rel(a, r) <= tol

        spec = [torch.zeros((3, g["nt"] // 2), dtype=torch.float64, device="cuda") for g in grids]

        def step():
            for (name, p, al, n, seed), e in zip(CASES, ens):
                S.sfhk_sample_into(ctx, e, al, seed, seed, sp)
            S.sfhk_batch_launch(b, sp)
            for e, g, o in zip(ens, grids, spec):
                vz_ptr, _ = S.sfhk_dipole_device(e)
                S.sfhk_spectrum_device(vz_ptr, g["nt"], g["dt"], g["t_origin"], 0.5 * g["Tp"],
                                       o[0].data_ptr(), o[1].data_ptr(), o[2].data_ptr(),
                                       g["nt"] // 2, sp)

        with torch.cuda.stream(stream):
            step()
        torch.cuda.synchronize()
        eager_vz = [S.sfhk_dipole(ctx, e, g["nt"]) for e, g in zip(ens, grids)]
        eager_y = [o[1].cpu().numpy().copy() for o in spec]
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            step()
        for _ in range(2):
            for o in spec:
                o.zero_()
            graph.replay()
            torch.cuda.synchronize()
            for e, g, v, y, o in zip(ens, grids, eager_vz, eager_y, spec):
                assert _rel(S.sfhk_dipole(ctx, e, g["nt"]), v) <= tol
                assert np.max(np.abs(o[1].cpu().numpy() - y)) <= 1e-12 * max(y.max(), 1e-300)
        del graph
        S.sfhk_batch_destroy(b)
    for e in ens:
        S.sfhk_destroy_ensemble(e)
    S.sfhk_destroy(ctx)
