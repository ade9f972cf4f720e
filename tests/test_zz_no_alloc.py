"""The allocation-free spectrum entry point (sfhk_spectrum_noalloc).

Some callers cannot allocate device memory while they call the library -- a
latency-bound serving loop that must not hit an allocation's device
synchronisation, or a process whose device memory is reserved up front by
another framework's allocator.  For them the spectrum has a variant whose
scratch lives in a fixed device array.  This test calls it through the C ABI
and checks it against the ordinary device-buffer sfhk_spectrum on two calls
in a row (different sizes and inputs, so stale scratch would show), and that
a size above the fixed maximum is refused.  It sits in a file of its own
that pytest collects last.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_spectrum_matches_allocating_path_twice():
    import torch
    from paper_2608_13686_b300 import _build
    _build.build()
    from paper_2608_13686_b300 import sfhk as S

    rng = np.random.default_rng(31)
    stream = torch.cuda.current_stream().cuda_stream
    for nt in (6620, 997):                     # two calls in a row
        dt, t0 = 0.05, -0.5 * (nt - 1) * 0.05
        tau = 0.5 * nt * dt
        n_out = nt // 2
        vz = torch.tensor(rng.normal(size=nt) * np.exp(-np.linspace(-3, 3, nt) ** 2),
                          dtype=torch.float64, device="cuda")
        ref = torch.zeros((3, n_out), dtype=torch.float64, device="cuda")
        out = torch.full((3, n_out), float("nan"), dtype=torch.float64, device="cuda")
        S.sfhk_spectrum_device(vz.data_ptr(), nt, dt, t0, tau, ref[0].data_ptr(),
                               ref[1].data_ptr(), ref[2].data_ptr(), n_out, stream)
        S.sfhk_spectrum_noalloc(vz.data_ptr(), nt, dt, t0, tau, out[0].data_ptr(),
                                out[1].data_ptr(), out[2].data_ptr(), n_out, stream)
        torch.cuda.synchronize()
        r, o = ref.cpu().numpy(), out.cpu().numpy()
        assert np.allclose(o[0], r[0], rtol=1e-15, atol=0.0)
        assert np.max(np.abs(o[1] - r[1])) <= 1e-11 * r[1].max()
        big = r[1] > 1e-12 * r[1].max()
        dph = np.angle(np.exp(1j * (o[2] - r[2])))
        assert np.max(np.abs(dph[big])) < 1e-9

    too_big = S.SFHK_NOALLOC_MAX_NT + 1
    buf = torch.zeros(too_big, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SfhkError) as e:
        S.sfhk_spectrum_noalloc(buf.data_ptr(), too_big, 0.05, 0.0, 1.0, buf.data_ptr(), 0, 0,
                                10, stream)
    assert e.value.code == S.SFHK_E_INVAL
