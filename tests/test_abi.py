"""The C-ABI library loads and exports every entry point include/sfhk.h
declares (CPU only: no compute calls)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sfhk.h")).read()
    return sorted(set(re.findall(r"^SFHK_API\s+[\w\s\*]+?\b(sfhk_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("sfhk_create_target", "sfhk_set_pulse", "sfhk_sample_initial",
                     "sfhk_propagate", "sfhk_dipole", "sfhk_spectrum"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2608_13686_b300 import _build
    _build.build()
    import ctypes
    lib = ctypes.CDLL(_build.OUT)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_every_symbol():
    from paper_2608_13686_b300 import sfhk as S
    assert sorted(S.EXPORTED) == _declared()


def test_no_device_means_loud_error():
    from paper_2608_13686_b300 import sfhk as S
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    with pytest.raises(S.SfhkError) as e:
        S.sfhk_create(0, 0)
    assert e.value.code == S.SFHK_E_CUDA
