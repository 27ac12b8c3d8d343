"""Host-side argument checks of the Python binding (no GPU needed): the element type of fields and
registers must be the context's, and the time-step arrays float64 CUDA tensors long enough for
every patch -- the library addresses them with those assumptions."""
import types

import pytest
import torch

import paper_1412_0934_gb300 as hy


def fake_ctx(dtype):
    return types.SimpleNamespace(dtype=dtype)


def test_element_type_must_match_the_context():
    c64, c32 = fake_ctx(torch.float64), fake_ctx(torch.float32)
    t64 = torch.zeros((5, 2, 2, 2), dtype=torch.float64)
    t32 = torch.zeros((5, 2, 2, 2), dtype=torch.float32)
    hy._same_dtype(c64, t64, [t64, [t64]])
    hy._same_dtype(c32, [t32, t32])
    with pytest.raises(ValueError):
        hy._same_dtype(c64, t64, [t32])
    with pytest.raises(ValueError):
        hy._same_dtype(c32, (t64,))


def test_time_step_arrays():
    assert hy._f64(None, 3, "dt") is None
    with pytest.raises(ValueError):  # float32
        hy._f64(torch.zeros(4, dtype=torch.float32), 1, "dt")
    with pytest.raises(ValueError):  # too short for the patches
        hy._f64(torch.zeros(2, dtype=torch.float64), 3, "dt")
    with pytest.raises(ValueError):  # not contiguous
        hy._f64(torch.zeros(8, dtype=torch.float64)[::2], 1, "dt")
    with pytest.raises(ValueError):  # host memory
        hy._f64(torch.zeros(3, dtype=torch.float64), 3, "dt")
