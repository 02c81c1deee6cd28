"""The binding refuses buffers that the library would overrun or misread (wrong element
count, dtype, layout, device, or mixed host and device halves of one output), before any
library call.  CPU only: these checks need no GPU."""
import numpy as np
import pytest

from paper_2103_11050_gb300 import binding as B


def test_pointer_checks_on_host_arrays():
    a = np.zeros((2, 3, 4))
    p, mem = B._ptr(a, 24)
    assert mem == B.MEM_HOST and p.value == a.ctypes.data
    with pytest.raises(ValueError, match="expected 25 values"):
        B._ptr(a, 25)
    with pytest.raises(ValueError, match="float64"):
        B._ptr(a.astype(np.float32), 24)
    with pytest.raises(ValueError, match="contiguous"):
        B._ptr(np.zeros((4, 6))[:, ::2], 12)
    with pytest.raises(TypeError):
        B._ptr([0.0] * 24, 24)


def test_pointer_checks_on_cpu_tensors():
    torch = pytest.importorskip("torch")
    t = torch.zeros((2, 3, 4), dtype=torch.float64)
    p, mem = B._ptr(t, 24)
    assert mem == B.MEM_HOST and p.value == t.data_ptr()
    with pytest.raises(ValueError, match="expected 23 values"):
        B._ptr(t, 23)
    with pytest.raises(ValueError, match="float64"):
        B._ptr(t.float(), 24)
    with pytest.raises(ValueError, match="contiguous"):
        B._ptr(t.transpose(0, 2), 24)
