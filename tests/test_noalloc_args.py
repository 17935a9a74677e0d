"""The binding of the allocation-free level refuses buffers the kernel cannot
safely read, before the library is called (no GPU needed).

The kernel reads A and the points on the device, so a host array, a wrong
element count, n beyond the points or an output of the wrong type would make
it read or write outside a buffer.  A stand-in object with the attributes of
a CUDA tensor lets the checks after the first one run without a device; it
has no ``data_ptr``, so a check that let it through would fail loudly with
AttributeError instead of reaching the library.
"""

import numpy as np
import pytest


class FakeCuda:
    """Looks like a contiguous CUDA tensor to the binding's checks."""

    def __init__(self, shape, dtype="torch.float32", device="cuda:0"):
        self.shape = tuple(shape)
        self.dtype = dtype
        self.device = device
        self.is_cuda = True

    def is_contiguous(self):
        return True

    def numel(self):
        return int(np.prod(self.shape))

    def dim(self):
        return len(self.shape)


def _call(**kw):
    from paper_1712_03084_gb300 import ftr
    args = dict(A=FakeCuda((32, 32, 32)), grid_n=(32, 32, 32), bbox=(0, 0, 0, 1, 1, 1),
                points=FakeCuda((10, 3)))
    args.update(kw)
    return ftr.ftr_iso_level_noalloc(**args)


def test_host_arrays_are_refused():
    with pytest.raises(ValueError):
        _call(A=np.zeros((32, 32, 32), np.float32))
    with pytest.raises(ValueError):
        _call(points=np.zeros((10, 3), np.float32))
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError):
        _call(points=torch.zeros((10, 3)))


def test_wrong_dtypes_and_devices_are_refused():
    with pytest.raises(ValueError):
        _call(A=FakeCuda((32, 32, 32), dtype="torch.float64"))
    with pytest.raises(ValueError):
        _call(points=FakeCuda((10, 3), device="cuda:1"))


def test_sizes_are_checked_against_the_grid_and_the_points():
    with pytest.raises(ValueError):
        _call(A=FakeCuda((32, 32, 31)))
    with pytest.raises(ValueError):
        _call(points=FakeCuda((10, 2)))
    with pytest.raises(ValueError):
        _call(n=11)
    with pytest.raises(ValueError):
        _call(n=-1)
    with pytest.raises(ValueError):
        _call(grid_n=(32, 32))


def test_level_out_must_hold_a_float64():
    with pytest.raises(ValueError):
        _call(level_out=np.zeros(1, np.float32))
    with pytest.raises(ValueError):
        _call(level_out=np.zeros(0, np.float64))
    with pytest.raises(ValueError):
        _call(level_out=FakeCuda((1,), dtype="torch.float32"))
