"""Host-side checks of the Python binding (no GPU): inputs of the wrong size
are refused before any pointer reaches the library, which would otherwise
read past the end of a short host array."""
import numpy as np
import pytest

from paper_1803_07822_gb300 import lattice
from paper_1803_07822_gb300.lattice import CurvedLattice, CurvedLattice2D


@pytest.fixture(autouse=True)
def torch_without_device(monkeypatch):
    """The binding refuses to run without CUDA (tested below); the
    marshalling checks here need torch only."""
    import torch
    monkeypatch.setattr(lattice, "_torch", lambda: torch)


def test_no_device_no_fallback(monkeypatch):
    monkeypatch.undo()
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lattice._torch()


def _bare(cls, n):
    obj = object.__new__(cls)  # no device: only the marshalling is used
    obj.n = tuple(n)
    obj.N = int(np.prod(n))
    obj.device = None
    return obj


def test_3d_inputs_of_the_wrong_size_are_refused():
    g = _bare(CurvedLattice, (4, 5, 6))
    p, d, k = g._arg(np.zeros((6, 120)), 6 * 120)
    assert d == 0 and k.size == 720 and p == k.ctypes.data
    with pytest.raises(ValueError):
        g._arg(np.zeros((6, 119)), 6 * 120)
    assert g._arg(None, 10)[0] is None


def test_2d_inputs_of_the_wrong_size_are_refused():
    g = _bare(CurvedLattice2D, (8, 5))
    p, d, k = g._arg(np.zeros((3, 40)), 3 * 40)
    assert d == 0 and k.size == 120
    for bad in (np.zeros((3, 39)), np.zeros(3)):
        with pytest.raises(ValueError):
            g._arg(bad, 3 * 40)
    import torch
    p, d, k = g._arg(torch.zeros(2, 5, dtype=torch.float32), 10)  # a CPU tensor is a host array
    assert d == 0 and k.dtype == np.float64 and k.size == 10
