"""The Python binding refuses buffers that the C library would read or write past
(wrong dtype, too short, not contiguous, host memory where device memory is
expected).  Host logic only: no CUDA call is made."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1809_05637_gb300._lib import _require_doubles  # noqa: E402


def test_host_buffers():
    _require_doubles("rho", np.zeros(10), 10, "host")
    _require_doubles("rho", np.zeros(12), 10, "host")  # longer is harmless
    _require_doubles("rho", torch.zeros(10, dtype=torch.float64), 10, "host")
    with pytest.raises(ValueError, match="holds 9 values"):
        _require_doubles("rho", np.zeros(9), 10, "host")
    with pytest.raises(ValueError, match="float64"):
        _require_doubles("rho", np.zeros(10, dtype=np.float32), 10, "host")
    with pytest.raises(ValueError, match="float64"):
        _require_doubles("rho", np.zeros(20)[::2], 10, "host")  # strided view
    with pytest.raises(ValueError, match="float64"):
        _require_doubles("rho", torch.zeros(10, dtype=torch.float32), 10, "host")
    with pytest.raises(TypeError):
        _require_doubles("rho", [0.0] * 10, 10, "host")


def test_device_buffers_refuse_host_memory():
    for x in (np.zeros(10), torch.zeros(10, dtype=torch.float64)):
        with pytest.raises(ValueError, match="CUDA tensor on cuda:0"):
            _require_doubles("rho_out", x, 10, "device", 0)


def test_empty_system_passes_through():
    """An unbuilt context has nval = 0: an empty buffer passes here and the library
    itself reports the argument error."""
    _require_doubles("rho", np.zeros(0), 0, "host")
