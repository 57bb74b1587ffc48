"""The binding's argument marshalling on the CPU: vectors reach the C ABI as
column-major N x nrhs FP64 arrays, and complex vectors (the Helmholtz kernel)
as the interleaved real vectors of the 2 x 2 embedding (real part at 2j,
imaginary part at 2j + 1), the layout the oracle's embedding uses."""
import numpy as np
import pytest
import torch

from oracle import helmholtz as hz
from paper_1307_2666_gb300 import api


def _is_colmajor(t):
    return t.ndim == 1 or t.shape[1] == 1 or (t.stride(0) == 1 and t.stride(1) >= t.shape[0])


def test_colmajor_keeps_values_and_gives_column_major():
    x = torch.arange(12, dtype=torch.float64).reshape(4, 3)          # row-major
    y = api._colmajor(x)
    assert _is_colmajor(y) and torch.equal(y, x)
    z = api._colmajor(y)
    assert z.data_ptr() == y.data_ptr()                                # already column-major: no copy
    v = torch.arange(5, dtype=torch.float64)
    assert torch.equal(api._colmajor(v), v)
    with pytest.raises(TypeError):
        api._colmajor(x.float())


def test_complex_vectors_interleave_like_the_embedding():
    rng = np.random.default_rng(4)
    zc = rng.standard_normal((6, 3)) + 1j * rng.standard_normal((6, 3))
    z = torch.as_tensor(zc)
    r = api._to_real(z)
    assert r.shape == (12, 3) and _is_colmajor(r)
    np.testing.assert_array_equal(r.numpy(), hz.to_real(zc))
    np.testing.assert_array_equal(api._to_complex(r).numpy(), zc)
    v = torch.as_tensor(zc[:, 0].copy())
    np.testing.assert_array_equal(api._to_real(v).numpy(), hz.to_real(zc[:, 0]))
    np.testing.assert_array_equal(api._to_complex(api._to_real(v)).numpy(), zc[:, 0])


def test_output_buffers_are_column_major():
    x = api._colmajor(torch.zeros(7, 4, dtype=torch.float64))
    y = api._empty_like_cm(x)
    assert y.shape == (7, 4) and _is_colmajor(y)
    assert api._empty_like_cm(torch.zeros(5, dtype=torch.float64)).shape == (5,)
