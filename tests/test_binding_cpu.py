"""The Python binding's argument checks, without a GPU: values that a cast to
int32 would wrap onto other values, coordinates off the grid in wider dtypes,
non-integer data, and k-NN output buffers of the wrong shape, dtype, layout or
device are refused before anything reaches the library."""
import numpy as np
import pytest
import torch

from paper_2112_06188_gb300 import forest as F


def test_int32_inputs_pass_through_unchanged():
    x = torch.tensor([[0, (1 << 20) - 1]], dtype=torch.int32)
    assert F._coords_i32(x) is x          # no cast, no device reduction
    ids = np.array([-3, 7, 2**31 - 1], np.int32)
    assert F._ids_i32(ids).tolist() == [-3, 7, 2**31 - 1]


def test_wide_coordinates_checked_before_the_cast():
    with pytest.raises(ValueError):
        F._coords_i32(np.array([[2**32 + 3, 0]], np.int64))     # would wrap to 3
    with pytest.raises(ValueError):
        F._coords_i32(np.array([[-1, 0]], np.int64))
    with pytest.raises(ValueError):
        F._coords_i32(np.array([[1 << 20, 0]], np.int64))
    ok = F._coords_i32(np.array([[0, (1 << 20) - 1]], np.int64))
    assert ok.dtype == torch.int32 and ok.tolist() == [[0, (1 << 20) - 1]]


def test_wide_ids_checked_before_the_cast():
    with pytest.raises(ValueError):
        F._ids_i32(np.array([2**32 + 5], np.int64))             # would wrap to 5
    with pytest.raises(ValueError):
        F._ids_i32(np.array([-(2**31) - 1], np.int64))
    assert F._ids_i32(np.array([-4, 9], np.int64)).tolist() == [-4, 9]   # ignored by erase, not refused


def test_non_integer_data_refused():
    with pytest.raises(TypeError):
        F._coords_i32(np.array([[1.5, 2.0]]))
    with pytest.raises(TypeError):
        F._ids_i32(torch.tensor([True, False]))


def test_forest_calls_refuse_wrapping_values_before_device_work():
    f = F.Forest.__new__(F.Forest)      # no library call: the checks come first
    f.dim, f.device, f.stream, f._h = 2, torch.device("cuda", 0), None, None
    with pytest.raises(ValueError):
        f.erase(np.array([2**32 + 5], np.int64))
    with pytest.raises(ValueError):
        f.insert(np.array([[2**32 + 3, 1]], np.int64))
    with pytest.raises(ValueError):
        f.knn(np.array([[0, 2**33]], np.int64), 4)


def test_knn_output_buffers_checked():
    m, k, dev = 5, 3, torch.device("cuda", 0)
    oi = torch.empty((m, k), dtype=torch.int32)
    od = torch.empty((m, k), dtype=torch.int64)
    with pytest.raises(ValueError):                  # host memory, not the forest's device
        F._check_out(oi, od, m, k, dev)
    with pytest.raises(ValueError):                  # too short
        F._check_out(oi[:2], od[:2], m, k, "cpu")
    with pytest.raises(ValueError):                  # dtypes swapped
        F._check_out(od, oi, m, k, "cpu")
    with pytest.raises(ValueError):                  # not contiguous
        F._check_out(torch.empty((k, m), dtype=torch.int32).t(), od, m, k, "cpu")
    with pytest.raises(TypeError):
        F._check_out(None, od, m, k, "cpu")
