"""Host-side argument checks of the Python binding (CPU): maps handed to the C ABI as bare
pointers must be CUDA tensors, and the batch's output-check cache compares tensor identity."""
import pytest

torch = pytest.importorskip("torch")

from paper_1901_09593_gb300 import batch, msbm  # noqa: E402


def test_maps_must_be_cuda_tensors():
    with pytest.raises(TypeError):
        msbm._check_map(torch.empty((2, 3), dtype=torch.int16), 3, 2, torch.int16, "d")   # host tensor
    with pytest.raises(TypeError):
        msbm._check_map(None, 3, 2, torch.int16, "d")
    with pytest.raises(TypeError):
        msbm._check_image(torch.empty((2, 3), dtype=torch.uint8), 3, 2, "left")


def test_batch_output_cache_compares_identity():
    a, b = torch.empty(1), torch.empty(1)
    assert batch._same([a, b], [a, b])
    assert not batch._same([a, b], [a, torch.empty(1)])
    assert not batch._same([a], [a, b])
    assert batch._same(None, None) and not batch._same(None, [a])
