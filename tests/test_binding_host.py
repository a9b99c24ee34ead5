"""The Python binding fails loudly instead of falling back (no GPU needed)."""
import pytest

from paper_1902_00090_gb300 import _build, binding


def test_missing_library_raises(monkeypatch):
    # no CPU path exists: without libddgmres.so every call raises
    monkeypatch.setattr(_build, "LIB", "/nonexistent/libddgmres.so")
    monkeypatch.setattr(binding, "_LIB", None)
    with pytest.raises(RuntimeError, match="is missing"):
        binding.load()


def test_calls_refuse_to_run_without_a_gpu():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    with pytest.raises(RuntimeError, match="needs a CUDA device"):
        binding.Context()
    with pytest.raises(RuntimeError, match="needs a CUDA device"):
        binding.Predictor(k=2, channels=(4,) * 6)


def test_device_pointers_only_from_contiguous_cuda_tensors_of_the_right_type():
    torch = pytest.importorskip("torch")
    with pytest.raises(ValueError, match="contiguous CUDA tensor"):
        binding._dev_ptr(torch.zeros(4, dtype=torch.complex128), torch.complex128, "x", 4)
    with pytest.raises(ValueError, match="contiguous CUDA tensor"):
        binding._dev_ptr(torch.zeros(4, dtype=torch.complex64), torch.complex128, "x", 4)
