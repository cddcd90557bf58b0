"""Host-side argument checks of the allocation-free solve's Python binding.

The C entry point launches on the current device and uses that device's
scratch array, so a tensor on another GPU, a stream of another GPU or a
non-contiguous row mask must be refused before the call.  Stand-in tensors
(device, dtype, contiguity, size) exercise the checks without a GPU.
"""
import pytest

torch = pytest.importorskip("torch")

from paper_2103_14870_gb300 import graphfem  # noqa: E402


class FakeCuda:
    def __init__(self, n, dtype, device=0, contiguous=True):
        self.n, self.dtype, self.device, self.contig = n, dtype, torch.device("cuda", device), contiguous

    def numel(self):
        return self.n

    def is_contiguous(self):
        return self.contig


def args(n=4, **over):
    a = dict(row_ptr=FakeCuda(n + 1, torch.int32), col=FakeCuda(n, torch.int32),
             values=FakeCuda(9 * n, torch.float64), b=FakeCuda(3 * n, torch.float64),
             x=FakeCuda(3 * n, torch.float64), fixed=FakeCuda(n, torch.uint8))
    a.update(over)
    return a


@pytest.fixture(autouse=True)
def fake_cuda_predicate(monkeypatch):
    monkeypatch.setattr(graphfem, "_is_torch_cuda", lambda t: isinstance(t, FakeCuda))


def test_accepts_tensors_on_the_current_device():
    assert graphfem._static_solve_args(**args(), device=0, stream_device=0) == 4
    assert graphfem._static_solve_args(**args(fixed=None), device=0, stream_device=None) == 4


@pytest.mark.parametrize("name", ["row_ptr", "col", "values", "b", "x", "fixed"])
def test_rejects_a_tensor_on_another_device(name):
    a = args()
    a[name] = FakeCuda(a[name].n, a[name].dtype, device=1)
    with pytest.raises(ValueError, match=name):
        graphfem._static_solve_args(**a, device=0, stream_device=0)


def test_rejects_a_stream_of_another_device():
    with pytest.raises(ValueError, match="stream"):
        graphfem._static_solve_args(**args(), device=0, stream_device=1)


@pytest.mark.parametrize("name", ["fixed", "x", "values"])
def test_rejects_non_contiguous_tensors(name):
    a = args()
    a[name] = FakeCuda(a[name].n, a[name].dtype, contiguous=False)
    with pytest.raises(TypeError, match=name):
        graphfem._static_solve_args(**a, device=0, stream_device=0)


def test_rejects_wrong_dtype_and_sizes():
    with pytest.raises(TypeError, match="fixed"):
        graphfem._static_solve_args(**args(fixed=FakeCuda(4, torch.bool)), device=0, stream_device=0)
    with pytest.raises(ValueError, match="3 \\* n_rows"):
        graphfem._static_solve_args(**args(b=FakeCuda(11, torch.float64)), device=0, stream_device=0)
