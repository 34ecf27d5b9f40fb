"""The Python binding has no CPU path: without the built library it raises,
and every call rejects host tensors before it reaches the library (the
binding only marshals device pointers).  Shape mismatches are caught before
the call.  No GPU is needed for any of this."""
import numpy as np
import pytest
import torch

from paper_2404_00774_gb300 import binding


@pytest.fixture(scope="module", autouse=True)
def _library():
    # the calls below load libsoar.so (host code only): build it if this
    # module runs before any other that does
    from paper_2404_00774_gb300 import build
    build.build()


def test_missing_library_raises_instead_of_falling_back(monkeypatch, tmp_path):
    monkeypatch.setattr(binding, "LIB_PATH", str(tmp_path / "libsoar.so"))
    monkeypatch.setattr(binding, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        binding.load()
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        binding.soar_exact_mips(torch.zeros(4, 2), torch.zeros(1, 2), 1)


def _cpu(*shape, dtype=torch.float32):
    return torch.zeros(shape, dtype=dtype)


CALLS = {
    "soar_train_centroids": lambda: binding.soar_train_centroids(_cpu(20, 4), 2, 1, _cpu(2, dtype=torch.int32),
                                                                 out=_cpu(2, 4)),
    "soar_assign": lambda: binding.soar_assign(_cpu(20, 4), _cpu(3, 4), 1.0, 1, out=_cpu(20, 2, dtype=torch.int32)),
    "soar_index_build": lambda: binding.soar_index_build(_cpu(20, 4), _cpu(3, 4), _cpu(20, 2, dtype=torch.int32)),
    "soar_exact_mips": lambda: binding.soar_exact_mips(_cpu(20, 4), _cpu(3, 4), 2),
    "soar_merge_topk": lambda: binding.soar_merge_topk(_cpu(3, 2, 5, dtype=torch.int64), _cpu(3, 2, 5), 4),
    "soar_quantize_fp8": lambda: binding.soar_quantize_fp8(_cpu(6, 8)),
    "soar_mlp_forward": lambda: binding.soar_mlp_forward(_cpu(binding.soar_mlp_param_count(4, 8)), 4, 8,
                                                         _cpu(3, 4)),
    "soar_mlp_backward": lambda: binding.soar_mlp_backward(_cpu(binding.soar_mlp_param_count(4, 8)), 4, 8,
                                                           _cpu(3, 4), _cpu(3)),
    "soar_mlp_adam": lambda: binding.soar_mlp_adam(_cpu(10), _cpu(10), _cpu(10), _cpu(10), 1, 1e-3),
    "soar_mlp_predict_probes": lambda: binding.soar_mlp_predict_probes(_cpu(binding.soar_mlp_param_count(4, 8)), 4,
                                                                       8, _cpu(3, 4), 1.0, 10),
}


@pytest.mark.parametrize("name", sorted(CALLS))
def test_host_tensors_are_rejected(name):
    before = binding.soar_kernel_launches()
    with pytest.raises(TypeError, match="must be a CUDA tensor"):
        CALLS[name]()
    assert binding.soar_kernel_launches() == before        # nothing reached the library's launch path


def test_shape_mismatches_are_caught_before_the_call():
    with pytest.raises(ValueError, match="disagree on d"):
        binding.soar_assign(_cpu(20, 4), _cpu(3, 5), 1.0, 1)
    with pytest.raises(ValueError, match="one row per datapoint"):
        binding.soar_index_build(_cpu(20, 4), _cpu(3, 4), _cpu(19, 2, dtype=torch.int32))
    with pytest.raises(ValueError, match="same shape"):
        binding.soar_merge_topk(_cpu(3, 2, 5, dtype=torch.int64), _cpu(3, 2, 4), 4)
    with pytest.raises(ValueError, match="one entry per list"):
        binding.soar_merge_topk(_cpu(3, 2, 5, dtype=torch.int64), _cpu(3, 2, 5), 4,
                                id_offsets=_cpu(3, dtype=torch.int64))


def test_unsupported_vector_dtypes_are_rejected():
    with pytest.raises(TypeError, match="float32 or bfloat16"):
        binding._dtype(torch.from_numpy(np.zeros((2, 2))))
    assert binding._dtype(_cpu(2, 2)) == binding.SOAR_F32
    assert binding._dtype(_cpu(2, 2, dtype=torch.bfloat16)) == binding.SOAR_BF16
