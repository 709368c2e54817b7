"""The binding's buffer checks (CPU): a device buffer with the wrong dtype,
shape or size, or one that is not contiguous or not on the GPU, raises
ValueError in the binding, before the C call could read or write past it."""
import pytest

torch = pytest.importorskip("torch")

from paper_2403_11367_gb300 import reloc  # noqa: E402


def test_ptr_checks_dtype_shape_size_layout_and_device():
    f32 = torch.zeros((3, 4, 5), dtype=torch.float32)
    with pytest.raises(ValueError, match="dtype"):
        reloc._ptr(torch.zeros(8, dtype=torch.float64), reloc._F32, name="x")
    with pytest.raises(ValueError, match="shape"):
        reloc._ptr(f32, reloc._F32, shape=(3, 5, 4), name="x")
    with pytest.raises(ValueError, match="elements"):
        reloc._ptr(f32, reloc._F32, numel=61, name="x")
    with pytest.raises(ValueError, match="contiguous"):
        reloc._ptr(f32.transpose(1, 2), reloc._F32, name="x")
    with pytest.raises(ValueError, match="CUDA"):
        reloc._ptr(f32, reloc._F32, shape=(3, 4, 5), numel=60, name="x")
    assert reloc._ptr(None, reloc._F32) is None
    # BF16 network buffers may be passed as bfloat16 or as 16-bit integers
    for dt in (torch.bfloat16, torch.int16):
        with pytest.raises(ValueError, match="CUDA"):
            reloc._ptr(torch.zeros(4, dtype=dt), reloc._U16, name="x")


def test_noalloc_wrapper_rejects_bad_image_shape():
    with pytest.raises(ValueError, match="expected"):
        reloc.reloc_ncc_images_noalloc(torch.zeros((2, 4, 8, 8)), torch.zeros((3, 8, 8)), torch.zeros(2, dtype=torch.float64))
    with pytest.raises(ValueError, match="expected"):
        reloc.reloc_ncc_images_noalloc(torch.zeros((3, 8, 8)), torch.zeros((3, 8, 8)), torch.zeros(2, dtype=torch.float64))
