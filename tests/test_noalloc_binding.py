"""The Python binding of the allocation-free transcoder refuses, before calling the library,
tensors that the C function would misread: a source that is not bytes, a destination whose
elements are not 16-bit units (the capacity is counted in them), a result smaller than one
gbu_result, and tensors off the current CUDA device.  Runs without a GPU: every tensor here
is refused on the host."""
import pytest

torch = pytest.importorskip("torch")

from paper_2111_08692_gb300 import GbuError, convert_utf8_to_utf16le_noalloc  # noqa: E402


def _args(src_dtype=torch.uint8, dst_dtype=torch.int16, result_elems=2):
    return (torch.zeros(64, dtype=src_dtype), torch.zeros(64, dtype=dst_dtype),
            torch.zeros(result_elems, dtype=torch.int64))


def test_refuses_a_source_that_is_not_uint8():
    with pytest.raises(GbuError, match="uint8"):
        convert_utf8_to_utf16le_noalloc(*_args(src_dtype=torch.int16))


def test_refuses_a_destination_without_2_byte_elements():
    with pytest.raises(GbuError, match="2-byte"):
        convert_utf8_to_utf16le_noalloc(*_args(dst_dtype=torch.uint8))
    with pytest.raises(GbuError, match="2-byte"):
        convert_utf8_to_utf16le_noalloc(*_args(dst_dtype=torch.int32))


def test_refuses_a_result_smaller_than_16_bytes():
    with pytest.raises(GbuError, match="16 bytes"):
        convert_utf8_to_utf16le_noalloc(*_args(result_elems=1))


def test_refuses_tensors_off_the_current_cuda_device():
    # host tensors: never on a CUDA device
    with pytest.raises(GbuError, match="current CUDA device"):
        convert_utf8_to_utf16le_noalloc(*_args())
