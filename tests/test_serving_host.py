"""Host-side pieces of the transform server (no GPU)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1605_00561_gb300 import serving  # noqa: E402


def test_request_bytes_counts_output_and_ll_scratch():
    r = serving.Request(w=1001, h=999, levels=3, dtype="f32")
    w1, h1, h2 = 501, 500, 250
    pitch = (w1 * 4 + 127) // 128 * 128
    # output rows of 4004 bytes padded to 4096
    assert serving.request_bytes(r) == 4096 * 999 + pitch * (h1 + h2) + 1024
    # one level needs no LL ping-pong
    assert serving.request_bytes(serving.Request(w=64, h=64, levels=1, dtype="i32")) == 64 * 64 * 4
    assert serving.request_bytes(serving.Request(w=64, h=64, levels=2, dtype="f16s")) == \
        64 * 64 * 2 + 128 * (32 + 16) + 1024
    assert serving.request_bytes(serving.Request(w=65, h=3, levels=1, dtype="f16s")) == 256 * 3


def test_output_pitch_is_128_byte_rows():
    assert serving.out_pitch(1, "f32") == 128
    assert serving.out_pitch(32, "f32") == 128
    assert serving.out_pitch(33, "f32") == 256
    assert serving.out_pitch(64, "f16s") == 128
    assert serving.out_pitch(65, "f16s") == 256


def test_percentile_nearest_rank():
    xs = list(range(101))
    assert serving.percentile(xs, 50) == 50
    assert serving.percentile(xs, 99) == 99
    assert serving.percentile([3.0], 99) == 3.0


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU error")
def test_server_refuses_without_cuda():
    with pytest.raises(RuntimeError):
        serving.Server()
