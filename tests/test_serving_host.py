"""Host-side pieces of the transform server (no GPU)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1605_00561_gb300 import serving  # noqa: E402


def work(cw, ch):
    """Work-list bound of one level with cw x ch quadruples."""
    nrs = (ch + 1) // 2
    return 1024 + 8 * ((cw + 119) // 120) * nrs + 12 * nrs


def test_request_bytes_counts_output_ll_buffers_and_work_list():
    r = serving.Request(w=1001, h=999, levels=3, dtype="f32")
    # output rows of 4004 bytes padded to 4096; LL of levels 1 and 2:
    # 501 x 500 (rows of 2004 -> 2048 bytes) and 251 x 250 (1004 -> 1024)
    assert serving.request_bytes(r) == (4096 * 999 + 2048 * 500 + 1024 * 250 +
                                        work(501, 500) + work(251, 250) + work(126, 125))
    # one level has no LL buffer
    assert serving.request_bytes(serving.Request(w=64, h=64, levels=1, dtype="i32")) == \
        64 * 64 * 4 + work(32, 32)
    # 32 x 32 float16 LL: 64-byte rows padded to 128
    assert serving.request_bytes(serving.Request(w=64, h=64, levels=2, dtype="f16s")) == \
        64 * 64 * 2 + 128 * 32 + work(32, 32) + work(16, 16)
    assert serving.request_bytes(serving.Request(w=65, h=3, levels=1, dtype="f16s")) == 256 * 3 + work(33, 2)
    # narrow and tall: every level's rows round up to 128 bytes
    assert serving.request_bytes(serving.Request(w=8, h=4096, levels=4, dtype="f32")) == \
        128 * 4096 + 128 * (2048 + 1024 + 512) + work(4, 2048) + work(2, 1024) + work(1, 512) + work(1, 256)


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
