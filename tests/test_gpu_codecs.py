"""GPU storage codecs against the oracle's codecs: every one of the 2^32 FP32
bit patterns is encoded on the GPU and compared code by code with the
oracle, and every one of the 65536 codes is decoded and compared bit by bit.
For IEEE FP16 / FP16S a NaN input must give a NaN code and a NaN code must
decode to NaN (the NaN payload is not part of the format's definition)."""
import numpy as np
import pytest

import __graft_entry__
import oracle

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FORMATS = ["FP16", "FP16S", "FP16C", "P16_0S", "P16_1S", "P16_2C", "P16_0", "P16_1"]
CHUNK = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    __graft_entry__.build()


def _is_nan_code(c):
    return ((c & 0x7C00) == 0x7C00) & ((c & 0x03FF) != 0)


@pytest.mark.parametrize("fmt", FORMATS)
def test_encode_all_fp32_inputs(fmt):
    import paper_2112_08926_gb300 as P
    ieee = fmt in ("FP16", "FP16S")
    out = torch.empty(CHUNK, dtype=torch.int16, device="cuda")
    for first in range(0, 1 << 32, CHUNK):
        P.codec_encode_bits(fmt, first, CHUNK, out=out)
        got = out.cpu().numpy().view(np.uint16)
        ref = oracle.encode_bits_range(fmt, first, CHUNK)
        if ieee:
            bits = np.arange(first, first + CHUNK, dtype=np.uint64).astype(np.uint32)
            nan_in = (bits & 0x7F800000) == 0x7F800000
            nan_in &= (bits & 0x007FFFFF) != 0
            assert np.all(_is_nan_code(got[nan_in]))
            ok = ~nan_in
            mism = np.flatnonzero(got[ok] != ref[ok])
        else:
            mism = np.flatnonzero(got != ref)
        if mism.size:
            k = mism[0]
            pytest.fail(f"{fmt}: {mism.size} mismatches in chunk {first:#x}, first at bits "
                        f"{first + int(k):#010x}: gpu {got[k]:#06x} oracle {ref[k]:#06x}")


@pytest.mark.parametrize("fmt", ["P16_0S", "P16_1S", "P16_2C", "P16_0", "P16_1"])
def test_table_encoder_all_fp32_inputs(fmt):
    """The paired kernel's table-driven posit encoder, over all 2^32 inputs."""
    import paper_2112_08926_gb300 as P
    out = torch.empty(CHUNK, dtype=torch.int16, device="cuda")
    for first in range(0, 1 << 32, CHUNK):
        P.codec_encode_bits(fmt, first, CHUNK, out=out, table=True)
        got = out.cpu().numpy().view(np.uint16)
        ref = oracle.encode_bits_range(fmt, first, CHUNK)
        mism = np.flatnonzero(got != ref)
        if mism.size:
            k = mism[0]
            pytest.fail(f"{fmt}: {mism.size} mismatches in chunk {first:#x}, first at bits "
                        f"{first + int(k):#010x}: gpu {got[k]:#06x} oracle {ref[k]:#06x}")


@pytest.mark.parametrize("fmt", FORMATS)
def test_decode_all_codes(fmt):
    import paper_2112_08926_gb300 as P
    codes = np.arange(1 << 16, dtype=np.uint16)
    got = P.codec_decode(fmt, torch.from_numpy(codes.view(np.int16)).cuda()).cpu().numpy()
    ref = oracle.decode(fmt, codes)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.uint32), ref[~nan].view(np.uint32))


@pytest.mark.parametrize("fmt", FORMATS)
def test_encode_array_entry_point(fmt):
    import paper_2112_08926_gb300 as P
    rng = np.random.default_rng(4)
    x = (np.exp2(rng.uniform(-40, 3, 1 << 20)) * np.where(rng.uniform(size=1 << 20) < 0.5, -1, 1)).astype(np.float32)
    got = P.codec_encode(fmt, torch.from_numpy(x).cuda()).cpu().numpy().view(np.uint16)
    assert np.array_equal(got, oracle.encode(fmt, x))
