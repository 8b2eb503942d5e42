"""Compressed dump to a host file and load back: every chunk's stream in the
file is byte-identical to the oracle's for that chunk, and the loaded values
are bit-identical to decompressing each chunk."""
import struct

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
from paper_2201_13020_b300 import dump, inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_dump_and_load_round_trip(tmp_path, dtype):
    n = 3 * (1 << 18) + 123
    x = inputs.sinusoid_1d(n, seed=4).astype(dtype)
    eb = inputs.rel_to_abs(x, 1e-3)
    xt = torch.from_numpy(x).cuda()
    path = tmp_path / "field.szx"
    info = dump.dump(xt, eb, str(path), chunk_values=1 << 18)
    assert info["chunks"] == 4 and info["file_bytes"] == path.stat().st_size
    data = path.read_bytes()
    head = struct.calcsize("<8sIIQdQQ")
    pos = head
    u = np.uint32 if dtype == np.float32 else np.uint64
    expect = []
    for k in range(4):
        nbytes = struct.unpack_from("<Q", data, pos)[0]
        stream = np.frombuffer(data, dtype=np.uint8, count=nbytes, offset=pos + 8)
        part = x[k << 18:(k + 1) << 18]
        ref = oracle.compress(part, eb, 128)
        assert np.array_equal(stream, ref), f"chunk {k}: stream differs from the oracle"
        expect.append(oracle.decompress(ref))
        pos += 8 + nbytes
    assert pos == len(data)
    y = dump.load(str(path)).cpu().numpy()
    assert np.array_equal(y.view(u), np.concatenate(expect).view(u))
