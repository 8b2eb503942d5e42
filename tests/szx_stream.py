"""Pure-Python reader of the compressed stream, used by the tests.

It parses every section and rebuilds each block's truncated words t_i from the
lead codes and mid-byte planes, so the tests can check what each stored field
means (Eq. 4 reqBits, identical-leading-byte counts, the Eq. 5 shift, the
byte-count formula) against its definition.  It is written from the format
description alone and shares no code with the C oracle or the CUDA library.
Slow: for small streams only.
"""
import struct
from dataclasses import dataclass, field

import numpy as np

HEADER = 64
MAGIC = 0x42585A53


def pad16(x):
    return (x + 15) // 16 * 16


@dataclass
class Block:
    k: int
    length: int
    state: int            # 0 constant, 1 non-constant (raw included)
    mu_bits: int
    req: int = 0          # reqBits, 0xFF raw, 0 constant
    L: list = field(default_factory=list)
    t: list = field(default_factory=list)
    raw: bytes = b""
    mid_bytes: int = 0


@dataclass
class Stream:
    dtype: int
    w: int
    W: int
    E: int
    M: int
    block: int
    G: int
    n: int
    e_bits: int
    nn: int
    nraw: int
    nesc: int
    total: int
    nb: int
    ntiles: int
    off_state: int
    off_mu: int
    off_index: int
    off_rec: int
    index: list
    blocks: list


def tile_blocks(block, w):
    return max(8, 32768 // (block * w))


def parse(buf):
    buf = bytes(buf)
    magic, version, dtype = struct.unpack_from("<IBB", buf, 0)
    assert magic == MAGIC and version == 1, "bad magic/version"
    block, G, n, e_bits, nn, nraw, nesc, total = struct.unpack_from("<IIQQQQQQ", buf, 8)
    w, W, E, M = (4, 32, 8, 23) if dtype == 0 else (8, 64, 11, 52)
    assert total == len(buf), (total, len(buf))
    nb = -(-n // block)
    ntiles = -(-nb // G)
    off_state = HEADER
    off_mu = off_state + pad16(-(-nb // 8))
    off_index = off_mu + pad16(nb * w)
    off_rec = off_index + pad16(8 * (ntiles + 1))
    index = list(struct.unpack_from(f"<{ntiles + 1}Q", buf, off_index))
    blocks = []
    for tile in range(ntiles):
        k0, k1 = tile * G, min(nb, tile * G + G)
        rec = buf[off_rec + index[tile]: off_rec + index[tile + 1]]
        states = [(buf[off_state + k // 8] >> (k % 8)) & 1 for k in range(k0, k1)]
        nn_t = sum(states)
        lead = rec[: nn_t * (block // 4)]
        reqs = rec[nn_t * (block // 4): nn_t * (block // 4 + 1)]
        cur = nn_t * (block // 4 + 1)
        rank = 0
        for k in range(k0, k1):
            length = min(block, n - k * block)
            mu_bits = int.from_bytes(buf[off_mu + k * w: off_mu + k * w + w], "little")
            b = Block(k, length, states[k - k0], mu_bits)
            if b.state:
                b.req = reqs[rank]
                codes = lead[rank * (block // 4): (rank + 1) * (block // 4)]
                b.L = [(codes[i >> 2] >> (2 * (i & 3))) & 3 for i in range(block)]
                rank += 1
                if b.req == 0xFF:
                    b.raw = rec[cur: cur + length * w]
                    cur += length * w
                    b.mid_bytes = length * w
                else:
                    s = (8 - b.req % 8) % 8
                    q = (b.req + s) // 8
                    own = [[None] * q for _ in range(length)]
                    for j in range(q):
                        for i in range(length):
                            if b.L[i] <= j:
                                own[i][j] = rec[cur]
                                cur += 1
                                b.mid_bytes += 1
                    prev = [0] * q
                    for i in range(length):
                        row = [own[i][j] if own[i][j] is not None else prev[j] for j in range(q)]
                        prev = row
                        word = 0
                        for j in range(q):
                            word |= row[j] << (W - 8 - 8 * j)
                        b.t.append(word)
            blocks.append(b)
        assert pad16(cur) == len(rec), "record size mismatch"
        assert all(x == 0 for x in rec[cur:]), "non-zero pad"
    return Stream(dtype, w, W, E, M, block, G, n, e_bits, nn, nraw, nesc, total, nb, ntiles,
                  off_state, off_mu, off_index, off_rec, index, blocks)


def bits_to_float(bits, w):
    if w == 4:
        return float(np.array([bits], dtype=np.uint32).view(np.float32)[0])
    return float(np.array([bits], dtype=np.uint64).view(np.float64)[0])


def float_bits(x, w):
    if w == 4:
        return int(np.array([x], dtype=np.float32).view(np.uint32)[0])
    return int(np.array([x], dtype=np.float64).view(np.uint64)[0])
