"""What the shared parity inputs exercise, counted on the oracle's streams (CPU
only).  The GPU parity tests compare the CUDA path with the oracle on these
inputs; this file checks that they reach every placement of a lead code, so
that a placement mistake in the kernel cannot pass unseen."""
import numpy as np
import pytest

import oracle
import szx_stream as ss
from cases import VALUE_RELS, bound_for, value_distribution_cases


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_value_distributions_put_every_lead_code_at_every_place(dtype):
    # Sec. V-A: 2-bit lead codes, four to a byte and sixteen to a 32-bit word.
    # For q = 2, 3 and 4 the cases put every code the bound allows
    # (0 .. min(q, 3)) at each of the sixteen places of a word.
    seen = {}
    for v in value_distribution_cases(dtype).values():
        x = v.astype(dtype)
        for rel in VALUE_RELS:
            st = ss.parse(bytes(oracle.compress(x, bound_for(x, rel), 128)))
            for bl in st.blocks:
                if bl.state and bl.req != 0xFF and bl.L:
                    q = (bl.req + ((8 - (bl.req & 7)) & 7)) >> 3
                    for i, code in enumerate(bl.L):
                        seen.setdefault((q, i % 16), set()).add(code)
    for q in (2, 3, 4):
        for place in range(16):
            assert seen.get((q, place)) == set(range(min(q, 3) + 1)), (q, place, seen.get((q, place)))
