"""BETWEEN (Sec. 4.2.2) on the GPU: [lo <= x <= hi] on every slot of 4
ciphertexts (one tile of 3 and a ragged tail of 1) with the bounds, values just
outside them, 0 and (p-1)/2 in the inputs; the tail's ciphertext bit for bit
against the oracle's product (1 - LT(x, lo)) (1 - LT(hi, x)) of its two LT
evaluations (through the SHA-256 the oracle wrote into
tests/golden/between_n4096.txt, see make_between_digest.py); bound errors and
the empty range lo > hi."""
import hashlib

import numpy as np
import pytest

from paper_2602_24271_b300 import build, hp
from tests.conftest import read_golden_kv
from tests.golden.make_between_digest import CT, HALF, HI, LO, LOGN, SEED_ENC, SEED_KEY, between_inputs

pytestmark = pytest.mark.gpu


def test_between_closed_form_and_oracle_parity():
    import torch

    build.build()
    ctx = hp.Context(LOGN, max_tile_ct=3)
    ctx.keygen(SEED_KEY)
    N = ctx.N
    x = between_inputs(N)
    cx = ctx.encrypt(x.reshape(-1, N), seed=SEED_ENC)
    out = ctx.between(cx, LO, HI)
    torch.cuda.synchronize()
    ctx.check_status()
    assert ctx.launch_count() > 0
    assert np.array_equal(ctx.decrypt(out).reshape(-1), ((x >= LO) & (x <= HI)).astype(np.uint32))
    gold = read_golden_kv("between_n4096.txt")
    assert gold["lo"] == LO and gold["hi"] == HI and gold["ciphertext"] == CT
    digest = hashlib.sha256(np.ascontiguousarray(hp.to_u64(out[CT]), dtype=np.uint64).tobytes()).hexdigest()
    assert digest == gold["sha256"]
    with pytest.raises(hp.HpError) as e:
        ctx.between(cx, 0, HALF + 1)
    assert e.value.code == hp.HP_ERR_ARG
    with pytest.raises(hp.HpError) as e:
        ctx.between(cx, HI, LO)
    assert e.value.code == hp.HP_ERR_ARG
    ctx.close()
