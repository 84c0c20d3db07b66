"""The allocation-free squaring entry point (hp_square_noalloc) against the
regular one (hp_run with HP_SQUARE), through the C ABI.

hp_square_noalloc serves callers that cannot allocate device memory when they
need the operation (a memory pool already owns the GPU, or a fixed-footprint
serving loop); its scratch is a fixed array inside the library.  Results must
be bit-identical to hp_run's, on two calls in a row (the shared scratch keeps
the first call's contents when the second runs).  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

from paper_2602_24271_b300 import build, hp

pytestmark = pytest.mark.gpu


def _noalloc(ctx, x, out):
    rc = ctx.lib.hp_square_noalloc(ctx.h, x.data_ptr(), out.data_ptr(), None)
    if rc != hp.HP_OK:
        raise hp.HpError(rc, ctx.lib.hp_last_error(ctx.h).decode())


def test_noalloc_square_matches_hp_run_twice():
    import torch

    build.build()
    ctx = hp.Context(12, max_tile_ct=1)
    ctx.keygen(77)
    rng = np.random.default_rng(12)
    slots = rng.integers(0, hp.T, (2, ctx.N)).astype(np.uint32)
    cts = ctx.encrypt(slots, seed=5)
    # call 1: a fresh ciphertext
    ref1 = ctx.run(hp.HP_SQUARE, cts[0:1])
    got1 = torch.empty_like(ref1)
    _noalloc(ctx, cts[0], got1[0])
    torch.cuda.synchronize()
    assert np.array_equal(hp.to_u64(got1), hp.to_u64(ref1))
    # call 2 right after: another input, the scratch still holds call 1's data
    ref2 = ctx.run(hp.HP_SQUARE, cts[1:2])
    got2 = torch.empty_like(ref2)
    _noalloc(ctx, cts[1], got2[0])
    torch.cuda.synchronize()
    assert np.array_equal(hp.to_u64(got2), hp.to_u64(ref2))
    assert not np.array_equal(hp.to_u64(got1), hp.to_u64(got2))
    # the squaring is 13 launches: lift, tensor, scale-and-round, key-switch
    # multiply-accumulate and mod-down, plus four two-pass transforms
    assert ctx.launch_count() == 13
    # in place (ct_out aliasing ct_in), again bit for bit against hp_run
    inplace = cts[0:1].clone()
    _noalloc(ctx, inplace[0], inplace[0])
    torch.cuda.synchronize()
    assert np.array_equal(hp.to_u64(inplace), hp.to_u64(ref1))
    ctx.check_status()
    ctx.close()


def test_noalloc_rejects_ring_degree_above_limit():
    import torch

    build.build()
    ctx = hp.Context(13, max_tile_ct=1)
    ctx.keygen(78)
    x = ctx.ct_empty(1)
    with pytest.raises(hp.HpError) as e:
        _noalloc(ctx, x[0], x[0])
    assert e.value.code == hp.HP_ERR_UNSUPPORTED
    assert b"scratch" in ctx.lib.hp_last_error(ctx.h)
    torch.cuda.synchronize()
    ctx.close()
