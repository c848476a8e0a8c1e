"""sqd_build_strings_noalloc: the string filter for callers that cannot
allocate device memory (its scratch is a fixed array inside the library).

Collected last on purpose, so that a run stopping at its first failure has
already run every other test.  Each case calls the entry point twice in a
row through the C ABI, on output buffers allocated beforehand, and compares
both results with sqd_build_strings bit for bit (the tolerance of the other
string tests).
"""
import numpy as np
import pytest
import torch

import sqd_inputs as si

pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(3)
    w = si.workload("h2o29")
    yield w.raw_a, 29, 5
    w = si.workload("scale36")
    yield w.raw_a, 36, 15
    junk = rng.integers(0, 1 << 22, size=5000, dtype=np.uint64)
    yield np.concatenate([junk, si.sample_strings(20, 6, 300, si.weights_exp(20), 2)[0]]), 20, 6
    yield np.array([0b1, 0b11], dtype=np.uint64), 6, 3  # nothing valid
    raw = si.sample_strings(40, 12, 60000, si.weights_fermi(40, 12.0, 3.0), 9)[0]
    assert raw.size <= 1 << 18
    yield raw, 40, 12


def test_noalloc_matches_build_strings_twice():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2601_16169_gb300 as sqd
    torch.cuda.set_device(0)
    ctx = sqd.Context(0)
    for raw, norb, ne in _cases():
        d_raw = torch.tensor(raw.view(np.int64), device="cuda")
        ref = sqd.build_strings(ctx, d_raw, norb, ne).cpu()
        outs = [torch.full_like(d_raw, -1) for _ in range(2)]
        for out in outs:  # two calls in a row on the shared scratch
            n = sqd.build_strings_noalloc(ctx, d_raw, norb, ne, out)
            assert n == ref.numel()
            assert torch.equal(out[:n].cpu(), ref)
    ctx.close()


def test_noalloc_in_place_twice():
    # the output buffer may be the input buffer, as for sqd_build_strings:
    # the raw strings reach the scratch array before the output is written
    import paper_2601_16169_gb300 as sqd
    torch.cuda.set_device(0)
    ctx = sqd.Context(0)
    for raw, norb, ne in _cases():
        d_raw = torch.tensor(raw.view(np.int64), device="cuda")
        ref = sqd.build_strings(ctx, d_raw, norb, ne).cpu()
        buf = d_raw.clone()
        for _ in range(2):  # the second call filters the first call's output in place
            n = sqd.build_strings_noalloc(ctx, buf, norb, ne, buf)
            assert n == ref.numel()
            assert torch.equal(buf[:n].cpu(), ref)
            buf = buf[:n].clone() if n else buf[:0]
    ctx.close()


def test_noalloc_rejects_inputs_over_its_limit():
    import paper_2601_16169_gb300 as sqd
    ctx = sqd.Context(0)
    big = torch.zeros((1 << 18) + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(sqd.SQDError) as e:
        sqd.build_strings_noalloc(ctx, big, 20, 3, torch.empty_like(big))
    assert e.value.code == sqd.SQD_EINVAL and "262144" in str(e.value)
    ctx.close()
