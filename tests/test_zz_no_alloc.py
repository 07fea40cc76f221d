"""The allocation-free merge entry point agrees with the allocating one.

pp_merge_terms_noalloc serves callers that may not allocate device memory
while they run: a serving loop whose device memory is sized once at start-up
(an allocation later could fail under load or stall the device), or an
application that hands out every device allocation from its own pool.  Its
scratch lives in a static device array inside the library.  Here it is called
through the C ABI twice in a row, on different inputs, and each result is
compared with pp_merge_terms on the same input.  The second call also checks
that the scratch left by the first call is cleared before it is reused.

This file is named so that pytest collects it after every other test file.
"""
import numpy as np
import pytest

import paper_2512_12094_gb300 as pp
import pp_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pp.build()
    pp.load()


def _keys(n, m, seed):
    rng = np.random.default_rng(seed)
    strings = []
    for i in range(m):
        w = int(rng.integers(0, min(n, 6) + 1))
        letters = ["I"] * n
        for q in rng.choice(n, size=w, replace=False):
            letters[q] = "XYZ"[int(rng.integers(0, 3))]
        strings.append("".join(letters))
    x, z = pi.to_masks(strings, n)
    keys = np.ascontiguousarray(np.concatenate([x, z], axis=1))
    coef = rng.normal(size=m)
    return keys, coef, (n + 63) // 64


def _as_dict(keys, coef):
    return {tuple(int(v) for v in keys[i]): float(coef[i]) for i in range(len(coef))}


@pytest.mark.parametrize("calls", [((20, 1, 3000, 1), (70, 2, 5000, 2))])
def test_noalloc_merge_matches_allocating_merge_twice(calls):
    import torch
    for n, group, m, seed in calls:
        keys, coef, W = _keys(n, m, seed)
        d_k = torch.from_numpy(keys.view(np.int64)).cuda()
        d_c = torch.from_numpy(coef).cuda()
        ref_k, ref_c = torch.empty_like(d_k), torch.empty_like(d_c)
        m_ref = pp.pp_merge_terms(n, group, m, d_k, d_c, ref_k, ref_c)
        out_k, out_c = torch.empty_like(d_k), torch.empty_like(d_c)
        m_dev = torch.full((1,), -7, dtype=torch.int64, device="cuda")
        stream = torch.cuda.current_stream()
        pp.pp_merge_terms_noalloc(n, group, m, d_k, d_c, out_k, out_c, m_dev, stream)
        stream.synchronize()
        m_got = int(m_dev.cpu()[0])
        assert m_got == m_ref
        got = _as_dict(out_k[:m_got].cpu().numpy().view(np.uint64), out_c[:m_got].cpu().numpy())
        want = _as_dict(ref_k[:m_ref].cpu().numpy().view(np.uint64), ref_c[:m_ref].cpu().numpy())
        assert set(got) == set(want)
        assert max(abs(got[k] - want[k]) for k in want) < 1e-12


def test_noalloc_merge_rejects_oversized_input():
    import torch
    m_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(pp.PPError) as e:
        pp.pp_merge_terms_noalloc(16, 0, 524289, 1, 1, 1, 1, m_dev)
    assert e.value.status == 1
    assert "524288" in str(e.value)


def test_noalloc_merge_allocates_nothing():
    """Free device memory is the same before and after a call (after a first
    call on the device, which looks up the scratch address), and that call's
    result matches pp_merge_terms on the same input."""
    import torch
    n, group, m = 24, 1, 4000
    keys, coef, W = _keys(n, m, 11)
    d_k = torch.from_numpy(keys.view(np.int64)).cuda()
    d_c = torch.from_numpy(coef).cuda()
    out_k, out_c = torch.empty_like(d_k), torch.empty_like(d_c)
    m_dev = torch.zeros(1, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        pp.pp_merge_terms_noalloc(n, group, m, d_k, d_c, out_k, out_c, m_dev, stream)
    stream.synchronize()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    pp.pp_merge_terms_noalloc(n, group, m, d_k, d_c, out_k, out_c, m_dev, stream)
    stream.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref_k, ref_c = torch.empty_like(d_k), torch.empty_like(d_c)
    m_ref = pp.pp_merge_terms(n, group, m, d_k, d_c, ref_k, ref_c)
    m_got = int(m_dev.cpu()[0])
    assert m_got == m_ref
    got = _as_dict(out_k[:m_got].cpu().numpy().view(np.uint64), out_c[:m_got].cpu().numpy())
    want = _as_dict(ref_k[:m_ref].cpu().numpy().view(np.uint64), ref_c[:m_ref].cpu().numpy())
    assert set(got) == set(want)
    assert max(abs(got[k] - want[k]) for k in want) < 1e-12
