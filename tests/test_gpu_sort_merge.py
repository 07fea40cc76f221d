"""The sort-based merge (radix sort + segmented FP64 reduce) against the oracle.

The merge loop of Algorithms 2 and 3 accumulates every string into its orbit
representative.  The sorted merge must give the oracle's representatives
exactly and its sums within 1e-12 (the oracle adds orbit members in hash-map
order).  Its own summation order is documented: a run of at most 64 equal keys
is added left to right in input order, a longer run by 32 lanes (lane l adds
elements l, l + 32, ... in order) followed by a butterfly over the lanes.  The
tests rebuild that order with Python floats (IEEE double addition) and require
equality bit for bit, so the output is reproducible from call to call.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2512_12094_gb300 as pp
import pp_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pp.build()
    pp.load()
    oracle.build()


def as_dict(x, z, c):
    x = np.asarray(x).reshape(len(c), -1)
    z = np.asarray(z).reshape(len(c), -1)
    d = {tuple(int(v) for v in x[i]) + tuple(int(v) for v in z[i]): float(c[i])
        for i in range(len(c))}
    assert len(d) == len(c), "a string appears twice in the table"
    return d


def rand_strings(n, m, seed, pool=None):
    """m random strings of n qubits (mixed weights); with pool, drawn with
    repetition from `pool` distinct strings so that keys repeat."""
    rng = np.random.default_rng(seed)

    def one():
        w = int(rng.integers(0, min(n, 8) + 1))
        letters = ["I"] * n
        for q in rng.choice(n, size=w, replace=False):
            letters[q] = "XYZ"[int(rng.integers(0, 3))]
        return "".join(letters)

    if pool is None:
        return [one() for _ in range(m)]
    base = [one() for _ in range(pool)]
    return [base[int(rng.integers(0, pool))] for _ in range(m)]


def device_merge(n, group, strings, coef, sorted_merge=True):
    import torch
    x, z = pi.to_masks(strings, n)
    W = x.shape[1]
    keys = np.ascontiguousarray(np.concatenate([x, z], axis=1))
    d_k = torch.from_numpy(keys.view(np.int64)).cuda()
    d_c = torch.from_numpy(np.asarray(coef, dtype=np.float64)).cuda()
    out_k = torch.empty_like(d_k)
    out_c = torch.empty_like(d_c)
    fn = pp.pp_merge_terms_sorted if sorted_merge else pp.pp_merge_terms
    m = fn(n, group, len(strings), d_k, d_c, out_k, out_c)
    ok = out_k[:m].cpu().numpy().view(np.uint64)
    return ok[:, :W], ok[:, W:], out_c[:m].cpu().numpy(), x, z


def packed_order(n, ox, oz):
    """The sort key the merge orders by: x | z << 32 (n <= 32), else (z, x)."""
    if n <= 32:
        return [int(a) | (int(b) << 32) for a, b in zip(ox[:, 0], oz[:, 0])]
    return [(int(b) << 64) | int(a) for a, b in zip(ox[:, 0], oz[:, 0])]


def groups_for(n):
    g = [0, 1, 2, 3]
    if n % 4 == 0 and n >= 8:
        g.append(oracle.torus_group(4))
    return g


@pytest.mark.parametrize("n", [5, 12, 31, 32, 33, 64])
def test_sorted_merge_matches_oracle(n):
    for group in groups_for(n):
        strings = rand_strings(n, 5000, seed=n * 10 + (group & 7), pool=1500)
        coef = np.random.default_rng(n + group).normal(size=len(strings))
        ox, oz, oc, x, z = device_merge(n, group, strings, coef)
        got = as_dict(ox, oz, oc)
        assert len(got) == len(oc)  # distinct keys
        want = oracle.OracleState(n, x, z, coef, group=group).as_dict()
        assert set(got) == set(want), group
        assert max(abs(got[k] - want[k]) for k in want) < 1e-12
        order = packed_order(n, ox, oz)
        assert order == sorted(order)
        # the hash merge finds the same strings
        hx, hz, hc, _, _ = device_merge(n, group, strings, coef, sorted_merge=False)
        assert set(as_dict(hx, hz, hc)) == set(got)


def lane_tree_sum(vals):
    """The documented order of a run longer than 64: 32 lane partials, then a
    butterfly (offsets 16, 8, 4, 2, 1); lane 0's value."""
    part = [0.0] * 32
    for lane in range(32):
        s = 0.0
        for j in range(lane, len(vals), 32):
            s = s + vals[j]
        part[lane] = s
    for o in (16, 8, 4, 2, 1):
        part = [part[lane] + part[lane ^ o] for lane in range(32)]
    return part[0]


def documented_sums(strings, coef):
    runs = {}
    for s, c in zip(strings, coef):
        runs.setdefault(s, []).append(float(c))
    out = {}
    for s, vals in runs.items():
        if len(vals) <= 64:
            acc = 0.0
            for v in vals:
                acc = acc + v
            out[s] = acc
        else:
            out[s] = lane_tree_sum(vals)
    return out


@pytest.mark.parametrize("n,m,pool", [(20, 9000, 40), (32, 5000, 2000), (48, 6000, 30)])
def test_sorted_merge_sums_in_documented_order_bitexact(n, m, pool):
    """Without a group, every run is one string; sums (short and long runs) must
    equal the documented order bit for bit, and two calls agree bit for bit."""
    strings = rand_strings(n, m, seed=7 + n, pool=pool)
    coef = np.random.default_rng(n).normal(size=m) * np.exp(np.random.default_rng(1).normal(size=m) * 3)
    ox, oz, oc, _, _ = device_merge(n, 0, strings, coef)
    got = dict(zip(pi.from_masks(ox, oz, n), oc.tolist()))
    want = documented_sums(strings, coef)
    assert set(got) == set(want)
    bad = [k for k in want if got[k] != want[k]]
    assert not bad, [(got[k], want[k]) for k in bad[:3]]
    ox2, oz2, oc2, _, _ = device_merge(n, 0, strings, coef)
    np.testing.assert_array_equal(ox2, ox)
    np.testing.assert_array_equal(oz2, oz)
    assert oc2.tobytes() == oc.tobytes()


@pytest.mark.parametrize("m", [1, 2, 2047, 2048, 2049, 4097])
def test_sorted_merge_ragged_sizes(m):
    n = 16
    strings = rand_strings(n, m, seed=m, pool=max(1, m // 3))
    coef = np.random.default_rng(m).normal(size=m)
    ox, oz, oc, x, z = device_merge(n, 0, strings, coef)
    want = documented_sums(strings, coef)
    assert dict(zip(pi.from_masks(ox, oz, n), oc.tolist())) == want


def test_sorted_merge_one_long_run_and_empty():
    import torch
    n = 64
    strings = ["XY" + "I" * (n - 2)] * 10000
    coef = np.random.default_rng(3).normal(size=len(strings))
    ox, oz, oc, _, _ = device_merge(n, 0, strings, coef)
    assert len(oc) == 1 and oc[0] == lane_tree_sum(coef.tolist())
    d = torch.zeros((0, 2), dtype=torch.int64, device="cuda")
    c = torch.zeros(0, dtype=torch.float64, device="cuda")
    assert pp.pp_merge_terms_sorted(n, 0, 0, d, c, d, c) == 0


def test_sorted_merge_sn_many_to_one():
    """S_64 maps every string with the same letter counts to one
    representative: long runs through the warp reduce."""
    n = 64
    strings = rand_strings(n, 20000, seed=5)
    coef = np.random.default_rng(5).normal(size=len(strings))
    ox, oz, oc, x, z = device_merge(n, 2, strings, coef)
    got = as_dict(ox, oz, oc)
    want = oracle.OracleState(n, x, z, coef, group=2).as_dict()
    assert set(got) == set(want) and len(want) <= math.comb(n + 3, 3)
    assert max(abs(got[k] - want[k]) for k in want) < 1e-11


def test_sorted_merge_rejects_wide_strings():
    import torch
    d = torch.zeros((4, 4), dtype=torch.int64, device="cuda")
    c = torch.zeros(4, dtype=torch.float64, device="cuda")
    with pytest.raises(pp.PPError) as e:
        pp.pp_merge_terms_sorted(65, 0, 4, d, c, d, c)
    assert e.value.status == 1


# ------------------------------------------------ contexts merging by sort

def run_both(wl, group, steps=None, **kw):
    n = wl.circuit.n
    ox, oz, oc = wl.observable.arrays()
    prop = pp.Propagator.from_workload(wl, symmetry=group, merge_method=pp.MERGE_SORT, **kw)
    st = oracle.OracleState(n, ox, oz, oc, group=group, eps=wl.eps, max_weight=wl.max_weight)
    L = len(wl.circuit.layers) if steps is None else steps
    for layer in reversed(range(L)):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        prop.apply_layer(gx, gz, th, boundary=True)
        st.apply_layer(gx, gz, th, wl.noise_mode, wl.noise_p, group=group)
        yield prop, st


def assert_close(prop, st, eps, atol=1e-12):
    g = as_dict(*prop.export())
    o = st.as_dict()
    for k in set(o) ^ set(g):
        v = o.get(k, g.get(k))
        assert eps > 0 and abs(abs(v) - eps) <= 1e-9 * eps, ("term sets differ", v)
    for k in set(g) & set(o):
        assert abs(g[k] - o[k]) <= atol, (g[k], o[k])


@pytest.mark.parametrize("n,steps,eps,wmax", [(8, 4, 0.0, -1), (12, 4, 1e-4, 6), (33, 2, 1e-3, 5),
                                              (64, 2, 1e-3, 4)])
def test_context_zn_sort_merge_matches_oracle(n, steps, eps, wmax):
    wl = pi.config1_ring(n=n, steps=steps, eps=eps, max_weight=wmax, symmetry=1)
    for prop, st in run_both(wl, 1):
        assert_close(prop, st, eps)
        assert prop.expect(wl.state.bloch) == pytest.approx(st.expect(wl.state.bloch), abs=1e-10)


def test_context_sn_sort_merge_matches_oracle():
    n = 7
    wl = pi.config0_heisenberg(n=n, dt=0.05, steps=2)
    wl.observable = pi.mean_z(n)
    wl.state = pi.neel_state(n)
    for prop, st in run_both(wl, 2):
        assert_close(prop, st, 0.0)
        assert prop.expect(wl.state.bloch) == pytest.approx(st.expect(wl.state.bloch), abs=1e-10)


def test_context_sort_merge_with_table_growth():
    """From a one-entry table the first layers outgrow their room (the table is
    regrown, and a gate may stop for capacity and resume); every queued sorted
    merge still matches the oracle."""
    n = 24
    wl = pi.config1_ring(n=n, steps=4, eps=1e-6, max_weight=-1, symmetry=1)
    for prop, st in run_both(wl, 1):
        assert_close(prop, st, wl.eps)
    assert prop.stats()["regrows"] > 0


def test_context_sort_and_hash_merges_agree_on_ring32():
    """Eight Trotter steps of the ring workload at n = 32 (over 10^4
    representatives), merged by sort and by hash: the same strings and
    coefficients within 1e-12."""
    wl = pi.config1_ring(n=32, steps=8, symmetry=1)
    out = []
    for method in (pp.MERGE_SORT, pp.MERGE_HASH):
        prop = pp.Propagator.from_workload(wl, symmetry=1, merge_method=method)
        val = prop.run(wl)
        out.append((as_dict(*prop.export()), val))
        prop.close()
    (a, va), (b, vb) = out
    assert set(a) == set(b) and len(a) > 1000
    assert max(abs(a[k] - b[k]) for k in a) < 1e-12
    assert va == pytest.approx(vb, abs=1e-12)


@pytest.mark.parametrize("f32", [False, True])
def test_batched_rows_sort_merge(f32):
    n, B = 12, 16
    angles = pi.batched_ring_angles(B, 2)
    gx, gz, _ = pi.Circuit(n, [pi.ring_layer(n, 0.0, 0.0, 0.0)]).gate_arrays(0)
    th = np.zeros((3 * n, B))
    th[:n], th[n:2 * n], th[2 * n:] = angles[:, 0], angles[:, 1], angles[:, 2]
    x, z, c = pi.mean_z(n).arrays()
    coef = np.repeat(c[:, None], B, axis=1)
    eps = 0.0 if f32 else 1e-4
    prop = pp.Propagator(n, x, z, coef, symmetry=1, eps=eps, max_weight=5, batch=B, f32=f32,
                         merge_method=pp.MERGE_SORT)
    st = oracle.BatchedOracleState(n, B, x, z, coef, group=1, eps=eps, max_weight=5)
    for _ in range(3):
        prop.apply_layer(gx, gz, th, boundary=True)
        st.apply_layer(gx, gz, th, group=1)
    gxo, gzo, gc = prop.export()
    oxo, ozo, oc = st.export()
    g = {tuple(int(v) for v in gxo[i]) + tuple(int(v) for v in gzo[i]): gc[i] for i in range(len(gc))}
    o = {tuple(int(v) for v in oxo[i]) + tuple(int(v) for v in ozo[i]): oc[i] for i in range(len(oc))}
    assert set(g) == set(o) and len(o) > 10
    tol = 1e-5 if f32 else 1e-12
    assert max(float(np.max(np.abs(g[k] - o[k]))) for k in o) < tol
    bloch = pi.neel_state(n).bloch
    got, want = prop.expect(bloch), st.expect(bloch)
    assert np.all(np.abs(got - want) <= (1e-5 * np.abs(want) + 1e-6 if f32 else 1e-10))
