"""Dihedral (D_n) and torus-translation groups: CUDA path vs the oracle.

Representatives are integer work, so they must match bit for bit, including
strings with a nontrivial stabiliser (palindromes, strings periodic along a
ring or along torus rows and columns), at one to four words per mask.
Merges and overlaps sum in FP64 (merges with atomics): coefficients within
1e-12, <O> within 1e-10.  Propagation with merging is compared step by step,
and without truncation it must equal the unmerged run (Theorem 1).
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
    if len(c) == 0:
        return {}
    x = np.asarray(x).reshape(len(c), -1)
    z = np.asarray(z).reshape(len(c), -1)
    d = {tuple(int(v) for v in x[i]) + tuple(int(v) for v in z[i]): c[i] for i in range(len(c))}
    assert len(d) == len(c), "a string appears twice in the table"
    return d


def strings_for(n, m, seed, lx=None):
    """Random strings of every weight, plus strings with a stabiliser:
    palindromes and period-4 rings (D_n), or rows or columns repeated (torus)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(m):
        kind = i % 4
        if kind == 0:
            w = int(rng.integers(0, n + 1))
        else:
            w = int(rng.integers(0, min(n, 6) + 1))
        letters = ["I"] * n
        for q in rng.choice(n, size=w, replace=False):
            letters[q] = "XYZ"[int(rng.integers(0, 3))]
        if kind == 2:
            if lx is None:
                half = letters[:(n + 1) // 2]
                letters = half + half[:n // 2][::-1]           # palindrome
            else:
                letters = letters[:lx] * (n // lx)             # every row the same
        elif kind == 3:
            if lx is None and n % 4 == 0:
                letters = letters[:4] * (n // 4)               # period 4 on the ring
            elif lx is not None:
                ly = n // lx
                col = [letters[lx * y] for y in range(ly)]
                letters = [col[q // lx] for q in range(n)]     # every column the same
        out.append("".join(letters))
    return out


def keys_of(strings, n):
    x, z = pi.to_masks(strings, n)
    return x, z, np.ascontiguousarray(np.concatenate([x, z], axis=1)), (n + 63) // 64


DN_SIZES = [2, 3, 5, 8, 31, 32, 33, 63, 64, 65, 100, 128, 200, 256]
TORI = [(2, 2), (4, 3), (3, 4), (8, 4), (4, 8), (6, 6), (8, 8), (16, 4), (5, 13), (10, 10),
        (16, 8), (12, 12), (16, 16)]


def canonical_on_gpu(n, code, keys):
    import torch
    d_in = torch.from_numpy(keys.view(np.int64)).cuda()
    d_out = torch.empty_like(d_in)
    pp.pp_canonical_keys(n, code, len(keys), d_in, d_out)
    torch.cuda.synchronize()
    return d_out.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("n", DN_SIZES)
def test_dihedral_canonical_keys_bitexact(n):
    x, z, keys, W = keys_of(strings_for(n, 400, seed=n), n)
    got = canonical_on_gpu(n, pp.SYM_DN, keys)
    ox, oz = oracle.canonical(n, oracle.DN, x, z)
    np.testing.assert_array_equal(got[:, :W], ox)
    np.testing.assert_array_equal(got[:, W:], oz)


@pytest.mark.parametrize("lx,ly", TORI)
def test_torus_canonical_keys_bitexact(lx, ly):
    n = lx * ly
    x, z, keys, W = keys_of(strings_for(n, 300, seed=n + lx, lx=lx), n)
    got = canonical_on_gpu(n, pp.sym_torus(lx), keys)
    ox, oz = oracle.canonical(n, oracle.torus_group(lx), x, z)
    np.testing.assert_array_equal(got[:, :W], ox)
    np.testing.assert_array_equal(got[:, W:], oz)


def test_orbit_counts_on_gpu():
    """All 4^n strings: the number of distinct GPU representatives is the
    orbit count (4-colour bracelets of 6 beads; 3 x 2 torus)."""
    import itertools
    for n, code, want in ((6, pp.SYM_DN, 430), (6, pp.sym_torus(3), 700)):
        strings = ["".join(t) for t in itertools.product("IXYZ", repeat=n)]
        _, _, keys, _ = keys_of(strings, n)
        got = canonical_on_gpu(n, code, keys)
        assert len({tuple(r) for r in got.tolist()}) == want


@pytest.mark.parametrize("n,code,ocode", [(10, pp.SYM_DN, oracle.DN), (70, pp.SYM_DN, oracle.DN),
                                          (12, pp.sym_torus(4), oracle.torus_group(4)),
                                          (80, pp.sym_torus(8), oracle.torus_group(8))])
def test_merge_and_overlap_match_oracle(n, code, ocode):
    import torch
    lx = (code >> 8) or None
    x, z, keys, W = keys_of(strings_for(n, 3000, seed=n, lx=lx), n)
    coef = np.random.default_rng(1).normal(size=len(keys))
    d_k = torch.from_numpy(keys.view(np.int64)).cuda()
    d_c = torch.from_numpy(coef).cuda()
    out_k = torch.empty_like(d_k)
    out_c = torch.empty_like(d_c)
    m = pp.pp_merge_terms(n, code, len(keys), d_k, d_c, out_k, out_c)
    ok = out_k[:m].cpu().numpy().view(np.uint64)
    got = as_dict(ok[:, :W], ok[:, W:], out_c[:m].cpu().numpy())
    want = oracle.OracleState(n, x, z, coef, group=ocode).as_dict()
    assert set(got) == set(want)
    assert max(abs(got[k] - want[k]) for k in want) < 1e-12
    st = pi.random_product_state(n, 9)  # not invariant: the orbit average is taken
    d_b = torch.from_numpy(np.ascontiguousarray(st.bloch.reshape(-1))).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    pp.pp_overlap_sum(n, code, len(keys), d_k, d_c, d_b, out)
    ref = float(np.dot(coef, oracle.sym_overlap(n, ocode, x, z, st.bloch)))
    assert float(out.cpu()[0]) == pytest.approx(ref, abs=1e-10)


def run_both(wl, code, ocode, **kw):
    n = wl.circuit.n
    ox, oz, oc = wl.observable.arrays()
    prop = pp.Propagator.from_workload(wl, symmetry=code, **kw)
    st = oracle.OracleState(n, ox, oz, oc, group=ocode, eps=wl.eps, max_weight=wl.max_weight)
    for layer in reversed(range(len(wl.circuit.layers))):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        prop.apply_layer(gx, gz, th, boundary=True)
        st.apply_layer(gx, gz, th, wl.noise_mode, wl.noise_p, group=ocode)
        yield prop, st


def assert_close(prop, st, eps, atol=1e-12):
    g = as_dict(*prop.export())
    o = st.as_dict()
    for k in set(o) - set(g):
        assert eps > 0 and abs(abs(o[k]) - eps) <= 1e-9 * eps, ("missing", o[k])
    for k in set(g) - set(o):
        assert eps > 0 and abs(abs(g[k]) - eps) <= 1e-9 * eps, ("extra", g[k])
    for k in set(g) & set(o):
        assert abs(g[k] - o[k]) <= atol, (g[k], o[k])


@pytest.mark.parametrize("n,eps,wmax,state", [(12, 1e-4, 6, "zero"), (33, 1e-3, 5, "neel"),
                                              (70, 1e-3, 4, "random")])
def test_dihedral_ring_propagation_matches_oracle(n, eps, wmax, state):
    wl = pi.config1_ring(n=n, steps=3, eps=eps, max_weight=wmax)
    wl.state = {"zero": pi.zero_state(n), "neel": pi.neel_state(n),
                "random": pi.random_product_state(n, 4)}[state]
    for prop, st in run_both(wl, pp.SYM_DN, oracle.DN):
        assert_close(prop, st, eps)
        assert float(prop.expect(wl.state.bloch)) == pytest.approx(
            st.expect(wl.state.bloch, oracle.DN), abs=1e-10)
    prop.close()


@pytest.mark.parametrize("lx,ly,eps,wmax", [(4, 3, 1e-4, 6), (8, 8, 1e-3, 4), (10, 8, 1e-3, 4)])
def test_torus_propagation_matches_oracle(lx, ly, eps, wmax):
    wl = pi.torus_ising(lx, ly, steps=2, eps=eps, max_weight=wmax)
    n = lx * ly
    for state in (pi.zero_state(n), pi.random_product_state(n, 6)):
        wl.state = state
        for prop, st in run_both(wl, pp.sym_torus(lx), oracle.torus_group(lx)):
            assert_close(prop, st, eps)
            assert float(prop.expect(state.bloch)) == pytest.approx(
                st.expect(state.bloch, oracle.torus_group(lx)), abs=1e-10)
        prop.close()


@pytest.mark.parametrize("kind", ["dn", "torus"])
def test_theorem1_merged_equals_plain_on_gpu(kind):
    """No truncation, exactly symmetric layers: the merged operator gives the
    unmerged expectation, also on a state that is not invariant (through the
    group-averaged overlap)."""
    if kind == "dn":
        wl, code = pi.config1_ring(n=8, steps=3, eps=0.0, max_weight=-1), pp.SYM_DN
    else:
        wl, code = pi.torus_ising(3, 3, steps=2), pp.sym_torus(3)
    plain = pp.Propagator.from_workload(wl, symmetry=0)
    merged = pp.Propagator.from_workload(wl, symmetry=code)
    plain.run(wl)
    merged.run(wl)
    for state in (wl.state, pi.random_product_state(wl.circuit.n, 12)):
        np.testing.assert_allclose(float(merged.expect(state.bloch)),
                                   float(plain.expect(state.bloch)), atol=1e-12, rtol=0)
    assert merged.num_terms()[0] < plain.num_terms()[0]
    plain.close()
    merged.close()


def test_batched_dihedral_merge_matches_batched_oracle():
    n, B = 12, 8
    angles = pi.batched_ring_angles(B, 3)
    layer = pi.ring_layer(n, 0.0, 0.0, 0.0)
    gx, gz, _ = pi.Circuit(n, [layer]).gate_arrays(0)
    th = np.zeros((3 * n, B))
    th[:n] = angles[:, 0]
    th[n:2 * n] = angles[:, 1]
    th[2 * n:] = angles[:, 2]
    x, z, c = pi.mean_z(n).arrays()
    coef = np.repeat(c[:, None], B, axis=1)
    prop = pp.Propagator(n, x, z, coef, symmetry=pp.SYM_DN, eps=1e-4, max_weight=5, batch=B)
    st = oracle.BatchedOracleState(n, B, x, z, coef, group=oracle.DN, eps=1e-4, max_weight=5)
    for _ in range(3):
        prop.apply_layer(gx, gz, th, True)
        st.apply_layer(gx, gz, th, group=oracle.DN)
    g = as_dict(*prop.export())
    o = as_dict(*st.export())
    assert set(g) == set(o)
    for k in o:
        np.testing.assert_allclose(g[k], o[k], atol=1e-12, rtol=0)
    bloch = pi.random_product_state(n, 2).bloch
    np.testing.assert_allclose(prop.expect(bloch), st.expect(bloch), atol=1e-10, rtol=0)
    prop.close()


def test_layers_that_break_the_group_are_rejected():
    n = 8
    # X_i Y_{i+1} on every bond: invariant under translations, not reflections
    chiral = [(pi.pauli(n, {i: "X", (i + 1) % n: "Y"}), 0.3) for i in range(n)]
    gx, gz, th = pi.Circuit(n, [chiral]).gate_arrays(0)
    x, z, c = pi.mean_z(n).arrays()
    zn = pp.Propagator(n, x, z, c, symmetry=pp.SYM_ZN)
    zn.apply_layer(gx, gz, th, True)
    dn = pp.Propagator(n, x, z, c, symmetry=pp.SYM_DN)
    with pytest.raises(pp.PPError) as e:
        dn.apply_layer(gx, gz, th, True)
    assert e.value.status == 4  # PP_ERR_SYMMETRY
    # the ring layer on 4 x 2 sites is not invariant under torus translations
    ring = pi.ring_layer(n, 0.4, 0.6, 0.3)
    gx, gz, th = pi.Circuit(n, [ring]).gate_arrays(0)
    tor = pp.Propagator(n, x, z, c, symmetry=pp.sym_torus(4))
    with pytest.raises(pp.PPError) as e:
        tor.apply_layer(gx, gz, th, True)
    assert e.value.status == 4
    for p in (zn, dn, tor):
        p.close()
