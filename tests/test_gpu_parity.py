"""CUDA path vs the CPU oracle, through the C ABI (needs a GB300).

Tolerances (see also the module docstring of tests/parity_util.py):
* Gates only (no symmetry merge): each coefficient is updated by exactly one
  thread as cos*c_Q +- sin*c_R in FP64 without FMA, the same operations the
  oracle performs, so term sets AND coefficients must be bit-identical, with
  or without truncation.
* Symmetry / identical-string merges sum coefficients with FP64 atomics in a
  run-dependent order: coefficients within 1e-12 absolute, term sets equal
  (a term whose oracle |c| is within 1e-9 relative of eps may flip).
* Expectation values: 1e-10 absolute (FP64 target).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import paper_2512_12094_gb300 as pp
import pp_inputs as pi
from oracle import statevector as sv

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


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


def run_both(wl, group, steps=None, **gpu_kw):
    """Propagate wl layer by layer on GPU and in the oracle; yield both states."""
    n = wl.circuit.n
    ox, oz, oc = wl.observable.arrays()
    prop = pp.Propagator.from_workload(wl, symmetry=group, **gpu_kw)
    st = oracle.OracleState(n, ox, oz, oc, group=group, eps=wl.eps, max_weight=wl.max_weight)
    L = len(wl.circuit.layers) if steps is None else steps
    for layer in reversed(range(L)):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        prop.apply_layer(gx, gz, th, boundary=True)
        st.apply_layer(gx, gz, th, wl.noise_mode, wl.noise_p, group=group)
        yield prop, st


def assert_bitexact(prop, st):
    g = as_dict(*prop.export())
    o = st.as_dict()
    assert set(g) == set(o)
    bad = [k for k in o if not (g[k] == o[k])]
    assert not bad, (len(bad), [(g[k], o[k]) for k in bad[:5]])


def assert_close(prop, st, eps, atol=1e-12):
    g = as_dict(*prop.export())
    o = st.as_dict()
    only_g = set(g) - set(o)
    only_o = set(o) - set(g)
    for k in only_o:
        assert eps > 0 and abs(abs(o[k]) - eps) <= 1e-9 * eps, ("missing", o[k])
    for k in only_g:
        assert eps > 0 and abs(abs(g[k]) - eps) <= 1e-9 * eps, ("extra", g[k])
    for k in set(g) & set(o):
        assert abs(g[k] - o[k]) <= atol, (g[k], o[k])


# ------------------------------------------------------------ gates only

def test_heisenberg_n8_bitexact_each_step():
    wl = pi.config0_heisenberg(n=8, dt=0.05, steps=3)
    ref = sv.statevector_expectations(wl.circuit.layers, wl.observable.terms, wl.state.bloch)
    gold = json.load(open(os.path.join(GOLDEN, "heisenberg_a2a_n8.json")))["plain"]
    for k, (prop, st) in enumerate(run_both(wl, 0)):
        assert_bitexact(prop, st)
        e = prop.expect(wl.state.bloch)
        assert e == pytest.approx(st.expect(wl.state.bloch), abs=1e-12)
        assert e == pytest.approx(ref[k], abs=1e-10)
        assert prop.num_terms()[0] == gold[k]["terms"]
        assert e == pytest.approx(gold[k]["expect"], abs=1e-12)


@pytest.mark.parametrize("n", [5, 63, 64, 65, 130, 256])
@pytest.mark.parametrize("noise", [0, 1, 2])
def test_random_circuits_bitexact(n, noise):
    seed = 1000 * n + noise
    circ = pi.random_circuit(n, n_layers=3, gates_per_layer=12, seed=seed, max_support=4)
    obs = pi.random_observable(n, 40, seed=seed + 1, max_weight=4)
    wl = pi.Workload("rand", circ, obs, pi.random_product_state(n, seed + 2),
                     noise_p=0.05 if noise else 0.0, noise_mode=noise)
    for prop, st in run_both(wl, 0):
        assert_bitexact(prop, st)
    assert prop.expect(wl.state.bloch) == pytest.approx(st.expect(wl.state.bloch), abs=1e-12)


@pytest.mark.parametrize("eps,wmax", [(1e-3, -1), (0.0, 3), (2e-3, 4)])
def test_truncation_bitexact(eps, wmax):
    n = 20
    circ = pi.random_circuit(n, n_layers=4, gates_per_layer=25, seed=7, max_support=3)
    obs = pi.random_observable(n, 30, seed=8, max_weight=3)
    wl = pi.Workload("trunc", circ, obs, pi.zero_state(n), eps=eps, max_weight=wmax)
    for prop, st in run_both(wl, 0):
        assert_bitexact(prop, st)


@pytest.mark.parametrize("symmetry", [0, 1])
def test_launch_paths_agree(symmetry):
    """Cooperative layer kernel (blocks of 256 and of 1024 threads), per-gate
    kernels from CUDA graphs (PDL) and per-gate direct launches give
    bit-identical tables and the same update
    statistics (live terms and live anticommuting terms entering each gate,
    counted from values before the gate, so no path depends on timing)."""
    wl = pi.config1_ring(n=32 if symmetry == 0 else 16, steps=5, eps=1e-4 if symmetry == 0 else 1e-5,
                         max_weight=10 if symmetry == 0 else 8)
    runs, stats = [], []
    for kw in (dict(layer_kernel=True, block_threads=256), dict(layer_kernel=False, use_graphs=True),
               dict(layer_kernel=False, use_graphs=False), dict(layer_kernel=True, block_threads=1024)):
        p = pp.Propagator.from_workload(wl, symmetry=symmetry, **kw)
        p.run(wl)
        runs.append(as_dict(*p.export()))
        st = p.stats()
        stats.append((st["gate_updates"], st["anticommuting_terms"]))
        p.close()
    assert len(set(stats)) == 1, stats
    if symmetry == 0:
        assert runs[0] == runs[1] == runs[2] == runs[3]
    else:  # merges sum with atomics: same keys, coefficients to rounding
        for r in runs[1:]:
            assert set(r) == set(runs[0])
            assert max(abs(r[k] - runs[0][k]) for k in r) < 1e-13


def test_ring_n32_plain_full_matches_oracle_trajectory():
    """The full translation-symmetric ring workload (n=32, 20 steps, eps=1e-4,
    weight <= 10), plain propagation, as timed by bench.py: per-step live
    terms must equal the oracle's and <O> agree to 1e-10."""
    gold = json.load(open(os.path.join(GOLDEN, "ring_n32.json")))["plain"]
    wl = pi.config1_ring()
    prop = pp.Propagator.from_workload(wl, symmetry=0)
    vals = prop.run(wl, record_each_step=True)
    # run() records after every layer; compare counts at the end too
    for k, row in enumerate(gold):
        assert vals[k] == pytest.approx(row["expect"], abs=1e-10)
    assert prop.num_terms()[0] == gold[-1]["terms"]
    assert prop.stats()["gate_updates"] == gold[-1]["updates"]


# ------------------------------------------------------- symmetry merges

@pytest.mark.parametrize("n,steps,eps,wmax", [(8, 4, 0.0, -1), (12, 4, 1e-4, 6), (33, 2, 1e-3, 5)])
def test_ring_zn_merge_matches_oracle(n, steps, eps, wmax):
    wl = pi.config1_ring(n=n, steps=steps, eps=eps, max_weight=wmax, symmetry=1)
    for prop, st in run_both(wl, 1):
        assert_close(prop, st, eps)
        assert prop.expect(wl.state.bloch) == pytest.approx(st.expect(wl.state.bloch), abs=1e-10)


@pytest.mark.parametrize("state", ["neel", "plus"])
def test_a2a_sn_merge_matches_oracle(state):
    n = 7
    wl = pi.config0_heisenberg(n=n, dt=0.05, steps=2)
    wl.observable = pi.mean_z(n)
    wl.state = pi.neel_state(n) if state == "neel" else pi.plus_state(n)
    for prop, st in run_both(wl, 2):
        assert_close(prop, st, 0.0)
        assert prop.expect(wl.state.bloch) == pytest.approx(st.expect(wl.state.bloch), abs=1e-10)
    assert prop.num_terms()[0] <= math.comb(n + 3, 3)


def test_theorem1_merged_equals_plain_on_gpu():
    n = 8
    wl = pi.config1_ring(n=n, steps=3, eps=0.0, max_weight=-1)
    plain = pp.Propagator.from_workload(wl, symmetry=0).run(wl, record_each_step=True)
    merged = pp.Propagator.from_workload(wl, symmetry=1).run(wl, record_each_step=True)
    np.testing.assert_allclose(merged, plain, atol=1e-12, rtol=0)
    ref = sv.statevector_expectations(wl.circuit.layers, wl.observable.terms, wl.state.bloch)
    np.testing.assert_allclose(plain, ref, atol=1e-10, rtol=0)


def test_ring_n32_zn_full_matches_oracle_trajectory():
    data = json.load(open(os.path.join(GOLDEN, "ring_n32.json")))
    if "zn" not in data:
        pytest.skip("merged trajectory not stored")
    gold = data["zn"]
    wl = pi.config1_ring(symmetry=1)
    prop = pp.Propagator.from_workload(wl, symmetry=1)
    vals = prop.run(wl, steps=len(gold), record_each_step=True)
    for k, row in enumerate(gold):
        assert vals[k] == pytest.approx(row["expect"], abs=1e-10)
    assert prop.num_terms()[0] == gold[-1]["terms"]


@pytest.mark.parametrize("group", [1, 2])
def test_ingest_merges_by_representative(group):
    n = 10
    x, z, c = pi.random_observable(n, 3000, seed=3).arrays()
    h = pp.pp_create(pp.pp_config_default(n_qubits=n, symmetry=group), x, z, c)
    got = as_dict(*pp.pp_export(h, n))
    want = oracle.OracleState(n, x, z, c, group=group).as_dict()
    pp.pp_destroy(h)
    assert set(got) == set(want)
    assert max(abs(got[k] - want[k]) for k in want) < 1e-12


@pytest.mark.parametrize("group", [1, 2])
def test_explicit_canonicalize_and_merge_calls(group):
    """A layer applied without the boundary merge leaves non-representative
    strings; pp_canonicalize + pp_merge must then equal the oracle's merge."""
    n = 8
    if group == 1:
        wl = pi.config1_ring(n=n, steps=2, eps=0.0, max_weight=-1)
    else:
        wl = pi.config0_heisenberg(n=n, dt=0.05, steps=2)
        wl.observable = pi.mean_z(n)
    x, z, c = wl.observable.arrays()
    h = pp.pp_create(pp.pp_config_default(n_qubits=n, symmetry=group), x, z, c)
    st = oracle.OracleState(n, x, z, c, group=group)
    gx, gz, th = wl.circuit.gate_arrays(0)
    pp.pp_apply_layer(h, pp.pack_gates(gx, gz), th, False)
    st.apply_layer(gx, gz, th, group=0)
    assert as_dict(*pp.pp_export(h, n)) == st.as_dict()  # gates only: bit-exact
    pp.pp_canonicalize(h)
    pp.pp_merge(h)
    st.symmetry_merge(group)
    got = as_dict(*pp.pp_export(h, n))
    want = st.as_dict()
    pp.pp_destroy(h)
    assert set(got) == set(want)
    assert max(abs(got[k] - want[k]) for k in want) < 1e-12


def test_truncate_call_matches_oracle():
    n = 12
    obs = pi.random_observable(n, 5000, seed=5)
    x, z, c = obs.arrays()
    h = pp.pp_create(pp.pp_config_default(n_qubits=n), x, z, c)
    pp.pp_truncate(h, 0.5, 7)
    st = oracle.OracleState(n, x, z, c)
    st.truncate(0.5, 7)
    assert as_dict(*pp.pp_export(h, n)) == st.as_dict()
    pp.pp_destroy(h)


# --------------------------------------------------- stateless entry points

def _rand_keys(n, m, seed, periodic=False):
    rng = np.random.default_rng(seed)
    W = (n + 63) // 64
    strings = []
    for i in range(m):
        if periodic and n % 4 == 0:
            block = "".join(rng.choice(list("IXYZ"), size=4))
            s = block * (n // 4)
        else:
            w = int(rng.integers(0, n + 1)) if i % 2 else int(rng.integers(0, min(n, 6) + 1))
            letters = ["I"] * n
            for q in rng.choice(n, size=w, replace=False):
                letters[q] = "XYZ"[int(rng.integers(0, 3))]
            s = "".join(letters)
        strings.append(s)
    x, z = pi.to_masks(strings, n)
    keys = np.concatenate([x, z], axis=1)  # [m][2W]
    return x, z, np.ascontiguousarray(keys), W


@pytest.mark.parametrize("n", [1, 2, 3, 8, 31, 32, 33, 63, 64, 65, 100, 128, 200, 256])
@pytest.mark.parametrize("group", [1, 2])
def test_canonical_keys_bitexact(n, group):
    import torch
    x, z, keys, W = _rand_keys(n, 600, seed=n * 7 + group, periodic=(n % 8 == 0))
    d_in = torch.from_numpy(keys.view(np.int64)).cuda()
    d_out = torch.empty_like(d_in)
    pp.pp_canonical_keys(n, group, len(keys), d_in, d_out)
    torch.cuda.synchronize()
    got = d_out.cpu().numpy().view(np.uint64)
    ox, oz = oracle.canonical(n, group, x, z)
    np.testing.assert_array_equal(got[:, :W], ox)
    np.testing.assert_array_equal(got[:, W:], oz)


def test_orbit_counts_on_gpu():
    import itertools
    import torch
    n = 8
    strings = ["".join(t) for t in itertools.product("IXYZ", repeat=n)]
    x, z = pi.to_masks(strings, n)
    keys = np.ascontiguousarray(np.concatenate([x, z], axis=1))
    d_in = torch.from_numpy(keys.view(np.int64)).cuda()
    for group, want in ((1, 8230), (2, math.comb(n + 3, 3))):
        d_out = torch.empty_like(d_in)
        pp.pp_canonical_keys(n, group, len(keys), d_in, d_out)
        got = d_out.cpu().numpy()
        assert len({tuple(r) for r in got.tolist()}) == want


@pytest.mark.parametrize("n,group", [(10, 0), (10, 1), (10, 2), (70, 1), (70, 2)])
def test_merge_terms_matches_oracle(n, group):
    import torch
    x, z, keys, W = _rand_keys(n, 5000, seed=n + group)
    coef = np.random.default_rng(1).normal(size=len(keys))
    d_k = torch.from_numpy(keys.view(np.int64)).cuda()
    d_c = torch.from_numpy(coef).cuda()
    out_k = torch.empty_like(d_k)
    out_c = torch.empty_like(d_c)
    m = pp.pp_merge_terms(n, group, len(keys), d_k, d_c, out_k, out_c)
    ok = out_k[:m].cpu().numpy().view(np.uint64)
    oc = out_c[:m].cpu().numpy()
    got = as_dict(ok[:, :W], ok[:, W:], oc)
    want = oracle.OracleState(n, x, z, coef, group=group).as_dict()
    assert set(got) == set(want)
    assert max(abs(got[k] - want[k]) for k in want) < 1e-12


@pytest.mark.parametrize("n,group", [(6, 0), (6, 1), (6, 2), (40, 1), (40, 2), (90, 0), (90, 1)])
def test_overlap_sum_matches_oracle(n, group):
    import torch
    x, z, keys, W = _rand_keys(n, 3000, seed=n * 3 + group)
    coef = np.random.default_rng(2).normal(size=len(keys))
    st = pi.random_product_state(n, 9)
    d_k = torch.from_numpy(keys.view(np.int64)).cuda()
    d_c = torch.from_numpy(coef).cuda()
    d_b = torch.from_numpy(np.ascontiguousarray(st.bloch.reshape(-1))).cuda()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    pp.pp_overlap_sum(n, group, len(keys), d_k, d_c, d_b, out)
    got = float(out.cpu()[0])
    want = float(np.dot(coef, oracle.sym_overlap(n, group, x, z, st.bloch)))
    assert got == pytest.approx(want, abs=1e-10)


# ------------------------------------------------------------ edge cases

def test_empty_observable():
    n = 8
    cfg = pp.pp_config_default(n_qubits=n)
    h = pp.pp_create(cfg, np.zeros((0, 1)), np.zeros((0, 1)), np.zeros(0))
    wl = pi.config1_ring(n=n, steps=1)
    gx, gz, th = wl.circuit.gate_arrays(0)
    pp.pp_apply_layer(h, pp.pack_gates(gx, gz), th, True)
    assert pp.pp_expect(h, pi.zero_state(n).bloch) == 0.0
    assert pp.pp_num_terms(h) == (0, 0)
    pp.pp_destroy(h)


def test_single_qubit_and_identity_terms():
    n = 1
    x, z = pi.to_masks(["Z", "I"], 1)
    h = pp.pp_create(pp.pp_config_default(n_qubits=1), x, z, np.array([1.0, 0.25]))
    th = np.array([0.7, 0.0])
    gx, gz = pi.to_masks(["X", "I"], 1)  # second gate is the identity generator
    pp.pp_apply_layer(h, pp.pack_gates(gx, gz), th, False)
    got = dict(zip(pi.from_masks(*pp.pp_export(h, 1)[:2], 1), pp.pp_export(h, 1)[2]))
    assert got["I"] == 0.25
    assert got["Z"] == math.cos(0.7) and got["Y"] == math.sin(0.7)
    pp.pp_destroy(h)


def test_rejects_bits_beyond_n():
    x = np.array([[1 << 5]], dtype=np.uint64)
    with pytest.raises(pp.PPError) as e:
        pp.pp_create(pp.pp_config_default(n_qubits=5), x, np.zeros((1, 1)), np.ones(1))
    assert e.value.status == 1


def test_budget_exceeded_is_a_clean_error():
    wl = pi.config1_ring(n=32, steps=20)
    prop = pp.Propagator.from_workload(wl, symmetry=0, budget=6 << 20)
    with pytest.raises(pp.PPError) as e:
        prop.run(wl)
    assert e.value.status == 3
    live, stored = prop.num_terms()  # context still usable
    assert live >= 0 and stored >= live
    prop.expect(wl.state.bloch)


def test_symmetry_checks():
    n = 8
    wl = pi.config1_ring(n=n, steps=1)
    prop = pp.Propagator.from_workload(wl, symmetry=2)  # ring layer is not S_n-invariant
    gx, gz, th = wl.circuit.gate_arrays(0)
    with pytest.raises(pp.PPError) as e:
        prop.apply_layer(gx, gz, th)
    assert e.value.status == 4
    # Z_0 is not Z_n-invariant and neither is the Neel state
    x, z = pi.to_masks([pi.pauli(n, {0: "Z"})], n)
    p2 = pp.Propagator(n, x, z, np.ones(1), symmetry=1)
    p2.apply_layer(gx, gz, th)
    with pytest.raises(pp.PPError) as e:
        p2.expect(pi.neel_state(n).bloch)
    assert e.value.status == 4
    p2.expect(pi.zero_state(n).bloch)  # invariant state is fine


def test_regrow_from_tiny_capacity():
    wl = pi.config1_ring(n=24, steps=6, eps=1e-6, max_weight=-1)
    prop = pp.Propagator.from_workload(wl, symmetry=0)
    ox, oz, oc = wl.observable.arrays()
    st = oracle.OracleState(24, ox, oz, oc, eps=wl.eps, max_weight=wl.max_weight)
    for layer in reversed(range(6)):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        prop.apply_layer(gx, gz, th)
        st.apply_layer(gx, gz, th)
    assert prop.stats()["regrows"] > 0
    assert_bitexact(prop, st)
