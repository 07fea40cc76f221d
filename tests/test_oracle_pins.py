"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Every check here compares the oracle with something other than itself: a
dense state-vector or density-matrix simulation, a matrix exponential, a
closed form, a count given by Burnside's lemma, the paper's printed example,
or brute force over group elements.  No GPU is used.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import pp_inputs as pi
from oracle import statevector as sv

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _single(oracle_lib, n, q_string, gates, noise_mode=0, p=0.0, eps=0.0, wmax=-1):
    x, z = pi.to_masks([q_string], n)
    st = oracle_lib.OracleState(n, x, z, np.array([1.0]), eps=eps, max_weight=wmax)
    for s, th in gates:  # Heisenberg order: caller passes gates last-to-first
        gx, gz = pi.to_masks([s], n)
        st.apply_gate(gx[0], gz[0], th, noise_mode, p)
    x, z, c = st.export()
    return dict(zip(pi.from_masks(x, z, n), c))


# ------------------------------------------------ single-gate closed forms
# App. A / Prop. 1 proof, read with U = exp(-i theta P / 2):
# U^dag Q U = cos(theta) Q + sin(theta) (i P Q) for anticommuting P, Q.

@pytest.mark.parametrize("theta", [0.3, -1.1, 2.5])
def test_rz_on_x(oracle_lib, theta):
    out = _single(oracle_lib, 1, "X", [("Z", theta)])
    assert out["X"] == pytest.approx(math.cos(theta), abs=1e-15)
    assert out["Y"] == pytest.approx(-math.sin(theta), abs=1e-15)


@pytest.mark.parametrize("theta", [0.3, -1.1, 2.5])
def test_rx_on_z_and_y(oracle_lib, theta):
    out = _single(oracle_lib, 1, "Z", [("X", theta)])
    assert out["Z"] == pytest.approx(math.cos(theta), abs=1e-15)
    assert out["Y"] == pytest.approx(math.sin(theta), abs=1e-15)
    out = _single(oracle_lib, 1, "Y", [("X", theta)])
    assert out["Y"] == pytest.approx(math.cos(theta), abs=1e-15)
    assert out["Z"] == pytest.approx(-math.sin(theta), abs=1e-15)


@pytest.mark.parametrize("n,q", [(70, 67), (130, 129)])
def test_rz_on_x_beyond_the_first_mask_word(oracle_lib, n, q):
    """The same closed form on a qubit held in the second or third 64-bit
    word of the masks: strings of more than 64 qubits take several words."""
    theta = 0.3
    out = _single(oracle_lib, n, pi.pauli(n, {q: "X"}), [(pi.pauli(n, {q: "Z"}), theta)])
    assert out[pi.pauli(n, {q: "X"})] == pytest.approx(math.cos(theta), abs=1e-15)
    assert out[pi.pauli(n, {q: "Y"})] == pytest.approx(-math.sin(theta), abs=1e-15)
    assert len(out) == 2


def test_commuting_gate_is_identity(oracle_lib):
    out = _single(oracle_lib, 3, "ZZI", [("ZZZ", 0.7), ("XXI", 0.4)])
    assert out == {"ZZI": 1.0}


def test_random_rotations_match_matrix_conjugation(oracle_lib):
    """Sign rule of i P Q for multi-qubit P, Q: compare with U^dag Q U built
    from dense matrices and decomposed over all 4^n strings."""
    rng = np.random.default_rng(7)
    n = 3
    for trial in range(40):
        q = "".join(rng.choice(list("IXYZ"), size=n))
        gates = []
        for _ in range(3):
            p = "".join(rng.choice(list("IXYZ"), size=n))
            if p == "I" * n:
                p = "X" + p[1:]
            gates.append((p, float(rng.uniform(-3, 3))))
        want = sv.heisenberg_decompose(n, gates, q)
        got = _single(oracle_lib, n, q, list(reversed(gates)))
        keys = set(want) | {k for k, v in got.items() if abs(v) > 1e-13}
        for k in keys:
            assert got.get(k, 0.0) == pytest.approx(want.get(k, 0.0), abs=1e-12), (q, gates, k)


# ------------------------------------------------- state-vector checks

def test_config0_heisenberg_matches_statevector(oracle_lib):
    wl = pi.config0_heisenberg(n=8, dt=0.05, steps=3)
    _, vals = oracle_lib.run_workload(wl, record_each_step=True)
    ref = sv.statevector_expectations(wl.circuit.layers, wl.observable.terms, wl.state.bloch)
    np.testing.assert_allclose(vals, ref, atol=1e-10, rtol=0)


def test_two_qubit_heisenberg_closed_form(oracle_lib):
    """n = 2: H = XX + YY + ZZ = 2 SWAP - 1; from |01>, <Z_0>(t) = cos 4t.
    The three rotations on one pair commute, so Trotter steps are exact."""
    dt = 0.13
    wl = pi.config0_heisenberg(n=2, dt=dt, steps=6)
    _, vals = oracle_lib.run_workload(wl, record_each_step=True)
    want = [math.cos(4 * (k + 1) * dt) for k in range(6)]
    np.testing.assert_allclose(vals, want, atol=1e-13, rtol=0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_circuit_matches_statevector(oracle_lib, seed):
    n = 6
    circ = pi.random_circuit(n, n_layers=3, gates_per_layer=8, seed=seed, max_support=4)
    obs = pi.random_observable(n, 5, seed=seed + 100, max_weight=3)
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    wl = pi.Workload("rand", circ, obs, pi.ProductState(n, v))
    _, vals = oracle_lib.run_workload(wl, record_each_step=True)
    # run_workload applies the *last* layer first and reads <O> after each
    # Heisenberg layer; the state vector reads after each time layer.  The
    # k-th Heisenberg value is the expectation after layers L-k..L-1 in time.
    L = len(circ.layers)
    for k in range(L):
        layers = circ.layers[L - 1 - k:]
        ref = sv.statevector_expectations(layers, obs.terms, v)[-1]
        assert vals[k] == pytest.approx(ref, abs=1e-10)


# ------------------------------------------------------- noise pins

def test_per_gate_noise_matches_density_matrix(oracle_lib):
    n = 4
    circ = pi.random_circuit(n, n_layers=2, gates_per_layer=6, seed=11, max_support=2)
    obs = pi.random_observable(n, 4, seed=12, max_weight=2)
    st = pi.random_product_state(n, 13)
    wl = pi.Workload("noisy", circ, obs, st, noise_p=0.07, noise_mode=1)
    _, vals = oracle_lib.run_workload(wl, record_each_step=True)
    ref = sv.density_expectations(n, circ.layers, obs.terms, st.bloch, p_gate=0.07)
    assert vals[-1] == pytest.approx(ref[-1], abs=1e-12)


def test_per_layer_noise_matches_density_matrix(oracle_lib):
    n = 4
    circ = pi.random_circuit(n, n_layers=3, gates_per_layer=5, seed=21, max_support=2)
    obs = pi.random_observable(n, 4, seed=22, max_weight=3)
    st = pi.random_product_state(n, 23)
    wl = pi.Workload("noisy", circ, obs, st, noise_p=0.2, noise_mode=2)
    _, vals = oracle_lib.run_workload(wl, record_each_step=True)
    ref = sv.density_expectations(n, circ.layers, obs.terms, st.bloch, gamma_layer=0.2)
    assert vals[-1] == pytest.approx(ref[-1], abs=1e-12)


# ------------------------------------------- orbit representatives

def _all_strings(n):
    return ["".join(t) for t in itertools.product("IXYZ", repeat=n)]


def _necklaces(n):
    return sum(4 ** math.gcd(j, n) for j in range(1, n + 1)) // n


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_zn_representative_count_is_necklace_number(oracle_lib, n):
    """Burnside / Example B.2: |R^{Z_n}_n| = (1/n) sum_j 4^gcd(j, n)."""
    strings = _all_strings(n)
    x, z = pi.to_masks(strings, n)
    ox, oz = oracle_lib.canonical(n, 1, x, z)
    reps = {tuple(a) + tuple(b) for a, b in zip(ox.tolist(), oz.tolist())}
    assert len(reps) == _necklaces(n)
    if n == 3:
        assert len(reps) == 24  # the paper's worked example
    if n in (5, 7):  # prime n: (4^n + 4(n-1)) / n, Example 1
        assert len(reps) == (4 ** n + 4 * (n - 1)) // n


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_sn_representative_count_is_tetrahedral(oracle_lib, n):
    """Example B.3: |R^{S_n}_n| = C(n+3, 3)."""
    strings = _all_strings(n)
    x, z = pi.to_masks(strings, n)
    ox, oz = oracle_lib.canonical(n, 2, x, z)
    reps = {tuple(a) + tuple(b) for a, b in zip(ox.tolist(), oz.tolist())}
    assert len(reps) == math.comb(n + 3, 3)


def _int_value(s):
    # Definition "Lowest integer representation": I,X,Y,Z -> 0,1,2,3; qubit q has weight 4^q
    return sum("IXYZ".index(ch) * 4 ** q for q, ch in enumerate(s))


@pytest.mark.parametrize("n", [2, 3, 4, 5, 6])
def test_sn_representative_is_argmin_over_all_permutations(oracle_lib, n):
    """Algorithm 3 counts letters instead of enumerating n! permutations; the
    result must equal the brute-force argmin of int() over every permutation."""
    rng = np.random.default_rng(n)
    strings = ["".join(rng.choice(list("IXYZ"), size=n)) for _ in range(40)]
    x, z = pi.to_masks(strings, n)
    ox, oz = oracle_lib.canonical(n, 2, x, z)
    got = pi.from_masks(ox, oz, n)
    for s, g in zip(strings, got):
        best = min(("".join(s[i] for i in perm) for perm in itertools.permutations(range(n))),
                   key=_int_value)
        assert g == best


@pytest.mark.parametrize("n", [3, 5, 8, 70, 130])
def test_zn_representative_is_argmin_and_invariant(oracle_lib, n):
    rng = np.random.default_rng(100 + n)
    strings = ["".join(rng.choice(list("IXYZ"), size=n)) for _ in range(60)]
    x, z = pi.to_masks(strings, n)
    got = pi.from_masks(*oracle_lib.canonical(n, 1, x, z), n)
    for s, g in zip(strings, got):
        rots = [s[j:] + s[:j] for j in range(n)]
        assert g == min(rots, key=_int_value)
        # shifting the input does not change the representative
        t = s[1:] + s[:1]
        xt, zt = pi.to_masks([t], n)
        assert pi.from_masks(*oracle_lib.canonical(n, 1, xt, zt), n)[0] == g


def test_paper_z3_representatives_lie_in_distinct_orbits(oracle_lib):
    with open(os.path.join(GOLDEN, "z3_representatives.txt")) as f:
        listed = [ln.strip() for ln in f if ln.strip() and not ln.startswith("#")]
    assert len(listed) == 24
    x, z = pi.to_masks(listed, 3)
    reps = pi.from_masks(*oracle_lib.canonical(3, 1, x, z), 3)
    assert len(set(reps)) == 24


# ---------------------------------------------- Theorem 1 and observations

def _symmetric_sn_layer(n, a, b, c):
    """exp(-i a sum_{i<j} ZZ / 2) (commuting, so exactly S_n-invariant), then
    RX(b) and RZ(c) on every qubit."""
    gates = [(pi.pauli(n, {i: "Z", j: "Z"}), a) for i in range(n) for j in range(i + 1, n)]
    gates += [(pi.pauli(n, {i: "X"}), b) for i in range(n)]
    gates += [(pi.pauli(n, {i: "Z"}), c) for i in range(n)]
    return gates


@pytest.mark.parametrize("state", ["zero", "neel"])
def test_theorem1_zn_merge_is_exact_on_ring(oracle_lib, state):
    n = 6
    wl = pi.config1_ring(n=n, steps=3, eps=0.0, max_weight=-1)
    wl.state = pi.zero_state(n) if state == "zero" else pi.neel_state(n)
    plain_st, plain = oracle_lib.run_workload(wl, group=0, record_each_step=True)
    merged_st, merged = oracle_lib.run_workload(wl, group=1, record_each_step=True)
    np.testing.assert_allclose(merged, plain, atol=1e-12, rtol=0)
    ref = sv.statevector_expectations(wl.circuit.layers, wl.observable.terms, wl.state.bloch)
    np.testing.assert_allclose(plain, ref, atol=1e-10, rtol=0)
    assert len(merged_st) < len(plain_st)


@pytest.mark.parametrize("state", ["plus", "neel"])
def test_theorem1_sn_merge_is_exact_on_symmetric_layer(oracle_lib, state):
    n = 5
    layer = _symmetric_sn_layer(n, 0.37, 0.81, -0.45)
    circ = pi.Circuit(n, [list(layer) for _ in range(2)])
    st = pi.plus_state(n) if state == "plus" else pi.neel_state(n)
    wl = pi.Workload("sn", circ, pi.mean_z(n), st)
    _, plain = oracle_lib.run_workload(wl, group=0, record_each_step=True)
    merged_st, merged = oracle_lib.run_workload(wl, group=2, record_each_step=True)
    np.testing.assert_allclose(merged, plain, atol=1e-12, rtol=0)
    assert len(merged_st) <= math.comb(n + 3, 3)


@pytest.mark.parametrize("every,sub", [(1, False), (2, False), (4, False), (1, True), (5, True)])
def test_theorem1_any_merge_cadence_is_exact(oracle_lib, every, sub):
    """Merging after every k-th symmetric layer (or after every RZZ / RX / RZ
    sublayer) leaves <O> unchanged without truncation: each merge happens at a
    boundary where the operator is invariant, so Theorem 1 applies at any
    cadence.  Checked against the state vector."""
    n, steps = 6, 4
    wl = pi.config1_ring(n=n, steps=steps, eps=0.0, max_weight=-1)
    run = pi.split_sublayers(wl) if sub else wl
    L = len(run.circuit.layers)
    flags = pi.merge_schedule(L, every)
    ox, oz, oc = wl.observable.arrays()
    st = oracle_lib.OracleState(n, ox, oz, oc, group=1)
    for a, layer in enumerate(reversed(range(L))):
        gx, gz, th = run.circuit.gate_arrays(layer)
        st.apply_layer(gx, gz, th, group=1 if flags[a] else 0)
    ref = sv.statevector_expectations(wl.circuit.layers, wl.observable.terms, wl.state.bloch)[-1]
    assert st.expect(wl.state.bloch, 1) == pytest.approx(ref, abs=1e-12)


def test_merge_schedule_and_sublayers():
    assert pi.merge_schedule(5, 2) == [False, True, False, True, True]
    assert pi.merge_schedule(3, 1) == [True, True, True]
    wl = pi.config1_ring(n=5, steps=2)
    sub = pi.split_sublayers(wl)
    assert len(sub.circuit.layers) == 6
    assert [g for layer in sub.circuit.layers for g in layer] == \
        [g for layer in wl.circuit.layers for g in layer]
    assert {s.replace("I", "") for s, _ in sub.circuit.layers[1]} == {"X"}


def test_observation1_orbit_supported_operator_is_unchanged(oracle_lib):
    n = 5
    rng = np.random.default_rng(5)
    strings = ["".join(rng.choice(list("IXYZ"), size=n)) for _ in range(30)]
    x, z = pi.to_masks(strings, n)
    reps = sorted(set(pi.from_masks(*oracle_lib.canonical(n, 1, x, z), n)))
    xr, zr = pi.to_masks(reps, n)
    coef = rng.normal(size=len(reps))
    st = oracle_lib.OracleState(n, xr, zr, coef, group=1)
    got = dict(zip(pi.from_masks(*st.export()[:2], n), st.export()[2]))
    assert got == pytest.approx(dict(zip(reps, coef)))


def test_observation2_merged_count_lower_bound(oracle_lib):
    """1/|G| <= N~/N: the merged operator never has fewer than N/|G| terms."""
    n = 6
    wl = pi.config1_ring(n=n, steps=4, eps=0.0, max_weight=-1)
    ox, oz, oc = wl.observable.arrays()
    plain = oracle_lib.OracleState(n, ox, oz, oc, group=0)
    for layer in range(4):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        plain.apply_layer(gx, gz, th, group=0)
        x, z, c = plain.export()
        merged = oracle_lib.OracleState(n, x, z, c, group=1)
        assert len(merged) * n >= len(plain)
        assert len(merged) <= len(plain)


# ------------------------------------------------------ overlaps

@pytest.mark.parametrize("n", [3, 4, 5])
def test_sn_orbit_average_matches_permutation_bruteforce(oracle_lib, n):
    st = pi.random_product_state(n, 31 + n)
    strings = []
    for nx in range(n + 1):
        for ny in range(n + 1 - nx):
            for nz in range(n + 1 - nx - ny):
                strings.append("Z" * nz + "Y" * ny + "X" * nx + "I" * (n - nx - ny - nz))
    x, z = pi.to_masks(strings, n)
    got = oracle_lib.sym_overlap(n, 2, x, z, st.bloch)
    for s, g in zip(strings, got):
        vals = []
        for perm in itertools.permutations(range(n)):
            t = "".join(s[perm[q]] for q in range(n))
            v = 1.0
            for q, ch in enumerate(t):
                if ch != "I":
                    v *= st.bloch[q, "XYZ".index(ch)]
            vals.append(v)
        assert g == pytest.approx(float(np.mean(vals)), abs=1e-14)


def test_sym_overlap_equals_plain_for_invariant_state(oracle_lib):
    n = 6
    rng = np.random.default_rng(3)
    strings = ["".join(rng.choice(list("IXYZ"), size=n)) for _ in range(50)]
    x, z = pi.to_masks(strings, n)
    for st in (pi.plus_state(n), pi.zero_state(n)):
        plain = oracle_lib.sym_overlap(n, 0, x, z, st.bloch)
        for g in (1, 2):
            np.testing.assert_allclose(oracle_lib.sym_overlap(n, g, x, z, st.bloch), plain,
                                       atol=1e-15)


def test_total_spin_normalisation(oracle_lib):
    """<+|S^2|+> = n(n+2)/4 (normalisation S_0^2 of Fig. 2)."""
    for n in (4, 7, 36):
        obs = pi.total_spin_squared(n)
        x, z, c = obs.arrays()
        st = oracle_lib.OracleState(n, x, z, c)
        assert st.expect(pi.plus_state(n).bloch) == pytest.approx(n * (n + 2) / 4, rel=1e-14)


# ------------------------------------------------------ truncation rules

def test_truncation_threshold_and_weight(oracle_lib):
    n = 4
    strings = ["ZIII", "XXII", "YYYI", "ZZZZ"]
    x, z = pi.to_masks(strings, n)
    coef = np.array([1e-3, 1e-4, 0.5, 0.9])
    st = oracle_lib.OracleState(n, x, z, coef, eps=1e-3, max_weight=3)
    got = dict(zip(pi.from_masks(*st.export()[:2], n), st.export()[2]))
    # |c| >= eps kept (ZIII at exactly eps), XXII below eps, ZZZZ too heavy
    assert got == {"ZIII": 1e-3, "YYYI": 0.5}


def test_truncation_follows_the_symmetry_merge(oracle_lib):
    """The coefficient rule applies to the operator held after a merge (Alg. 1
    step 2b gives O~, whose coefficients are orbit sums, Eq. O-merging): on
    n = 3 with Z_3, 0.6 ZII - 0.55 IZI + 0.3 ZZI passes eps = 0.1 term by term,
    but ZII and IZI share an orbit whose sum 0.05 is below eps, so after a
    layer of RZ gates (which commute with every term) and the merge only the
    representative ZZI remains, with 0.3."""
    n = 3
    strings = ["ZII", "IZI", "ZZI"]
    x, z = pi.to_masks(strings, n)
    st = oracle_lib.OracleState(n, x, z, np.array([0.6, -0.55, 0.3]), eps=0.1)
    assert len(st) == 3
    layer = [(pi.pauli(n, {q: "Z"}), 0.7) for q in range(n)]
    gx, gz, th = pi.Circuit(n, [layer]).gate_arrays(0)
    st.apply_layer(gx, gz, th, group=1)
    got = dict(zip(pi.from_masks(*st.export()[:2], n), st.export()[2]))
    assert got == {"ZZI": 0.3}
    # batched rows: a merged row is kept iff some column reaches eps
    rows = np.array([[0.6, 0.5], [-0.55, -0.45], [0.3, 0.01]])
    bst = oracle_lib.BatchedOracleState(n, 2, x, z, rows, eps=0.1)
    assert len(bst) == 3
    bst.apply_layer(gx, gz, np.repeat(th[:, None], 2, axis=1), group=1)
    bx, bz, bc = bst.export()
    assert pi.from_masks(bx, bz, n) == ["ZZI"]
    assert bc.tolist() == [[0.3, 0.01]]


def test_truncation_never_drops_zero_when_off(oracle_lib):
    n = 2
    x, z = pi.to_masks(["ZI", "XI"], n)
    st = oracle_lib.OracleState(n, x, z, np.array([0.0, 1.0]))
    assert len(st) == 2


def test_s2_invariant_for_symmetric_heisenberg_a2a(oracle_lib):
    """S^2 commutes with each exp(-i dt (XX+YY+ZZ)) pair gate (Heisenberg
    all-to-all, config 0 family), so <S^2> stays n(n+2)/4 from |+>^n."""
    n = 5
    wl = pi.config0_heisenberg(n=n, dt=0.07, steps=2)
    wl.observable = pi.total_spin_squared(n)
    wl.state = pi.plus_state(n)
    _, vals = oracle_lib.run_workload(wl, record_each_step=True)
    np.testing.assert_allclose(vals, [n * (n + 2) / 4] * 2, rtol=1e-12)


# ------------------------------------------------------ batched angle sets

def _ring_angles(B, seed):
    return pi.batched_ring_angles(B, seed)


def _ring_theta(n, angles):
    """[K=3n, B] angles of one ring layer for B angle triples (theta_J, theta_x, theta_z)."""
    B = len(angles)
    th = np.zeros((3 * n, B))
    th[:n] = angles[:, 0]
    th[n:2 * n] = angles[:, 1]
    th[2 * n:] = angles[:, 2]
    return th


def test_batched_columns_equal_single_runs_bitexact(oracle_lib):
    n, B, L = 6, 5, 3
    angles = _ring_angles(B, 3)
    gx, gz, _ = pi.Circuit(n, [pi.ring_layer(n, 0, 0, 0)]).gate_arrays(0)
    obs = pi.mean_z(n)
    x, z, c = obs.arrays()
    bst = oracle_lib.BatchedOracleState(n, B, x, z, np.repeat(c[:, None], B, axis=1))
    th = _ring_theta(n, angles)
    for _ in range(L):
        bst.apply_layer(gx, gz, th)
    bx, bz, bc = bst.export()
    bkeys = [tuple(a) + tuple(b) for a, b in zip(bx.tolist(), bz.tolist())]
    for b in range(B):
        st = oracle_lib.OracleState(n, x, z, c)
        for _ in range(L):
            st.apply_layer(gx, gz, th[:, b])
        want = st.as_dict()
        got = {k: bc[i, b] for i, k in enumerate(bkeys)}
        assert set(want) <= set(got)
        for k, v in got.items():
            assert v == want.get(k, 0.0)
    ref = sv.statevector_expectations(
        [[(s, angles[1][0] if g < n else (angles[1][1] if g < 2 * n else angles[1][2]))
          for g, (s, _) in enumerate(pi.ring_layer(n, 0, 0, 0))]] * L,
        obs.terms, pi.zero_state(n).bloch)[-1]
    assert bst.expect(pi.zero_state(n).bloch)[1] == pytest.approx(ref, abs=1e-12)


def test_batched_single_column_equals_single_state_with_truncation(oracle_lib):
    n = 10
    wl = pi.config1_ring(n=n, steps=4, eps=1e-3, max_weight=5)
    x, z, c = wl.observable.arrays()
    bst = oracle_lib.BatchedOracleState(n, 1, x, z, c[:, None], eps=wl.eps,
                                        max_weight=wl.max_weight)
    st = oracle_lib.OracleState(n, x, z, c, eps=wl.eps, max_weight=wl.max_weight)
    for layer in range(4):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        bst.apply_layer(gx, gz, th[:, None])
        st.apply_layer(gx, gz, th)
    bx, bz, bc = bst.export()
    sx, sz, sc = st.export()
    np.testing.assert_array_equal(bx, sx)
    np.testing.assert_array_equal(bz, sz)
    np.testing.assert_array_equal(bc[:, 0], sc)


def _column_layers(circ, angles_per_gate, b):
    """The circuit's layers with gate k of the flattened circuit at angle
    angles_per_gate[k, b] (time order)."""
    out, k = [], 0
    for layer in circ.layers:
        row = []
        for s, _ in layer:
            row.append((s, float(angles_per_gate[k, b])))
            k += 1
        out.append(row)
    return out


@pytest.mark.parametrize("p", [0.07, 0.3])
def test_batched_per_gate_noise_matches_density_matrix_per_column(oracle_lib, p):
    """Batched rows with per-gate depolarising damping: every column is its own
    noisy circuit (own angles, same gates), so column b must equal the density
    matrix evolved with column b's angles and the channel after every gate on
    its support.  Damping applied after the rotation instead of before it, or
    with the support count of the wrong string, changes these values."""
    n, B = 4, 3
    circ = pi.random_circuit(n, n_layers=2, gates_per_layer=6, seed=31, max_support=2)
    n_gates = sum(len(l) for l in circ.layers)
    angles = np.random.default_rng(32).uniform(-math.pi, math.pi, size=(n_gates, B))
    obs = pi.random_observable(n, 4, seed=33, max_weight=2)
    state = pi.random_product_state(n, 34)
    x, z, c = obs.arrays()
    bst = oracle_lib.BatchedOracleState(n, B, x, z, np.repeat(c[:, None], B, axis=1))
    k_end = n_gates
    for li in reversed(range(len(circ.layers))):
        K = len(circ.layers[li])
        gx, gz = pi.to_masks([s for s, _ in circ.layers[li]], n)
        bst.apply_layer(gx, gz, angles[k_end - K:k_end], noise_mode=1, p=p)
        k_end -= K
    got = bst.expect(state.bloch)
    for b in range(B):
        ref = sv.density_expectations(n, _column_layers(circ, angles, b), obs.terms, state.bloch,
                                      p_gate=p)[-1]
        assert got[b] == pytest.approx(ref, abs=1e-12)
    assert len(set(np.round(got, 9))) == B  # the columns really differ


def test_batched_noise_single_column_equals_single_state(oracle_lib):
    """One column with per-gate damping and truncation is the single-column
    oracle, coefficient for coefficient."""
    n = 6
    wl = pi.config1_ring(n=n, steps=3, eps=1e-3, max_weight=4)
    x, z, c = wl.observable.arrays()
    bst = oracle_lib.BatchedOracleState(n, 1, x, z, c[:, None], eps=wl.eps,
                                        max_weight=wl.max_weight)
    st = oracle_lib.OracleState(n, x, z, c, eps=wl.eps, max_weight=wl.max_weight)
    for layer in range(3):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        bst.apply_layer(gx, gz, th[:, None], noise_mode=1, p=0.05)
        st.apply_layer(gx, gz, th, noise_mode=1, p=0.05)
    bx, bz, bc = bst.export()
    sx, sz, sc = st.export()
    np.testing.assert_array_equal(bx, sx)
    np.testing.assert_array_equal(bz, sz)
    np.testing.assert_array_equal(bc[:, 0], sc)


def test_batched_truncation_keeps_a_term_if_any_column_is_large(oracle_lib):
    n = 3
    x, z = pi.to_masks(["ZII", "XII", "IYI"], n)
    coef = np.array([[1e-4, 2e-2], [1e-4, 1e-4], [0.5, 0.5]])
    bst = oracle_lib.BatchedOracleState(n, 2, x, z, coef, eps=1e-2)
    bx, bz, bc = bst.export()
    got = dict(zip(pi.from_masks(bx, bz, n), map(tuple, bc)))
    assert got == {"ZII": (1e-4, 2e-2), "IYI": (0.5, 0.5)}


@pytest.mark.parametrize("n", [3, 5, 7])
def test_ising_counts_saturate_at_the_orbit_numbers(oracle_lib, n):
    """The periodic Ising example (Fig. 1 and its caption, Example "Translation
    symmetry Z_n"): without truncation, propagating Z at site ceil(n/2) through
    the Trotter layers fills the whole traceless operator space, so the plain
    count saturates at 4^n - 1 strings and the merged count at the number of
    Z_n orbits of non-identity strings, (4^n + 4(n-1))/n - 1 for prime n
    (Burnside).  At every layer the merged count is at most the plain one,
    and below it from the second layer on."""
    wl = pi.config1_ring(n=n, steps=7, theta_j=0.37, theta_x=0.81, theta_z=0.53, eps=0.0,
                         max_weight=-1)
    x, z = pi.to_masks([pi.pauli(n, {(n + 1) // 2 - 1: "Z"})], n)
    counts = {}
    for group in (0, 1):
        st = oracle_lib.OracleState(n, x, z, np.array([1.0]), group=group)
        counts[group] = []
        for layer in reversed(range(len(wl.circuit.layers))):
            gx, gz, th = wl.circuit.gate_arrays(layer)
            st.apply_layer(gx, gz, th, group=group)
            counts[group].append(len(st))
    assert counts[0][-1] == 4 ** n - 1
    assert counts[1][-1] == (4 ** n + 4 * (n - 1)) // n - 1
    assert all(m <= p for m, p in zip(counts[1], counts[0]))
    assert all(m < p for m, p in zip(counts[1][1:], counts[0][1:]))


# -------------------------- ingest, the update count, batched merging

def test_ingest_accumulates_repeated_strings(oracle_lib):
    """Algorithm 1 step 1 starts from O = sum_s c_s s: a string listed twice
    stands for the sum of its coefficients.  The ingested table holds the
    sums (single column and batched rows), and <O> after a random circuit on
    a mixed product state is the density-matrix value of the same list of
    terms."""
    n = 4
    terms = [("ZIII", 0.25), ("XYII", 0.5), ("ZIII", 0.5), ("IIXZ", 1.0), ("XYII", -0.125)]
    x, z = pi.to_masks([t for t, _ in terms], n)
    st = oracle_lib.OracleState(n, x, z, np.array([c for _, c in terms]))
    ex, ez, ec = st.export()
    assert dict(zip(pi.from_masks(ex, ez, n), ec.tolist())) == {
        "ZIII": 0.75, "XYII": 0.375, "IIXZ": 1.0}
    circ = pi.random_circuit(n, n_layers=2, gates_per_layer=5, seed=41, max_support=2)
    state = pi.random_product_state(n, 42)
    for li in reversed(range(len(circ.layers))):
        gx, gz, th = circ.gate_arrays(li)
        st.apply_layer(gx, gz, th)
    ref = sv.density_expectations(n, circ.layers, terms, state.bloch)[-1]
    assert st.expect(state.bloch) == pytest.approx(ref, abs=1e-12)

    coef = np.array([[0.25, -1.0], [0.5, 0.0], [0.5, 2.0], [1.0, 1.0], [-0.125, 0.5]])
    bst = oracle_lib.BatchedOracleState(n, 2, x, z, coef)
    bx, bz, bc = bst.export()
    assert dict(zip(pi.from_masks(bx, bz, n), map(tuple, bc.tolist()))) == {
        "ZIII": (0.75, 1.0), "XYII": (0.375, 0.5), "IIXZ": (1.0, 1.0)}


def test_update_count_is_the_live_terms_entering_each_gate(oracle_lib):
    """The throughput unit: one update is one live term entering one gate.
    Closed form for X_0 under RZ_0, RZ_0, RZ_1 (Heisenberg order): one term
    enters the first gate and leaves it as {X_0, Y_0}, two enter each later
    gate (1, 3, 5).  With a threshold that drops the sin branch, one term
    enters every gate (1, 2, 3).  On a truncated ring circuit the count grows
    at every gate by the number of terms stored just before it."""
    n = 2
    x, z = pi.to_masks(["XI"], n)
    gates = [pi.pauli(n, {0: "Z"}), pi.pauli(n, {0: "Z"}), pi.pauli(n, {1: "Z"})]
    for eps, th, want in [(0.0, 0.7, [1, 3, 5]), (0.5, 0.1, [1, 2, 3])]:
        st = oracle_lib.OracleState(n, x, z, np.array([1.0]), eps=eps)
        bst = oracle_lib.BatchedOracleState(n, 2, x, z, np.array([[1.0, 0.5]]), eps=eps)
        got, bgot = [], []
        for g in gates:
            gx, gz = pi.to_masks([g], n)
            st.apply_gate(gx[0], gz[0], th)
            bst.apply_layer(gx, gz, np.array([[th, th]]))
            got.append(st.updates)
            bgot.append(bst.updates)
        assert got == want and bgot == want

    wl = pi.config1_ring(n=8, steps=2, eps=1e-3, max_weight=4)
    x, z, c = wl.observable.arrays()
    st = oracle_lib.OracleState(8, x, z, c, eps=wl.eps, max_weight=wl.max_weight)
    bst = oracle_lib.BatchedOracleState(8, 1, x, z, c[:, None], eps=wl.eps,
                                        max_weight=wl.max_weight)
    for layer in reversed(range(2)):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        for g in reversed(range(len(th))):
            before, bbefore = len(st), len(bst)
            u, bu = st.updates, bst.updates
            st.apply_gate(gx[g], gz[g], th[g])
            bst.apply_layer(gx[g:g + 1], gz[g:g + 1], th[g:g + 1, None])
            assert st.updates - u == before and bst.updates - bu == bbefore
    assert st.updates > 100


def test_batched_symmetry_merge_keeps_every_column_exact(oracle_lib):
    """Batched rows merged by Z_n representatives after every ring step (Eq.
    O-merging, column by column): without truncation every column's <O> is
    the state-vector value for its own angles (Theorem 1; the Neel state is
    not invariant, so the overlap is the orbit average), and the merged
    table is smaller than the unmerged one."""
    n, B, L = 6, 3, 2
    angles = _ring_angles(B, 5)
    gx, gz, _ = pi.Circuit(n, [pi.ring_layer(n, 0, 0, 0)]).gate_arrays(0)
    obs = pi.mean_z(n)
    x, z, c = obs.arrays()
    state = pi.neel_state(n)
    th = _ring_theta(n, angles)
    rows = np.repeat(c[:, None], B, axis=1)
    merged = oracle_lib.BatchedOracleState(n, B, x, z, rows, group=1)
    plain = oracle_lib.BatchedOracleState(n, B, x, z, rows)
    for _ in range(L):
        merged.apply_layer(gx, gz, th, group=1)
        plain.apply_layer(gx, gz, th)
    got = merged.expect(state.bloch, 1)
    for b in range(B):
        layer = [(s, float(th[g, b])) for g, (s, _) in enumerate(pi.ring_layer(n, 0, 0, 0))]
        ref = sv.statevector_expectations([layer] * L, obs.terms, state.bloch)[-1]
        assert got[b] == pytest.approx(ref, abs=1e-12)
    assert len(set(np.round(got, 9))) == B
    assert len(merged) < len(plain)


def test_batched_sn_merge_keeps_every_column_exact(oracle_lib):
    """Batched rows merged by S_n representatives after every layer of the
    permutation-invariant layer (all-pairs ZZ, then RX and RZ on every qubit)
    with different angles per column: without truncation every column's <O>
    is the state-vector value for its own angles (Theorem 1; from the Neel
    state, which is not S_n-invariant, through the orbit-averaged overlap),
    and the merged table holds at most C(n+3, 3) representatives."""
    n, B, L = 5, 3, 2
    cols = [(0.37, 0.81, -0.45), (-0.6, 0.2, 1.1), (1.3, -0.9, 0.25)]
    layers = [_symmetric_sn_layer(n, *a) for a in cols]
    gx, gz, _ = pi.Circuit(n, [layers[0]]).gate_arrays(0)
    th = np.array([[layers[b][g][1] for b in range(B)] for g in range(len(layers[0]))])
    obs = pi.mean_z(n)
    x, z, c = obs.arrays()
    state = pi.neel_state(n)
    merged = oracle_lib.BatchedOracleState(n, B, x, z, np.repeat(c[:, None], B, axis=1), group=2)
    for _ in range(L):
        merged.apply_layer(gx, gz, th, group=2)
    got = merged.expect(state.bloch, 2)
    for b in range(B):
        ref = sv.statevector_expectations([layers[b]] * L, obs.terms, state.bloch)[-1]
        assert got[b] == pytest.approx(ref, abs=1e-12)
    assert len(set(np.round(got, 9))) == B
    assert len(merged) <= math.comb(n + 3, 3)


# ------------------------------------------ the stored expected values

def _trajectory(oracle_lib, wl, group, layers):
    ox, oz, oc = wl.observable.arrays()
    st = oracle_lib.OracleState(wl.circuit.n, ox, oz, oc, group=group, eps=wl.eps,
                                max_weight=wl.max_weight)
    rows = []
    for layer in list(reversed(range(len(wl.circuit.layers))))[:layers]:
        gx, gz, th = wl.circuit.gate_arrays(layer)
        st.apply_layer(gx, gz, th, wl.noise_mode, wl.noise_p, group=group)
        rows.append({"terms": len(st), "expect": st.expect(wl.state.bloch, group),
                     "updates": st.updates})
    return rows


def test_stored_heisenberg_trajectory_is_the_oracles_and_the_state_vectors(oracle_lib):
    """tests/golden/heisenberg_a2a_n8.json was written by write_golden.py from
    the oracle: the oracle still gives it exactly, and it is the state-vector
    result (n = 8, 3 Trotter steps, no truncation)."""
    gold = json.load(open(os.path.join(GOLDEN, "heisenberg_a2a_n8.json")))["plain"]
    wl = pi.config0_heisenberg()
    assert _trajectory(oracle_lib, wl, 0, len(gold)) == gold
    ref = sv.statevector_expectations(wl.circuit.layers, wl.observable.terms, wl.state.bloch)
    np.testing.assert_allclose([r["expect"] for r in gold], ref, atol=1e-12, rtol=0)


def test_stored_ring_trajectories_start_as_the_oracles(oracle_lib):
    """The first steps of tests/golden/ring_n32.json (plain and Z_32) are what
    the oracle computes now; the first two steps agree between plain and merged
    (no term is near eps yet), as Theorem 1 says without truncation."""
    data = json.load(open(os.path.join(GOLDEN, "ring_n32.json")))
    wl = pi.config1_ring()
    assert _trajectory(oracle_lib, wl, 0, 3) == data["plain"][:3]
    assert _trajectory(oracle_lib, wl, 1, 3) == data["zn"][:3]
    for k in range(2):
        assert data["zn"][k]["expect"] == pytest.approx(data["plain"][k]["expect"], abs=1e-14)
