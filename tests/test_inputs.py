"""The seeded input recipes: every workload has the sizes, angles, noise and
truncation settings it is documented with, and the generators are
deterministic in their seeds.  CPU only; no propagation arithmetic."""
import math

import numpy as np
import pytest

import pp_inputs as pi


def letters(s):
    return {q: ch for q, ch in enumerate(s) if ch != "I"}


def test_mask_encoding_round_trip():
    n = 70
    rng = np.random.default_rng(3)
    strings = ["".join(rng.choice(list("IXYZ"), size=n)) for _ in range(50)]
    x, z = pi.to_masks(strings, n)
    assert x.shape == (50, 2) and z.shape == (50, 2)
    assert pi.from_masks(x, z, n) == strings
    # X sets x, Z sets z, Y sets both; qubit q is bit q % 64 of word q // 64
    gx, gz = pi.to_masks([pi.pauli(n, {0: "X", 64: "Y", 65: "Z"})], n)
    assert gx[0].tolist() == [1, 1] and gz[0].tolist() == [0, 3]


def test_config0_heisenberg_recipe():
    wl = pi.config0_heisenberg()
    n = wl.circuit.n
    assert n == 8 and len(wl.circuit.layers) == 3
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    want = [(pi.pauli(n, {i: p, j: p}), 0.1) for (i, j) in pairs for p in "XYZ"]
    for layer in wl.circuit.layers:
        assert len(layer) == 84
        assert [g[0] for g in layer] == [w[0] for w in want]
        assert all(g[1] == pytest.approx(0.1, abs=1e-15) for g in layer)
    assert wl.observable.terms == [(pi.pauli(n, {0: "Z"}), 1.0)]
    assert wl.state.basis.tolist() == [q % 2 for q in range(n)]
    assert wl.eps == 0.0 and wl.max_weight == -1 and wl.noise_mode == 0


def test_config1_ring_recipe():
    wl = pi.config1_ring()
    n = wl.circuit.n
    assert n == 32 and len(wl.circuit.layers) == 20
    for layer in wl.circuit.layers:
        assert len(layer) == 96
        for i in range(n):
            assert letters(layer[i][0]) == {i: "Z", (i + 1) % n: "Z"} and layer[i][1] == 0.4
            assert letters(layer[n + i][0]) == {i: "X"} and layer[n + i][1] == 0.6
            assert letters(layer[2 * n + i][0]) == {i: "Z"} and layer[2 * n + i][1] == 0.3
    assert len(wl.observable.terms) == n
    assert all(letters(s) == {q: "Z"} and c == 1.0 / n for q, (s, c) in enumerate(wl.observable.terms))
    assert wl.state.basis.tolist() == [0] * n
    assert wl.eps == 1e-4 and wl.max_weight == 10


def test_config2_all_to_all_recipe():
    wl = pi.config2_all_to_all()
    n = wl.circuit.n
    assert n == 64 and len(wl.circuit.layers) == 10
    layer = wl.circuit.layers[0]
    assert len(layer) == 2016 * 3 == 6048
    assert all(g[1] == pytest.approx(0.04, abs=1e-15) for g in layer)
    assert wl.noise_mode == 1 and wl.noise_p == 0.01 and wl.eps == 1e-5
    assert wl.state.basis.tolist() == [q % 2 for q in range(n)]
    assert [len(letters(g[0])) for g in layer] == [2] * 6048


@pytest.mark.parametrize("n", [6, 36])
@pytest.mark.parametrize("split", [False, True])
def test_xxz_recipe_and_normalisation(n, split):
    dt, J, Delta = 0.05, 1.0, -1.8
    wl = pi.xxz_all_to_all(n, dt, 2, split=split)
    npairs = n * (n - 1) // 2
    if split:
        assert len(wl.circuit.layers) == 6
        for k, layer in enumerate(wl.circuit.layers):
            p = "XYZ"[k % 3]
            assert len(layer) == npairs
            assert all(set(letters(g[0]).values()) == {p} for g in layer)
    else:
        assert len(wl.circuit.layers) == 2 and len(wl.circuit.layers[0]) == 3 * npairs
    for layer in wl.circuit.layers:
        for s, th in layer:
            p = set(letters(s).values()).pop()
            want = -2 * J * dt if p in "XY" else -2 * J * (Delta + 1) * dt
            assert th == pytest.approx(want, abs=1e-15)
    # <+|O|+> = 1: only strings of I and X overlap |+>^n, each with value 1
    plus = sum(c for s, c in wl.observable.terms if set(s) <= {"I", "X"})
    assert plus == pytest.approx(1.0, abs=1e-13)
    assert np.allclose(wl.state.bloch, [[1.0, 0.0, 0.0]] * n)


def test_torus_layer_is_translation_invariant():
    lx, ly = 4, 3
    n = lx * ly
    layer = pi.torus_layer(lx, ly, 0.4, 0.6, 0.3)
    assert len(layer) == 2 * n + 2 * n

    def shifted(s, dx, dy):
        out = ["I"] * n
        for q, ch in enumerate(s):
            x, y = q % lx, q // lx
            out[(x + dx) % lx + lx * ((y + dy) % ly)] = ch
        return "".join(out)

    base = sorted(layer)
    for dx, dy in [(1, 0), (0, 1), (3, 2)]:
        assert sorted((shifted(s, dx, dy), th) for s, th in layer) == base


def test_batched_angles_recipe():
    a = pi.batched_ring_angles(256, 0)
    assert a.shape == (256, 3)
    assert a.min() >= 0.0 and a.max() <= math.pi / 2
    np.testing.assert_array_equal(a, pi.batched_ring_angles(256, 0))
    assert not np.array_equal(a, pi.batched_ring_angles(256, 1))


def test_serving_stream_recipe():
    jobs = pi.serving_stream(2000, 200.0, 0)
    assert jobs == pi.serving_stream(2000, 200.0, 0)
    t = np.array([j["arrival"] for j in jobs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    # exponential gaps of mean 1/200 s: the sample mean of 2000 is within
    # 5 standard errors (sd / sqrt(2000) = mean / 44.7)
    assert abs(gaps.mean() - 1 / 200) < 5 * (1 / 200) / math.sqrt(2000)
    assert {j["n"] for j in jobs} == {16, 32, 64, 128}
    assert {j["family"] for j in jobs} == {"ring", "a2a"}
    assert min(j["steps"] for j in jobs) >= 5 and max(j["steps"] for j in jobs) <= 40
    assert all(1e-6 <= j["eps"] <= 1e-3 for j in jobs)
    assert all(not (j["family"] == "ring" and j["group"] == 2) for j in jobs)
    assert {j["group"] for j in jobs} == {0, 1, 2}


def test_random_generators_are_seeded():
    a = pi.random_circuit(10, 3, 20, seed=4)
    b = pi.random_circuit(10, 3, 20, seed=4)
    assert a.layers == b.layers
    assert a.layers != pi.random_circuit(10, 3, 20, seed=5).layers
    o1, o2 = pi.random_observable(12, 30, 7), pi.random_observable(12, 30, 7)
    assert o1.terms == o2.terms
    s = pi.random_product_state(9, 2).bloch
    np.testing.assert_array_equal(s, pi.random_product_state(9, 2).bloch)
    assert np.all(np.linalg.norm(s, axis=1) <= 1.0 + 1e-12)
