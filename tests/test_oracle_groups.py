"""Pins of the oracle's dihedral (D_n) and 2D-translation (Z_Lx x Z_Ly) groups.

The paper names both as further symmetry groups for the method: reflections of
a ring (dihedral symmetry, Appendix B) and translations along x and y for the
XXZ lattice figure.  The oracle finds representatives and symmetrised
overlaps by enumerating group elements; these tests pin it to facts
computed here independently: Burnside's orbit counts (from cycle counts of
permutations built in this file), invariance under every element, the
relation of D_n to Z_n, brute-force overlap averages, and Theorem 1 (merging
is exact on symmetric layers without truncation).
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import pp_inputs as pi
from oracle import statevector as sv


@pytest.fixture(scope="module")
def oracle_lib():
    oracle.build()
    return oracle


def dihedral_maps(n):
    """All 2n site maps of D_n, built here: q -> q + j and q -> -q + j (mod n)."""
    maps = []
    for j in range(n):
        maps.append([(q + j) % n for q in range(n)])
        maps.append([(-q + j) % n for q in range(n)])
    return maps


def torus_maps(lx, ly):
    maps = []
    for dx in range(lx):
        for dy in range(ly):
            maps.append([((q % lx) + dx) % lx + lx * (((q // lx) + dy) % ly) for q in range(lx * ly)])
    return maps


def cycles(m):
    seen, c = set(), 0
    for q in range(len(m)):
        if q not in seen:
            c += 1
            while q not in seen:
                seen.add(q)
                q = m[q]
    return c


def burnside(maps):
    """Number of orbits of 4-letter strings: (1/|G|) sum_g 4^{cycles(g)}."""
    total = sum(4 ** cycles(m) for m in maps)
    assert total % len(maps) == 0
    return total // len(maps)


def apply(s, m):
    r = [None] * len(s)
    for q, ch in enumerate(s):
        r[m[q]] = ch
    return "".join(r)


def canon_strings(oracle_lib, n, group, strings):
    x, z = pi.to_masks(strings, n)
    ox, oz = oracle_lib.canonical(n, group, x, z)
    return pi.from_masks(ox, oz, n)


def all_strings(n):
    return ["".join(t) for t in itertools.product("IXYZ", repeat=n)]


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7])
def test_dihedral_representative_count_is_burnside(oracle_lib, n):
    reps = set(canon_strings(oracle_lib, n, oracle.DN, all_strings(n)))
    assert len(reps) == burnside(dihedral_maps(n))
    # bracelets with 4 colours, the textbook closed form
    neck = sum(4 ** math.gcd(j, n) for j in range(1, n + 1))
    refl = n * 4 ** ((n + 1) // 2) if n % 2 else (n // 2) * (4 ** (n // 2 + 1) + 4 ** (n // 2))
    assert len(reps) == (neck + refl) // (2 * n)


@pytest.mark.parametrize("lx,ly", [(2, 2), (2, 3), (3, 2), (3, 3), (4, 2)])
def test_torus_representative_count_is_burnside(oracle_lib, lx, ly):
    n = lx * ly
    reps = set(canon_strings(oracle_lib, n, oracle.torus_group(lx), all_strings(n)))
    assert len(reps) == burnside(torus_maps(lx, ly))
    # closed form: translation (dx, dy) has n / order cycles
    want = 0
    for dx in range(lx):
        for dy in range(ly):
            order = math.lcm(lx // math.gcd(dx, lx), ly // math.gcd(dy, ly))
            want += 4 ** (n // order)
    assert len(reps) == want // n


@pytest.mark.parametrize("group,n,maps", [
    (oracle.DN, 9, dihedral_maps(9)), (oracle.DN, 12, dihedral_maps(12)),
    (oracle.torus_group(4), 12, torus_maps(4, 3)), (oracle.torus_group(3), 12, torus_maps(3, 4))])
def test_representative_is_invariant_minimal_and_in_orbit(oracle_lib, group, n, maps):
    rng = np.random.default_rng(5)
    strings = ["".join(rng.choice(list("IXYZ"), size=n)) for _ in range(60)]
    reps = canon_strings(oracle_lib, n, group, strings)
    digits = {"I": 0, "X": 1, "Y": 2, "Z": 3}

    def as_int(s):
        return sum(digits[ch] * 4 ** q for q, ch in enumerate(s))

    for s, r in zip(strings, reps):
        images = [apply(s, m) for m in maps]
        assert r in images                                   # in the orbit
        assert as_int(r) == min(as_int(t) for t in images)   # lowest integer
        assert canon_strings(oracle_lib, n, group, images[1:4]) == [r] * 3  # invariant


@pytest.mark.parametrize("n", [5, 8, 11])
def test_dihedral_is_min_of_ring_and_reflected_ring(oracle_lib, n):
    rng = np.random.default_rng(n)
    strings = ["".join(rng.choice(list("IXYZ"), size=n)) for _ in range(80)]
    dn = canon_strings(oracle_lib, n, oracle.DN, strings)
    zn = canon_strings(oracle_lib, n, oracle.ZN, strings)
    zr = canon_strings(oracle_lib, n, oracle.ZN, [s[::-1] for s in strings])
    digits = {"I": 0, "X": 1, "Y": 2, "Z": 3}

    def key(s):
        return [digits[ch] for ch in reversed(s)]

    for d, a, b in zip(dn, zn, zr):
        assert d == min(a, b, key=key)


@pytest.mark.parametrize("group,n,maps", [(oracle.DN, 7, dihedral_maps(7)),
                                          (oracle.torus_group(3), 9, torus_maps(3, 3))])
def test_symmetrised_overlap_is_brute_force_average(oracle_lib, group, n, maps):
    rng = np.random.default_rng(11)
    strings = ["".join(rng.choice(list("IXYZ"), size=n)) for _ in range(40)]
    bloch = pi.random_product_state(n, 3).bloch
    b = np.asarray(bloch).reshape(n, 3)
    col = {"X": 0, "Y": 1, "Z": 2}

    def prod(s):
        v = 1.0
        for q, ch in enumerate(s):
            if ch != "I":
                v *= b[q, col[ch]]
        return v

    want = [np.mean([prod(apply(s, m)) for m in maps]) for s in strings]
    x, z = pi.to_masks(strings, n)
    got = oracle_lib.sym_overlap(n, group, x, z, bloch)
    np.testing.assert_allclose(got, want, atol=1e-14, rtol=1e-12)
    # for an invariant state the average is the plain overlap
    inv = pi.plus_state(n).bloch
    np.testing.assert_allclose(oracle_lib.sym_overlap(n, group, x, z, inv),
                               oracle_lib.sym_overlap(n, 0, x, z, inv), atol=1e-15)


@pytest.mark.parametrize("state", ["zero", "neel", "random"])
def test_theorem1_dihedral_merge_is_exact_on_ring(oracle_lib, state):
    n = 6
    wl = pi.config1_ring(n=n, steps=3, eps=0.0, max_weight=-1)
    wl.state = {"zero": pi.zero_state(n), "neel": pi.neel_state(n),
                "random": pi.random_product_state(n, 7)}[state]
    plain_st, plain = oracle_lib.run_workload(wl, group=0, record_each_step=True)
    merged_st, merged = oracle_lib.run_workload(wl, group=oracle.DN, record_each_step=True)
    zn_st, _ = oracle_lib.run_workload(wl, group=oracle.ZN, record_each_step=True)
    np.testing.assert_allclose(merged, plain, atol=1e-12, rtol=0)
    assert len(merged_st) <= len(zn_st) < len(plain_st)


@pytest.mark.parametrize("lx,ly", [(3, 2), (2, 3)])
def test_theorem1_torus_merge_is_exact(oracle_lib, lx, ly):
    wl = pi.torus_ising(lx, ly, steps=2)
    n = lx * ly
    for state in (pi.zero_state(n), pi.random_product_state(n, 2)):
        wl.state = state
        plain_st, plain = oracle_lib.run_workload(wl, group=0, record_each_step=True)
        merged_st, merged = oracle_lib.run_workload(wl, group=oracle.torus_group(lx),
                                                    record_each_step=True)
        np.testing.assert_allclose(merged, plain, atol=1e-12, rtol=0)
        assert len(merged_st) < len(plain_st)
    ref = sv.statevector_expectations(wl.circuit.layers, wl.observable.terms, pi.zero_state(n).bloch)
    wl.state = pi.zero_state(n)
    _, plain = oracle_lib.run_workload(wl, group=0, record_each_step=True)
    np.testing.assert_allclose(plain, ref, atol=1e-10, rtol=0)


# ------------------------------------------------- XXZ workload (total spin)

@pytest.mark.parametrize("split", [True, False])
def test_xxz_total_spin_against_statevector_and_conservation(oracle_lib, split):
    """All-to-all XXZ with alpha = 0: H = -J (2 S^2 + 2 Delta S_z^2) + const.

    Split into XX / YY / ZZ sublayers each step is exp(-i t S_a^2) up to a
    phase: every sublayer is a product of commuting gates that S_n maps onto
    itself, so merging after it is exact (Theorem 1), and each commutes with
    S^2, so without truncation <S^2>/S_0^2 stays exactly 1.

    In the pair-by-pair order (pairs outer, XX YY ZZ inner) the gate multiset
    is S_n-invariant but the ordered product of non-commuting pair gates is
    not, so merging after the layer is exact only up to Trotter error.  The
    paper merges after such layers too; the pin records that the merged value
    then differs from the plain one, while the plain one matches the state
    vector and drifts from 1 by Trotter error."""
    n = 6
    wl = pi.xxz_all_to_all(n, 0.1, 3, eps=0.0, symmetry=2, split=split)
    plain_st, plain = oracle_lib.run_workload(wl, group=0, record_each_step=True)
    merged_st, merged = oracle_lib.run_workload(wl, group=2, record_each_step=True)
    ref = sv.statevector_expectations(wl.circuit.layers, wl.observable.terms, wl.state.bloch)
    np.testing.assert_allclose(plain, ref, atol=1e-10, rtol=0)
    assert len(merged_st) < len(plain_st)
    if split:
        np.testing.assert_allclose(merged, plain, atol=1e-12, rtol=0)
        np.testing.assert_allclose(plain, 1.0, atol=1e-12, rtol=0)
    else:
        assert max(abs(v - 1.0) for v in plain) > 1e-3
        assert max(abs(a - b) for a, b in zip(merged, plain)) > 1e-3
