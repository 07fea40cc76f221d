"""Host-side symmetry checks on the CPU (no GPU).

pp_create and pp_apply_layer refuse (PP_ERR_SYMMETRY) a layer whose gate
multiset, with angles, the declared group does not map onto itself, and an
observable / state pair of which neither is invariant (the condition of
Theorem 1).  They test only the group's generators.  The code sits in
paper_2512_12094_gb300/csrc/pp_symmetry_host.h; here the same header is
compiled into a small driver (tests/symmetry_main.cpp) and compared with
brute force over every element of the group, built in this file from the
group's definition: the generators must generate the whole group, and
invariance under the generators must equal invariance under every element.
"""
import collections
import itertools
import os
import shutil
import subprocess

import numpy as np
import pytest

import pp_inputs as pi

HERE = os.path.dirname(os.path.abspath(__file__))
ZN, SN, DN, TORUS = 1, 2, 3, 4


def torus(lx):
    return TORUS | (lx << 8)


def elements(group, n):
    """Every element of the group as a site map (the letter of q moves to m[q])."""
    kind, lx = group & 0xFF, group >> 8
    if kind == ZN:
        return {tuple((q + j) % n for q in range(n)) for j in range(n)}
    if kind == DN:
        return ({tuple((q + j) % n for q in range(n)) for j in range(n)} |
                {tuple((j - q) % n for q in range(n)) for j in range(n)})
    if kind == SN:
        return set(itertools.permutations(range(n)))
    if kind == TORUS:
        ly = n // lx
        return {tuple((q % lx + dx) % lx + lx * ((q // lx + dy) % ly) for q in range(n))
                for dx in range(lx) for dy in range(ly)}
    raise ValueError(group)


def act(m, s):
    out = [None] * len(s)
    for q, ch in enumerate(s):
        out[m[q]] = ch
    return "".join(out)


@pytest.fixture(scope="module", params=["plain", "asan_ubsan"])
def driver(request, tmp_path_factory):
    """The driver built plainly, and with AddressSanitizer and
    UndefinedBehaviorSanitizer (no recovery: an invalid access or undefined
    behaviour ends the run with an error)."""
    if shutil.which("g++") is None:
        pytest.skip("no g++")
    flags = ["-O1", "-std=c++17", "-Wall", "-Wextra", "-Werror"]
    if request.param == "asan_ubsan":
        flags += ["-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
                  "-fno-omit-frame-pointer"]
    exe = str(tmp_path_factory.mktemp("symmetry_" + request.param) / "symmetry")
    r = subprocess.run(["g++", *flags, os.path.join(HERE, "symmetry_main.cpp"), "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0 and request.param == "asan_ubsan":
        pytest.skip("g++ without sanitizer runtimes: " + r.stderr.strip()[-200:])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1", UBSAN_OPTIONS="print_stacktrace=1")

    def run(text):
        out = subprocess.run([exe], input=text, capture_output=True, text=True, timeout=120,
                             env=env)
        assert out.returncode == 0, out.stderr
        assert "runtime error" not in out.stderr and "AddressSanitizer" not in out.stderr
        return out.stdout.strip().splitlines()
    return run


def multiset_request(group, n, gates):
    x, z = pi.to_masks([s for s, _ in gates], n)
    lines = [" ".join(str(int(w)) for w in list(x[i]) + list(z[i])) + " " + repr(float(v))
             for i, (_, v) in enumerate(gates)]
    return f"multiset {group} {n} {len(gates)}\n" + "".join(ln + "\n" for ln in lines)


def brute_invariant(group, n, gates):
    base = collections.Counter(gates)
    return all(collections.Counter((act(m, s), v) for s, v in gates) == base
               for m in elements(group, n))


CASES = [(ZN, 1), (ZN, 2), (ZN, 3), (ZN, 5), (ZN, 8), (SN, 2), (SN, 3), (SN, 4), (SN, 5),
         (DN, 3), (DN, 4), (DN, 6), (torus(2), 6), (torus(3), 9), (torus(4), 8), (torus(1), 3)]


@pytest.mark.parametrize("group,n", CASES)
def test_generators_generate_the_group(driver, group, n):
    out = driver(f"gens {group} {n}\n")
    gens = [tuple(int(v) for v in line.split()) for line in out[1:]]
    assert int(out[0]) == len(gens)
    want = elements(group, n)
    if n < 2:
        assert gens == []
        return
    assert all(g in want for g in gens)
    closure, frontier = {tuple(range(n))}, [tuple(range(n))]
    while frontier:
        nxt = []
        for a in frontier:
            for g in gens:
                c = tuple(g[a[q]] for q in range(n))
                if c not in closure:
                    closure.add(c)
                    nxt.append(c)
        frontier = nxt
    assert closure == want


@pytest.mark.parametrize("group,n", CASES)
def test_multiset_invariance_equals_brute_force(driver, group, n):
    """Orbit-closed gate multisets with one angle per orbit are invariant;
    dropping a gate, changing one angle, duplicating a gate or adding a
    random gate breaks that (almost always).  The driver's answer, from the
    generators, must equal brute force over every element in every case."""
    rng = np.random.default_rng(1000 * group + n)
    els = sorted(elements(group, n))
    req, want = [], []
    for _ in range(12):
        gates = []
        for _ in range(int(rng.integers(1, 4))):
            s = "".join(rng.choice(list("IXYZ"), size=n))
            angle = float(rng.choice([0.1, 0.25, -0.7]))
            gates += [(t, angle) for t in sorted({act(m, s) for m in els})]
        extra = ("".join(rng.choice(list("XYZ"), size=n)), 0.1)
        variants = [gates, gates[1:], gates + [gates[0]], gates + [extra]]
        k = int(rng.integers(len(gates)))
        variants.append(gates[:k] + [(gates[k][0], gates[k][1] + 1.0)] + gates[k + 1:])
        for v in variants:
            req.append(multiset_request(group, n, v))
            want.append(brute_invariant(group, n, v))
    got = [line == "1" for line in driver("".join(req))]
    assert got == want
    assert any(want)
    if len(els) > 1:
        assert not all(want)


def test_layers_of_the_workloads(driver):
    """The ring layer is invariant under translations and reflections but not
    under all permutations; the all-to-all Heisenberg layer is invariant
    under all permutations; a chiral ring layer (X on q, Y on q+1) is
    invariant under translations only.  Also for 70 qubits (two words)."""
    for n in (6, 70):
        ring = pi.ring_layer(n, 0.4, 0.6, 0.3)
        chiral = [(pi.pauli(n, {q: "X", (q + 1) % n: "Y"}), 0.2) for q in range(n)]
        heis = pi.heisenberg_layer(n, 0.1, 0.1, 0.1) if n <= 8 else None
        req = [multiset_request(g, n, ring) for g in (ZN, DN, SN)]
        req += [multiset_request(g, n, chiral) for g in (ZN, DN)]
        if heis is not None:
            req += [multiset_request(g, n, heis) for g in (SN, ZN)]
        got = [line == "1" for line in driver("".join(req))]
        want = [True, True, False, True, False] + ([True, True] if heis is not None else [])
        assert got == want


@pytest.mark.parametrize("group,n", CASES)
def test_product_state_invariance_equals_brute_force(driver, group, n):
    rng = np.random.default_rng(7 + n + group)
    states = [np.tile([0.0, 0.0, 1.0], (n, 1)),                         # |0...0>
              np.array([[0.0, 0.0, (-1.0) ** q] for q in range(n)]),     # Neel
              rng.normal(size=(n, 3))]
    els = elements(group, n)
    req, want = [], []
    for b in states:
        req.append(f"bloch {group} {n}\n" + " ".join(repr(float(v)) for v in b.reshape(-1)) + "\n")
        want.append(all(np.array_equal(b[list(m)], b) for m in els))
    assert [line == "1" for line in driver("".join(req))] == want


def test_group_codes(driver):
    cases = [(0, 5, True), (ZN, 5, True), (SN, 5, True), (DN, 5, True), (torus(2), 6, True),
             (torus(3), 6, True), (torus(6), 6, True), (torus(4), 6, False), (torus(0), 6, False),
             (torus(7), 6, False), (TORUS + 1, 6, False), (-1, 6, False), (ZN | (2 << 8), 6, False)]
    got = driver("".join(f"valid {c} {n}\n" for c, n, _ in cases))
    assert [line == "1" for line in got] == [w for _, _, w in cases]
