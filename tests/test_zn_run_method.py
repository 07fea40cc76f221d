"""The Z_n representative method of the CUDA kernels, checked on the CPU.

Algorithm 2 takes the translation of a string with the lowest digit integer
(I=0, X=1, Y=2, Z=3, qubit q the digit of weight 4^q) by trying all n
translations.  The kernels reach the same string without trying them all:

* the lowest translation has the smallest digit d present on its top qubit,
  and the longer its top run of d's the lower it is, so only translations
  that put a longest cyclic run of d on qubits n-L..n-1 are candidates;
* the longest runs are found by walking the gaps between the sites that
  differ from d (when at most 12 do) or by shrinking the mask of d's,
  cur &= T cur, until one more step would empty it;
* the candidates are narrowed on the next two digits below the run (high
  bit of the digit, then low bit), and any still tied are compared whole.

This file restates those steps in Python on digit lists -- independently of
the CUDA source and of the oracle -- and compares the result with the
brute-force minimum over every translation, on random, low-weight, periodic
and one-letter strings for n = 1 to 70 and a few larger n.  The CUDA path
itself is compared with the oracle bit for bit by the GPU tests.
"""
import numpy as np
import pytest

GAP_WALK_MAX = 12  # at most this many sites differ from d: walk the gaps
NARROW = 2         # digits below the run compared on masks


def digit_int(s):
    return sum(d << (2 * q) for q, d in enumerate(s))


def translate(s, j):
    """T^j: qubit q takes the digit of site q + j (mod n)."""
    n = len(s)
    return [s[(q + j) % n] for q in range(n)]


def brute_force(s):
    return min((translate(s, j) for j in range(len(s))), key=digit_int)


def longest_runs_by_gaps(s, d):
    """Translations j that end a longest cyclic run of d just before site j."""
    n = len(s)
    others = [q for q in range(n) if s[q] != d]
    L, cand = -1, set()

    def take(gap, j):
        nonlocal L, cand
        if gap > L:
            L, cand = gap, set()
        if gap == L:
            cand.add(j)

    for prev, q in zip(others, others[1:]):
        take(q - prev - 1, q)
    take(others[0] + n - others[-1] - 1, others[0])  # the run wrapping past qubit n-1
    return L, cand


def longest_runs_by_shrinking(s, d):
    n = len(s)
    cur = {q for q in range(n) if s[q] == d}
    L = 1
    while True:
        nxt = {p for p in cur if (p + 1) % n in cur}  # cur & T cur
        if not nxt:
            break
        cur, L = nxt, L + 1
    # bit p marks a window p..p+L-1 of d's; the translation starts after it
    return L, {(p + L) % n for p in cur}


def run_method(s):
    n = len(s)
    d = min(s)
    n_other = sum(1 for v in s if v != d)
    if n_other == 0:
        return list(s)
    if n_other <= GAP_WALK_MAX:
        L, cand = longest_runs_by_gaps(s, d)
    else:
        L, cand = longest_runs_by_shrinking(s, d)
    for kk in range(1, NARROW + 1):
        if kk > n - L or len(cand) < 2:
            break
        # the kk-th digit below the run of translation j sits at site j - L - kk
        below = {j: s[(j - L - kk) % n] for j in cand}
        hi0 = {j for j in cand if below[j] >> 1 == 0}
        if hi0:
            cand = hi0
        lo0 = {j for j in cand if below[j] & 1 == 0}
        if lo0:
            cand = lo0
    return min((translate(s, j) for j in sorted(cand)), key=digit_int)


def _cases(n, rng):
    out = [list(rng.integers(0, 4, n)) for _ in range(40)]  # random letters
    for _ in range(40):  # low weight: mostly I, a few letters (gap walk)
        s = [0] * n
        for q in rng.choice(n, size=int(rng.integers(0, min(n, 14) + 1)), replace=False):
            s[int(q)] = int(rng.integers(1, 4))
        out.append(s)
    for _ in range(20):  # periodic: several translations give the same string
        p = int(rng.integers(1, n + 1))
        if n % p == 0:
            block = list(rng.integers(0, 4, p))
            out.append(block * (n // p))
    for _ in range(20):  # no identity: d = X, Y or Z, long runs of it
        s = list(rng.integers(1, 4, n))
        for _ in range(int(rng.integers(0, 3))):
            a, ln = int(rng.integers(0, n)), int(rng.integers(1, n + 1))
            for t in range(ln):
                s[(a + t) % n] = s[a]
        out.append(s)
    out += [[v] * n for v in range(4)]  # one letter everywhere
    return [[int(v) for v in s] for s in out]


@pytest.mark.parametrize("n", list(range(1, 71)) + [96, 128, 130, 256])
def test_run_method_equals_the_lowest_translation(n):
    rng = np.random.default_rng(7000 + n)
    for s in _cases(n, rng):
        assert run_method(s) == brute_force(s), s


def test_both_run_finders_agree():
    """Where both apply, the gap walk and the shrinking mask find the same
    longest runs."""
    rng = np.random.default_rng(5)
    for _ in range(2000):
        n = int(rng.integers(2, 40))
        s = [int(v) for v in rng.integers(0, 4, n)]
        d = min(s)
        if all(v == d for v in s):
            continue
        assert longest_runs_by_gaps(s, d) == longest_runs_by_shrinking(s, d), s
