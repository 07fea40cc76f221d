"""The popcount sign rule of the CUDA gate pass, checked on the CPU.

For a gate exp(-i theta P / 2) and a string Q that anticommutes with P, the
child term is sin(theta) (i P Q) with i P Q = sigma R, R = (xP ^ xQ, zP ^ zQ)
and sigma = +-1 (App. A, Prop. 1 proof).  The kernels take sigma from bit
masks: with one site written as i^(x z) X^x Z^z,

    P Q = i^E R,  E = popc(xP & zP) + popc(xQ & zQ) + 2 popc(zP & xQ)
                      - popc((xP ^ xQ) & (zP ^ zQ)),

so i P Q = i^(E+1) R, and E + 1 is even when P and Q anticommute.  This file
restates that formula in Python and compares sigma with the one read off
dense Pauli matrices (Kronecker products) for every pair of strings on one
and two qubits and for random pairs on up to six qubits.
"""
import itertools

import numpy as np
import pytest

MATS = {
    "I": np.eye(2, dtype=complex),
    "X": np.array([[0, 1], [1, 0]], dtype=complex),
    "Y": np.array([[0, -1j], [1j, 0]], dtype=complex),
    "Z": np.array([[1, 0], [0, -1]], dtype=complex),
}


def masks(s):
    """(x, z) bit masks of a letter string, qubit q in bit q."""
    x = sum(1 << q for q, ch in enumerate(s) if ch in "XY")
    z = sum(1 << q for q, ch in enumerate(s) if ch in "YZ")
    return x, z


def letters(x, z, n):
    return "".join("IXZY"[((x >> q) & 1) | (((z >> q) & 1) << 1)] for q in range(n))


def dense(s):
    m = np.eye(1, dtype=complex)
    for ch in reversed(s):  # qubit 0 is the least significant factor
        m = np.kron(m, MATS[ch])
    return m


def popc(v):
    return bin(v).count("1")


def sigma_popcount(p, q):
    (px, pz), (qx, qz) = masks(p), masks(q)
    e = popc(px & pz) + popc(qx & qz) + 2 * popc(pz & qx) - popc((px ^ qx) & (pz ^ qz))
    return 1 if ((e + 1) & 3) == 0 else -1


def sigma_dense(p, q):
    """i P Q = sigma R from the matrices; None when P and Q commute."""
    n = len(p)
    P, Q = dense(p), dense(q)
    if np.allclose(P @ Q, Q @ P):
        return None
    (px, pz), (qx, qz) = masks(p), masks(q)
    R = dense(letters(px ^ qx, pz ^ qz, n))
    c = np.trace(R.conj().T @ (1j * P @ Q)) / 2 ** n
    assert np.allclose(1j * P @ Q, c * R)
    assert abs(c.imag) < 1e-12 and abs(abs(c.real) - 1) < 1e-12
    return int(round(c.real))


@pytest.mark.parametrize("n", [1, 2])
def test_every_anticommuting_pair(n):
    seen = 0
    for p in itertools.product("IXYZ", repeat=n):
        for q in itertools.product("IXYZ", repeat=n):
            p_s, q_s = "".join(p), "".join(q)
            want = sigma_dense(p_s, q_s)
            if want is None:
                continue
            seen += 1
            assert sigma_popcount(p_s, q_s) == want, (p_s, q_s)
    # every P other than I anticommutes with half of the 4^n strings
    assert seen == (4 ** n - 1) * 4 ** n // 2


def test_random_pairs_up_to_six_qubits():
    rng = np.random.default_rng(11)
    checked = 0
    while checked < 300:
        n = int(rng.integers(3, 7))
        p = "".join(rng.choice(list("IXYZ"), size=n))
        q = "".join(rng.choice(list("IXYZ"), size=n))
        want = sigma_dense(p, q)
        if want is None:
            continue
        assert sigma_popcount(p, q) == want, (p, q)
        checked += 1
