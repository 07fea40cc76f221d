"""Dense Schroedinger-picture simulation used to pin the oracle (test infrastructure).

A state vector (n <= ~12) or density matrix (n <= ~6) evolved gate by gate in
time order with numpy, and <O> = Tr[rho O] read at the end.  It shares no
arithmetic with the oracle's Heisenberg map: gates are applied to the state as
U = cos(theta/2) I - i sin(theta/2) P built from the 2x2 Pauli matrices, and
depolarising noise is the channel rho -> (1-p) rho + p Tr_q(rho) (x) I/2.
"""
from __future__ import annotations

import numpy as np

_I = np.eye(2, dtype=complex)
_X = np.array([[0, 1], [1, 0]], dtype=complex)
_Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
_Z = np.array([[1, 0], [0, -1]], dtype=complex)
PAULI = {"I": _I, "X": _X, "Y": _Y, "Z": _Z}


def _apply_1q(psi: np.ndarray, M: np.ndarray, q: int) -> np.ndarray:
    out = np.tensordot(M, psi, axes=([1], [q]))
    return np.moveaxis(out, 0, q)


def apply_pauli(psi: np.ndarray, p: str) -> np.ndarray:
    """P |psi> for a letter string P; psi has shape [2] * n."""
    for q, ch in enumerate(p):
        if ch != "I":
            psi = _apply_1q(psi, PAULI[ch], q)
    return psi


def product_state_vector(bloch: np.ndarray) -> np.ndarray:
    """Pure product state from unit Bloch vectors [n, 3] -> tensor [2]*n."""
    psi = np.ones((), dtype=complex)
    for bx, by, bz in bloch:
        r = np.sqrt(bx * bx + by * by + bz * bz)
        if abs(r - 1.0) > 1e-12:
            raise ValueError("state-vector needs pure (unit) Bloch vectors")
        th = np.arccos(np.clip(bz, -1.0, 1.0))
        ph = np.arctan2(by, bx)
        v = np.array([np.cos(th / 2), np.exp(1j * ph) * np.sin(th / 2)])
        psi = np.multiply.outer(psi, v)
    return psi


def evolve_state(psi: np.ndarray, gates) -> np.ndarray:
    """Apply exp(-i theta P / 2) for (P, theta) in time order."""
    for p, th in gates:
        psi = np.cos(th / 2) * psi - 1j * np.sin(th / 2) * apply_pauli(psi, p)
    return psi


def expect_state(psi: np.ndarray, terms) -> float:
    """<psi| sum c_s s |psi>."""
    flat = psi.reshape(-1)
    acc = 0.0
    for p, c in terms:
        acc += c * np.vdot(flat, apply_pauli(psi, p).reshape(-1)).real
    return float(acc)


def statevector_expectations(circuit_layers, observable_terms, bloch):
    """<O> after each successive layer (time order) from a pure product state."""
    psi = product_state_vector(np.asarray(bloch, dtype=float))
    vals = []
    for layer in circuit_layers:
        psi = evolve_state(psi, layer)
        vals.append(expect_state(psi, observable_terms))
    return vals


# ------------------------------------------------------------ density matrix

def full_matrix(p: str) -> np.ndarray:
    """Dense 2^n x 2^n matrix of a letter string, qubit 0 as the first factor."""
    m = np.ones((1, 1), dtype=complex)
    for ch in p:
        m = np.kron(m, PAULI[ch])
    return m


def product_density(bloch: np.ndarray) -> np.ndarray:
    rho = np.ones((1, 1), dtype=complex)
    for bx, by, bz in bloch:
        r1 = 0.5 * (_I + bx * _X + by * _Y + bz * _Z)
        rho = np.kron(rho, r1)
    return rho


def depolarize(rho: np.ndarray, n: int, q: int, p: float) -> np.ndarray:
    """rho -> (1-p) rho + p Tr_q(rho) (x) I_q / 2 on qubit q."""
    t = rho.reshape([2] * (2 * n))
    tr = np.trace(t, axis1=q, axis2=n + q)  # shape [2]*(2n-2)
    # re-insert identity/2 on qubit q
    eye = 0.5 * np.eye(2, dtype=complex)
    full = np.multiply.outer(tr, eye)  # axes: others..., q, q'
    # move the two new axes to positions q and n+q
    dims = full.ndim
    full = np.moveaxis(full, [dims - 2, dims - 1], [q, n + q])
    return (1 - p) * rho + p * full.reshape(rho.shape)


def density_expectations(n, circuit_layers, observable_terms, bloch, p_gate=0.0, gamma_layer=0.0):
    """<O> after each layer with per-gate depolarising noise on the gate's
    support (strength p_gate) and/or per-layer noise on every qubit with
    1 - p = exp(-gamma_layer)."""
    rho = product_density(np.asarray(bloch, dtype=float))
    dim = 2 ** n
    O = np.zeros((dim, dim), dtype=complex)
    for s, c in observable_terms:
        O += c * full_matrix(s)
    vals = []
    for layer in circuit_layers:
        for s, th in layer:
            U = np.cos(th / 2) * np.eye(dim) - 1j * np.sin(th / 2) * full_matrix(s)
            rho = U @ rho @ U.conj().T
            if p_gate > 0:
                for q, ch in enumerate(s):
                    if ch != "I":
                        rho = depolarize(rho, n, q, p_gate)
        if gamma_layer > 0:
            for q in range(n):
                rho = depolarize(rho, n, q, 1.0 - np.exp(-gamma_layer))
        vals.append(float(np.trace(rho @ O).real))
    return vals


def heisenberg_decompose(n: int, gates, q_string: str):
    """Pauli coefficients of U^dag Q U (U = gates in time order) by brute force
    over all 4^n strings: c_R = Tr[R U^dag Q U] / 2^n.  Tiny n only."""
    dim = 2 ** n
    U = np.eye(dim, dtype=complex)
    for s, th in gates:
        G = np.cos(th / 2) * np.eye(dim) - 1j * np.sin(th / 2) * full_matrix(s)
        U = G @ U
    H = U.conj().T @ full_matrix(q_string) @ U
    out = {}
    import itertools
    for letters in itertools.product("IXYZ", repeat=n):
        r = "".join(letters)
        c = np.trace(full_matrix(r) @ H).real / dim
        if abs(c) > 1e-13:
            out[r] = c
    return out
