"""Seeded synthetic inputs for Pauli propagation: circuits, observables, states.

This module holds no propagation arithmetic.  It only builds inputs: Pauli
strings (as letter strings and as X/Z bit masks), gate lists with rotation
angles, observables and product states.  Both the CPU oracle tests and the
CUDA path read their inputs from here, so the two sides see the same data.

Conventions
-----------
* A Pauli string over ``n`` qubits is a string of letters ``I X Y Z``;
  character ``q`` is qubit ``q`` (qubit 0 first).
* Bit-mask form (the symplectic encoding of Appendix E, "Lowest integer
  representation"): ``W = ceil(n/64)`` words per mask; qubit ``q`` lives in
  word ``q // 64``, bit ``q % 64``.  X sets x, Z sets z, Y sets both.
* A gate is a Pauli rotation ``exp(-i theta P / 2)`` given by ``(P, theta)``.
  Layers are lists of gates in *time order*.
* Product states are per-qubit Bloch vectors ``(bx, by, bz)``;
  ``rho = prod_q (I + bx X + by Y + bz Z) / 2``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

LETTERS = "IXYZ"


def words_for(n: int) -> int:
    """Number of 64-bit words per mask for ``n`` qubits."""
    if n < 1:
        raise ValueError("n must be >= 1")
    return (n + 63) // 64


def pauli(n: int, sites: dict) -> str:
    """Build an n-qubit letter string from {qubit: letter}."""
    s = ["I"] * n
    for q, p in sites.items():
        s[q] = p
    return "".join(s)


def to_masks(strings: Sequence[str], n: int) -> Tuple[np.ndarray, np.ndarray]:
    """Letter strings -> (x, z) uint64 arrays of shape [len(strings), W]."""
    W = words_for(n)
    m = len(strings)
    x = np.zeros((m, W), dtype=np.uint64)
    z = np.zeros((m, W), dtype=np.uint64)
    for i, s in enumerate(strings):
        if len(s) != n:
            raise ValueError(f"string {s!r} has length {len(s)}, expected {n}")
        xw = [0] * W
        zw = [0] * W
        for q, ch in enumerate(s):
            if ch in "XY":
                xw[q >> 6] |= 1 << (q & 63)
            if ch in "ZY":
                zw[q >> 6] |= 1 << (q & 63)
            if ch not in LETTERS:
                raise ValueError(f"bad letter {ch!r}")
        x[i] = xw
        z[i] = zw
    return x, z


def from_masks(x: np.ndarray, z: np.ndarray, n: int) -> List[str]:
    """(x, z) uint64 arrays [m, W] -> letter strings."""
    x = np.asarray(x, dtype=np.uint64).reshape(len(x), -1)
    z = np.asarray(z, dtype=np.uint64).reshape(len(z), -1)
    out = []
    for i in range(x.shape[0]):
        chars = []
        for q in range(n):
            xb = (int(x[i, q >> 6]) >> (q & 63)) & 1
            zb = (int(z[i, q >> 6]) >> (q & 63)) & 1
            chars.append(LETTERS[(xb and not zb) * 1 + (xb and zb) * 2 + ((not xb) and zb) * 3])
        out.append("".join(chars))
    return out


@dataclass
class Circuit:
    """A layered circuit of Pauli rotations; every layer is in time order."""
    n: int
    layers: List[List[Tuple[str, float]]] = field(default_factory=list)

    def gate_arrays(self, layer: int):
        """(gx [K, W] uint64, gz [K, W] uint64, theta [K] float64) of one layer."""
        gates = self.layers[layer]
        gx, gz = to_masks([g[0] for g in gates], self.n)
        th = np.array([g[1] for g in gates], dtype=np.float64)
        return gx, gz, th


@dataclass
class Observable:
    n: int
    terms: List[Tuple[str, float]]

    def arrays(self):
        x, z = to_masks([t[0] for t in self.terms], self.n)
        c = np.array([t[1] for t in self.terms], dtype=np.float64)
        return x, z, c


@dataclass
class ProductState:
    """Per-qubit Bloch vectors; ``basis`` holds the bits when it is a basis state."""
    n: int
    bloch: np.ndarray  # [n, 3] float64
    basis: np.ndarray | None = None  # [n] uint8 or None


# ---------------------------------------------------------------- states

def basis_state(bits: Sequence[int]) -> ProductState:
    bits = np.asarray(bits, dtype=np.uint8)
    n = len(bits)
    b = np.zeros((n, 3))
    b[:, 2] = 1.0 - 2.0 * bits
    return ProductState(n, b, bits.copy())


def neel_state(n: int) -> ProductState:
    """|0101...>: qubit q is |1> for odd q."""
    return basis_state([q % 2 for q in range(n)])


def zero_state(n: int) -> ProductState:
    return basis_state([0] * n)


def plus_state(n: int) -> ProductState:
    b = np.zeros((n, 3))
    b[:, 0] = 1.0
    return ProductState(n, b, None)


def random_product_state(n: int, seed: int) -> ProductState:
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v *= rng.uniform(0.3, 1.0, size=(n, 1))
    return ProductState(n, v, None)


# ---------------------------------------------------------- observables

def z_site(n: int, q: int = 0) -> Observable:
    return Observable(n, [(pauli(n, {q: "Z"}), 1.0)])


def mean_z(n: int) -> Observable:
    """(1/n) sum_i Z_i."""
    return Observable(n, [(pauli(n, {q: "Z"}), 1.0 / n) for q in range(n)])


def total_spin_squared(n: int) -> Observable:
    """S^2 = sum_mu (sum_i P_mu,i / 2)^2 written in Pauli strings (Eq. s2)."""
    terms = [("I" * n, 3.0 * n / 4.0)]
    for i in range(n):
        for j in range(i + 1, n):
            for p in "XYZ":
                terms.append((pauli(n, {i: p, j: p}), 0.5))
    return Observable(n, terms)


def random_observable(n: int, n_terms: int, seed: int, max_weight: int | None = None) -> Observable:
    rng = np.random.default_rng(seed)
    seen = {}
    while len(seen) < n_terms:
        if max_weight is None:
            letters = rng.integers(0, 4, size=n)
        else:
            letters = np.zeros(n, dtype=np.int64)
            w = int(rng.integers(1, max_weight + 1))
            sites = rng.choice(n, size=min(w, n), replace=False)
            letters[sites] = rng.integers(1, 4, size=len(sites))
        s = "".join(LETTERS[v] for v in letters)
        seen[s] = float(rng.normal())
    return Observable(n, list(seen.items()))


# -------------------------------------------------------------- circuits

def heisenberg_layer(n: int, theta_xx: float, theta_yy: float, theta_zz: float,
                     pairs: Sequence[Tuple[int, int]] | None = None):
    """One first-order Trotter step of sum_{i<j} (a XX + b YY + c ZZ).

    Pairs are taken in lexicographic order (outer loop), and for each pair the
    XX, YY, ZZ rotations follow in that order (inner loop).
    """
    if pairs is None:
        pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    gates = []
    for (i, j) in pairs:
        for p, th in (("X", theta_xx), ("Y", theta_yy), ("Z", theta_zz)):
            gates.append((pauli(n, {i: p, j: p}), th))
    return gates


def ring_layer(n: int, theta_j: float, theta_x: float, theta_z: float):
    """RZZ(theta_j) on bonds (i, i+1 mod n), then RX(theta_x), then RZ(theta_z)."""
    gates = []
    for i in range(n):
        gates.append((pauli(n, {i: "Z", (i + 1) % n: "Z"}) if n > 1 else "Z", theta_j))
    for i in range(n):
        gates.append((pauli(n, {i: "X"}), theta_x))
    for i in range(n):
        gates.append((pauli(n, {i: "Z"}), theta_z))
    return gates


def torus_layer(lx: int, ly: int, theta_j: float, theta_x: float, theta_z: float):
    """One Trotter step on an lx x ly torus (qubit q = x + lx y): RZZ on every
    horizontal bond, then on every vertical bond, then RX and RZ on every
    site.  Each group of gates commutes and is mapped onto itself by the
    lattice translations."""
    n = lx * ly
    gates = []
    for y in range(ly):
        for x in range(lx):
            gates.append((pauli(n, {x + lx * y: "Z", (x + 1) % lx + lx * y: "Z"}), theta_j))
    for y in range(ly):
        for x in range(lx):
            gates.append((pauli(n, {x + lx * y: "Z", x + lx * ((y + 1) % ly): "Z"}), theta_j))
    gates += [(pauli(n, {q: "X"}), theta_x) for q in range(n)]
    gates += [(pauli(n, {q: "Z"}), theta_z) for q in range(n)]
    return gates


def tilted_ising_layer(n: int, delta: float, hx: float = 1.4, hz: float = 0.9045):
    """Trotter layer of H = -sum ZZ - hz sum Z - hx sum X on a ring.

    exp(-i d ZZ) exp(-i hz d Z) exp(-i hx d X) written as rotations
    exp(-i theta P / 2) with theta = 2 * delta * coupling.
    """
    gates = []
    for i in range(n):
        gates.append((pauli(n, {i: "Z", (i + 1) % n: "Z"}), 2.0 * delta))
    for i in range(n):
        gates.append((pauli(n, {i: "Z"}), 2.0 * hz * delta))
    for i in range(n):
        gates.append((pauli(n, {i: "X"}), 2.0 * hx * delta))
    return gates


def random_circuit(n: int, n_layers: int, gates_per_layer: int, seed: int,
                   max_support: int = 3) -> Circuit:
    """Random Pauli rotations with random supports (1..max_support qubits)."""
    rng = np.random.default_rng(seed)
    layers = []
    for _ in range(n_layers):
        gates = []
        for _ in range(gates_per_layer):
            k = int(rng.integers(1, min(max_support, n) + 1))
            sites = rng.choice(n, size=k, replace=False)
            d = {int(q): LETTERS[int(rng.integers(1, 4))] for q in sites}
            gates.append((pauli(n, d), float(rng.uniform(-math.pi, math.pi))))
        layers.append(gates)
    return Circuit(n, layers)


# ---------------------------------------------------- named workloads

@dataclass
class Workload:
    name: str
    circuit: Circuit
    observable: Observable
    state: ProductState
    eps: float = 0.0
    max_weight: int = -1
    noise_p: float = 0.0
    noise_mode: int = 0  # 0 none, 1 per gate, 2 per layer
    symmetry: int = 0    # 0 none, 1 Z_n, 2 S_n


def config0_heisenberg(n: int = 8, dt: float = 0.05, steps: int = 3) -> Workload:
    """All-to-all Heisenberg, theta = 2 dt for XX, YY, ZZ; Z_0; Neel; plain FP64."""
    layer = heisenberg_layer(n, 2 * dt, 2 * dt, 2 * dt)
    return Workload("heisenberg_a2a_n%d_dt%g_x%d" % (n, dt, steps),
                    Circuit(n, [list(layer) for _ in range(steps)]),
                    z_site(n, 0), neel_state(n))


def config1_ring(n: int = 32, steps: int = 20, theta_j: float = 0.4, theta_x: float = 0.6,
                 theta_z: float = 0.3, eps: float = 1e-4, max_weight: int = 10,
                 symmetry: int = 0) -> Workload:
    """Translation-symmetric ring: RZZ, RX, RZ layers; (1/n) sum Z; |0...0>."""
    layer = ring_layer(n, theta_j, theta_x, theta_z)
    return Workload("ring_n%d_x%d" % (n, steps), Circuit(n, [list(layer) for _ in range(steps)]),
                    mean_z(n), zero_state(n), eps=eps, max_weight=max_weight, symmetry=symmetry)


def config2_all_to_all(n: int = 64, dt: float = 0.02, steps: int = 10, p: float = 0.01,
                       eps: float = 1e-5, noise_mode: int = 1, symmetry: int = 0) -> Workload:
    """All-to-all Heisenberg with per-gate depolarising damping; (1/n) sum Z; Neel."""
    layer = heisenberg_layer(n, 2 * dt, 2 * dt, 2 * dt)
    return Workload("heisenberg_a2a_n%d_x%d_p%g" % (n, steps, p),
                    Circuit(n, [list(layer) for _ in range(steps)]),
                    mean_z(n), neel_state(n), eps=eps, noise_p=p, noise_mode=noise_mode,
                    symmetry=symmetry)


def xxz_all_to_all(n: int, delta_t: float, steps: int, J: float = 1.0, Delta: float = -1.8,
                   eps: float = 0.0, symmetry: int = 0, gamma: float = 0.0,
                   split: bool = False) -> Workload:
    """Eq. hamXXZ with alpha = 0: h_ij = -J (XX + YY + (Delta+1) ZZ); S^2 / S_0^2; |+>^n.

    split=False: one layer per Trotter step, pairs (i, j) in lexicographic
    order with XX, YY, ZZ inner.  split=True: each step is three layers (all
    XX over the pairs, then all YY, then all ZZ).  Each of those is a set of
    commuting gates invariant under S_n, so a runner that merges at layer
    boundaries merges after every sublayer.  The per-step damping gamma is
    only defined for split=False.
    """
    th_xy = -2.0 * J * delta_t
    th_zz = -2.0 * J * (Delta + 1.0) * delta_t
    layer = heisenberg_layer(n, th_xy, th_xy, th_zz)
    if not split:
        layers = [list(layer) for _ in range(steps)]
    else:
        if gamma > 0:
            raise ValueError("per-step damping is defined for unsplit steps only")
        subs = [[g for g in layer if set(g[0].replace("I", "")) == {p}] for p in "XYZ"]
        layers = [list(sub) for _ in range(steps) for sub in subs]
    obs = total_spin_squared(n)
    s0 = (n / 2.0) * (n / 2.0 + 1.0)  # <+|S^2|+>: the figure's normalisation S_0^2
    obs = Observable(n, [(s, c / s0) for s, c in obs.terms])
    return Workload("xxz_a2a_n%d_x%d%s" % (n, steps, "_split" if split else ""), Circuit(n, layers),
                    obs, plus_state(n), eps=eps,
                    noise_p=gamma, noise_mode=2 if gamma > 0 else 0, symmetry=symmetry)


def split_sublayers(wl: Workload, parts: int = 3) -> Workload:
    """The same workload with every layer cut into `parts` consecutive
    sublayers of equal length, each applied as a layer of its own.  For the
    ring layer these are all RZZ, all RX and all RZ gates: each is a set of
    commuting gates mapped onto itself by the translations, so a merge may
    follow any of them."""
    layers = []
    for layer in wl.circuit.layers:
        if len(layer) % parts:
            raise ValueError("layer length is not a multiple of parts")
        k = len(layer) // parts
        layers.extend([list(layer[i * k:(i + 1) * k]) for i in range(parts)])
    return Workload(wl.name + "_sub%d" % parts, Circuit(wl.circuit.n, layers), wl.observable,
                    wl.state, eps=wl.eps, max_weight=wl.max_weight, noise_p=wl.noise_p,
                    noise_mode=wl.noise_mode, symmetry=wl.symmetry)


def merge_schedule(n_layers: int, every: int) -> List[bool]:
    """Merge flags in application order (the last layer of the circuit comes
    first): a symmetry merge after every `every`-th applied layer and after the
    final one."""
    if every < 1:
        raise ValueError("every must be >= 1")
    return [((a + 1) % every == 0) or (a == n_layers - 1) for a in range(n_layers)]


def torus_ising(lx: int, ly: int, steps: int, theta_j: float = 0.4, theta_x: float = 0.6,
                theta_z: float = 0.3, eps: float = 0.0, max_weight: int = -1,
                symmetry: int = 0) -> Workload:
    """The ring workload's gate set on an lx x ly torus: (1/n) sum Z_i, |0...0>."""
    n = lx * ly
    layer = torus_layer(lx, ly, theta_j, theta_x, theta_z)
    return Workload("torus_%dx%d_x%d" % (lx, ly, steps), Circuit(n, [list(layer) for _ in range(steps)]),
                    mean_z(n), zero_state(n), eps=eps, max_weight=max_weight, symmetry=symmetry)


def batched_ring_angles(n_sets: int = 256, seed: int = 0) -> np.ndarray:
    """[n_sets, 3] angle triples (theta_J, theta_x, theta_z) ~ U[0, pi/2]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(0.0, math.pi / 2, size=(n_sets, 3))


def serving_stream(n_jobs: int = 2000, rate: float = 200.0, seed: int = 0):
    """Poisson-arrival job descriptions for the serving workload."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += float(rng.exponential(1.0 / rate))
        n = int(rng.choice([16, 32, 64, 128]))
        family = "ring" if rng.uniform() < 0.5 else "a2a"
        steps = int(rng.integers(5, 41))
        eps = float(10 ** rng.uniform(-6, -3))
        group = int(rng.integers(0, 3))
        if family == "ring" and group == 2:
            group = 1
        if family == "a2a" and group == 1:
            group = 2
        angles = rng.uniform(0.0, math.pi / 2, size=3)
        jobs.append(dict(job=j, arrival=t, n=n, family=family, steps=steps, eps=eps,
                         group=group, angles=angles.tolist()))
    return jobs
