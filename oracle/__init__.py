"""CPU oracle for symmetry-merging Pauli propagation (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it.

``oracle.cpp`` is the plain restatement of the method (a hash map of Pauli
strings kept as per-qubit letters); ``statevector.py`` is an independent dense
simulation used to pin it.  The oracle follows, in order:

* Algorithm 1 (symmetry PP): ingest + merge O, then per layer propagate and
  merge by orbit representatives (Eq. O-merging), then Tr[rho O_0];
* Appendix A / Prop. 1 proof: per-gate Pauli-rotation branch rule;
* Algorithm 2 (Z_n) and Algorithm 3 (S_n): lowest-integer representatives.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

GROUP_NONE, GROUP_ZN, GROUP_SN = 0, 1, 2
NOISE_NONE, NOISE_PER_GATE, NOISE_PER_LAYER = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile oracle.cpp into liboracle.so (plain g++, no FMA contraction).

    With PP_ORACLE_SO set, that prebuilt library is used instead and nothing is
    compiled: the mutation test points the pins at copies of the oracle with a
    planted mistake this way."""
    override = os.environ.get("PP_ORACLE_SO")
    if override:
        return override
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared",
               _SRC, "-o", _LIB + ".tmp"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    P = ctypes.c_void_p
    u64p = ctypes.POINTER(ctypes.c_uint64)
    f64p = ctypes.POINTER(ctypes.c_double)
    lib.orc_create.restype = P
    lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_longlong, u64p, u64p, f64p, ctypes.c_int,
                               ctypes.c_double, ctypes.c_int]
    lib.orc_destroy.argtypes = [P]
    lib.orc_size.restype = ctypes.c_longlong
    lib.orc_size.argtypes = [P]
    lib.orc_updates.restype = ctypes.c_double
    lib.orc_updates.argtypes = [P]
    lib.orc_export.argtypes = [P, u64p, u64p, f64p]
    lib.orc_apply_gate.argtypes = [P, u64p, u64p, ctypes.c_double, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_int]
    lib.orc_damp_layer.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_int]
    lib.orc_symmetry_merge.argtypes = [P, ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lib.orc_truncate.argtypes = [P, ctypes.c_double, ctypes.c_int]
    lib.orc_apply_layer.argtypes = [P, ctypes.c_int, u64p, u64p, f64p, ctypes.c_int,
                                    ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    lib.orc_expect.restype = ctypes.c_double
    lib.orc_expect.argtypes = [P, f64p, ctypes.c_int]
    lib.orc_canonical.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_int, u64p, u64p,
                                  u64p, u64p]
    lib.orc_sym_overlap.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_int, u64p, u64p,
                                    f64p, f64p]
    lib.orcb_create.restype = P
    lib.orcb_create.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_int, u64p, u64p, f64p,
                                ctypes.c_int, ctypes.c_double, ctypes.c_int]
    lib.orcb_destroy.argtypes = [P]
    lib.orcb_size.restype = ctypes.c_longlong
    lib.orcb_size.argtypes = [P]
    lib.orcb_updates.restype = ctypes.c_double
    lib.orcb_updates.argtypes = [P]
    lib.orcb_apply_layer.argtypes = [P, ctypes.c_int, u64p, u64p, f64p, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
    lib.orcb_expect.argtypes = [P, f64p, ctypes.c_int, f64p]
    lib.orcb_export.argtypes = [P, u64p, u64p, f64p]
    _lib = lib
    return lib


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


# Group codes shared with the library's C ABI (plain integers): 1 = Z_n,
# 2 = S_n, 3 = D_n (rotations and reflections of a ring), and
# torus_group(Lx) = translations of an Lx x (n / Lx) torus, qubit q = x + Lx y.
ZN, SN, DN = 1, 2, 3


def torus_group(lx: int) -> int:
    return 4 | (lx << 8)


class OracleState:
    """Heisenberg-picture operator O = sum_s c_s s held by the C++ oracle."""

    def __init__(self, n: int, x, z, coef, group: int = 0, eps: float = 0.0,
                 max_weight: int = -1):
        lib = _load()
        self.n = n
        self.W = (n + 63) // 64
        xa, xp = _u64(np.asarray(x).reshape(-1, self.W))
        za, zp = _u64(np.asarray(z).reshape(-1, self.W))
        ca, cp = _f64(coef)
        self._h = lib.orc_create(n, len(ca), xp, zp, cp, group, eps, max_weight)
        self.group = group
        self.eps = eps
        self.max_weight = max_weight

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    def __len__(self):
        return int(_lib.orc_size(self._h))

    @property
    def updates(self) -> float:
        return float(_lib.orc_updates(self._h))

    def apply_gate(self, px, pz, theta, noise_mode=0, p=0.0):
        pa, pp = _u64(np.asarray(px).reshape(-1))
        qa, qp = _u64(np.asarray(pz).reshape(-1))
        _lib.orc_apply_gate(self._h, pp, qp, float(theta), noise_mode, p, self.eps,
                            self.max_weight)

    def apply_layer(self, gx, gz, theta, noise_mode=0, p=0.0, group: Optional[int] = None):
        """Gates in time order; applied last-to-first; then merge if group != 0."""
        g = self.group if group is None else group
        ga, gp = _u64(gx)
        ha, hp = _u64(gz)
        ta, tp = _f64(theta)
        _lib.orc_apply_layer(self._h, len(ta), gp, hp, tp, noise_mode, p, self.eps,
                             self.max_weight, g)

    def symmetry_merge(self, group: int):
        _lib.orc_symmetry_merge(self._h, group, self.eps, self.max_weight)

    def truncate(self, eps: float, max_weight: int):
        _lib.orc_truncate(self._h, eps, max_weight)

    def expect(self, bloch, group: Optional[int] = None) -> float:
        g = self.group if group is None else group
        ba, bp = _f64(np.asarray(bloch).reshape(-1))
        return float(_lib.orc_expect(self._h, bp, g))

    def export(self):
        """(x [m, W], z [m, W], coef [m]) sorted by the (x words, z words) tuple."""
        m = len(self)
        x = np.zeros((m, self.W), dtype=np.uint64)
        z = np.zeros((m, self.W), dtype=np.uint64)
        c = np.zeros(m, dtype=np.float64)
        if m:
            _lib.orc_export(self._h, x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                            z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                            c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return x, z, c

    def as_dict(self):
        """{(x words..., z words...): coef}"""
        x, z, c = self.export()
        return {tuple(int(v) for v in x[i]) + tuple(int(v) for v in z[i]): float(c[i])
                for i in range(len(c))}


class BatchedOracleState:
    """B angle sets on one circuit: every string carries B coefficients; a
    term is kept iff some column has |c| >= eps."""

    def __init__(self, n, B, x, z, coef, group=0, eps=0.0, max_weight=-1):
        lib = _load()
        self.n, self.B, self.W = n, B, (n + 63) // 64
        xa, xp = _u64(np.asarray(x).reshape(-1, self.W))
        za, zp = _u64(np.asarray(z).reshape(-1, self.W))
        ca, cp = _f64(np.asarray(coef, dtype=np.float64).reshape(-1, B))
        self._h = lib.orcb_create(n, xa.shape[0], B, xp, zp, cp, group, eps, max_weight)
        self.group, self.eps, self.max_weight = group, eps, max_weight

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orcb_destroy(h)
            self._h = None

    def __len__(self):
        return int(_lib.orcb_size(self._h))

    @property
    def updates(self) -> float:
        return float(_lib.orcb_updates(self._h))

    def apply_layer(self, gx, gz, theta, noise_mode=0, p=0.0, group=None):
        """theta: [K, B] angles (time order of the K gates)."""
        g = self.group if group is None else group
        ga, gp = _u64(gx)
        ha, hp = _u64(gz)
        ta, tp = _f64(np.asarray(theta, dtype=np.float64).reshape(-1, self.B))
        _lib.orcb_apply_layer(self._h, ta.shape[0], gp, hp, tp, noise_mode, p, self.eps,
                              self.max_weight, g)

    def expect(self, bloch, group=None):
        g = self.group if group is None else group
        ba, bp = _f64(np.asarray(bloch).reshape(-1))
        out = np.zeros(self.B)
        _lib.orcb_expect(self._h, bp, g, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return out

    def export(self):
        m = len(self)
        x = np.zeros((m, self.W), dtype=np.uint64)
        z = np.zeros((m, self.W), dtype=np.uint64)
        c = np.zeros((m, self.B), dtype=np.float64)
        if m:
            _lib.orcb_export(self._h, x.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                             z.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                             c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        return x, z, c


def canonical(n: int, group: int, x, z):
    """Orbit representatives of keys (x, z [m, W]) under Z_n or S_n."""
    lib = _load()
    W = (n + 63) // 64
    xa, xp = _u64(np.asarray(x).reshape(-1, W))
    za, zp = _u64(np.asarray(z).reshape(-1, W))
    ox = np.zeros_like(xa)
    oz = np.zeros_like(za)
    lib.orc_canonical(n, xa.shape[0], group, xp, zp,
                      ox.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                      oz.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    return ox, oz


def sym_overlap(n: int, group: int, x, z, bloch):
    lib = _load()
    W = (n + 63) // 64
    xa, xp = _u64(np.asarray(x).reshape(-1, W))
    za, zp = _u64(np.asarray(z).reshape(-1, W))
    ba, bp = _f64(np.asarray(bloch).reshape(-1))
    out = np.zeros(xa.shape[0])
    lib.orc_sym_overlap(n, xa.shape[0], group, xp, zp, bp,
                        out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    return out


def run_workload(wl, group: Optional[int] = None, steps: Optional[int] = None,
                 record_each_step: bool = False):
    """Propagate a pp_inputs.Workload through the oracle.

    Layers are applied from the last to the first (Heisenberg order).  Returns
    (state, [<O> after each layer]) when record_each_step, else (state, <O>).
    """
    g = wl.symmetry if group is None else group
    ox, oz, oc = wl.observable.arrays()
    st = OracleState(wl.circuit.n, ox, oz, oc, group=g, eps=wl.eps, max_weight=wl.max_weight)
    L = len(wl.circuit.layers) if steps is None else steps
    vals = []
    for layer in reversed(range(L)):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        st.apply_layer(gx, gz, th, wl.noise_mode, wl.noise_p, group=g)
        if record_each_step:
            vals.append(st.expect(wl.state.bloch, g))
    if record_each_step:
        return st, vals
    return st, st.expect(wl.state.bloch, g)
