"""Python binding of the GB300 Pauli propagation library (libpp.so).

Argument marshalling only: every step of the propagation runs in the CUDA
kernels behind the C ABI of ``include/pp.h``.  The functions below carry the
same names as the C entry points.  There is no CPU fallback: if the compiled
library is missing, :func:`load` raises.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_ROOT = os.path.dirname(_HERE)
_CSRC = os.path.join(_HERE, "csrc")
_LIB = os.path.join(_HERE, "libpp.so")
_SOURCES = ["pp_kernels.cu", "pp_api.cu", "pp_static.cu", "pp_batched.cu", "pp_server.cu",
            "pp_sort.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr"]

PP_OK = 0
STATUS = {0: "PP_OK", 1: "PP_ERR_ARG", 2: "PP_ERR_OOM", 3: "PP_ERR_CAPACITY",
          4: "PP_ERR_SYMMETRY", 5: "PP_ERR_CUDA", 6: "PP_ERR_TIMEOUT", 7: "PP_ERR_BUSY",
          8: "PP_ERR_REJECTED", 9: "PP_ERR_STATE", 10: "PP_ERR_INTERNAL"}
SYM_NONE, SYM_ZN, SYM_SN, SYM_DN, SYM_TORUS = 0, 1, 2, 3, 4
NOISE_NONE, NOISE_PER_GATE, NOISE_PER_LAYER = 0, 1, 2
MERGE_HASH, MERGE_SORT = 0, 1


def sym_torus(lx: int) -> int:
    """Group code of the translations of an lx x (n / lx) torus (PP_SYM_TORUS_LX)."""
    return SYM_TORUS | (int(lx) << 8)


_lib = None
_lock = threading.Lock()


class PPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile libpp.so in-tree for sm_103a (objects in parallel, then link)."""
    srcs = [os.path.join(_CSRC, s) for s in _SOURCES]
    deps = srcs + [os.path.join(_CSRC, h) for h in sorted(os.listdir(_CSRC))
                   if h.endswith((".h", ".cuh"))] + [os.path.join(_ROOT, "include", "pp.h")]
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= max(os.path.getmtime(d) for d in deps)):
        return _LIB
    bdir = os.path.join(_HERE, "_build")
    os.makedirs(bdir, exist_ok=True)
    nvcc = _nvcc()

    def compile_one(src):
        obj = os.path.join(bdir, os.path.basename(src) + ".o")
        cmd = [nvcc, *ARCH, *NVCC_FLAGS, "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            print(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(len(srcs)) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = _LIB + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", *objs, "-o", tmp]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, _LIB)
    return _LIB


class pp_config(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int), ("symmetry", ctypes.c_int), ("batch", ctypes.c_int),
                ("coef_type", ctypes.c_int), ("coeff_eps", ctypes.c_double),
                ("max_weight", ctypes.c_int), ("noise_mode", ctypes.c_int),
                ("noise_p", ctypes.c_double), ("mem_budget_bytes", ctypes.c_size_t),
                ("cuda_stream", ctypes.c_void_p), ("check_symmetry", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("profile_kernels", ctypes.c_int),
                ("layer_kernel", ctypes.c_int), ("merge_method", ctypes.c_int),
                ("block_threads", ctypes.c_int), ("wait_limit", ctypes.c_int),
                ("room_factor", ctypes.c_double)]


class pp_pauli(ctypes.Structure):
    _fields_ = [("x", ctypes.c_uint64 * 4), ("z", ctypes.c_uint64 * 4)]


class pp_job(ctypes.Structure):
    _fields_ = [("cfg", pp_config), ("n_terms", ctypes.c_int64), ("x", ctypes.c_void_p),
                ("z", ctypes.c_void_p), ("coef", ctypes.c_void_p), ("n_layer_gates", ctypes.c_int),
                ("gates", ctypes.c_void_p), ("theta", ctypes.c_void_p), ("n_layers", ctypes.c_int),
                ("symmetric_boundary", ctypes.c_int), ("bloch", ctypes.c_void_p),
                ("mem_bytes", ctypes.c_size_t)]


class pp_job_result(ctypes.Structure):
    _fields_ = [("done", ctypes.c_int), ("status", ctypes.c_int), ("value", ctypes.c_double),
                ("live_terms", ctypes.c_int64), ("gate_updates", ctypes.c_double),
                ("device_bytes", ctypes.c_size_t), ("reserved_bytes", ctypes.c_size_t),
                ("queue_ms", ctypes.c_double), ("run_ms", ctypes.c_double),
                ("latency_ms", ctypes.c_double), ("message", ctypes.c_char * 160),
                ("grows", ctypes.c_int), ("restarts", ctypes.c_int)]


class pp_stats_t(ctypes.Structure):
    _fields_ = [("live_terms", ctypes.c_int64), ("stored_terms", ctypes.c_int64),
                ("capacity", ctypes.c_int64), ("gate_updates", ctypes.c_double),
                ("gates_applied", ctypes.c_int64), ("merges", ctypes.c_int64),
                ("compactions", ctypes.c_int64), ("regrows", ctypes.c_int64),
                ("device_bytes", ctypes.c_size_t), ("anticommuting_terms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("gate_kernel_ms", ctypes.c_double),
                ("gate_kernels_timed", ctypes.c_int64), ("grid_scale", ctypes.c_double),
                ("skipped_updates", ctypes.c_double), ("gates_skipped", ctypes.c_int64),
                ("index_factor", ctypes.c_double), ("persistent", ctypes.c_int64),
                ("block_threads", ctypes.c_int64), ("stalls", ctypes.c_int64),
                ("index_slots", ctypes.c_int64)]


_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p

# name -> argtypes (all return pp_status unless listed in _RESTYPE)
_SIGS = {
    "pp_config_default": [ctypes.POINTER(pp_config)],
    "pp_create": [ctypes.POINTER(pp_config), ctypes.c_int64, _vp, _vp, _vp, ctypes.POINTER(_vp)],
    "pp_create_device": [ctypes.POINTER(pp_config), ctypes.c_int64, _vp, _vp, _vp,
                         ctypes.POINTER(_vp)],
    "pp_destroy": [_vp],
    "pp_apply_layer": [_vp, ctypes.c_int, _vp, _vp, ctypes.c_int],
    "pp_canonicalize": [_vp],
    "pp_merge": [_vp],
    "pp_truncate": [_vp, ctypes.c_double, ctypes.c_int],
    "pp_expect": [_vp, _vp, _f64p],
    "pp_expect_basis": [_vp, _vp, _f64p],
    "pp_import": [_vp, ctypes.c_int64, _vp, _vp, _vp],
    "pp_tune": [_vp, ctypes.c_int, _vp, _vp, _f64p],
    "pp_num_terms": [_vp, _i64p, _i64p],
    "pp_export": [_vp, ctypes.c_int64, _vp, _vp, _vp, _i64p],
    "pp_stats": [_vp, ctypes.POINTER(pp_stats_t)],
    "pp_set_budget": [_vp, ctypes.c_size_t],
    "pp_set_grid_fraction": [_vp, ctypes.c_double],
    "pp_synchronize": [_vp],
    "pp_last_error": [],
    "pp_debug_fail_alloc_after": [ctypes.c_int64],
    "pp_canonical_keys": [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _vp, _vp, _vp],
    "pp_merge_terms": [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _vp, _vp, _vp, _vp, _i64p, _vp],
    "pp_merge_terms_sorted": [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _vp, _vp, _vp, _vp, _i64p,
                              _vp],
    "pp_overlap_sum": [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp],
    "pp_merge_terms_noalloc": [ctypes.c_int, ctypes.c_int, ctypes.c_int64, _vp, _vp, _vp, _vp, _vp,
                               _vp],
    "pp_server_create": [ctypes.c_int, ctypes.c_size_t, ctypes.c_size_t, ctypes.POINTER(_vp)],
    "pp_submit": [_vp, ctypes.POINTER(pp_job), ctypes.POINTER(ctypes.c_uint64)],
    "pp_server_poll": [_vp, ctypes.c_uint64, ctypes.POINTER(pp_job_result)],
    "pp_server_wait": [_vp, ctypes.c_uint64, ctypes.POINTER(pp_job_result)],
    "pp_server_stats": [_vp, _i64p, _i64p, _i64p, ctypes.POINTER(ctypes.c_size_t)],
    "pp_server_destroy": [_vp],
}
_RESTYPE = {"pp_last_error": ctypes.c_char_p}

EXPORTED = sorted(_SIGS)


def load():
    """Load libpp.so (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB):
            raise RuntimeError(
                "libpp.so is not built: run paper_2512_12094_gb300.build() "
                "(the CUDA library is required; there is no CPU fallback)")
        lib = ctypes.CDLL(_LIB)
        for name, args in _SIGS.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = _RESTYPE.get(name, ctypes.c_int)
        _lib = lib
        return lib


def _check(st: int):
    if st != PP_OK:
        msg = load().pp_last_error().decode()
        raise PPError(st, msg)


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (host or device)."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    if isinstance(a, int):
        return a
    return a.ctypes.data


# ------------------------------------------------------------ C entry points

def pp_config_default(**kw) -> pp_config:
    cfg = pp_config()
    _check(load().pp_config_default(ctypes.byref(cfg)))
    for k, v in kw.items():
        if k == "cuda_stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream  # torch.cuda.Stream
        setattr(cfg, k, v)
    return cfg


def pp_create(cfg: pp_config, x, z, coef):
    """x, z: uint64 [m, W] host arrays; coef: float64 [m] or [m, batch]."""
    W = (cfg.n_qubits + 63) // 64
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint64).reshape(-1, W))
    z = np.ascontiguousarray(np.asarray(z, dtype=np.uint64).reshape(-1, W))
    c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).reshape(-1, cfg.batch))
    h = _vp()
    _check(load().pp_create(ctypes.byref(cfg), c.shape[0], _ptr(x), _ptr(z), _ptr(c),
                            ctypes.byref(h)))
    return h


def pp_create_device(cfg: pp_config, n_terms: int, x_dev, z_dev, coef_dev):
    """x_dev, z_dev, coef_dev: device tensors/pointers with the pp_create layout."""
    h = _vp()
    _check(load().pp_create_device(ctypes.byref(cfg), int(n_terms), _ptr(x_dev), _ptr(z_dev),
                                   _ptr(coef_dev), ctypes.byref(h)))
    return h


def pp_destroy(ctx):
    _check(load().pp_destroy(ctx))


def pack_gates(gx, gz) -> np.ndarray:
    """[K, W] x / z masks -> array of pp_pauli structs ([K, 8] uint64)."""
    gx = np.asarray(gx, dtype=np.uint64)
    gz = np.asarray(gz, dtype=np.uint64)
    K, W = gx.shape
    out = np.zeros((K, 8), dtype=np.uint64)
    out[:, :W] = gx
    out[:, 4:4 + W] = gz
    return out


def pp_apply_layer(ctx, gates_packed: np.ndarray, theta, symmetric_boundary: bool):
    """gates_packed from pack_gates (time order); theta float64 [K] or [K, batch]."""
    g = np.ascontiguousarray(gates_packed)
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    _check(load().pp_apply_layer(ctx, g.shape[0], _ptr(g), _ptr(th), int(bool(symmetric_boundary))))


def pp_canonicalize(ctx):
    _check(load().pp_canonicalize(ctx))


def pp_merge(ctx):
    _check(load().pp_merge(ctx))


def pp_truncate(ctx, eps: float, max_weight: int):
    _check(load().pp_truncate(ctx, float(eps), int(max_weight)))


def pp_expect(ctx, bloch, batch: int = 1):
    """Tr[rho O]: a float, or float64 [batch] for a batched context."""
    b = np.ascontiguousarray(np.asarray(bloch, dtype=np.float64).reshape(-1))
    out = np.zeros(batch, dtype=np.float64)
    _check(load().pp_expect(ctx, _ptr(b), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return float(out[0]) if batch == 1 else out


def pp_expect_basis(ctx, bits, batch: int = 1):
    """Tr[rho O] for the computational basis state with bits[q] in {0, 1}."""
    b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8).reshape(-1))
    out = np.zeros(batch, dtype=np.float64)
    _check(load().pp_expect_basis(ctx, _ptr(b), out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return float(out[0]) if batch == 1 else out


def pp_import(ctx, n_qubits: int, x, z, coef, batch: int = 1):
    """Replace the context's operator by the given terms (pp_create's layout)."""
    W = (n_qubits + 63) // 64
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint64).reshape(-1, W))
    z = np.ascontiguousarray(np.asarray(z, dtype=np.uint64).reshape(-1, W))
    c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).reshape(-1, batch))
    _check(load().pp_import(ctx, c.shape[0], _ptr(x), _ptr(z), _ptr(c)))


def pp_tune(ctx, packed_gates, theta) -> float:
    """Time the layer at each candidate launch size on a copy of the table and
    keep the fastest; returns the chosen scale."""
    g = np.ascontiguousarray(packed_gates)
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    out = ctypes.c_double(0.0)
    _check(load().pp_tune(ctx, g.shape[0], _ptr(g), _ptr(th), ctypes.byref(out)))
    return out.value


def pp_num_terms(ctx):
    live, stored = ctypes.c_int64(), ctypes.c_int64()
    _check(load().pp_num_terms(ctx, ctypes.byref(live), ctypes.byref(stored)))
    return live.value, stored.value


def pp_export(ctx, n_qubits: int, batch: int = 1):
    """(x [m, W], z [m, W], coef [m] or [m, batch]) of the live terms."""
    W = (n_qubits + 63) // 64
    m = ctypes.c_int64()
    st = load().pp_export(ctx, 0, None, None, None, ctypes.byref(m))
    if st not in (PP_OK, 1):
        _check(st)
    cap = m.value
    x = np.zeros((cap, W), dtype=np.uint64)
    z = np.zeros((cap, W), dtype=np.uint64)
    c = np.zeros((cap, batch) if batch > 1 else cap, dtype=np.float64)
    _check(load().pp_export(ctx, cap, _ptr(x), _ptr(z), _ptr(c), ctypes.byref(m)))
    return x[:m.value], z[:m.value], c[:m.value]


def pp_stats(ctx) -> dict:
    s = pp_stats_t()
    _check(load().pp_stats(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in pp_stats_t._fields_}


def pp_set_budget(ctx, nbytes: int):
    _check(load().pp_set_budget(ctx, int(nbytes)))


def pp_set_grid_fraction(ctx, fraction: float):
    _check(load().pp_set_grid_fraction(ctx, float(fraction)))


def pp_synchronize(ctx):
    _check(load().pp_synchronize(ctx))


def pp_last_error() -> str:
    return load().pp_last_error().decode()


def pp_debug_fail_alloc_after(n: int):
    """Make the allocation after the next n fail as out of memory (n < 0: off)."""
    _check(load().pp_debug_fail_alloc_after(int(n)))


def pp_canonical_keys(n_qubits: int, symmetry: int, m: int, keys_in, keys_out, stream=None):
    _check(load().pp_canonical_keys(n_qubits, symmetry, int(m), _ptr(keys_in), _ptr(keys_out),
                                    _stream(stream)))


def pp_merge_terms(n_qubits: int, symmetry: int, m: int, keys_in, coef_in, keys_out, coef_out,
                   stream=None) -> int:
    mo = ctypes.c_int64()
    _check(load().pp_merge_terms(n_qubits, symmetry, int(m), _ptr(keys_in), _ptr(coef_in),
                                 _ptr(keys_out), _ptr(coef_out), ctypes.byref(mo),
                                 _stream(stream)))
    return mo.value


def pp_merge_terms_sorted(n_qubits: int, symmetry: int, m: int, keys_in, coef_in, keys_out,
                          coef_out, stream=None) -> int:
    mo = ctypes.c_int64()
    _check(load().pp_merge_terms_sorted(n_qubits, symmetry, int(m), _ptr(keys_in), _ptr(coef_in),
                                        _ptr(keys_out), _ptr(coef_out), ctypes.byref(mo),
                                        _stream(stream)))
    return mo.value


def pp_overlap_sum(n_qubits: int, symmetry: int, m: int, keys, coef, bloch, out, stream=None):
    _check(load().pp_overlap_sum(n_qubits, symmetry, int(m), _ptr(keys), _ptr(coef), _ptr(bloch),
                                 _ptr(out), _stream(stream)))


def pp_merge_terms_noalloc(n_qubits: int, symmetry: int, m: int, keys_in, coef_in, keys_out,
                           coef_out, m_out_dev, stream=None):
    """Queue the allocation-free merge; the count lands in m_out_dev (device int64)."""
    _check(load().pp_merge_terms_noalloc(n_qubits, symmetry, int(m), _ptr(keys_in), _ptr(coef_in),
                                         _ptr(keys_out), _ptr(coef_out), _ptr(m_out_dev),
                                         _stream(stream)))


def pp_server_create(slots: int, mem_budget_bytes: int, default_job_bytes: int = 0):
    h = _vp()
    _check(load().pp_server_create(int(slots), int(mem_budget_bytes), int(default_job_bytes),
                                   ctypes.byref(h)))
    return h


def pp_server_destroy(server):
    _check(load().pp_server_destroy(server))


def make_job(cfg: pp_config, x, z, coef, gates_packed, theta, n_layers: int, bloch,
             symmetric_boundary: bool = True, mem_bytes: int = 0):
    """Build a pp_job; the returned tuple keeps the numpy buffers alive."""
    W = (cfg.n_qubits + 63) // 64
    x = np.ascontiguousarray(np.asarray(x, dtype=np.uint64).reshape(-1, W))
    z = np.ascontiguousarray(np.asarray(z, dtype=np.uint64).reshape(-1, W))
    c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64).reshape(-1, cfg.batch))
    g = np.ascontiguousarray(gates_packed)
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(bloch, dtype=np.float64).reshape(-1))
    job = pp_job(cfg=cfg, n_terms=c.shape[0], x=_ptr(x), z=_ptr(z), coef=_ptr(c),
                 n_layer_gates=g.shape[0], gates=_ptr(g), theta=_ptr(th), n_layers=int(n_layers),
                 symmetric_boundary=int(bool(symmetric_boundary)), bloch=_ptr(b),
                 mem_bytes=int(mem_bytes))
    return job, (x, z, c, g, th, b)


def pp_submit(server, job: "pp_job") -> int:
    jid = ctypes.c_uint64()
    _check(load().pp_submit(server, ctypes.byref(job), ctypes.byref(jid)))
    return jid.value


def _result(r: "pp_job_result") -> dict:
    out = {k: getattr(r, k) for k, _ in pp_job_result._fields_}
    out["message"] = r.message.decode(errors="replace")
    return out


def pp_server_poll(server, job_id: int) -> dict:
    r = pp_job_result()
    _check(load().pp_server_poll(server, int(job_id), ctypes.byref(r)))
    return _result(r)


def pp_server_wait(server, job_id: int) -> dict:
    r = pp_job_result()
    _check(load().pp_server_wait(server, int(job_id), ctypes.byref(r)))
    return _result(r)


def pp_server_stats(server) -> dict:
    q, r, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    b = ctypes.c_size_t()
    _check(load().pp_server_stats(server, ctypes.byref(q), ctypes.byref(r), ctypes.byref(c),
                                  ctypes.byref(b)))
    return {"queued": q.value, "running": r.value, "completed": c.value, "reserved_bytes": b.value}


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


# ------------------------------------------------------------- convenience

class Propagator:
    """Owns one pp_ctx; runs a pp_inputs.Workload through the C ABI."""

    def __init__(self, n_qubits, x, z, coef, symmetry=SYM_NONE, eps=0.0, max_weight=-1,
                 noise_mode=NOISE_NONE, noise_p=0.0, budget=0, stream=None, use_graphs=True,
                 check_symmetry=True, profile=False, layer_kernel=True, batch=1, f32=False,
                 merge_method=MERGE_HASH, block_threads=0, wait_limit=0, room_factor=0.0):
        self.n = n_qubits
        self.cfg = pp_config_default(n_qubits=n_qubits, symmetry=symmetry, coeff_eps=eps,
                                     max_weight=max_weight, noise_mode=noise_mode,
                                     noise_p=noise_p, mem_budget_bytes=budget,
                                     cuda_stream=stream, use_graphs=int(use_graphs),
                                     check_symmetry=int(check_symmetry),
                                     profile_kernels=int(profile),
                                     layer_kernel=int(layer_kernel), batch=int(batch),
                                     coef_type=1 if f32 else 0, merge_method=int(merge_method),
                                     block_threads=int(block_threads), wait_limit=int(wait_limit),
                                     room_factor=float(room_factor))
        self.batch = int(batch)
        self.ctx = pp_create(self.cfg, x, z, coef)
        self._packed = {}

    @classmethod
    def from_workload(cls, wl, symmetry=None, **kw):
        ox, oz, oc = wl.observable.arrays()
        sym = wl.symmetry if symmetry is None else symmetry
        return cls(wl.circuit.n, ox, oz, oc, symmetry=sym, eps=wl.eps, max_weight=wl.max_weight,
                   noise_mode=wl.noise_mode, noise_p=wl.noise_p, **kw)

    def close(self):
        if self.ctx is not None:
            pp_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def apply_layer(self, gx, gz, theta, boundary=True, key=None):
        if key is not None and key in self._packed:
            g = self._packed[key]
        else:
            g = pack_gates(gx, gz)
            if key is not None:
                self._packed[key] = g
        pp_apply_layer(self.ctx, g, theta, boundary)

    def run(self, wl, steps=None, record_each_step=False):
        L = len(wl.circuit.layers) if steps is None else steps
        vals = []
        for layer in reversed(range(L)):
            gx, gz, th = wl.circuit.gate_arrays(layer)
            self.apply_layer(gx, gz, th, boundary=True, key=layer)
            if record_each_step:
                vals.append(self.expect(wl.state.bloch))
        if record_each_step:
            return vals
        return self.expect(wl.state.bloch)

    def expect(self, bloch):
        return pp_expect(self.ctx, bloch, self.batch)

    def num_terms(self):
        return pp_num_terms(self.ctx)

    def export(self):
        return pp_export(self.ctx, self.n, self.batch)

    def stats(self):
        return pp_stats(self.ctx)
