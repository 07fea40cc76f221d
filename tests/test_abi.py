"""The C-ABI library builds, loads and exports every entry point of include/pp.h.

No compute call is made here (no GPU); only host-side argument validation,
which returns before any CUDA call, is exercised.
"""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

import paper_2512_12094_gb300 as pp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    pp.build()
    return pp.load()


def _declared():
    txt = open(os.path.join(ROOT, "include", "pp.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pp_[a-z_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert len(declared) >= 18
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == sorted(pp.EXPORTED)


def test_exports_via_nm(lib):
    import subprocess
    out = subprocess.run(["nm", "-D", pp._LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pp_[a-z_]+)", out))
    assert set(_declared()) <= exported


def test_config_default(lib):
    cfg = pp.pp_config_default()
    assert cfg.batch == 1 and cfg.max_weight == -1 and cfg.use_graphs == 1
    assert cfg.check_symmetry == 1 and cfg.coeff_eps == 0.0


@pytest.mark.parametrize("fields", [dict(n_qubits=0), dict(n_qubits=257), dict(batch=0),
                                    dict(batch=513), dict(symmetry=5), dict(symmetry=4 | (3 << 8)),
                                    dict(symmetry=4), dict(symmetry=1 | (2 << 8)), dict(coef_type=2),
                                    dict(coeff_eps=-1.0), dict(noise_mode=7),
                                    dict(batch=4, noise_mode=2, noise_p=0.1),
                                    dict(coef_type=1, noise_mode=2, noise_p=0.1),
                                    dict(coeff_eps=float("nan")), dict(noise_mode=1, noise_p=-0.1),
                                    dict(noise_mode=2, noise_p=float("nan")), dict(merge_method=2),
                                    dict(wait_limit=-1), dict(room_factor=-1.0),
                                    dict(room_factor=float("nan")), dict(room_factor=float("inf")),
                                    dict(block_threads=512), dict(block_threads=-256)])
def test_create_rejects_bad_config_without_gpu(lib, fields):
    cfg = pp.pp_config_default(n_qubits=8)
    for field, value in fields.items():
        setattr(cfg, field, value)
    h = ctypes.c_void_p()
    st = lib.pp_create(ctypes.byref(cfg), 0, None, None, None, ctypes.byref(h))
    assert st == 1  # PP_ERR_ARG
    assert h.value is None
    assert lib.pp_last_error().decode() != ""


def test_group_codes_in_the_header_match_the_binding(lib):
    txt = open(os.path.join(ROOT, "include", "pp.h")).read()
    for name, value in (("PP_SYM_ZN", pp.SYM_ZN), ("PP_SYM_SN", pp.SYM_SN),
                        ("PP_SYM_DN", pp.SYM_DN), ("PP_SYM_TORUS", pp.SYM_TORUS)):
        assert re.search(r"\b%s = %d\b" % (name, value), txt), name
    assert pp.sym_torus(4) == 4 + 4 * 256
    # a torus width that does not divide n is rejected before any CUDA call
    assert lib.pp_canonical_keys(8, pp.sym_torus(3), 1, None, None, None) == 1


def test_status_codes_and_struct_sizes_match_the_header(lib):
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "pp.h")).read(), flags=re.S)
    body = re.search(r"typedef enum \{(.*?)\} pp_status;", txt, flags=re.S).group(1)
    declared = {int(v): k for k, v in re.findall(r"(PP_\w+)\s*=\s*(\d+)", body)}
    assert declared == pp.STATUS


def test_binding_structs_have_the_header_layout(tmp_path):
    """Every ctypes mirror has the size and field offsets that a C compiler
    gives the structs of include/pp.h."""
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [pp.pp_config, pp.pp_pauli, pp.pp_stats_t, pp.pp_job, pp.pp_job_result]
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "pp.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append('  printf("%s sizeof %%zu\\n", sizeof(%s));' % (name, name))
        for field in st._fields_:
            lines.append('  printf("%s %s %%zu\\n", offsetof(%s, %s));'
                         % (name, field[0], name, field[0]))
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    got = {}
    for ln in out.splitlines():
        name, field, value = ln.split()
        got[(name, field)] = int(value)
    for st in structs:
        name = st.__name__
        assert got[(name, "sizeof")] == ctypes.sizeof(st), name
        for field in st._fields_:
            assert got[(name, field[0])] == getattr(st, field[0]).offset, (name, field[0])


def test_stateless_calls_validate_arguments(lib):
    assert lib.pp_canonical_keys(0, 1, 1, None, None, None) == 1
    assert lib.pp_canonical_keys(8, 5, 1, None, None, None) == 1
    assert lib.pp_canonical_keys(8, 1, 0, None, None, None) == 0  # empty: nothing to do
    m = ctypes.c_int64(7)
    assert lib.pp_merge_terms(8, 0, 0, None, None, None, None, ctypes.byref(m), None) == 0
    assert m.value == 0
    assert lib.pp_overlap_sum(8, 0, 1, None, None, None, None, None) == 1


def test_null_context_is_an_argument_error(lib):
    assert lib.pp_destroy(None) == 0
    for name in ("pp_canonicalize", "pp_merge", "pp_synchronize"):
        assert getattr(lib, name)(None) == 1
    assert lib.pp_truncate(None, 0.0, -1) == 1


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without libpp.so every call raises: there is no CPU path to fall back on."""
    monkeypatch.setattr(pp, "_lib", None)
    monkeypatch.setattr(pp, "_LIB", str(tmp_path / "libpp.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        pp.load()
    with pytest.raises(RuntimeError):
        pp.pp_config_default(n_qubits=4)


def test_binding_argument_counts_match_the_prototypes():
    """Every prototype of include/pp.h and the binding's argtypes agree in arity."""
    txt = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "pp.h")).read(), flags=re.S)
    protos = re.findall(r"\n(?:pp_status|const char\*)\s+(pp_\w+)\s*\(([^;]*?)\)\s*;", txt,
                        flags=re.S)
    assert sorted(name for name, _ in protos) == pp.EXPORTED
    for name, args in protos:
        a = args.strip()
        arity = 0 if a in ("", "void") else len(a.split(","))
        assert arity == len(pp._SIGS[name]), name


def test_server_calls_validate_arguments(lib):
    h = ctypes.c_void_p()
    for slots, budget in ((0, 1 << 30), (257, 1 << 30), (4, 0)):
        assert lib.pp_server_create(slots, budget, 0, ctypes.byref(h)) == 1  # PP_ERR_ARG
        assert h.value is None
    assert lib.pp_server_create(4, 1 << 30, 0, None) == 1
    job, jid = pp.pp_job(), ctypes.c_uint64()
    assert lib.pp_submit(None, ctypes.byref(job), ctypes.byref(jid)) == 1
    assert lib.pp_last_error().decode() != ""


def test_calls_that_need_a_gpu_fail_loudly_without_one(lib):
    """Without a GPU a context or a server is not created: the call returns
    PP_ERR_CUDA with a message (no CPU fallback, no crash)."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert lib.pp_server_create(2, 1 << 30, 0, ctypes.byref(h)) == 5  # PP_ERR_CUDA
    assert h.value is None and lib.pp_last_error().decode() != ""
    cfg = pp.pp_config_default(n_qubits=8)
    x, z = (ctypes.c_uint64 * 1)(0), (ctypes.c_uint64 * 1)(1)
    c = (ctypes.c_double * 1)(1.0)
    assert lib.pp_create(ctypes.byref(cfg), 1, x, z, c, ctypes.byref(h)) == 5
    assert h.value is None and lib.pp_last_error().decode() != ""


def test_plain_c_program_builds_and_runs_against_the_library(lib, tmp_path):
    """tests/abi_example.c uses the library from C99 alone (create, apply
    three Z_n-merged layers, expect, destroy).  It compiles warning-free
    against include/pp.h and links against libpp.so; without a GPU it stops
    at pp_create with PP_ERR_CUDA and a message, with one it prints <O>."""
    import torch
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pkg = os.path.dirname(os.path.abspath(pp.__file__))
    exe = tmp_path / "abi_example"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "abi_example.c"), "-L", pkg, "-lpp",
                    "-Wl,-rpath," + pkg, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    if torch.cuda.is_available():
        assert r.returncode == 0, r.stderr
        assert r.stdout.startswith("<O> = ")
    else:
        assert r.returncode == 2, (r.returncode, r.stdout, r.stderr)
        assert r.stderr.startswith("pp_create failed: status 5: ") and len(r.stderr) > 30
