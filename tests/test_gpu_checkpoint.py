"""Checkpoint and resume through pp_export / pp_import, and pp_expect_basis.

A propagation stopped after some layers, exported, imported into a fresh
context and continued gives the table of the uninterrupted run: bit for bit
without symmetry (same gate arithmetic on the same terms), to 1e-12 with a
group (merges sum with FP64 atomics).
"""
import numpy as np
import pytest

import paper_2512_12094_gb300 as pp
import pp_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pp.build()
    pp.load()


def as_dict(x, z, c):
    if len(c) == 0:
        return {}
    x = np.asarray(x).reshape(len(c), -1)
    z = np.asarray(z).reshape(len(c), -1)
    d = {tuple(int(v) for v in x[i]) + tuple(int(v) for v in z[i]): c[i] for i in range(len(c))}
    assert len(d) == len(c), "a string appears twice in the table"
    return d


def layers_of(wl, start, stop):
    for layer in reversed(range(len(wl.circuit.layers))):
        k = len(wl.circuit.layers) - 1 - layer
        if start <= k < stop:
            yield wl.circuit.gate_arrays(layer)


@pytest.mark.parametrize("group", [0, 1])
def test_export_import_resume_equals_uninterrupted_run(group):
    n = 24
    wl = pi.config1_ring(n=n, steps=6, eps=1e-5, max_weight=8)
    full = pp.Propagator.from_workload(wl, symmetry=group)
    for gx, gz, th in layers_of(wl, 0, 6):
        full.apply_layer(gx, gz, th, True)
    first = pp.Propagator.from_workload(wl, symmetry=group)
    for gx, gz, th in layers_of(wl, 0, 3):
        first.apply_layer(gx, gz, th, True)
    x, z, c = first.export()
    first.close()
    # resume in a context created from some other observable
    other = pi.z_site(n, 5)
    ox, oz, oc = other.arrays()
    second = pp.Propagator(n, ox, oz, oc, symmetry=group, eps=wl.eps, max_weight=wl.max_weight)
    pp.pp_import(second.ctx, n, x, z, c)
    assert as_dict(*second.export()) == as_dict(x, z, c)
    for gx, gz, th in layers_of(wl, 3, 6):
        second.apply_layer(gx, gz, th, True)
    a, b = as_dict(*second.export()), as_dict(*full.export())
    assert set(a) == set(b)
    if group == 0:
        assert all(a[k] == b[k] for k in b)
    else:
        assert max(abs(a[k] - b[k]) for k in b) <= 1e-12
    st = pi.neel_state(n)  # not invariant under translations: the orbit average is used
    assert second.expect(st.bloch) == pytest.approx(full.expect(st.bloch), abs=1e-10)
    second.close()
    full.close()


def test_import_merges_duplicates_and_orbits_and_empties():
    n = 8
    strings = ["XIIIIIII", "IXIIIIII", "XIIIIIII", "ZZIIIIII"]
    x, z = pi.to_masks(strings, n)
    c = np.array([0.5, 0.25, 0.5, -1.0])
    p = pp.Propagator(n, *pi.mean_z(n).arrays()[:2], pi.mean_z(n).arrays()[2], symmetry=pp.SYM_ZN)
    pp.pp_import(p.ctx, n, x, z, c)
    got = as_dict(*p.export())
    xr, zr = pi.to_masks(["XIIIIIII", "ZZIIIIII"], n)
    want = as_dict(xr, zr, np.array([1.25, -1.0]))  # X on any site folds onto X_0
    assert got == want
    pp.pp_import(p.ctx, n, np.zeros((0, 1), np.uint64), np.zeros((0, 1), np.uint64), np.zeros(0))
    assert p.num_terms()[0] == 0
    assert p.expect(pi.zero_state(n).bloch) == 0.0
    p.close()


def test_import_batched_rows():
    n, B = 10, 3
    x, z, c = pi.random_observable(n, 20, 4).arrays()
    coef = np.stack([c, 2 * c, -c], axis=1)
    p = pp.Propagator(n, x, z, np.zeros_like(coef), batch=B)
    pp.pp_import(p.ctx, n, x, z, coef, batch=B)
    got = as_dict(*p.export())
    want = {}
    for i, k in enumerate(as_dict(x, z, np.arange(len(c)))):
        want[k] = want.get(k, 0) + coef[i]
    assert set(got) == set(want)
    for k in want:
        np.testing.assert_allclose(got[k], want[k], atol=1e-15, rtol=0)
    p.close()


def test_expect_basis_equals_bloch_form():
    n = 12
    wl = pi.config1_ring(n=n, steps=3, eps=1e-5, max_weight=8)
    for group in (0, 1):
        p = pp.Propagator.from_workload(wl, symmetry=group)
        p.run(wl)
        bits = np.array([(q * 5 + 1) % 3 == 0 for q in range(n)], dtype=np.uint8)
        bloch = np.zeros((n, 3))
        bloch[:, 2] = 1.0 - 2.0 * bits
        assert pp.pp_expect_basis(p.ctx, bits) == p.expect(bloch.reshape(-1))
        p.close()
