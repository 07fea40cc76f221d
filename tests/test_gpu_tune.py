"""pp_tune: the launch size is chosen by timing, results do not depend on it.

A tuned context (the layer timed at 0.5, 1, 2 and 4 times the default
number of blocks on a copy of its table) continues exactly like an untuned
one: same table bit for bit without symmetry, same statistics (the trials
are not counted), and the chosen scale is one of the candidates."""
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


def layers(wl):
    for layer in reversed(range(len(wl.circuit.layers))):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        yield pp.pack_gates(gx, gz), th


@pytest.mark.parametrize("group,layer_kernel", [(0, True), (1, True), (0, False)])
def test_tuned_context_continues_like_untuned(group, layer_kernel):
    wl = pi.config1_ring(n=24, steps=6, eps=1e-5, max_weight=8)
    tuned = pp.Propagator.from_workload(wl, symmetry=group, layer_kernel=layer_kernel)
    plain = pp.Propagator.from_workload(wl, symmetry=group, layer_kernel=layer_kernel)
    for k, (g, th) in enumerate(layers(wl)):
        if k == 2:  # a table of some size to time
            scale = pp.pp_tune(tuned.ctx, g, th)
            assert scale in (0.5, 1.0, 2.0, 4.0)
            st = tuned.stats()
            assert st["grid_scale"] == scale
            assert st["index_factor"] in (1.5, 3.0) and st["persistent"] in (0, 1)
            a, b = tuned.stats(), plain.stats()
            for key in ("gate_updates", "anticommuting_terms", "gates_applied", "live_terms"):
                assert a[key] == b[key], key
            assert as_dict(*tuned.export()) == as_dict(*plain.export())
        pp.pp_apply_layer(tuned.ctx, g, th, True)
        pp.pp_apply_layer(plain.ctx, g, th, True)
    a, b = as_dict(*tuned.export()), as_dict(*plain.export())
    assert set(a) == set(b)
    if group == 0:
        assert all(a[k] == b[k] for k in b)
    else:
        assert max(abs(a[k] - b[k]) for k in b) <= 1e-12
    sa, sb = tuned.stats(), plain.stats()
    for key in ("gate_updates", "anticommuting_terms", "gates_applied"):
        assert sa[key] == sb[key], key
    tuned.close()
    plain.close()


def test_tune_batched_rows_and_empty_table():
    n, B = 16, 64
    angles = pi.batched_ring_angles(B, 1)
    gx, gz, _ = pi.Circuit(n, [pi.ring_layer(n, 0.0, 0.0, 0.0)]).gate_arrays(0)
    th = np.zeros((3 * n, B))
    th[:n], th[n:2 * n], th[2 * n:] = angles[:, 0], angles[:, 1], angles[:, 2]
    x, z, c = pi.mean_z(n).arrays()
    coef = np.repeat(c[:, None], B, axis=1)
    g = pp.pack_gates(gx, gz)
    tuned = pp.Propagator(n, x, z, coef, eps=1e-5, batch=B)
    plain = pp.Propagator(n, x, z, coef, eps=1e-5, batch=B)
    for k in range(3):
        if k == 1:
            assert pp.pp_tune(tuned.ctx, g, th) in (0.5, 1.0, 2.0, 4.0)
        pp.pp_apply_layer(tuned.ctx, g, th, True)
        pp.pp_apply_layer(plain.ctx, g, th, True)
    a, b = as_dict(*tuned.export()), as_dict(*plain.export())
    assert set(a) == set(b)
    for k in b:
        np.testing.assert_array_equal(a[k], b[k])
    tuned.close()
    plain.close()
    empty = pp.Propagator(n, np.zeros((0, 1), np.uint64), np.zeros((0, 1), np.uint64), np.zeros(0))
    assert pp.pp_tune(empty.ctx, g, th[:, 0].copy()) == 1.0
    empty.close()
