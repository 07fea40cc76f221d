"""Merge cadence (the number of layers between symmetry merges) on the GPU.

The paper leaves the number of layers between merges free: a merge is exact
at any boundary where the layers so far are symmetric (Theorem 1).  For each
cadence -- after every k-th full Trotter layer, or after every RZZ / RX / RZ
(or XX / YY / ZZ) sublayer -- the GPU must give the oracle's table and <O>
when the oracle follows the same schedule.
"""
import numpy as np
import pytest

import oracle
import paper_2512_12094_gb300 as pp
import pp_inputs as pi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    pp.build()
    pp.load()
    oracle.build()


def as_dict(x, z, c):
    d = {tuple(int(v) for v in x[i]) + tuple(int(v) for v in z[i]): float(c[i])
        for i in range(len(c))}
    assert len(d) == len(c), "a string appears twice in the table"
    return d


def run_schedule(wl, group, every, merge_method=pp.MERGE_HASH):
    n = wl.circuit.n
    L = len(wl.circuit.layers)
    flags = pi.merge_schedule(L, every)
    ox, oz, oc = wl.observable.arrays()
    prop = pp.Propagator.from_workload(wl, symmetry=group, merge_method=merge_method)
    st = oracle.OracleState(n, ox, oz, oc, group=group, eps=wl.eps, max_weight=wl.max_weight)
    for a, layer in enumerate(reversed(range(L))):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        prop.apply_layer(gx, gz, th, boundary=flags[a])
        st.apply_layer(gx, gz, th, wl.noise_mode, wl.noise_p, group=group if flags[a] else 0)
    return prop, st


def check(prop, st, wl, group, atol=1e-12):
    g = as_dict(*prop.export())
    o = st.as_dict()
    for k in set(o) ^ set(g):
        v = o.get(k, g.get(k))
        assert wl.eps > 0 and abs(abs(v) - wl.eps) <= 1e-9 * wl.eps
    for k in set(o) & set(g):
        assert abs(g[k] - o[k]) <= atol
    assert prop.expect(wl.state.bloch) == pytest.approx(st.expect(wl.state.bloch, group), abs=1e-10)


@pytest.mark.parametrize("every,sub", [(1, False), (2, False), (4, False), (1, True), (3, True)])
@pytest.mark.parametrize("method", [pp.MERGE_HASH, pp.MERGE_SORT])
def test_ring_zn_cadence_matches_oracle(every, sub, method):
    wl = pi.config1_ring(n=16, steps=5, eps=1e-4, max_weight=8, symmetry=1)
    run = pi.split_sublayers(wl) if sub else wl
    prop, st = run_schedule(run, 1, every, method)
    check(prop, st, run, 1)


@pytest.mark.parametrize("every", [1, 3])
def test_xxz_sn_cadence_matches_oracle(every):
    wl = pi.xxz_all_to_all(12, 0.05, 3, eps=1e-3, symmetry=2, split=True)
    prop, st = run_schedule(wl, 2, every)
    check(prop, st, wl, 2, atol=1e-11)
