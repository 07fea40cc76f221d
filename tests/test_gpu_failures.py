"""Failure detection without a GPU fault.

* Every device wait is bounded.  A context whose bound is one microsecond
  makes the grid barrier of a multi-block layer run out: the kernel records the timeout
  and returns, the call reports PP_ERR_TIMEOUT, the context can be destroyed,
  and the next context on the same GPU computes the oracle's result.
* Device allocations can be made to fail on the host
  (pp_debug_fail_alloc_after).  A failure before any gate runs -- uploading a
  new layer's arguments, growing the tables -- returns PP_ERR_OOM and leaves
  the context as it was: the same layer applied again gives the oracle's table.
Nothing here traps, faults or hangs the GPU.
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


@pytest.fixture(autouse=True)
def _no_injection():
    yield
    pp.pp_debug_fail_alloc_after(-1)


def as_dict(x, z, c):
    d = {tuple(int(v) for v in x[i]) + tuple(int(v) for v in z[i]): float(c[i])
        for i in range(len(c))}
    assert len(d) == len(c), "a string appears twice in the table"
    return d


def oracle_after(wl, layers):
    ox, oz, oc = wl.observable.arrays()
    st = oracle.OracleState(wl.circuit.n, ox, oz, oc, eps=wl.eps, max_weight=wl.max_weight)
    for layer in layers:
        gx, gz, th = wl.circuit.gate_arrays(layer)
        st.apply_layer(gx, gz, th, group=0)
    return st.as_dict()


def test_grid_barrier_wait_runs_out_with_a_one_microsecond_bound():
    wl = pi.config1_ring(n=20, steps=6, eps=0.0, max_weight=6)
    ox, oz, oc = wl.observable.arrays()
    cfg = pp.pp_config_default(n_qubits=20, max_weight=6, wait_limit=1)
    ctx = pp.pp_create(cfg, ox, oz, oc)
    status = None
    for layer in reversed(range(6)):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        try:
            pp.pp_apply_layer(ctx, pp.pack_gates(gx, gz), th, False)
        except pp.PPError as e:
            status = e.status
            break
    assert status == 6, "no bounded wait ran out"  # PP_ERR_TIMEOUT
    assert "ran out" in pp.pp_last_error() or "wait" in pp.pp_last_error()
    pp.pp_destroy(ctx)
    # the GPU and the library are fine: a default context reproduces the oracle
    prop = pp.Propagator.from_workload(wl, symmetry=0)
    for layer in reversed(range(3)):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        prop.apply_layer(gx, gz, th, boundary=False)
    assert as_dict(*prop.export()) == oracle_after(wl, reversed(range(3)))


def test_rejects_a_negative_wait_limit():
    with pytest.raises(pp.PPError) as e:
        pp.pp_create(pp.pp_config_default(n_qubits=4, wait_limit=-1), [[0]], [[1]], [1.0])
    assert e.value.status == 1


def test_injected_oom_uploading_layer_arguments_leaves_context_usable():
    n = 6
    wl = pi.config1_ring(n=n, steps=2, eps=0.0, max_weight=-1)
    prop = pp.Propagator.from_workload(wl, symmetry=0)
    gx, gz, th = wl.circuit.gate_arrays(1)
    prop.apply_layer(gx, gz, th, boundary=False)
    before = as_dict(*prop.export())
    gx, gz, th = wl.circuit.gate_arrays(0)
    th = th + 0.25  # new angles: the layer's arguments are uploaded anew
    pp.pp_debug_fail_alloc_after(0)
    with pytest.raises(pp.PPError) as e:
        prop.apply_layer(gx, gz, th, boundary=False)
    assert e.value.status == 2  # PP_ERR_OOM
    assert as_dict(*prop.export()) == before
    prop.apply_layer(gx, gz, th, boundary=False)
    wl.circuit.layers[0] = [(s, t + 0.25) for s, t in wl.circuit.layers[0]]
    assert as_dict(*prop.export()) == oracle_after(wl, [1, 0])


def test_injected_oom_growing_the_tables_leaves_context_usable():
    n = 16
    wl = pi.config1_ring(n=n, steps=3, eps=0.0, max_weight=6)
    prop = pp.Propagator.from_workload(wl, symmetry=0)
    gx, gz, th = wl.circuit.gate_arrays(2)
    prop.apply_layer(gx, gz, th, boundary=False)
    cap0 = prop.stats()["capacity"]
    before = as_dict(*prop.export())
    gx, gz, th = wl.circuit.gate_arrays(1)
    pp.pp_debug_fail_alloc_after(0)  # the next table allocation fails
    with pytest.raises(pp.PPError) as e:
        prop.apply_layer(gx, gz, th, boundary=False)
    assert e.value.status == 2
    assert prop.stats()["capacity"] == cap0
    assert as_dict(*prop.export()) == before
    prop.apply_layer(gx, gz, th, boundary=False)  # grows this time
    assert prop.stats()["capacity"] > cap0
    assert as_dict(*prop.export()) == oracle_after(wl, [2, 1])
