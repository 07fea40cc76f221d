"""Contexts driven from different host threads at the same time, each on a
share of the GPU (pp_set_grid_fraction): every result equals the context run
alone, bit for bit (needs a GB300)."""
import threading

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
    d = {tuple(int(v) for v in x[i]) + tuple(int(v) for v in z[i]): float(c[i])
         for i in range(len(c))}
    assert len(d) == len(c), "a string appears twice in the table"
    return d


def layers_of(wl):
    return [wl.circuit.gate_arrays(l) for l in reversed(range(len(wl.circuit.layers)))]


def run(wl, group, stream=None, fraction=None, gate=None):
    x, z, c = wl.observable.arrays()
    p = pp.Propagator(wl.circuit.n, x, z, c, symmetry=group, eps=wl.eps,
                      max_weight=wl.max_weight, stream=stream)
    if fraction is not None:
        pp.pp_set_grid_fraction(p.ctx, fraction)
    if gate is not None:
        gate.wait()  # start the layers of both threads together
    for gx, gz, th in layers_of(wl):
        p.apply_layer(gx, gz, th, True)
    out = (as_dict(*p.export()), float(p.expect(wl.state.bloch)))
    p.close()
    return out


@pytest.mark.parametrize("fractions", [(0.5, 0.5), (0.25, 0.75), (0.1, 0.3)])
def test_threads_with_grid_fractions_match_alone(fractions):
    import torch
    wl = pi.config1_ring(n=32, steps=8)
    alone = [run(wl, g) for g in (0, 1)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    gate = threading.Barrier(2)
    got = [None, None]
    errors = []

    def work(g):
        try:
            got[g] = run(wl, g, stream=streams[g].cuda_stream, fraction=fractions[g],
                         gate=gate)
        except Exception as e:  # noqa: BLE001 - reported below
            errors.append(e)

    threads = [threading.Thread(target=work, args=(g,)) for g in (0, 1)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for g in (0, 1):
        assert got[g][0] == alone[g][0]
        # the overlap sums in table order, which depends on the order births
        # were appended in
        assert got[g][1] == pytest.approx(alone[g][1], abs=1e-12)


def test_grid_fraction_is_checked():
    wl = pi.config1_ring(n=32, steps=1)
    x, z, c = wl.observable.arrays()
    p = pp.Propagator(32, x, z, c)
    for bad in (0.0, -0.5, 1.5, float("nan")):
        with pytest.raises(pp.PPError) as e:
            pp.pp_set_grid_fraction(p.ctx, bad)
        assert e.value.status == 1  # PP_ERR_ARG
    pp.pp_set_grid_fraction(p.ctx, 1.0)
    p.close()


def test_bench_step_matches_the_oracle_trajectory():
    """The step bench.py times, through its own code: the plain and Z_32
    propagations of the full ring workload (n=32, 20 steps, eps 1e-4, weight
    <= 10) at the same time from two host threads on a quarter and three
    quarters of the GPU, the merged run taking the whole GPU once the plain
    run is done, from device-resident and from host inputs.  <O> must equal
    the oracle's stored trajectory to 1e-10, and the live-term and update
    counts must equal the oracle's."""
    import json
    import os
    import torch
    import bench
    data = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "ring_n32.json")))
    wl = pi.config1_ring()
    layers = [(pp.pack_gates(gx, gz), th) for gx, gz, th in layers_of(wl)]
    ox, oz, oc = wl.observable.arrays()
    dev = torch.device("cuda", 0)
    obs_dev = (torch.from_numpy(ox.view(np.int64)).to(dev),
               torch.from_numpy(oz.view(np.int64)).to(dev), torch.from_numpy(oc).to(dev))
    streams = [torch.cuda.Stream() for _ in range(2)]
    join = torch.cuda.Stream()
    for host_inputs in (False, True):
        vals, stats, _, _, end = bench.run_job_concurrent(pp, wl, layers, obs_dev, streams, join,
                                                          host_inputs, 0.25)
        end.synchronize()
        for g, key in enumerate(("plain", "zn")):
            gold = data[key][-1]
            assert vals[g] == pytest.approx(gold["expect"], abs=1e-10)
            assert stats[g]["live_terms"] == gold["terms"]
            assert stats[g]["gate_updates"] == gold["updates"]
