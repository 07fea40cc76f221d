"""The workloads beyond the ring benchmark, at their full sizes where the
oracle can follow, through the C ABI (needs a GB300).

* All-to-all Heisenberg, n=64, S_64, per-gate damping p=0.01, eps 1e-5, Neel
  state, 10 steps: GPU and oracle element by element after every step, merged
  and plain.  With per-gate damping a weight-1 string loses 0.99^189 per step,
  so the table empties within a few steps.  The per-layer damping variant
  (exp(-0.01 |Q|) once per step, the paper's noise model) is compared over its
  first step.  The merged operator is permutation symmetric and odd under a
  global spin flip and the state is Neel, so its <O> is 0 to rounding (the
  unmerged run truncates a non-symmetric operator and is not).
* Batched ring, n=64, B=256 angle sets in [0, pi/2], eps 1e-5 any-column: the
  table grows about tenfold per step (the any-column rule keeps the union of
  256 columns' strings), so the full 30 steps exceed any memory budget on one
  GPU.  The first two steps are compared with the batched oracle (FP64 rows
  bit for bit, FP32 rows within 1e-5 relative); a budget run checks that the
  growth stops with PP_ERR_CAPACITY and the context is restored.
* All-to-all XXZ (Delta = -1.8, |+>^n, S^2 / S_0^2), merged under S_n after
  every XX / YY / ZZ sublayer or after every full step, against the oracle at
  n = 8, 10 and at n = 36 over the first 16 sublayers.
* PP_ERR_CAPACITY leaves a context at its state before the call.
"""
import math

import numpy as np
import pytest

import oracle
import paper_2512_12094_gb300 as pp
import pp_inputs as pi

pytestmark = pytest.mark.gpu

GB = 1 << 30


@pytest.fixture(scope="module", autouse=True)
def _built():
    pp.build()
    pp.load()
    oracle.build()


def as_dict(x, z, c):
    if len(c) == 0:
        return {}
    x = np.asarray(x).reshape(len(c), -1)
    z = np.asarray(z).reshape(len(c), -1)
    d = {tuple(int(v) for v in x[i]) + tuple(int(v) for v in z[i]): c[i] for i in range(len(c))}
    assert len(d) == len(c), "a string appears twice in the table"
    return d


def assert_close(prop, st, eps, atol=1e-10):
    """Term sets equal up to terms whose oracle |c| is within 1e-9 relative of
    eps (merges sum in a different order); coefficients within atol, the FP64
    bar (merged coefficients are orbit sums and can be far above 1)."""
    g = as_dict(*prop.export())
    o = st.as_dict()
    for k in set(o) - set(g):
        assert eps > 0 and abs(abs(o[k]) - eps) <= 1e-9 * eps, ("missing", o[k])
    for k in set(g) - set(o):
        assert eps > 0 and abs(abs(g[k]) - eps) <= 1e-9 * eps, ("extra", g[k])
    for k in set(g) & set(o):
        assert abs(g[k] - o[k]) <= atol, (g[k], o[k])


def run_both(wl, group, layers=None):
    n = wl.circuit.n
    ox, oz, oc = wl.observable.arrays()
    prop = pp.Propagator.from_workload(wl, symmetry=group)
    st = oracle.OracleState(n, ox, oz, oc, group=group, eps=wl.eps, max_weight=wl.max_weight)
    L = len(wl.circuit.layers) if layers is None else layers
    for layer in reversed(range(L)):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        prop.apply_layer(gx, gz, th, boundary=True)
        st.apply_layer(gx, gz, th, wl.noise_mode, wl.noise_p, group=group)
        yield prop, st


# ------------------------------------------------ all-to-all Heisenberg, n=64

@pytest.mark.parametrize("group", [2, 0])
def test_a2a_n64_per_gate_noise_full_matches_oracle(group):
    wl = pi.config2_all_to_all()
    assert wl.circuit.n == 64 and len(wl.circuit.layers) == 10 and len(wl.circuit.layers[0]) == 6048
    bloch = wl.state.bloch
    for prop, st in run_both(wl, group):
        assert_close(prop, st, wl.eps)
        got, want = float(prop.expect(bloch)), st.expect(bloch, group)
        assert got == pytest.approx(want, abs=1e-10)
        if group == 2:
            # the merged operator is permutation symmetric and odd under a
            # global flip; its symmetrised overlap with Neel vanishes
            assert abs(got) <= 1e-12
            assert prop.num_terms()[0] <= math.comb(64 + 3, 3)
    prop.close()


def test_a2a_n64_per_layer_noise_first_step_matches_oracle():
    wl = pi.config2_all_to_all()
    wl.noise_mode = 2
    wl.noise_p = 0.01
    for prop, st in run_both(wl, 2, layers=1):
        assert_close(prop, st, wl.eps)
        assert float(prop.expect(wl.state.bloch)) == pytest.approx(
            st.expect(wl.state.bloch, 2), abs=1e-10)
    prop.close()


# ------------------------------------------- batched ring, n=64, B=256

def ring_batch(n, B, seed=0):
    angles = pi.batched_ring_angles(B, seed)
    layer = pi.ring_layer(n, 0.0, 0.0, 0.0)
    gx, gz, _ = pi.Circuit(n, [layer]).gate_arrays(0)
    th = np.zeros((3 * n, B))
    th[:n] = angles[:, 0]
    th[n:2 * n] = angles[:, 1]
    th[2 * n:] = angles[:, 2]
    x, z, c = pi.mean_z(n).arrays()
    return gx, gz, th, x, z, np.repeat(c[:, None], B, axis=1)


def test_batched_n64_b256_prefix_matches_batched_oracle():
    n, B, eps, steps = 64, 256, 1e-5, 2
    gx, gz, th, x, z, coef = ring_batch(n, B)
    st = oracle.BatchedOracleState(n, B, x, z, coef, group=0, eps=eps, max_weight=-1)
    p64 = pp.Propagator(n, x, z, coef, eps=eps, batch=B)
    p32 = pp.Propagator(n, x, z, coef, eps=eps, batch=B, f32=True)
    for _ in range(steps):
        st.apply_layer(gx, gz, th, group=0)
        p64.apply_layer(gx, gz, th, True)
        p32.apply_layer(gx, gz, th, True)
    o = as_dict(*st.export())
    g64 = as_dict(*p64.export())
    assert set(g64) == set(o) and len(o) > 1000
    for k in o:
        np.testing.assert_array_equal(g64[k], o[k])
    g32 = as_dict(*p32.export())
    assert set(g32) == set(o)
    worst = max(float(np.max(np.abs(g32[k] - o[k]) / np.maximum(np.abs(o[k]), 1e-3))) for k in o)
    assert worst < 1e-5
    bloch = pi.zero_state(n).bloch
    want = st.expect(bloch)
    np.testing.assert_allclose(p64.expect(bloch), want, atol=1e-12, rtol=0)
    got32 = p32.expect(bloch)
    assert np.all(np.abs(got32 - want) <= 1e-5 * np.abs(want) + 1e-7)
    p64.close()
    p32.close()


@pytest.mark.parametrize("f32", [False, True])
def test_batched_n64_b256_growth_stops_cleanly(f32):
    """The full 30 steps do not fit: with a 4 GiB budget the run stops with
    PP_ERR_CAPACITY, and the context still holds the last completed step."""
    n, B = 64, 256
    gx, gz, th, x, z, coef = ring_batch(n, B)
    p = pp.Propagator(n, x, z, coef, eps=1e-5, batch=B, f32=f32, budget=4 * GB)
    bloch = pi.zero_state(n).bloch
    done = 0
    with pytest.raises(pp.PPError) as e:
        for _ in range(30):
            before = p.expect(bloch)
            p.apply_layer(gx, gz, th, True)
            done += 1
    assert e.value.status == 3  # PP_ERR_CAPACITY
    assert 2 <= done < 30
    # the restored table is the same set of terms in another order; the
    # overlap sums in table order
    np.testing.assert_allclose(p.expect(bloch), before, atol=1e-12, rtol=0)
    p.close()


@pytest.mark.parametrize("batch,f32", [(1, False), (256, True), (256, False)])
def test_layers_that_stall_for_room_match_the_per_gate_path(batch, f32):
    """With almost no headroom asked for at a layer's start (room_factor
    0.01: room for twice the stored terms), every layer that more than
    doubles the table stops part way, grows it and goes on.  The persistent
    layer kernel then stops in every block at the same gate and resumes after
    the growth; the result equals the per-gate path's with the default
    headroom, entry for entry (the same rows in the same arithmetic)."""
    n, layers = 64, 4
    gx, gz, th, x, z, coef = ring_batch(n, max(batch, 2))
    if batch == 1:
        th, coef = th[:, 0].copy(), coef[:, 0].copy()

    def make(persistent, room):
        return pp.Propagator(n, x, z, coef, eps=1e-5, batch=batch, f32=f32,
                             layer_kernel=persistent, room_factor=room)

    ref = make(False, 0.0)
    p = make(True, 0.01)
    for _ in range(layers):
        ref.apply_layer(gx, gz, th, True)
        p.apply_layer(gx, gz, th, True)
    st = p.stats()
    assert st["persistent"] == 1 and st["stalls"] >= 2
    assert ref.stats()["stalls"] < st["stalls"]
    got, want = as_dict(*p.export()), as_dict(*ref.export())
    assert set(got) == set(want) and len(want) > 1000
    for k in want:
        np.testing.assert_array_equal(got[k], want[k])
    bloch = pi.zero_state(n).bloch
    # the overlap sums in table order, which the stalls' compactions change
    np.testing.assert_allclose(p.expect(bloch), ref.expect(bloch), atol=1e-12, rtol=0)
    p.close()
    ref.close()


# ------------------------------------------------------ XXZ, S_n, sublayers

@pytest.mark.parametrize("n,eps,split,layers", [(8, 1e-4, True, None), (8, 1e-4, False, None),
                                                (10, 1e-5, True, None), (10, 1e-4, False, None),
                                                (36, 0.05, True, 16)])
def test_xxz_sn_matches_oracle(n, eps, split, layers):
    wl = pi.xxz_all_to_all(n, 0.05, 4 if n < 36 else 6, eps=eps, symmetry=2, split=split)
    bloch = wl.state.bloch
    for prop, st in run_both(wl, 2, layers=layers):
        assert_close(prop, st, eps)
        assert float(prop.expect(bloch)) == pytest.approx(st.expect(bloch, 2), abs=1e-10)
    assert prop.num_terms()[0] <= math.comb(n + 3, 3)
    prop.close()


# ------------------------------------------- capacity errors restore state

@pytest.mark.parametrize("batch", [1, 4])
def test_capacity_error_restores_the_context(batch):
    wl = pi.config1_ring(n=32, steps=8)
    x, z, c = wl.observable.arrays()
    coef = np.repeat(c[:, None], batch, axis=1) if batch > 1 else c

    def cols(th):
        return np.repeat(th[:, None], batch, axis=1) if batch > 1 else th

    def make(budget):
        return pp.Propagator(32, x, z, coef, symmetry=0, eps=wl.eps, max_weight=wl.max_weight,
                             budget=budget, batch=batch)

    ref = make(0)
    for layer in reversed(range(8)):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        ref.apply_layer(gx, gz, cols(th), True)
    budget = ref.stats()["device_bytes"] // 4  # the run outgrows this part way
    ref.close()
    ref, p = make(0), make(budget)
    bloch = wl.state.bloch
    failed = 0
    for layer in reversed(range(8)):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        before = as_dict(*p.export())
        e_before = p.expect(bloch)
        try:
            p.apply_layer(gx, gz, cols(th), True)
        except pp.PPError as e:
            assert e.status == 3  # PP_ERR_CAPACITY
            failed += 1
            after = as_dict(*p.export())
            assert set(after) == set(before)
            for k in before:
                np.testing.assert_array_equal(after[k], before[k])
            np.testing.assert_allclose(p.expect(bloch), e_before, atol=1e-12, rtol=0)
            pp.pp_set_budget(p.ctx, 0)  # lift the ceiling and apply the same layer again
            p.apply_layer(gx, gz, cols(th), True)
        ref.apply_layer(gx, gz, cols(th), True)
        a_, b_ = as_dict(*p.export()), as_dict(*ref.export())
        assert set(a_) == set(b_)
        for k in b_:
            np.testing.assert_array_equal(a_[k], b_[k])
    assert failed == 1
    p.close()
    ref.close()
