"""Batched angle sets (B coefficient columns per string) vs the batched oracle.

* FP64 rows, gates only: the same per-column arithmetic as the oracle, so
  term sets and every coefficient are bit-identical.
* FP32 rows: gate arithmetic in FP32, merges and overlaps in FP64; with
  truncation off the term sets equal the FP64 oracle's and <O> per column
  agrees within 1e-5 relative (the FP32 target), plus an absolute floor.
"""
import math

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


def ring_theta(n, angles):
    B = len(angles)
    th = np.zeros((3 * n, B))
    th[:n] = angles[:, 0]
    th[n:2 * n] = angles[:, 1]
    th[2 * n:] = angles[:, 2]
    return th


def run_batched(n, B, steps, eps, wmax, group, f32, seed=0, state=None, noise_p=0.0):
    angles = pi.batched_ring_angles(B, seed)
    layer = pi.ring_layer(n, 0.0, 0.0, 0.0)
    gx, gz, _ = pi.Circuit(n, [layer]).gate_arrays(0)
    th = ring_theta(n, angles)
    obs = pi.mean_z(n)
    x, z, c = obs.arrays()
    coef = np.repeat(c[:, None], B, axis=1)
    mode = pp.NOISE_PER_GATE if noise_p > 0 else pp.NOISE_NONE
    prop = pp.Propagator(n, x, z, coef, symmetry=group, eps=eps, max_weight=wmax, batch=B, f32=f32,
                         noise_mode=mode, noise_p=noise_p)
    st = oracle.BatchedOracleState(n, B, x, z, coef, group=group, eps=eps, max_weight=wmax)
    for _ in range(steps):
        prop.apply_layer(gx, gz, th, boundary=True)
        st.apply_layer(gx, gz, th, noise_mode=mode, p=noise_p, group=group)
    return prop, st


def rows_dict(x, z, c):
    d = {tuple(int(v) for v in x[i]) + tuple(int(v) for v in z[i]): c[i] for i in range(len(c))}
    assert len(d) == len(c), "a string appears twice in the table"
    return d


@pytest.mark.parametrize("n,B,eps,wmax", [(10, 5, 1e-4, 6), (12, 33, 0.0, 5), (64, 8, 1e-3, 4)])
def test_batched_fp64_gates_bitexact(n, B, eps, wmax):
    prop, st = run_batched(n, B, 3, eps, wmax, 0, False)
    g = rows_dict(*prop.export())
    o = rows_dict(*st.export())
    assert set(g) == set(o)
    for k in o:
        np.testing.assert_array_equal(g[k], o[k])
    bloch = pi.zero_state(n).bloch
    np.testing.assert_allclose(prop.expect(bloch), st.expect(bloch), atol=1e-12, rtol=0)


@pytest.mark.parametrize("n,B", [(12, 16), (64, 8)])
def test_batched_fp64_zn_merge(n, B):
    prop, st = run_batched(n, B, 3, 1e-4, 5, 1, False)
    g = rows_dict(*prop.export())
    o = rows_dict(*st.export())
    assert set(g) == set(o)
    for k in o:
        np.testing.assert_allclose(g[k], o[k], atol=1e-12, rtol=0)
    bloch = pi.zero_state(n).bloch
    np.testing.assert_allclose(prop.expect(bloch), st.expect(bloch), atol=1e-10, rtol=0)


@pytest.mark.parametrize("group", [0, 1])
def test_batched_fp32_storage_within_fp32_tolerance(group):
    n, B = 10, 24
    prop, st = run_batched(n, B, 3, 0.0, 6, group, True)
    g = rows_dict(*prop.export())
    o = rows_dict(*st.export())
    assert set(g) == set(o)
    worst = max(float(np.max(np.abs(g[k] - o[k]))) for k in o)
    assert worst < 1e-5
    bloch = pi.zero_state(n).bloch
    got, want = prop.expect(bloch), st.expect(bloch)
    assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + 1e-6)


def test_fp32_single_column():
    n = 12
    prop, st = run_batched(n, 1, 3, 0.0, 5, 0, True)
    bloch = pi.zero_state(n).bloch
    assert abs(float(prop.expect(bloch)) - float(st.expect(bloch)[0])) < 1e-5


def test_batched_column_equals_unbatched_run():
    """Column b of a batched FP64 run without truncation equals the plain
    single-angle-set GPU run with column b's angles."""
    n, B = 9, 6
    prop, _ = run_batched(n, B, 2, 0.0, -1, 0, False, seed=5)
    angles = pi.batched_ring_angles(B, 5)
    bx, bz, bc = prop.export()
    bd = rows_dict(bx, bz, bc)
    for b in (0, 3, 5):
        wl = pi.config1_ring(n=n, steps=2, theta_j=angles[b, 0], theta_x=angles[b, 1],
                             theta_z=angles[b, 2], eps=0.0, max_weight=-1)
        single = pp.Propagator.from_workload(wl, symmetry=0)
        single.run(wl)
        sd = rows_dict(*single.export())
        for k, v in sd.items():
            assert bd[k][b] == v
        assert math.isclose(float(single.expect(wl.state.bloch)),
                            float(prop.expect(wl.state.bloch)[b]), abs_tol=1e-13)


@pytest.mark.parametrize("f32", [False, True])
def test_batched_at_the_maximum_batch(f32):
    """B = 512, the largest batch the ABI accepts: FP64 rows bit for bit, FP32
    rows within the FP32 tolerance (truncation off, so that no term sits on the
    threshold), overlaps of all 512 columns."""
    n, B = 8, 512
    prop, st = run_batched(n, B, 2, 0.0 if f32 else 1e-5, -1, 1, f32, seed=9)
    g = rows_dict(*prop.export())
    o = rows_dict(*st.export())
    assert set(g) == set(o) and len(o) > 10
    for k in o:
        if f32:
            assert float(np.max(np.abs(g[k] - o[k]))) < 1e-5
        else:
            np.testing.assert_allclose(g[k], o[k], atol=1e-12, rtol=0)
    bloch = pi.neel_state(n).bloch
    got, want = prop.expect(bloch), st.expect(bloch)
    assert got.shape == (B,)
    tol = 1e-5 * np.abs(want) + 1e-6 if f32 else 1e-10
    assert np.all(np.abs(got - want) <= tol)


@pytest.mark.parametrize("n,B,eps,wmax,group", [(10, 8, 1e-4, 6, 0), (12, 16, 1e-4, 5, 1),
                                                 (64, 8, 1e-3, 4, 0)])
def test_batched_fp64_per_gate_noise_bitexact(n, B, eps, wmax, group):
    """Per-gate depolarising damping (1-p)^k on batched FP64 rows: the same
    per-column operations as the batched oracle, so without a merge the term
    sets and coefficients are bit-identical; with a Z_n merge (FP64 atomics)
    within 1e-12."""
    prop, st = run_batched(n, B, 3, eps, wmax, group, False, seed=4, noise_p=0.02)
    g = rows_dict(*prop.export())
    o = rows_dict(*st.export())
    assert set(g) == set(o) and len(o) > 10
    for k in o:
        if group == 0:
            np.testing.assert_array_equal(g[k], o[k])
        else:
            np.testing.assert_allclose(g[k], o[k], atol=1e-12, rtol=0)
    bloch = pi.neel_state(n).bloch
    np.testing.assert_allclose(prop.expect(bloch), st.expect(bloch), atol=1e-10, rtol=0)


@pytest.mark.parametrize("group", [0, 1])
def test_batched_fp32_per_gate_noise_within_fp32_tolerance(group):
    """FP32 rows with per-gate damping: the damping factors and the rotation are
    applied in FP32, merges and overlaps in FP64.  Truncation is off so that no
    term sits on the threshold; <O> per column agrees with the FP64 oracle
    within 1e-5 relative (plus a 1e-6 floor)."""
    n, B = 10, 24
    prop, st = run_batched(n, B, 3, 0.0, 6, group, True, seed=6, noise_p=0.05)
    g = rows_dict(*prop.export())
    o = rows_dict(*st.export())
    assert set(g) == set(o)
    worst = max(float(np.max(np.abs(g[k] - o[k]))) for k in o)
    assert worst < 1e-5
    bloch = pi.neel_state(n).bloch
    got, want = prop.expect(bloch), st.expect(bloch)
    assert np.all(np.abs(got - want) <= 1e-5 * np.abs(want) + 1e-6)


@pytest.mark.parametrize("f32,noise", [(False, 0.0), (False, 0.03), (True, 0.0)])
def test_batched_launch_paths_agree(f32, noise):
    """All gates of a layer in one persistent cooperative launch, and one kernel
    per gate replayed from CUDA graphs, give the same rows bit for bit and the
    same update statistics (gates the occupancy test skips included)."""
    n, B = 14, 40
    angles = pi.batched_ring_angles(B, 11)
    gx, gz, _ = pi.Circuit(n, [pi.ring_layer(n, 0.0, 0.0, 0.0)]).gate_arrays(0)
    th = ring_theta(n, angles)
    x, z, c = pi.mean_z(n).arrays()
    coef = np.repeat(c[:, None], B, axis=1)
    runs, stats = [], []
    for layer_kernel in (True, False):
        prop = pp.Propagator(n, x, z, coef, eps=1e-4, max_weight=6, batch=B, f32=f32,
                             layer_kernel=layer_kernel,
                             noise_mode=pp.NOISE_PER_GATE if noise else pp.NOISE_NONE,
                             noise_p=noise)
        for _ in range(3):
            prop.apply_layer(gx, gz, th, boundary=False)
        runs.append(rows_dict(*prop.export()))
        st = prop.stats()
        stats.append((st["gate_updates"], st["anticommuting_terms"], st["gates_applied"]))
        prop.close()
    assert stats[0] == stats[1]
    assert set(runs[0]) == set(runs[1]) and len(runs[0]) > 50
    for k in runs[0]:
        np.testing.assert_array_equal(runs[0][k], runs[1][k])
