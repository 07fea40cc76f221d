"""Benchmark: Pauli-term gate updates/s on the translation-symmetric ring.

Workload (one "step" = one whole job): the n=32 ring circuit (RZZ(0.4) on
all bonds, RX(0.6), RZ(0.3) on all qubits; 20 Trotter steps = 1920 gates),
observable (1/n) sum Z_i, state |0...0>, coefficient truncation 1e-4, Pauli
weight <= 10, FP64.  It is propagated twice, plain and Z_32-merged, and
<O> is read for both.  One gate update = one (live term, gate) pair.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  ``value`` is measured with the observable
already in device memory; ``e2e`` goes through the host-buffer C-ABI calls
(pp_create from host arrays, pp_expect back to the host).  Both timed regions
run the job without instrumentation.  ``roofline`` is for the layer kernel,
timed with CUDA events around every layer kernel on the context's stream in a
separate pass of the same jobs.  ``cpu_baseline`` times the CPU
oracle on a bounded prefix of the same workload.  ``served`` (one GPU only)
is the serving part of the metric: a scaled Poisson stream of 300 jobs
through pp_submit after the main job, with jobs/s and latency p50/p99
(``--no-serving`` leaves it out).  ``other_workloads`` (one GPU only) times the
all-to-all n=64, the batched-angle ring n=64 and the XXZ n=36 workloads once
each (``--no-others`` leaves them out).  With N > 1 (torchrun) every rank runs an
independent replica of the job (the path does not shard).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import pp_inputs as pi  # noqa: E402

WORKLOAD = "ring_n32_20steps_eps1e-4_w10_plain+Z32"
METRIC = "pauli_term_gate_updates_per_s"
UNIT = "updates/s"
KEY_BYTES = 16   # one uint64 X word + one uint64 Z word (n = 32)
COEF_BYTES = 8   # FP64
# per live anticommuting term: its coefficient read and rescaled (2C), the
# child's key and coefficient written (K + C), and one insert: a key compared
# and one index slot (K + C)
BYTES_PER_ANTICOMMUTING = 2 * COEF_BYTES + KEY_BYTES + COEF_BYTES + KEY_BYTES + COEF_BYTES


def algorithmic_bytes(updates, skipped_updates, anticommuting):
    """The layer kernel's algorithmic bytes: the key of every live term
    entering a scanned gate, plus BYTES_PER_ANTICOMMUTING per live
    anticommuting term.  Updates in gates the occupancy test skipped move no
    bytes (every string commutes with the gate and nothing is read)."""
    return KEY_BYTES * (updates - skipped_updates) + BYTES_PER_ANTICOMMUTING * anticommuting
# DRAM bytes (read + write) per algorithmic byte of layer_kernel<1>, from one
# ncu capture (dram__bytes_read.sum + dram__bytes_write.sum) of the last layer
# of the Z_32-merged job, taken with the kernel sources whose digest is
# recorded beside it.  When the sources differ from that digest the figure no
# longer describes the kernel and the JSON line reports traffic as null.
TRAFFIC_CAPTURE = {"ratio": 2.595, "sources_sha16": "97da5ada6879b7ac"}  # 7.956 GB / 3.066 GB
KERNEL_SOURCES = ["paper_2512_12094_gb300/csrc/pp_kernels.cu",
                  "paper_2512_12094_gb300/csrc/pp_device.cuh",
                  "paper_2512_12094_gb300/csrc/pp_internal.h"]


def kernel_sources_sha16():
    """Digest of the sources that define layer_kernel<1>."""
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


HBM_NOMINAL_GBS = 7900.0  # GB300 HBM3e data-sheet bandwidth, for context beside the measured peak


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 100 ms."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.proc = None
        self.lines = []
        self.index = index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


GROUPS = {"both": (0, 1), "plain": (0,), "zn": (1,)}


def run_job(pp, wl, layers, obs_dev, stream, host_inputs, profile, marks=None, only="both",
            block_threads=0):
    """One job: plain then Z_n-merged propagation of the whole circuit.
    marks: optional [event, event, event] recorded before, between, after."""
    n = wl.circuit.n
    stats = []
    vals = []
    for gi, group in enumerate(GROUPS[only]):
        if marks is not None:
            marks[gi].record(stream)
        cfg = pp.pp_config_default(n_qubits=n, symmetry=group, coeff_eps=wl.eps,
                                   max_weight=wl.max_weight, cuda_stream=stream,
                                   profile_kernels=int(profile), block_threads=block_threads)
        if host_inputs:
            ox, oz, oc = wl.observable.arrays()
            ctx = pp.pp_create(cfg, ox, oz, oc)
        else:
            dx, dz, dc = obs_dev
            ctx = pp.pp_create_device(cfg, len(wl.observable.terms), dx, dz, dc)
        for packed, th in layers:
            pp.pp_apply_layer(ctx, packed, th, True)
        vals.append(pp.pp_expect(ctx, wl.state.bloch))
        stats.append(pp.pp_stats(ctx))
        pp.pp_destroy(ctx)
    if marks is not None:
        marks[2].record(stream)
    return vals, stats


def trace_layers(args):
    """One JSON line per layer of the config-1 job (plain, then Z_32): live and
    stored terms after the layer, the layer's gate updates and anticommuting
    strings, the layer kernels' time (CUDA events around each launch) and the
    whole layer's time (events around pp_apply_layer, merge included), and the
    layer kernels' algorithmic bandwidth against the measured copy peak."""
    import torch
    import paper_2512_12094_gb300 as pp
    torch.cuda.set_device(0)
    pp.build()
    pp.load()
    wl = pi.config1_ring()
    layers = []
    for layer in reversed(range(len(wl.circuit.layers))):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        layers.append((pp.pack_gates(gx, gz), th))
    ox, oz, oc = wl.observable.arrays()
    hbm, kind = peaks()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        for label, group in (("plain", 0), ("Z32", 1)):
            cfg = pp.pp_config_default(n_qubits=32, symmetry=group, coeff_eps=wl.eps,
                                       max_weight=wl.max_weight, cuda_stream=stream,
                                       profile_kernels=1)
            ctx = pp.pp_create(cfg, ox, oz, oc)
            prev = pp.pp_stats(ctx)
            for k, (packed, th) in enumerate(layers):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                pp.pp_apply_layer(ctx, packed, th, True)
                e1.record(stream)
                e1.synchronize()
                st = pp.pp_stats(ctx)
                upd = st["gate_updates"] - prev["gate_updates"]
                skip = st["skipped_updates"] - prev["skipped_updates"]
                ac = st["anticommuting_terms"] - prev["anticommuting_terms"]
                kms = st["gate_kernel_ms"] - prev["gate_kernel_ms"]
                alg = algorithmic_bytes(upd, skip, ac)
                gbs = alg / (kms / 1e3) / 1e9 if kms > 0 else None
                print(json.dumps({"job": label, "layer": k, "live_terms": st["live_terms"],
                                  "stored_terms": st["stored_terms"], "gate_updates": upd,
                                  "skipped_updates": skip, "anticommuting_terms": ac,
                                  "layer_kernel_ms": kms, "layer_ms": e0.elapsed_time(e1),
                                  "algorithmic_gbs": gbs,
                                  "frac": (gbs / hbm) if gbs else None, "peak_kind": kind,
                                  "stalls": st["stalls"] - prev["stalls"]}), flush=True)
                prev = st
            pp.pp_destroy(ctx)


def run_job_concurrent(pp, wl, layers, obs_dev, streams, join, host_inputs, plain_share,
                       block_threads=0):
    """One job with its two propagations (plain and Z_n-merged) at the same
    time, each driven by its own host thread on its own stream.  The plain
    run's persistent layer launches take the fraction plain_share of the GPU
    and the merged run's the rest (pp_set_grid_fraction), so both fit at once;
    when the plain run's last layer has returned, the merged run takes the
    whole GPU from its next layer on.  Returns (vals, stats, start, ends, end):
    CUDA events on the joining stream (start, end) and each run's own end."""
    import threading
    import torch
    n = wl.circuit.n
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    start.record(join)
    for s_ in streams:
        s_.wait_event(start)
    vals, stats, errors = [None, None], [None, None], []
    plain_done = threading.Event()

    def run(gi):
        try:
            stream = streams[gi]
            cfg = pp.pp_config_default(n_qubits=n, symmetry=gi, coeff_eps=wl.eps,
                                       max_weight=wl.max_weight, cuda_stream=stream,
                                       block_threads=block_threads)
            if host_inputs:
                ox, oz, oc = wl.observable.arrays()
                ctx = pp.pp_create(cfg, ox, oz, oc)
            else:
                dx, dz, dc = obs_dev
                ctx = pp.pp_create_device(cfg, len(wl.observable.terms), dx, dz, dc)
            share = plain_share if gi == 0 else 1.0 - plain_share
            pp.pp_set_grid_fraction(ctx, share)
            for packed, th in layers:
                if gi == 1 and share < 1.0 and plain_done.is_set():
                    share = 1.0  # the plain run's layer launches are all finished
                    pp.pp_set_grid_fraction(ctx, share)
                pp.pp_apply_layer(ctx, packed, th, True)
            if gi == 0:
                plain_done.set()
            vals[gi] = pp.pp_expect(ctx, wl.state.bloch)
            stats[gi] = pp.pp_stats(ctx)
            pp.pp_destroy(ctx)
            ends[gi].record(stream)
        except Exception as e:  # noqa: BLE001 - re-raised below
            plain_done.set()
            errors.append(e)

    threads = [threading.Thread(target=run, args=(gi,)) for gi in (0, 1)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    if errors:
        raise errors[0]
    for e in ends:
        join.wait_event(e)
    end.record(join)
    return vals, stats, start, ends, end


def bench_ours(args):
    import torch
    import paper_2512_12094_gb300 as pp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    pp.build()
    pp.load()

    wl = pi.config1_ring()
    L = len(wl.circuit.layers)
    layers = []
    for layer in reversed(range(L)):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        layers.append((pp.pack_gates(gx, gz), th))
    ox, oz, oc = wl.observable.arrays()
    dev = torch.device("cuda", local)
    obs_dev = (torch.from_numpy(ox.view(np.int64)).to(dev), torch.from_numpy(oz.view(np.int64)).to(dev),
               torch.from_numpy(oc).to(dev))
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    concurrent = args.only == "both" and args.plain_share > 0.0
    job_streams = [torch.cuda.Stream(device=dev) for _ in range(2)]

    def timed_job(host_inputs, profile):
        """(vals, stats, total ms, [plain ms, merged ms]); the two propagations
        run at the same time unless profiling or --plain-share 0."""
        flush.zero_()
        barrier()
        if concurrent and not profile:
            vals, stats, start, ends, end = run_job_concurrent(
                pp, wl, layers, obs_dev, job_streams, stream, host_inputs, args.plain_share,
                block_threads=args.block_threads)
            end.synchronize()
            return vals, stats, start.elapsed_time(end), [start.elapsed_time(e) for e in ends]
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        if args.only != "both":
            ev[1] = ev[0]
        vals, stats = run_job(pp, wl, layers, obs_dev, stream, host_inputs, profile, marks=ev,
                              only=args.only, block_threads=args.block_threads)
        ev[2].synchronize()
        return vals, stats, ev[0].elapsed_time(ev[2]), [ev[0].elapsed_time(ev[1]),
                                                         ev[1].elapsed_time(ev[2])]

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            timed_job(False, False)
        barrier()
        clocks = ClockSampler(local)
        clocks.start()
        ms_total, upd, launches = 0.0, 0.0, 0
        split = [0.0, 0.0]
        vals = stats = None
        for _ in range(args.steps):
            # no per-kernel events here: the job exactly as a user runs it
            vals, stats, ms, parts = timed_job(False, False)
            ms_total += ms
            if args.only == "both":
                split[0] += parts[0]
                split[1] += parts[1]
            for st in stats:
                upd += st["gate_updates"]
                launches += st["kernel_launches"]
        barrier()
        # end to end through the host-buffer API (inputs copied in, result read back)
        e2e_ms = 0.0
        if not args.no_e2e:
            for _ in range(args.steps):
                _, _, ms, _ = timed_job(True, False)
                e2e_ms += ms
        clk = clocks.stop()  # both timed regions
        barrier()
        # roofline pass: the same jobs with CUDA events around every layer kernel
        # on the job's stream (separate from the timed regions above)
        pupd = ac = gate_ms = skipped = 0.0
        gate_n = gates_skipped = 0
        for _ in range(args.steps):
            _, pstats, _, _ = timed_job(False, True)
            for st in pstats:
                pupd += st["gate_updates"]
                skipped += st["skipped_updates"]
                gates_skipped += st["gates_skipped"]
                ac += st["anticommuting_terms"]
                gate_ms += st["gate_kernel_ms"]
                gate_n += st["gate_kernels_timed"]

    value, e2e_value, ms_max, e2e_max, total_upd = replica_throughput(dist, ms_total, e2e_ms, upd,
                                                                      dev)
    upd_per_rank = upd / args.steps  # one job's updates (the same on every rank)
    hbm, peak_kind = peaks()
    # gates the occupancy test skipped read nothing: their updates count in the
    # metric (every string is processed: it commutes) but add no bytes
    bytes_alg = algorithmic_bytes(pupd, skipped, ac)
    achieved = bytes_alg / (gate_ms / 1e3) / 1e9 if gate_ms > 0 else None
    gates_per_job = len(GROUPS[args.only]) * sum(len(l[1]) for l in layers)
    h2d = len(GROUPS[args.only]) * (ox.nbytes + oz.nbytes + oc.nbytes + wl.state.bloch.nbytes +
                                     sum(p.nbytes + th.nbytes for p, th in layers))
    d2h = len(GROUPS[args.only]) * (8 + L * 512)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    served = None
    if world == 1 and not args.no_serving:
        try:
            served = served_summary(pp)
        except Exception as e:  # the headline line is printed whatever happens here
            served = {"error": f"{type(e).__name__}: {e}"}
    others = None
    if world == 1 and not args.no_others:
        try:
            others = other_workloads_summary(pp)
        except Exception as e:  # the headline line is printed whatever happens here
            others = {"error": f"{type(e).__name__}: {e}"}
    cpu = cpu_baseline(seconds=args.cpu_seconds) if (world == 1 and not args.no_cpu) else None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.only == "both" else WORKLOAD + ":" + args.only,
                   "n_qubits": 32, "trotter_steps": 20, "gates_per_job": gates_per_job,
                   "coeff_eps": 1e-4, "max_weight": 10, "updates_per_job": upd_per_rank,
                   "l2": "flushed (256 MB write) before every timed job",
                   "parallelism": "replicas" if world > 1 else "single"},
        "breakdown_ms_per_step": {"plain": split[0] / args.steps, "zn": split[1] / args.steps,
                                  "layer_kernels_instrumented_pass": gate_ms / args.steps},
        "schedule": ({"propagations": "plain and Z_32 at the same time, one host thread and "
                                      "stream each; breakdown = each run's own span",
                      "plain_grid_fraction": args.plain_share}
                     if concurrent else {"propagations": "plain, then Z_32, on one stream"}),
        "result": result_summary(vals, stats, args.only),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": (achieved / hbm) if achieved else None,
                     "traffic": traffic_per_launch(bytes_alg / max(gate_n, 1)),
                     "traffic_basis": "ncu DRAM bytes per algorithmic byte of the last layer "
                                      "of the Z_32 job x this run's average launch; null when "
                                      "the kernel sources differ from the captured ones",
                     "kernel": "layer_kernel<1>", "block_threads": stats[-1]["block_threads"],
                     "peak_kind": peak_kind,
                     "peak_nominal": HBM_NOMINAL_GBS,
                     "frac_nominal": (achieved / HBM_NOMINAL_GBS) if achieved else None,
                     "bytes_model": "16 B key per live term entering a scanned gate + 64 B per "
                                    "live anticommuting term (gates skipped by the occupancy "
                                    "test move no bytes)",
                     "skipped_updates_fraction": (skipped / pupd) if pupd else None,
                     "gates_skipped_per_job": gates_skipped / max(args.steps, 1),
                     "avg_launch_us": 1e3 * gate_ms / max(gate_n, 1),
                     "algorithmic_bytes_per_launch": bytes_alg / max(gate_n, 1),
                     "timing": "CUDA events around every layer kernel, in a pass of the "
                               "same jobs after the timed regions"},
        "clocks": clk,
        "cpu_baseline": cpu,
        "served": served,
        "other_workloads": others,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def traffic_per_launch(alg_bytes_per_launch):
    """DRAM bytes per launch scaled from the capture's ratio, or None when the
    kernel sources changed since that capture."""
    if TRAFFIC_CAPTURE["sources_sha16"] != kernel_sources_sha16():
        return None
    return TRAFFIC_CAPTURE["ratio"] * alg_bytes_per_launch


def result_summary(vals, stats, only):
    """<O> and live terms of each run; with both runs, the expectation
    difference between the plain and the Z_32-merged propagation."""
    out = {"expect": vals, "live_terms": [st["live_terms"] for st in stats]}
    if only == "both" and len(vals) == 2:
        out["plain_minus_merged"] = vals[0] - vals[1]
        out["abs_error_merged_vs_plain"] = abs(vals[0] - vals[1])
        out["live_terms_merged_over_plain"] = stats[1]["live_terms"] / max(stats[0]["live_terms"], 1)
    return out


def host_cpu():
    """The host the CPU baseline ran on: logical CPUs, architecture and the
    CPU model as /proc/cpuinfo names it (x86: "model name"; Arm: the
    implementer and part numbers), for the baseline's record."""
    import platform
    info = {"nproc": os.cpu_count(), "arch": platform.machine()}
    try:
        with open("/proc/cpuinfo") as f:
            fields = {}
            for ln in f:
                k, _, v = ln.partition(":")
                k, v = k.strip(), v.strip()
                if k and v and k not in fields:
                    fields[k] = v
        if "model name" in fields:
            info["model"] = fields["model name"]
        elif "CPU part" in fields:
            info["model"] = "implementer %s part %s" % (fields.get("CPU implementer", "?"),
                                                        fields["CPU part"])
    except Exception:  # a record only: the baseline is reported without it
        pass
    return info


def cpu_baseline(seconds=20.0):
    """The CPU oracle, as it stands, on a bounded prefix of the same workload:
    plain and Z_32-merged propagation, layer by layer, each run stopped once
    it has used seconds/2 of CPU time."""
    import oracle
    oracle.build()
    wl = pi.config1_ring()
    total_upd = 0.0
    total_t = 0.0
    done = []
    for group in (0, 1):
        ox, oz, oc = wl.observable.arrays()
        st = oracle.OracleState(32, ox, oz, oc, group=group, eps=wl.eps, max_weight=wl.max_weight)
        t0 = time.process_time()
        k = 0
        for layer in reversed(range(len(wl.circuit.layers))):
            gx, gz, th = wl.circuit.gate_arrays(layer)
            st.apply_layer(gx, gz, th, group=group)
            k += 1
            if time.process_time() - t0 > seconds / 2:
                break
        total_t += time.process_time() - t0
        total_upd += st.updates
        done.append(k)
    return {"value": total_upd / total_t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "first %d (plain) and %d (Z_32) of 20 Trotter steps of the job, "
                      "%.1f s CPU, %.3g updates" % (done[0], done[1], total_t, total_upd),
            "seconds": total_t, "host": host_cpu()}


def profile_layer(args):
    """Run the Z_n-merged job once and bracket layer K (application order)
    with cudaProfilerStart/Stop, so that `ncu --profile-from-start off`
    captures exactly that layer's kernels.  Prints the layer's algorithmic
    bytes (same model as the roofline) for comparison with ncu's counters."""
    import torch
    import paper_2512_12094_gb300 as pp
    pp.build()
    pp.load()
    wl = pi.config1_ring()
    ox, oz, oc = wl.observable.arrays()
    cfg = pp.pp_config_default(n_qubits=32, symmetry=pp.SYM_ZN, coeff_eps=wl.eps,
                               max_weight=wl.max_weight, profile_kernels=1)
    ctx = pp.pp_create(cfg, ox, oz, oc)
    L = len(wl.circuit.layers)
    for k, layer in enumerate(reversed(range(L))):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        before = pp.pp_stats(ctx)
        if k == args.profile_layer:
            torch.cuda.synchronize()
            torch.cuda.profiler.start()
        pp.pp_apply_layer(ctx, pp.pack_gates(gx, gz), th, True)
        if k == args.profile_layer:
            torch.cuda.synchronize()
            torch.cuda.profiler.stop()
            after = pp.pp_stats(ctx)
            upd = after["gate_updates"] - before["gate_updates"]
            skip = after["skipped_updates"] - before["skipped_updates"]
            ac = after["anticommuting_terms"] - before["anticommuting_terms"]
            # the roofline's model: updates in gates the occupancy test skipped move no bytes
            print(json.dumps({"profile_layer": k, "updates": upd, "skipped_updates": skip,
                              "anticommuting_terms": ac,
                              "algorithmic_bytes": algorithmic_bytes(upd, skip, ac),
                              "layer_kernel_ms": after["gate_kernel_ms"] - before["gate_kernel_ms"],
                              "launches": after["gate_kernels_timed"] - before["gate_kernels_timed"],
                              "live_terms": after["live_terms"]}), flush=True)
    pp.pp_destroy(ctx)


A2A_N = {16: 8, 32: 10, 64: 12, 128: 16}


def serving_specs(n_jobs, rate, seed=0):
    """The Poisson job stream of the serving workload, scaled so that every
    job finishes in well under a second: ring jobs keep n in {16..128} with
    steps <= 20, weight <= 8 and eps >= 1e-4; all-to-all jobs use n in
    {8, 10, 12, 16} (mapped from {16, 32, 64, 128}) and <= 4 steps."""
    out = []
    for j in pi.serving_stream(n_jobs, rate, seed):
        a = j["angles"]
        eps = max(j["eps"], 1e-4)
        if j["family"] == "ring":
            wl = pi.config1_ring(n=j["n"], steps=min(j["steps"], 20), theta_j=a[0], theta_x=a[1],
                                 theta_z=a[2], eps=eps, max_weight=8, symmetry=j["group"])
        else:
            n = A2A_N[j["n"]]
            wl = pi.config0_heisenberg(n=n, dt=0.02 + 0.02 * a[0], steps=min(j["steps"], 4))
            wl.observable = pi.mean_z(n)
            wl.state = pi.neel_state(n)
            wl.eps = eps
            wl.symmetry = j["group"]
        out.append((j["arrival"], wl))
    return out


def serving_specs_full(n_jobs, rate, seed=0):
    """The serving workload at its stated sizes: the first n_jobs of the seeded
    2000-job Poisson stream.  Ring jobs are the translation-symmetric ring
    circuit with the job's three angles, Pauli weight <= 10, (1/n) sum Z and
    |0...0>; all-to-all jobs are the Heisenberg circuit with per-gate
    depolarising damping p = 0.01, (1/n) sum Z and the Neel state, with a step
    dt in [0.01, 0.03] from the job's first angle.  n, steps, eps and the group
    are the job's own."""
    out = []
    for j in pi.serving_stream(2000, rate, seed)[:n_jobs]:
        a = j["angles"]
        if j["family"] == "ring":
            wl = pi.config1_ring(n=j["n"], steps=j["steps"], theta_j=a[0], theta_x=a[1],
                                 theta_z=a[2], eps=j["eps"], max_weight=10, symmetry=j["group"])
        else:
            wl = pi.config2_all_to_all(n=j["n"], dt=0.01 + 0.02 * a[0] / (np.pi / 2),
                                       steps=j["steps"], p=0.01, eps=j["eps"], noise_mode=1,
                                       symmetry=j["group"])
        out.append((j["arrival"], wl))
    return out


def serve_stream(pp, specs, slots, full, check_every=None):
    """Serve `specs` (arrival time, workload) through pp_submit on a server
    with `slots` workers and a 150 GB budget, submitting each job at its
    arrival time; then run a sample of the same jobs (every check_every-th;
    by default all of them for the scaled stream and about 50 for the
    full-size one) one after the other on one slot to check their results
    against the job run alone.  Returns (results, wall s, results alone,
    wall s alone, the sample's indices or None for all)."""
    jobs = []
    for _, wl in specs:
        cfg = pp.pp_config_default(n_qubits=wl.circuit.n, symmetry=wl.symmetry, coeff_eps=wl.eps,
                                   max_weight=wl.max_weight, noise_mode=wl.noise_mode,
                                   noise_p=wl.noise_p)
        x, z, c = wl.observable.arrays()
        gx, gz, th = wl.circuit.gate_arrays(0)
        # no reservation named: the server estimates it from the observable and
        # grows it with the job's live-term count
        jobs.append(pp.make_job(cfg, x, z, c, pp.pack_gates(gx, gz), th, len(wl.circuit.layers),
                                wl.state.bloch, True, 0))

    def run(slots, paced, subset=None):
        server = pp.pp_server_create(slots, 150 << 30, 0)
        t0 = time.perf_counter()
        ids = []
        picked = range(len(jobs)) if subset is None else subset
        for k in picked:
            (arrival, _), (job, _bufs) = specs[k], jobs[k]
            if paced:
                delay = t0 + arrival - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
            ids.append(pp.pp_submit(server, job))
        res = [pp.pp_server_wait(server, i) for i in ids]
        t1 = time.perf_counter()
        pp.pp_server_destroy(server)
        return res, t1 - t0

    def report_failures(tag, res):
        bad = [r for r in res if r["status"] != 0]
        if bad:
            hist = {}
            for r in bad:
                hist[r["status"]] = hist.get(r["status"], 0) + 1
            print(f"{tag}: {len(bad)} failed jobs, statuses {hist}; first: {bad[0]['message']}",
                  file=sys.stderr, flush=True)

    if not full:
        warm, _ = run(slots, False)  # warm-up (builds graphs, pools)
        report_failures("warm-up", warm)
    res, wall = run(slots, True)
    report_failures("timed", res)
    if check_every is None and full:
        check_every = max(1, len(jobs) // 50)
    subset = None if check_every is None else list(range(0, len(jobs), check_every))
    seq, seq_wall = run(1, False, subset)
    return res, wall, seq, seq_wall, subset


def served_max_diff(res, seq, subset):
    pairs = zip(res if subset is None else [res[k] for k in subset], seq)
    ok = [(a, b) for a, b in pairs if a["status"] == 0 and b["status"] == 0]
    return max((abs(a["value"] - b["value"]) for a, b in ok), default=None)


def served_summary(pp, n_jobs=300, rate=200.0, slots=8):
    """The serving part of the metric, measured beside the headline job: the
    scaled Poisson stream (n_jobs jobs at `rate`/s, every job well under a
    second) through pp_submit.  Jobs/s over the stream's wall time, latency
    p50/p99 from submission to result, and every result against the same
    job run alone."""
    specs = serving_specs(n_jobs, rate)
    res, wall, seq, _, subset = serve_stream(pp, specs, slots, False, check_every=5)
    lat = np.array([r["latency_ms"] for r in res])
    return {"workload": "serving_stream_scaled", "jobs": len(res), "rate_per_s": rate,
            "slots": slots,
            "sizes": "ring n in {16,32,64,128}, <= 20 steps, weight <= 8, eps >= 1e-4; "
                     "all-to-all Heisenberg n in {8,10,12,16}, <= 4 steps",
            "jobs_per_s": len(res) / wall,
            "latency_ms": {"p50": float(np.percentile(lat, 50)),
                           "p99": float(np.percentile(lat, 99)), "max": float(lat.max())},
            "failed": int(sum(r["status"] != 0 for r in res)),
            "max_abs_diff_vs_alone": served_max_diff(res, seq, subset),
            "checked_alone": len(seq),
            "timing": "host wall clock from each job's submission to its result"}


def bench_serving(args):
    import torch
    import paper_2512_12094_gb300 as pp
    torch.cuda.set_device(0)
    pp.build()
    pp.load()
    full = args.serving_full > 0
    specs = serving_specs_full(args.serving_full, args.rate) if full else \
        serving_specs(args.serving, args.rate)
    res, wall, seq, seq_wall, subset = serve_stream(pp, specs, args.slots, full)
    lat = np.array([r["latency_ms"] for r in res])
    err = served_max_diff(res, seq, subset)
    line = {"metric": "served_jobs_per_s", "value": len(res) / wall, "unit": "jobs/s",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": "serving_stream_full_sizes" if full else "serving_stream_scaled",
                       "jobs": len(res), "rate_per_s": args.rate,
                       "slots": args.slots, "budget_bytes": 150 << 30,
                       "reservations": "estimated from each observable, grown with its live terms"},
            "families": {f: sum(1 for _, wl in specs if (wl.noise_mode == 1) == (f == "a2a"))
                         for f in ("ring", "a2a")},
            "grows_total": int(sum(r["grows"] for r in res)),
            "restarts_total": int(sum(r["restarts"] for r in res)),
            "max_reserved_gb": max(r["reserved_bytes"] for r in res) / 1e9,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "max": float(lat.max())},
            "run_ms": {"p50": float(np.percentile([r["run_ms"] for r in res], 50))},
            "failed": int(sum(r["status"] != 0 for r in res)),
            "sequential_per_job": ({"jobs_per_s": len(seq) / seq_wall, "wall_s": seq_wall}
                                   if subset is None else
                                   {"jobs_checked_alone": len(seq), "wall_s": seq_wall}),
            "offered_load_wall_s": float(specs[-1][0]),
            "max_abs_diff_vs_sequential": err}
    print(json.dumps(line), flush=True)
    if args.serving_dump:
        stream = pi.serving_stream(2000, args.rate, 0) if full else None
        recs = []
        for k, ((arrival, wl), r) in enumerate(zip(specs, res)):
            rec = {"arrival_s": arrival, "n": wl.circuit.n, "layers": len(wl.circuit.layers),
                   "gates_per_layer": len(wl.circuit.layers[0]), "eps": wl.eps,
                   "group": wl.symmetry, "noise_mode": wl.noise_mode,
                   "family": "a2a" if wl.noise_mode == 1 else "ring"}
            if stream is not None:
                rec["steps"] = stream[k]["steps"]
            rec.update({key: r[key] for key in ("status", "latency_ms", "queue_ms", "run_ms",
                                                "grows", "restarts", "reserved_bytes",
                                                "device_bytes", "live_terms", "gate_updates")
                        if key in r})
            recs.append(rec)
        with open(args.serving_dump, "w") as f:
            json.dump(recs, f)


def replica_throughput(dist, ms_total, e2e_ms, upd, device):
    """Whole-job rate of N independent replicas (one per rank): the updates
    of all ranks over the slowest rank's time, for the device-timed and the
    end-to-end regions.  dist is torch.distributed (or None for one rank).
    Returns (value, e2e_value, ms_max, e2e_max, total_updates)."""
    import torch
    t = torch.tensor([ms_total, e2e_ms], dtype=torch.float64, device=device)
    u = torch.tensor([upd], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(u, op=dist.ReduceOp.SUM)
    ms_max, e2e_max, total = float(t[0]), float(t[1]), float(u[0])
    value = total / (ms_max / 1e3)
    e2e_value = total / (e2e_max / 1e3) if e2e_max > 0 else None
    return value, e2e_value, ms_max, e2e_max, total


def _timed_run(pp, make, layers, boundary=True, bloch=None):
    """Propagate through `layers` (packed gates, angles) on a fresh context
    from make(); CUDA-event time of the whole run (creation included)."""
    import torch
    stream = torch.cuda.current_stream()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    prop = make()
    for packed, th in layers:
        pp.pp_apply_layer(prop.ctx, packed, th, boundary)
    val = prop.expect(bloch) if bloch is not None else None
    t1.record(stream)
    torch.cuda.synchronize()
    st = prop.stats()
    live = prop.num_terms()[0]
    prop.close()
    return t0.elapsed_time(t1), st, live, val


def _packed_layers(pp, wl, count=None):
    """The workload's layers in application (Heisenberg) order as (packed
    gates, angles), the first `count` of them if given."""
    L = len(wl.circuit.layers)
    out = []
    for k, layer in enumerate(reversed(range(L))):
        if count is not None and k >= count:
            break
        gx, gz, th = wl.circuit.gate_arrays(layer)
        out.append((pp.pack_gates(gx, gz), th))
    return out


def _ring64_batched(pp):
    """Ring n=64 with 256 angle sets in [0, pi/2] (seed 0): (packed gates,
    angles [192, 256], x, z, single-column coefficients, rows [n, 256])."""
    n, B = 64, 256
    angles = pi.batched_ring_angles(B, 0)
    gx, gz, _ = pi.Circuit(n, [pi.ring_layer(n, 0.0, 0.0, 0.0)]).gate_arrays(0)
    th = np.zeros((3 * n, B))
    th[:n], th[n:2 * n], th[2 * n:] = angles[:, 0], angles[:, 1], angles[:, 2]
    x, z, c = pi.mean_z(n).arrays()
    return pp.pack_gates(gx, gz), th, x, z, c, np.repeat(c[:, None], B, axis=1)


def other_workloads_summary(pp):
    """The other full-size workloads through the same C ABI, measured beside
    the headline job: one warm-up run, then one run timed with CUDA events
    (context creation included).
    * all-to-all Heisenberg n=64, 10 steps (60,480 gates), per-gate damping
      p=0.01, eps 1e-5, Neel, merged under S_64;
    * ring n=64 with 256 angle sets (eps 1e-5 on any column), its first three
      steps, FP64 and FP32 rows (the table grows about tenfold per step and
      the 30 steps do not fit one GPU);
    * all-to-all XXZ n=36, eps 0.05, merged under S_36 after each of its
      first 16 XX/YY/ZZ sublayers."""
    out = {}
    wl = pi.config2_all_to_all()
    layers = _packed_layers(pp, wl)
    make = lambda: pp.Propagator.from_workload(wl, symmetry=2)  # noqa: E731
    _timed_run(pp, make, layers[:1])
    ms, st, live, val = _timed_run(pp, make, layers, bloch=wl.state.bloch)
    out["a2a64_S64_per_gate_noise_10steps"] = {
        "ms": ms, "value": st["gate_updates"] / (ms / 1e3), "unit": "updates/s",
        "gates": len(layers) * 6048, "expect": val, "live_terms": live}
    packed, th, x, z, _, rows = _ring64_batched(pp)
    for f32 in (False, True):
        make = lambda: pp.Propagator(64, x, z, rows, eps=1e-5, batch=256, f32=f32)  # noqa: E731
        _timed_run(pp, make, [(packed, th)])
        ms, st, live, _ = _timed_run(pp, make, [(packed, th)] * 3)
        out["ring64_B256_%s_3steps" % ("fp32" if f32 else "fp64")] = {
            "ms": ms, "value": st["gate_updates"] * 256 / (ms / 1e3),
            "unit": "column updates/s (live strings x gates x 256 columns)", "live_terms": live}
    wl = pi.xxz_all_to_all(36, 0.05, 6, eps=0.05, symmetry=2, split=True)
    layers = _packed_layers(pp, wl, 16)
    make = lambda: pp.Propagator.from_workload(wl, symmetry=2)  # noqa: E731
    _timed_run(pp, make, layers[:3])
    ms, st, live, val = _timed_run(pp, make, layers, bloch=wl.state.bloch)
    out["xxz36_S36_16_sublayers"] = {"ms": ms, "value": st["gate_updates"] / (ms / 1e3),
                                     "unit": "updates/s", "S2_over_S02": val, "live_terms": live}
    return out


def bench_workload(args):
    """The other workloads through the same C ABI, one JSON line each (one
    GPU; not the headline).  a2a64: all-to-all Heisenberg n=64, 10 steps,
    eps 1e-5, Neel, per-gate damping p=0.01, merged under S_64 and plain,
    and the per-layer damping variant.  batched64: ring n=64, 256 angle sets
    in [0, pi/2], eps 1e-5 any-column, the first three steps (the table grows
    about tenfold per step), FP64 and FP32 rows; columns64: the same 256
    angle sets run one column at a time.  canon64: representatives of 2^24
    random n=64 strings under Z_64, D_64 and S_64 (pp_canonical_keys).  xxz36: all-to-all XXZ n=36, dt 0.05,
    S^2/S_0^2, |+>^n, eps 0.05, merged after each of the first 16 XX/YY/ZZ
    sublayers."""
    import torch
    import paper_2512_12094_gb300 as pp
    torch.cuda.set_device(0)
    pp.build()
    pp.load()

    def packed_layers(wl, count=None):
        return _packed_layers(pp, wl, count)

    def line(name, ms, updates, extra):
        d = {"metric": "pauli_term_gate_updates_per_s", "value": updates / (ms / 1e3),
             "unit": "updates/s", "n_gpus": 1, "ms_per_run": ms, "higher_is_better": True,
             "dtype": "f64", "data": "synthetic", "config": {"workload": name}}
        d.update(extra)
        print(json.dumps(d), flush=True)

    names = args.workload.split(",")
    if "a2a64" in names:
        for label, group, mode in (("a2a64_S64_per_gate_noise", 2, 1), ("a2a64_plain_per_gate_noise", 0, 1),
                                   ("a2a64_S64_per_layer_noise", 2, 2)):
            wl = pi.config2_all_to_all()
            wl.noise_mode = mode
            layers = packed_layers(wl)
            make = lambda: pp.Propagator.from_workload(wl, symmetry=group)  # noqa: E731
            _timed_run(pp, make, layers[:1])  # warm-up
            ms, st, live, val = _timed_run(pp, make, layers, bloch=wl.state.bloch)
            line(label, ms, st["gate_updates"], {"result": {"expect": val, "live_terms": live},
                                                 "gates_per_run": len(layers) * 6048})
    if "batched64" in names or "columns64" in names:
        n, B, steps = 64, 256, 3
        packed, th, x, z, c, coef = _ring64_batched(pp)
        for f32 in ((False, True) if "batched64" in names else ()):
            make = lambda: pp.Propagator(n, x, z, coef, eps=1e-5, batch=B, f32=f32)  # noqa: E731
            _timed_run(pp, make, [(packed, th)])
            ms, st, live, _ = _timed_run(pp, make, [(packed, th)] * steps)
            line("ring64_B256_%s_3steps" % ("fp32" if f32 else "fp64"), ms, st["gate_updates"] * B,
                 {"unit_note": "column updates (live strings x gates x 256 columns)",
                  "result": {"live_terms": live}})
        # the same 256 angle sets, one single-column context each
        total_ms, total_upd = 0.0, 0.0
        for b in (range(B) if "columns64" in names else ()):
            thb = np.ascontiguousarray(th[:, b])
            make = lambda: pp.Propagator(n, x, z, c, eps=1e-5)  # noqa: E731
            if b == 0:
                _timed_run(pp, make, [(packed, thb)])
            ms, st, _, _ = _timed_run(pp, make, [(packed, thb)] * steps)
            total_ms += ms
            total_upd += st["gate_updates"]
        if "columns64" in names:
            line("ring64_256_columns_one_at_a_time_3steps", total_ms, total_upd,
                 {"unit_note": "column updates; each column truncated on its own"})
    if "canon64" in names:
        # representatives of 2^24 random n=64 strings (16 B each) and 2^23
        # random n=128 strings (32 B each), resident in HBM: 512 MB read +
        # written per call, far above L2
        hbm, kind = peaks()
        rng = np.random.default_rng(3)
        cases = []
        for m, n in ((1 << 24, 64), (1 << 23, 128)):
            W = n // 64
            keys = torch.from_numpy(rng.integers(0, 2 ** 63, size=(m, 2 * W), dtype=np.int64)).cuda()
            for label, code in (("Z", pp.SYM_ZN), ("D", pp.SYM_DN), ("S", pp.SYM_SN)):
                cases.append((m, n, keys, "%s%d" % (label, n), code))
        # 2^22 strings of weight <= 10 on 64 qubits, the shape of propagated
        # tables (mostly I): the Z_n search walks the gaps between their sites
        m = 1 << 22
        sites = rng.integers(0, 64, size=(m, 10))
        letters = rng.integers(0, 4, size=(m, 10))  # 0 leaves the site as I
        bit = np.left_shift(np.uint64(1), sites.astype(np.uint64))
        xw = np.bitwise_or.reduce(np.where((letters == 1) | (letters == 2), bit, np.uint64(0)), axis=1)
        zw = np.bitwise_or.reduce(np.where((letters == 2) | (letters == 3), bit, np.uint64(0)), axis=1)
        keys = torch.from_numpy(np.stack([xw, zw], axis=1).view(np.int64)).cuda()
        for label, code in (("Z", pp.SYM_ZN), ("S", pp.SYM_SN)):
            cases.append((m, 64, keys, "%s64w10" % label, code))
        for m, n, keys, label, code in cases:
            out = torch.empty_like(keys)
            pp.pp_canonical_keys(n, code, m, keys, out)
            torch.cuda.synchronize()
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record()
            for _ in range(5):
                pp.pp_canonical_keys(n, code, m, keys, out)
            t1.record()
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1) / 5
            gbs = 2 * 16 * (n // 64) * m / (ms / 1e3) / 1e9
            print(json.dumps({"metric": "canonical_keys_per_s", "value": m / (ms / 1e3),
                              "unit": "keys/s", "n_gpus": 1, "ms_per_call": ms,
                              "higher_is_better": True, "data": "synthetic",
                              "config": {"workload": "canonical_keys_n%d_%s_%dM"
                                         % (n, label, m >> 20)},
                              "hbm": {"achieved_gbs": gbs, "peak_gbs": hbm, "frac": gbs / hbm,
                                      "peak_kind": kind}}), flush=True)
    if "merge32" in names:
        # the Z_32 boundary merge of the ring job: the table after the gates of
        # the last layer (before its merge), merged by hash and by sort
        wl = pi.config1_ring(symmetry=1)
        layers = packed_layers(wl)
        prop = pp.Propagator.from_workload(wl, symmetry=1)
        for packed, th in layers[:-1]:
            pp.pp_apply_layer(prop.ctx, packed, th, True)
        pp.pp_apply_layer(prop.ctx, layers[-1][0], layers[-1][1], False)
        x, z, c = prop.export()
        prop.close()
        m = len(c)
        keys = torch.from_numpy(np.ascontiguousarray(np.concatenate([x, z], axis=1)).view(np.int64)).cuda()
        coef = torch.from_numpy(c).cuda()
        out_k, out_c = torch.empty_like(keys), torch.empty_like(coef)
        res = {}
        for label, fn in (("hash", pp.pp_merge_terms), ("sort", pp.pp_merge_terms_sorted)):
            for _ in range(2):
                res[label + "_distinct"] = fn(32, 1, m, keys, coef, out_k, out_c)
            t0 = torch.cuda.Event(enable_timing=True)
            t1 = torch.cuda.Event(enable_timing=True)
            t0.record()
            for _ in range(5):
                fn(32, 1, m, keys, coef, out_k, out_c)
            t1.record()
            torch.cuda.synchronize()
            res[label + "_ms"] = t0.elapsed_time(t1) / 5
        print(json.dumps({"metric": "boundary_merge_ms", "unit": "ms", "n_gpus": 1,
                          "data": "synthetic", "higher_is_better": False,
                          "config": {"workload": "ring_n32_Z32_last_boundary_merge",
                                     "input_terms": m},
                          "result": res}), flush=True)
        # the whole Z_32 job with each merge method
        for method, label in ((pp.MERGE_HASH, "hash"), (pp.MERGE_SORT, "sort")):
            make = lambda: pp.Propagator.from_workload(wl, symmetry=1, merge_method=method)  # noqa: E731
            _timed_run(pp, make, layers)
            ms = [_timed_run(pp, make, layers, bloch=wl.state.bloch) for _ in range(3)]
            line("ring_n32_Z32_job_merge_" + label, min(r[0] for r in ms), ms[0][1]["gate_updates"],
                 {"result": {"expect": ms[0][3], "live_terms": ms[0][2]},
                  "ms_all": [r[0] for r in ms]})
    if "rows64" in names:
        # batched rows (ring n=64, B = 256, 3 steps) merged by hash and by sort
        n, B, steps = 64, 256, 3
        packed, th, x, z, c, coef = _ring64_batched(pp)
        for f32 in (False, True):
            for method, label in ((pp.MERGE_HASH, "hash"), (pp.MERGE_SORT, "sort")):
                make = lambda: pp.Propagator(n, x, z, coef, symmetry=1, eps=1e-5, batch=B,  # noqa: E731
                                             f32=f32, merge_method=method)
                _timed_run(pp, make, [(packed, th)])
                ms, st, live, _ = _timed_run(pp, make, [(packed, th)] * steps)
                line("ring64_B256_%s_Z64_3steps_merge_%s" % ("fp32" if f32 else "fp64", label), ms,
                     st["gate_updates"] * B, {"unit_note": "column updates",
                                              "result": {"live_terms": live}})
    if "cadence" in names:
        # merge cadence: a symmetry merge after every k-th layer (or sublayer);
        # GPU time and table sizes, and <O> next to the oracle on the same schedule
        def sweep(wl, group, schedules, with_oracle, label):
            for every, sub in schedules:
                run = pi.split_sublayers(wl) if sub else wl
                L = len(run.circuit.layers)
                flags = pi.merge_schedule(L, every)
                layers_r = packed_layers(run)

                def job(record=False):
                    prop = pp.Propagator.from_workload(run, symmetry=group)
                    peak = 0
                    for (packed, th), f in zip(layers_r, flags):
                        pp.pp_apply_layer(prop.ctx, packed, th, f)
                        if record:
                            peak = max(peak, prop.num_terms()[0])
                    return prop, peak

                prop, peak = job(record=True)
                val = prop.expect(run.state.bloch)
                live = prop.num_terms()[0]
                prop.close()
                times = []
                for _ in range(3):
                    torch.cuda.synchronize()
                    t0 = torch.cuda.Event(enable_timing=True)
                    t1 = torch.cuda.Event(enable_timing=True)
                    t0.record()
                    prop, _ = job()
                    prop.expect(run.state.bloch)
                    t1.record()
                    torch.cuda.synchronize()
                    st = prop.stats()
                    prop.close()
                    times.append(t0.elapsed_time(t1))
                res = {"expect": val, "live_terms": live, "peak_live_terms": peak,
                       "merges": int(sum(flags))}
                if with_oracle:
                    import oracle
                    t = time.perf_counter()
                    ox, oz, oc = run.observable.arrays()
                    ost = oracle.OracleState(run.circuit.n, ox, oz, oc, group=group, eps=run.eps,
                                             max_weight=run.max_weight)
                    for layer, f in zip(reversed(range(L)), flags):
                        gx, gz, th = run.circuit.gate_arrays(layer)
                        ost.apply_layer(gx, gz, th, run.noise_mode, run.noise_p,
                                        group=group if f else 0)
                    ov = ost.expect(run.state.bloch, group)
                    res.update({"oracle_expect": ov, "abs_error_vs_oracle": abs(val - ov),
                                "oracle_s": time.perf_counter() - t})
                line("%s_merge_every_%d%s" % (label, every, "_sublayers" if sub else "_layers"),
                     min(times), st["gate_updates"], {"result": res, "ms_all": times})

        sched = [(1, False), (2, False), (4, False), (1, True), (2, True)]
        sweep(pi.config1_ring(n=32, symmetry=1), 1, sched, False, "ring32_Z32")
        sweep(pi.config1_ring(n=16, steps=10, eps=1e-4, max_weight=8, symmetry=1), 1, sched, True,
              "ring16_Z16")
        sweep(pi.xxz_all_to_all(20, 0.05, 4, eps=0.01, symmetry=2, split=True), 2,
              [(1, False), (3, False)], True, "xxz20_S20_12_sublayers")
    if "xxz36" in names:
        wl = pi.xxz_all_to_all(36, 0.05, 6, eps=0.05, symmetry=2, split=True)
        layers = packed_layers(wl, 16)
        make = lambda: pp.Propagator.from_workload(wl, symmetry=2)  # noqa: E731
        _timed_run(pp, make, layers[:3])
        ms, st, live, val = _timed_run(pp, make, layers, bloch=wl.state.bloch)
        line("xxz36_split_eps0.05_16_sublayers", ms, st["gate_updates"],
             {"result": {"S2_over_S02": val, "live_terms": live}})


def bench_reference(args):
    """The oracle as the reference arm, on the host cores (rank 0 only)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per = max(4.0, 60.0 / max(args.steps + args.warmup, 1))
    for _ in range(args.warmup):
        cpu_baseline(seconds=per)
    vals = [cpu_baseline(seconds=per) for _ in range(args.steps)]
    v = statistics.mean(x["value"] for x in vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.mean(x["seconds"] for x in vals),
            "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "step": "a bounded prefix of the job (CPU time per step fixed)"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": vals[-1]["sample"], "host": vals[-1]["host"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true",
                    help="leave out the scaled serving stream measured after the main job")
    ap.add_argument("--no-others", action="store_true",
                    help="leave out the other workloads measured after the main job")
    ap.add_argument("--only", default="both", choices=sorted(GROUPS))
    ap.add_argument("--trace-layers", action="store_true",
                    help="one JSON line per layer of the config-1 job (no timing contract)")
    ap.add_argument("--plain-share", type=float, default=0.25,
                    help="run the plain and Z_32 propagations of a job at the same time, the "
                         "plain one on this fraction of the GPU's co-resident blocks (0: one "
                         "after the other)")
    ap.add_argument("--block-threads", type=int, default=0, choices=[0, 256, 1024],
                    help="block size of the persistent layer kernel (0: the library default)")
    ap.add_argument("--serving", type=int, default=0,
                    help="serve N jobs of the scaled Poisson stream instead of the main job")
    ap.add_argument("--serving-full", type=int, default=0,
                    help="serve the first N jobs of the 2000-job stream at their stated sizes")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--slots", type=int, default=8)
    ap.add_argument("--serving-dump", default="",
                    help="with --serving/--serving-full: write every job's description and "
                         "result to this JSON file")
    ap.add_argument("--workload", default="",
                    help="comma list of a2a64, batched64, columns64, xxz36, canon64, merge32, "
                         "rows64, cadence: time those")
    ap.add_argument("--profile-layer", type=int, default=-1,
                    help="run the Z_n job once, bracketing layer K for ncu --profile-from-start off")
    args = ap.parse_args()
    if args.workload:
        bench_workload(args)
    elif args.serving > 0 or args.serving_full > 0:
        bench_serving(args)
    elif args.profile_layer >= 0:
        profile_layer(args)
    elif args.trace_layers:
        trace_layers(args)
    elif args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
