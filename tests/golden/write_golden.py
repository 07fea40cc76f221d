"""Write the stored expected values under tests/golden/ from the CPU oracle.

Every value in the JSON files written here comes from ``oracle/`` (and the
seeded inputs of ``pp_inputs``); nothing comes from the CUDA library.

    python tests/golden/write_golden.py [--skip-merged]
"""
import argparse
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import pp_inputs as pi  # noqa: E402


def trajectory(wl, group):
    ox, oz, oc = wl.observable.arrays()
    st = oracle.OracleState(wl.circuit.n, ox, oz, oc, group=group, eps=wl.eps,
                            max_weight=wl.max_weight)
    rows = []
    t0 = time.time()
    for layer in reversed(range(len(wl.circuit.layers))):
        gx, gz, th = wl.circuit.gate_arrays(layer)
        st.apply_layer(gx, gz, th, wl.noise_mode, wl.noise_p, group=group)
        rows.append({"terms": len(st), "expect": st.expect(wl.state.bloch, group),
                     "updates": st.updates})
        print(wl.name, group, len(rows), rows[-1], "%.1fs" % (time.time() - t0), flush=True)
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--skip-merged", action="store_true")
    args = ap.parse_args()
    oracle.build()
    out = {}
    wl0 = pi.config0_heisenberg()
    out["heisenberg_a2a_n8"] = {
        "source": "oracle/oracle.cpp via oracle.OracleState; inputs pp_inputs.config0_heisenberg()",
        "plain": trajectory(wl0, 0)}
    with open(os.path.join(HERE, "heisenberg_a2a_n8.json"), "w") as f:
        json.dump(out["heisenberg_a2a_n8"], f, indent=1)

    wl1 = pi.config1_ring()
    res = {"source": "oracle/oracle.cpp via oracle.OracleState; inputs pp_inputs.config1_ring()",
           "plain": trajectory(wl1, 0)}
    with open(os.path.join(HERE, "ring_n32.json"), "w") as f:
        json.dump(res, f, indent=1)
    if not args.skip_merged:
        res["zn"] = trajectory(wl1, 1)
        with open(os.path.join(HERE, "ring_n32.json"), "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    main()
