"""Write oracle reference values of Im Sigma on the two wide-shape workloads at their full q lists.

The split tensor-core forms are held to the 1e-4 relative target against these
values on sampled k (the oracle needs minutes per workload, so the values are
stored rather than recomputed in each GPU test run).  Only the CPU oracle is
called here.

* diamond_nw8: nw = 8, two atoms, 249 Re = Rp, the stored 2000-k band-edge list,
  60^3 grid + 1e5 random q (316,000), sigma = 10 meV, T = 300 K; 8 sampled k.
* hex_nw5: nw = 5, three atoms, the hexagonal R shells, 20^3 k x 40^3 q,
  sigma = 15 meV, T = 50 K; 8 sampled k.

Run:  python tests/golden/make_wide_reference.py   (writes wide_reference.json beside it)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads as W  # noqa: E402

SAMPLES = {
    "diamond_nw8": [0, 5, 42, 611, 1024, 1333, 1777, 1999],
    "hex_nw5": [0, 17, 400, 1234, 3999, 5555, 7000, 7999],
}


def main():
    oracle.build()
    out = {}
    for name, idx in SAMPLES.items():
        wl = W.make_workload(name)
        t0 = time.time()
        ref = oracle.linewidth(wl.model, wl.k[idx], wl.q, wl.wq, wl.T, wl.EF, wl.sigma)
        print(name, f"{len(idx)} k x {len(wl.q)} q in {time.time() - t0:.0f} s", flush=True)
        out[name] = {"k_index": idx, "nq": int(len(wl.q)), "T": wl.T, "EF": wl.EF, "sigma": wl.sigma,
                     "imsigma": np.asarray(ref).tolist()}
    with open(os.path.join(HERE, "wide_reference.json"), "w") as f:
        json.dump(out, f, indent=1)


if __name__ == "__main__":
    main()
