"""Write oracle reference samples for the full-size parity tests.

Calls only ``oracle/`` and ``synth`` (no CUDA path).  For each workload it
runs the FP64 oracle for the stated number of iterations and stores the
Frobenius norm of the reconstructed image and its values at seeded sample
positions, so a GPU test can compare the same entries without rerunning a
multi-minute oracle.

Usage: python tests/golden/make_golden.py [workload ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import synth  # noqa: E402
from oracle import admm  # noqa: E402

N_SAMPLES = 4096
RUNS = {"shlr_12c_256": 30, "shlrv_12c_256": 30, "shlrvp_8c_192_8e": 30, "unrolled_03": 10, "unrolled_11": 10}


def make(name, n_iter):
    wl = synth.unrolled_instance(name) if name.startswith("unrolled_") else synth.get_config(name)
    inp = synth.make_inputs(wl)
    t0 = time.time()
    if wl.model in ("SHLR", "SHLR_V", "SHLR_S", "SHLR_SV"):
        X, K, rels = admm.shlr(inp["Y"], inp["mask"], wl, n_iter=n_iter)
    else:
        X, K, iters = admm.shlr_p(inp["Y"], inp["mask"], wl, n_iter=n_iter)
        rels = []
    rng = np.random.default_rng(12345)
    idx = np.sort(rng.choice(X.size, N_SAMPLES, replace=False))
    out = os.path.join(HERE, f"{name}_{n_iter}it.npz")
    np.savez_compressed(out, idx=idx, values=X.ravel()[idx], norm=np.linalg.norm(X), n_iter=n_iter,
                        rels=np.asarray(rels), workload=name, seconds=time.time() - t0)
    print(out, f"{time.time() - t0:.1f}s")


if __name__ == "__main__":
    names = sys.argv[1:] or list(RUNS)
    for nm in names:
        make(nm, RUNS[nm])
