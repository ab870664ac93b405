"""Writes c2_32x6_oracle.txt beside this script: the FP64 oracle's whole
decomposition of the 32^6 benchmark tensor (synth config c2_32x6: ranks
(1, 8, 16, 16, 16, 8, 1), 200 multiplicative-update iterations per stage from
the counter-RNG initial factors) and its Eq. (3) relative error.

Calls only oracle/ and synth/.  Run from the repository root:

    python tests/golden/make_c2_32x6_oracle.py

(about a quarter of an hour on 8 host cores and 30 GB of host memory).
"""

import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synth  # noqa: E402


def main():
    c = synth.CONFIGS["c2_32x6"]
    t0 = time.time()
    A, _ = synth.tt_tensor(c["dims"], c["ranks"], c["core_dist"], c["noise"], c["data_seed"])
    cores, finals = oracle.ntt_decompose(A.astype(np.float64), c["ranks"], c["iters"], seed=c["init_seed"],
                                         record=False)
    eps = oracle.rel_error(A, cores)
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c2_32x6_oracle.txt")
    with open(out, "w") as f:
        f.write("# FP64 oracle (oracle.ntt_decompose, record=False) on synth config c2_32x6:\n")
        f.write("# 32^6 tensor, ranks (1,8,16,16,16,8,1), 200 MU iterations per stage, init seed 102.\n")
        f.write("# Written by tests/golden/make_c2_32x6_oracle.py; Eq. (3) relative error, then the\n")
        f.write("# final objective 1/2 ||X_l - W_l H_l||^2 of every stage.\n")
        f.write(f"rel_error {eps!r}\n")
        for s, v in enumerate(finals):
            f.write(f"stage_objective {s} {float(np.ravel(v)[-1])!r}\n")
    print(f"rel error {eps:.8f} in {time.time() - t0:.0f} s -> {out}")


if __name__ == "__main__":
    main()
