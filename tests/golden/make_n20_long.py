"""Write the stored oracle results for the n = 20 configuration's long schedules
(T = 40 and T = 160 at dt = 0.05: 800 and 3200 Strang steps), which the
complex128 oracle needs tens of minutes to produce.

Calls only ``oracle`` and ``satgen``: planted n = 20 instance ``planted_n20_s0``,
uniform start, linear schedule s_k = (k + 1/2)/K.  Stores the normalised
ground-state probability, the norm, <H_P>, <H_B> and the amplitudes at 256
seeded indices plus the planted solution.  Run from the repository root:

    python tests/golden/make_n20_long.py
"""

import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import satgen  # noqa: E402

N, DT = 20, 0.05


def main():
    inst = satgen.load_instance("planted_n20_s0")
    cl = inst["clauses"]
    e = oracle.violated_counts(N, cl)
    sol = int(np.flatnonzero(e == 0)[0])
    idx = np.sort(np.random.default_rng(2011).choice(1 << N, size=256, replace=False))
    idx = np.unique(np.append(idx, sol))
    for T in (40.0, 160.0):
        K = int(round(T / DT))
        psi = oracle.evolve_strang(N, cl, T, K, energies=e)
        out = {
            "source": "oracle.evolve_strang (complex128), planted_n20_s0, uniform start, s_k = (k + 1/2)/K",
            "n": N, "T": T, "steps": K, "dt": DT,
            "norm": float(oracle.norm(psi)),
            "success_prob": float(oracle.success_prob(psi, e)),
            "expect_hp": float(oracle.expect_hp(psi, e)),
            "expect_hb": float(oracle.expect_hb(N, psi)),
            "solution": sol,
            "indices": [int(i) for i in idx],
            "amplitudes": [[float(psi[i].real), float(psi[i].imag)] for i in idx],
        }
        path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"n20_T{int(T)}.json")
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(path, out["success_prob"], flush=True)


if __name__ == "__main__":
    main()
