"""Writes tests/golden/oracle_200bus.json from the CPU oracle only.

Run:  python tests/golden/make_golden.py
The fixture pins the oracle's outputs on the 200-bus synthetic case (seed
200) so that any later change to the oracle's arithmetic shows up as a
regression; it is never produced from the CUDA path.
"""
import hashlib
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import gridgen  # noqa: E402
import oracle  # noqa: E402


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def main():
    s = gridgen.grid_200()
    out = {"case": "gridgen.grid_200(seed=200)", "modes": {}}
    for mode, name in ((oracle.REDUCED, "reduced"), (oracle.EXTENDED, "extended")):
        ext = mode == oracle.EXTENDED
        rec = {"states": []}
        for k in range(6):
            x = gridgen.flat_state(s, ext) if k == 0 else gridgen.perturbed_state(s, k, ext)
            F = oracle.residual(s, x, mode)
            rp, ci, jv = oracle.jacobian(s, x, mode)
            if k == 0:
                rec["n_rows"] = int(F.shape[0])
                rec["nnz"] = int(rp[-1])
                rec["rowptr_sha256"] = sha(rp.astype(np.int32))
                rec["colind_sha256"] = sha(ci.astype(np.int32))
            rec["states"].append({
                "state": "flat" if k == 0 else f"perturbed seed {k}",
                "F_every_17th": [float(v) for v in F[::17]],
                "J_every_97th": [float(v) for v in jv[::97]],
                "F_inf": float(np.abs(F).max()),
                "J_abs_sum": float(np.abs(jv).sum()),
            })
        out["modes"][name] = rec
    xs, hist = oracle.newton_dense(s, gridgen.flat_state(s))
    out["newton_reduced_flat"] = {"iterations": len(hist) - 1, "final_inf": hist[-1],
                                  "V_min": float(xs[s.n_bus:].min())}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_200bus.json")
    with open(path, "w") as fh:
        json.dump(out, fh, indent=1)
    print("wrote", path)


if __name__ == "__main__":
    main()
