"""Writes multi_charge_sphere_oracle.json: the FP64 oracle's dense-LU solution
of the 20-charge sphere (icosphere level 5, radius 10 A, 10,242 vertices) for
the cases of Table 1 that the sphere workload runs, under quadrature plan D0.

Only the oracle runs here (dense assembly, dense preconditioned LU). Stored per
case: Delta G (paper units and kcal/mol), the M-norms of the interior traces
and the traces at 64 seeded vertices, which the GPU tests compare with. For
the cases in TRACE_CASES the whole interior traces (u_int, v_int at every
vertex) go to multi_charge_sphere_traces.npz, so that the GPU tests can take
the M-norm of the difference itself.

    python tests/golden/make_sphere_oracle.py           # ~30 min on 8 cores, ~25 GB
    python tests/golden/make_sphere_oracle.py --traces  # only the npz (TRACE_CASES)
"""
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from oracle import oracle as O  # noqa: E402
from oracle.closed_forms import kirkwood_energy  # noqa: E402
from synth import multi_charge_sphere  # noqa: E402

CASES = (2, 10, 12, 13, 14, 15, 19, 20, 23)
TRACE_CASES = (2, 10, 20)
SAMPLE_SEED = 11
N_SAMPLE = 64


def traces(out=os.path.join(HERE, "multi_charge_sphere_traces.npz")):
    """Full interior traces of the TRACE_CASES solutions (dense LU)."""
    phys = O.Physics()
    v, t, xq, q = multi_charge_sphere()
    t0 = time.time()
    ops = oracle.assemble(v, t, phys.kappa)
    print(f"assembled {len(v)} vertices in {time.time() - t0:.0f} s", flush=True)
    arrays = {}
    for case in TRACE_CASES:
        t1 = time.time()
        r = O.solve(v, t, xq, q, phys, case=case, ops=ops)
        u, w = O.interior_traces(O.CASES[case][0], r.x, phys)
        arrays[f"u_int_{case}"] = u
        arrays[f"v_int_{case}"] = w
        arrays[f"dG_kcal_{case}"] = np.array(r.dG_kcal)
        print(f"case {case}: dG {r.dG_kcal:.8f} kcal/mol ({time.time() - t1:.0f} s)", flush=True)
    np.savez_compressed(out, **arrays)


def main(out=os.path.join(HERE, "multi_charge_sphere_oracle.json")):
    phys = O.Physics()
    v, t, xq, q = multi_charge_sphere()
    t0 = time.time()
    ops = oracle.assemble(v, t, phys.kappa)
    print(f"assembled {len(v)} vertices in {time.time() - t0:.0f} s", flush=True)
    idx = np.sort(np.random.default_rng(SAMPLE_SEED).choice(len(v), size=N_SAMPLE, replace=False))
    res = {
        "_doc": "FP64 oracle (dense assembly, dense LU of the preconditioned system) on the multi-charge sphere; "
                "written by make_sphere_oracle.py, which calls only oracle/ and synth/.",
        "workload": "icosphere level 5, radius 10 A, 20 charges uniform in r <= 8 A (seed 2), q ~ U[-1, 1] e",
        "physics": {"eps_int": phys.eps_int, "eps_ext": phys.eps_ext, "kappa": phys.kappa},
        "plan": "far 6-point degree-4 rule; singular maps with 4 Gauss points per dimension",
        "n_verts": int(len(v)), "n_tris": int(len(t)),
        "kirkwood_series_dG_paper": float(kirkwood_energy(10.0, xq, q, phys.eps_int, phys.eps_ext, phys.kappa)),
        "sample_vertices": idx.tolist(),
        "cases": {},
    }
    for case in CASES:
        t1 = time.time()
        r = O.solve(v, t, xq, q, phys, case=case, ops=ops)
        form = O.CASES[case][0]
        u, w = O.interior_traces(form, r.x, phys)
        res["cases"][str(case)] = {
            "form": form, "precond": O.CASES[case][1],
            "dG_paper": r.dG, "dG_kcal": r.dG_kcal,
            "u_int_M_norm": float(np.sqrt(u @ ops.M @ u)), "v_int_M_norm": float(np.sqrt(w @ ops.M @ w)),
            "u_int_sample": u[idx].tolist(), "v_int_sample": w[idx].tolist(),
        }
        print(f"case {case}: dG {r.dG_kcal:.8f} kcal/mol ({time.time() - t1:.0f} s)", flush=True)
        with open(out, "w") as f:
            json.dump(res, f, indent=1)


if __name__ == "__main__":
    if "--traces" in sys.argv:
        traces()
    else:
        main()
