"""Small runs of every workload family through the C ABI, saved to an .npz file: tally batches
(int64 fixed point, so the result does not depend on the order of the atomics) and counters.  Run
by test_gpu_checked.py twice, once with MCGB_CHECKED=1 (the bounds-checked library) and once
without, in child processes so that each loads its own library.

    python tests/checked_cases.py OUT.npz
"""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

from paper_2305_07636_gb300 import mc  # noqa: E402
from paper_2305_07636_gb300 import problems as P  # noqa: E402


def largest_lattice():
    prob = P.lattice_absorber_3d(n=64, nz=16, pitch=0.1, pitch_z=0.5, radius=0.035, point=(3.2, 3.2, 4.0))
    for m in prob["materials"]:
        m["sigma_s"] = [[0.6 * m["sigma_t"][0]]]
    return prob


def cases():
    """(name, problem, histories, run options); every option set is one code path."""
    return [
        ("config1", P.config1(), 200_000, {}),
        ("config1_history", P.config1(), 200_000, {"algorithm": "history"}),
        ("config2", P.config2(), 200_000, {}),
        ("config2_fp64", P.config2(), 20_000, {"precision": "fp64"}),
        ("config2_crossing", P.config2_crossing(), 200_000, {}),
        ("config2_implicit", P.config2(), 100_000, {"implicit_capture": 1}),
        ("config3", P.config3(), 100_000, {}),
        ("azurv1_pc", P.azurv1(t_end=10.0, n_tbins=10), 100_000, {"census_times": [2.5, 5.0, 7.5]}),
        ("axial_lattice", P.axial_lattice(), 50_000, {}),
        ("dogleg", P.dogleg_duct(), 100_000, {}),
        ("quadrics", P.quadric_assembly(), 100_000, {}),
        ("largest_lattice", largest_lattice(), 20_000, {}),
        ("ww_stack", P.slab_stack(thickness=8.0, n_layers=4, detector=2.0, ww_bin=1.0, name="thin"), 50_000,
         {"ww_enable": 1, "bank_capacity": 1 << 22}),  # room enough that no split is ever held
    ]


def main(out):
    res = {}
    for name, prob, n, opts in cases():
        p = mc.Problem(prob)
        if opts.get("ww_enable"):
            p.set_weight_windows(P.exponential_ww(prob, decay=0.8))
        p.run(n, 5, **opts)
        c = p.counters()
        c.pop("iterations")
        res[name + "/tally"] = p.tally_batches(0)
        res[name + "/counters"] = np.array([c[k] for k in sorted(c)], dtype=np.int64)
        p.close()
    # k-eigenvalue cycles
    p = mc.Problem(P.pin_cell())
    k, sites, km, _ = p.run_eigen(20_000, 2, 3, 6)
    res["eigen/k"] = k
    res["eigen/sites"] = sites.astype(np.int64)
    p.close()
    # the batched launch over a few uneven problems
    probs, nh = P.config5()
    probs, nh = probs[:: 32], [min(int(h), 30_000) for h in nh[:: 32]]
    ps = [mc.Problem(q) for q in probs]
    mc.run_batch([q.h for q in ps], nh, 7)
    for i, q in enumerate(ps):
        res[f"batch{i}/tally"] = q.tally_batches(0)
        q.close()
    np.savez(out, **res)


if __name__ == "__main__":
    main(sys.argv[1])
