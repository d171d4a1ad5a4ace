"""Write pr1_chaos_envelope.json: how far the FP64 oracle's own 5-iteration ICM
on config PR1 moves when the count calibration kappa is perturbed by 1e-5
(relative), and when its image and ratio are stored in bfloat16 / float16.  ICM with MAP-LM is sensitive to perturbations of the data (LM
decisions at the edge of a decrease, voxels switching between local minima),
so an end-to-end float32 run is compared with this envelope.  Calls only the
oracle.  Run from the repository root: python tests/golden/make_pr1_chaos_envelope.py
"""
import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import kcs_synth as S  # noqa: E402
from oracle import icm as OI  # noqa: E402
from oracle import osl as OO  # noqa: E402
from cases import pr1_problem, rel_l2  # noqa: E402

EPS = 1e-5


def main():
    P = pr1_problem()
    kappa = float(np.float32(P["kappa"]))
    a = OI.icm(P["g"], P["counts"], kappa, P["ts"], P["te"], S.FENG, 5, 10, 0.1, 0.1, 0.01)
    b = OI.icm(P["g"], P["counts"], kappa * (1 + EPS), P["ts"], P["te"], S.FENG, 5, 10,
               0.1, 0.1, 0.01)

    def ll(x):
        return OO.loglik(P["g"], x, P["counts"], kappa, P["dt"])

    out = {"perturbation": f"kappa x (1 + {EPS:g})", "iterations": 5, "n_lm": 10,
           "image_rel_l2": rel_l2(b[0], a[0]), "model_tac_rel_l2": rel_l2(b[3], a[3]),
           "loglik_rel": abs(ll(b[0]) / ll(a[0]) - 1)}
    # The same oracle run with the image and ratio stored on the bfloat16 /
    # float16 grid (per-frame scale = max of the start image): how far storage
    # rounding alone moves the ICM trajectory.
    lab = S.labels_pr1()
    inside = lab > 0
    # (the maximum over three stored runs with kappa x (1, 1 + EPS, 1 - EPS): a
    # chaotic quantity needs more than one sample to bound)
    out["storage"] = {}
    for kind in ("bf16", "f16"):
        worst = {}
        for f in (1.0, 1 + EPS, 1 - EPS):
            c = OI.icm(P["g"], P["counts"], kappa * f, P["ts"], P["te"], S.FENG, 5, 10, 0.1, 0.1,
                       0.01, storage=kind)
            m = {"image_rel_l2": rel_l2(c[0], a[0]), "model_tac_rel_l2": rel_l2(c[3], a[3]),
                 "K1_rel_l2": rel_l2(c[1][0, 0][inside], a[1][0, 0][inside]),
                 "k3_rel_l2": rel_l2(c[1][2, 0][inside], a[1][2, 0][inside]),
                 "Ki_rel_l2": rel_l2(c[2][0][inside], a[2][0][inside]),
                 "Ki_class_mean_rel": float(max(
                     abs(c[2][0][lab == k].mean() / a[2][0][lab == k].mean() - 1)
                     for k in (1, 2, 3)))}
            worst = {k: max(v, worst.get(k, 0.0)) for k, v in m.items()}
        out["storage"][kind] = worst
    # the same sensitivity for the other two methods of Sec. IV-A
    # (maximum over kappa x (1 + EPS) and kappa x (1 - EPS))
    out["methods"] = {}
    for method in ("direct", "indirect"):
        c = OI.icm(P["g"], P["counts"], kappa, P["ts"], P["te"], S.FENG, 5, 10, 0.1, 0.1, 0.01,
                   method=method)
        worst = {}
        for f in (1 + EPS, 1 - EPS):
            d = OI.icm(P["g"], P["counts"], kappa * f, P["ts"], P["te"], S.FENG, 5, 10,
                       0.1, 0.1, 0.01, method=method)
            m = {"image_rel_l2": rel_l2(d[0], c[0]), "model_tac_rel_l2": rel_l2(d[3], c[3]),
                 "loglik_rel": abs(ll(d[0]) / ll(c[0]) - 1),
                 "Ki_class_mean_rel": float(max(
                     abs(d[2][0][lab == k].mean() / c[2][0][lab == k].mean() - 1)
                     for k in (1, 2, 3)))}
            worst = {k: max(v, worst.get(k, 0.0)) for k, v in m.items()}
        out["methods"][method] = worst
    with open(os.path.join(HERE, "pr1_chaos_envelope.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
