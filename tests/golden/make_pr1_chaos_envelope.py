"""Write pr1_chaos_envelope.json: how far the FP64 oracle's own 5-iteration ICM
on config PR1 moves when the count calibration kappa is perturbed by 1e-5
(relative).  ICM with MAP-LM is sensitive to perturbations of the data (LM
decisions at the edge of a decrease, voxels switching between local minima),
so an end-to-end float32 run is judged against this envelope.  Calls only the
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
    with open(os.path.join(HERE, "pr1_chaos_envelope.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(out)


if __name__ == "__main__":
    main()
