"""Write pr1_chaos_envelope.json: how far the FP64 oracle's own 5-iteration ICM
(10 MAP-LM steps each) on config PR1 moves under small perturbations, the
yardstick of the end-to-end GPU tests.  Calls only the oracle.  Run from the
repository root:  python tests/golden/make_pr1_chaos_envelope.py

Sections:
  "stable", "stable_direct"  KCS and DIRECT at the weights where the
      alternation is stable at PR1's count level (beta_kp = 0.01, beta_h = 1e4,
      delta = 0.01): the largest change of the image series, the model TACs,
      the maps, the log-likelihood and the share of voxels whose maps leave the
      1e-3 band, when the count calibration kappa is multiplied by 1 +- 1e-6
      and 1 +- 1e-5.
  "storage"  the same KCS run with the image series and each subset's ratio
      stored on the bfloat16 / float16 grid (per-frame scale = max of the start
      image): its distance from the float64 run (what storage rounding alone
      does to the trajectory) and, as "sensitivity", its own largest change
      under kappa x (1 +- 1e-5).
  "unstable"  KCS at beta_kp = 0.1, beta_h = 0.1 (the weights of the config
      text): the change under kappa x (1 + 1e-5), recorded to show that no
      end-to-end tolerance is meaningful there.
"""
import json
import os
import sys
from concurrent.futures import ProcessPoolExecutor

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

STABLE = dict(beta_kp=0.01, beta_h=1e4, delta=0.01)
UNSTABLE = dict(beta_kp=0.1, beta_h=0.1, delta=0.01)
FLOOR = 1e-2 * np.array([0.06, 0.10, 0.04, 0.03])[:, None, None, None]


def _run(job):
    """One oracle ICM run: (weights, method, kappa factor, storage)."""
    import kcs_synth as S
    from oracle import icm as OI
    from cases import pr1_problem
    w, method, f, storage = job
    P = pr1_problem()
    kappa = float(np.float32(P["kappa"]))
    return OI.icm(P["g"], P["counts"], kappa * f, P["ts"], P["te"], S.FENG, 5, 10, w["beta_kp"],
                  w["beta_h"], w["delta"], method=method, storage=storage)


def _compare(a, b, ll, inside, lab):
    off = np.any(np.abs(b[1] - a[1]) > 1e-3 * np.maximum(np.abs(a[1]), FLOOR), axis=0)
    from cases import rel_l2
    return {"image_rel_l2": rel_l2(b[0], a[0]), "model_tac_rel_l2": rel_l2(b[3], a[3]),
            "maps_rel_l2": rel_l2(b[1], a[1]), "loglik_rel": abs(ll(b[0]) / ll(a[0]) - 1),
            "map_voxels_outside_1e-3": float(off.mean()),
            "K1_rel_l2": rel_l2(b[1][0, 0][inside], a[1][0, 0][inside]),
            "k3_rel_l2": rel_l2(b[1][2, 0][inside], a[1][2, 0][inside]),
            "Ki_rel_l2": rel_l2(b[2][0][inside], a[2][0][inside]),
            "Ki_class_mean_rel": float(max(abs(b[2][0][lab == k].mean() / a[2][0][lab == k].mean()
                                               - 1) for k in (1, 2, 3)))}


def _worst(ms):
    out = {}
    for m in ms:
        out = {k: max(v, out.get(k, 0.0)) for k, v in m.items()}
    return out


def main():
    import kcs_synth as S
    from oracle import osl as OO
    from cases import pr1_problem
    P = pr1_problem()
    kappa = float(np.float32(P["kappa"]))
    lab = S.labels_pr1()
    inside = lab > 0

    def ll(x):
        return OO.loglik(P["g"], x, P["counts"], kappa, P["dt"])

    jobs = {}
    for method in ("kcs", "direct"):
        jobs[(method, 1.0)] = (STABLE, method, 1.0, None)
        for eps in (1e-6, 1e-5):
            for f in (1 + eps, 1 - eps):
                jobs[(method, f)] = (STABLE, method, f, None)
    for kind in ("bf16", "f16"):
        for f in (1.0, 1 + 1e-5, 1 - 1e-5):
            jobs[(kind, f)] = (STABLE, "kcs", f, kind)
    jobs[("unstable", 1.0)] = (UNSTABLE, "kcs", 1.0, None)
    jobs[("unstable", 1 + 1e-5)] = (UNSTABLE, "kcs", 1 + 1e-5, None)
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    with ProcessPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 1)) as ex:
        res = dict(zip(jobs, ex.map(_run, jobs.values())))

    def cmp(a, b):
        return _compare(res[a], res[b], ll, inside, lab)

    out = {"iterations": 5, "n_lm": 10}
    for method, name in (("kcs", "stable"), ("direct", "stable_direct")):
        sec = {"weights": STABLE, "method": method}
        for eps in (1e-6, 1e-5):
            sec[f"kappa_rel_{eps:g}"] = _worst([cmp((method, 1.0), (method, f))
                                               for f in (1 + eps, 1 - eps)])
        out[name] = sec
    out["storage"] = {"weights": STABLE}
    for kind in ("bf16", "f16"):
        out["storage"][kind] = {
            "vs_float64": cmp(("kcs", 1.0), (kind, 1.0)),
            "sensitivity": _worst([cmp((kind, 1.0), (kind, f)) for f in (1 + 1e-5, 1 - 1e-5)])}
    out["unstable"] = dict(cmp(("unstable", 1.0), ("unstable", 1 + 1e-5)), weights=UNSTABLE,
                           perturbation="kappa x (1 + 1e-5)")
    with open(os.path.join(HERE, "pr1_chaos_envelope.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    main()
