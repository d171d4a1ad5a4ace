"""bench.py's JSON contract on the CPU: the reference arm (the float64 oracle
on a bounded sample of the full-size workload) prints one JSON line with the
metric, unit and config of the GPU arm, a cpu_baseline description and an e2e
object with no host<->device traffic; and the nominal LM flop count and the
traffic table of the GPU arm are well formed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0"], capture_output=True, text=True,
                         timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    assert d["impl"] == "reference"
    assert d["metric"] == bench.METRIC and d["unit"] == "iter/s"
    assert d["higher_is_better"] is True and d["n_gpus"] == 1 and d["steps"] == 1
    assert d["value"] > 0 and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"] == {"value": d["value"], "unit": "iter/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}
    assert d["config"]["workload"] == bench.WORKLOAD


def test_gpu_arm_tables_well_formed():
    import bench
    # one model + Jacobian evaluation per frame and step, solve and Huber terms
    assert 2000 < bench.LM_FLOPS_PER_VOXEL_STEP < 3000
    for name, t in bench.TRAFFIC.items():
        assert t["src"] in ("projector.cu", "kinetics.cu") and len(t["sha"]) == 16
        got = bench._traffic(name)
        # None only when the kernel source changed since the counters were taken
        assert got is None or got > 1.0, name


def test_joseph_nonzero_count_matches_oracle_matrix():
    """The bench's count of Joseph-matrix nonzeros (the frame vectors the
    projectors move through the SM data path) equals the number of stored
    entries of the oracle's system matrix, over all angles, for bins equal to
    and finer than the voxels."""
    from types import SimpleNamespace

    import bench
    from oracle import projector as OP
    for n_bins, bin_mm, n_angles, n_subsets in ((40, 2.0, 36, 4), (48, 1.7, 30, 5)):
        W = SimpleNamespace(nx=32, ny=28, vox_mm=2.0, n_bins=n_bins, bin_mm=bin_mm,
                            n_angles=n_angles, n_subsets=n_subsets)
        nnz = OP.system_matrix(W.nx, W.ny, W.vox_mm, n_bins, n_angles, bin_mm).nnz
        got = bench.joseph_nnz_per_subset(W) * n_subsets
        print(f"bins {n_bins} x {bin_mm} mm: bench {got:.0f}, oracle {nnz}")
        assert abs(got - nnz) <= 1e-3 * nnz
