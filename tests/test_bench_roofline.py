"""bench.py's roofline arithmetic on CPU: the algorithmic bytes per kernel
family written out from the operations each family must do, the choice of
the dominant family, and the recorded-traffic lookup."""
import os
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

N, M, J = 1024, 8, 4
Q = lambda j: (N >> j) ** 2   # subband side^2 at level j


def test_analysis_level1_bytes():
    # read the gradient image (N^2), read B_k and B_k-1 and write B_k+1 over
    # the 3 detail subbands of every basis (3 x 3 M (N/2)^2), write the M
    # level-1 approximations ((N/2)^2 each): 84 bytes per pixel in FP32
    want = (N * N + 9 * M * Q(1) + M * Q(1)) * 4
    assert want == 84 * N * N
    assert bench.family_bytes("analysis_l1", N, M, J, 4, None) == want


def test_coarse_analysis_and_synthesis_bytes():
    ana = sum(M * Q(j - 1) + 9 * M * Q(j) + (M * Q(j) if j < J else 3 * M * Q(j))
              for j in range(2, J + 1)) * 8
    assert bench.family_bytes("analysis", N, M, J, 8, None) == ana
    syn = sum(3 * M * Q(j) + M * Q(j) + M * Q(j - 1) for j in range(2, J + 1)) * 4
    assert bench.family_bytes("synth", N, M, J, 4, None) == syn
    # level 1 reads all M bases' coefficients (M N^2) and writes the image
    assert bench.family_bytes("synth_l1", N, M, J, 4, None) == (M + 1) * N * N * 4


def test_spectral_step_bytes_fused_and_unfused():
    half = N * (N // 2 + 1)
    # fused: read Z, X_k-1, B (complex) and K (real), write Z and X_k
    assert bench.family_bytes("spec_mul", N, M, J, 4, None) == (2 + 2 + 2 + 1 + 2 + 2) * 4 * half
    assert bench.family_bytes("fft_r2c", N, M, J, 4, None) == N * N * 4 + half * 8
    # N not a power of two: cuFFT transforms, the unfused step reads X_k,
    # X_k-1, B, K and writes S
    n = 48
    assert bench.family_bytes("spec_mul", n, M, 3, 4, None) == 9 * 4 * n * (n // 2 + 1)
    assert bench.family_bytes("fft_r2c", n, M, 3, 4, None) is None


@pytest.mark.parametrize("n,rsz,fused", [(16, 4, True), (1024, 4, True), (8192, 4, True),
                                         (8192, 8, False), (48, 4, False), (8, 4, False)])
def test_fused_rule(n, rsz, fused):
    assert bench.fused_spectral_step(n, rsz) == fused


def test_dominant_family_and_fraction():
    # (launches, total ms) per family; the dominant family has the most time
    prof = {"synth": (10, 0.40), "analysis_l1": (10, 0.37), "fft_grid": (2, 5.0),
            "spec_mul": (10, 0.19), "fft_r2c": (10, 0.08)}
    w = types.SimpleNamespace(npix=N)
    args = types.SimpleNamespace(precision="fp32")
    r = bench.roofline_of(prof, w, None, args)
    assert r["kernel"] == "synth"   # the operator's cuFFT time is not ours
    hbm, _ = bench._peaks()
    b = bench.family_bytes("synth", N, M, J, 4, None)
    assert r["achieved"] == pytest.approx(b / (0.40 / 10 / 1e3) / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / hbm)
    assert set(r["frac_by_family"]) == {"synth", "analysis_l1", "spec_mul", "fft_r2c"}


def test_recorded_traffic_needs_matching_precision():
    assert bench.recorded_traffic("synth", "fp64") is None
    assert bench.recorded_traffic("grid", "fp32") is None   # not a per-pass family


class _FakePlan:
    """partition counts and gridding layout of a plan, without a GPU"""

    def partition_counts(self, chan=0):
        return {"L": 3000, "H": 5000, "LH": 100, "ALL": 7900}

    def partition_layout(self, part, chan=0):
        return {"L": 7, "H": 11}[part], 38 * 38, 8


def test_gridding_and_fold_bytes():
    plan = _FakePlan()
    rows = (3000 + 5000) / 2
    grid = 4 * N * N * 2 * 4
    # per row: packed cell (4 B) + two offsets + one complex value (FP32)
    assert bench.family_bytes("grid", N, M, J, 4, plan) == rows * (4 + 4 * 4) + grid
    # degridding also reads the observed value and writes the residual
    assert bench.family_bytes("degrid", N, M, J, 4, plan) == rows * (4 + 2 * 4 + 4 * 4) + grid
    # the fold reads every work item's (T + 6)^2 tile once and writes the grid
    fold = ((7 + 11) / 2) * 38 * 38 * 8 + grid
    assert bench.family_bytes("fold", N, M, J, 4, plan) == fold


def test_host_cores_reports_the_machine():
    nproc, cores = bench.host_cores()
    assert nproc == os.cpu_count() and 1 <= cores <= nproc


def test_oracle_phases_run_in_a_pinned_child(tmp_path):
    """The oracle timing child sees one BLAS thread and reports its phases
    (a tiny sample, no FISTA or 128-pixel run)."""
    import numpy as np
    import synth
    w = synth.tiny(npix=32, n_ant=8, n_dumps=6, seed=1)
    path = str(tmp_path / "s.npz")
    np.savez(path, u=w.u[0], v=w.v[0], vis=w.vis[0], npix=32, pixel_size=w.pixel_size)
    one = bench.run_oracle_phases({"data": path, "rows": 100}, 1)
    assert one["threads"] == 1 and one["grid_degrid"]["rows"] == 100
    assert one["grid_degrid"]["vis_per_s"] > 0 and one["fft_ng2_pair_ms"] > 0
    two = bench.run_oracle_phases({"data": path, "rows": 100, "pool": 2}, 2)
    assert two["grid_degrid"]["processes"] == 2 and two["grid_degrid"]["rows"] == 100
