"""Host-side logic that needs no GPU: the benchmark's traffic record lookup and the input
generators the multi-right-hand-side solves use."""
import os
import shutil

import numpy as np

from conftest import ROOT


def test_traffic_record_is_used_only_for_the_kernel_sources_it_was_taken_on(tmp_path, monkeypatch):
    """bench.py reports a committed ncu traffic figure only while the pass kernels' sources hash to
    the value recorded beside it; a record for other sources reads as missing."""
    import bench
    src = os.path.join(ROOT, "profiles", "kf_r2r_cols_fp32_compact_n4096.txt")
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    shutil.copytree(os.path.join(ROOT, "paper_2107_03958_gb300", "csrc"), root / "paper_2107_03958_gb300" / "csrc")
    shutil.copy(src, root / "profiles" / "rec.txt")
    monkeypatch.setattr(bench, "ROOT", str(root))
    text = open(src).read()
    recorded = float(next(l.split(":", 1)[1] for l in text.splitlines() if l.startswith("traffic_bytes_per_launch")))
    current = bench.kernel_source_hash()
    # the copy hashes like the repository's sources
    (root / "profiles" / "rec.txt").write_text(
        "\n".join(("kernel_source_hash: " + current) if l.startswith("kernel_source_hash") else l
                  for l in text.splitlines()))
    assert bench.recorded_traffic("rec.txt") == recorded
    # a changed pass-kernel source voids it
    with open(root / "paper_2107_03958_gb300" / "csrc" / "fft_engine.cuh", "a") as f:
        f.write("\n// changed\n")
    assert bench.kernel_source_hash() != current
    assert bench.recorded_traffic("rec.txt") is None
    # a host-only source (the LS solver) does not
    with open(root / "paper_2107_03958_gb300" / "csrc" / "fft_engine.cuh", "w") as f:
        f.write(open(os.path.join(ROOT, "paper_2107_03958_gb300", "csrc", "fft_engine.cuh")).read())
    with open(root / "paper_2107_03958_gb300" / "csrc" / "ls.cu", "a") as f:
        f.write("\n// changed\n")
    assert bench.kernel_source_hash() == current
    assert bench.recorded_traffic("rec.txt") == recorded
    assert bench.recorded_traffic("absent.txt") is None


def test_plane_wave_directions():
    from paper_2107_03958_gb300 import inputs
    n, kappa = 32, 7.0
    X1, X2 = inputs.grid(n)
    w0 = inputs.plane_wave(n, kappa)
    assert np.allclose(w0, np.exp(1j * kappa * X1))
    assert np.allclose(inputs.plane_wave(n, kappa, 0.0), w0)
    w90 = inputs.plane_wave(n, kappa, np.pi / 2)
    assert np.allclose(w90, np.exp(1j * kappa * X2), atol=1e-12)
    w = inputs.plane_wave(n, kappa, 0.7)
    assert np.allclose(np.abs(w), 1.0)
    # the phase advances by kappa along the unit direction (cos 0.7, sin 0.7)
    h = 1.0 / n
    assert np.allclose(w[1:, :] / w[:-1, :], np.exp(1j * kappa * h * np.cos(0.7)))


def test_fault_injection_arguments_are_checked():
    """conv_fault_inject arms host-side faults only for the known kinds and non-negative counts
    (the call touches no device)."""
    from paper_2107_03958_gb300 import _native as N
    from paper_2107_03958_gb300 import build
    build.build()
    lib = N.load()
    assert lib.conv_fault_inject(99, 1) == 1
    assert lib.conv_fault_inject(N.FAULT["alloc"], -1) == 1
    for k in N.FAULT.values():
        assert lib.conv_fault_inject(k, 0) == 0


def test_committed_traffic_records_match_the_current_kernels():
    """The dominant kernels' traffic records in profiles/ were taken on the current pass-kernel
    sources (so the benchmark reports them), and each record's algorithmic bytes are the column
    pass's byte model: read and write the batch's n x (L/2 + 1) spectra, read the multiplier
    quadrant once."""
    import types
    import bench
    for prec, esz in (("fp64", 16), ("fp32", 8)):
        name = "kf_r2r_cols_%s_compact_n4096.txt" % prec
        assert bench.recorded_traffic(name) is not None, name
        text = open(os.path.join(ROOT, "profiles", name)).read()
        alg = int(next(l.split(":", 1)[1] for l in text.splitlines() if l.startswith("algorithmic_bytes_per_launch")))
        n, L, B = 4096, 8192, 16
        h = L // 2 + 1
        assert alg == B * 2 * h * n * esz + h * h * (esz // 2)
        fake = types.SimpleNamespace(n=n, precision=prec, info=types.SimpleNamespace(transform_len=L))
        assert bench.r2r_bytes(fake, B) == alg


def test_period3_schedule_bytes():
    """The effective-bandwidth view: FP32 65 n^2 per R2R convolution and 102 n^2 per Helmholtz
    one; the column pass 24 n^2 per density plus a 9 n^2 quadrant per launch; FP64 twice."""
    import bench
    n, B = 4096, 16
    v32 = bench.period3_view(n, B, "fp32", col_ms=1.0, step_ms=1.0, hbm=1000.0)
    v64 = bench.period3_view(n, B, "fp64", col_ms=1.0, step_ms=1.0, hbm=1000.0)
    nn = n * n
    assert v32["col_bytes_per_launch"] == (24 * B + 9) * nn
    assert v32["step_bytes"] == B * (4 * 65 + 102) * nn
    assert v64["step_bytes"] == 2 * v32["step_bytes"]
    assert abs(v32["col_gbs"] - v32["col_bytes_per_launch"] / 1e-3 / 1e9) < 1e-6
    assert abs(v32["step_frac"] - v32["step_gbs"] / 1000.0) < 1e-12
