"""Host-side pieces of bench.py, on the CPU: the algorithmic-bytes model of
each kernel (against the counts of the 64^3 bench problem: m = 230,400 rays,
N = 64^3 voxels, nnz = 19,477,604) and the digest that keys the captured
traffic to the kernel code."""
import pytest

import bench

M, N, NNZ = 230_400, 64 ** 3, 19_477_604


def test_plain_kernel_bytes():
    f, b = bench.plain_launch_bytes(M, N, NNZ, "fp32")
    # forward: 8 B per entry, 8 B per row pointer, x gathered once, b read, r written
    assert f == 8 * NNZ + 8 * (M + 1) + 4 * N + 8 * M
    assert b == 8 * NNZ + 8 * (N + 1) + 4 * M + 8 * N
    assert round(f / 1e6, 1) == 160.6 and round(b / 1e6, 1) == 160.9
    f16, b16 = bench.plain_launch_bytes(M, N, NNZ, "bf16")
    # bfloat16 values: 2 B less per entry, plus the row scale and the scaled residual
    assert f - f16 == 2 * NNZ - 8 * M and b - b16 == 2 * NNZ


@pytest.mark.parametrize("method,bwd,fwd", [("gpbb", 169.3, 173.0), ("upn", 167.2, 171.7),
                                            ("gp", 167.2, 166.8)])
def test_solver_kernel_bytes(method, bwd, fwd):
    b, f = bench.solver_launch_bytes(M, N, NNZ, "fp32", method)
    assert (round(b / 1e6, 1), round(f / 1e6, 1)) == (bwd, fwd)


def test_kernel_digest_ignores_comments_but_not_code(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    (tmp_path / "k.cu").write_text("int f(int a) {\n  return a + 1;  // one\n}\n/* note */\n")
    d0 = bench.kernel_source_digest(["k.cu"])
    (tmp_path / "k.cu").write_text("// header\nint f(int a) {\n  return a + 1;  /* one */\n}\n")
    assert bench.kernel_source_digest(["k.cu"]) == d0
    (tmp_path / "k.cu").write_text("int f(int a) {\n  return a + 2;\n}\n")
    assert bench.kernel_source_digest(["k.cu"]) != d0


def test_trial_and_backprojection_bytes_follow_the_scope_table():
    # f-only trial 8 nnz + 12 m + 8 N, 12 B per voxel for the projected step,
    # 12 more per voxel for UPN's extrapolation; back projection 8 nnz + 4 m + 8 N
    g = bench.trial_bytes(M, N, NNZ, "fp32", "gpbb")
    u = bench.trial_bytes(M, N, NNZ, "fp32", "upn")
    assert round(g / 1e6, 1) == 163.8 and u - g == 12 * N
    assert round(bench.backprojection_bytes(M, N, NNZ, "fp32") / 1e6, 1) == 158.8
    assert g - bench.trial_bytes(M, N, NNZ, "bf16", "gpbb") == 2 * NNZ


def test_both_arms_print_the_same_config():
    import synth
    cfg = synth.get_config("c64")
    a = bench.bench_config(cfg, 1e-4, NNZ, "fp32", 1, 1)
    assert a == bench.bench_config(cfg, 1e-4, NNZ, "fp32", True, 1)
    assert a["m"] == M and a["N"] == N and a["nnz"] == NNZ
