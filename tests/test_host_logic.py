"""Host-side checks that need no GPU: the product never touches the oracle, and
the bench's roofline model (pure functions) computes what its design states."""
import ast
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2107_01715_b300")


def test_product_package_never_imports_the_oracle():
    for dirpath, _, files in os.walk(PKG):
        for f in files:
            path = os.path.join(dirpath, f)
            if f.endswith(".py"):
                tree = ast.parse(open(path).read())
                for node in ast.walk(tree):
                    if isinstance(node, ast.Import):
                        assert all(not a.name.startswith("oracle") for a in node.names), path
                    if isinstance(node, ast.ImportFrom):
                        assert not (node.module or "").startswith("oracle"), path
            if f.endswith((".cu", ".cuh", ".h", ".cpp")):
                assert "or_search" not in open(path).read() and "bcts_oracle" not in open(path).read(), path


def test_binding_import_does_not_load_the_oracle():
    code = ("import sys; import paper_2107_01715_b300.bcts as b; "
            "print(any(m == 'oracle' or m.startswith('oracle.') for m in sys.modules))")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True)
    if out.returncode != 0 and "libbcts" in out.stderr:
        pytest.skip("library not built")
    assert out.stdout.strip() == "False", out.stderr


@pytest.fixture(scope="module")
def bench():
    sys.path.insert(0, ROOT)
    import bench as b
    return b


def test_class_nodes_split_conv1_when_partial_maps_ran(bench):
    n, A, d = 32, 18, 3
    with_z = {"conv1_leaf": 6}
    assert bench.class_nodes("conv1_leaf", n, A, d, with_z) == n * A ** d
    assert bench.class_nodes("conv1_partial", n, A, d, with_z) == n * A ** (d - 1)
    assert bench.class_nodes("conv1", n, A, d, with_z) == n + n * A
    assert bench.class_nodes("conv2", n, A, d, with_z) == n + n * A + n * A ** d
    assert bench.class_nodes("conv1", n, A, d, {}) == n + n * A + n * A ** d


def test_roofline_picks_the_binding_resource(bench):
    pk = {"hbm_gbs": 6000.0, "bf16_tflops_sustained": 1000.0, "sm_max_mhz": 2000.0}
    # leaf conv1 from the partial maps is a streaming pass: no contraction, 54,124 bytes per
    # leaf in split mode (state + 1/18 of the parent's FP32 map + the hi/lo output map)
    macs, mma, rd, wr = bench.layer_model("conv1_leaf", "fp32", 18)
    assert macs == 0 and rd + wr == pytest.approx(80 + 51200 / 18 + 51200)
    r = bench.roofline_for("conv1_leaf", "fp32", 18, 1000, 1.0, 1, pk, "measured")
    assert r["bound"] == "hbm" and r["achieved"] == pytest.approx((rd + wr) * 1000 / 1e-3 / 1e9)
    # conv2 in split mode: 3 MMAs per MAC on the tap-pair kernel's padded grid (100 rows
    # per 81 kept, 127 kept of each 128-row tile) -> tensor-bound; achieved and frac count
    # the method's own FLOPs (2 x MACs), executed_frac the executed MMAs
    r = bench.roofline_for("conv2", "fp32", 18, 1000, 1.0, 1, pk, "measured")
    assert r["bound"] == "tensor"
    assert r["achieved"] == pytest.approx(2 * 81 * 64 * 512 * 1000 / 1e-3 / 1e12)
    assert r["frac"] == pytest.approx(r["achieved"] / 1000.0)
    assert r["executed_frac"] == pytest.approx(3 * 100 / 81 * 128 / 127 * r["frac"])
    # E4M3 doubles the tensor peak; the plain FP32 network is ALU-bound
    r8 = bench.roofline_for("conv2", "fp8", 18, 1000, 1.0, 1, pk, "measured")
    assert r8["min_time_ms"]["tensor_or_alu_executed"] == pytest.approx(
        1e3 * 2 * 81 * 64 * 512 * 1000 * (100 / 81) / 2000e12)
    assert bench.roofline_for("conv2", "fp32_simt", 18, 10 ** 6, 1.0, 1, pk, "measured")["bound"] == "alu"
