"""The C ABI from a plain C program (gcc, no Python binding, no GPU): the
host entry points on the paper's D_G example (CPU only)."""

import os
import shutil
import subprocess

import pytest

from tests.helpers import golden

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1807_07691_b300")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_c_client_on_dg_example(tmp_path):
    exe = str(tmp_path / "c_client")
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_client.c"), "-L", PKG, "-lgsmat", "-Wl,-rpath," + PKG,
                    "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout.splitlines()
    lines = {ln.split(" ", 1)[0]: ln.split(" ", 1)[1] if " " in ln else "" for ln in out}
    g = golden("dg_example.json")
    nums = [int(x) for x in lines["triples"].split(":")[1].split()]
    assert [nums[i:i + 3] for i in range(0, len(nums), 3)] == g["cube_spo"]
    assert lines["sizes"] == "3 7"
    assert lines["decode"] == "A I2 C B"  # the answer (X, W, Z, Y) decoded, Sec. 6.3
    assert lines["decode_bad"] == "1"
    pats = " ".join(f"({s} {p} {o} {sv} {ov})" for s, p, o, sv, ov in g["query"])
    assert lines["bgp"] == f"4 4: {pats}"
    assert lines["vars"] == "x y z w proj 4 distinct 0"
    assert lines["plan"] == " ".join(str(i) for i in g["plan_order"])
    # the same keys and statistics as the client's (likes: 3 entries over 2
    # subjects and 2 objects; follows: 4 over 3 and 3)
    import oracle.planner as oplan

    st = [dict(nnz=3, nr_s=2, nr_o=2) if p[1] == 1 else dict(nnz=4, nr_s=3, nr_o=3) for p in g["query"]]
    keys = [x["nnz"] for x in st]
    assert lines["plan_cost"] == " ".join(str(i) for i in oplan.cost_plan_order(g["query"], keys, st))
    assert lines["unsupported"] == "2"
    assert out[-1] == "ok"
