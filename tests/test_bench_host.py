"""Host logic of bench.py that runs without a GPU: the oracle errors of several
solutions in one pass, the oracle-error status of the method variants (direct
errors, else the bound from the main solve), the reference arm's line and the
roofline of a traced solve."""
import numpy as np
import pytest

import bench
from oracle import formats as F
from oracle import fullgrid as fg
from oracle import operator as op
from paper_2006_09314_gb300.inputs import make_problem


def _exact_cp(p):
    """The oracle's exact solution of problem p as a canonical tensor of rank n^2."""
    lams, Vs = zip(*[op.eig(*op.assemble(p.coeffs[l])) for l in range(3)])
    u = fg.solve_exact(F.cp_full(p.yw, p.yU), lams, Vs, p.alpha, p.beta)
    n = p.n
    U = [np.zeros((n, n * n)) for _ in range(3)]
    for j in range(n):
        for k in range(n):
            c = j + n * k
            U[0][:, c] = u[:, j, k]
            U[1][j, c] = 1.0
            U[2][k, c] = 1.0
    return np.ones(n * n), U


@pytest.fixture(scope="module")
def pool():
    p = bench._pool(2)
    yield p
    p.close()


def test_oracle_errors_of_several_solutions_in_one_pass(pool):
    """bench.oracle_errors: the exact solution has error ~0, a 1% scaled one 0.01."""
    p = make_problem(8, 0.5, 1e-2, 2, 5)
    w, U = _exact_cp(p)
    e = bench.oracle_errors(p, [(w, U), (1.01 * w, U)], pool)
    assert e[0] < 1e-12 and abs(e[1] - 0.01) < 1e-9


def test_verify_variants_direct_errors_and_bound():
    errs = [5e-7, 5e-7]
    variants = {"learned_pre": {"rel_diff_to_main": [2e-6, 1e-7], "solves_per_s": 10.0},
                "fp64_sinc": {"rel_diff_to_main": [1e-7, 7e-7], "solves_per_s": 4.0},
                "aniso_pre": {"rel_diff_to_main": [1e-7, 1e-7], "solves_per_s": 2.0},
                "learned_operator": {"accepted": 0}}
    direct = {"learned_pre": [8e-7, 2e-6], "fp64_sinc": [3e-7, None]}
    bench.verify_variants(variants, direct, errs)
    lp, sc, an = variants["learned_pre"], variants["fp64_sinc"], variants["aniso_pre"]
    # direct errors decide, whatever the distance to the main solve says
    assert lp["rel_err_vs_oracle"] == [8e-7, 2e-6] and "err_bound_vs_oracle" not in lp
    assert lp["verified_le_1e-6"] == 1 and lp["verified_solves_per_s"] == 5.0
    # an incomplete direct check leaves the bound: main error + distance
    assert sc["err_bound_vs_oracle"] == pytest.approx([6e-7, 1.2e-6])
    assert sc["verified_le_1e-6"] == 1
    assert an["verified_le_1e-6"] == 2 and an["verified_solves_per_s"] == 2.0
    assert "verified_le_1e-6" not in variants["learned_operator"]


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` (the oracle timed on the host) prints one JSON
    line with the keys of the benchmark contract."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--n", "16"], cwd=root, capture_output=True,
                         text=True, timeout=300, check=True).stdout.strip().splitlines()
    line = json.loads(out[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"


def test_roofline_from_trace_divides_each_kernel_by_its_own_pipe():
    """Tensor-core GEMMs against the BF16 peak (digit products), FP64 GEMMs against
    the FP64 pipe, byte-modelled kernels against HBM; the largest modelled kernel
    gives the roofline object, whose frac is its work / time / peak."""
    rep = {"tcg_kernel": {"launches": 10, "ms": 5.0, "flops": 1e11, "mma_flops": 2.1e12, "bytes": 0.0},
           "dgemm_kernel": {"launches": 100, "ms": 4.0, "flops": 4e8, "mma_flops": 0.0, "bytes": 1e8},
           "split_kernel": {"launches": 20, "ms": 1.0, "flops": 0.0, "mma_flops": 0.0, "bytes": 3e9},
           "jacobi_kernel": {"launches": 3, "ms": 9.0, "flops": 0.0, "mma_flops": 0.0, "bytes": 0.0}}
    iso, roof = bench.roofline_from_trace(rep)
    peaks = bench._pipe_peaks()
    k = iso["kernels"]
    assert k["tcg_kernel"]["bound"] == "tensor"
    assert k["tcg_kernel"]["achieved"] == pytest.approx(2.1e12 / 5e-3 / 1e12, rel=1e-3)
    assert k["dgemm_kernel"]["bound"] == "alu"
    assert k["dgemm_kernel"]["frac"] == pytest.approx(4e8 / 4e-3 / 1e12 / peaks["alu"][0], rel=1e-3)
    assert k["split_kernel"]["bound"] == "hbm"
    assert k["split_kernel"]["achieved"] == pytest.approx(3e9 / 1e-3 / 1e9, rel=1e-3)
    assert "bound" not in k["jacobi_kernel"] and k["jacobi_kernel"]["share"] == pytest.approx(0.4737, abs=1e-3)
    # the jacobi kernel leads but has no work model: the roofline is the tensor-core GEMM
    assert roof["kernel"] == "tcg_kernel" and roof["bound"] == "tensor"
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert roof["work_per_launch"] == pytest.approx(2.1e11)
    assert roof["ms_per_launch"] == pytest.approx(0.5)
