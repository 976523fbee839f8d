"""Baseline study of the factorizations on the GPU path (small N): the
paper's qualitative results hold on the kernels — FP16 Linzer-Feig with the
1e-7 clamp and the cosine table are non-finite ("divergent", Table I), the
dual-select FP16 error stays below its Eq. 11 bound and below 4e-3, and in
FP32 all three tables give ~1e-7 (Section V)."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rows():
    import bench
    return bench.error_study(log2ns=(10, 12), precisions=("fp32", "fp16", "bf16"))


def _row(rows, n, prec, fac, eps=None):
    for r in rows:
        if r["N"] == n and r["precision"] == prec and r["factorization"] == fac and (
                eps is None or r["lf_eps"] == eps):
            return r
    raise KeyError((n, prec, fac, eps))


@pytest.mark.parametrize("n", [1024, 4096])
def test_fp16_lf_and_cosine_are_non_finite(rows, n):
    lf = _row(rows, n, "fp16", "linzer_feig_clamped", 1e-7)
    cos = _row(rows, n, "fp16", "cosine")
    assert lf["nonfinite_table_entries"] > 0 and lf["nonfinite_out_uniform"] > 0
    assert cos["nonfinite_table_entries"] > 0 and cos["nonfinite_out_uniform"] > 0


@pytest.mark.parametrize("n", [1024, 4096])
def test_fp16_dual_select_within_bound(rows, n):
    ds = _row(rows, n, "fp16", "dual_select")
    assert ds["t_max"] == 1.0                              # Theorem 1, exactly 1 at k = N/8
    assert ds["nonfinite_out_uniform"] == 0 and ds["nonfinite_out_gaussian"] == 0
    assert ds["rel_l2_uniform"] < 4e-3 and ds["rel_l2_gaussian"] < 4e-3
    assert ds["rel_l2_uniform"] < ds["bound_eq11"]
    assert math.isclose(ds["bound_eq11"], (1 + 2.0 ** -11) ** int(np.log2(n)) - 1)


def test_fp16_lf_with_larger_clamp_is_finite_and_worse_bound(rows):
    lf = _row(rows, 1024, "fp16", "linzer_feig_clamped", 2.0 ** -14)
    ds = _row(rows, 1024, "fp16", "dual_select")
    assert lf["nonfinite_out_uniform"] == 0
    assert lf["t_max"] > 100 and lf["bound_eq11"] > 50 * ds["bound_eq11"]


@pytest.mark.parametrize("fac,eps", [("dual_select", None), ("linzer_feig_clamped", 1e-7), ("cosine", None)])
def test_fp32_all_tables_near_1e7(rows, fac, eps):
    r = _row(rows, 1024, "fp32", fac, eps)
    assert r["nonfinite_out_uniform"] == 0
    assert r["rel_l2_uniform"] < 1e-6 and r["rel_l2_gaussian"] < 1e-6
