"""GPU twiddle-table builder against the oracle's tables (Algorithm 1 and
Eqs. 4-9) and the paper's Table I values."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import FAC, FMT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


def _ulp_diff(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    ia = a.view(np.int64)
    ib = b.view(np.int64)
    ia = np.where(ia < 0, np.int64(-0x8000000000000000) - ia, ia)
    ib = np.where(ib < 0, np.int64(-0x8000000000000000) - ib, ib)
    return np.abs(ia - ib)


@pytest.mark.parametrize("fac", ["dual_select", "linzer_feig_clamped", "cosine"])
@pytest.mark.parametrize("N", [2, 8, 1024, 1 << 14, 1 << 20])
def test_fp64_stage_matches_host(dsfft, fac, N):
    """The GPU's FP64 cos/sin/divide agree with the host's within 2 ulp (the
    cosine table's near-singular k = N/4 entry excepted) and the path flags are
    equal away from the exact ties k = N/8, 3N/8."""
    t, m, p = dsfft.twiddle_fp64(N, fac)
    to, mo, po = orc.table(N, FAC[fac], orc.FP64)
    k = np.arange(N // 2)
    tie = (k * 8 == N) | (k * 8 == 3 * N)
    assert np.array_equal(p[~tie], po[~tie])
    same = p == po
    near_sing = np.abs(to) > 1e6
    assert np.max(_ulp_diff(m[same], mo[same]), initial=0) <= 2
    assert np.max(_ulp_diff(t[same & ~near_sing], to[same & ~near_sing]), initial=0) <= 4


def test_dual_select_table1_on_gpu(dsfft):
    """Table I on the GPU table: |t| <= 1 with max exactly 1 at N = 1024."""
    for prec in ("fp32", "fp16", "bf16"):
        plan = dsfft.Plan(1024, prec, "dual_select", scale_forward=False)
        t, m, p = plan.table(-1)
        assert np.max(np.abs(t)) == 1.0
        info = plan.info()
        assert info["cos_count"] + info["sin_count"] == 512
        assert abs(info["cos_count"] - 256) <= 1


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("fac", ["dual_select", "linzer_feig_clamped", "cosine"])
def test_rounding_once_matches_oracle_rounding(dsfft, prec, fac):
    """Rounded entries are RN-even of the GPU's FP64 values (one rounding)."""
    N = 4096
    t64, m64, p64 = dsfft.twiddle_fp64(N, fac)
    for scaled in (False, True):
        plan = dsfft.Plan(N, prec, fac, scale_forward=scaled)
        t, m, p = plan.table(-1)
        assert np.array_equal(p, p64)
        np.testing.assert_array_equal(t, orc.round_array(t64, FMT[prec]))
        np.testing.assert_array_equal(m, orc.round_array(m64 * (0.5 if scaled else 1.0), FMT[prec]))


def test_inverse_table_is_conjugate(dsfft):
    for prec in ("fp32", "fp16"):
        plan = dsfft.Plan(2048, prec, "dual_select", scale_forward=False, scale_inverse=False)
        tf, mf, pf = plan.table(-1)
        ti, mi, pi = plan.table(1)
        assert np.array_equal(pf, pi)
        np.testing.assert_array_equal(ti, -tf)
        np.testing.assert_array_equal(mi, np.where(pf == 1, -mf, mf))


def test_packed_words_consistent(dsfft):
    """The packed words carry (-t, t), (sigma m, m) and the swap selector."""
    plan = dsfft.Plan(1024, "fp16", "dual_select")
    raw = plan.raw_table(-1)
    lo_t, hi_t = raw[:, 0] & 0xFFFF, raw[:, 0] >> 16
    assert np.all((lo_t ^ hi_t) == 0x8000)
    lo_m, hi_m = raw[:, 1] & 0xFFFF, raw[:, 1] >> 16
    sine = raw[:, 2] == 0x3210
    assert np.all(sine | (raw[:, 2] == 0x1032))
    assert np.all(((lo_m ^ hi_m) == 0x8000) == sine)
    assert np.all(raw[:, 3] == (raw[:, 1] ^ 0x80008000))
    _, _, p = plan.table(-1)
    assert np.array_equal(p, sine.astype(np.int32))


@pytest.mark.parametrize("fac", ["dual_select", "linzer_feig_clamped", "cosine"])
@pytest.mark.parametrize("log2n", [10, 16, 20, 24])
def test_rounded_entries_gpu_vs_host_counted(dsfft, fac, log2n, capsys):
    """Counts (and prints) the rounded FP32/FP16/BF16 entries where the GPU
    plan's table differs from the oracle's table built with the host's libm.
    The two FP64 stages may differ by an ulp (CUDA's and glibc's cos/sin), and
    the exact ties |w_r| = |w_i| at k = N/8 and 3N/8 may take different paths;
    a rounded entry may differ only where its FP64 inputs differ."""
    N = 1 << log2n
    k = np.arange(N // 2)
    tie = (k * 8 == N) | (k * 8 == 3 * N)
    t64, m64, p64 = dsfft.twiddle_fp64(N, fac)
    to64, mo64, po64 = orc.table(N, FAC[fac], orc.FP64)
    fp64_differs = (t64 != to64) | (m64 != mo64) | (p64 != po64)
    lines = []
    for prec in ("fp32", "fp16", "bf16"):
        plan = dsfft.Plan(N, prec, fac, scale_forward=False)
        t, m, p = plan.table(-1)
        to, mo, po = orc.table(N, FAC[fac], FMT[prec])
        both_nan = np.isnan(t) & np.isnan(to)
        differs = ((t != to) & ~both_nan) | (m != mo) | (p != po)
        assert not np.any(differs & ~fp64_differs), "a rounded entry differs while its FP64 values agree"
        assert not np.any((p != po) & ~tie), "paths differ away from the exact ties"
        ties = ", ".join(f"k={int(i)}: path gpu {int(p[i])} host {int(po[i])}" for i in np.flatnonzero(tie))
        lines.append(f"table-diff N=2^{log2n} {fac} {prec}: {int(differs.sum())} of {N // 2} rounded entries differ "
                     f"(FP64 stage differs at {int(fp64_differs.sum())}; ties {ties or 'none'})")
        plan.close()
    with capsys.disabled():
        print("\n" + "\n".join(lines))
