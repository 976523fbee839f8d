"""GPU parity of the fused (N <= 2^14) path against the CPU oracle.

Bit-exact: the library's output equals the oracle's op-by-op emulation of the
same 6-FMA Stockham FFT fed with the plan's own rounded table.
Tolerance: dual-select FP32 within relative L2 2e-6 of the FP64 DFT, FP16
(x0.5 per pass) within 4e-3 of DFT/N; BF16 is measured against its own bound
(unit roundoff 2^-8 makes 4e-3 unreachable, see the emulated study)."""
import numpy as np
import pytest

import oracle as orc
from gpu_util import FAC, FMT, assert_bitexact, emulate, gpu_fft
from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu

NS = [2, 4, 8, 16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384]


def _batch_for(N):
    # several blocks plus a ragged tail for every shape
    return max(3, min(37, (1 << 16) // N + 3))


@pytest.fixture(scope="module")
def dsfft():
    import torch
    assert torch.cuda.is_available()
    import paper_2604_00567_b300 as m
    m.lib()
    return m


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("N", NS)
def test_dual_select_bitexact(dsfft, prec, N):
    x = signals.signal(100 + N, _batch_for(N), N, prec)
    plan = dsfft.Plan(N, prec, "dual_select")
    for d in (-1, 1):
        y = gpu_fft(plan, x, d)
        assert_bitexact(y, emulate(plan, x, d), f"N={N} {prec} dir={d}")


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("fac", ["linzer_feig_clamped", "cosine"])
@pytest.mark.parametrize("N", [16, 1024, 4096])
def test_other_tables_bitexact(dsfft, prec, fac, N):
    """The same kernels with the Linzer-Feig and cosine tables (only the table
    changes); FP16 results are non-finite, and must be non-finite in the same
    places."""
    x = signals.signal(200 + N, 5, N, prec)
    plan = dsfft.Plan(N, prec, fac)
    y = gpu_fft(plan, x, -1)
    assert_bitexact(y, emulate(plan, x, -1), f"{fac} N={N} {prec}")


@pytest.mark.parametrize("prec", ["fp32", "fp16", "bf16"])
@pytest.mark.parametrize("scale", [(False, False), (True, True), (False, True)])
def test_scaling_options_bitexact(dsfft, prec, scale):
    N = 2048
    x = signals.signal(300, 6, N, prec)
    plan = dsfft.Plan(N, prec, "dual_select", scale_forward=scale[0], scale_inverse=scale[1])
    for d in (-1, 1):
        assert_bitexact(gpu_fft(plan, x, d), emulate(plan, x, d), f"{prec} scale={scale} dir={d}")


def test_gaussian_and_subnormal_inputs_bitexact(dsfft):
    """Gaussian sigma = 0.25 inputs and FP16 inputs with subnormal values (the
    x0.5 scaling rounds those)."""
    N = 1024
    for prec in ("fp16", "bf16", "fp32"):
        x = signals.signal(400, 9, N, prec, dist="gaussian", sigma=0.25)
        plan = dsfft.Plan(N, prec, "dual_select")
        assert_bitexact(gpu_fft(plan, x), emulate(plan, x), f"gaussian {prec}")
    x0 = signals.signal(401, 4, N, "fp16") * (2.0 ** -16)
    x = np.empty_like(x0)
    x.real = signals.round_storage(x0.real, "fp16")
    x.imag = signals.round_storage(x0.imag, "fp16")
    plan = dsfft.Plan(N, "fp16", "dual_select")
    assert_bitexact(gpu_fft(plan, x), emulate(plan, x), "fp16 subnormal")


@pytest.mark.parametrize("prec,tol", [("fp32", 2e-6), ("fp16", 4e-3), ("bf16", 1.5e-2)])
@pytest.mark.parametrize("N", [1024, 4096, 16384])
def test_accuracy_vs_fp64(dsfft, prec, tol, N):
    x = signals.signal(500 + N, 4, N, prec)
    plan = dsfft.Plan(N, prec, "dual_select")
    y = gpu_fft(plan, x)
    ref = orc.fft_fp64(x) / (N if plan.scale_forward else 1)
    assert orc.rel_l2(y, ref) < tol


def test_round_trip_fp32(dsfft):
    """Forward then inverse, divided by N: ~1e-7 relative L2 (Section V)."""
    N = 4096
    x = signals.signal(600, 8, N, "fp32")
    plan = dsfft.Plan(N, "fp32", "dual_select")
    y = gpu_fft(plan, gpu_fft(plan, x, -1), 1) / N
    assert orc.rel_l2(y, x) < 3e-7


def test_inplace_matches_out_of_place(dsfft):
    for prec in ("fp32", "fp16"):
        for N in (8, 1024, 16384):
            x = signals.signal(700 + N, 5, N, prec)
            plan = dsfft.Plan(N, prec, "dual_select")
            assert_bitexact(gpu_fft(plan, x, inplace=True), gpu_fft(plan, x), f"inplace {prec} {N}")


def test_impulse_and_constant(dsfft):
    N = 4096
    x = np.zeros((2, N), dtype=np.complex128)
    x[0, 0] = 1.0
    x[1, :] = 0.375 - 0.25j
    for prec in ("fp32", "fp16", "bf16"):
        plan = dsfft.Plan(N, prec, "dual_select")
        y = gpu_fft(plan, x)
        s = 1.0 / N if plan.scale_forward else 1.0
        assert np.all(y[0] == s)
        assert y[1, 0] == (0.375 - 0.25j) * N * s and np.all(y[1, 1:] == 0)


def test_batch_zero_and_argument_errors(dsfft):
    import torch
    plan = dsfft.Plan(256, "fp32", "dual_select")
    x = torch.zeros((0, 256), dtype=torch.complex64, device="cuda")
    plan.exec(x)  # no-op
    L = dsfft.lib()
    h = plan.handle
    assert L.fft_exec(h, None, None, 1, -1, None) == 1          # null pointers
    xx = torch.zeros((1, 256), dtype=torch.complex64, device="cuda")
    assert L.fft_exec(h, xx.data_ptr(), xx.data_ptr(), -1, -1, None) == 1   # negative batch
    assert L.fft_exec(h, xx.data_ptr(), xx.data_ptr(), 1, 0, None) == 1     # bad direction
    assert L.fft_exec(h, xx.data_ptr() + 4, xx.data_ptr(), 1, -1, None) == 1  # misaligned
    for bad_n in (0, 1, 3, 1000, 1 << 25):
        with pytest.raises(dsfft.DsfftError) as e:
            dsfft.Plan(bad_n, "fp32", "dual_select")
        assert e.value.status == 2


def test_plan_info(dsfft):
    plan = dsfft.Plan(1024, "fp16", "dual_select")
    info = plan.info()
    assert info["n"] == 1024 and info["log2n"] == 10 and info["kernel"] == 0
    assert info["cos_count"] + info["sin_count"] == 512
    assert info["element_bytes"] == 4


@pytest.mark.parametrize("prec", ["fp32", "fp16"])
@pytest.mark.parametrize("N", [256, 4096, 16384])
def test_output_not_16_byte_aligned(dsfft, prec, N):
    """An output pointer that is element- but not 16-byte-aligned takes the
    direct-store path; results equal the aligned (bulk-store) path."""
    import torch
    x = signals.signal(900 + N, 5, N, prec)
    plan = dsfft.Plan(N, prec, "dual_select")
    xt = signals.to_torch(x, prec, "cuda")
    ref = plan.exec(xt)
    if prec == "fp32":
        buf = torch.zeros((5 * N + 1,), dtype=torch.complex64, device="cuda")
        out = buf[1:].view(5, N)
    else:
        buf = torch.zeros((5 * N + 1, 2), dtype=torch.float16, device="cuda")
        out = buf[1:].view(5, N, 2)
    assert out.data_ptr() % 16 != 0
    plan.exec(xt, out=out)
    torch.cuda.synchronize()
    assert_bitexact(signals.from_torch(out, prec), signals.from_torch(ref, prec), "unaligned out")
