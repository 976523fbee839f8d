"""Helpers shared by the GPU parity tests (no FFT arithmetic here)."""
from __future__ import annotations

import numpy as np

import oracle as orc
from paper_2604_00567_b300 import signals

FMT = {"fp32": orc.FP32, "fp16": orc.FP16, "bf16": orc.BF16}
FAC = {"dual_select": orc.DS, "linzer_feig_clamped": orc.LF, "cosine": orc.COS}


def gpu_fft(plan, x: np.ndarray, direction: int = -1, inplace: bool = False) -> np.ndarray:
    """Run the library on host values ``x`` (complex128, (batch, N)) and
    return the output as complex128."""
    import torch
    xt = signals.to_torch(x, plan.precision, device="cuda")
    if inplace:
        y = plan.exec(xt, direction=direction, out=xt)
    else:
        y = plan.exec(xt, direction=direction)
    torch.cuda.synchronize()
    return signals.from_torch(y, plan.precision)


def emulate(plan, x: np.ndarray, direction: int = -1) -> np.ndarray:
    """The oracle's op-by-op emulation fed with the plan's own rounded table."""
    t, m, p = plan.table(direction)
    scaled = plan.scale_forward if direction < 0 else plan.scale_inverse
    return orc.emulate_fft(x, FMT[plan.precision], t, m, p, scaled=scaled, threads=8)


def emulate_async(pool, plan, x: np.ndarray, direction: int = -1):
    """:func:`emulate` on a thread pool: the plan's table is downloaded here
    (on the calling thread), the emulation runs on ``pool`` (ctypes releases
    the GIL, so several emulations run in parallel).  Returns a future."""
    t, m, p = plan.table(direction)
    scaled = plan.scale_forward if direction < 0 else plan.scale_inverse
    return pool.submit(orc.emulate_fft, x, FMT[plan.precision], t, m, p, scaled, 1)


def assert_bitexact(y: np.ndarray, ref: np.ndarray, what: str = ""):
    """Equal values, equal NaN positions and equal signs of zeros."""
    for part in ("real", "imag"):
        a = getattr(y, part)
        b = getattr(ref, part)
        na, nb = np.isnan(a), np.isnan(b)
        bad = (na != nb) | (~na & (a != b)) | (~na & (a == 0) & (np.signbit(a) != np.signbit(b)))
        if np.any(bad):
            idx = np.argwhere(bad)[:5]
            raise AssertionError(f"{what} {part}: {int(bad.sum())} mismatches, first at {idx.tolist()}: "
                                 f"gpu {a[tuple(idx[0])]!r} vs oracle {b[tuple(idx[0])]!r}")
