"""Seeded synthetic signals shared by the tests, the benchmark and the oracle.

This module holds no FFT arithmetic: it draws numbers and rounds them to the
storage format of an input.  Both the CUDA path and the CPU oracle receive the
same (already rounded) values.

Host generator: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) evaluated as a counter-based
function of (seed, index), so any slice of a stream can be regenerated alone.
Uniform variates take the top 53 bits; Gaussian variates use Box-Muller.

Device generator (large benchmark batches only): ``torch.Generator`` on the
GPU, seeded; its draws are not SplitMix64 and are copied back to the host when
a test needs them.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

PRECISIONS = ("fp32", "fp16", "bf16")


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream for ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def round_storage(x: np.ndarray, precision: str) -> np.ndarray:
    """Round FP64 values to the storage precision of an input (fp32: RN-even
    cast; fp16: numpy's RN-even cast; bf16: RN-even of the fp32 value),
    returned as float64 holding exactly representable values."""
    x = np.asarray(x, dtype=np.float64)
    if precision == "fp64":
        return x.copy()
    if precision == "fp32":
        return x.astype(np.float32).astype(np.float64)
    if precision == "fp16":
        return x.astype(np.float16).astype(np.float64)
    if precision == "bf16":
        f = x.astype(np.float32)
        u = f.view(np.uint32).astype(np.uint64)
        lsb = (u >> np.uint64(16)) & np.uint64(1)
        r = ((u + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
        r = r.astype(np.uint32)
        nan = np.isnan(f)
        r[nan] = 0x7FC00000
        return r.view(np.float32).astype(np.float64)
    raise ValueError(f"unknown precision {precision!r}")


def signal(seed: int, batch: int, N: int, precision: str = "fp32", dist: str = "uniform",
           sigma: float = 0.25, start_transform: int = 0) -> np.ndarray:
    """Complex signals of shape ``(batch, N)`` (complex128 holding values of
    ``precision``).  Real and imaginary parts are i.i.d.; ``uniform`` draws
    U[-1, 1), ``gaussian`` draws N(0, sigma^2).  Transform ``b`` uses stream
    positions starting at ``2 N (start_transform + b)`` so slices regenerate."""
    n = 2 * batch * N
    start = 2 * N * start_transform
    if dist == "uniform":
        v = 2.0 * uniform01(seed, start, n) - 1.0
    elif dist == "gaussian":
        u1 = uniform01(seed, 2 * start, n)
        u2 = uniform01(seed ^ 0x5DEECE66D, 2 * start, n)
        u1 = np.maximum(u1, 2.0 ** -60)
        v = sigma * np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    else:
        raise ValueError(f"unknown distribution {dist!r}")
    v = round_storage(v, precision)
    out = np.empty(batch * N, dtype=np.complex128)
    out.real = v[0::2]      # assigned, not computed: keeps the sign of zeros
    out.imag = v[1::2]
    return out.reshape(batch, N)


def to_torch(x: np.ndarray, precision: str, device="cpu"):
    """Pack complex128 values (exactly representable) into the library's
    storage layout: fp32 -> complex64 ``(batch, N)``; fp16/bf16 -> real tensor
    ``(batch, N, 2)`` with interleaved (re, im)."""
    import torch
    x = np.asarray(x, dtype=np.complex128)
    if precision == "fp32":
        return torch.from_numpy(x.astype(np.complex64)).to(device)
    pair = np.stack([x.real, x.imag], axis=-1)
    if precision == "fp16":
        return torch.from_numpy(pair.astype(np.float16)).to(device)
    if precision == "bf16":
        return torch.from_numpy(pair.astype(np.float32)).to(torch.bfloat16).to(device)
    raise ValueError(precision)


def from_torch(t, precision: str) -> np.ndarray:
    """Inverse of :func:`to_torch`: storage tensor -> complex128 values."""
    import torch
    t = t.detach().to("cpu")
    if precision == "fp32":
        return t.numpy().astype(np.complex128)
    f = t.to(torch.float32).numpy().astype(np.float64)
    out = np.empty(f.shape[:-1], dtype=np.complex128)
    out.real = f[..., 0]    # assigned, not computed: x + 1j*y turns -0 into +0
    out.imag = f[..., 1]
    return out


def device_signal(batch: int, N: int, precision: str, seed: int, dist: str = "uniform",
                  sigma: float = 0.25, device="cuda"):
    """Large seeded batch drawn on the GPU with ``torch.Generator`` (used where
    a host SplitMix64 draw of a full 1 GiB batch would be too slow)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    dt = {"fp32": torch.float32, "fp16": torch.float16, "bf16": torch.bfloat16}[precision]
    if dist == "uniform":
        v = torch.rand((batch, N, 2), generator=g, device=device, dtype=torch.float32) * 2.0 - 1.0
    else:
        v = torch.randn((batch, N, 2), generator=g, device=device, dtype=torch.float32) * sigma
    v = v.to(dt)
    if precision == "fp32":
        return torch.view_as_complex(v.contiguous())
    return v.contiguous()
