"""Host-memory batches (fft_pipeline_*): chunked copy-in / transform /
copy-out on several streams gives exactly the bytes of transforming the same
batch on the device, for ragged chunk counts, in-place host buffers, both
directions and the fused, cluster and sweep paths."""
import pytest

from paper_2604_00567_b300 import signals

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dsfft():
    import paper_2604_00567_b300 as m
    m.lib()
    return m


@pytest.mark.parametrize("prec,log2n,batch,chunk,depth", [
    ("fp16", 10, 37, 8, 3), ("fp32", 12, 10, 3, 2), ("bf16", 14, 5, 2, 3), ("fp16", 15, 6, 4, 3),
    ("fp16", 17, 3, 1, 2), ("fp32", 16, 2, 5, 1)])
def test_pipeline_matches_device_exec(dsfft, prec, log2n, batch, chunk, depth):
    import torch
    n = 1 << log2n
    x = signals.device_signal(batch, n, prec, seed=log2n)
    plan = dsfft.Plan(n, prec, "dual_select")
    pipe = dsfft.Pipeline(plan, chunk, depth)
    hin = x.cpu().pin_memory()
    word = torch.int32 if prec == "fp32" else torch.int16
    for d in (-1, 1):
        hout = torch.empty_like(hin).pin_memory()
        pipe.exec(hin, hout, direction=d)
        ref = plan.exec(x, direction=d)
        torch.cuda.synchronize()
        assert torch.equal(hout.view(word), ref.cpu().view(word)), d
    # in place on the host buffer
    hio = hin.clone().pin_memory()
    pipe.exec(hio, hio)
    ref = plan.exec(x)
    torch.cuda.synchronize()
    assert torch.equal(hio.view(word), ref.cpu().view(word))
    pipe.close()


def test_pipeline_validation(dsfft):
    import torch
    plan = dsfft.Plan(1024, "fp16", "dual_select")
    with pytest.raises(dsfft.DsfftError):
        dsfft.Pipeline(plan, 0, 2)
    with pytest.raises(dsfft.DsfftError):
        dsfft.Pipeline(plan, 4, 9)
    pipe = dsfft.Pipeline(plan, 4, 2)
    with pytest.raises(ValueError):
        pipe.exec(torch.zeros(2, 1024, 2, dtype=torch.float16, device="cuda"),
                  torch.zeros(2, 1024, 2, dtype=torch.float16))
