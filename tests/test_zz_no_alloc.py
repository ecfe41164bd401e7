"""fse_extrapolate_noalloc, the entry point for callers that cannot allocate
device memory (for example plug-ins whose host owns the device-memory budget,
or loops that must not call cudaMalloc because it can synchronize the device).
It must give what the ordinary entry point gives, call after call, while its
scratch lives in one static device array that every call reuses."""
import numpy as np
import pytest

import paper_2207_00238_gb300 as fse
from paper_2207_00238_gb300 import synth

pytestmark = pytest.mark.gpu


def _jobs():
    rng = synth.Rng(synth.SEED_BASE + 77)
    img = synth.image(96, 72, rng, structure=True)
    defects = dict(image=img, mask=synth.defect_mask(96, 72, 0.01, 2, rng),
                   params=synth.params(4, 14, 32, 100, n_tiles=2, overlap=16))
    return [synth.plain_64()[0], synth.tiled_1024(W=160, H=128, K=80, n_tiles=4)[0], defects]


def _device_job(job, torch):
    dev = torch.device("cuda", 0)
    img = torch.from_numpy(job["image"]).to(dev)
    msk = torch.from_numpy(job["mask"]).to(dev)
    out = torch.zeros_like(img)
    g = torch.zeros(img.shape, dtype=torch.float32, device=dev)
    return (img, msk, out, g), fse.make_job(img, msk, out, job["params"], out_f32=g)


def test_noalloc_matches_batch_entry_on_two_calls():
    import torch
    fse.build()
    jobs = _jobs()
    # reference: the ordinary entry point (context with its own arena)
    ctx = fse.Context(0, arena_bytes=256 << 20)
    ref_bufs, ref_jobs = zip(*[_device_job(j, torch) for j in jobs])
    ctx.extrapolate(list(ref_jobs))
    torch.cuda.synchronize()
    ctx.close()
    ref = [(b[2].cpu().numpy(), b[3].cpu().numpy()) for b in ref_bufs]
    bufs, cjobs = zip(*[_device_job(j, torch) for j in jobs])
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        for b in bufs:
            b[2].zero_()
            b[3].zero_()
        fse.extrapolate_noalloc(list(cjobs), stream=stream)
        # the same kernels on the same inputs: identical bytes and model values
        for (out, g), b, j in zip(ref, bufs, jobs):
            got, gg = b[2].cpu().numpy(), b[3].cpu().numpy()
            assert (got == out).all(), f"call {call}: output bytes differ"
            np.testing.assert_array_equal(gg, g, err_msg=f"call {call}: model values differ")
            lost = j["mask"] > 0
            assert (got[~lost] == j["image"][~lost]).all()


def test_noalloc_rejects_calls_beyond_its_scratch():
    import torch
    big = synth.tiled_1024(W=4096, H=4096, K=10, n_tiles=1)[0]
    _, job = _device_job(big, torch)
    with pytest.raises(fse.FseError) as e:
        fse.extrapolate_noalloc([job])
    assert e.value.code == fse.ENOMEM
    assert "static scratch" in str(e.value)
