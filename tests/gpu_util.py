"""Helpers for the GPU tests: run jobs through the C ABI on device tensors."""
import numpy as np

import paper_2207_00238_gb300 as fse


def run_gpu(ctx, jobs, precision=32, f64=False, stream=None):
    """jobs: list of dict(image, mask, params).  Returns list of dict(out, g) and stats."""
    import torch
    dev = torch.device("cuda", 0)
    keep, cjobs, res = [], [], []
    for j in jobs:
        img = torch.from_numpy(np.ascontiguousarray(j["image"])).to(dev)
        msk = torch.from_numpy(np.ascontiguousarray(j["mask"])).to(dev)
        out = torch.empty_like(img)
        H, W = img.shape
        gf = torch.empty((H, W), dtype=torch.float64 if f64 else torch.float32, device=dev)
        p = dict(j["params"])
        p["precision"] = precision
        kw = {"out_f64": gf} if f64 else {"out_f32": gf}
        cjobs.append(fse.make_job(img, msk, out, p, **kw))
        keep += [img, msk, out, gf]
        res.append((out, gf))
    st = ctx.extrapolate(cjobs, stream=stream)
    torch.cuda.synchronize()
    return [dict(out=o.cpu().numpy(), g=g.cpu().numpy()) for o, g in res], st


def psnr(a, b, sel):
    err = a.astype(np.float64)[sel] - b.astype(np.float64)[sel]
    mse = np.mean(err ** 2)
    return float("inf") if mse == 0 else 10 * np.log10(255.0 ** 2 / mse)


def oracle_run(oracle, job, report=True, **over):
    p = dict(job["params"])
    p.update(over)
    return oracle.fse_image(job["image"], job["mask"], block=p["block"], border=p["border"],
                            fft=p["fft"], K=p["K"], rho=p["rho"], delta=p["delta"],
                            gamma=p["gamma"], order=p["order"], n_tiles=p["n_tiles"],
                            overlap=p["overlap"], report=report, tiling=p.get("tiling", "alg1"))
