"""Serving loop on the GPU: resident scenes, Poisson arrivals, continuous
batching over concurrent slots.  Every served image equals the standalone
render of its camera bit for bit, whatever batch it landed in."""
import numpy as np
import pytest
import torch

from paper_2412_00578_gb300 import synth

pytestmark = pytest.mark.gpu


def test_served_results_equal_standalone_renders():
    from paper_2412_00578_gb300 import build

    build.build()
    from paper_2412_00578_gb300 import raster, serve

    scenes = {"s20k": synth.blob_scene(20_000, seed=80, n_blobs=20).to("cuda:0"),
              "s50k": synth.blob_scene(50_000, seed=81, n_blobs=30).to("cuda:0")}
    res = [(64, 48), (160, 120), (97, 61), (200, 150)]

    def cam_fn(gen):
        w, h = res[int(torch.randint(len(res), (1,), generator=gen))]
        return synth.orbit_camera(gen, w, h)

    reqs = serve.poisson_requests(3000.0, 0.03, list(scenes), cam_fn, seed=82)
    assert len(reqs) > 40
    sch = serve.Scheduler({k: v.n for k, v in scenes.items()}, max_batch=8)
    ex = serve.GpuExecutor(scenes, "cuda:0", slots=3)
    done, stats = serve.serve(reqs, sch, ex)
    assert stats["requests"] == len(reqs)
    assert stats["mean_batch"] > 1.0
    ref = raster.Renderer("cuda:0")
    for q in done:
        img = ref.render(scenes[q.scene], q.camera, "accutile", 16).image
        assert torch.equal(q.result, img), q.rid
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    # a sample of served images, one per resolution and scene where present,
    # against the FP32 oracle directly
    import oracle

    cpu = {k: synth.blob_scene(v.n, seed=80 if k == "s20k" else 81, n_blobs=20 if k == "s20k" else 30)
           for k, v in scenes.items()}
    seen = set()
    for q in done:
        key = (q.scene, q.camera.width, q.camera.height)
        if key in seen:
            continue
        seen.add(key)
        o = oracle.render(cpu[q.scene], q.camera, 16, 2, prec64=False)
        err = np.abs(q.result.cpu().numpy().astype(np.float64) - o["image"]).max()
        assert err <= 1e-4, (key, err)
    assert len(seen) >= 4
    print(stats)
