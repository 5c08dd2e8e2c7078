"""gs_intersect_noalloc: key emission for callers that cannot allocate device
memory (for example a plug-in whose host application owns every GPU
allocation, or a real-time loop that must not stall on one).  It keeps its
working memory in a fixed array built into the library instead of the
frame's scratch buffer.  Checked here through the C ABI against gs_intersect
on the same inputs, on two calls in a row (the second call runs on the array
the first one left behind)."""
import numpy as np
import pytest
import torch

from paper_2412_00578_gb300 import synth

pytestmark = pytest.mark.gpu


def test_intersect_noalloc_matches_intersect_on_two_calls_in_a_row():
    from paper_2412_00578_gb300 import build

    build.build()
    from paper_2412_00578_gb300 import raster

    rast = raster.Rasterizer("cuda:0")
    cases = [(synth.small_box_workload(), 2), (synth.small_box_workload(seed=7), 0)]
    for (scene, cam), mode in cases:
        ds = scene.to("cuda:0")
        cfg = raster.cfg_struct(16, mode)
        cap = 200_000
        ref = raster.Frame(scene.n, cam.width, cam.height, 16, cap, "cuda:0")
        rast.gs_preprocess(ds, cam, cfg, ref)
        K_ref = rast.gs_intersect(cam, cfg, ref, sync=True)
        keys_ref = ref.keys[:K_ref].cpu().numpy().view(np.uint64).copy()
        vals_ref = ref.vals[:K_ref].cpu().numpy().view(np.uint32).copy()

        out = raster.Frame(scene.n, cam.width, cam.height, 16, cap, "cuda:0")
        rast.gs_preprocess(ds, cam, cfg, out)
        out.keys.fill_(-1)
        fs = raster.GsFrame.from_buffer_copy(out.struct)
        fs.scratch = None  # the caller provides no working memory at all
        # nor the buffers of the later stages, which this stage never touches
        fs.ranges = fs.image = fs.final_T = fs.last = None
        K = rast.gs_intersect_noalloc(cam, cfg, fs)
        torch.cuda.synchronize()
        assert K == K_ref > 0
        assert np.array_equal(out.keys[:K].cpu().numpy().view(np.uint64), keys_ref)
        assert np.array_equal(out.vals[:K].cpu().numpy().view(np.uint32), vals_ref)


def test_intersect_noalloc_rejects_sizes_beyond_its_limit():
    from paper_2412_00578_gb300 import build

    build.build()
    from paper_2412_00578_gb300 import raster

    rast = raster.Rasterizer("cuda:0")
    _, cam = synth.small_box_workload()
    f = raster.GsFrame()
    f.n_capacity, f.key_capacity = (1 << 24) + 1, 16
    f.width, f.height, f.tile = cam.width, cam.height, 16
    with pytest.raises(raster.GsError) as ei:
        rast.gs_intersect_noalloc(cam, raster.cfg_struct(16, 2), f)
    assert ei.value.status == 1 and "16777216" in str(ei.value)
