"""PUP sensitivity (Sec. 4.2, Eq. pup_score) on the GPU against the FP64
oracle (itself pinned by finite differences of the image): the accumulated
6 x 6 (mu, s) blocks over several views, and their log determinants, plus
the relation to the efficient score of Sec. 4.2.1."""
import numpy as np
import pytest
import torch

import oracle
from paper_2412_00578_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def raster():
    from paper_2412_00578_gb300 import build

    build.build()
    from paper_2412_00578_gb300 import raster as r

    return r


def views(count=4, seed=95, res=(96, 72)):
    gen = torch.Generator().manual_seed(seed)
    return [synth.orbit_camera(gen, *res) for _ in range(count)]


@pytest.mark.parametrize("mode,tile", [(2, 16), (0, 8), (4, 16)])
def test_pup_hessian_and_logdet_against_oracle(raster, mode, tile):
    scene = synth.blob_scene(3000, seed=96, n_blobs=6, log_scale_mu=-2.5)
    cams = views()
    r = raster.Renderer("cuda:0")
    ds = scene.to("cuda:0")
    H, score = raster.pup_scores(r, ds, cams, mode=mode, tile=tile)
    H = H.cpu().numpy().astype(np.float64)
    score = score.cpu().numpy()
    ref = oracle.pup(scene, cams, tile, mode)
    seen = np.abs(ref).sum(0) > 0
    assert seen.sum() > 500
    rel = np.linalg.norm(H - ref) / np.linalg.norm(ref)
    assert rel <= 1e-3, rel
    # no Gaussian the oracle leaves untouched gets a value, and vice versa
    assert np.array_equal(np.abs(H).sum(0) > 0, seen)
    # log det where the block is well conditioned
    M = oracle.pup_full(ref)
    ev = np.linalg.eigvalsh(M)
    # (the FP32 sums carry a relative error near 1e-6 of the block's largest
    # eigenvalue, so log det is compared where the condition number is < 1e3)
    good = (ev[:, 0] > 0) & (ev[:, -1] < 1e3 * ev[:, 0])
    assert good.sum() > 100
    want = np.linalg.slogdet(M[good])[1]
    assert np.abs(score[good] - want).max() <= 1e-2
    # a block that is not positive definite scores -inf
    assert np.all(np.isneginf(score[~seen]))
    print(f"mode {mode} tile {tile}: rel {rel:.2e}, {good.sum()} well-conditioned blocks")


def test_single_view_block_is_singular_and_scores_relate(raster):
    """One view: every block has rank <= 5 (the image sees the 5 parameters
    of the 2D Gaussian), so U_i = -inf or a huge negative number; the
    efficient score is the same per-pixel weight sum_ch (dC/dg)^2 without the
    geometric factor, so both rank Gaussians that no pixel sees last."""
    scene = synth.blob_scene(3000, seed=97, n_blobs=6, log_scale_mu=-2.5)
    cams = views(count=1, seed=98)
    r = raster.Renderer("cuda:0")
    ds = scene.to("cuda:0")
    H, _ = raster.pup_scores(r, ds, cams)
    M = oracle.pup_full(H.cpu().numpy().astype(np.float64))
    ev = np.linalg.eigvalsh(M)
    seen = ev[:, -1] > 0
    assert seen.sum() > 200
    assert np.all(ev[seen, 0] <= 1e-4 * ev[seen, -1])
