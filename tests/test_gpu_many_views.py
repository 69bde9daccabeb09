"""A scene seen by more views than one group of eight: the record -> vertex
adjoint reads the touched flags eight views at a time and sums a survivor's
views over lanes. The gradient of a batch is the sum of its views' gradients
(each view alone, same upstream), and every view's image is the one it has
alone, bit for bit."""

import numpy as np
import pytest
import torch

import synth
from parity import gpu_run

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("normals", [False, True])
def test_views_of_two_groups_sum_to_the_batch_gradient(normals):
    from paper_2406_01579_b300 import Params
    sc = synth.scene_sphere16()
    cams = [synth.orbit_camera(15.0 + 31.0 * i, 10.0 + 7.0 * (i % 4), 48, 40) for i in range(11)]
    up = synth.upstream_grads(5, cams)
    if normals:
        rng = np.random.default_rng(17)
        up = [u + (rng.normal(size=(3, 40, 48)).astype(np.float32),) for u in up]
    p = Params(s=175.0, tile=8, normals=normals)
    allv = gpu_run([sc], [(c, 0) for c in cams], p, upstream=up)
    gsum = None
    for i, c in enumerate(cams):
        one = gpu_run([sc], [(c, 0)], p, upstream=[up[i]])
        for a, b in zip(allv["views"][i], one["views"][0]):
            assert np.array_equal(a, b)
        g = one["grads"][0]
        gsum = list(g) if gsum is None else [x + y for x, y in zip(gsum, g)]
    for name, a, b in zip(("dV", "df", "drgb"), allv["grads"][0], gsum):
        scale = float(np.abs(b).max())
        assert scale > 0.0
        np.testing.assert_allclose(a, b, rtol=1e-4, atol=1e-5 * scale, err_msg=name)
    torch.cuda.synchronize()
