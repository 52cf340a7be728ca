"""Plans on a second GPU of the same process.  The fused pass's launch attributes (its dynamic
shared memory above 48 KB) are set once per device, so a plan on cuda:1 made after one on cuda:0
must solve as well, and give the same image bit for bit.  Skipped when one GPU is visible."""
import numpy as np
import pytest

import gen

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.mark.parametrize("shape", [2, 4])   # MISR_TILE_32x32, MISR_TILE_STREAM
def test_plan_on_a_second_device_after_the_first(orc, shape):
    if torch.cuda.device_count() < 2:
        pytest.skip("one GPU visible")
    from paper_2108_04315_b300 import binding as B
    h, w, f = 40, 56, 2
    sh, psf = gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5)
    P = orc.Problem(h, w, f, sh, psf, lam=0.01)
    y = (P.forward_all(gen.phantom(f * h, f * w, 90)) + gen.gaussian_noise((4, h, w), 0.01, 91)).astype(np.float32)
    images = []
    for dev in (0, 1):
        with torch.cuda.device(dev):
            plan = B.Plan(h, w, f, sh, psf, lam=0.01, iters=8, tile_shape=shape)
            x, st = plan.solve(torch.from_numpy(y).to(f"cuda:{dev}"))
            torch.cuda.synchronize(dev)
            assert st["iters_done"] == 8
            images.append(x.cpu().numpy())
            plan.close()
    assert np.array_equal(images[0], images[1])
