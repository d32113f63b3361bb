"""The solves' noise stream pinned on the GPU (reading R15 of the noise
generator: Philox4x32-10 per Salmon et al., SC'11, and Box-Muller): the
Philox words the kernel's device functions produce for 10^6 counters are
bit-equal to the oracle's independently written Philox, and the normals are
within the error of their binary32 elementary functions.

Bound on a normal: n = r (cos, sin)(2 pi u_b) with r = sqrt(-2 ln u_a).  The
kernel takes -2 ln u_a without a branch (Cody-Waite reduction and the atanh
series: within 2 ulp with an exact division, host test; about 3.5 ulp with
the device's MUFU reciprocal), the radius as x rsqrt(x) (2 ulp for rsqrt,
one rounding), the sin / cos of 2 pi u_b from u_b's bits (within 0.75 ulp
of 1, host test) and one product: about 6 ulp of the radius in all, so
|n_gpu - n_oracle| <= 2^-20 r (8 to 16 ulp of r); the uniform maps are
exact on both sides."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300
    paper_2508_05773_gb300.load()
    return paper_2508_05773_gb300


@pytest.mark.parametrize("seed,counter", [(0, 0), (0x123456789ABCDEF, 4242), (2**64 - 1, 2**32 - 1)])
def test_noise_stream_matches_the_oracle(pkg, seed, counter):
    import torch
    n_samples, H, n_blocks = 2000, 50, 10  # 10^6 Philox blocks
    dev = torch.device("cuda:0")
    words = torch.empty((n_samples, H, n_blocks, 4), dtype=torch.int32, device=dev)
    normals = torch.empty((n_samples, H, n_blocks, 4), dtype=torch.float32, device=dev)
    assert pkg.brmppi_noise_blocks(seed, counter, n_samples, H, n_blocks, words, normals) == 0
    torch.cuda.synchronize()
    gw = words.cpu().numpy().view(np.uint32)
    gn = normals.cpu().numpy().astype(np.float64)
    ow, on = oracle.noise_table(seed, counter, n_samples, H, n_blocks)
    assert np.array_equal(gw, ow)
    r = np.repeat(np.hypot(on[..., 0::2], on[..., 1::2]), 2, axis=-1)
    err = np.abs(gn - on)
    assert np.all(err <= 2.0 ** -20 * r + 1e-30), float(np.max(err / r))
    print(f"noise stream: largest |n_gpu - n_oracle| / r = {float(np.max(err / r)):.3e}")


def test_noise_stream_words_only_and_rejections(pkg):
    import torch
    dev = torch.device("cuda:0")
    words = torch.empty((3, 4, 2, 4), dtype=torch.int32, device=dev)
    assert pkg.brmppi_noise_blocks(9, 1, 3, 4, 2, words, None) == 0
    torch.cuda.synchronize()
    ow, _ = oracle.noise_table(9, 1, 3, 4, 2)
    assert np.array_equal(words.cpu().numpy().view(np.uint32), ow)
    assert pkg.brmppi_noise_blocks(9, 1, -1, 4, 2, words, None) == pkg.BRMPPI_EINVAL
    assert pkg.brmppi_noise_blocks(9, 1, 0, 4, 2, None, None) == 0  # nothing to do
