"""The library's clover site arithmetic run on the host (the same
__host__ __device__ code as its kernels) against the oracle: the blocks
C(x) for random links, the uniform-flux closed form, and the per-site
inverses (1 + C(x))^{-1}.  No GPU needed."""
import numpy as np
import pytest

from oracle import clover as CL
from paper_2106_01275_gb300 import inputs


@pytest.mark.parametrize("dims,seed", [([2, 3, 2, 4], 1), ([4, 4, 4, 4], 2), ([3, 1, 5, 2], 3)])
def test_blocks_match_the_oracle(ptlib, dims, seed):
    U = inputs.gauge_links(dims, seed, eps=0.8)
    kappa, csw = 0.125, 1.7
    got = ptlib.clover_blocks_host(dims, U, kappa, csw)
    want = CL.clover_blocks(U, dims, kappa, csw)
    assert np.abs(got - want).max() < 1e-14 * max(1.0, np.abs(want).max())
    assert np.abs(want).max() > 1e-2                                  # not trivially zero


def test_uniform_flux_closed_form(ptlib):
    dims = [4, 6, 2, 2]
    U, phi = CL.uniform_abelian_links(dims, 1, (0, 1))
    got = ptlib.clover_blocks_host(dims, U, 0.13, 2.0)
    want = -0.13 * 2.0 * np.sin(phi) * np.kron(CL.sigma(0, 1), np.eye(3))
    assert np.allclose(got, want[None], atol=1e-14)
    assert np.abs(ptlib.clover_blocks_host(dims, inputs.unit_links(dims), 0.13, 2.0)).max() == 0.0


def test_site_inverses(ptlib):
    dims = [2, 2, 2, 4]
    U = inputs.gauge_links(dims, 4, eps=0.9)
    C = CL.clover_blocks(U, dims, 0.13, 1.9)
    inv = ptlib.site_blocks_invert_host(C, 1.0)
    want = np.linalg.inv(np.eye(12)[None] + C)
    assert np.abs(inv - want).max() < 1e-13
    rng = np.random.default_rng(5)
    B = rng.standard_normal((3, 12, 12)) + 1j * rng.standard_normal((3, 12, 12))    # pivoting needed
    B[:, 0, 0] = 0.0
    assert np.allclose(ptlib.site_blocks_invert_host(B, 0.0) @ B, np.eye(12)[None], atol=1e-12)
    B[1] = 0.0
    with pytest.raises(ptlib.PtraceError):
        ptlib.site_blocks_invert_host(B, 0.0)
