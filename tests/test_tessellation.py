"""The exact tessellate tiling schedule of the 1D sweeps (Section 3.4).

stencil_tessellation_counts reports, from the same range functions the two
kernels use, how many of a pass's b steps each point of a tile takes in the
triangle stage and in the inverted-triangle stage.  These CPU tests pin it to
the update profiles the paper draws and to the invariants of the scheme; the
GPU parity of the tessellated runs is in test_gpu_sweeps.py.
"""

import pytest


@pytest.fixture(scope="module")
def binding():
    from paper_2103_09235_gb300 import build, binding as b
    build.build()
    return b


def test_tessellation_profile_of_the_paper(binding):
    """4 steps of a radius-1 stencil on a 9-point tile: 0,1,2,3,4,3,2,1,0 in
    the triangles and 4,3,2,1,0,1,2,3,4 in the inverted triangles."""
    s1, s2 = binding.tessellation_counts(9, 4, 1)
    assert s1 == [0, 1, 2, 3, 4, 3, 2, 1, 0]
    assert s2 == [4, 3, 2, 1, 0, 1, 2, 3, 4]


@pytest.mark.parametrize("W,b,R", [(8, 4, 1), (64, 5, 3), (2048, 32, 16), (4096, 6, 12),
                                   (100, 7, 2)])
def test_tessellation_every_point_takes_b_steps(binding, W, b, R):
    """Every point takes exactly b steps over the two stages, and stage 1
    gives a point min(b, d // R) steps for its distance d to the nearer tile
    edge: a triangle step only reads points of its own tile that are already
    at the previous level."""
    s1, s2 = binding.tessellation_counts(W, b, R)
    for i in range(W):
        d = min(i, W - 1 - i)
        assert s1[i] == min(b, d // R)
        assert s1[i] + s2[i] == b


def test_tessellation_rejects_narrow_tiles(binding):
    with pytest.raises(binding.StencilError):
        binding.tessellation_counts(7, 4, 1)
