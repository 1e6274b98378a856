"""Pins of the oracle's field resampling between node grids of one rectangle."""
import numpy as np

from oracle import grids


def _centres(n, L):
    return (np.arange(n) + 0.5) * L / n


def test_affine_fields_are_reproduced_away_from_the_clamped_edge():
    # an affine field sampled at the source cell centres is interpolated exactly at every
    # target centre that lies between source centres (bilinear interpolation of an affine
    # function), for refinement and coarsening
    Lx, Lz = 3.0, 2.0
    for (nx0, nz0), (nx1, nz1) in [((12, 8), (30, 20)), ((30, 20), (12, 8)), ((17, 9), (40, 23))]:
        x0, z0 = _centres(nx0, Lx), _centres(nz0, Lz)
        f = lambda x, z: 1.5 + 0.7 * x - 2.0 * z
        src = f(x0[None, :], z0[:, None])
        out = grids.resample(src, nx1, nz1)
        x1, z1 = _centres(nx1, Lx), _centres(nz1, Lz)
        inside = ((z1 >= z0[0]) & (z1 <= z0[-1]))[:, None] & ((x1 >= x0[0]) & (x1 <= x0[-1]))[None, :]
        ref = f(x1[None, :], z1[:, None])
        assert np.allclose(out[inside], ref[inside], rtol=0, atol=1e-12)
        # clamped edge: the nearest source row / column's value along the clamped axis
        assert np.allclose(out[0, :][(x1 >= x0[0]) & (x1 <= x0[-1])],
                           f(x1[(x1 >= x0[0]) & (x1 <= x0[-1])], max(z1[0], z0[0])), rtol=0, atol=1e-12)


def test_same_grid_is_the_identity_and_constants_are_kept():
    g = np.random.default_rng(0).normal(size=(7, 11))
    assert np.allclose(grids.resample(g, 11, 7), g, rtol=0, atol=1e-15)
    assert np.allclose(grids.resample(np.full((5, 9), 2.5), 23, 13), 2.5, rtol=0, atol=1e-15)
