"""Host logic of the FWI driver (Alg. 1, Sec. 3.2, 4.2, 5.1), checked on the CPU: the
regulariser schedule per frequency window, the Rademacher weights of the simultaneous
sources, and the grid of a window at about ten points per shortest wavelength."""
import numpy as np
import pytest

from paper_2405_17696_gb300 import fwi as FWI
from paper_2405_17696_gb300 import media


def test_regulariser_schedule_one_value_or_one_per_window():
    cfg = FWI.FwiConfig(windows=[[3.0], [4.0], [5.0]], reg_kind=2, reg_alpha=1e17)
    assert FWI.regulariser_schedule(cfg) == ([2, 2, 2], [1e17] * 3)
    # R_high on the first sweeps, then R_diff (the order of Sec. 5.3)
    cfg = FWI.FwiConfig(windows=[[3.0], [4.0], [5.0]], reg_kind=[2, 2, 1], reg_alpha=[1e17, 1e17, 1e14])
    assert FWI.regulariser_schedule(cfg) == ([2, 2, 1], [1e17, 1e17, 1e14])
    assert FWI.regulariser_schedule(FWI.FwiConfig(windows=[[3.0]])) == ([0], [0.0])


@pytest.mark.parametrize("kind,alpha", [([1, 2], 1.0), (1, [1.0, 2.0]), (3, 1.0), (1.5, 1.0), (1, -1.0),
                                        (1, float("nan"))])
def test_regulariser_schedule_rejects(kind, alpha):
    with pytest.raises(ValueError):
        FWI.regulariser_schedule(FWI.FwiConfig(windows=[[3.0]], reg_kind=kind, reg_alpha=alpha))


def test_rademacher_weights():
    w = FWI.rademacher(16, 40, media.rng(7))
    assert w.shape == (16, 40) and w.dtype == np.float32
    assert set(np.unique(w)) == {-1.0, 1.0}
    assert np.array_equal(w, FWI.rademacher(16, 40, media.rng(7)))     # seeded
    # E[w_ks w_kt] = delta_st: the trace estimator of Sec. 3.2 is unbiased
    big = FWI.rademacher(20000, 4, media.rng(3)).astype(np.float64)
    assert np.allclose(big.T @ big / len(big), np.eye(4), atol=0.03)


def test_window_grid_has_ten_points_per_wavelength():
    lx, lz = 7680.0, 3840.0
    for f in (2.0, 4.0, 8.0):
        nx, nz, hx, hz = FWI.window_grid_size(lx, lz, f)
        assert nx % 16 == 0 and nz % 16 == 0
        assert abs(nx * hx - lx) < 1e-6 and abs(nz * hz - lz) < 1e-6
        h = 1500.0 / (10 * f)
        assert abs(hx - h) <= 0.1 * h and abs(hz - h) <= 0.1 * h
