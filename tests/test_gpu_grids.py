"""Several grids at once (per-frequency grids of the FWI windows): helm_resample
against the oracle's resampling, element by element, and helm_solve_multi, whose
contexts of different sizes solve to the tolerance in one call with the iteration
counts of separate solves."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import grids, helmholtz as H  # noqa: E402
from paper_2405_17696_gb300 import media  # noqa: E402


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_17696_gb300 import build
    build.build()
    from paper_2405_17696_gb300 import native as n
    return n


@pytest.mark.parametrize("shape0,shape1", [((1024, 512), (336, 176)), ((336, 176), (1024, 512)), ((97, 45), (97, 45)),
                                           ((64, 32), (100, 60))])
def test_resample_parity(native, shape0, shape1):
    (nx0, nz0), (nx1, nz1) = shape0, shape1
    g = np.random.default_rng(nx0 + nx1)
    src = media.gaussian_smooth(g.normal(size=(nz0, nx0)), 3.0).astype(np.float32)
    base = g.normal(size=(nz1, nx1)).astype(np.float32)
    ref = grids.resample(src.astype(np.float64), nx1, nz1)
    d = torch.from_numpy(base.copy()).cuda()
    native.helm_resample(torch.from_numpy(src).cuda(), nx0, nz0, d, nx1, nz1, 2.0, 1.0)
    got = d.cpu().numpy().astype(np.float64)
    want = 2.0 * ref + base
    assert np.all(np.abs(got - want) <= 2e-6 * (np.abs(want) + np.abs(ref).max()))


def test_solve_multi_over_grids_of_different_sizes(native):
    ctxs, rhs, xs, meta = [], [], [], []
    try:
        for (nx, nz, f) in [(64, 32, 4.0), (128, 64, 5.0), (96, 48, 6.0)]:
            w = media.crop_workload(nx, nz, freqs=(f,), width=8)
            stream = torch.cuda.Stream()
            ctx = native.helm_setup(torch.from_numpy(w.kappa).cuda(), torch.from_numpy(w.gamma).cuda(), nx, nz, w.h,
                                    w.h, torch.tensor([2 * math.pi * f], dtype=torch.float32, device="cuda"),
                                    opts=native.helm_default_opts(mg_levels=3, max_iter=800,
                                                                  stream=stream.cuda_stream))
            ctxs.append(ctx)
            b = torch.from_numpy(w.rhs()).cuda()
            rhs.append(b)
            xs.append(torch.zeros(b.shape, dtype=torch.complex128, device="cuda"))
            meta.append((w, stream))
        torch.cuda.synchronize()
        status, outs = native.helm_solve_multi(ctxs, rhs, xs, [b.shape[0] for b in rhs], tol=1e-6,
                                               flags=native.HELM_SOLVE_ZERO_X0)
        assert status == native.HELM_OK
        for ctx, b, x, (w, _), (it, rel, st) in zip(ctxs, rhs, xs, meta, outs):
            # the same batch alone
            x1 = torch.zeros_like(x)
            s1, it1, rel1, _ = native.helm_solve(ctx, b, x1, b.shape[0], None, 1e-6, native.HELM_SOLVE_ZERO_X0)
            assert s1 == native.HELM_OK and np.array_equal(it, it1)
            xh, bh = x.cpu().numpy(), b.cpu().numpy()
            om = float(np.float32(w.omegas[0]))
            for k in range(bh.shape[0]):
                rr = H.relative_residual(xh[k], bh[k], w.kappa.astype(np.float64), w.gamma.astype(np.float64), om,
                                         w.h, w.h)
                assert rr <= 1e-6
    finally:
        for c in ctxs:
            native.helm_destroy(c)
