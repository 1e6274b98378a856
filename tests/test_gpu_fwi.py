"""GPU parity of the Gauss-Newton FWI pieces (Sec. 3.2-3.3, Alg. 1) against the
oracle, through the C ABI: synthetic data, the sensitivity products J v and J^T w
(Eq. 3.10 written out from the operator of Eq. 3.1), simultaneous sources, and one
Gauss-Newton iteration (conjugate gradients on the normal equations).

Solves run to a tight tolerance (1e-8) so that the comparison is of the products
themselves; the bounds follow the solver's accuracy (complex64 Krylov vectors,
FP64 residual), 1e-5 for data and 1e-4 for products of two solves.  At the paper's
sensitivity tolerance 1e-4 a solve's error is bounded by the condition number of H
times 1e-4 (about 25 times on this problem, measured), so those products are held to 1e-2."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import fwi  # noqa: E402
from paper_2405_17696_gb300 import media  # noqa: E402


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_17696_gb300 import build
    build.build()
    from paper_2405_17696_gb300 import native as n
    return n


def _f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _case(hx=20.0, hz=20.0):
    nx, nz = 64, 32
    c_true = media.layered_velocity(nx, nz, seed=4, n_layers=6)
    c0 = media.gaussian_smooth(c_true, 4.0)
    gamma = media.abl_gamma(nx, nz, 8)
    freqs = [3.0, 5.0]
    src = [2 * nx + 4 + 8 * s for s in range(8)]
    rcv = [2 * nx + ix for ix in range(1, nx, 2)]
    return nx, nz, hx, hz, media.kappa_of(c_true), media.kappa_of(c0), gamma, freqs, src, rcv


def _ctx(native, nx, nz, hx, hz, kappa, gamma, freqs, **opts):
    om = torch.from_numpy(np.asarray([2 * math.pi * f for f in freqs], np.float32)).cuda()
    return native.helm_setup(torch.from_numpy(np.asarray(kappa, np.float32)).cuda(),
                             torch.from_numpy(np.asarray(gamma, np.float32)).cuda(), nx, nz, hx, hz, om,
                             opts=native.helm_default_opts(mg_levels=3, **opts))


def _sources(nx, nz, hx, hz, src, w=None):
    g = np.zeros((len(src), nz * nx), np.complex128)
    for s, k in enumerate(src):
        g[s, k] = 1.0 / (hx * hz)
    g = g.reshape(len(src), nz, nx)
    return g if w is None else np.tensordot(np.asarray(w, np.float64), g, axes=1)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("sim", [False, True])
def test_forward_data_and_sensitivities(native, sim):
    nx, nz, hx, hz, k_true, k0, gamma, freqs, src, rcv = _case()
    om = [float(np.float32(2 * math.pi * f)) for f in freqs]
    w = np.where(np.random.default_rng(1).random((4, len(src))) < 0.5, -1.0, 1.0) if sim else None
    g = _sources(nx, nz, hx, hz, src, w)
    k64, gam = _f32(k0), _f32(gamma)
    d_ref, _ = fwi.forward_data(k64, gam, om, hx, hz, g, np.array(rcv))
    rng = np.random.default_rng(2)
    dm = (rng.normal(size=(nz, nx)) * k64 ** 2 * 1e-2).astype(np.float32)
    dd_in = (rng.normal(size=d_ref.shape) + 1j * rng.normal(size=d_ref.shape)).astype(np.complex64)
    jv_ref = fwi.jacobian_apply(k64, gam, om, hx, hz, g, np.array(rcv), _f32(dm))
    jt_ref = fwi.jacobian_adjoint(k64, gam, om, hx, hz, g, np.array(rcv), dd_in.astype(np.complex128))
    sv = native.Survey(src, rcv, w)
    ctx = _ctx(native, nx, nz, hx, hz, k0, gamma, freqs)
    try:
        d = np.zeros(d_ref.shape, np.complex64)
        iters = native.fwi_forward_data(ctx, sv, d, tol=1e-8)
        jv = np.zeros(d_ref.shape, np.complex64)
        native.fwi_jacobian(ctx, sv, dm, jv, tol=1e-8)
        jt = np.zeros((nz, nx), np.float32)
        native.fwi_jacobian_adjoint(ctx, sv, dd_in, jt, tol=1e-8)
        jv4 = np.zeros(d_ref.shape, np.complex64)
        native.fwi_jacobian(ctx, sv, dm, jv4, tol=1e-4)
        jt4 = np.zeros((nz, nx), np.float32)
        native.fwi_jacobian_adjoint(ctx, sv, dd_in, jt4, tol=1e-4)
    finally:
        native.helm_destroy(ctx)
    assert iters > 0
    assert _rel(d, d_ref) <= 1e-5
    assert _rel(jv, jv_ref) <= 1e-4
    assert _rel(jt, jt_ref) <= 1e-4
    assert _rel(jv4, jv_ref) <= 1e-2 and _rel(jt4, jt_ref) <= 1e-2
    # the adjoint identity on the GPU's own products
    lhs = float(np.real(np.vdot(dd_in.astype(np.complex128), jv.astype(np.complex128))))
    rhs = float(np.sum(_f32(dm) * _f32(jt)))
    assert abs(lhs - rhs) <= 1e-4 * abs(lhs)


def test_gauss_newton_iteration_matches_the_oracle(native):
    """One Gauss-Newton iteration (3 CG steps, full step accepted) against the oracle's
    direction; the misfit drops and the iteration counts are reported per phase."""
    nx, nz, hx, hz, k_true, k0, gamma, freqs, src, rcv = _case()
    om = [float(np.float32(2 * math.pi * f)) for f in freqs]
    g = _sources(nx, nz, hx, hz, src)
    d_obs, _ = fwi.forward_data(_f32(k_true), _f32(gamma), om, hx, hz, g, np.array(rcv))
    dm_ref, phi_ref, _ = fwi.gauss_newton_direction(_f32(k0), _f32(gamma), om, hx, hz, g, np.array(rcv), d_obs, 3)
    sv = native.Survey(src, rcv)
    m = (np.asarray(k0, np.float32) ** 2).astype(np.float32)
    m0 = m.copy()
    ctx = _ctx(native, nx, nz, hx, hz, k0, gamma, freqs)
    try:
        info = native.fwi_gn_iteration(ctx, sv, np.ascontiguousarray(d_obs, np.complex64), m,
                                       native.fwi_default_gn_opts(tol=1e-8, tol_sens=1e-8, cg_iters=3,
                                                                  max_backtracks=0))
    finally:
        native.helm_destroy(ctx)
    assert abs(info["misfit_before"] - phi_ref) <= 1e-5 * phi_ref
    assert info["step"] == 1.0 and info["misfit_after"] < info["misfit_before"]
    assert info["cg_iters"] == 3
    assert min(info["iters_forward"], info["iters_adjoint"], info["iters_sensitivity"]) > 0
    assert _rel(_f32(m) - _f32(m0), dm_ref) <= 1e-3


@pytest.mark.parametrize("kind,alpha,hz", [(1, 4e16, 20.0), (2, 3e19, 20.0), (1, 1.87e17, 30.0), (2, 2.52e20, 30.0)])
def test_regularised_gauss_newton_iteration_matches_the_oracle(native, kind, alpha, hz):
    """One Gauss-Newton iteration on Phi + alpha R with R_diff (kind 1) or R_high (kind 2)
    of Sec. 5.1 about a smoother reference model, against the oracle's direction.  The
    weights make alpha grad R about a third of grad Phi, so the direction moves far from
    the unregularised one (by 0.77 to 0.96 of its norm in the oracle); the objective Phi +
    alpha R before the step is checked against the oracle's R.  hz = 30: an anisotropic
    grid, whose Laplacian weighs the two axes differently."""
    nx, nz, hx, hz, k_true, k0, gamma, freqs, src, rcv = _case(hz=hz)
    om = [float(np.float32(2 * math.pi * f)) for f in freqs]
    g = _sources(nx, nz, hx, hz, src)
    d_obs, _ = fwi.forward_data(_f32(k_true), _f32(gamma), om, hx, hz, g, np.array(rcv))
    c_ref = media.gaussian_smooth(media.layered_velocity(nx, nz, seed=4, n_layers=6), 10.0)
    m_ref = (np.asarray(media.kappa_of(c_ref), np.float32) ** 2).astype(np.float32)
    alpha = float(np.float32(alpha))
    dm_ref, phi_ref, _ = fwi.gauss_newton_direction(_f32(k0), _f32(gamma), om, hx, hz, g, np.array(rcv), d_obs, 3,
                                                    reg_kind=kind, alpha=alpha, m_ref=_f32(m_ref))
    sv = native.Survey(src, rcv)
    m = (np.asarray(k0, np.float32) ** 2).astype(np.float32)
    m0 = m.copy()
    R_ref = fwi.regularizer(_f32(m0), _f32(m_ref), hx, hz, kind)[0]
    ctx = _ctx(native, nx, nz, hx, hz, k0, gamma, freqs)
    try:
        info = native.fwi_gn_iteration(ctx, sv, np.ascontiguousarray(d_obs, np.complex64), m,
                                       native.fwi_default_gn_opts(tol=1e-8, tol_sens=1e-8, cg_iters=3,
                                                                  max_backtracks=0, reg_kind=kind, alpha=alpha),
                                       m_ref=torch.from_numpy(m_ref).cuda())
    finally:
        native.helm_destroy(ctx)
    assert abs(info["misfit_before"] - phi_ref) <= 1e-5 * phi_ref
    obj_ref = info["misfit_before"] + alpha * R_ref
    assert abs(info["objective_before"] - obj_ref) <= 1e-9 * obj_ref
    assert info["step"] == 1.0 and info["objective_after"] < info["objective_before"]
    assert info["cg_iters"] == 3
    assert _rel(_f32(m) - _f32(m0), dm_ref) <= 1e-3


def test_gauss_newton_rejects_invalid_regulariser_options(native):
    """reg_kind outside {0, 1, 2} and a negative weight are refused before any work."""
    nx, nz, hx, hz, k_true, k0, gamma, freqs, src, rcv = _case()
    sv = native.Survey(src, rcv)
    m = (np.asarray(k0, np.float32) ** 2).astype(np.float32)
    d = np.zeros((len(freqs), len(src), len(rcv)), np.complex64)
    ctx = _ctx(native, nx, nz, hx, hz, k0, gamma, freqs)
    try:
        for bad in (dict(reg_kind=3, alpha=1.0), dict(reg_kind=-1, alpha=1.0), dict(reg_kind=1, alpha=-1.0)):
            with pytest.raises(native.HelmError) as e:
                native.fwi_gn_iteration(ctx, sv, d, m, native.fwi_default_gn_opts(**bad))
            assert e.value.status == native.HELM_EINVAL
    finally:
        native.helm_destroy(ctx)


def test_frequency_continuation_lowers_the_misfit(native):
    """Alg. 1 through the driver: two frequency windows of Gauss-Newton iterations with
    simultaneous sources, MG-FGMRES and CNN-FGMRES with Alg. 2 retraining after each
    iteration; the model error to the true medium drops and the Helmholtz iterations of
    every phase are counted."""
    from paper_2405_17696_gb300 import fwi as FWI
    nx, nz, hx, hz, k_true, k0, gamma, _, src, rcv = _case()
    freqs = [3.0, 4.0]
    d_obs, _ = FWI.observed_data(native, k_true, gamma, nx, nz, hx, hz, freqs, native.Survey(src, rcv))
    m_true = torch.from_numpy((np.asarray(k_true, np.float64) ** 2).astype(np.float32)).cuda()
    results = {}
    for label, retrain in (("mg", None), ("cnn", 4)):
        m = torch.from_numpy((np.asarray(k0, np.float64) ** 2).astype(np.float32)).cuda()
        err0 = float(torch.linalg.norm(m - m_true) / torch.linalg.norm(m_true))
        net = native.cnn_create(3, (16, 32, 64), seed=media.SEED_CNN) if retrain else None
        try:
            cfg = FWI.FwiConfig(windows=[[3.0], [4.0]], gn_iters=2, cg_iters=3, sim_sources=4,
                                retrain_steps=retrain or 0, retrain_initial=8, max_rhs=8)
            hist = FWI.run(native, m, gamma, nx, nz, hx, hz, src, rcv, d_obs, freqs, cfg, net=net)
        finally:
            if net is not None:
                native.cnn_destroy(net)
        err1 = float(torch.linalg.norm(m - m_true) / torch.linalg.norm(m_true))
        results[label] = (err0, err1, hist)
        assert err1 < err0, (label, err0, err1)
        assert len(hist.rows) == 4 and hist.total_iterations > 0
        for r in hist.rows:
            assert r["misfit_after"] <= r["misfit_before"]
        if retrain:
            assert all("retrain_loss" in r for r in hist.rows)


def test_windows_on_their_own_grids(native):
    """Alg. 1 with a grid per frequency window (coarser for the lower frequency): the fine
    model moves toward the truth and each window reports its grid."""
    from paper_2405_17696_gb300 import fwi as FWI
    nx0, nz0, h0 = 192, 96, 20.0
    c_true = media.layered_velocity(nx0, nz0, seed=4, n_layers=6)
    c0 = media.gaussian_smooth(c_true, 6.0)
    lx, lz = nx0 * h0, nz0 * h0
    m = torch.from_numpy((1.0 / c0.astype(np.float64) ** 2).astype(np.float32)).cuda()
    m_true = torch.from_numpy((1.0 / c_true.astype(np.float64) ** 2).astype(np.float32)).cuda()
    windows = []
    for f in (3.0, 5.0):
        nx, nz, hx, hz = FWI.window_grid_size(lx, lz, f)
        kt = torch.empty((nz, nx), dtype=torch.float32, device="cuda")
        native.helm_resample(torch.from_numpy(media.kappa_of(c_true)).cuda(), nx0, nz0, kt, nx, nz)
        gam = media.abl_gamma(nx, nz, max(4, nx // 16))
        src = [2 * nx + 2 + (nx - 4) * s // 8 for s in range(8)]
        rcv = [2 * nx + ix for ix in range(1, nx - 1, 2)]
        d, _ = FWI.observed_data(native, kt, gam, nx, nz, hx, hz, [f], native.Survey(src, rcv))
        windows.append(FWI.WindowGrid([f], nx, nz, hx, hz, gam, src, rcv, d))
    assert (windows[0].nx, windows[0].nz) != (windows[1].nx, windows[1].nz)
    err0 = float(torch.linalg.norm(m - m_true) / torch.linalg.norm(m_true))
    cfg = FWI.FwiConfig(windows=[], gn_iters=2, cg_iters=3, sim_sources=4, max_rhs=8)
    hist = FWI.run_windows(native, m, nx0, nz0, windows, cfg)
    err1 = float(torch.linalg.norm(m - m_true) / torch.linalg.norm(m_true))
    assert [r["grid"] for r in hist.rows] == [[w.nx, w.nz] for w in windows for _ in range(2)]
    for r in hist.rows:
        assert r["misfit_after"] <= r["misfit_before"], r
    assert err1 < err0, (err0, err1)


def test_regulariser_schedule_across_window_grids(native):
    """Alg. 1 with R_high on the first window and R_diff on the second (the order of
    Sec. 5.3), each window on its own grid, the reference model the initial guess resampled
    to that grid: on the first iteration of the first window m = m_ref, so the objective is
    the misfit; on the second window's grid the model has moved, so alpha R > 0; every
    accepted step lowers the objective and the model still moves toward the truth."""
    from paper_2405_17696_gb300 import fwi as FWI
    nx0, nz0, h0 = 192, 96, 20.0
    c_true = media.layered_velocity(nx0, nz0, seed=4, n_layers=6)
    c0 = media.gaussian_smooth(c_true, 6.0)
    lx, lz = nx0 * h0, nz0 * h0
    m = torch.from_numpy((1.0 / c0.astype(np.float64) ** 2).astype(np.float32)).cuda()
    m_true = torch.from_numpy((1.0 / c_true.astype(np.float64) ** 2).astype(np.float32)).cuda()
    windows = []
    for f in (3.0, 5.0):
        nx, nz, hx, hz = FWI.window_grid_size(lx, lz, f)
        kt = torch.empty((nz, nx), dtype=torch.float32, device="cuda")
        native.helm_resample(torch.from_numpy(media.kappa_of(c_true)).cuda(), nx0, nz0, kt, nx, nz)
        gam = media.abl_gamma(nx, nz, max(4, nx // 16))
        src = [2 * nx + 2 + (nx - 4) * s // 8 for s in range(8)]
        rcv = [2 * nx + ix for ix in range(1, nx - 1, 2)]
        d, _ = FWI.observed_data(native, kt, gam, nx, nz, hx, hz, [f], native.Survey(src, rcv))
        windows.append(FWI.WindowGrid([f], nx, nz, hx, hz, gam, src, rcv, d))
    err0 = float(torch.linalg.norm(m - m_true) / torch.linalg.norm(m_true))
    cfg = FWI.FwiConfig(windows=[], gn_iters=2, cg_iters=3, sim_sources=0, max_rhs=8,
                        reg_kind=[2, 1], reg_alpha=[1e17, 1e14])
    hist = FWI.run_windows(native, m, nx0, nz0, windows, cfg)
    err1 = float(torch.linalg.norm(m - m_true) / torch.linalg.norm(m_true))
    rows = hist.rows
    assert len(rows) == 4
    assert rows[0]["objective_before"] == rows[0]["misfit_before"]
    assert rows[2]["objective_before"] > rows[2]["misfit_before"]
    for r in rows:
        assert r["objective_after"] <= r["objective_before"], r
        assert r["objective_after"] >= r["misfit_after"]
    assert err1 < err0, (err0, err1)
    with pytest.raises(ValueError):
        FWI.run(native, m, windows[0].gamma, windows[0].nx, windows[0].nz, windows[0].hx, windows[0].hz,
                windows[0].src_idx, windows[0].rcv_idx, windows[0].d_obs, [3.0],
                FWI.FwiConfig(windows=[[3.0]], reg_kind=[1, 2], reg_alpha=1.0))
