"""helm_residual_noalloc against helm_residual, through the C ABI.

The allocation-free entry point serves callers that cannot allocate device
memory (their budget is owned by another allocator, or an allocation is not
acceptable in their loop).  Its output must equal the context-based
helm_residual on the same inputs, on two calls in a row (the second call
reuses the shared scratch array, whose counters it must clear first)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def native():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_17696_gb300 import build
    build.build()
    from paper_2405_17696_gb300 import native as n
    return n


def test_noalloc_residual_matches_helm_residual(native):
    from paper_2405_17696_gb300 import media
    w = media.crop_workload(200, 96, freqs=(3.0, 6.0), width=12)
    nb = 5
    fi = np.array([0, 1, 1, 0, 1], np.int32)
    om = np.asarray(w.omegas, dtype=np.float32)
    kap = torch.from_numpy(w.kappa).cuda()
    gam = torch.from_numpy(w.gamma).cuda()
    ctx = native.helm_setup(kap, gam, w.nx, w.nz, w.h, w.h, torch.from_numpy(om).cuda(),
                            opts=native.helm_default_opts(mg_levels=2))
    try:
        for call in range(2):
            b = torch.from_numpy(media.complex_normal((nb, w.nz, w.nx), seed=40 + call)).cuda()
            x = torch.from_numpy(media.complex_normal((nb, w.nz, w.nx), seed=50 + call).astype(np.complex128)).cuda()
            x = x * (10.0 ** (3 + call))
            r_ref = torch.zeros((nb, w.nz, w.nx), dtype=torch.complex64, device="cuda")
            rel_ref = native.helm_residual(ctx, b, x, r_ref, nb, fi)
            r = torch.full((nb, w.nz, w.nx), 7.0, dtype=torch.complex64, device="cuda")
            rel = torch.full((nb,), -1.0, dtype=torch.float64, device="cuda")
            om_rhs = torch.from_numpy(om[fi]).cuda()
            native.helm_residual_noalloc(kap, gam, w.nx, w.nz, w.h, w.h, om_rhs, b, x, r, rel, nb)
            torch.cuda.synchronize()
            rel = rel.cpu().numpy()
            scale = r_ref.abs().max().item()
            assert (r - r_ref).abs().max().item() <= 1e-6 * scale
            assert np.all(np.abs(rel - rel_ref) <= 1e-12 * rel_ref), (rel, rel_ref)
    finally:
        native.helm_destroy(ctx)


def test_noalloc_rejects_sizes_beyond_the_scratch(native):
    nx, nz, nb = 512, 256, 1025          # 1025 x 64 tiles > 65536 partial sums
    kap = torch.zeros((nz, nx), dtype=torch.float32, device="cuda")
    om = torch.zeros((nb,), dtype=torch.float32, device="cuda")
    b = torch.zeros((1,), dtype=torch.complex64, device="cuda")
    x = torch.zeros((1,), dtype=torch.complex128, device="cuda")
    rel = torch.zeros((1,), dtype=torch.float64, device="cuda")
    with pytest.raises(native.HelmError) as e:
        native.helm_residual_noalloc(kap, kap, nx, nz, 10.0, 10.0, om, b, x, b, rel, nb)
    assert e.value.status == native.HELM_EINVAL
    assert "scratch" in str(e.value)


def test_noalloc_rejects_host_arrays(native):
    """Nothing is staged: an array in host memory is refused before any launch."""
    nx, nz, nb = 64, 32, 1
    kap = torch.zeros((nz, nx), dtype=torch.float32, device="cuda")
    kap_host = torch.zeros((nz, nx), dtype=torch.float32)
    om = torch.zeros((nb,), dtype=torch.float32, device="cuda")
    b = torch.zeros((nb, nz, nx), dtype=torch.complex64, device="cuda")
    x = torch.zeros((nb, nz, nx), dtype=torch.complex128, device="cuda")
    rel = torch.zeros((nb,), dtype=torch.float64, device="cuda")
    with pytest.raises(native.HelmError) as e:
        native.helm_residual_noalloc(kap_host, kap, nx, nz, 10.0, 10.0, om, b, x, b, rel, nb)
    assert e.value.status == native.HELM_EINVAL
    assert "device memory" in str(e.value)
