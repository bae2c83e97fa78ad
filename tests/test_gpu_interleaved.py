"""The interleaved two-image pipeline and its two new minor-cycle problems
(Eq. LowRes on V_H, the mirrored Eq. FullRes on V_L) against the oracle
(GPU)."""
import numpy as np
import pytest

import synth
from oracle import gridding as og
from oracle import imaging as oi
from oracle import interleaved as oil
from oracle import solver as osv
from oracle.wavelets import Dictionary

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ms():
    import torch
    import paper_2406_18356_gb300 as pkg
    from paper_2406_18356_gb300 import _build
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    _build.build()
    pkg.load_library()
    return pkg


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-4)])
@pytest.mark.parametrize("step,part", [("low_h", "H"), ("full_l", "L")])
def test_new_minor_cycle_problems_match_oracle(ms, precision, tol, step, part):
    """LOW_H: Eq. LowRes on V_H's PSF; FULL_L: Eq. FullRes on V_L with the
    filters' sides exchanged (data below ell - delta, prior above)."""
    J, M, iters = 3, 8, 30
    w = synth.tiny(npix=32, n_ant=12, n_dumps=10, seed=4)
    plan = ms.Plan(w.u[0], w.v[0], 32, w.pixel_size, w.ell_px, w.delta_px, precision=precision,
                   levels=J, n_bases=M)
    in_l, in_h = og.partition(w.u[0], w.v[0], 32, w.pixel_size, w.ell_px, w.delta_px)
    mask = in_h if part == "H" else in_l
    A = og.GriddedOperator(w.u[0][mask], w.v[0][mask], 32, w.pixel_size)
    res = A.dirty(w.vis[0][mask])
    lam = 0.05 * np.linalg.norm(res) * 2
    W = Dictionary(32, M, J)
    Hhat = osv.psf_spectrum(A.psf())
    s2 = osv.sigma2_hat(res)
    e2 = 1e-3 * s2
    prior = 0.4 * res + 0.01 * np.random.default_rng(1).standard_normal(res.shape)
    if step == "low_h":
        prob = osv.Problem("low", W, Hhat, res, lam)
    else:
        data, ph = oil.mirrored_filters(32, w.ell_px, w.delta_px, s2, e2)
        prob = osv.Problem("full", W, Hhat, res, lam, gl=ph, gh=data, l_low=prior)
    ref = osv.fista(prob, iters)
    model, st = plan.minor_cycle(step, cuda(res).to(plan.real_dtype), lam, iters,
                                 l_low=cuda(prior).to(plan.real_dtype) if step == "full_l" else None,
                                 sigma2=s2, eta2=e2)
    np.testing.assert_allclose(st.trace, ref.objective, rtol=tol)
    e = rel(model.double().cpu().numpy(), W.synth(ref.beta))
    print(f"{step} {precision}: model image {e:.2e}")
    assert e <= (1e-8 if precision == "fp64" else 1e-4)
    assert abs(st.theta - prob.lipschitz_closed_form()) <= 1e-6 * st.theta
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 1e-4)])
def test_interleaved_pipeline_matches_oracle(ms, precision, tol):
    """Both nodes' images and the combined image of three major cycles
    (the two nodes' minor cycles as one batched launch per cycle)."""
    w = synth.tiny(npix=32, n_ant=12, n_dumps=10, seed=9)
    plan = ms.Plan(w.u[0], w.v[0], 32, w.pixel_size, w.ell_px, w.delta_px, precision=precision,
                   levels=3, n_bases=8)
    opts = ms.ReconOptions(n_major=3, fista_iters=25)
    ro = oi.ReconOptions(n_major=3, fista_iters=25, levels=3)
    img, node_l, node_h, st = plan.reconstruct_interleaved(cuda(w.vis[0]).to(plan.complex_dtype),
                                                            opts)
    ref = oil.reconstruct_interleaved(w.vis[0], w.u[0], w.v[0], 32, w.pixel_size, w.ell_px,
                                      w.delta_px, ro)
    errs = [rel(node_l.double().cpu().numpy(), ref.node_l.image),
            rel(node_h.double().cpu().numpy(), ref.node_h.image),
            rel(img.double().cpu().numpy(), ref.image)]
    print(f"interleaved {precision}: node L {errs[0]:.2e} node H {errs[1]:.2e} "
          f"combined {errs[2]:.2e}")
    assert max(errs) <= tol
    for s, node in zip(st, (ref.node_l, ref.node_h)):
        assert s.total_iterations == 3 * 25
        assert s.sigma2 == pytest.approx(node.sigma2, rel=1e-9 if precision == "fp64" else 1e-4)
    plan.close()


def test_interleaved_pipeline_recovers_the_sky_with_complete_coverage(ms):
    """Every image frequency sampled, lambda = 0: the combined image of 6
    cycles is within 1e-4 of the sky (FP64), as in the oracle's pin."""
    rng = np.random.default_rng(4)
    N, dl = 16, 1e-4
    k = np.arange(-N // 2, N // 2)
    kx, ky = np.meshgrid(k, k)
    u, v = kx.ravel() / (N * dl), ky.ravel() / (N * dl)
    sky = rng.standard_normal((N, N))
    vis = og.GriddedOperator(u, v, N, dl).forward(sky)
    plan = ms.Plan(u, v, N, dl, 4.0, 1.5, precision="fp64", levels=2, n_bases=2)
    opts = ms.ReconOptions(n_major=6, fista_iters=300, lambda_low=0.0, lambda_full=0.0)
    img, _, _, _ = plan.reconstruct_interleaved(cuda(vis), opts)
    e = rel(img.cpu().numpy(), sky)
    print(f"interleaved, complete coverage: {e:.2e}")
    assert e <= 1e-4
    plan.close()


@pytest.mark.parametrize("N,convolution", [(32, "linear"), (48, "circular")])
def test_interleaved_pipeline_without_the_batched_form_matches_oracle(ms, N, convolution):
    """Plans the batched form does not serve (the linear PSF operator; N = 48,
    not a power of two) run the two nodes' minor cycles one after the other:
    the same images as the oracle's pipeline (FP64)."""
    w = synth.tiny(npix=N, n_ant=12, n_dumps=10, seed=9)
    plan = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px, precision="fp64",
                   levels=3, n_bases=4, convolution=convolution)
    opts = ms.ReconOptions(n_major=3, fista_iters=20)
    ro = oi.ReconOptions(n_major=3, fista_iters=20, levels=3, n_bases=4, convolution=convolution)
    img, node_l, node_h, st = plan.reconstruct_interleaved(cuda(w.vis[0]), opts)
    ref = oil.reconstruct_interleaved(w.vis[0], w.u[0], w.v[0], N, w.pixel_size, w.ell_px,
                                      w.delta_px, ro)
    errs = [rel(node_l.cpu().numpy(), ref.node_l.image), rel(node_h.cpu().numpy(), ref.node_h.image),
            rel(img.cpu().numpy(), ref.image)]
    print(f"interleaved {convolution} N={N}: node L {errs[0]:.2e} node H {errs[1]:.2e} "
          f"combined {errs[2]:.2e}")
    assert max(errs) <= 1e-8
    assert [s.total_iterations for s in st] == [60, 60]
    plan.close()
