"""The minor cycle with the linear PSF operator (MS_CONV_LINEAR) against the
oracle's linear reading (the convolution that A^H A / sum(w) is on the
N x N field, through the PSF of a 2N x 2N field)."""
import numpy as np
import pytest

import synth
from oracle import gridding as og
from oracle import imaging as oi
from oracle import solver as osv
from oracle.wavelets import Dictionary

pytestmark = pytest.mark.gpu

IMAGE_TOL = {"fp64": 1e-8, "fp32": 1e-4}


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


def _setup(ms, precision="fp64", N=32, J=3, M=8, seed=4):
    w = synth.tiny(npix=N, n_ant=12, n_dumps=10, seed=seed)
    plan = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px, precision=precision,
                   levels=J, n_bases=M, convolution="linear")
    return w, plan


def _mask(w, part):
    in_l, in_h = og.partition(w.u[0], w.v[0], w.npix, w.pixel_size, w.ell_px, w.delta_px)
    return {"L": in_l, "H": in_h, "ALL": np.ones_like(in_l)}[part]


def _linear_problem(w, kind, J, M, lam, part, res, l_low=None, s2=None, e2=None):
    m = _mask(w, part)
    u, v = w.u[0][m], w.v[0][m]
    Hhat = osv.psf_spectrum(og.GriddedOperator(u, v, w.npix, w.pixel_size).psf())
    Hhat2 = osv.psf_spectrum(og.GriddedOperator(u, v, 2 * w.npix, w.pixel_size).psf())
    W = Dictionary(w.npix, M, J)
    if kind == "low":
        return osv.Problem("low", W, Hhat, res, lam, Hhat2=Hhat2)
    gl, gh = osv.filter_responses(w.npix, w.ell_px, w.delta_px, s2, e2)
    return osv.Problem("full", W, Hhat, res, lam, gl=gl, gh=gh, l_low=l_low, Hhat2=Hhat2)


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
@pytest.mark.parametrize("step,part", [("low", "L"), ("single", "ALL"), ("full", "H")])
def test_linear_step_size_matches_oracle(ms, precision, tol, step, part):
    """The step size of the linear operator: 100 power iterations from the
    SplitMix64 start on both sides (each implements the generator), so the
    estimates agree to rounding; below the oracle's bound."""
    w, plan = _setup(ms, precision)
    res = np.zeros((32, 32))
    s2, e2 = 2.0e-3, 2.0e-6
    prob = _linear_problem(w, "full" if step == "full" else "low", 3, 8, 0.0, part, res,
                           l_low=res, s2=s2, e2=e2)
    used, _ = plan.lipschitz(step, sigma2=s2, eta2=e2, power_iters=0)
    want = oi._step_size(prob, None)
    print(f"linear step size {step} {precision}: {used / want - 1:+.2e} "
          f"(bound / used {prob.lipschitz_closed_form() / used:.2f})")
    assert abs(used - want) <= tol * want
    assert used <= prob.lipschitz_closed_form()
    plan.close()


@pytest.mark.parametrize("step,part", [("low", "L"), ("full", "H")])
def test_linear_power_iteration_reaches_the_top_eigenvalue(ms, step, part):
    """Power iteration on the linear operator (the step size the minor cycle
    uses, 100 iterations, and a 500-iteration run): within 2 % of, and not
    above, 2 M lambda_max(K) with K = H H (or H G_H^2 H + G_L^2) built densely
    from the oracle's operator on a 16 x 16 field (W W^H = M I gives
    lambda_max(W^H K W) = M lambda_max(K))."""
    N, J, M = 16, 2, 4
    w = synth.tiny(npix=N, n_ant=10, n_dumps=8, seed=11)
    s2, e2 = 1.0, 1.2
    plan = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px, precision="fp64",
                   levels=J, n_bases=M, convolution="linear")
    prob = _linear_problem(w, "full" if step == "full" else "low", J, M, 0.0, part,
                           np.zeros((N, N)), l_low=np.zeros((N, N)), s2=s2, e2=e2)
    K = np.zeros((N * N, N * N))
    for i in range(N * N):
        e = np.zeros(N * N)
        e[i] = 1.0
        x = e.reshape(N, N)
        if step == "full":
            y = prob.H(prob.GH(prob.GH(prob.H(x)))) + prob.GL(prob.GL(x))
        else:
            y = prob.H(prob.H(x))
        K[:, i] = y.ravel()
    top = float(np.linalg.eigvalsh(0.5 * (K + K.T))[-1])
    exact = 2.0 * M * top
    used, power = plan.lipschitz(step, sigma2=s2, eta2=e2, power_iters=500)
    print(f"linear {step}: used {used:.6e} 500 iterations {power:.6e} exact {exact:.6e} "
          f"bound {prob.lipschitz_closed_form():.6e}")
    for est in (used, power):
        assert est <= exact * (1 + 1e-9)
        assert est >= 0.98 * exact
    assert exact <= prob.lipschitz_closed_form()
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-4)])
@pytest.mark.parametrize("step,part", [("low", "L"), ("single", "ALL"), ("full", "H")])
def test_linear_minor_cycle_matches_oracle(ms, precision, tol, step, part):
    """Objective trace F(beta_0..beta_K) and W beta_K of one minor cycle with
    the linear PSF operator against the oracle's Algorithm 1 on the same
    problem and step size."""
    J, M, iters = 3, 8, 30
    w, plan = _setup(ms, precision, J=J, M=M)
    m = _mask(w, part)
    A = og.GriddedOperator(w.u[0][m], w.v[0][m], 32, w.pixel_size)
    res = A.dirty(w.vis[0][m])
    lam = 0.05 * np.linalg.norm(res) * 2
    rng = np.random.default_rng(0)
    l_low = 0.5 * res + 0.01 * rng.standard_normal(res.shape)
    s2 = osv.sigma2_hat(res)
    e2 = 1e-3 * s2
    prob = _linear_problem(w, "full" if step == "full" else "low", J, M, lam, part, res,
                           l_low=l_low, s2=s2, e2=e2)
    theta = oi._step_size(prob, None)
    ref = osv.fista(prob, iters, theta=theta)
    model, st = plan.minor_cycle(step, cuda(res).to(plan.real_dtype), lam, iters,
                                 l_low=cuda(l_low).to(plan.real_dtype) if step == "full" else None,
                                 sigma2=s2, eta2=e2)
    assert st.iterations == iters
    np.testing.assert_allclose(st.trace, ref.objective, rtol=tol)
    e_model = rel(model.cpu().numpy(), prob.W.synth(ref.beta))
    print(f"linear minor cycle {step} {precision}: model image {e_model:.2e}")
    assert e_model <= IMAGE_TOL[precision]
    assert abs(st.theta - theta) <= 1e-5 * theta
    plan.close()


@pytest.mark.parametrize("N,J", [(64, 4), (128, 4), (48, 3)])
def test_linear_minor_cycle_larger_images_match_oracle(ms, N, J):
    """Several row blocks and ragged 2N x 2N transforms (N = 48: 2N = 96)."""
    M, iters = 4, 20
    w = synth.tiny(npix=N, n_ant=16, n_dumps=12, seed=5)
    plan = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px, precision="fp64",
                   levels=J, n_bases=M, convolution="linear")
    m = _mask(w, "L")
    A = og.GriddedOperator(w.u[0][m], w.v[0][m], N, w.pixel_size)
    res = A.dirty(w.vis[0][m])
    lam = 0.05 * np.linalg.norm(res) * 2
    prob = _linear_problem(w, "low", J, M, lam, "L", res)
    ref = osv.fista(prob, iters, theta=oi._step_size(prob, None))
    model, st = plan.minor_cycle("low", cuda(res), lam, iters)
    np.testing.assert_allclose(st.trace, ref.objective, rtol=1e-9)
    assert rel(model.cpu().numpy(), prob.W.synth(ref.beta)) <= IMAGE_TOL["fp64"]
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 1e-4)])
def test_linear_two_step_and_single_step_small(ms, precision, tol):
    """The whole method with the linear operator (major cycles, both steps,
    the single-step baseline) against the oracle's convolution="linear"."""
    w, plan = _setup(ms, precision, seed=9)
    u, v, vis = w.u[0], w.v[0], w.vis[0]
    opts = ms.ReconOptions(n_major=3, fista_iters=25)
    ro = oi.ReconOptions(n_major=3, fista_iters=25, levels=3, convolution="linear")
    tv = cuda(vis).to(plan.complex_dtype)
    low, img, st = plan.reconstruct_two_step(tv, opts)
    o_low, o_full = oi.reconstruct_two_step(vis, u, v, 32, w.pixel_size, w.ell_px, w.delta_px, ro)
    print(f"linear two-step {precision}: low {rel(low.cpu().numpy(), o_low.image):.2e} "
          f"full {rel(img.cpu().numpy(), o_full.image):.2e}")
    assert rel(low.cpu().numpy(), o_low.image) <= tol
    assert rel(img.cpu().numpy(), o_full.image) <= tol
    assert st.total_iterations == 2 * 3 * 25
    single, _ = plan.reconstruct_single_step(tv, opts)
    o_single = oi.reconstruct_single_step(vis, u, v, 32, w.pixel_size, ro)
    assert rel(single.cpu().numpy(), o_single.image) <= tol
    plan.close()


def test_linear_needs_the_daubechies_dictionary(ms):
    w = synth.tiny(npix=32, n_ant=8, n_dumps=4, seed=1)
    with pytest.raises(ms.MsError):
        ms.Plan(w.u[0], w.v[0], 32, w.pixel_size, w.ell_px, w.delta_px, dictionary="iuwt",
                convolution="linear")
