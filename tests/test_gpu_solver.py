"""Parity of the CUDA minor cycle and the two-step / single-step
reconstructions with the FP64 oracle, through the C ABI (GPU)."""
import numpy as np
import pytest

import synth
from oracle import gridding as og
from oracle import imaging as oi
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


# Model images W beta_K after a minor cycle: the final-image bar of the
# benchmark definition (1e-4 relative L2) for the FP32 form, 1e-8 for FP64.
IMAGE_TOL = {"fp64": 1e-8, "fp32": 1e-4}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def cuda(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _setup(ms, precision="fp64", N=32, J=3, M=8, seed=4):
    w = synth.tiny(npix=N, n_ant=12, n_dumps=10, seed=seed)
    plan = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px, precision=precision,
                   levels=J, n_bases=M)
    return w, plan


def _oracle_problem(w, kind, J, M, lam, part, res, l_low=None, s2=None, e2=None):
    u, v = w.u[0], w.v[0]
    in_l, in_h = og.partition(u, v, w.npix, w.pixel_size, w.ell_px, w.delta_px)
    mask = {"L": in_l, "H": in_h, "ALL": np.ones_like(in_l)}[part]
    A = og.GriddedOperator(u[mask], v[mask], w.npix, w.pixel_size)
    Hhat = osv.psf_spectrum(A.psf())
    W = Dictionary(w.npix, M, J)
    if kind == "low":
        return osv.Problem("low", W, Hhat, res, lam)
    gl, gh = osv.filter_responses(w.npix, w.ell_px, w.delta_px, s2, e2)
    return osv.Problem("full", W, Hhat, res, lam, gl=gl, gh=gh, l_low=l_low)


@pytest.mark.parametrize("step,part", [("low", "L"), ("single", "ALL"), ("full", "H")])
def test_lipschitz_closed_form_matches_oracle(ms, step, part):
    w, plan = _setup(ms)
    res = np.zeros((32, 32))
    s2, e2 = 2.0e-3, 2.0e-6
    prob = _oracle_problem(w, "full" if step == "full" else "low", 3, 8, 0.0, part, res,
                           l_low=res, s2=s2, e2=e2)
    closed, power = plan.lipschitz(step, sigma2=s2, eta2=e2, power_iters=300)
    assert abs(closed - prob.lipschitz_closed_form()) <= 1e-10 * closed
    # the power iteration approaches the closed form from below
    assert power <= closed * (1 + 1e-9)
    assert power >= 0.97 * closed
    plan.close()


def _separated_case(N=32, dl=1e-4, n_dc=10, n_rand=300, seed=7):
    """Rows at the uv origin plus uniformly random rows: the DC term of every
    partition's PSF spectrum stands well above the rest, so the largest
    eigenvalue of the normal operator is separated from the next one."""
    rng = np.random.default_rng(seed)
    u1, v1 = synth.random_uv(n_rand, N, dl, rng, frac_of_grid=0.2)
    return (np.concatenate([np.zeros(n_dc), u1]), np.concatenate([np.zeros(n_dc), v1]))


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 1e-5)])
@pytest.mark.parametrize("step,part", [("low", "L"), ("single", "ALL"), ("full", "H")])
def test_power_iteration_reaches_the_closed_form(ms, precision, tol, step, part):
    """Sect. 3.4: with orthogonal bases and circulant operators the Lipschitz
    constant is 2 M max K^; the library's power iteration through W (FP64
    reductions) must reach it on a spectrum whose top eigenvalue is separated
    (ratio of the next one checked on the oracle's K^; 300 iterations shrink
    the Rayleigh-quotient error by that ratio to the power 600)."""
    N, dl, ell, delta, s2, e2 = 32, 1e-4, 1.0, 0.5, 1.0, 1.2
    u, v = _separated_case(N, dl)
    in_l, in_h = og.partition(u, v, N, dl, ell, delta)
    mask = {"L": in_l, "H": in_h, "ALL": np.ones_like(in_l)}[part]
    A = og.GriddedOperator(u[mask], v[mask], N, dl)
    Hhat = osv.psf_spectrum(A.psf())
    if step == "full":
        gl, gh = osv.filter_responses(N, ell, delta, s2, e2)
        K = (gh * Hhat) ** 2 + gl ** 2
    else:
        K = Hhat ** 2
    top = np.sort(np.unique(np.round(K.ravel() / K.max(), 12)))[::-1]
    assert top[1] <= 0.9, top[:3]
    plan = ms.Plan(u, v, N, dl, ell, delta, precision=precision, levels=3, n_bases=8)
    closed, power = plan.lipschitz(step, sigma2=s2, eta2=e2, power_iters=300)
    err = abs(power - closed) / closed
    print(f"power iteration {step} {precision}: {err:.2e} (next/top {top[1]:.3f})")
    assert abs(closed - 2 * 8 * K.max()) <= (1e-10 if precision == "fp64" else 1e-5) * closed
    assert err <= tol
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-4)])
@pytest.mark.parametrize("step,part", [("low", "L"), ("single", "ALL"), ("full", "H")])
def test_minor_cycle_matches_oracle(ms, precision, tol, step, part):
    """Objective trace F(beta_0..beta_K) and the model W beta_K of one minor
    cycle (Algorithm 1 with Eqs. GradL / GradH) against the oracle."""
    J, M, iters = 3, 8, 30
    w, plan = _setup(ms, precision, J=J, M=M)
    u, v = w.u[0], w.v[0]
    in_l, in_h = og.partition(u, v, 32, w.pixel_size, w.ell_px, w.delta_px)
    mask = {"L": in_l, "H": in_h, "ALL": np.ones_like(in_l)}[part]
    A = og.GriddedOperator(u[mask], v[mask], 32, w.pixel_size)
    res = A.dirty(w.vis[0][mask])
    lam = 0.05 * np.linalg.norm(res) * 2
    rng = np.random.default_rng(0)
    l_low = 0.5 * res + 0.01 * rng.standard_normal(res.shape)
    s2 = osv.sigma2_hat(res)
    e2 = 1e-3 * s2
    prob = _oracle_problem(w, "full" if step == "full" else "low", J, M, lam, part, res,
                           l_low=l_low, s2=s2, e2=e2)
    ref = osv.fista(prob, iters)
    model, st = plan.minor_cycle(step, cuda(res).to(plan.real_dtype), lam, iters,
                                 l_low=cuda(l_low).to(plan.real_dtype) if step == "full" else None,
                                 sigma2=s2, eta2=e2)
    assert st.iterations == iters
    np.testing.assert_allclose(st.trace, ref.objective, rtol=tol)
    e_model = rel(model.cpu().numpy(), prob.W.synth(ref.beta))
    print(f"minor cycle {step} {precision}: model image {e_model:.2e}")
    assert e_model <= IMAGE_TOL[precision]
    assert abs(st.theta - prob.lipschitz_closed_form()) <= 1e-6 * st.theta
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-4)])
@pytest.mark.parametrize("N,J", [(48, 4), (128, 4), (512, 4), (16, 2), (64, 4), (256, 4),
                                 (1024, 4)])
def test_minor_cycle_larger_images_match_oracle(ms, precision, tol, N, J):
    """48 (level sides 48, 24, 12, 6; 2-D cuFFT spectral step), and the
    powers of two 16 ... 1024, whose spectral step runs the column transforms
    in shared memory with every last-stage radix (16: one radix-16 stage;
    64, 128, 512, 1024: radix 4, 8, 2, 4 after radix-16 stages; 256: two
    radix-16 stages).  At 512 pixels and above the level-1 analysis uses
    32-wide tiles whose interior input windows are staged by TMA (edge
    windows by wrapped loads), and synthesis uses 32- and 64-wide tiles."""
    M, iters = 8, 12
    w = synth.tiny(npix=N, n_ant=12, n_dumps=10, seed=11)
    plan = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px,
                   precision=precision, levels=J, n_bases=M)
    A = og.GriddedOperator(w.u[0], w.v[0], N, w.pixel_size)
    res = A.dirty(w.vis[0])
    lam = 0.05 * np.linalg.norm(res) * 2
    prob = osv.Problem("low", Dictionary(N, M, J), osv.psf_spectrum(A.psf()), res, lam)
    ref = osv.fista(prob, iters)
    model, st = plan.minor_cycle("single", cuda(res).to(plan.real_dtype), lam, iters)
    np.testing.assert_allclose(st.trace, ref.objective, rtol=tol)
    e_model = rel(model.cpu().numpy(), prob.W.synth(ref.beta))
    print(f"minor cycle {N} px {precision}: model image {e_model:.2e}")
    assert e_model <= IMAGE_TOL[precision]
    plan.close()


_WIDE = {}


def _wide_reference(N):
    """Oracle FISTA at N = 2048 / 4096 (2 bases, 2 levels, 3 iterations),
    computed once per size."""
    if N not in _WIDE:
        w = synth.tiny(npix=N, n_ant=12, n_dumps=10, seed=11)
        A = og.GriddedOperator(w.u[0], w.v[0], N, w.pixel_size)
        res = A.dirty(w.vis[0])
        lam = 0.05 * np.linalg.norm(res) * 2
        prob = osv.Problem("low", Dictionary(N, 2, 2), osv.psf_spectrum(A.psf()), res, lam)
        _WIDE[N] = (w, res, lam, prob, osv.fista(prob, 3))
    return _WIDE[N]


@pytest.mark.slow
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-4)])
@pytest.mark.parametrize("N", [2048, 4096])
def test_minor_cycle_wide_images_match_oracle(ms, precision, tol, N):
    """The spectral step's transforms at 2048 and 4096 pixels: last radix 4
    and 8, one column per block, and (FP64 at 4096) the column kernel
    without the shared-memory prefetch of X^_{k-1}, K^ and B^."""
    w, res, lam, prob, ref = _wide_reference(N)
    plan = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px,
                   precision=precision, levels=2, n_bases=2)
    model, st = plan.minor_cycle("single", cuda(res).to(plan.real_dtype), lam, 3)
    np.testing.assert_allclose(st.trace, ref.objective, rtol=tol)
    e_model = rel(model.cpu().numpy(), prob.W.synth(ref.beta))
    print(f"minor cycle {N} px {precision}: model image {e_model:.2e}")
    assert e_model <= IMAGE_TOL[precision]
    plan.close()


def test_minor_cycle_relative_tolerance_stop_and_warm_start(ms):
    J, M = 3, 8
    w, plan = _setup(ms, J=J, M=M)
    u, v = w.u[0], w.v[0]
    A = og.GriddedOperator(u, v, 32, w.pixel_size)
    res = A.dirty(w.vis[0])
    lam = 0.02 * np.linalg.norm(res) * 2
    prob = _oracle_problem(w, "low", J, M, lam, "ALL", res)
    ref = osv.fista(prob, 500, rel_tol=1e-5)
    model, st = plan.minor_cycle("single", cuda(res), lam, 500, rel_tol=1e-5)
    assert st.converged and st.iterations == ref.iterations
    np.testing.assert_allclose(st.trace, ref.objective, rtol=1e-9)
    # warm start from a given beta: the oracle from the same start
    beta0 = np.random.default_rng(1).standard_normal((M, 32, 32)) * 1e-3
    ref2 = osv.fista(prob, 12, beta0=beta0)
    b = cuda(beta0)
    _, st2 = plan.minor_cycle("single", cuda(res), lam, 12, beta=b)
    np.testing.assert_allclose(st2.trace, ref2.objective, rtol=1e-9)
    np.testing.assert_allclose(b.cpu().numpy(), ref2.beta, atol=1e-10)
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 1e-4), ("fp32_kahan", 1e-4)])
def test_two_step_and_single_step_small(ms, precision, tol):
    w, plan = _setup(ms, precision, seed=9)
    u, v, vis = w.u[0], w.v[0], w.vis[0]
    opts = ms.ReconOptions(n_major=3, fista_iters=25)
    ro = oi.ReconOptions(n_major=3, fista_iters=25, levels=3)
    tv = cuda(vis).to(plan.complex_dtype)
    low, img, st = plan.reconstruct_two_step(tv, opts)
    o_low, o_full = oi.reconstruct_two_step(vis, u, v, 32, w.pixel_size, w.ell_px, w.delta_px, ro)
    assert rel(low.cpu().numpy(), o_low.image) <= tol
    assert rel(img.cpu().numpy(), o_full.image) <= tol
    assert abs(st.sigma2 - o_full.sigma2) <= 1e-6 * o_full.sigma2 * (1 if precision == "fp64" else 100)
    assert st.total_iterations == 2 * 3 * 25
    single, st1 = plan.reconstruct_single_step(tv, opts)
    o_single = oi.reconstruct_single_step(vis, u, v, 32, w.pixel_size, ro)
    assert rel(single.cpu().numpy(), o_single.image) <= tol
    plan.close()


@pytest.mark.slow
def test_small_fp64_workload_end_to_end(ms):
    """The 128-pixel, 31,744-row workload: two-step and single-step FISTA,
    200 iterations x 5 major cycles, lambda = 1e-3 max|dirty| (held), FP64,
    against the oracle: final images within 1e-4 relative L2."""
    w = synth.small_fp64()
    u, v, vis = w.u[0], w.v[0], w.vis[0]
    plan = ms.Plan(u, v, 128, w.pixel_size, w.ell_px, w.delta_px, precision="fp64")
    opts = ms.ReconOptions(n_major=5, fista_iters=200, lambda_rule="max_fixed",
                           lambda_low=1e-3, lambda_full=1e-3, lambda_single=1e-3)
    ro = oi.ReconOptions(n_major=5, fista_iters=200, lambda_rule="max_fixed",
                         lambda_low=1e-3, lambda_full=1e-3, lambda_single=1e-3)
    tv = cuda(vis)
    low, img, st = plan.reconstruct_two_step(tv, opts)
    o_low, o_full = oi.reconstruct_two_step(vis, u, v, 128, w.pixel_size, w.ell_px, w.delta_px, ro)
    e_low, e_img = rel(low.cpu().numpy(), o_low.image), rel(img.cpu().numpy(), o_full.image)
    single, _ = plan.reconstruct_single_step(tv, opts)
    o_single = oi.reconstruct_single_step(vis, u, v, 128, w.pixel_size, ro)
    e_single = rel(single.cpu().numpy(), o_single.image)
    print(f"small fp64 end to end: low {e_low:.2e} full {e_img:.2e} single {e_single:.2e}")
    assert e_low <= 1e-4 and e_img <= 1e-4 and e_single <= 1e-4
    plan.close()


def test_two_step_needs_both_partitions(ms):
    w = synth.tiny(npix=32, n_ant=8, n_dumps=6, seed=5)
    # ell - delta above every baseline: V_H is empty
    plan = ms.Plan(w.u[0], w.v[0], 32, w.pixel_size, 40.0, 2.0)
    assert plan.partition_counts()["H"] == 0
    with pytest.raises(ms.MsError) as e:
        plan.reconstruct_two_step(cuda(w.vis[0]))
    assert e.value.status == ms.MS_ERR_ARG
    plan.close()


def test_complete_coverage_recovers_the_sky(ms):
    """One noise-free visibility at every image frequency and lambda = 0: the
    library's single-step image equals the sky and its two-step image
    converges to it, as the oracle's do (the exact-recovery pins of the
    oracle); FP64."""
    N, dl = 16, 1e-4
    k = np.arange(-N // 2, N // 2)
    kx, ky = np.meshgrid(k, k)
    u, v = kx.ravel() / (N * dl), ky.ravel() / (N * dl)
    sky = np.random.default_rng(4).standard_normal((N, N))
    vis = og.GriddedOperator(u, v, N, dl).forward(sky)
    plan = ms.Plan(u, v, N, dl, 4.0, 1.5, precision="fp64", levels=2, n_bases=2)
    tv = cuda(vis)
    single, _ = plan.reconstruct_single_step(
        tv, ms.ReconOptions(n_major=3, fista_iters=100, lambda_single=0.0))
    assert rel(single.cpu().numpy(), sky) <= 1e-10
    opts = ms.ReconOptions(n_major=6, fista_iters=300, lambda_low=0.0, lambda_full=0.0,
                           sigma2=1.0, eta2=1e-3)
    low, img, st = plan.reconstruct_two_step(tv, opts)
    ro = oi.ReconOptions(n_major=6, fista_iters=300, lambda_low=0.0, lambda_full=0.0, levels=2,
                         n_bases=2, sigma2=1.0, eta2=1e-3)
    o_low, o_full = oi.reconstruct_two_step(vis, u, v, N, dl, 4.0, 1.5, ro)
    assert rel(img.cpu().numpy(), o_full.image) <= 1e-8
    assert rel(img.cpu().numpy(), sky) <= 1e-5
    plan.close()


def _warm_net(ms, side, seed=3):
    """A network whose head is not zero (so its start differs from the
    step-one image)."""
    net = ms.WarmStartNet(levels=2, width=8, max_side=side, seed=seed)
    p = net.get_params()
    n_head = 8 * 9 + 1   # the head's weights [1][3][3][8] and bias, stored last
    p[-n_head:-1] = np.random.default_rng(seed).standard_normal(n_head - 1) * 0.05
    net.set_params(p)
    return net


def test_warm_start_coefficients_follow_the_network(ms):
    """ms_warm_start_coefficients: x0 = s net([i^_L, i~_H1] / s) with s =
    max|i~_H1| (the network against the oracle's network), and beta = W^H x0 / M
    (the oracle's dictionary on the library's x0), FP64 plan."""
    import torch
    from oracle import unet as ou
    w, plan = _setup(ms, "fp64", N=32, J=3, M=8, seed=9)
    tv = cuda(w.vis[0])
    low, _, _ = plan.reconstruct_two_step(tv, ms.ReconOptions(n_major=2, fista_iters=20))
    res = plan.grid("H", tv)
    net = _warm_net(ms, 32)
    beta, x0 = plan.warm_start_coefficients(net, low, res)
    lo, r = low.cpu().numpy(), res.cpu().numpy()
    s = np.max(np.abs(r))
    xin = np.stack([lo, r], axis=2).astype(np.float32).astype(np.float64) / s
    params = []
    flat, off = net.get_params().astype(np.float64), 0
    spec = ou.UNetSpec(levels=2, width=8)
    for co, ci in spec.conv_shapes():
        nw = co * 9 * ci
        params.append({"w": flat[off:off + nw].reshape(co, 3, 3, ci), "b": flat[off + nw:off + nw + co]})
        off += nw + co
    y, _ = ou.forward(spec, params, np.stack([lo, r], axis=2).astype(np.float32).astype(np.float64)
                      * np.float32(1.0 / s), quantize=True)
    x0_ref = y * s
    e_x0 = rel(x0.cpu().numpy(), x0_ref)
    assert e_x0 <= 2e-3, e_x0
    Wd = Dictionary(32, 8, 3)
    b_ref = Wd.analysis(x0.cpu().numpy()) / 8
    assert rel(beta.cpu().numpy(), b_ref) <= 1e-12
    assert rel(Wd.synth(beta.cpu().numpy()), x0.cpu().numpy()) <= 1e-12   # W beta = x0
    net.close()
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-8), ("fp32", 1e-4)])
def test_two_step_with_warm_start_handle_matches_oracle(ms, precision, tol):
    """ms_reconstruct_two_step with a network in the options: step two's first
    minor cycle starts from the network's coefficients; the oracle's two-step
    method started from the same beta_0 gives the same images."""
    w, plan = _setup(ms, precision, seed=9)
    u, v, vis = w.u[0], w.v[0], w.vis[0]
    tv = cuda(vis).to(plan.complex_dtype)
    net = _warm_net(ms, 32)
    opts = ms.ReconOptions(n_major=3, fista_iters=25, warm_start=net)
    low, img, st = plan.reconstruct_two_step(tv, opts)
    # the start the library used: the network on its own i^_L and i~_H1
    beta0, _ = plan.warm_start_coefficients(net, low, plan.grid("H", tv))
    ro = oi.ReconOptions(n_major=3, fista_iters=25, levels=3)
    o_low, o_full = oi.reconstruct_two_step(vis, u, v, 32, w.pixel_size, w.ell_px, w.delta_px, ro,
                                            beta0_full=beta0.double().cpu().numpy())
    e_low, e_img = rel(low.cpu().numpy(), o_low.image), rel(img.cpu().numpy(), o_full.image)
    print(f"two-step with warm start {precision}: low {e_low:.2e} full {e_img:.2e}")
    assert e_low <= tol and e_img <= tol
    # the start changed the answer's path: without it the image differs
    _, img0, _ = plan.reconstruct_two_step(tv, ms.ReconOptions(n_major=3, fista_iters=25))
    assert rel(img0.cpu().numpy(), img.cpu().numpy()) > 10 * tol
    net.close()
    plan.close()


def test_lambda_entry_point_matches_the_rule(ms):
    w, plan = _setup(ms, "fp64", seed=9)
    res = plan.grid("L", cuda(w.vis[0]))
    r = res.cpu().numpy()
    assert abs(plan.lam(res, 0.05, 3) - 0.05 * np.linalg.norm(r) * 8) <= 1e-12 * np.linalg.norm(r)
    assert abs(plan.lam(res, 1e-3, 2, rule="max_fixed") - 1e-3 * np.abs(r).max()) <= 1e-15
    plan.close()
