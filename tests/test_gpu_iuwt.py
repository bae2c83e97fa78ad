"""The IUWT dictionary on the GPU (App. A.1's alternative to the Daubechies
dictionary; Sect. 3.4's power-iteration step size) against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest

import synth
from oracle import gridding as og
from oracle import iuwt as oiu
from oracle import solver as osv

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


TOL = {"fp64": 1e-12, "fp32": 1e-6}


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N,J", [(32, 1), (64, 3), (256, 4), (48, 3)])
def test_transforms_match_oracle(ms, precision, N, J):
    w = synth.tiny(npix=N, n_ant=8, n_dumps=4, seed=2)
    plan = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px, precision=precision,
                   levels=J, dictionary="iuwt")
    assert plan.n_bases == J + 1
    rng = np.random.default_rng(N + J)
    x = rng.standard_normal((N, N))
    a = rng.standard_normal((J + 1, N, N))
    got_a = plan.dictionary_analysis(cuda(x).to(plan.real_dtype)).double().cpu().numpy()
    assert rel(got_a, oiu.iuwt(x, J)) <= TOL[precision]
    got_x = plan.dictionary_synthesis(cuda(a).to(plan.real_dtype)).double().cpu().numpy()
    assert rel(got_x, oiu.iuwt_adjoint(a, J)) <= TOL[precision]
    plan.close()


def _case(ms, precision, N=64, J=3, seed=3):
    w = synth.tiny(npix=N, n_ant=14, n_dumps=12, seed=seed)
    plan = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px, precision=precision,
                   levels=J, dictionary="iuwt")
    return w, plan


@pytest.mark.parametrize("step,part", [("low", "L"), ("single", "ALL"), ("full", "H")])
def test_power_iteration_step_size(ms, step, part):
    """The step size the minor cycle uses (100 power iterations) and a long
    power iteration, against the Fourier-space value max_k K(k) S(k) of the
    oracle (S the symbol of T^H T)."""
    N, J = 64, 3
    w, plan = _case(ms, "fp64", N, J)
    s2, e2 = 1.0, 1e-3
    in_l, in_h = og.partition(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px)
    mask = {"L": in_l, "H": in_h, "ALL": np.ones_like(in_l)}[part]
    A = og.GriddedOperator(w.u[0][mask], w.v[0][mask], N, w.pixel_size)
    Hhat = osv.psf_spectrum(A.psf())
    if step == "full":
        gl, gh = osv.filter_responses(N, w.ell_px, w.delta_px, s2, e2)
        K = (gh * Hhat) ** 2 + gl ** 2
    else:
        K = Hhat ** 2
    want = oiu.lipschitz_fourier(K, N, J)
    used, power = plan.lipschitz(step, sigma2=s2, eta2=e2, power_iters=2000)
    print(f"IUWT step size {step}: used {used / want - 1:+.2e}, 2000 iterations {power / want - 1:+.2e}")
    assert power <= want * (1 + 1e-9) and power >= want * (1 - 1e-6)
    assert used <= want * (1 + 1e-9) and used >= want * (1 - 1e-2)
    plan.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-9), ("fp32", 2e-4)])
@pytest.mark.parametrize("step", ["single", "full"])
def test_minor_cycle_matches_oracle(ms, precision, tol, step):
    """FISTA (Algorithm 1) with W = T^H, the step size the library chose
    handed to the oracle: objective traces and the model image."""
    N, J, iters = 64, 3, 25
    w, plan = _case(ms, precision, N, J)
    u, v = w.u[0], w.v[0]
    in_l, in_h = og.partition(u, v, N, w.pixel_size, w.ell_px, w.delta_px)
    mask = in_h if step == "full" else np.ones_like(in_l)
    A = og.GriddedOperator(u[mask], v[mask], N, w.pixel_size)
    res = A.dirty(w.vis[0][mask])
    lam = 0.02 * np.linalg.norm(res) * 2
    Wd = oiu.IUWTDictionary(N, J)
    Hhat = osv.psf_spectrum(A.psf())
    kw = {}
    if step == "full":
        s2 = osv.sigma2_hat(res)
        e2 = 1e-3 * s2
        l_low = 0.5 * res
        gl, gh = osv.filter_responses(N, w.ell_px, w.delta_px, s2, e2)
        prob = osv.Problem("full", Wd, Hhat, res, lam, gl=gl, gh=gh, l_low=l_low)
        kw = {"l_low": cuda(l_low).to(plan.real_dtype), "sigma2": s2, "eta2": e2}
    else:
        prob = osv.Problem("low", Wd, Hhat, res, lam)
    model, st = plan.minor_cycle(step, cuda(res).to(plan.real_dtype), lam, iters, **kw)
    ref = osv.fista(prob, iters, theta=st.theta)
    np.testing.assert_allclose(st.trace, ref.objective, rtol=tol)
    e = rel(model.double().cpu().numpy(), Wd.synth(ref.beta))
    print(f"IUWT minor cycle {step} {precision}: model image {e:.2e}")
    assert e <= (1e-8 if precision == "fp64" else 1e-4)
    plan.close()


def test_warm_start_needs_daubechies(ms):
    import torch
    w, plan = _case(ms, "fp64", 32, 2)
    net = ms.WarmStartNet(levels=2, width=8, max_side=32, seed=0)
    z = torch.zeros((32, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(ms.MsError) as e:
        plan.warm_start_coefficients(net, z, z)
    assert e.value.status == ms.MS_ERR_ARG
    net.close()
    plan.close()
