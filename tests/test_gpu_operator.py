"""Parity of the CUDA measurement operator, partition and dictionary with the
FP64 oracle, through the C ABI (GPU)."""
import numpy as np
import pytest

import synth
from oracle import gridding as og
from oracle import wavelets as ow

pytestmark = pytest.mark.gpu

# tolerances: FP64 path agrees with the oracle to rounding (1e-12 relative L2);
# FP32 operator outputs within 1e-5 relative L2
TOL = {"fp64": 1e-12, "fp32": 1e-5, "fp32_kahan": 1e-5}


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


def _plan(ms, w, precision="fp64", **kw):
    return ms.Plan(w.u[0], w.v[0], w.npix, w.pixel_size, w.ell_px, w.delta_px,
                   precision=precision, **kw)


def _edge_workload(N=32, n=1500, seed=0):
    """Random uv out to the edge of the oversampled grid (footprints wrap)."""
    rng = np.random.default_rng(seed)
    dl = 1e-3
    u, v = synth.random_uv(n, N, dl, rng, frac_of_grid=0.49)
    w = synth.tiny(npix=N)
    w.u, w.v = u[None], v[None]
    w.pixel_size = dl
    w.vis = (rng.standard_normal(n) + 1j * rng.standard_normal(n))[None]
    w.ell_px = 0.2 * N
    w.delta_px = 2.0
    return w


CASES = {
    "tiny32": lambda: synth.tiny(npix=32, n_ant=10, n_dumps=8, seed=1),
    "edge32": lambda: _edge_workload(32, 1500, 0),
    "edge48": lambda: _edge_workload(48, 2222, 1),      # Ng = 96: 16-cell tiles
    "c1": lambda: synth.small_fp64(),
}


@pytest.mark.parametrize("tile", [16, 32])
@pytest.mark.parametrize("case", list(CASES))
def test_partition_rows_match_oracle(ms, case, tile):
    """Bit-exact: every partition holds exactly the oracle's rows; the plan
    order is by tile, then by anchor cell inside the tile (row, column), rows
    sharing an anchor in original order (both tile sides)."""
    w = CASES[case]()
    if (2 * w.npix) % tile:
        pytest.skip("grid side not a multiple of the tile")
    plan = _plan(ms, w, tile=tile)
    in_l, in_h = og.partition(w.u[0], w.v[0], w.npix, w.pixel_size, w.ell_px, w.delta_px)
    counts = plan.partition_counts()
    assert counts["L"] == in_l.sum() and counts["H"] == in_h.sum()
    assert counts["LH"] == (in_l & in_h).sum() and counts["ALL"] == w.nvis
    Ng = 2 * w.npix
    T = tile
    A = og.GriddedOperator(w.u[0], w.v[0], w.npix, w.pixel_size)
    cu = (A.c0u + Ng // 2) % Ng
    cv = (A.c0v + Ng // 2) % Ng
    tile = (cv // T) * (Ng // T) + cu // T
    anchor = (tile.astype(np.int64) * T + cv % T) * T + cu % T
    for part, mask in (("L", in_l), ("H", in_h), ("ALL", np.ones_like(in_l))):
        rows = plan.partition_rows(part)
        np.testing.assert_array_equal(np.sort(rows), np.flatnonzero(mask))
        key = anchor[rows] * (1 << 32) + rows
        assert np.all(np.diff(key) > 0)
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_kahan"])
@pytest.mark.parametrize("case", list(CASES))
def test_degrid_matches_oracle(ms, case, precision):
    import torch
    w = CASES[case]()
    plan = _plan(ms, w, precision)
    rng = np.random.default_rng(7)
    x = rng.standard_normal((w.npix, w.npix))
    A = og.GriddedOperator(w.u[0], w.v[0], w.npix, w.pixel_size)
    ref = A.forward(x)
    out = plan.degrid("ALL", cuda(x).to(plan.real_dtype))
    got = out.cpu().numpy().astype(np.complex128)
    assert rel(got, ref) <= TOL[precision], rel(got, ref)
    # residual form and partition subset: only the partition's rows are written
    in_l, _ = og.partition(w.u[0], w.v[0], w.npix, w.pixel_size, w.ell_px, w.delta_px)
    obs = cuda(w.vis[0]).to(plan.complex_dtype)
    fill = torch.full_like(obs, 7.0)
    plan.degrid("L", cuda(x).to(plan.real_dtype), vis_obs=obs, out=fill)
    got = fill.cpu().numpy().astype(np.complex128)
    np.testing.assert_array_equal(got[~in_l], 7.0)
    want = w.vis[0][in_l] - ref[in_l]
    assert rel(got[in_l], want) <= TOL[precision] * max(1.0, np.linalg.norm(ref[in_l]) / np.linalg.norm(want))
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_kahan"])
@pytest.mark.parametrize("case", list(CASES))
def test_grid_matches_oracle(ms, case, precision):
    w = CASES[case]()
    plan = _plan(ms, w, precision)
    in_l, in_h = og.partition(w.u[0], w.v[0], w.npix, w.pixel_size, w.ell_px, w.delta_px)
    vis = cuda(w.vis[0]).to(plan.complex_dtype)
    for part, mask in (("ALL", np.ones_like(in_l)), ("L", in_l), ("H", in_h)):
        if mask.sum() == 0:
            continue
        A = og.GriddedOperator(w.u[0][mask], w.v[0][mask], w.npix, w.pixel_size)
        ref = A.dirty(w.vis[0][mask])
        got = plan.grid(part, vis).cpu().numpy().astype(np.float64)
        assert rel(got, ref) <= TOL[precision], (part, rel(got, ref))
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_residual_image_and_psf(ms, precision):
    w = synth.small_fp64()
    plan = _plan(ms, w, precision)
    in_l, in_h = og.partition(w.u[0], w.v[0], w.npix, w.pixel_size, w.ell_px, w.delta_px)
    rng = np.random.default_rng(1)
    model = rng.standard_normal((w.npix, w.npix)) * 0.01
    A = og.GriddedOperator(w.u[0][in_h], w.v[0][in_h], w.npix, w.pixel_size)
    ref = A.residual_image(w.vis[0][in_h], model)
    got = plan.residual_image("H", cuda(w.vis[0]).to(plan.complex_dtype),
                              cuda(model).to(plan.real_dtype)).cpu().numpy()
    assert rel(got, ref) <= 10 * TOL[precision]
    psf = plan.psf("H").cpu().numpy()
    assert rel(psf, A.psf()) <= TOL[precision]
    plan.close()


def test_adjointness_on_gpu_fp64(ms):
    """<A x, y> = <x, A^H y> for the CUDA operator (FP64), 1e-12."""
    w = _edge_workload(32, 1500, 3)
    plan = _plan(ms, w)
    rng = np.random.default_rng(2)
    x = rng.standard_normal((32, 32))
    y = rng.standard_normal(1500) + 1j * rng.standard_normal(1500)
    Ax = plan.degrid("ALL", cuda(x)).cpu().numpy()
    AHy = plan.grid("ALL", cuda(y)).cpu().numpy() * 1500
    lhs = np.real(np.vdot(Ax, y))
    rhs = float(np.sum(x * AHy))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    plan.close()


def test_flagged_rows_are_excluded(ms):
    w = synth.tiny(npix=32, n_ant=10, n_dumps=8, seed=2)
    flags = (np.random.default_rng(0).random(w.nvis) < 0.3).astype(np.uint8)
    plan = ms.Plan(w.u[0], w.v[0], 32, w.pixel_size, w.ell_px, w.delta_px, flags=flags)
    keep = flags == 0
    assert plan.partition_counts()["ALL"] == keep.sum()
    A = og.GriddedOperator(w.u[0][keep], w.v[0][keep], 32, w.pixel_size)
    got = plan.grid("ALL", cuda(w.vis[0])).cpu().numpy()
    assert rel(got, A.dirty(w.vis[0][keep])) <= 1e-12
    plan.close()


@pytest.mark.parametrize("chunk", [1, 7, 100])
def test_work_item_split_does_not_change_result(ms, chunk):
    """Hot tiles split into many work items (ragged last item) give the same
    dirty image as the oracle: the fold sums every item of a tile."""
    w = synth.tiny(npix=32, n_ant=10, n_dumps=8, seed=4)
    plan = ms.Plan(w.u[0], w.v[0], 32, w.pixel_size, w.ell_px, w.delta_px, chunk=chunk)
    ref = og.GriddedOperator(w.u[0], w.v[0], 32, w.pixel_size).dirty(w.vis[0])
    assert rel(plan.grid("ALL", cuda(w.vis[0])).cpu().numpy(), ref) <= 1e-12
    plan.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("N,J,M", [(32, 4, 8), (64, 3, 8), (128, 4, 8), (16, 4, 3),
                                   (48, 4, 8), (80, 4, 5), (512, 4, 8), (1024, 4, 8)])
def test_dictionary_matches_oracle(ms, precision, N, J, M):
    """Every tile size of the wavelet kernels: 16- to 64-wide synthesis tiles
    and 8- to 32-wide analysis tiles (the 1024-pixel case has the widest);
    48 and 80 pixels give level sides that are not powers of two."""
    w = synth.tiny(npix=N)
    plan = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px, precision=precision,
                   levels=J, n_bases=M)
    rng = np.random.default_rng(N)
    x = rng.standard_normal((N, N))
    W = ow.Dictionary(N, M, J)
    ana = plan.dictionary_analysis(cuda(x).to(plan.real_dtype)).cpu().numpy()
    assert rel(ana, W.analysis(x)) <= TOL[precision]
    a = rng.standard_normal((M, N, N))
    syn = plan.dictionary_synthesis(cuda(a).to(plan.real_dtype)).cpu().numpy()
    assert rel(syn, W.synth(a)) <= TOL[precision]
    plan.close()


def test_sigma2_hat_matches_oracle(ms):
    from oracle.solver import sigma2_hat
    w = synth.tiny(npix=64)
    plan = _plan(ms, w)
    img = np.random.default_rng(0).standard_normal((64, 64))
    assert abs(plan.sigma2_hat(cuda(img)) - sigma2_hat(img)) <= 1e-12 * sigma2_hat(img)
    plan.close()


def test_large_sampled_degrid_fp32(ms):
    """At the 1024-pixel, 9.27M-row workload, sampled visibilities of the
    FP32 degridder match the exact FP64 model computed row by row."""
    w = synth.ska_mid_like(max_rows=None, device="cuda")
    plan = ms.Plan(w.u[0], w.v[0], w.npix, w.pixel_size, w.ell_px, w.delta_px,
                   precision="fp32")
    rng = np.random.default_rng(0)
    x = np.zeros((w.npix, w.npix))
    pts = rng.integers(300, 700, size=(50, 2))
    x[pts[:, 0], pts[:, 1]] = rng.uniform(0.1, 1.0, 50)
    out = plan.degrid("ALL", cuda(x).float()).cpu().numpy()
    idx = rng.choice(w.nvis, 2000, replace=False)
    # exact model of the point image, row by row: sum_s f_s exp(-2 pi i (u l_s + v m_s))
    p, q = np.nonzero(x)
    l = (q - w.npix // 2) * w.pixel_size
    m = (p - w.npix // 2) * w.pixel_size
    exact = np.exp(-2j * np.pi * (np.outer(w.u[0][idx], l) + np.outer(w.v[0][idx], m))) @ x[p, q]
    assert rel(out[idx], exact) <= 1e-5
    plan.close()


def test_plans_of_different_dictionary_sizes_coexist(ms):
    """The device's Daubechies filter table is shared by every plan on it: a
    plan with fewer bases built later must leave an earlier plan's
    transforms intact."""
    N, J = 32, 3
    w = synth.tiny(npix=N)
    big = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px, precision="fp64",
                  levels=J, n_bases=8)
    small = ms.Plan(w.u[0], w.v[0], N, w.pixel_size, w.ell_px, w.delta_px, precision="fp64",
                    levels=J, n_bases=1)
    a = np.random.default_rng(3).standard_normal((8, N, N))
    syn = big.dictionary_synthesis(cuda(a)).cpu().numpy()
    assert rel(syn, ow.Dictionary(N, 8, J).synth(a)) <= TOL["fp64"]
    small.close()
    big.close()
