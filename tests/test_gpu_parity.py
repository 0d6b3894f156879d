"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.  Tolerance: relative error <= 1e-5 per magnification
(FP32 rays and accumulation against FP64 throughout), 1e-9 for point-source
magnifications (FP64 polish and validation)."""
import numpy as np
import pytest

from paper_2510_02639_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def G():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2510_02639_gb300 import build as B
    B.build()
    from paper_2510_02639_gb300 import icrs
    return icrs


def run_gpu(icrs, params, t, grid):
    import torch
    n_lens = int(params[0]["n_lens"])
    pd = icrs.params_to_device(params)
    tt = torch.tensor(np.asarray(t, dtype=np.float64).reshape(len(params), -1), device="cuda")
    A, st = icrs.magnification(pd, tt, icrs.grid_from_dict(grid, n_lens))
    torch.cuda.synchronize()
    return A.cpu().numpy(), st.cpu().numpy()


def assert_parity(A, Ao, tol=TOL, what=""):
    rel = np.abs(A / Ao - 1.0)
    bad = np.argwhere(rel > tol)
    assert np.all(np.isfinite(A)), what
    assert len(bad) == 0, f"{what}: {len(bad)} of {rel.size} above {tol}; worst {rel.max():.3e} at {np.unravel_index(rel.argmax(), rel.shape)}"


# Status bits that the GPU and the oracle define the same way: illegal image
# count, merged sectors (cap), grid edge, non-finite result.  (Non-convergence
# depends on each side's own iteration; table overflow exists on the GPU only.)
SHARED_BITS = 2 | 4 | 8 | 16


def assert_status(st, so, what=""):
    a = np.asarray(st).astype(np.int64) & SHARED_BITS
    b = np.asarray(so).astype(np.int64) & SHARED_BITS
    bad = np.argwhere(a != b)
    assert len(bad) == 0, f"{what}: status bits differ at {bad[:5].tolist()}: gpu {a[tuple(bad[0])]} oracle {b[tuple(bad[0])]}"


def test_point_source_binary(G, oracle_mod):
    import torch
    rng = np.random.default_rng(21)
    for q, s in [(1e-3, 1.0), (0.3, 0.8), (1e-5, 1.2)]:
        p = I.binary(q=q, s=s)
        w = rng.uniform(-0.3, 0.3, 300) + 1j * rng.uniform(-0.3, 0.3, 300)
        wd = torch.tensor(np.stack([w.real, w.imag], -1)[None], device="cuda")
        A, imgs, n, st = G.point_source(G.params_to_device([p]), wd, G.grid_from_dict(I.grid(), 2), 2)
        Ao, no, zo, so = oracle_mod.point_source(p, I.grid(), w)
        A = A.cpu().numpy()[0]; n = n.cpu().numpy()[0]; imgs = imgs.cpu().numpy()[0]
        np.testing.assert_array_equal(n, no)
        np.testing.assert_allclose(A, Ao, rtol=1e-9)
        for i in range(len(w)):
            zg = imgs[i, : n[i], 0] + 1j * imgs[i, : n[i], 1]
            for z in zo[i, : no[i]]:
                assert np.min(np.abs(zg - z)) < 1e-9


def test_point_source_triple(G, oracle_mod):
    import torch
    rng = np.random.default_rng(22)
    p = I.triple()
    w = rng.uniform(-0.2, 0.2, 200) + 1j * rng.uniform(-0.2, 0.2, 200)
    wd = torch.tensor(np.stack([w.real, w.imag], -1)[None], device="cuda")
    A, imgs, n, st = G.point_source(G.params_to_device([p]), wd, G.grid_from_dict(I.grid(), 3), 3)
    Ao, no, zo, so = oracle_mod.point_source(p, I.grid(), w)
    np.testing.assert_array_equal(n.cpu().numpy()[0], no)
    np.testing.assert_allclose(A.cpu().numpy()[0], Ao, rtol=1e-9)


def test_caustic_crossing_curve(G, oracle_mod):
    """Binary s=1, q=1e-3, rho=1e-3, u=0.5: all 500 epochs, 64 x 256 grid."""
    params, t = I.caustic_crossing_binary()
    g = I.grid()
    A, st = run_gpu(G, params, t, g)
    Ao, so = oracle_mod.magnification(params, t, g)
    assert_parity(A, Ao, what="caustic crossing")
    assert_status(st, so, what="caustic crossing")
    assert not np.any(st & 16)


def test_binary_batch_small(G, oracle_mod):
    """Five sets from the 64-set batch distribution with a ragged epoch count
    (several blocks, partial chunks), epochs concentrated near the lens."""
    params, t = I.binary_batch(n_sets=5, n_epochs=173, seed=12)
    t = np.stack([np.sort(np.random.default_rng(i).uniform(-3, 3, 173)) for i in range(5)])
    g = I.grid()
    A, st = run_gpu(G, params, t, g)
    Ao, so = oracle_mod.magnification(params, t, g)
    assert_parity(A, Ao, what="binary batch")
    assert_status(st, so, what="binary batch")


def test_triple_curve(G, oracle_mod):
    """Triple lens q2=1e-3, q3=3e-4: 250 of the 2000 epochs."""
    params, t = I.triple_curve()
    t = t[:, ::8]
    g = I.grid()
    A, st = run_gpu(G, params, t, g)
    Ao, so = oracle_mod.magnification(params, t, g)
    assert_parity(A, Ao, what="triple")
    assert_status(st, so, what="triple")


def test_uniform_and_grid_variants(G, oracle_mod):
    """Uniform rule; non-power-of-two grids (ragged rows and segments)."""
    params, t = I.caustic_crossing_binary(n_epochs=60)
    for g in (I.grid(uniform=1), I.grid(n_r=37, n_theta=500), I.grid(n_r=20, n_theta=1100, n_limb=300)):
        A, st = run_gpu(G, params, t, g)
        Ao, so = oracle_mod.magnification(params, t, g)
        assert_parity(A, Ao, what=str(g))
        assert_status(st, so, what=str(g))


def test_ring_and_origin_cases(G, oracle_mod):
    """Source over a single lens (ring image, full-circle sector and r-gap
    filling) and an equal-mass binary whose origin maps inside the source."""
    ring = I.binary(q=1e-5, s=10.0, u0=0.0, alpha=0.0, t0=0.0, tE=1.0, rho=0.01, u1=0.5)
    t = np.linspace(-0.02, 0.02, 21)
    A, _ = run_gpu(G, [ring], t, I.grid())
    Ao, _ = oracle_mod.magnification([ring], t, I.grid())
    assert_parity(A, Ao, what="ring")
    eq = I.binary(q=1.0, s=1.0, u0=0.0, alpha=0.3, t0=0.0, tE=1.0, rho=0.05, u1=0.5)
    t = np.linspace(-0.04, 0.04, 9)
    A, _ = run_gpu(G, [eq], t, I.grid())
    Ao, _ = oracle_mod.magnification([eq], t, I.grid())
    assert_parity(A, Ao, what="origin inside")


def test_full_batch_sampled(G, oracle_mod):
    """The 64 sets x 10,000 epochs batch in the benchmark's launch
    configuration; the oracle checks 160 sampled epochs (the highest-
    magnification epoch of each set plus random ones)."""
    params, t = I.binary_batch()
    g = I.grid()
    A, st = run_gpu(G, params, t, g)
    rng = np.random.default_rng(99)
    picks = [(s, int(np.argmax(A[s]))) for s in range(len(params))]
    picks += [(int(rng.integers(len(params))), int(rng.integers(t.shape[1]))) for _ in range(96)]
    for s, e in picks:
        Ao, _ = oracle_mod.magnification([params[s]], [t[s, e]], g)
        assert abs(A[s, e] / Ao[0, 0] - 1.0) <= TOL, (s, e, A[s, e], Ao[0, 0])


@pytest.fixture(scope="module")
def headline(G):
    """The benchmark's headline launch: the 64 x 10,000 batch in one call at
    n_r = 1024, n_theta = 2048 (warm starts along each light curve)."""
    params, t = I.binary_batch()
    g = I.grid(n_r=1024, n_theta=2048)
    A, st = run_gpu(G, params, t, g)
    return params, t, g, A, st


def test_headline_grid_full_batch_sampled(headline, oracle_mod):
    """The oracle recomputes 24 sampled epochs of the headline launch on the
    same grid: the highest-magnification epoch of 8 sets and 16 random ones."""
    params, t, g, A, st = headline
    assert np.all(np.isfinite(A))
    rng = np.random.default_rng(7)
    picks = [(s, int(np.argmax(A[s]))) for s in range(0, len(params), 8)]
    picks += [(int(rng.integers(len(params))), int(rng.integers(t.shape[1]))) for _ in range(16)]
    for s, e in picks:
        Ao, so = oracle_mod.magnification([params[s]], [t[s, e]], g)
        assert abs(A[s, e] / Ao[0, 0] - 1.0) <= TOL, (s, e, A[s, e], Ao[0, 0])
        assert (int(st[s, e]) & SHARED_BITS) == (int(so[0, 0]) & SHARED_BITS), (s, e, st[s, e], so[0, 0])


def test_headline_merged_sector_epochs(G, headline, oracle_mod):
    """Every epoch of the headline launch whose sectors reached the cap and
    were merged (ICRS_ST_SECTCAP), the epochs where the sector rule is most
    sensitive to the image-limb points: each against the oracle (cold roots)
    at 1e-5 with the same status bits, and the indexed launch of just those
    epochs (roots warm-started from an unrelated epoch) equal to the full
    launch to 1e-7."""
    import torch
    params, t, g, A, st = headline
    idx = [(int(s), int(e)) for s, e in np.argwhere(st & 4)]
    assert idx, "the headline workload has merged-sector epochs"
    for s, e in idx:
        Ao, so = oracle_mod.magnification([params[s]], [t[s, e]], g)
        assert abs(A[s, e] / Ao[0, 0] - 1.0) <= TOL, (s, e, A[s, e], Ao[0, 0])
        assert (int(st[s, e]) & SHARED_BITS) == (int(so[0, 0]) & SHARED_BITS), (s, e, st[s, e], so[0, 0])
    S, E = t.shape
    pd = G.params_to_device(params)
    tt = torch.tensor(t, device="cuda")
    items = torch.tensor([s * E + e for s, e in idx], dtype=torch.int32, device="cuda")
    Ai = torch.full((S, E), float("nan"), dtype=torch.float64, device="cuda")
    sti = torch.zeros((S, E), dtype=torch.int32, device="cuda")
    G.magnification_indexed(pd, tt, G.grid_from_dict(g, 2), items, len(idx), Ai, sti)
    Ai = Ai.cpu().numpy()
    for s, e in idx:
        assert abs(Ai[s, e] / A[s, e] - 1.0) <= 1e-7, (s, e, Ai[s, e], A[s, e])


def test_wide_theta_grid(G, oracle_mod):
    """n_theta = 8192 at N_limb = 500 (the paper's finest angular resolution
    is 8000): the 768-thread binary layout does not fit in shared memory
    there, so the launch takes the 512-thread instantiation.  8 epochs of the
    caustic-crossing curve against the oracle on the same grid."""
    params, t = I.caustic_crossing_binary(n_epochs=8)
    g = I.grid(n_r=64, n_theta=8192)
    A, st = run_gpu(G, params, t, g)
    Ao, so = oracle_mod.magnification(params, t, g)
    assert_parity(A, Ao, what="n_theta 8192")


def test_empty_and_invalid(G):
    import torch
    pd = G.params_to_device([I.binary()])
    t = torch.zeros((1, 0), dtype=torch.float64, device="cuda")
    A, st = G.magnification(pd, t, G.make_grid())
    assert A.shape == (1, 0)
    with pytest.raises(G.IcrsError):
        G.magnification(pd, torch.zeros((1, 3), dtype=torch.float64, device="cuda"), G.make_grid(n_theta=4))


def test_quadratic_limb_darkening_and_split_rule(G, oracle_mod):
    """Quadratic limb darkening (u2 = 0.25) on the caustic-crossing curve,
    with the literal per-point rule and the split-profile rule, and the
    linear law with the split rule: each against the oracle at 1e-5 with the
    same status bits.  The derivative entry points refuse the split rule."""
    import torch
    base, t = I.caustic_crossing_binary(n_epochs=60)
    for u2, split in ((0.25, 0), (0.25, 1), (0.0, 1)):
        params = [dict(base[0], u2=u2)]
        g = I.grid(ld_split=split)
        A, st = run_gpu(G, params, t, g)
        Ao, so = oracle_mod.magnification(params, t, g)
        assert_parity(A, Ao, what=f"u2={u2} split={split}")
        assert_status(st, so, what=f"u2={u2} split={split}")
    pd = G.params_to_device(base)
    tt = torch.tensor(t, device="cuda")
    with pytest.raises(G.IcrsError):
        G.magnification_vjp(pd, tt, G.grid_from_dict(I.grid(ld_split=1), 2), torch.ones_like(tt))


@pytest.mark.parametrize("coef", [(0.6, 0.0, 0.0, 0.0), (0.3, 0.2, -0.1, 0.05), (0.0, 0.3, 0.0, 0.2)])
def test_power_series_profiles(G, oracle_mod, coef):
    """The power-series law in mu^(1/2) (coefficients a1..a4 on top of u1 =
    0.2; half-integer powers take the kernel's generic instantiation and its
    paired half-power sweep, integer ones the linear instantiation) on the
    caustic-crossing curve and on 64 batch epochs,
    with the literal and the split-profile rules: against the oracle at 1e-5
    with the same status bits."""
    a = dict(a1=coef[0], a2=coef[1], a3=coef[2], a4=coef[3])
    base, t = I.caustic_crossing_binary(n_epochs=40)
    bp, bt = I.binary_batch()
    sel = [(s_, e) for s_ in range(0, 64, 8) for e in range(0, 10000, 1250)]
    cases = [([dict(base[0], u1=0.2, **a)], t),
             ([dict(bp[s_], u1=0.2, **a) for s_, _ in sel], np.array([[bt[s_, e]] for s_, e in sel]))]
    for split in (0, 1):
        g = I.grid(ld_split=split)
        for params, tt in cases:
            A, st = run_gpu(G, params, tt, g)
            Ao, so = oracle_mod.magnification(params, tt, g)
            assert_parity(A, Ao, what=f"a={coef} split={split}")
            assert_status(st, so, what=f"a={coef} split={split}")


@pytest.mark.parametrize("spot", [(0.3, -0.2, 0.4, 0.7), (-0.5, 0.1, 0.3, 0.5), (0.0, 0.0, 1.0, 0.6)])
def test_spotted_sources(G, oracle_mod, spot):
    """A circular spot (centre, radius in rho, contrast) on a linearly
    limb-darkened source, on the caustic-crossing curve and on 64 batch
    epochs (one with a power-series law too): against the oracle at 1e-5
    with the same status bits; a spot outside the disk gives NaN and
    ICRS_ST_NAN on both sides."""
    sx, sy, sr, sc = spot
    sp = dict(spot_x=sx, spot_y=sy, spot_r=sr, spot_c=sc)
    base, t = I.caustic_crossing_binary(n_epochs=40)
    bp, bt = I.binary_batch()
    sel = [(s_, e) for s_ in range(0, 64, 8) for e in range(0, 10000, 1250)]
    cases = [([dict(base[0], **sp)], t),
             ([dict(bp[s_], **sp) for s_, _ in sel], np.array([[bt[s_, e]] for s_, e in sel])),
             ([dict(base[0], a1=0.3, a3=-0.1, **sp)], t[:, ::4])]
    g = I.grid()
    for params, tt in cases:
        A, st = run_gpu(G, params, tt, g)
        Ao, so = oracle_mod.magnification(params, tt, g)
        assert_parity(A, Ao, what=f"spot {spot}")
        assert_status(st, so, what=f"spot {spot}")
    bad = [dict(base[0], spot_x=0.8, spot_y=0.0, spot_r=0.3, spot_c=0.5)]
    A, st = run_gpu(G, bad, t[:, :3], g)
    Ao, so = oracle_mod.magnification(bad, t[:, :3], g)
    assert np.all(np.isnan(A)) and np.all(np.isnan(Ao))
    assert np.all(st & 16) and np.all(so & 16)


def test_qualification_sample_at_headline_grid(G):
    """The 512-epoch qualification sample of the batch (peak epochs, random
    epochs, small sources at moderate magnification, sources inside a
    caustic; tests/golden/batch_qualification.json, written by a script that
    calls only the oracle) at the headline grid, one launch with one set per
    epoch (cold roots): every epoch against the stored oracle value on the
    same grid at 1e-5."""
    import json
    import os
    import torch
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "batch_qualification.json")
    gold = json.load(open(path))
    params, t = I.binary_batch()
    rows = gold["epochs"]
    g = I.grid(**gold["grids"][0])
    ps = [params[r["set"]] for r in rows]
    tt = np.array([[t[r["set"], r["epoch"]]] for r in rows])
    A, st = run_gpu(G, ps, tt, g)
    Ao = np.array([[r["A"][0]] for r in rows])
    so = np.array([[r["status"][0]] for r in rows])
    assert_parity(A, Ao, what="qualification sample")
    assert_status(st, so, what="qualification sample")


def test_interval_first_edge_epochs(G):
    """Five epochs of the 5000 x 2000 scoring batch whose lowest image angle
    lies within 1e-7 rad above the first edge of its angular interval
    (tests/golden/interval_edge_epochs.json, written by a script that calls
    only the oracle and checks that property): the FP32 angle of that point
    can fall below the edge while its FP64 angle bins it inside, and the
    sector must still span the whole image.  Each epoch against the stored
    oracle value at 1e-5 with the same status bits."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "interval_edge_epochs.json")
    gold = json.load(open(path))
    params, t = I.binary_batch(**gold["batch"])
    rows = gold["epochs"]
    g = I.grid(**gold["grid"])
    ps = [params[r["set"]] for r in rows]
    tt = np.array([[t[r["set"], r["epoch"]]] for r in rows])
    A, st = run_gpu(G, ps, tt, g)
    Ao = np.array([[r["A"]] for r in rows])
    so = np.array([[r["status"]] for r in rows])
    assert_parity(A, Ao, what="interval first-edge epochs")
    assert_status(st, so, what="interval first-edge epochs")


def test_near_critical_pair_epochs(G):
    """Four epochs of the 5000 x 2000 scoring batch with a limb point just
    inside a fold caustic, whose close image pair (up to 2.6e-2 apart) the
    FP32 polynomial can round into a pair of false roots
    (tests/golden/near_critical_epochs.json, oracle values).  Each epoch
    cold (one launch, one set per epoch) and at the end of its light curve
    run from the first epoch (the set repeated once per SM, so that every
    block runs the whole curve in order with warm-started roots): both
    against the stored oracle value at 1e-5 with the same status bits."""
    import json
    import os
    import torch
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "near_critical_epochs.json")
    gold = json.load(open(path))
    params, t = I.binary_batch(**gold["batch"])
    rows = gold["epochs"]
    g = I.grid(**gold["grid"])
    Ao = np.array([[r["A"]] for r in rows])
    so = np.array([[r["status"]] for r in rows])
    A, st = run_gpu(G, [params[r["set"]] for r in rows], np.array([[t[r["set"], r["epoch"]]] for r in rows]), g)
    assert_parity(A, Ao, what="near-critical epochs, cold")
    assert_status(st, so, what="near-critical epochs, cold")
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    for r, a_o, s_o in zip(rows, Ao[:, 0], so[:, 0]):
        s_, e = r["set"], r["epoch"]
        Aw, sw = run_gpu(G, [params[s_]] * nsm, np.tile(t[s_, :e + 1], (nsm, 1)), g)
        assert_parity(Aw[:, e:e + 1], np.full((nsm, 1), a_o), what=f"near-critical epoch {s_}/{e}, warm")
        assert_status(sw[:, e:e + 1], np.full((nsm, 1), s_o), what=f"near-critical epoch {s_}/{e}, warm")


def test_triple_at_qualified_grid(G):
    """The triple-lens curve (rho = 5e-4) at 1024 x 2048 with N_limb = 500 (it
    fits in shared memory since the per-sector offset table holds at most
    256 columns): 32 epochs (the 16 of highest point-source magnification and
    16 spread along the curve, tests/golden/triple_qualification.json) in one
    launch, each against the stored oracle value on the same grid at 1e-5,
    and within 1e-4 of the oracle at 4096 x 8192 up to that reference's own
    Richardson bound."""
    import json
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "triple_qualification.json")
    gold = json.load(open(path))
    params, t = I.triple_curve()
    rows = gold["epochs"]
    g = I.grid(**gold["grids"][0])
    tt = np.array([[t[0, r["epoch"]] for r in rows]])
    A, st = run_gpu(G, params, tt, g)
    Ao = np.array([[r["A"][0] for r in rows]])
    so = np.array([[r["status"][0] for r in rows]])
    assert_parity(A, Ao, what="triple at 1024 x 2048")
    assert_status(st, so, what="triple at 1024 x 2048")
    ref = np.array([r["A"][-1] for r in rows])
    bound = np.abs(np.array([r["A"][-1] / r["A"][-2] - 1.0 for r in rows]))
    err = np.abs(A[0] / ref - 1.0)
    assert np.all(err <= 1e-4 + bound), (err.max(), bound[err.argmax()])


@pytest.mark.parametrize("q", [1e-5, 1e-3, 1e-1])
def test_root_stage_error_of_fp32_coefficients(G, oracle_mod, q):
    """The root stage forms the polynomial coefficients in FP32 (about the
    lightest lens) and refines each image by a double-float Newton step, with
    FP64 fallbacks.  Its image-limb points (r, theta) against the oracle's
    FP64 ones, for a source crossing the central caustic (8 epochs, 500 limb
    points each): same image count at every limb point, and positions equal
    to the FP32 rounding of the FP64 values (relative 2^-23) -- the sector
    bounds are then taken from FP64-polished or double-float values."""
    import torch
    p = I.binary(q=q, s=1.0, rho=1e-3, u0=0.0, alpha=0.3, t0=0.0, tE=20.0)
    t = np.linspace(-0.03, 0.03, 8)
    g = I.grid()
    pd = G.params_to_device([p])
    tt = torch.tensor(t[None, :], device="cuda")
    _, _, _, _, pts = G.magnification_diag(pd, tt, G.grid_from_dict(g, 2), points=True)
    pts = pts.cpu().numpy()[0]
    worst = 0.0
    for e in range(len(t)):
        lp = oracle_mod.limb_points(p, t[e], g)          # [N_limb, 5, (r, theta, valid)]
        gp = pts[e].reshape(lp.shape[0], 5, 4)
        for k in range(lp.shape[0]):
            vo = lp[k][lp[k, :, 2] > 0][:, :2]
            vg = gp[k][(gp[k, :, 2].astype(int) & 1) > 0][:, :2].astype(np.float64)
            assert len(vo) == len(vg), (e, k, len(vo), len(vg))
            zo = vo[:, 0] * np.exp(1j * vo[:, 1])
            zg = vg[:, 0] * np.exp(1j * vg[:, 1])
            for z in zo:
                d = np.min(np.abs(zg - z)) / max(1.0, abs(z))
                worst = max(worst, d)
    print(f"q={q}: worst image-limb point error {worst:.2e} (relative to max(1, |z|))")
    assert worst <= 4 * 2.0 ** -23
