"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1803_02132_gb300 as bisp  # noqa: E402
import synthcat  # noqa: E402
from oracle import estimator as E  # noqa: E402

# tolerance: per multipole, max relative error <= 1e-4 over bins with
# |B| > 1% of the multipole's maximum |B|
TOL = 1e-4


def rel_err(gpu, ref):
    """max relative error over bins above 1% of the multipole's max |ref|, per multipole."""
    out = []
    for g, r in zip(gpu, ref):
        m = np.abs(r) > 0.01 * np.abs(r).max()
        out.append(float(np.max(np.abs(g[m] - r[m]) / np.abs(r[m]))) if m.any() else 0.0)
    return out


# bins below 1% of their multipole's maximum (cancellation) are held to this fraction of that
# maximum instead: the shell sums of the shot-noise terms carry FP32 per-mode rounding of ~1e-6 of
# each sum, and a shot-noise bin is a difference of such sums
FLOOR = 1e-5


def assert_close(gpu, ref, tol=TOL, what=""):
    errs = rel_err(gpu, ref)
    assert max(errs) <= tol, f"{what}: max rel err per multipole {errs}"
    for i, (g, r) in enumerate(zip(gpu, ref)):
        scale = np.abs(r).max()
        bad = np.abs(g - r) > np.maximum(tol * np.abs(r), FLOOR * scale)
        worst = float(np.max(np.abs(g - r)) / scale) if scale > 0 else 0.0
        assert not bad.any(), (f"{what}: multipole {i}: {int(bad.sum())} bins beyond max(tol |ref|, {FLOOR} max|ref|); "
                               f"max |err| / max|ref| = {worst:.2e}")


def _plan(p, **kw):
    return bisp.Plan(nmesh=p.N, box_len=p.L, k_edges=p.edges, ells=p.ells, los=p.los, observer=p.observer,
                     mas=p.mas, interlace=p.interlace, fkp_P0=p.P0, want_window=p.window, **kw)


def _assign(plan, which, cat, device=True):
    xyz = cat["xyz"]
    w = cat.get("w")
    nb = cat.get("nbar")
    if device:
        t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
        plan.assign(which, t(xyz), t(w), t(nb))
    else:
        plan.assign(which, xyz, w, nb)


# ----------------------------------------------------------------------------------
def test_cell_order_bit_exact():
    N, L = 64, 1000.0
    rng = np.random.default_rng(11)
    xyz = (rng.random((100_000, 3)) * L).astype(np.float32)
    xyz[:2000] = np.round(xyz[:2000] / (L / N)) * np.float32(L / N)  # on nodes
    xyz[2000:4000] = (np.floor(xyz[2000:4000] / (L / N)) + 0.5) * np.float32(L / N)  # half-cell ties
    xyz = np.mod(xyz, np.float32(L)).astype(np.float32)
    xyz[xyz >= L] = 0
    xyz[4000:6000] = xyz[6000:8000]  # duplicate positions: stability
    xd = torch.from_numpy(xyz).cuda()
    for mas in (1, 2, 3):
        keys, order = bisp.cell_order(N, L, mas, xd)
        ok = E.cell_keys(xyz, N, L, mas)
        oo = np.argsort(ok, kind="stable")
        assert np.array_equal(order.cpu().numpy().astype(np.int64), oo)
        assert np.array_equal(keys.cpu().numpy().astype(np.int64), ok[oo])


def test_cell_order_empty_and_ragged():
    for n in (0, 1, 4095, 4097):
        xyz = (np.random.default_rng(n).random((n, 3)) * 100.0).astype(np.float32)
        if n == 0:
            continue
        keys, order = bisp.cell_order(16, 100.0, 3, torch.from_numpy(xyz).cuda())
        ok = E.cell_keys(xyz, 16, 100.0, 3)
        assert np.array_equal(order.cpu().numpy(), np.argsort(ok, kind="stable"))


@pytest.mark.parametrize("mas,interlace", [(1, False), (2, False), (3, True)])
def test_mesh_and_spectrum_parity(mas, interlace, monkeypatch):
    monkeypatch.setenv("BISP_DEBUG", "BISP_DEBUG_KEEP_MESH")
    N, L = 32, 500.0
    rng = np.random.default_rng(3)
    xyz = (rng.random((20_000, 3)) * L).astype(np.float32)
    w = (0.5 + rng.random(20_000)).astype(np.float32)
    p = E.Params(N=N, L=L, edges=[0.02, 0.05], ells=[(0, 0, 0)], mas=mas, interlace=interlace)
    with _plan(p) as plan:
        _assign(plan, 0, {"xyz": xyz, "w": w})
        mesh = plan.fetch_mesh(0, 0)
        ref = E.assign(xyz, w.astype(np.float64), N, L, mas, 0.0)
        assert np.max(np.abs(mesh - ref)) <= 2e-6 * np.max(np.abs(ref))
        spec = plan.fetch_spectrum(0, 0)
        refk = E.spectrum(p, xyz, w.astype(np.float64))[:, :, : N // 2]
        assert np.max(np.abs(spec - refk)) <= 1e-5 * np.max(np.abs(refk))


def _survey(seed, N, L, ngal, nran, P0=1e4):
    obs = (0.5 * L, 0.5 * L, -0.3 * L)
    gal, ran = synthcat.survey_catalogs(N, L, obs, ngal, nran, seed, r_min=0.35 * L, r_max=1.25 * L,
                                        half_angle_deg=40.0, r_mean=0.8 * L, sigma=0.2 * L)
    return gal, ran, obs


CASES = {
    "box_cic": dict(N=32, L=1000.0, mas=2, interlace=False, los="global", np_=30_000,
                    ells=[(0, 0, 0), (2, 0, 2), (1, 1, 0), (2, 2, 2)]),
    "box_tsc_ilv": dict(N=32, L=1000.0, mas=3, interlace=True, los="global", np_=30_000,
                        ells=[(0, 0, 0), (1, 1, 0), (2, 2, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2)]),
    "survey_local": dict(N=32, L=2000.0, mas=3, interlace=True, los="local", np_=20_000,
                         ells=[(0, 0, 0), (2, 0, 2), (1, 1, 2)]),
}


@pytest.mark.parametrize("case", list(CASES))
def test_estimator_parity_small(case):
    c = CASES[case]
    N, L = c["N"], c["L"]
    kf = 2 * np.pi / L
    edges = kf * np.array([1.0, 2.5, 4.0, 5.5, 7.0, 8.5, 11.0, 15.5])  # 7 bins, last one ragged
    if c["los"] == "global":
        gal = {"xyz": synthcat.periodic_catalog(N, L, c["np_"], seed=100 + N)}
        ran = None
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="global", mas=c["mas"], interlace=c["interlace"])
    else:
        gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="local", observer=obs, mas=c["mas"],
                     interlace=c["interlace"], P0=1e4, window=True)
    ref = E.measure(p, gal, ran)
    with _plan(p) as plan:
        _assign(plan, 0, gal)
        if ran is not None:
            _assign(plan, 1, ran)
        out = plan.measure()
        out2 = plan.measure()
        info = plan.info()
    assert info["norm_I"] == pytest.approx(ref["I"], rel=1e-6)
    assert np.array_equal(out["nmodes"], ref["nmodes"])
    assert_close(out["B"], ref["B"], what="B")
    assert_close(out["shot"], ref["shot"], what="shot")
    assert np.array_equal(out["B"], out2["B"])  # bitwise reproducible
    if ran is not None:
        assert_close(out["window"], ref["window"], what="window")
        assert_close(out["window_shot"], ref["window_shot"], what="window shot")


@pytest.mark.parametrize("case,ells", [("survey_local", None),
                                       ("box_cic", [(0, 0, 0), (2, 0, 2), (1, 1, 0)])])
def test_estimator_parity_tcgen05(case, ells, monkeypatch):
    """The opt-in tcgen05 contraction kernel against the oracle (jobs of at most 8 terms on
    at most 4 bare components: the survey set B000, B202, B112 and a box set)."""
    monkeypatch.setenv("BISP_PAIR_KERNEL", "tcgen05")
    c = CASES[case]
    N, L = c["N"], c["L"]
    ells = ells or c["ells"]
    kf = 2 * np.pi / L
    edges = kf * np.array([1.0, 2.5, 4.0, 5.5, 7.0, 8.5, 11.0, 15.5])
    if c["los"] == "global":
        gal = {"xyz": synthcat.periodic_catalog(N, L, c["np_"], seed=100 + N)}
        ran = None
        p = E.Params(N=N, L=L, edges=edges, ells=ells, los="global", mas=c["mas"], interlace=c["interlace"])
    else:
        gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
        p = E.Params(N=N, L=L, edges=edges, ells=ells, los="local", observer=obs, mas=c["mas"],
                     interlace=c["interlace"], P0=1e4, window=True)
    ref = E.measure(p, gal, ran)
    with _plan(p) as plan:
        _assign(plan, 0, gal)
        if ran is not None:
            _assign(plan, 1, ran)
        out = plan.measure()
        out2 = plan.measure()
        info = plan.info()
    assert info["pair_kernel"] == 2
    assert_close(out["B"], ref["B"], what="B")
    assert_close(out["shot"], ref["shot"], what="shot")
    assert np.array_equal(out["B"], out2["B"])
    if ran is not None:
        assert_close(out["window"], ref["window"], what="window")
        assert_close(out["window_shot"], ref["window_shot"], what="window shot")


@pytest.mark.parametrize("case,block", [("box_cic", 0), ("box_tsc_ilv", 0), ("survey_local", 0),
                                        ("survey_local", 3)])
def test_estimator_parity_fp64(case, block, monkeypatch):
    """The plain FP64 form (cuFFT Z2D fields, one FP64 mesh sum per bin pair and 3j term)
    against the oracle and against the fused FP32 path; block > 0 holds shell fields for
    blocks of that many bins (7 bins: a ragged last block)."""
    if block:
        monkeypatch.setenv("BISP_FP64_BLOCK_BINS", str(block))
    else:
        monkeypatch.delenv("BISP_FP64_BLOCK_BINS", raising=False)
    c = CASES[case]
    N, L = c["N"], c["L"]
    kf = 2 * np.pi / L
    edges = kf * np.array([1.0, 2.5, 4.0, 5.5, 7.0, 8.5, 11.0, 15.5])
    if c["los"] == "global":
        gal = {"xyz": synthcat.periodic_catalog(N, L, c["np_"], seed=100 + N)}
        ran = None
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="global", mas=c["mas"], interlace=c["interlace"])
    else:
        gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="local", observer=obs, mas=c["mas"],
                     interlace=c["interlace"], P0=1e4, window=True)
    ref = E.measure(p, gal, ran)
    outs = {}
    for prec in ("fp64", "fp32"):
        with _plan(p, precision=prec) as plan:
            _assign(plan, 0, gal)
            if ran is not None:
                _assign(plan, 1, ran)
            outs[prec] = plan.measure()
            if prec == "fp64":
                again = plan.measure()
                assert plan.info()["pair_kernel"] == 3
                assert np.array_equal(outs[prec]["B"], again["B"])  # fixed-order sums
    o64, o32 = outs["fp64"], outs["fp32"]
    assert np.array_equal(o64["nmodes"], ref["nmodes"])
    keys = ["B", "shot"] + (["window", "window_shot"] if ran is not None else [])
    for k in keys:
        assert_close(o64[k], ref[k], what=f"fp64 {k}")
        assert_close(o32[k], o64[k], what=f"fp32 vs fp64 {k}")


@pytest.mark.parametrize("case,block,nbins", [("survey_local", 3, 7), ("box_tsc_ilv", 2, 7), ("box_cic", 0, 34)])
def test_estimator_parity_blocked(case, block, nbins, monkeypatch):
    """Shell fields held for blocks of bins (two blocks resident, one pair launch per union):
    forced blocks of 3 (7 bins: a one-bin last block) and 2, and 34 bins (more than one pair
    launch covers: blocks of 16), against the oracle and against the unblocked path."""
    c = CASES[case]
    N, L = c["N"], c["L"]
    kf = 2 * np.pi / L
    edges = kf * (np.array([1.0, 2.5, 4.0, 5.5, 7.0, 8.5, 11.0, 15.5]) if nbins == 7
                  else np.linspace(1.0, 15.5, nbins + 1))
    if c["los"] == "global":
        gal = {"xyz": synthcat.periodic_catalog(N, L, c["np_"], seed=100 + N)}
        ran = None
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="global", mas=c["mas"], interlace=c["interlace"])
    else:
        gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="local", observer=obs, mas=c["mas"],
                     interlace=c["interlace"], P0=1e4, window=True)
    ref = E.measure(p, gal, ran)
    outs = {}
    for blocked in (True, False):
        if blocked and block:
            monkeypatch.setenv("BISP_BLOCK_BINS", str(block))
        else:
            monkeypatch.delenv("BISP_BLOCK_BINS", raising=False)
        if not blocked and nbins > 32:
            continue
        with _plan(p) as plan:
            _assign(plan, 0, gal)
            if ran is not None:
                _assign(plan, 1, ran)
            outs[blocked] = plan.measure()
            assert plan.info()["pair_kernel"] == 1
    assert np.array_equal(outs[True]["nmodes"], ref["nmodes"])
    keys = ["B", "shot"] + (["window", "window_shot"] if ran is not None else [])
    for k in keys:
        assert_close(outs[True][k], ref[k], what=f"blocked {k}")
        if False in outs:
            assert_close(outs[True][k], outs[False][k], tol=1e-6, what=f"blocked vs unblocked {k}")


@pytest.mark.parametrize("case,r0", [("box_tsc_ilv", False), ("survey_local", False), ("survey_local", True)])
def test_threept_parity(case, r0, monkeypatch):
    """Three-point-function multipoles zeta and window multipoles Q (Sec. 4.3, Sec. 6.1)
    against the oracle: r-bins of mesh separations (a first bin [0, H/2) holds s = 0 only),
    shot noise on r_a = r_b, separation counts exact."""
    from oracle import threept as T

    monkeypatch.delenv("BISP_BLOCK_BINS", raising=False)
    c = CASES[case]
    N, L = c["N"], c["L"]
    H = L / N
    edges = H * np.array(([0.0, 0.5] if r0 else [0.9]) + [1.5, 2.05, 2.95, 4.1, 6.0, 8.5])
    if c["los"] == "global":
        gal = {"xyz": synthcat.periodic_catalog(N, L, c["np_"], seed=100 + N)}
        ran = None
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="global", mas=c["mas"], interlace=c["interlace"])
    else:
        gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="local", observer=obs, mas=c["mas"],
                     interlace=c["interlace"], P0=1e4, window=True)
    ref = T.measure(p, gal, ran)
    with _plan(p, estimator="threept") as plan:
        _assign(plan, 0, gal)
        if ran is not None:
            _assign(plan, 1, ran)
        out = plan.measure()
        again = plan.measure()
    assert np.array_equal(out["nmodes"], ref["nr"])
    assert np.array_equal(out["B"], again["B"])
    assert_close(out["B"], ref["zeta"], what="zeta")
    assert_close(out["shot"], ref["shot"], what="zeta shot")
    if ran is not None:
        assert_close(out["window"], ref["window"], what="Q")
        assert_close(out["window_shot"], ref["window_shot"], what="Q shot")


@pytest.mark.parametrize("case,block,estimator", [("survey_local", 3, "bispectrum"), ("box_cic", 2, "bispectrum"),
                                                  ("box_tsc_ilv", 0, "threept")])
def test_diagonal_only(case, block, estimator, monkeypatch):
    """diagonal_only: the k1 = k2 (r1 = r2) outputs match the oracle, every other output is NaN;
    with blocks of bins each block is measured alone."""
    from oracle import threept as T

    if block:
        monkeypatch.setenv("BISP_BLOCK_BINS", str(block))
    else:
        monkeypatch.delenv("BISP_BLOCK_BINS", raising=False)
    c = CASES[case]
    N, L = c["N"], c["L"]
    three = estimator == "threept"
    edges = (L / N * np.array([0.9, 1.5, 2.05, 2.95, 4.1, 6.0, 8.5]) if three
             else 2 * np.pi / L * np.array([1.0, 2.5, 4.0, 5.5, 7.0, 8.5, 11.0, 15.5]))
    if c["los"] == "global":
        gal = {"xyz": synthcat.periodic_catalog(N, L, c["np_"], seed=100 + N)}
        ran = None
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="global", mas=c["mas"], interlace=c["interlace"])
    else:
        gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="local", observer=obs, mas=c["mas"],
                     interlace=c["interlace"], P0=1e4, window=True)
    ref = T.measure(p, gal, ran) if three else E.measure(p, gal, ran)
    with _plan(p, estimator=estimator, diagonal_only=True) as plan:
        _assign(plan, 0, gal)
        if ran is not None:
            _assign(plan, 1, ran)
        out = plan.measure()
    keys = [("B", "zeta" if three else "B"), ("shot", "shot")]
    if ran is not None:
        keys += [("window", "window"), ("window_shot", "window_shot")]
    nb = len(edges) - 1
    off = ~np.eye(nb, dtype=bool)
    for k, rk in keys:
        d = np.diagonal(out[k], axis1=1, axis2=2)
        assert_close(d, np.diagonal(ref[rk], axis1=1, axis2=2), what=f"diagonal {k}")
        assert np.all(np.isnan(out[k][:, off]))


def test_default_pair_kernel_is_mma_sync(monkeypatch):
    monkeypatch.delenv("BISP_PAIR_KERNEL", raising=False)
    c = CASES["box_cic"]
    N, L = c["N"], c["L"]
    gal = {"xyz": synthcat.periodic_catalog(N, L, c["np_"], seed=100 + N)}
    edges = 2 * np.pi / L * np.array([1.0, 2.5, 4.0, 5.5])
    p = E.Params(N=N, L=L, edges=edges, ells=[(0, 0, 0)], los="global", mas=2, interlace=False)
    with _plan(p) as plan:
        _assign(plan, 0, gal)
        plan.measure()
        assert plan.info()["pair_kernel"] == 1


def test_measure_batch_matches_single_measures():
    """bisp_measure_batch over independent realisations on meshes of two sizes (measured
    concurrently by worker threads) gives each plan's bisp_measure result exactly, and reports a
    failing plan by index."""
    L = 1000.0
    kf = 2 * np.pi / L
    edges = kf * np.array([1.0, 2.5, 4.0, 5.5, 7.0])
    plans = []
    try:
        for seed, N in ((21, 32), (22, 64), (23, 32), (24, 64), (25, 32)):
            p = E.Params(N=N, L=L, edges=edges, ells=[(0, 0, 0), (2, 0, 2)], los="global", mas=3, interlace=True)
            pl = _plan(p)
            _assign(pl, 0, {"xyz": synthcat.periodic_catalog(N, L, 20_000, seed=seed)})
            plans.append(pl)
        single = [pl.measure() for pl in plans]
        for _ in range(2):
            batch = bisp.measure_batch(plans)
            for a, b in zip(single, batch):
                for k in ("B", "shot", "nmodes"):
                    assert np.array_equal(a[k], b[k])
        p = E.Params(N=32, L=L, edges=edges, ells=[(0, 0, 0), (2, 0, 2)], los="global", mas=3, interlace=True)
        empty = _plan(p)
        plans.insert(3, empty)
        with pytest.raises(bisp.BispError, match="BISP_ESTATE.*plan 3"):
            bisp.measure_batch(plans)
        with pytest.raises(bisp.BispError, match="BISP_EINVAL.*repeats"):
            bisp.measure_batch([plans[0], plans[0]])
    finally:
        for pl in plans:
            pl.close()


def test_two_plans_from_two_host_threads():
    """Two plans (a local-line-of-sight survey with window and a periodic box, different meshes)
    driven at the same time from two host threads on their own streams give exactly the results
    of measuring each alone: no launch of one plan reads the other's job tables."""
    import threading

    c = CASES["survey_local"]
    kf = 2 * np.pi / c["L"]
    gal, ran, obs = _survey(7, c["N"], c["L"], c["np_"], 4 * c["np_"])
    ps = E.Params(N=c["N"], L=c["L"], edges=kf * np.array([1.0, 2.5, 4.0, 5.5, 7.0, 8.5]), ells=c["ells"],
                  los="local", observer=obs, mas=3, interlace=True, P0=1e4, window=True)
    Lb = 1000.0
    pb = E.Params(N=64, L=Lb, edges=2 * np.pi / Lb * np.array([1.0, 3.0, 5.0, 8.0, 12.0]),
                  ells=[(0, 0, 0), (2, 0, 2), (2, 2, 2)], los="global", mas=2, interlace=False)
    box = {"xyz": synthcat.periodic_catalog(64, Lb, 100_000, seed=31)}
    with _plan(ps) as a, _plan(pb) as b:
        _assign(a, 0, gal)
        _assign(a, 1, ran)
        _assign(b, 0, box)
        ref = [a.measure(), b.measure()]
        got = [[], []]

        def run(i, pl):
            for _ in range(4):
                got[i].append(pl.measure())

        th = [threading.Thread(target=run, args=(0, a)), threading.Thread(target=run, args=(1, b))]
        for t in th:
            t.start()
        for t in th:
            t.join()
    for i in range(2):
        assert len(got[i]) == 4
        for r in got[i]:
            for k in ref[i]:
                assert np.array_equal(r[k], ref[i][k]), (i, k)


def test_covariance_of_gpu_batch_matches_oracle():
    """Covariance of bispectrum multipoles over a batch of realisations measured on the GPU
    (bisp_measure_batch) and formed by bisp_covariance (Sec. 5.5, Eq. Covariance) against the
    oracle's covariance (oracle/stats.py) of the oracle's outputs on the same seeds; the
    Hartlap-scaled chi^2 of one realisation (App. E) against both."""
    from oracle import stats as ST

    N, L = 32, 1000.0
    kf = 2 * np.pi / L
    edges = kf * np.array([1.0, 2.5, 4.0, 5.5])
    p = E.Params(N=N, L=L, edges=edges, ells=[(0, 0, 0), (2, 0, 2)], los="global", mas=3, interlace=True)
    seeds = list(range(300, 320))
    cats = [{"xyz": synthcat.periodic_catalog(N, L, 20_000, seed=s)} for s in seeds]
    plans = []
    try:
        for cat in cats:
            pl = _plan(p)
            _assign(pl, 0, cat)
            plans.append(pl)
        outs = bisp.measure_batch(plans)
    finally:
        for pl in plans:
            pl.close()
    iu = np.triu_indices(len(edges) - 1)
    vec = lambda B: np.concatenate([B[0][iu], np.diagonal(B[1])])  # B000 on k1 <= k2, B202 on k1 = k2
    Xg = np.array([vec(o["B"]) for o in outs])
    Xo = np.array([vec(E.measure(p, cat, None)["B"]) for cat in cats])
    cg = bisp.covariance(Xg, n_par=2)
    mo, co, ro = ST.covariance(Xo)
    sd = np.sqrt(np.diag(co))
    assert np.all(np.abs(cg["mean"] - mo) <= 1e-4 * np.abs(Xo).max(axis=0))
    assert np.all(np.abs(cg["cov"] - co) <= 1e-3 * np.outer(sd, sd))
    assert np.all(np.abs(cg["corr"] - ro) <= 2e-3)
    x_th = mo
    assert bisp.chi2(cg["cov"], len(seeds), Xg[0], cg["mean"]) == pytest.approx(
        ST.chi2(co, len(seeds), Xo[0], x_th), rel=1e-2)
    assert cg["hartlap"] == pytest.approx(ST.hartlap(len(seeds), Xg.shape[1]), rel=1e-12)


def test_cfg1_box_64_cic_fp():
    # 1000 Mpc/h box, 64^3, 2e5 particles, CIC, no interlacing, global LOS, B000 and B202 on
    # 10 bins with edges 0.01..0.21 h/Mpc
    N, L = 64, 1000.0
    gal = {"xyz": synthcat.periodic_catalog(N, L, 200_000, seed=1000)}
    edges = np.linspace(0.01, 0.21, 11)
    p = E.Params(N=N, L=L, edges=edges, ells=[(0, 0, 0), (2, 0, 2)], los="global", mas=2, interlace=False)
    ref = E.measure(p, gal, None)
    with _plan(p) as plan:
        _assign(plan, 0, gal, device=False)   # host pointers through the C ABI
        out = plan.measure()
    assert_close(out["B"], ref["B"], what="B")
    assert_close(out["shot"], ref["shot"], what="shot")


def test_errors_are_reported():
    p = E.Params(N=16, L=100.0, edges=[0.1, 0.3], ells=[(0, 0, 0)], los="local", mas=3)
    with _plan(p) as plan:
        with pytest.raises(bisp.BispError) as e:
            plan.measure()
        assert e.value.status == bisp.BISP_ESTATE
        bad = np.array([[1.0, 2.0, 3.0], [np.nan, 1.0, 1.0], [150.0, 1.0, 1.0]], np.float32)
        with pytest.raises(bisp.BispError) as e:
            plan.assign(0, bad)
        assert e.value.status == bisp.BISP_EINVAL and "2 particles" in str(e.value)
        plan.assign(0, np.array([[1.0, 2.0, 3.0]], np.float32))
        with pytest.raises(bisp.BispError) as e:  # local LOS needs randoms
            plan.measure()
        assert e.value.status == bisp.BISP_ESTATE


HIGH_ELLS = [(4, 0, 4), (3, 1, 2), (2, 2, 4), (4, 4, 0)]


@pytest.mark.parametrize("los", ["global", "local"])
def test_estimator_parity_high_multipoles(los, monkeypatch):
    """Multipoles with l = 3 and 4, the largest the header admits (Table 1's selection rules):
    B404, B312, B224, B440; the local line of sight needs the L = 4 channels (15 delta n and 15 N
    meshes, deposited in groups) and contraction jobs split over several launches."""
    monkeypatch.delenv("BISP_BLOCK_BINS", raising=False)
    monkeypatch.delenv("BISP_PAIR_FP32", raising=False)
    c = CASES["box_tsc_ilv" if los == "global" else "survey_local"]
    N, L = c["N"], c["L"]
    edges = 2 * np.pi / L * np.array([1.0, 2.5, 4.0, 5.5, 7.0, 8.5, 11.0, 15.5])
    if los == "global":
        gal = {"xyz": synthcat.periodic_catalog(N, L, c["np_"], seed=100 + N)}
        ran = None
        p = E.Params(N=N, L=L, edges=edges, ells=HIGH_ELLS, los="global", mas=c["mas"], interlace=c["interlace"])
    else:
        gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
        p = E.Params(N=N, L=L, edges=edges, ells=HIGH_ELLS, los="local", observer=obs, mas=c["mas"],
                     interlace=c["interlace"], P0=1e4, window=True)
    ref = E.measure(p, gal, ran)
    with _plan(p) as plan:
        _assign(plan, 0, gal)
        if ran is not None:
            _assign(plan, 1, ran)
        out = plan.measure()
    assert_close(out["B"], ref["B"], what="B")
    assert_close(out["shot"], ref["shot"], what="shot")
    if ran is not None:
        assert_close(out["window"], ref["window"], what="window")
        assert_close(out["window_shot"], ref["window_shot"], what="window shot")


_SHAPE_REF = {}


@pytest.mark.parametrize("ksplit,ells,dual,tail", [("0", None, "-1", "1"), ("1", None, "-1", "1"),
                                                  ("2", None, "-1", "1"), ("0", None, "0", "1"),
                                                  ("0", None, "-1", "0"), ("1", [(0, 0, 0)], "-1", "1"),
                                                  ("2", [(0, 0, 0)], "-1", "1")])
def test_tma_contraction_launch_shapes(ksplit, ells, dual, tail, monkeypatch):
    """The TMA contraction at 25 bins, the headline workload's tile shape (two 16-row by four
    8-column tiles per term), on a small survey with window: the cell halves of a chunk split by
    the balancing rule, on one warp or on two (BISP_PAIR_KSPLIT), for the survey's five terms (two
    staged chunks) and for B000 alone (one term, three staged chunks); the unit-shell launch's
    ten terms (two G sets) in two-term warps by default and one term per warp with
    BISP_PAIR_DUAL=0; the 25th bin's column by FP32 FMAs by default and on the tensor cores with
    BISP_PAIR_TAIL=0; against the oracle."""
    monkeypatch.setenv("BISP_PAIR_KSPLIT", ksplit)
    monkeypatch.setenv("BISP_PAIR_DUAL", dual)
    monkeypatch.setenv("BISP_PAIR_TAIL", tail)
    monkeypatch.delenv("BISP_BLOCK_BINS", raising=False)
    c = CASES["survey_local"]
    N, L = c["N"], c["L"]
    ells = ells or c["ells"]
    edges = 2 * np.pi / L * np.linspace(1.0, 15.5, 26)
    key = tuple(ells)
    if key not in _SHAPE_REF:
        gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
        p = E.Params(N=N, L=L, edges=edges, ells=ells, los="local", observer=obs, mas=c["mas"],
                     interlace=c["interlace"], P0=1e4, window=True)
        _SHAPE_REF[key] = (p, gal, ran, E.measure(p, gal, ran))
    p, gal, ran, ref = _SHAPE_REF[key]
    with _plan(p) as plan:
        _assign(plan, 0, gal)
        _assign(plan, 1, ran)
        out = plan.measure()
        assert plan.info()["pair_kernel"] == 1
    for k in ("B", "shot", "window", "window_shot"):
        assert_close(out[k], ref[k], what=k)


@pytest.mark.parametrize("case", ["survey_local", "box_tsc_ilv"])
def test_fp32_fma_contraction_kernel(case, monkeypatch):
    """The FP32-FMA contraction (k_pair, forced with BISP_PAIR_FP32=1; otherwise used for jobs
    outside the tensor-core layout) against the oracle."""
    monkeypatch.setenv("BISP_PAIR_FP32", "1")
    monkeypatch.delenv("BISP_BLOCK_BINS", raising=False)
    c = CASES[case]
    N, L = c["N"], c["L"]
    edges = 2 * np.pi / L * np.array([1.0, 2.5, 4.0, 5.5, 7.0, 8.5, 11.0, 15.5])
    if c["los"] == "global":
        gal = {"xyz": synthcat.periodic_catalog(N, L, c["np_"], seed=100 + N)}
        ran = None
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="global", mas=c["mas"], interlace=c["interlace"])
    else:
        gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
        p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="local", observer=obs, mas=c["mas"],
                     interlace=c["interlace"], P0=1e4, window=True)
    ref = E.measure(p, gal, ran)
    with _plan(p) as plan:
        _assign(plan, 0, gal)
        if ran is not None:
            _assign(plan, 1, ran)
        out = plan.measure()
        assert plan.info()["pair_kernel"] == 0
    assert_close(out["B"], ref["B"], what="B")
    assert_close(out["shot"], ref["shot"], what="shot")
    if ran is not None:
        assert_close(out["window"], ref["window"], what="window")
        assert_close(out["window_shot"], ref["window_shot"], what="window shot")


@pytest.mark.parametrize("los_object", [1, 2])
def test_los_on_x1_x2(los_object, monkeypatch):
    """The line of sight on x1 or x2 (App. B): the y_L^{M*} weight on the k1 or k2 object, with the
    contraction over that object's (m, M) done in k space and the shot-noise terms following the
    weighted object, against oracle/los.py on the local-line-of-sight survey with window; the L = 0
    multipole does not depend on the choice."""
    from oracle import los as LS

    monkeypatch.delenv("BISP_BLOCK_BINS", raising=False)
    c = CASES["survey_local"]
    N, L = c["N"], c["L"]
    edges = 2 * np.pi / L * np.array([1.0, 2.5, 4.0, 5.5, 7.0, 8.5, 11.0, 15.5])
    ells = [(0, 0, 0), (2, 0, 2), (1, 1, 2), (2, 2, 2), (3, 1, 2)]
    gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
    p = E.Params(N=N, L=L, edges=edges, ells=ells, los="local", observer=obs, mas=c["mas"],
                 interlace=c["interlace"], P0=1e4, window=True)
    ref = LS.measure(p, gal, ran, los_object)
    with _plan(p, los_object=los_object) as plan:
        _assign(plan, 0, gal)
        _assign(plan, 1, ran)
        out = plan.measure()
        again = plan.measure()
    for k, rk in (("B", "B"), ("shot", "shot"), ("window", "window"), ("window_shot", "window_shot")):
        assert_close(out[k], ref[rk], what=f"x{los_object} {k}")
    assert np.array_equal(out["B"], again["B"])
    with _plan(p) as plan3:  # L = 0: the same for every choice
        _assign(plan3, 0, gal)
        _assign(plan3, 1, ran)
        o3 = plan3.measure()
    assert_close(out["B"][:1], o3["B"][:1], tol=1e-5, what="B000 x1/x2 vs x3")


def test_autotuned_zpass_groups_do_not_change_results(monkeypatch):
    """The autotuner picks the z pass's row groups per CTA by timing candidates on the plan's
    largest shell batch; every candidate computes the same fields, so measurements with the tuned
    value and with fixed values (BISP_ZGROUPS) are identical bit for bit."""
    c = CASES["survey_local"]
    N, L = c["N"], c["L"]
    edges = 2 * np.pi / L * np.array([1.0, 2.5, 4.0, 5.5, 7.0, 8.5, 11.0, 15.5])
    gal, ran, obs = _survey(7, N, L, c["np_"], 4 * c["np_"])
    p = E.Params(N=N, L=L, edges=edges, ells=c["ells"], los="local", observer=obs, mas=3, interlace=True, P0=1e4,
                 window=True)
    outs, groups = [], []
    for fixed in (None, "1", "2", "16"):
        if fixed:
            monkeypatch.setenv("BISP_ZGROUPS", fixed)
        else:
            monkeypatch.delenv("BISP_ZGROUPS", raising=False)
        with _plan(p) as plan:
            _assign(plan, 0, gal)
            _assign(plan, 1, ran)
            outs.append(plan.measure())
            groups.append(plan.info()["zpass_groups"])
    assert groups[0] > 0
    for o in outs[1:]:
        for k in ("B", "shot", "window", "window_shot"):
            assert np.array_equal(o[k], outs[0][k]), k
