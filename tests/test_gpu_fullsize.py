"""Parity at the full sizes of the benchmark workloads, in the launch configuration that
bench.py times: sampled outputs the FP64 oracle can compute one by one, and properties
that hold at any size."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import bench  # noqa: E402
import paper_1803_02132_gb300 as bisp  # noqa: E402
import synthcat  # noqa: E402
from oracle import estimator as E  # noqa: E402

TOL = 1e-4


def _dev(a):
    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _plan_for(w, **kw):
    args = dict(los="local" if w["kind"] == "survey" else "global", observer=w.get("observer", (0, 0, 0)),
                mas=w["mas"], interlace=w["interlace"], fkp_P0=w["P0"], want_window=w["window"])
    args.update(kw)
    return bisp.Plan(w["N"], w["L"], w["edges"], w["ells"], **args)


def test_box256_sampled_pairs_against_oracle():
    # 1000 Mpc/h box, 256^3, 4e6 particles, TSC + interlacing, six multipoles on 20 bins
    w = bench.WORKLOADS["box256"]
    gal, _ = bench.make_inputs(w, seed=1002)
    with _plan_for(w) as plan:
        plan.assign(bisp.DATA, _dev(gal["xyz"]))
        out = plan.measure()
    p = E.Params(N=w["N"], L=w["L"], edges=w["edges"], ells=w["ells"], los="global", mas=3, interlace=True)
    sd = E.catalogue_spectra(p, gal, None)["data"]
    samples = {(0, 0, 0): [(2, 17), (19, 19)], (1, 1, 0): [(5, 5)], (2, 0, 2): [(12, 4)],
               (1, 1, 2): [(9, 14)], (2, 2, 2): [(19, 19)], (2, 2, 0): [(0, 11)]}
    for mult, pairs in samples.items():
        im = w["ells"].index(mult)
        q = E.Params(N=p.N, L=p.L, edges=p.edges, ells=[mult], los="global", mas=3, interlace=True)
        raw = E.bispectrum_raw_fft(q, sd, pairs)[0]
        shot = E.shot_noise_fft(q, sd, pairs)[0]
        scale = np.abs(out["B"][im]).max()
        for b1, b2 in pairs:
            ref = raw[b1, b2] - shot[b1, b2]
            assert abs(out["shot"][im, b1, b2] - shot[b1, b2]) <= TOL * abs(shot[b1, b2]), (mult, b1, b2)
            # 1e-4 of the value, or 1e-5 of the multipole's largest |value| for bins in cancellation
            assert abs(out["B"][im, b1, b2] - ref) <= max(TOL * abs(ref), 1e-5 * scale), (
                mult, b1, b2, out["B"][im, b1, b2], ref, scale)


def _direct_dft(mesh, n_vecs, N):
    """sum_x m(x) e^{-2 pi i n.x / N} at a few integer wavevectors (separable contraction)."""
    x = np.arange(N)
    out = []
    for n in n_vecs:
        ez = np.exp(-2j * np.pi * n[2] * x / N)
        ey = np.exp(-2j * np.pi * n[1] * x / N)
        ex = np.exp(-2j * np.pi * n[0] * x / N)
        out.append(np.einsum("i,ijk,j,k->", ex, mesh, ey, ez, optimize=True))
    return np.array(out)


def test_survey512_full_size_spectra_and_properties():
    w = bench.WORKLOADS["survey512"]
    gal, ran = bench.make_inputs(w, seed=1002)
    N, L = w["N"], w["L"]
    with _plan_for(w) as plan:
        plan.assign(bisp.DATA, _dev(gal["xyz"]), None, _dev(gal["nbar"]))
        plan.assign(bisp.RANDOMS, _dev(ran["xyz"]), None, _dev(ran["nbar"]))
        out = plan.measure()
        out2 = plan.measure()
        spec_g = plan.fetch_spectrum(bisp.DATA, 0)
        spec_r = plan.fetch_spectrum(bisp.RANDOMS, 0)
        info = plan.info()
    # bitwise reproducible
    for k in ("B", "shot", "window", "window_shot"):
        assert np.array_equal(out[k], out2[k]), k
    # B_{l l L}(k1, k2) = B_{l l L}(k2, k1): the two orders are summed independently
    for im, (l1, l2, _) in enumerate(w["ells"]):
        if l1 == l2:
            Bm = out["B"][im]
            m = np.abs(Bm) > 0.01 * np.abs(Bm).max()
            assert np.max(np.abs(Bm - Bm.T)[m] / np.abs(Bm)[m]) <= TOL
    # mode counts equal the oracle's shell counts
    p = E.Params(N=N, L=L, edges=w["edges"], ells=w["ells"], los="local", observer=w["observer"], mas=3,
                 interlace=True, P0=w["P0"])
    bins = E.bin_grid(p)
    assert np.array_equal(out["nmodes"], np.bincount(bins[bins >= 0].ravel(), minlength=len(w["edges"]) - 1))
    del bins
    # sampled modes of the deconvolved spectra against the oracle's FP64 mesh (direct DFT)
    modes = [(1, 0, 0), (3, -2, 5), (-7, 11, 2), (20, 13, 30), (-40, 5, 60), (100, -90, 77)]
    for cat, spec in ((gal, spec_g), (ran, spec_r)):
        wts = E.object_weights(cat, w["P0"])
        m0 = E.assign(cat["xyz"], wts, N, L, 3, 0.0)
        d0 = _direct_dft(m0, modes, N)
        del m0
        m1 = E.assign(cat["xyz"], wts, N, L, 3, 0.5)
        d1 = _direct_dft(m1, modes, N)
        del m1
        nn = np.array(modes)
        D = 0.5 * (d0 + np.exp(-1j * np.pi * nn.sum(1) / N) * d1)
        W = np.prod(np.sinc(nn / N), axis=1) ** 3
        D = D / W
        got = np.array([spec[n[0] % N, n[1] % N, n[2]] for n in modes])
        scale = np.abs(spec[1:, 1:, 1:]).max()
        assert np.max(np.abs(got - D)) <= 2e-5 * scale, (np.abs(got - D), scale)
    # far observer: the local line of sight tends to the global one (same catalogues)
    with _plan_for(w, observer=(1500.0, 1500.0, -1e9), want_window=False) as pl, \
            _plan_for(w, los="global", want_window=False) as pg:
        for pln in (pl, pg):
            pln.assign(bisp.DATA, _dev(gal["xyz"]), None, _dev(gal["nbar"]))
            pln.assign(bisp.RANDOMS, _dev(ran["xyz"]), None, _dev(ran["nbar"]))
        bl, bg = pl.measure()["B"], pg.measure()["B"]
    for im in range(len(w["ells"])):
        m = np.abs(bg[im]) > 0.01 * np.abs(bg[im]).max()
        assert np.max(np.abs(bl[im] - bg[im])[m] / np.abs(bg[im])[m]) <= 1e-4
    assert info["norm_I"] > 0


def test_survey512_sampled_pairs_against_oracle():
    """The headline workload at its full size, in bench.py's launch configuration: the 512^3
    survey (local line of sight, FKP weights, TSC with interlacing, 1e6 galaxies and 5e7 randoms,
    window pass) against FP64 oracle values at sampled bin pairs of B000, B202 (both orders of
    l1 != l2) and B112, next to and at the top bin: B, its shot noise, the window bispectrum and its
    shot noise, each within 1e-4 of itself or 1e-6 of its multipole's largest |value|.  The oracle values are stored in tests/golden/survey512_sampled_pairs.json, written
    by tests/golden/make_survey512_sampled_pairs.py (the oracle only) from the same seeded
    catalogues, whose checksums the test checks first."""
    import hashlib
    import json
    import os

    path = os.path.join(os.path.dirname(__file__), "golden", "survey512_sampled_pairs.json")
    gold = json.load(open(path))
    w = bench.WORKLOADS["survey512"]
    gw = gold["workload"]
    assert gw["N"] == w["N"] and gw["L"] == w["L"] and gw["n_gen"] == w["n_gen"]
    assert gw["n_gal"] == w["n_gal"] and gw["n_ran"] == w["n_ran"] and gw["P0"] == w["P0"]
    assert np.allclose(gw["edges"], w["edges"]) and [tuple(e) for e in gw["ells"]] == w["ells"]
    gal, ran = bench.make_inputs(w, seed=gw["seed"])
    for nm, cat in (("gal", gal), ("ran", ran)):
        for k in ("xyz", "nbar"):
            dig = hashlib.sha256(np.ascontiguousarray(cat[k]).tobytes()).hexdigest()
            assert dig == gold["catalogue_sha256"][f"{nm}_{k}"], f"{nm} {k}: the generator gives another catalogue"
    with _plan_for(w) as plan:
        plan.assign(bisp.DATA, _dev(gal["xyz"]), None, _dev(gal["nbar"]))
        plan.assign(bisp.RANDOMS, _dev(ran["xyz"]), None, _dev(ran["nbar"]))
        out = plan.measure()
        info = plan.info()
    assert info["norm_I"] == pytest.approx(gold["norm_I"], rel=1e-6)
    assert info["alpha"] == pytest.approx(gold["alpha"], rel=1e-9)
    for rec in gold["values"]:
        im = w["ells"].index(tuple(rec["ells"]))
        b1, b2 = rec["b1"], rec["b2"]
        for key in ("B", "shot", "window", "window_shot"):
            ref = rec[key]
            got = out[key][im, b1, b2]
            # every sampled value: 1e-4 of itself, or 1e-6 of the multipole's largest |value| for
            # values deep in cancellation (most sampled pairs lie below 1% of that largest value,
            # where the parity tests' relative bound alone would not apply)
            scale = np.abs(out[key][im]).max()
            assert abs(got - ref) <= max(TOL * abs(ref), 1e-6 * scale), (rec["ells"], b1, b2, key, got, ref, scale)


def test_box1024_blocked_fp32_against_fp64_form(monkeypatch):
    """The 1024^3 box workload (2000 Mpc/h, 1.2e8 particles, TSC + interlacing, B000, B202,
    B112, B222) at its full mesh and catalogue, in its blocked launch configuration (bins held in
    blocks, one contraction per block union), on its first four bins: the fused FP32 path against
    the plain FP64 form (FP64 inverse transforms and one FP64 mesh sum per bin pair and 3j term)
    on the same assignment.  Holds the 1024^3 instantiations of the pruned inverse passes and the
    few-bin contraction shapes to the FP64 transforms and mesh sums."""
    w = dict(bench.WORKLOADS["box1024"])
    w["edges"] = w["edges"][:5]
    gal, _ = bench.make_inputs(w, seed=1002)
    xyz = _dev(gal["xyz"])
    outs = {}
    for prec in ("fp32", "fp64"):
        if prec == "fp32":
            monkeypatch.setenv("BISP_BLOCK_BINS", "2")
            monkeypatch.delenv("BISP_FP64_BLOCK_BINS", raising=False)
        else:
            monkeypatch.delenv("BISP_BLOCK_BINS", raising=False)
            monkeypatch.setenv("BISP_FP64_BLOCK_BINS", "1")
        with _plan_for(w, precision=prec) as plan:
            plan.assign(bisp.DATA, xyz)
            outs[prec] = plan.measure()
            assert plan.info()["pair_kernel"] == (1 if prec == "fp32" else 3)
    assert np.array_equal(outs["fp32"]["nmodes"], outs["fp64"]["nmodes"])
    for key in ("B", "shot"):
        for im, mult in enumerate(w["ells"]):
            ref = outs["fp64"][key][im]
            got = outs["fp32"][key][im]
            m = np.abs(ref) > 0.01 * np.abs(ref).max()
            err = np.max(np.abs(got[m] - ref[m]) / np.abs(ref[m]))
            assert err <= TOL, (key, mult, err)
            # every other bin within 1e-5 of the multipole's largest |value|
            assert np.all(np.abs(got - ref) <= np.maximum(TOL * np.abs(ref), 1e-5 * np.abs(ref).max())), (key, mult)
