"""Write tests/golden/survey512_sampled_pairs.json: FP64 oracle values of the 512^3 survey
workload (3000 Mpc/h box, observer at (1500, 1500, -300) Mpc/h, 1e6 galaxies and 5e7 randoms
from synthcat seed 1002, FKP P0 = 1e4, TSC with interlacing, local line of sight, 25 bins of
0.01 h/Mpc from 0.01 h/Mpc, window pass) at sampled bin pairs of B000, B202 and B112: the
shot-noise-subtracted B, its shot noise, the window bispectrum and the window's shot noise.

Calls only the oracle (oracle/sampled.py, which evaluates oracle/estimator.py with its spectra
kept in files) and the seeded input generator.  Hours of CPU time and about 50 GB of disk for
the spectra: run it by hand, e.g.
    python tests/golden/make_survey512_sampled_pairs.py <scratch directory>
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synthcat  # noqa: E402
from oracle import estimator as E  # noqa: E402
from oracle import sampled as S  # noqa: E402

WORKLOAD = dict(N=512, L=3000.0, n_gen=256, observer=[1500.0, 1500.0, -300.0], n_gal=1_000_000,
                n_ran=50_000_000, seed=1002, edges=[round(float(e), 6) for e in np.linspace(0.01, 0.26, 26)],
                ells=[[0, 0, 0], [2, 0, 2], [1, 1, 2]], mas=3, interlace=True, P0=1e4)
# bin pairs: both orders of l1 != l2, pairs at and next to the top bin
PAIRS = {(0, 0, 0): [(3, 17), (24, 24)], (2, 0, 2): [(5, 20), (20, 5), (23, 24)], (1, 1, 2): [(2, 9), (24, 22)]}
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "survey512_sampled_pairs.json")


def digest(a):
    return hashlib.sha256(np.ascontiguousarray(a).tobytes()).hexdigest()


def main(workdir):
    w = WORKLOAD
    t0 = time.time()
    gal, ran = synthcat.survey_catalogs(w["n_gen"], w["L"], tuple(w["observer"]), w["n_gal"], w["n_ran"], w["seed"])
    sums = {f"{nm}_{k}": digest(c[k]) for nm, c in (("gal", gal), ("ran", ran)) for k in ("xyz", "nbar")}
    print(f"catalogues {len(gal['xyz'])} + {len(ran['xyz'])} in {time.time() - t0:.0f} s", flush=True)
    p = E.Params(N=w["N"], L=w["L"], edges=w["edges"], ells=[tuple(e) for e in w["ells"]], los="local",
                 observer=tuple(w["observer"]), mas=w["mas"], interlace=w["interlace"], P0=w["P0"], window=True)
    specs = S.catalogue_spectra_on_disk(p, gal, ran, workdir)
    print(f"spectra in {time.time() - t0:.0f} s", flush=True)
    del gal, ran
    values = []
    for mult, prs in PAIRS.items():
        for pr in prs:
            rec = S.measure_pairs(p, specs, {mult: [pr]})[mult + pr]
            values.append({"ells": list(mult), "b1": pr[0], "b2": pr[1], **rec})
            print(mult, pr, rec, f"{time.time() - t0:.0f} s", flush=True)
    doc = {"description": __doc__.split("\n\n")[0], "workload": w, "catalogue_sha256": sums,
           "norm_I": specs["data"].I, "alpha": specs["data"].alpha, "values": values,
           "cpu_seconds": round(time.time() - t0)}
    with open(OUT, "w") as f:
        json.dump(doc, f, indent=1)
    print("wrote", OUT)


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else os.path.join(ROOT, "_work", "oracle512"))
