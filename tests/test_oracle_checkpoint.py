"""Checkpointed oracle runs: an interrupted run resumes after its last completed k1 row and ends
with the same result as one uninterrupted measurement; a checkpoint of other inputs is refused."""
import numpy as np
import pytest

from oracle import checkpoint as CK
from oracle import estimator as E

L_BOX = 1000.0
KF = 2 * np.pi / L_BOX


def _case():
    rng = np.random.default_rng(9)
    gal = {"xyz": (rng.random((300, 3)) * L_BOX).astype(np.float32), "w": (0.5 + rng.random(300)).astype(np.float32)}
    ran = {"xyz": (rng.random((900, 3)) * L_BOX).astype(np.float32), "w": (0.5 + rng.random(900)).astype(np.float32)}
    p = E.Params(N=16, L=L_BOX, edges=[1.5 * KF, 2.5 * KF, 3.5 * KF, 4.6 * KF], ells=[(0, 0, 0), (2, 0, 2)],
                 los="local", observer=(500.0, 400.0, -900.0), mas=3, interlace=True, window=True)
    return p, gal, ran


def test_interrupted_run_resumes_to_the_same_result(tmp_path):
    p, gal, ran = _case()
    ref = E.measure(p, gal, ran)
    path = str(tmp_path / "ck.npz")
    assert CK.measure_rows(p, gal, ran, path, max_rows=1) is None
    assert CK.measure_rows(p, gal, ran, path, max_rows=1) is None
    st = np.load(path)
    assert st["done"].tolist() == [True, True, False]
    out = CK.measure_rows(p, gal, ran, path)
    for k in ("B", "shot", "window", "window_shot", "nmodes"):
        assert np.array_equal(out[k], ref[k]), k


def test_checkpoint_of_other_inputs_is_refused(tmp_path):
    p, gal, ran = _case()
    path = str(tmp_path / "ck.npz")
    CK.measure_rows(p, gal, ran, path, max_rows=1)
    gal2 = {k: v.copy() for k, v in gal.items()}
    gal2["w"][0] += 1.0
    with pytest.raises(ValueError, match="different measurement"):
        CK.measure_rows(p, gal2, ran, path)
