"""The C-ABI library builds for sm_103a, loads, and exports every function that
include/bisp.h declares (no GPU needed: nothing here calls into CUDA)."""
import os
import re

import pytest

import paper_1803_02132_gb300 as bisp


def test_library_exports_every_header_function():
    names = bisp.header_functions()
    assert {"bisp_plan_create", "bisp_assign", "bisp_measure", "bisp_plan_destroy", "bisp_last_error"} <= set(names)
    lib = bisp.lib()
    for n in names:
        assert hasattr(lib, n), n


def test_header_is_plain_c():
    txt = open(os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "bisp.h")).read()
    assert 'extern "C"' in txt
    assert "torch" not in txt and "at::" not in txt
    # every declared function is documented by a comment block just above it
    for m in re.finditer(r"^(?:bisp_status|const char\*)\s+(bisp_\w+)\s*\(", txt, re.M):
        before = txt[: m.start()].rstrip().splitlines()[-1]
        assert before.strip().endswith("*/") or before.strip().startswith("enum") or "}" in before, m.group(1)


def test_plan_create_rejects_bad_params_without_touching_the_gpu():
    # validation happens before any CUDA call: these fail with BISP_EINVAL even without a GPU
    with pytest.raises(bisp.BispError) as e:
        bisp.Plan(nmesh=48, box_len=1000.0, k_edges=[0.01, 0.02], ells=[(0, 0, 0)])
    assert e.value.status == bisp.BISP_EINVAL
    with pytest.raises(bisp.BispError) as e:
        bisp.Plan(nmesh=64, box_len=1000.0, k_edges=[0.02, 0.01], ells=[(0, 0, 0)])
    assert e.value.status == bisp.BISP_EINVAL
    with pytest.raises(bisp.BispError) as e:
        bisp.Plan(nmesh=64, box_len=1000.0, k_edges=[0.01, 0.02], ells=[(2, 1, 2)])
    assert e.value.status == bisp.BISP_EINVAL and "selection rules" in str(e.value)
    with pytest.raises(bisp.BispError) as e:
        bisp.Plan(nmesh=64, box_len=-1.0, k_edges=[0.01, 0.02], ells=[(0, 0, 0)])
    assert e.value.status == bisp.BISP_EINVAL


def test_oracle_is_not_imported_by_the_product():
    src_dir = os.path.dirname(bisp.__file__)
    for root, _, files in os.walk(src_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                txt = open(os.path.join(root, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle", txt, re.M), f


def test_new_plan_options_are_validated_without_the_gpu():
    with pytest.raises(bisp.BispError) as e:
        bisp.Plan(nmesh=64, box_len=1000.0, k_edges=[0.01, 0.02], ells=[(0, 0, 0)], estimator=5)
    assert e.value.status == bisp.BISP_EINVAL and "estimator" in str(e.value)
    with pytest.raises(bisp.BispError) as e:  # the FP64 form covers the bispectrum only
        bisp.Plan(nmesh=64, box_len=1000.0, k_edges=[10.0, 20.0], ells=[(0, 0, 0)], estimator="threept",
                  precision="fp64")
    assert e.value.status == bisp.BISP_EUNSUPPORTED
    with pytest.raises(bisp.BispError) as e:  # r edges may start at 0 but not below
        bisp.Plan(nmesh=64, box_len=1000.0, k_edges=[-1.0, 20.0], ells=[(0, 0, 0)], estimator="threept")
    assert e.value.status == bisp.BISP_EINVAL and "r edges" in str(e.value)
    with pytest.raises(bisp.BispError) as e:  # k edges must be positive
        bisp.Plan(nmesh=64, box_len=1000.0, k_edges=[0.0, 0.02], ells=[(0, 0, 0)])
    assert e.value.status == bisp.BISP_EINVAL
    with pytest.raises(bisp.BispError) as e:
        bisp.Plan(nmesh=64, box_len=1000.0, k_edges=[0.01, 0.02], ells=[(0, 0, 0)], precision=7)
    assert e.value.status == bisp.BISP_EINVAL


def test_checked_build_compiles():
    """The kernels with device bounds checks (-DBISP_CHECKED, relocatable device code) compile for
    sm_103a: the translation units that carry checks (object files discarded)."""
    import concurrent.futures as cf
    import shutil
    import subprocess

    from paper_1803_02132_gb300 import build as B

    if not shutil.which(B.nvcc()) and not os.path.exists(B.nvcc()):
        pytest.skip("nvcc not available")

    def one(src):
        cmd = [B.nvcc(), *B.ARCH, *B.FLAGS, "-DBISP_CHECKED", "-rdc=true", "-c", os.path.join(B.CSRC, src),
               "-o", os.devnull]
        return src, subprocess.run(cmd, capture_output=True, text=True)

    with cf.ThreadPoolExecutor(max_workers=5) as ex:
        for src, r in ex.map(one, ["assign.cu", "fft.cu", "measure.cu", "pair.cu", "plan.cu"]):
            assert r.returncode == 0, f"{src}: {r.stderr[-2000:]}"
