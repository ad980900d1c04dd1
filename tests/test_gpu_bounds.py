"""The bounds-checked build (every global access of the pass kernels checked against
its buffer) runs odd shapes, strides, offsets, parameters and batches with no access
outside any buffer, and gives the same bits as the normal build."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_bounds_checked_build_clean_and_identical(tmp_path):
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    sys.path.insert(0, ROOT)
    from paper_2108_13656_gb300 import build_lib
    lib = build_lib.build(force=True, extra_flags=["-DDC_BOUNDS_CHECK"], lib_path=str(tmp_path / "libdc_bc.so"),
                          obj_dir=str(tmp_path / "obj"))
    npz = str(tmp_path / "bc.npz")
    env = dict(os.environ, DC_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(HERE, "_bounds_cases.py"), npz], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    assert "bounds checked=1 flags=0" in r.stdout, r.stdout
    checked = dict(np.load(npz))
    import _bounds_cases
    import paper_2108_13656_gb300 as dc
    assert dc.debug_bounds() == (False, 0)  # the normal build has no checks
    normal = _bounds_cases.run()
    assert sorted(checked) == sorted(normal)
    for k in normal:
        assert np.array_equal(checked[k], normal[k], equal_nan=True), k
