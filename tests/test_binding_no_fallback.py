"""The Python binding only marshals arguments: CPU tensors are refused before any library call
(there is no CPU path for the device entry points), the host-buffer calls refuse device or
non-float64 tensors, and a missing library fails the import with a message instead of
falling back to anything."""
import os
import shutil
import subprocess
import sys

import pytest
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sbq():
    from paper_2310_00889_gb300 import build
    build.build()
    from paper_2310_00889_gb300 import sbq as mod
    return mod


def test_device_entry_points_refuse_cpu_tensors(sbq):
    x = torch.zeros((3, 8), dtype=torch.float64)
    w = torch.ones(8, dtype=torch.float64)
    with pytest.raises(TypeError):
        sbq.sl_apply(x, w, x, x)
    with pytest.raises(TypeError):
        sbq.dl_apply(x, x, w, x, x)
    with pytest.raises(TypeError):
        sbq.combined_apply(x, x, w, x, x, 1.0, 1.0)
    with pytest.raises(TypeError):
        sbq.laplace_apply(x, x, w, torch.zeros(8, dtype=torch.float64), x)
    with pytest.raises(TypeError):
        sbq.StokesTree(x, w)
    with pytest.raises(TypeError):
        sbq.StokesOp(x, x, w, 1.0)


def test_host_entry_points_refuse_other_tensors(sbq):
    x32 = torch.zeros((3, 8), dtype=torch.float32)
    w = torch.ones(8, dtype=torch.float64)
    x = torch.zeros((3, 8), dtype=torch.float64)
    with pytest.raises(TypeError):
        sbq.apply_host(x32, x, w, x, 1.0)
    with pytest.raises(ValueError):
        sbq.apply_host(x[:, :4], x, w, x, 1.0)
    with pytest.raises(TypeError):
        sbq.solve_host(x, x, w.to(torch.float32), x, 1.0)


def test_missing_library_fails_the_import(tmp_path):
    """A copy of the package without its built library: importing the binding raises."""
    dst = tmp_path / "paper_2310_00889_gb300"
    shutil.copytree(os.path.join(ROOT, "paper_2310_00889_gb300"), dst,
                    ignore=shutil.ignore_patterns("_lib", "__pycache__", "csrc", "rules"))
    r = subprocess.run([sys.executable, "-c", "import paper_2310_00889_gb300.sbq"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0
    assert "libsbq.so is not built" in r.stderr
