"""The product path has no CPU fallback: the binding refuses to import without
the CUDA library, and refuses host tensors instead of computing on the host."""
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def cs():
    from paper_2110_10156_gb300 import build
    build.build()
    from paper_2110_10156_gb300 import cs_ngf
    return cs_ngf


def test_import_fails_loudly_without_the_library(tmp_path):
    """A copy of the package without libcs_ngf.so cannot be imported."""
    pkg = tmp_path / "paper_2110_10156_gb300"
    pkg.mkdir()
    for name in ("__init__.py", "cs_ngf.py"):
        shutil.copy(os.path.join(ROOT, "paper_2110_10156_gb300", name), pkg / name)
    code = "import paper_2110_10156_gb300.cs_ngf"
    res = subprocess.run([sys.executable, "-c", code], cwd=tmp_path, capture_output=True, text=True,
                         env={**os.environ, "PYTHONPATH": str(tmp_path)})
    assert res.returncode != 0
    assert "ImportError" in res.stderr and "libcs_ngf.so is missing" in res.stderr


def _host_pair():
    A = torch.zeros((8, 8, 8), dtype=torch.float32)
    M = torch.ones((8, 8, 8), dtype=torch.uint8)
    return A, M


def test_host_tensors_are_refused(cs):
    A, M = _host_pair()
    with pytest.raises(TypeError, match="CUDA tensor"):
        cs.prepare_fixed(A, M)
    with pytest.raises(TypeError, match="CUDA tensor"):
        cs.global_align(A, M, A, M)
    q = np.array([[1.0, 0.0, 0.0, 0.0]])
    with pytest.raises(TypeError, match="CUDA tensor"):
        cs.score_rotations_noalloc(A, M, A, M, q)


def test_numpy_arrays_are_refused(cs):
    A = np.zeros((8, 8, 8), np.float32)
    M = np.ones((8, 8, 8), np.uint8)
    with pytest.raises(TypeError, match="CUDA tensor"):
        cs.prepare_fixed(A, M)
    with pytest.raises(TypeError, match="CUDA tensor"):
        cs.score_rotations_noalloc(A, M, A, M, np.array([[1.0, 0.0, 0.0, 0.0]]))
    with pytest.raises(TypeError, match="CUDA tensor"):
        cs.global_align(A, M, A, M)


def test_noalloc_refuses_mismatched_shapes_and_outputs_before_any_launch(cs):
    """The allocation-free call reads B and the masks with A's dims and writes
    R results, so the binding refuses any other shape up front (these host
    tensors would be refused later too; the shape check comes first)."""
    A, M = _host_pair()
    q = np.array([[1.0, 0.0, 0.0, 0.0]] * 2)
    small = torch.zeros((8, 8, 7), dtype=torch.float32)
    with pytest.raises(ValueError, match="shape"):
        cs.score_rotations_noalloc(A, M, small, M, q)
    with pytest.raises(ValueError, match="shape"):
        cs.score_rotations_noalloc(A, M, A, torch.ones((8, 7, 8), dtype=torch.uint8), q)
    with pytest.raises(ValueError, match="shape"):
        cs.score_rotations_noalloc(A, torch.ones((9, 8, 8), dtype=torch.uint8), A, M, q)
    with pytest.raises(ValueError, match="nz"):
        cs.score_rotations_noalloc(A[0], M[0], A[0], M[0], q)
    with pytest.raises(ValueError, match="best_score"):
        cs.score_rotations_noalloc(A, M, A, M, q, out_score=torch.zeros(1))
    with pytest.raises(ValueError, match="best_shift"):
        cs.score_rotations_noalloc(A, M, A, M, q, out_shift=torch.zeros((2, 2), dtype=torch.int32))
