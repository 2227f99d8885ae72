import os
import re
import shutil
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (B300, sm_103a)")


def _has_gpu() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


def pytest_collection_modifyitems(config, items):
    if _has_gpu():
        return
    skip = pytest.mark.skip(reason="no CUDA GPU in this environment")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture
def repo_tmp(request):
    """A scratch directory inside the repository's git-ignored build folder
    (tests keep their files under the repository)."""
    name = re.sub(r"[^A-Za-z0-9_.-]", "_", request.node.name)
    path = os.path.join(ROOT, "_build", "test_tmp", name)
    shutil.rmtree(path, ignore_errors=True)
    os.makedirs(path)
    return path


def build_c_client(out_dir: str) -> str:
    """Compile tests/c_client/stem_client.c (C99) against include/stem.h and
    link it with libstem.so and the CUDA runtime; return the executable."""
    import subprocess
    pkg = os.path.join(ROOT, "paper_1706_08563_b300")
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    exe = os.path.join(out_dir, "stem_client")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-O2", "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(cuda, "include"), os.path.join(ROOT, "tests", "c_client", "stem_client.c"),
           "-L", pkg, "-lstem", "-L", os.path.join(cuda, "lib64"), "-lcudart", "-Wl,-rpath," + pkg,
           "-Wl,-rpath," + os.path.join(cuda, "lib64"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe
