"""The product path has no CPU fallback: it never reaches the oracle, and it fails with an error when its
CUDA library is missing or no GPU can be used."""
import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2304_09409_gb300")


def _python_files():
    for d, _, files in os.walk(PKG):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(d, f)


def test_package_never_imports_the_oracle():
    for path in _python_files():
        tree = ast.parse(open(path).read(), path)
        for node in ast.walk(tree):
            names = []
            if isinstance(node, ast.Import):
                names = [a.name for a in node.names]
            elif isinstance(node, ast.ImportFrom):
                names = [node.module or ""]
            assert not any(n == "oracle" or n.startswith("oracle.") for n in names), path
            if isinstance(node, ast.Constant) and isinstance(node.value, str):
                assert "libdporacle" not in node.value and "dp_oracle" not in node.value, path


def test_cuda_sources_never_reach_the_oracle():
    for d, _, files in os.walk(os.path.join(PKG, "csrc")):
        for f in files:
            src = open(os.path.join(d, f)).read()
            assert "dp_oracle" not in src and "orc_" not in src and "libdporacle" not in src, f


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_2304_09409_gb300 import dpgb
    from paper_2304_09409_gb300 import inputs as I
    monkeypatch.setattr(dpgb, "LIB_PATH", str(tmp_path / "libdpgb.so"))
    monkeypatch.setattr(dpgb, "_lib", None)
    cfg = I.water_model()
    with pytest.raises(RuntimeError, match="not built"):
        dpgb.Model(cfg, I.make_params(cfg, 0), precision="fp64")


def test_no_gpu_raises():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: the GPU tests cover this path")
    from paper_2304_09409_gb300 import build, dpgb
    from paper_2304_09409_gb300 import inputs as I
    if not os.path.exists(dpgb.LIB_PATH):
        build.build()
    cfg = I.water_model()
    with pytest.raises(dpgb.DPError):
        dpgb.Model(cfg, I.make_params(cfg, 0), precision="fp64")


def test_oracle_includes_nothing_of_the_cuda_path():
    """The oracle and the CUDA path share no code: the oracle's source includes system headers only."""
    src = open(os.path.join(ROOT, "oracle", "dp_oracle.cpp")).read()
    for line in src.splitlines():
        if line.strip().startswith("#include"):
            assert "<" in line and '"' not in line, line
