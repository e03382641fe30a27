"""The product path and the oracle stay apart, and the product path fails
loudly without its library.  No GPU.

* No module of the package imports the oracle, and no CUDA/C++ source of the
  library includes anything from it; the oracle imports nothing from the
  package (the seeded input generators are the only shared code, and the
  tests call them on both sides).
* With libpmgb.so missing, loading the binding raises instead of falling
  back to anything else, and a ParticleMesh on a machine without CUDA raises.
"""

import ast
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2211_09958_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _python_imports(path):
    tree = ast.parse(open(path).read(), path)
    names = set()
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            names.update(a.name.split(".")[0] for a in node.names)
        elif isinstance(node, ast.ImportFrom) and node.level == 0 and node.module:
            names.add(node.module.split(".")[0])
    return names


def _files(top, exts):
    for d, _, fs in os.walk(top):
        if "__pycache__" in d or os.sep + "_lib" in d:
            continue
        for f in fs:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_package_does_not_import_the_oracle():
    py = list(_files(PKG, (".py",)))
    assert len(py) >= 6
    for path in py:
        assert "oracle" not in _python_imports(path), path


def test_library_sources_do_not_include_the_oracle():
    src = list(_files(os.path.join(PKG, "csrc"), (".cu", ".cuh", ".cpp", ".h")))
    src += list(_files(os.path.join(ROOT, "include"), (".h",)))
    assert len(src) >= 8
    for path in src:
        for inc in re.findall(r'#\s*include\s*[<"]([^>"]+)[>"]', open(path).read()):
            assert "oracle" not in inc, (path, inc)


def test_oracle_does_not_import_the_package_or_torch():
    py = list(_files(ORACLE, (".py",)))
    assert len(py) >= 5
    for path in py:
        imports = _python_imports(path)
        assert "paper_2211_09958_gb300" not in imports, path
        assert "torch" not in imports, path


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_2211_09958_gb300 import _pmgb
    monkeypatch.setattr(_pmgb, "_LIB_PATH", str(tmp_path / "libpmgb.so"))
    monkeypatch.setattr(_pmgb, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _pmgb.load()


def test_particle_mesh_needs_cuda(monkeypatch):
    import torch
    from paper_2211_09958_gb300.pm import ParticleMesh, PMError
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    with pytest.raises(PMError, match="CUDA"):
        ParticleMesh(8, 16, 32.0)
