"""Static and CPU checks of the product path's boundary rules: the package and
the input generators never import the oracle, and the binding refuses to run
without the compiled library (there is no CPU fallback)."""

import ast
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def python_files(*dirs):
    for d in dirs:
        for base, _, files in os.walk(os.path.join(ROOT, d)):
            for f in files:
                if f.endswith(".py"):
                    yield os.path.join(base, f)


def imported_modules(path):
    tree = ast.parse(open(path).read(), filename=path)
    for node in ast.walk(tree):
        if isinstance(node, ast.Import):
            for a in node.names:
                yield a.name
        elif isinstance(node, ast.ImportFrom) and node.module and node.level == 0:
            yield node.module


def test_package_and_generators_never_import_the_oracle():
    for path in python_files("paper_2110_01614_gb300", "synth"):
        for mod in imported_modules(path):
            assert mod.split(".")[0] != "oracle", (path, mod)


def test_native_sources_never_name_the_oracle():
    csrc = os.path.join(ROOT, "paper_2110_01614_gb300", "csrc")
    for f in os.listdir(csrc):
        if f.endswith((".cu", ".cuh", ".h", ".cpp")):
            assert "oracle" not in open(os.path.join(csrc, f)).read().lower(), f
    for f in os.listdir(os.path.join(ROOT, "include")):
        assert "oracle" not in open(os.path.join(ROOT, "include", f)).read().lower(), f


def test_oracle_never_imports_the_product():
    for path in python_files("oracle"):
        for mod in imported_modules(path):
            assert mod.split(".")[0] != "paper_2110_01614_gb300", (path, mod)


def test_binding_refuses_to_run_without_the_library(tmp_path, monkeypatch):
    from paper_2110_01614_gb300 import _abi
    monkeypatch.setattr(_abi, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _abi.load(str(tmp_path / "libnsdf.so"))
