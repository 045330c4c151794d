"""The oracle and the CUDA path share no code: nothing in the package (Python,
CUDA, headers) imports, includes or loads the oracle, and nothing in the oracle
uses the package.  The only module both sides use is the seeded input generator
(synth.py), which draws inputs and computes none of the method.  And the product
path has no fallback: without the built library, importing the binding fails.
Static checks on the sources; CPU only."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1008_0502_b300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(d, exts):
    for dirpath, _, files in os.walk(d):
        if "__pycache__" in dirpath:
            continue
        for f in files:
            if f.endswith(exts):
                p = os.path.join(dirpath, f)
                with open(p, errors="replace") as fh:
                    yield p, fh.read()


def test_package_never_uses_the_oracle():
    pat = re.compile(r"^\s*(import\s+oracle|from\s+oracle\b|from\s+\.+\s*import\s+oracle)|"
                     r"#\s*include\s*[<\"][^>\"]*oracle|liboracle|orc_[a-z_]+\s*\(", re.M)
    hits = [p for p, src in _sources(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")) if pat.search(src)]
    with open(os.path.join(ROOT, "include", "seg.h")) as f:
        assert not pat.search(f.read())
    assert not hits, hits


def test_oracle_never_uses_the_package():
    pat = re.compile(r"paper_1008_0502_b300|libseg|#\s*include\s*[<\"][^>\"]*seg(_internal)?\.(h|cuh)|"
                     r"\bseg_[a-z_]+\s*\(", re.M)
    hits = [p for p, src in _sources(ORACLE, (".py", ".c", ".h")) if pat.search(src)]
    assert not hits, hits


def test_shared_input_generator_imports_neither_side():
    with open(os.path.join(PKG, "synth.py")) as f:
        src = f.read()
    imports = re.findall(r"^\s*(?:import|from)\s+([\w.]+)", src, re.M)
    assert imports and not any(m.startswith(".") or m.split(".")[0] in ("oracle", "paper_1008_0502_b300", "torch")
                               for m in imports), imports


def test_binding_fails_loudly_without_the_library(tmp_path):
    # a copy of the binding next to no built library must refuse to import
    pkg = tmp_path / "paper_1008_0502_b300"
    pkg.mkdir()
    for f in ("__init__.py", "seg.py"):
        with open(os.path.join(PKG, f)) as src, open(pkg / f, "w") as dst:
            dst.write(src.read())
    r = subprocess.run([sys.executable, "-c", "import paper_1008_0502_b300.seg"], cwd=tmp_path,
                       capture_output=True, text=True, env=dict(os.environ, PYTHONPATH=str(tmp_path)))
    assert r.returncode != 0 and "CUDA library not built" in r.stderr, r.stderr[-500:]
