"""The oracle and the CUDA path stay independent, and the product has no CPU
fallback (checked statically and in a fresh interpreter; no GPU needed):

* no module of the package imports the oracle, and the oracle imports
  nothing of the package but the seeded input generator (synth), which holds
  none of the method's arithmetic;
* the CUDA sources include nothing from oracle/ and the oracle's C source
  includes nothing from the package or include/ (no shared header, table or
  helper);
* bench.py reaches the oracle only from its CPU-baseline and reference-arm
  functions, and __graft_entry__ only from build() (which compiles it) and
  smoke() (which checks against it);
* with libhe.so missing, the first library call raises instead of computing
  anything on the host."""
import ast
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2109_14704_gb300")


def _imports(path):
    """(module name, enclosing top-level function or None) of every import."""
    tree = ast.parse(open(path).read(), path)
    out = []

    def visit(node, fn):
        for child in ast.iter_child_nodes(node):
            name = fn
            if isinstance(child, (ast.FunctionDef, ast.AsyncFunctionDef)) and fn is None:
                name = child.name
            if isinstance(child, ast.Import):
                out.extend((a.name, name) for a in child.names)
            elif isinstance(child, ast.ImportFrom):
                mod = ("." * child.level) + (child.module or "")
                out.append((mod, name))
                out.extend((f"{mod}.{a.name}", name) for a in child.names)
            visit(child, name)

    visit(tree, None)
    return out


def _py_files(d):
    for base, dirs, files in os.walk(d):
        dirs[:] = [x for x in dirs if not x.startswith(("_", "."))]
        for f in files:
            if f.endswith(".py"):
                yield os.path.join(base, f)


def test_package_never_imports_the_oracle():
    files = list(_py_files(PKG))
    assert len(files) >= 5
    for path in files:
        for mod, _ in _imports(path):
            assert not re.match(r"(\.*)oracle\b", mod), (path, mod)


def test_oracle_imports_only_the_input_generator_from_the_package():
    for path in _py_files(os.path.join(ROOT, "oracle")):
        for mod, _ in _imports(path):
            if "paper_2109_14704_gb300" in mod:
                assert mod in ("paper_2109_14704_gb300.synth", "paper_2109_14704_gb300.synth.Rng"), (path, mod)


def test_no_shared_native_code():
    inc = re.compile(r'^\s*#\s*include\s*[<"]([^>"]+)[>"]', re.M)
    csrc = os.path.join(PKG, "csrc")
    for f in os.listdir(csrc):
        for h in inc.findall(open(os.path.join(csrc, f)).read()):
            assert "oracle" not in h, (f, h)
    # the oracle's C source uses the C standard library alone
    oracle_c = os.path.join(ROOT, "oracle", "he_oracle.c")
    headers = set(inc.findall(open(oracle_c).read()))
    assert headers and headers <= {"stdint.h", "stddef.h", "stdlib.h", "string.h", "stdio.h"}, headers


def test_oracle_reached_only_from_the_baseline_and_the_checks():
    seen = {}
    for path, allowed in ((os.path.join(ROOT, "bench.py"), {"cpu_baseline", "run_reference", "_ntt_moduli"}),
                          (os.path.join(ROOT, "__graft_entry__.py"), {"build", "smoke"})):
        fns = {fn for mod, fn in _imports(path) if re.match(r"oracle\b", mod)}
        assert None not in fns, path                       # no module-level import
        assert fns <= allowed, (path, fns - allowed)
        seen[os.path.basename(path)] = fns
    assert {"cpu_baseline", "run_reference"} <= seen["bench.py"]


def test_missing_library_fails_loudly(tmp_path):
    code = f"""
import sys
sys.path.insert(0, {ROOT!r})
from paper_2109_14704_gb300 import build as b, he
b.LIB = {str(tmp_path / "absent" / "libhe.so")!r}
he._build.LIB = b.LIB
try:
    he.load(build_if_needed=False)
except RuntimeError as e:
    print("raised:", e)
    sys.exit(0)
print("no error")
sys.exit(1)
"""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "CUDA library missing" in r.stdout, r.stdout + r.stderr
