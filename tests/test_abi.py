"""The C-ABI library builds, loads and exports every function include/phi4smc.h declares (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "phi4smc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s+\**([a-z][a-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_2511_15196_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("smc_init", "smc_temper_step", "ns_replace_step", "smc_log_evidence", "smc_observables"):
        assert required in names
    assert len(names) >= 20


def test_library_exports_every_declared_symbol(built):
    so = ctypes.CDLL(built)
    missing = [n for n in declared_functions() if not hasattr(so, n)]
    assert not missing, missing


def test_binding_signatures_cover_header(built):
    import paper_2511_15196_gb300 as p
    assert set(declared_functions()) == set(p.exported_symbols())
    lib = p.lib()
    assert lib.phi4_stage_name(0) == b"bisect_reweight"


def test_workspace_sizing_and_argument_checks(built):
    import paper_2511_15196_gb300 as p
    n = p.workspace_bytes(p.Config(L=8, N=1024))
    assert n > 1024 * 64 * 8 * 3
    big = p.workspace_bytes(p.Config(L=64, N=8192, precision=p.MIXED_BF16))
    assert big > 8192 * 4096 * 4 * 3
    with pytest.raises(p.Phi4Error) as e:
        p.workspace_bytes(p.Config(L=0, N=16))
    assert e.value.status == p.PHI4_ERR_ARG
    with pytest.raises(p.Phi4Error):
        p.workspace_bytes(p.Config(L=8, N=16, ess_target=1.5))
    assert b"ess_target" in p.lib().phi4_last_error()
    with pytest.raises(p.Phi4Error):
        p.workspace_bytes(p.Config(L=8, N=16, kind=p.NS_SLICE, ns_n_delete=16))
    assert b"ns_n_delete" in p.lib().phi4_last_error()


def test_inner_kernel_configuration_rules_and_workspace(built):
    # SMC-IRMH: FP64, D <= 1024; SMC-HMC: FP64 or FP32, D <= 4096; both SMC moves, so the Z2
    # flag is accepted. Their extra buffers (whitened norms, leapfrog scales) are in the
    # workspace.
    import paper_2511_15196_gb300 as p
    rw = p.workspace_bytes(p.Config(L=8, N=1024))
    assert p.workspace_bytes(p.Config(L=8, N=1024, kind=p.SMC_IRMH)) >= rw + 2 * 1024 * 8
    assert p.workspace_bytes(p.Config(L=8, N=1024, kind=p.SMC_HMC)) >= rw + 64 * 8
    assert p.workspace_bytes(p.Config(L=64, N=64, kind=p.SMC_HMC, precision=p.FP32)) > 0
    assert p.workspace_bytes(p.Config(L=32, N=64, kind=p.SMC_IRMH, flags=p.FLAG_Z2_FLIP)) > 0
    for bad, word in ((p.Config(L=8, N=64, kind=p.SMC_IRMH, precision=p.FP32), b"SMC-IRMH"),
                      (p.Config(L=33, N=64, kind=p.SMC_IRMH), b"SMC-IRMH"),
                      (p.Config(L=8, N=64, kind=p.SMC_HMC, precision=p.MIXED_BF16), b"SMC-HMC"),
                      (p.Config(L=65, N=64, kind=p.SMC_HMC), b"SMC-HMC"),
                      (p.Config(L=8, N=64, kind=4), b"kind")):
        with pytest.raises(p.Phi4Error):
            p.workspace_bytes(bad)
        assert word in p.lib().phi4_last_error()


def _imports_of(tree):
    """Absolute module names imported anywhere under an AST node."""
    import ast
    out = []
    for n in ast.walk(tree):
        if isinstance(n, ast.Import):
            out += [a.name for a in n.names]
        elif isinstance(n, ast.ImportFrom) and n.level == 0:
            out.append(n.module or "")
    return [m.split(".")[0] for m in out]


def test_product_and_oracle_are_separate():
    # the product (the package and its CUDA sources) never imports or names the oracle;
    # the oracle imports nothing of the product; bench.py reaches the oracle only inside
    # its CPU-baseline function (the reference arm and the cpu_baseline leg)
    import ast

    def parsed(path):
        return ast.parse(open(path).read())
    pkg = os.path.join(ROOT, "paper_2511_15196_gb300")
    for name in sorted(os.listdir(pkg)):
        if name.endswith(".py"):
            assert "oracle" not in _imports_of(parsed(os.path.join(pkg, name))), name
    csrc = os.path.join(pkg, "csrc")
    for name in sorted(os.listdir(csrc)):
        assert "oracle" not in open(os.path.join(csrc, name)).read().lower(), name
    odir = os.path.join(ROOT, "oracle")
    for name in sorted(os.listdir(odir)):
        if name.endswith(".py"):
            mods = _imports_of(parsed(os.path.join(odir, name)))
            assert not {"paper_2511_15196_gb300", "torch", "ctypes"} & set(mods), name
    bench = parsed(os.path.join(ROOT, "bench.py"))
    for node in bench.body:
        if isinstance(node, ast.FunctionDef) and "oracle" in _imports_of(node):
            assert node.name == "cpu_baseline", node.name
        elif not isinstance(node, ast.FunctionDef):
            assert "oracle" not in _imports_of(node)


def test_binding_structs_match_the_header_layout(tmp_path):
    # the ctypes mirrors of phi4_config and phi4_obs have the C compiler's size and field
    # offsets (a field added, dropped or reordered on one side only would shift the rest)
    import shutil
    import subprocess
    import paper_2511_15196_gb300 as p
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = {"phi4_config": p.CConfig, "phi4_obs": p.CObs}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "phi4smc.h"', "int main(void) {"]
    for cname, cls in structs.items():
        lines.append('printf("%s sizeof %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            cf = "lambda" if f == "lambda_" else f
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, cf))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        s, f, v = line.split()
        got[(s, f)] = int(v)
    for cname, cls in structs.items():
        assert got[(cname, "sizeof")] == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert got[(cname, f)] == getattr(cls, f).offset, (cname, f)


def test_static_resampling_array_holds_the_scratch_of_its_largest_call(built):
    # the allocation-free resampler's built-in array (PHI4_RESAMPLE_STATIC_MAX_N 64-bit
    # words) is exactly the scratch the allocating entry point asks for at that N
    import paper_2511_15196_gb300 as p
    text = open(HEADER).read()
    max_n = int(re.search(r"#define PHI4_RESAMPLE_STATIC_MAX_N (\d+)", text).group(1))
    lib = p.lib()
    assert lib.phi4_resample_scratch_bytes(max_n) == 8 * max_n == 512 * 1024
    for n in (1, 2, 1000, 8192, 131072):
        assert lib.phi4_resample_scratch_bytes(n) == 8 * n
    assert lib.phi4_bisect_scratch_bytes(8192) > 0
