"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/lbm_gb300.h declares; the ctypes structs match the C layout.  CPU only: no
compute call is made."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    import paper_2210_07501_gb300 as pkg
    pkg.build()
    return pkg.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lbm_create", "lbm_step", "lbm_fields", "lbm_destroy", "lbm_diag", "lbm_init_fields"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    import paper_2210_07501_gb300 as pkg
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in pkg.SIGNATURES, f"binding lacks {name}"
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (lbm_[a-z_0-9]+)", out))
    assert set(declared_functions()) <= exported


def test_library_targets_sm_103a():
    import paper_2210_07501_gb300 as pkg
    pkg.build()
    out = subprocess.run(["cuobjdump", "--list-elf", pkg.LIB_PATH], capture_output=True, text=True).stdout
    assert "sm_103a" in out


def test_struct_layout_matches_c(tmp_path):
    import ctypes

    import paper_2210_07501_gb300 as pkg
    src = tmp_path / "layout.c"
    fields_d = [f for f, _ in pkg.LbmDomain._fields_]
    fields_p = [f for f, _ in pkg.LbmParams._fields_]
    body = "#include <stdio.h>\n#include <stddef.h>\n#include \"lbm_gb300.h\"\nint main(void){\n"
    body += 'printf("%zu %zu\\n", sizeof(lbm_domain), sizeof(lbm_params));\n'
    for f in fields_d:
        body += f'printf("%zu\\n", offsetof(lbm_domain, {f}));\n'
    for f in fields_p:
        body += f'printf("%zu\\n", offsetof(lbm_params, {f}));\n'
    body += "return 0;}\n"
    src.write_text(body)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    vals = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    assert int(vals[0]) == ctypes.sizeof(pkg.LbmDomain)
    assert int(vals[1]) == ctypes.sizeof(pkg.LbmParams)
    offs = [int(v) for v in vals[2:]]
    expect = [getattr(pkg.LbmDomain, f).offset for f in fields_d] + [getattr(pkg.LbmParams, f).offset for f in fields_p]
    assert offs == expect


def test_product_never_imports_the_oracle():
    """The CUDA path and the oracle share nothing: no import of oracle from the package."""
    pkg_dir = os.path.join(ROOT, "paper_2210_07501_gb300")
    for dirpath, _, files in os.walk(pkg_dir):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text and "lbm_oracle" not in text, f


def test_invalid_arguments_rejected_before_any_device_work(lib):
    """Parameter validation happens on the host, before the first CUDA call."""
    import ctypes

    import lbm_workloads as WL
    import paper_2210_07501_gb300 as pkg
    w = WL.workload("srf-channel-128x32")
    bad = [dict(nx=2), dict(ny=1), dict(q_phi=7), dict(q_T=3), dict(W=0.0), dict(b=0.0), dict(b=40.0),
           dict(precision=5), dict(tau_flow=0.5), dict(tau_T=0.2), dict(tau_phi=0.5), dict(visc_ratio=0.0),
           dict(rho_top=-1.0), dict(sigma0=float("nan"))]
    for over in bad:
        d = dict(w["domain"])
        p = dict(w["params"])
        prec = over.pop("precision", 0)
        for k, v in over.items():
            (d if k in d else p)[k] = v
        h = ctypes.c_void_p()
        rc = lib.lbm_create(ctypes.byref(pkg.make_domain(d, prec)), ctypes.byref(pkg.make_params(p)), None,
                            ctypes.byref(h))
        assert rc == pkg.LBM_EINVAL, over
        assert not h.value
    assert lib.lbm_step(None, 1) == pkg.LBM_EINVAL
    assert lib.lbm_fields(None, None, None, None, None, None) == pkg.LBM_EINVAL
    lib.lbm_destroy(None)
    assert lib.lbm_strerror(pkg.LBM_EIO) == b"checkpoint I/O error"


def test_sweep_generator_matches_the_stated_distribution():
    import lbm_workloads as WL
    cases = WL.sweep_cases(96, seed=0)
    assert len(cases) == 96
    for c in cases:
        d, p = c["domain"], c["params"]
        assert d["nx"] in (256, 512, 1024) and d["ny"] in (64, 128, 256)
        assert -2e-5 <= p["sigma1"] <= 2e-5 and -4e-4 <= p["sigma2"] <= 0.0
        assert 0.5 <= p["cond_ratio"] <= 4.0 and 0.5 <= p["visc_ratio"] <= 4.0
        ab = (d["ny"] - d["b"]) / d["b"]
        assert 0.2 <= ab <= 4.5
    assert WL.sweep_cases(96, seed=0) == cases            # seeded
    assert len({(c["domain"]["nx"], c["domain"]["ny"]) for c in cases}) == 9
