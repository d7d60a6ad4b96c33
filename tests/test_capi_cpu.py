"""CPU-side checks of the C ABI library: it builds, loads, exports every
symbol include/dmrg.h declares, and reports a clean error without a GPU."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "dmrg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dmrg_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2103_09976_gb300 import build, capi
    if not os.path.exists(capi.LIB_PATH):
        build.build()
    return capi.LIB_PATH


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("dmrg_create", "dmrg_destroy", "dmrg_load_synthetic", "dmrg_sigma", "dmrg_davidson",
              "dmrg_build_blocks", "dmrg_sweep", "dmrg_psi_layout", "dmrg_last_error"):
        assert f in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = set(l.split()[-1] for l in out.splitlines() if l.strip())
    missing = [f for f in declared_functions() if f not in exported]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libpath):
    from paper_2103_09976_gb300 import capi
    L = capi.lib()
    for f in declared_functions():
        assert f in capi.SIGNATURES, f
        getattr(L, f)


def test_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2103_09976_gb300 import capi
    with pytest.raises(capi.DMRGError) as e:
        capi.dmrg_create()
    assert e.value.status in (capi.DMRG_ECUDA, capi.DMRG_EINVAL)


def test_server_create_without_gpu_fails_cleanly(libpath):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2103_09976_gb300 import capi
    with pytest.raises(capi.DMRGError):
        capi.dmrg_server_create(0, 2, 1 << 30)


def test_default_opts(libpath):
    from paper_2103_09976_gb300 import capi
    o = capi.dmrg_default_opts()
    assert o.dav_max_space == 24 and o.dav_max_iter == 200 and o.sigma_prec == capi.DMRG_FP64
    assert o.mixed_cut == -1 and o.graphs == 1 and o.keep_one_per_q == 0
    assert o.tc_chain == 0 and o.tc_producers == 0


def test_option_checks_come_before_the_device(libpath):
    """Invalid options are rejected with EINVAL whether or not a GPU is present."""
    from paper_2103_09976_gb300 import capi
    for kw in ({"mixed_cut": -2}, {"keep_one_per_q": 2}, {"noise": -1.0}, {"dav_max_space": 2}, {"tc_chain": -2},
               {"tc_producers": 2}, {"tc_producers": -1}):
        with pytest.raises(capi.DMRGError) as e:
            capi.dmrg_create(**kw)
        assert e.value.status == capi.DMRG_EINVAL, kw


@pytest.mark.parametrize("module", ["sweeps", "serve", "precision_sweep", "profile_sigma", "bond_energy"])
def test_command_line_tools_start_without_a_gpu(module):
    """The user-facing tools parse their arguments and import the binding
    without touching the device (the device is needed only to run them)."""
    import sys
    r = subprocess.run([sys.executable, "-m", f"paper_2103_09976_gb300.{module}", "--help"], capture_output=True,
                       text=True, timeout=120, cwd=os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    assert r.returncode == 0 and "usage" in r.stdout
