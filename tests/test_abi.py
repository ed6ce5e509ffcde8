"""CPU checks of the C ABI: the library loads, exports every function the
header declares, the ctypes mirror of ng_params matches the C layout, and
host-side validation rejects bad parameters before touching a GPU."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ngravs.h")


@pytest.fixture(scope="module")
def binding():
    from paper_1502_07442_gb300 import build
    build.build()
    from paper_1502_07442_gb300 import binding as b
    b.lib()
    return b


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ng_[a-z_]+)\s*\(", text)))


def test_header_functions_are_exported(binding):
    L = binding.lib()
    names = _declared()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert sorted(binding.exported_symbols()) == names


def test_params_layout_matches_c(binding, tmp_path):
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "ngravs.h"\n'
                   'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(ng_params),'
                   ' offsetof(ng_params,G), offsetof(ng_params,law), offsetof(ng_params,eps),'
                   ' offsetof(ng_params,theta), offsetof(ng_params,opening), offsetof(ng_params,alpha),'
                   ' offsetof(ng_params,pure_tree), offsetof(ng_params,beta), offsetof(ng_params,accumulate_fp64));return 0;}\n')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = list(map(int, subprocess.check_output([str(exe)]).split()))
    P = binding.NgParams
    want = [ctypes.sizeof(P), P.G.offset, P.law.offset, P.eps.offset, P.theta.offset,
            P.opening.offset, P.alpha.offset, P.pure_tree.offset, P.beta.offset,
            P.accumulate_fp64.offset]
    assert got == want


@pytest.mark.parametrize("field,value,needle", [
    ("D", 0, "D=0"), ("D", 7, "D=7"), ("eps", 0.0, "eps"), ("box", -1.0, "box"),
    ("pm_mesh", 48, "pm_mesh"), ("leaf_size", 65, "leaf_size"), ("theta", -0.1, "theta"),
    ("rcut_over_rs", 1000.0, "r_cut"), ("opening", 2, "opening"), ("reserved1", 1, "reserved1"),
    ("accumulate_fp64", 2, "accumulate_fp64"), ("reserved2", 1, "reserved2"),
    ("pure_tree", 1, "pm_mesh"), ("pure_tree", 3, "pure_tree"), ("ignore_nperp", 3, "ignore_nperp"),
])
def test_create_rejects_bad_params(binding, field, value, needle):
    p = binding.make_params(2, np.ones((2, 2)), eps=1e-3, pm_mesh=32)
    setattr(p, field, value)
    ctx = ctypes.c_void_p()
    rc = binding.lib().ng_create(ctypes.byref(ctx), ctypes.byref(p), None)
    assert rc == binding.NG_EINVAL
    assert not ctx.value
    assert needle in binding.lib().ng_last_error(None).decode()


@pytest.mark.parametrize("alpha", [0.0, -1.0, float("inf"), float("nan")])
def test_relative_opening_needs_positive_alpha(binding, alpha):
    p = binding.make_params(2, np.ones((2, 2)), eps=1e-3, opening=binding.NG_OPEN_RELATIVE,
                            alpha=alpha)
    ctx = ctypes.c_void_p()
    assert binding.lib().ng_create(ctypes.byref(ctx), ctypes.byref(p), None) == binding.NG_EINVAL
    assert "alpha" in binding.lib().ng_last_error(None).decode()


@pytest.mark.parametrize("law,beta,needle", [
    ([[3, 3], [3, 3]], 1e-3, "pure tree"),                       # Mahalo outside pure tree mode
    ([[0, 3], [3, 0]], 1e-3, "no cored species"),
    ([[0, 3], [3, 3]], 0.0, "beta"),
])
def test_mahalo_validation(binding, law, beta, needle):
    pure = needle != "pure tree"
    p = binding.make_params(2, np.ones((2, 2)), eps=1e-3, pm_mesh=0 if pure else 32, law=law,
                            pure_tree=1 if pure else 0, beta=beta)
    ctx = ctypes.c_void_p()
    assert binding.lib().ng_create(ctypes.byref(ctx), ctypes.byref(p), None) == binding.NG_EINVAL
    assert needle in binding.lib().ng_last_error(None).decode()


@pytest.mark.parametrize("law,yl,needle", [
    ([[3, 3], [3, 3]], 0.05, "Mahalo"),          # Mahalo laws have no lattice corrections
    ([[1, 1], [1, 1]], 0.2, "yuk_l"),            # Yukawa image sums need yuk_l <= L/8
])
def test_lattice_mode_validation(binding, law, yl, needle):
    p = binding.make_params(2, np.ones((2, 2)), eps=1e-3, pm_mesh=0, law=law, yuk_a=np.ones((2, 2)),
                            yuk_l=np.full((2, 2), yl), pure_tree=2, beta=1e-3)
    ctx = ctypes.c_void_p()
    assert binding.lib().ng_create(ctypes.byref(ctx), ctypes.byref(p), None) == binding.NG_EINVAL
    assert needle in binding.lib().ng_last_error(None).decode()


def test_yukawa_needs_positive_range(binding):
    p = binding.make_params(1, np.ones((1, 1)), eps=1e-3, law=[[1]], yuk_a=[[0.2]], yuk_l=[[0.0]])
    ctx = ctypes.c_void_p()
    assert binding.lib().ng_create(ctypes.byref(ctx), ctypes.byref(p), None) == binding.NG_EINVAL
    assert "Yukawa" in binding.lib().ng_last_error(None).decode()


def test_calls_reject_null_context(binding):
    L = binding.lib()
    assert L.ng_build_tree(None, 10, None, None, None, None, None) == binding.NG_EINVAL
    assert L.ng_tree_force(None, None, None) == binding.NG_EINVAL
    assert L.ng_pm_force(None, None) == binding.NG_EINVAL
    assert L.ng_destroy(None) == binding.NG_OK
    assert "sm_103a" in binding.ng_version()


def test_stage_names_follow_the_header(binding, tmp_path):
    # the binding's stage names are the header's NG_STAGE_* enumerators, in order
    text = open(HEADER).read()
    names = re.findall(r"NG_STAGE_([A-Z_]+)", text)
    seen = []
    for s in names:
        if s.lower() not in seen:
            seen.append(s.lower())
    assert tuple(seen) == binding.STAGES
    src = tmp_path / "st.c"
    src.write_text('#include <stdio.h>\n#include "ngravs.h"\n'
                   'int main(void){printf("%d %d\\n", (int)NG_NSTAGES, (int)NG_STAGE_WALK);return 0;}\n')
    exe = tmp_path / "st"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    n, walk = map(int, subprocess.check_output([str(exe)]).split())
    assert n == len(binding.STAGES) and walk == n - 1
