"""Host-side checks of the C ABI (no GPU needed): the library loads, exports every
symbol include/eslbm.h declares, and validates configurations."""
import ctypes
import os
import re

import pytest

from paper_2403_13406_gb300 import build as cuda_build
from paper_2403_13406_gb300 import eslbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    cuda_build.build()
    return eslbm.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "eslbm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(eslbm_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(eslbm.EXPORTS)


def test_abi_version_and_status_strings(L):
    assert L.eslbm_abi_version() == 3
    for s in (0, 1, 2, 3, 4, 5, 100, 77):
        assert L.eslbm_status_string(s)


def q(**kw):
    base = dict(dim=1, system="burgers", nx=256, V=1.5)
    base.update(kw)
    return eslbm.make_config(**base)


def test_query_sizes(L):
    sz = eslbm.query(q(precision="fp32"))
    assert (sz.q, sz.M, sz.planes, sz.ncell) == (2, 1, 2, 256)
    assert sz.state_bytes == 2 * 256 * 4
    assert sz.stages_per_step == 18 and sz.step_cells == 24
    sz = eslbm.query(q(system="sw", nx=1 << 20, precision="fp64", V=4.0, g=9.81))
    assert sz.planes == 4 and sz.state_bytes == 4 * (1 << 20) * 8
    sz = eslbm.query(eslbm.make_config(2, "sw", 100, 50, V=8.0, g=9.81))
    assert (sz.q, sz.M, sz.ncell) == (4, 3, 5000)
    sz = eslbm.query(eslbm.make_config(2, "euler", 64, 64, V=6.21))
    assert sz.planes == 16
    assert eslbm.query(q(scheme="III")).stages_per_step == 27
    assert eslbm.query(q(scheme="IV")).stages_per_step == 36
    assert eslbm.query(q(scheme="plain")).stages_per_step == 1
    assert eslbm.query(q(scheme="plain")).step_cells == 1
    assert eslbm.query(q(scheme="B")).step_cells == 4


@pytest.mark.parametrize("bad,status", [
    (dict(dim=3), eslbm.ERR_ARG),
    (dict(nx=0), eslbm.ERR_ARG),
    (dict(V=-1.0), eslbm.ERR_ARG),
    (dict(scheme=9), eslbm.ERR_ARG),
    (dict(kappa=0), eslbm.ERR_ARG),
    (dict(system="sw", g=0.0), eslbm.ERR_ARG),
    (dict(system="linear", a=(1.6, 0.0)), eslbm.ERR_DOMAIN),
    (dict(system="sw", V=4.0, g=9.81, u_ref=(-1.0, 0.0)), eslbm.ERR_DOMAIN),  # negative reference depth
    (dict(system="sw", V=4.0, g=9.81, u_ref=(1.0, 5.0)), eslbm.ERR_DOMAIN),   # |v| + sqrt(g h) > V
    (dict(system="burgers", V=1.0, u_ref=(1.2,)), eslbm.ERR_DOMAIN),          # |u| >= V (D1Q2)
    (dict(precision=3), eslbm.ERR_ARG),
])
def test_query_rejects(L, bad, status):
    cfg = q(**bad)
    with pytest.raises(eslbm.EslbmError) as e:
        eslbm.query(cfg)
    assert e.value.status == status


def test_shifted_reference_is_accepted(L):
    """The reference state of the shifted storage is checked on the host at query time."""
    assert eslbm.query(q(system="sw", V=4.0, g=9.81, u_ref=(1.0, 0.0))).planes == 4
    assert eslbm.query(eslbm.make_config(2, "euler", 16, 16, V=8.0, u_ref=(1.0, 1.0, 1.0, 3.5))).planes == 16
    bad = q(system="sw", V=4.0, g=9.81, u_ref=(1.0, 0.0))
    bad.shifted = 2
    with pytest.raises(eslbm.EslbmError) as e:
        eslbm.query(bad)
    assert e.value.status == eslbm.ERR_ARG


def test_mixed_precision_and_blocking_fields(L):
    """FP32_MIXED stores FP32 (same buffer sizes as FP32); blocking takes AUTO (0), OFF (1) or a largest
    group of stages per 2D launch (2..32)."""
    a = eslbm.query(q(system="sw", V=4.0, g=9.81, precision="fp32", omega_mode="entropic"))
    b = eslbm.query(q(system="sw", V=4.0, g=9.81, precision="fp32_mixed", omega_mode="entropic"))
    assert a.state_bytes == b.state_bytes == 4 * 256 * 4
    assert eslbm.query(q(blocking=False)).planes == 2
    assert eslbm.query(q(blocking=6)).planes == 2
    for v in (-1, 33):
        bad = q()
        bad.blocking = v
        with pytest.raises(eslbm.EslbmError) as e:
            eslbm.query(bad)
        assert e.value.status == eslbm.ERR_ARG


def test_structs_match_header(L, tmp_path):
    """The ctypes mirrors of the ABI structs have the C layout: sizes and field offsets printed by
    a C program compiled against include/eslbm.h."""
    import subprocess
    structs = {"eslbm_config": eslbm.Config, "eslbm_sizes": eslbm.Sizes, "eslbm_diagnostics": eslbm.Diagnostics,
               "eslbm_batch_sizes": eslbm.BatchSizes}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "eslbm.h"', 'int main(void) {']
    for cname, cls in structs.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in cls._fields_:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, cls in structs.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for f, _ in cls._fields_:
            assert int(got["%s.%s" % (cname, f)]) == getattr(cls, f).offset, (cname, f)


def test_entropic_euler_is_unsupported(L):
    with pytest.raises(eslbm.EslbmError) as e:
        eslbm.query(eslbm.make_config(2, "euler", 8, 8, V=6.0, omega_mode="entropic"))
    assert e.value.status == eslbm.ERR_UNSUPPORTED


def test_create_rejects_bad_buffers(L):
    cfg = q()
    h = ctypes.c_void_p()
    st = L.eslbm_create(ctypes.byref(cfg), None, None, None, None, ctypes.byref(h))
    assert st == eslbm.ERR_ARG and not h.value
    st = L.eslbm_create(ctypes.byref(cfg), 16, 16, 32, None, ctypes.byref(h))  # same buffer twice
    assert st == eslbm.ERR_ARG
    st = L.eslbm_create(ctypes.byref(cfg), 17, 48, 64, None, ctypes.byref(h))  # misaligned
    assert st == eslbm.ERR_ARG
    assert L.eslbm_destroy(None) == 0


@pytest.mark.parametrize("system,kw,precision,mode,blocking,nx,expected", [
    # AUTO: two stages a launch of the blocked 2D kernel for the 16-plane Euler state in FP32, fixed omega
    ("euler", dict(V=8.0, gamma=1.4), "fp32", "fixed", True, 8192, 9.0),
    ("euler", dict(V=8.0, gamma=1.4), "fp32", "fixed", False, 8192, 18.0),
    ("euler", dict(V=8.0, gamma=1.4), "fp64", "fixed", True, 8192, 18.0),
    ("euler", dict(V=8.0, gamma=1.4), "fp32", "fixed", True, 8190, 18.0),  # rows off 16-byte boundaries
    ("euler", dict(V=8.0, gamma=1.4), "fp32", "fixed", 6, 8192, 3.0),
    ("burgers", dict(V=3.0), "fp32", "fixed", True, 4096, 18.0),
    ("burgers", dict(V=3.0), "fp32", "entropic", True, 4096, 18.0),
    ("sw", dict(V=8.0, g=9.81), "fp32", "entropic", True, 1024, 18.0),
])
def test_blocking_choice_in_2d(system, kw, precision, mode, blocking, nx, expected):
    """Launches per composite step that the library reports for a 2D configuration (no device needed: the
    grouping of the stages is planned on the host)."""
    cfg = eslbm.make_config(2, system, nx, nx, precision=precision, omega_mode=mode, blocking=blocking, **kw)
    assert eslbm.query(cfg).launches_per_step == expected
