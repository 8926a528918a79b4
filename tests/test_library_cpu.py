"""CPU-side checks of the C ABI library: it builds, loads, exports every
function declared in include/*.h, and its host-only logic (parameter
validation, CSR validation, momentum scalar, status strings) behaves.  No
call here touches a GPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2409_13344_gb300 import build
    build.build()
    from paper_2409_13344_gb300 import appga
    return appga.load_library()


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(appga_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_exports_every_declared_symbol(lib):
    names = _declared_functions()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_header(lib):
    from paper_2409_13344_gb300 import appga
    assert set(_declared_functions()) <= set(appga.SIGNATURES)
    for name in _declared_functions():
        assert callable(getattr(appga, name, None)) or name in (
            "appga_status_string", "appga_last_error", "appga_version", "appga_params_default"), name


def test_struct_layouts_match_header(lib):
    from paper_2409_13344_gb300 import appga
    assert ctypes.sizeof(appga.appga_params) == 96
    assert ctypes.sizeof(appga.appga_stats) == 40
    assert ctypes.sizeof(appga.appga_matrix_info) == 72


def test_struct_layouts_match_c_compiler(lib, tmp_path):
    """sizeof and field offsets of every ABI struct as the C compiler lays
    them out, against the ctypes mirrors the binding passes."""
    import shutil
    import subprocess
    from paper_2409_13344_gb300 import appga
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [appga.appga_params, appga.appga_stats, appga.appga_matrix_info,
               appga.appga_batch_tuning, appga.appga_fom, appga.appga_afppa_stats,
               appga.appga_server_config,
               appga.appga_request_stats,
               appga.appga_server_summary]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "appga_server.h"',
             "int main(void) {"]
    for st in structs:
        lines.append(f'  printf("{st.__name__} %zu\\n", sizeof({st.__name__}));')
        for f, _ in st._fields_:
            lines.append(f'  printf("{st.__name__}.{f} %zu\\n", offsetof({st.__name__}, {f}));')
    lines.append("  return 0;\n}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                   check=True).stdout.splitlines())
    for st in structs:
        assert int(got[st.__name__]) == ctypes.sizeof(st), st.__name__
        for f, _ in st._fields_:
            assert int(got[f"{st.__name__}.{f}"]) == getattr(st, f).offset, (st.__name__, f)


def test_nofv_host(lib):
    from paper_2409_13344_gb300 import appga as A
    assert A.appga_nofv(5.0, 5.0, 1.0) == 1.0
    assert A.appga_nofv(1.0, 5.0, 1.0) == 0.0
    assert A.appga_nofv(3.0, 5.0, 1.0) == 0.5


def test_server_config_default(lib):
    from paper_2409_13344_gb300 import appga as A
    c = A.server_config()
    assert (c.slots_per_pool, c.steps_per_launch, c.a_precision, c.max_pools) == (64, 8, 0, 0)
    assert (c.hbm_budget_bytes, c.hbm_reserve_bytes) == (0, 1 << 30)


def test_params_default_and_validate(lib):
    from paper_2409_13344_gb300 import appga as A
    p = A.default_params()
    assert (p.lambda1, p.lambda2, p.eps, p.omega, p.a, p.b, p.beta) == (0.1, 0.05, 1e-3, 0.5, 0.125, 1.0, 1.0)
    assert A.appga_params_validate(p) == A.APPGA_OK
    bad = [dict(eps=0.0), dict(lambda1=-1.0), dict(beta=0.0), dict(omega=1.5), dict(omega=0.0),
           dict(a=0.0), dict(omega=1.0, a=0.5), dict(max_iters=-1), dict(precond_freeze_iter=0),
           dict(a_precision=7), dict(momentum=9), dict(rel_obj_tol=-1.0), dict(eps=math.nan),
           dict(b=-0.125, omega=1.0)]  # b = -a*1 makes t_1 = 0
    for kw in bad:
        q = A.default_params(**kw)
        assert A.appga_params_validate(q) == A.APPGA_EINVAL, kw
        assert lib.appga_last_error()


def test_gn_theta_host(lib):
    from paper_2409_13344_gb300 import appga as A
    for k in range(1, 50):
        assert A.appga_gn_theta(k, 0.125, 1.0, 1.0) == pytest.approx((k - 1) / (k + 8), abs=1e-15)
        assert A.appga_gn_theta(k, 0.125, 1.0, 0.5) == pytest.approx(
            math.sqrt(k - 1) / (math.sqrt(k) + 8), abs=1e-15)


def _csr_call(lib, m, d, rp, col, val):
    rp = np.ascontiguousarray(rp, np.int32)
    col = np.ascontiguousarray(col, np.int32)
    val = np.ascontiguousarray(val, np.float32)
    return lib.appga_validate_csr_host(m, d, rp.ctypes.data, col.ctypes.data, val.ctypes.data)


def test_csr_validator_rejects_corruption(lib):
    ok = ([0, 2, 2, 3], [0, 3, 1], [1.0, 0.5, 2.0])
    assert _csr_call(lib, 3, 4, *ok) == 0
    assert _csr_call(lib, 3, 4, [1, 2, 2, 3], ok[1], ok[2]) == 1          # row_ptr[0] != 0
    assert _csr_call(lib, 3, 4, [0, 2, 1, 3], ok[1], ok[2]) == 1          # decreasing
    assert _csr_call(lib, 3, 4, ok[0], [0, 4, 1], ok[2]) == 1             # col out of range
    assert _csr_call(lib, 3, 4, ok[0], [0, -1, 1], ok[2]) == 1
    assert _csr_call(lib, 3, 4, ok[0], ok[1], [1.0, -0.5, 2.0]) == 3      # negative entry
    assert _csr_call(lib, 3, 4, ok[0], ok[1], [1.0, math.nan, 2.0]) == 3  # NaN entry
    assert _csr_call(lib, 3, 4, ok[0], ok[1], [1.0, math.inf, 2.0]) == 3
    assert "range" in lib.appga_last_error().decode() or lib.appga_last_error()


def test_status_strings(lib):
    lib.appga_status_string.restype = ctypes.c_char_p
    for s in range(0, 9):
        assert lib.appga_status_string(s)
    assert lib.appga_status_string(3) == b"input outside the model's domain"


def test_no_device_is_reported_not_crashed(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2409_13344_gb300 import appga as A
    with pytest.raises(A.AppgaError) as ei:
        A.appga_ctx_create(0)
    assert ei.value.status == A.APPGA_ENODEV
