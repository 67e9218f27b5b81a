"""Host-side checks of the C ABI: the library builds, loads and exports every
symbol include/lbgb.h declares; argument validation needs no GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lbgb():
    from paper_2505_01126_gb300 import build

    build.build()
    from paper_2505_01126_gb300 import lbgb as mod

    return mod


def declared_functions():
    src = open(os.path.join(ROOT, "include", "lbgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lb_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lb_create", "lb_init", "lb_step", "lb_moments", "lb_destroy", "lb_diagnostics"):
        assert required in names


def test_header_is_plain_c99():
    """A C99 program (no C++) can include the header and name every declared
    function: the boundary needs no C++ or torch types (gcc, syntax only, source
    on stdin)."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not found")
    body = "\n".join(f"    (void)&{n};" for n in declared_functions())
    src = f'#include "lbgb.h"\nint main(void) {{\n{body}\n    return 0;\n}}\n'
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c",
                        "-I", os.path.join(ROOT, "include"), "-"], input=src, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_library_exports_every_declared_symbol(lbgb):
    lib = lbgb.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
    for name in lbgb.EXPORTS:
        assert name in declared_functions()


@pytest.mark.parametrize("args", [
    (0, 8, 8, 1.0, 0.1, 3.0, 0.01),
    (8, 8, 8, 0.5, 0.1, 3.0, 0.01),
    (8, 8, 8, 1.0, 0.0, 3.0, 0.01),
    (8, 8, 8, 1.0, 0.1, -1.0, 0.01),
    (8, 8, 8, 1.0, 0.1, 3.0, -0.01),
    (8, 8, 8, 1.0, 0.1, float("inf"), 0.01),
])
def test_create_rejects_invalid_parameters(lbgb, args):
    with pytest.raises(lbgb.LBError) as e:
        lbgb.Box(*args)
    assert e.value.code == lbgb.LB_EINVAL


def test_create_rejects_bad_storage_and_force(lbgb):
    with pytest.raises(lbgb.LBError) as e:
        lbgb.Box(8, 8, 8, 1.0, 0.1, 3.0, 0.01, storage=7)
    assert e.value.code == lbgb.LB_EINVAL
    with pytest.raises(lbgb.LBError) as e:
        lbgb.Box(8, 8, 8, 1.0, 0.1, 3.0, 0.01, force=lbgb.Force(kind=lbgb.LB_FORCE_LINEAR, T_relax=0))
    assert e.value.code == lbgb.LB_EINVAL


def test_batch_rejects_unknown_storage(lbgb):
    with pytest.raises(lbgb.LBError) as e:
        lbgb.Batch([(8, 8, 8)], 1.0, 0.1, 3.0, 0.01, storage=9)
    assert e.value.code == lbgb.LB_EINVAL


def test_null_context_calls_fail_cleanly(lbgb):
    lib = lbgb.lib()
    assert lib.lb_step(None, 1) == lbgb.LB_EINVAL
    assert lib.lb_sync(None) == lbgb.LB_EINVAL
    assert lib.lb_time(None) == -1
    lib.lb_destroy(None)
