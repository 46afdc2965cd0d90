"""Host-side checks of the C ABI: the library builds and loads, exports every
declared entry point, and rejects bad arguments before touching a GPU."""
import ctypes

import pytest

from tests._util import declared_symbols


@pytest.fixture(scope="module")
def L():
    from paper_2003_07504_gb300 import build, _lib
    build.build()
    return _lib.lib()


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert "ils_plan_create" in names and "ils_smooth" in names
    for n in names:
        assert hasattr(L, n), f"{n} declared in include/ but not exported"


def test_binding_signatures_cover_the_header():
    from paper_2003_07504_gb300 import _lib
    assert set(declared_symbols()) <= set(_lib.SIGNATURES), set(declared_symbols()) - set(_lib.SIGNATURES)


# The boundary calls of the hot path: plans (Eq. 11's c), Algorithm 1 from f or from a given
# u^0, uneven-frame batches, plan-owned checkpoints and the adjoint by f, status names.
BOUNDARY = {
    "ils_plan_create": 8, "ils_plan_destroy": 1, "ils_smooth": 4, "ils_smooth_from": 5,
    "ils_smooth_batched": 3, "ils_set_checkpointing": 2, "ils_backward": 5, "ils_status_string": 1,
    "ils_plan_c": 1,
}


def test_header_declares_the_boundary_calls():
    import os
    import re
    from tests._util import ROOT
    text = open(os.path.join(ROOT, "include", "ils.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    for name, nargs in BOUNDARY.items():
        m = re.search(r"\b" + name + r"\s*\(([^)]*)\)\s*;", text)
        assert m is not None, f"{name} is not declared"
        assert len(m.group(1).split(",")) == nargs, (name, m.group(1))
    assert re.search(r"ILS_ERR_FALLBACK_TAKEN\s*=\s*6", text)


def test_boundary_calls_validate_without_a_gpu(L):
    assert L.ils_set_checkpointing(None, 1) == 1
    assert L.ils_backward(None, None, None, None, None) == 1
    assert L.ils_backward_ckpt(None, None, None, None, None, None) == 1


def test_noalloc_source_calls_no_allocator():
    """The allocation-free entry point's translation unit names no allocating routine."""
    import os
    import re
    from tests._util import ROOT
    src = open(os.path.join(ROOT, "paper_2003_07504_gb300", "csrc", "ils_noalloc.cu")).read()
    code = re.sub(r"//[^\n]*", "", re.sub(r"/\*.*?\*/", "", src, flags=re.S))
    for bad in (r"\bcudaMalloc\w*", r"\bcudaFree\w*", r"\bcuMem\w*", r"\bmalloc\s*\(", r"\bcalloc\s*\(",
                r"\brealloc\s*\(", r"\bnew\b", r"\bstd::vector\b", r"\bstd::string\b", r"\bdev_alloc\b"):
        assert re.search(bad, code) is None, bad


def test_status_strings(L):
    for code, name in ((0, b"ILS_OK"), (1, b"ILS_ERR_INVALID_ARG"), (2, b"ILS_ERR_UNSUPPORTED_SIZE"),
                       (3, b"ILS_ERR_OOM"), (4, b"ILS_ERR_CUDA"), (5, b"ILS_ERR_TIMEOUT"),
                       (6, b"ILS_ERR_FALLBACK_TAKEN")):
        assert L.ils_status_string(code) == name


def _create(L, H, W, C=1, lam=1.0, p=0.8, eps=1e-4, N=4):
    h = ctypes.c_void_p()
    return L.ils_plan_create(H, W, C, lam, p, eps, N, ctypes.byref(h)), h


@pytest.mark.parametrize("args", [
    dict(C=0), dict(N=-1), dict(lam=-1.0), dict(lam=float("nan")), dict(eps=0.0), dict(eps=-1e-4),
    dict(p=0.0), dict(p=1.5), dict(p=-0.5), dict(lam=float("inf")),
])
def test_bad_parameters_are_rejected(L, args):
    kw = dict(H=16, W=16)
    kw.update(args)
    st, h = _create(L, **kw)
    assert st == 1 and not h.value


@pytest.mark.parametrize("H,W", [(7, 16), (16, 14), (16, 15), (1, 16), (16, 0), (16384, 16), (16, 16384), (22, 16)])
def test_unsupported_sizes_are_rejected(L, H, W):
    st, h = _create(L, H, W)
    assert st == 2 and not h.value


def test_null_arguments(L):
    assert L.ils_plan_create(16, 16, 1, 1.0, 0.8, 1e-4, 4, None) == 1
    assert L.ils_smooth(None, None, None, None) == 1
    assert L.ils_smooth_from(None, None, None, None, None) == 1
    assert L.ils_smooth_host(None, None, None, None) == 1
    assert L.ils_plan_destroy(None) == 0
    assert L.ils_plan_c(None) == -1.0


def test_header_is_plain_c_and_links(L, tmp_path):
    # a C99 program includes the header, links libils.so and calls entry points that must
    # answer without a GPU: status strings and argument validation
    import os
    import shutil
    import subprocess
    from paper_2003_07504_gb300 import _lib
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    lib_dir = os.path.dirname(_lib.LIB_PATH)
    src = tmp_path / "abi.c"
    src.write_text(r'''
#include <stdio.h>
#include <string.h>
#include "ils.h"
int main(void) {
  ils_plan* plan = NULL;
  if (strcmp(ils_status_string(ILS_OK), "ILS_OK") != 0) return 1;
  if (ils_plan_create(16, 16, 1, -1.0f, 0.8f, 1e-4f, 4, &plan) != ILS_ERR_INVALID_ARG || plan != NULL) return 2;
  if (ils_plan_create(14, 16, 1, 1.0f, 0.8f, 1e-4f, 4, &plan) != ILS_ERR_UNSUPPORTED_SIZE) return 3;
  if (ils_smooth(NULL, NULL, NULL, NULL) != ILS_ERR_INVALID_ARG) return 4;
  if (ils_plan_destroy(NULL) != ILS_OK) return 5;
  printf("ok\n");
  return 0;
}
''')
    exe = tmp_path / "abi"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(root, "include"), str(src),
                    "-o", str(exe), "-L", lib_dir, "-lils", f"-Wl,-rpath,{lib_dir}"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout, r.stderr)
