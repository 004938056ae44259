"""The C-ABI library builds, loads without a GPU, and exports every function
include/smap.h declares (no compute calls: this runs on CPU-only machines)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    hdr = open(os.path.join(ROOT, "include", "smap.h")).read()
    pat = re.compile(r"^(?:smap_status|void|int|uint64_t|const char\*)\s+(smap_\w+)\s*\(", re.M)
    return set(pat.findall(hdr))


@pytest.fixture(scope="module")
def libpath():
    if not __import__("shutil").which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    from paper_2312_08684_gb300 import build
    return build.build()


def test_library_exports_every_declared_function(libpath):
    names = _declared()
    assert len(names) >= 20
    lib = ctypes.CDLL(libpath)
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_2312_08684_gb300 import _binding
    assert set(_binding.EXPORTS) == _declared()
    _binding.load()
    for n in _binding.EXPORTS:
        assert hasattr(_binding, n), n


def test_host_only_calls(libpath):
    from paper_2312_08684_gb300 import _binding as abi
    assert abi.smap_status_string(0) == "ok"
    assert "non-finite" in abi.smap_status_string(6)
    assert abi.smap_num_variants() >= 1
    for v in range(abi.smap_num_variants()):
        ppt, maxt, tpp = abi.smap_variant_info(v)
        assert ppt >= 1 and maxt % 32 == 0 and tpp in (1, 2, 4, 8, 16, 32)
    with pytest.raises(abi.SmapError):
        abi.smap_variant_info(99)
    assert abi.smap_kernel_launches() == 0


def test_header_is_plain_c(tmp_path):
    """include/smap.h compiles as C99 with warnings as errors: plain types and
    pointers only, usable from any language with a C FFI."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "use_header.c"
    src.write_text('#include "smap.h"\n'
                   "int main(void) { smap_config c = {0}; (void)c; return SMAP_OK; }\n")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"),
                        "-c", str(src), "-o", str(tmp_path / "use_header.o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_no_device_fails_loudly(libpath):
    """Without a usable CUDA device the library refuses to create a handle
    (an error status, no silent CPU path)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    from paper_2312_08684_gb300 import _binding as abi, workloads as W
    wl = W.make_linear_gauss(B=2, T=4, N=16, L=3)
    with pytest.raises(abi.SmapError):
        abi.smap_create(wl.kind, wl.params, wl.N, wl.L, wl.step, 0, 1.0, 0, 1, 2, 4, wl.x0, None, 0)
