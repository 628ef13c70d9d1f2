"""The C ABI library loads and exports every function include/pss.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pss_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def libpath():
    from paper_2405_02410_gb300 import build
    return build.build()


def test_library_exports_every_declared_function(libpath):
    lib = ctypes.CDLL(libpath)
    names = _declared("pss.h")
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header(libpath):
    from paper_2405_02410_gb300 import pss
    assert sorted(pss.EXPORTS) == _declared("pss.h")


def test_create_rejects_bad_sizes_without_touching_the_gpu(libpath):
    # argument checks run before any CUDA call
    from paper_2405_02410_gb300 import pss
    for shape in [(6, 8), (2048,), (8, 8, 3)]:
        with pytest.raises(pss.PssError) as ei:
            pss.System(shape, dt=0.1)
        assert ei.value.code in (pss.PSS_EINVAL, pss.PSS_EUNSUPPORTED)
    with pytest.raises(pss.PssError):
        pss.System((8, 8), dt=-1.0)
