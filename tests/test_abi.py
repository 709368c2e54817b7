"""The C-ABI library loads and exports every symbol include/reloc.h declares
(no GPU needed: nothing is called but version and default-config)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "reloc.h")


def declared_functions(path=HEADER):
    text = open(path).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(reloc_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2403_11367_gb300.build import build
    path = build()
    return C.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["reloc_create", "reloc_destroy", "reloc_load_map", "reloc_select_block", "reloc_render",
                 "reloc_score", "reloc_localize", "reloc_localize_host", "reloc_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(lib):
    from paper_2403_11367_gb300 import reloc
    assert set(declared_functions()) <= set(reloc.SIGNATURES)


def test_version_and_default_config_without_gpu(lib):
    from paper_2403_11367_gb300 import reloc
    assert "sm_103a" in reloc.reloc_version()
    cfg = reloc.reloc_default_config()
    assert (cfg.tile_w, cfg.tile_h) == (16, 16)
    assert abs(cfg.alpha_min - 1 / 255) < 1e-9 and abs(cfg.alpha_max - 0.99) < 1e-7
    assert abs(cfg.t_min - 1e-4) < 1e-10 and cfg.cut == 3.0 and abs(cfg.near_plane - 0.2) < 1e-7


def test_create_rejects_bad_config_before_touching_a_device(lib):
    from paper_2403_11367_gb300 import reloc
    cfg = reloc.reloc_default_config(tile_w=12)
    with pytest.raises(reloc.RelocError) as e:
        reloc.Context(cfg)
    assert e.value.status == reloc.EINVAL
