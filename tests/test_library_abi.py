"""CPU checks of the C-ABI boundary: the library builds for sm_103a, loads without a GPU and
exports every function include/gbpic.h declares.  No compute call is made here."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "gbpic.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pic_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ["pic_create", "pic_load_species", "pic_set_external_field", "pic_set_plasma", "pic_step",
                 "pic_get_fields", "pic_get_moments", "pic_destroy", "pic_last_error", "pic_create_batch",
                 "pic_load_species_batch", "pic_set_external_field_batch", "pic_set_plasma_batch",
                 "pic_get_moments_run", "pic_autotune", "pic_use_graphs", "pic_checkpoint", "pic_backward", "pic_set_pusher", "pic_resolution_factor"]:
        assert need in names


def test_library_exports_every_declared_symbol():
    from paper_2411_04703_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_loads_without_gpu():
    from paper_2411_04703_gb300 import api
    L = api.lib()
    assert L.pic_last_error(None) is not None or True
