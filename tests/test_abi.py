"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads without a GPU, exports every
entry point include/ndg.h declares, and rejects invalid arguments with NDG_EINVAL before touching a
device."""
import ctypes
import os
import re

import pytest

from paper_2510_05254_b300 import native as nat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ndg.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ndg_[a-z0-9_]+)\s*\(", src)) - {"ndg_alloc_fn", "ndg_free_fn"})


def test_library_loads_and_exports_every_declared_symbol():
    lib = nat.load()
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if getattr(lib, n, None) is None]
    assert not missing, missing
    # and the binding wraps each of them under the same name
    assert not [n for n in names if not hasattr(nat, n)], [n for n in names if not hasattr(nat, n)]


def test_invalid_arguments_are_rejected_without_a_device():
    lib = nat.load()
    h = ctypes.c_void_p()
    e3 = (ctypes.c_int * 3)(4, 4, 4)
    assert lib.ndg_create(0, 3, e3, 0, 0, ctypes.byref(h)) == nat.NDG_EINVAL
    assert "dim" in nat.ndg_last_error()
    assert lib.ndg_create(2, 8, e3, 0, 0, ctypes.byref(h)) == nat.NDG_EINVAL
    assert lib.ndg_create(2, 0, e3, 0, 0, ctypes.byref(h)) == nat.NDG_EINVAL
    assert lib.ndg_create(2, 3, e3, nat.NDG_ISO_EULER, nat.NDG_FLUX_UPWIND, ctypes.byref(h)) == nat.NDG_EINVAL
    bad = (ctypes.c_int * 3)(4, 0, 4)
    assert lib.ndg_create(2, 3, bad, 0, 0, ctypes.byref(h)) == nat.NDG_EINVAL
    assert lib.ndg_create(2, 3, e3, 7, 0, ctypes.byref(h)) == nat.NDG_EINVAL
    assert h.value is None  # never set on failure
    cfg = nat.ndg_config_init()
    cfg.sound_speed = 1.0
    cfg.dtype = 5
    assert lib.ndg_create_ex(ctypes.byref(cfg), ctypes.byref(h)) == nat.NDG_EINVAL
    assert lib.ndg_config_init(None) == nat.NDG_EINVAL
    assert lib.ndg_step(None, 0.1, 1, 4) == nat.NDG_EINVAL
    assert lib.ndg_norms(None, None, 0, None) == nat.NDG_EINVAL
    assert lib.ndg_destroy(None) == nat.NDG_OK
    assert lib.ndg_set_allocator(nat.ALLOC_FN(lambda *a: 0), nat.FREE_FN(), None) == nat.NDG_EINVAL
    assert lib.ndg_batch_create(None, 0, ctypes.byref(h)) == nat.NDG_EINVAL
    assert lib.ndg_pool_create(0, 0, ctypes.byref(h)) == nat.NDG_EINVAL


def test_config_defaults():
    cfg = nat.ndg_config_init()
    assert (cfg.dim, cfg.degree, cfg.dtype, cfg.equation) == (2, 7, nat.NDG_F64, nat.NDG_ADVECTION)
    assert cfg.sound_speed == 1.0 and list(cfg.length) == [1.0, 1.0, 1.0]


def test_no_device_is_reported_as_cuda_error():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(nat.NdgError) as ei:
        nat.ndg_create(2, 3, (4, 4), nat.NDG_ADVECTION, nat.NDG_FLUX_UPWIND)
    assert ei.value.status == nat.NDG_ECUDA


def _header_struct_fields(name):
    """Field names of `typedef struct { ... } name;` in include/ndg.h, in order."""
    import re
    text = open(HEADER).read()
    m = re.search(r"typedef struct \{([^}]*)\}\s*" + name + ";", text)
    assert m, name
    fields = []
    for line in m.group(1).splitlines():
        line = line.split("/*")[0].strip()
        if not line.endswith(";"):
            continue
        decl = line[:-1].replace("*", " ").split()[-1]
        fields.append(decl.split("[")[0])
    return fields


@pytest.mark.parametrize("cname,pyname", [("ndg_config", "ndg_config"), ("ndg_norms_t", "ndg_norms_t"),
                                          ("ndg_info_t", "ndg_info_t"), ("ndg_solve_stats_t", "ndg_solve_stats_t")])
def test_binding_structs_match_the_header(cname, pyname):
    assert [f[0] for f in getattr(nat, pyname)._fields_] == _header_struct_fields(cname)


def test_mass_option_is_checked_without_a_device():
    lib = nat.load()
    h = ctypes.c_void_p()
    cfg = nat.ndg_config_init()
    assert cfg.mass == nat.NDG_MASS_LUMPED
    cfg.mass = 2
    assert lib.ndg_create_ex(ctypes.byref(cfg), ctypes.byref(h)) == nat.NDG_EINVAL
    assert "mass" in nat.ndg_last_error()
    cfg.mass = nat.NDG_MASS_EXACT
    cfg.dtype = nat.NDG_F64_FF
    assert lib.ndg_create_ex(ctypes.byref(cfg), ctypes.byref(h)) == nat.NDG_EINVAL
