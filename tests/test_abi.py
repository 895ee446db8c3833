"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point that include/rb.h declares; the Python binding has the same names.
No compute call is made here."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(rb_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_1110_4876_gb300 import build, rb

    path = build.build()
    lib = ctypes.CDLL(path)
    declared = _declared()
    assert {"rb_create", "rb_set_particles", "rb_step", "rb_get_particles", "rb_energy"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), name
        assert hasattr(rb, name), name


def test_create_rejects_bad_config_without_gpu():
    """Argument checks happen before any device call."""
    from paper_1110_4876_gb300 import rb

    rb.load()
    cfg = rb.make_config(theta=-1.0, box=(1.0, 1.0, 1.0))
    h = ctypes.c_void_p()
    assert rb.load().rb_create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == rb.RB_ERR_ARG
    assert "theta" in rb.rb_last_error(None)
    cfg = rb.make_config(box=(1.0, 2.0, 1.0))
    assert rb.load().rb_create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == rb.RB_ERR_ARG
    cfg = rb.make_config(integrator=rb.RB_INT_SEI, omega=0.0)
    assert rb.load().rb_create(ctypes.byref(cfg), 1, None, ctypes.byref(h)) == rb.RB_ERR_ARG


def test_sort_rejects_bad_arguments_without_gpu():
    """rb_sort_pairs_u64 checks its sizes and key width before any device
    call; an empty sort is a no-op."""
    from paper_1110_4876_gb300 import rb

    lib = rb.load()
    k = (ctypes.c_uint64 * 4)()
    assert lib.rb_sort_pairs_u64(-1, 4, 64, k, None, None) == rb.RB_ERR_ARG
    assert lib.rb_sort_pairs_u64(4, 3, 64, k, None, None) == rb.RB_ERR_ARG
    assert lib.rb_sort_pairs_u64(4, 4, 0, k, None, None) == rb.RB_ERR_ARG
    assert lib.rb_sort_pairs_u64(4, 4, 65, k, None, None) == rb.RB_ERR_ARG
    assert lib.rb_sort_pairs_u64(4, 1 << 30, 64, k, None, None) == rb.RB_ERR_ARG
    assert lib.rb_sort_pairs_u64(4, 4, 64, None, None, None) == rb.RB_ERR_ARG
    assert b"rb_sort_pairs_u64" in lib.rb_last_error(None)
    assert lib.rb_sort_pairs_u64(0, 0, 64, None, None, None) == rb.RB_OK
