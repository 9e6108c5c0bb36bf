"""The C-ABI library loads on a host without a GPU and exports every entry
point that include/gmcp.h declares; without a device it fails loudly (no CPU
fallback)."""
import ctypes as C

import pytest

from paper_2605_24339_b300 import binding


def test_library_exports_header_symbols():
    syms = binding.header_symbols()
    assert {"ipc_create", "ipc_candidates", "ipc_barrier_eval", "ipc_ccd_max_step",
            "ipc_newton_step", "ipc_destroy", "ipc_last_error", "ipc_profile"} <= set(syms)
    L = C.CDLL(binding.LIB_PATH)
    missing = [s for s in syms if not hasattr(L, s)]
    assert not missing, missing


def test_create_without_device_fails_loudly():
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2605_24339_b300 import scenes as S
    sc = S.tactile_indent(n_quads=2, side=1e-3, nz=1, thick=0.5e-3, sphere_subdiv=0, radius=1e-3)
    L = binding.lib()
    scn, keep = binding.scene_struct(sc)
    prm = binding.make_params(sc.params)
    h = C.c_void_p()
    st = L.ipc_create(C.byref(prm), C.byref(scn), C.byref(h))
    assert st == 2 and not h.value
    assert b"device" in L.ipc_last_error(None)


def test_null_arguments_rejected():
    L = binding.lib()
    h = C.c_void_p()
    assert L.ipc_create(None, None, C.byref(h)) == 1
    assert L.ipc_create(None, None, None) == 1
    assert L.ipc_candidates(None, None, None, None) == 1
    assert L.ipc_barrier_eval(None, None, None, None, None, None, None, None) == 1
    L.ipc_destroy(None)
