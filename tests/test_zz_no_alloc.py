"""The allocation-free additive-CCD entry point (ipc_accd_min_noalloc) gives
the same step bound as ipc_ccd_max_step's alpha_accd, call after call.

It is meant for callers that cannot allocate device memory while running
(a real-time control loop, a framework that owns every device allocation);
its scratch is an array built into the library, so this test also checks
that two calls in a row, which reuse that array, agree, and that the second
call leaves the device's free memory unchanged.  The file name makes pytest
collect it after every other test."""
import ctypes as C

import numpy as np
import pytest

from helpers import small_indent
from paper_2605_24339_b300 import scenes as S

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _noalloc(binding):
    L = binding.lib()
    f = L.ipc_accd_min_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_void_p] * 5 + [C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32)]
    return f


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_24339_b300 import binding
    binding.lib()
    return binding


def _batch3():
    """Three environments of different sizes: pairs must stay inside each."""
    parts, xs = [], []
    for k, (nq, press) in enumerate([(5, 0.05e-3), (7, 0.08e-3), (4, 0.04e-3)]):
        s, xx = small_indent(n_quads=nq, subdiv=2, press=press, seed=30 + k)
        parts.append(s)
        xs.append(xx)
    return S.concat_envs(parts), np.concatenate(xs)


@pytest.mark.parametrize("scene", ["one_env", "three_envs"])
@pytest.mark.parametrize("moving_master", [False, True])
def test_noalloc_matches_ccd_max_step(B, scene, moving_master):
    if scene == "one_env":
        sc, x = small_indent(n_quads=8, subdiv=2, press=0.06e-3, seed=5)
    else:
        sc, x = _batch3()
    ctx = B.Context(sc, precision="fp64")
    rng = np.random.default_rng(7)
    dx = np.zeros_like(x)
    if moving_master:
        xm1 = sc.Y0 + np.array([0.0, 0.0, 2.5e-4])
    else:
        dx[:, 2] = -(2e-4 + 2e-4 * rng.random(x.shape[0]))
        dx[:, :2] = 3e-5 * rng.normal(size=(x.shape[0], 2))
        xm1 = None
    ref = ctx.ccd_max_step(x, dx, sc.Y0, xm1)
    assert 0 < ref["alpha_accd"] < 1
    f = _noalloc(B)
    xt, dxt, xm0t = ctx._as(x), ctx._as(dx), ctx._as(sc.Y0)
    xm1t = ctx._as(xm1)
    torch.cuda.synchronize()
    for call in range(2):                    # two calls in a row share the scratch
        free0 = torch.cuda.mem_get_info()[0]
        a = C.c_double(-1.0)
        n = (C.c_int64 * 2)()
        cap = C.c_int32(-1)
        st = f(ctx.h, _ptr(xt), _ptr(dxt), _ptr(xm0t), _ptr(xm1t), C.byref(a), n, C.byref(cap))
        assert st == 0, B.lib().ipc_last_error(ctx.h)
        if call == 1:                        # the device's free memory did not move
            assert torch.cuda.mem_get_info()[0] == free0
        assert a.value == ref["alpha_accd"]  # ACCD results are bit-identical
        assert (n[0], n[1]) == (ref["n_pt"], ref["n_ee"])
        assert cap.value == int(ref["iter_cap_hit"]) == 0
    ctx.close()


def test_noalloc_reports_iteration_cap(B):
    """With an iteration cap of 1 the additive CCD stops at its first safe
    time on some pair: the flag says so, as ipc_ccd_max_step's does."""
    sc, x = small_indent(n_quads=6, subdiv=2, press=0.06e-3, seed=6)
    ctx = B.Context(sc, precision="fp64", params={"ccd_max_iter": 1})
    dx = np.zeros_like(x)
    dx[:, 2] = -3e-4
    ref = ctx.ccd_max_step(x, dx, sc.Y0)
    assert ref["iter_cap_hit"]
    f = _noalloc(B)
    a = C.c_double(-1.0)
    cap = C.c_int32(-1)
    xt, dxt, xm0t = ctx._as(x), ctx._as(dx), ctx._as(sc.Y0)   # kept alive across the call
    st = f(ctx.h, _ptr(xt), _ptr(dxt), _ptr(xm0t), None, C.byref(a), None, C.byref(cap))
    assert st == 0, B.lib().ipc_last_error(ctx.h)
    assert cap.value == 1 and a.value == ref["alpha_accd"]
    ctx.close()


def test_noalloc_rejects_oversized_moving_master(B):
    pad, _ = small_indent(n_quads=2, subdiv=1)
    Y, F = S.height_field(420, 20e-3, 0.5e-3, 2e-3, seed=2)   # 177,241 master vertices
    Y[:, 2] -= 1e-3
    pad.Y0, pad.mtris = Y, F
    pad.env_mvert_off = np.array([0, Y.shape[0]])
    pad.env_mtri_off = np.array([0, F.shape[0]])
    ctx = B.Context(pad, precision="fp64")
    f = _noalloc(B)
    x = ctx._as(pad.X)
    dx, Yt = torch.zeros_like(x), ctx._as(Y)
    a = C.c_double()
    st = f(ctx.h, _ptr(x), _ptr(dx), _ptr(Yt), _ptr(Yt), C.byref(a), None, None)
    assert st == 5
    assert b"174752" in B.lib().ipc_last_error(ctx.h)
    ctx.close()
