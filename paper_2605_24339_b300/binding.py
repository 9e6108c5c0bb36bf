"""Thin ctypes binding of libgmcp (C ABI in include/gmcp.h).

Argument marshalling only: every step of the contact pass runs in the CUDA
library.  PyTorch supplies device memory and the stream.  There is no CPU
fallback: :func:`lib` raises if the library has not been built, and the
library itself fails with IPC_ERR_CUDA when no usable device is present.
"""
from __future__ import annotations

import ctypes as C
import os
import re
from typing import Optional

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libgmcp.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "gmcp.h")

STATUS = {0: "IPC_OK", 1: "IPC_ERR_ARG", 2: "IPC_ERR_CUDA", 3: "IPC_ERR_OOM",
          4: "IPC_ERR_INFEASIBLE", 5: "IPC_ERR_CAPACITY", 6: "IPC_ERR_NOT_CONVERGED",
          7: "IPC_ERR_LINESEARCH", 8: "IPC_ERR_TIMEOUT"}
PREC = {"fp64": 0, "mixed": 1}


class GmcpError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("precision", C.c_int32), ("dhat", C.c_double), ("kappa", C.c_double),
                ("kappa_edge", C.c_double), ("kappa_point", C.c_double), ("delta_T", C.c_double),
                ("delta_e", C.c_double), ("face_rule_level", C.c_int32), ("h", C.c_double),
                ("density", C.c_double), ("youngs", C.c_double), ("poisson", C.c_double),
                ("gravity", C.c_double * 3), ("newton_tol", C.c_double), ("pcg_rel_tol", C.c_double),
                ("max_newton", C.c_int32), ("max_pcg", C.c_int32), ("max_halvings", C.c_int32),
                ("ccd_slack", C.c_double), ("ccd_max_iter", C.c_int32), ("dhat_guard", C.c_double),
                ("kappa_guard", C.c_double), ("device", C.c_int32), ("stream", C.c_void_p),
                ("use_graphs", C.c_int32), ("face_sampler", C.c_int32)]


class SceneC(C.Structure):
    _fields_ = [("n_env", C.c_int32), ("env_vert_off", C.c_void_p), ("env_tet_off", C.c_void_p),
                ("env_stri_off", C.c_void_p), ("env_mvert_off", C.c_void_p),
                ("env_mtri_off", C.c_void_p), ("n_vert", C.c_int64), ("n_tet", C.c_int64),
                ("n_stri", C.c_int64), ("n_mvert", C.c_int64), ("n_mtri", C.c_int64),
                ("pad_rest", C.c_void_p), ("tets", C.c_void_p), ("s_tris", C.c_void_p),
                ("dirichlet", C.c_void_p), ("m_rest", C.c_void_p), ("m_tris", C.c_void_p)]


class CandCounts(C.Structure):
    _fields_ = [("face", C.c_int64), ("edge", C.c_int64), ("point", C.c_int64),
                ("max_per_tri", C.c_int32 * 3)]


class SampleCounts(C.Structure):
    _fields_ = [("face", C.c_int64), ("edge", C.c_int64), ("point", C.c_int64),
                ("guard", C.c_int64), ("face_evaluated", C.c_int64), ("query_tris", C.c_int64)]


class BsrView(C.Structure):
    _fields_ = [("n_rows", C.c_int64), ("nnzb", C.c_int64), ("row_ptr_dev", C.c_void_p),
                ("col_idx_dev", C.c_void_p), ("vals_dev", C.c_void_p), ("dtype", C.c_int32)]


class CcdInfo(C.Structure):
    _fields_ = [("alpha", C.c_double), ("alpha_lin", C.c_double), ("alpha_accd", C.c_double),
                ("n_pairs_pt", C.c_int64), ("n_pairs_ee", C.c_int64), ("iter_cap_hit", C.c_int32),
                ("swept_tris", C.c_int64)]


class StepStats(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("pcg_iters_total", C.c_int32),
                ("line_search_halvings", C.c_int32), ("residual", C.c_double),
                ("res0", C.c_double), ("alpha0", C.c_double), ("last_alpha", C.c_double),
                ("energy", C.c_double), ("ms_total", C.c_double), ("pred_used", C.c_int32)]


class MasterBody(C.Structure):
    _fields_ = [("n_mtet", C.c_int64), ("m_tets", C.c_void_p), ("m_dirichlet", C.c_void_p),
                ("pattern_radius", C.c_double)]


class WsParams(C.Structure):
    _fields_ = [("params_host", C.c_void_p), ("lr", C.c_double), ("beta1", C.c_double),
                ("beta2", C.c_double), ("eps", C.c_double), ("pos_scale", C.c_double),
                ("disp_scale", C.c_double), ("force_scale", C.c_double)]


WS_NPARAM = 140803


# ipc_status values a time step may end with without a programming error
STEP_INFEASIBLE, STEP_NOT_CONVERGED, STEP_LINESEARCH = 4, 6, 7


_lib = None


def header_symbols():
    """Names of the functions declared in include/gmcp.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ipc_[a-z_0-9]+)\s*\(", txt)))


def lib():
    """Load libgmcp.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -m paper_2605_24339_b300.build`")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    L.ipc_create.restype = C.c_int
    L.ipc_create.argtypes = [C.POINTER(Params), C.POINTER(SceneC), C.POINTER(P)]
    L.ipc_destroy.restype = None; L.ipc_destroy.argtypes = [P]
    L.ipc_last_error.restype = C.c_char_p; L.ipc_last_error.argtypes = [P]
    L.ipc_candidates.restype = C.c_int
    L.ipc_candidates.argtypes = [P, P, P, C.POINTER(CandCounts)]
    L.ipc_candidates_copy.restype = C.c_int
    L.ipc_candidates_copy.argtypes = [P, C.c_int32, P, C.c_int64, C.POINTER(C.c_int64)]
    L.ipc_barrier_eval.restype = C.c_int
    L.ipc_barrier_eval.argtypes = [P, P, P, P, C.POINTER(C.c_double), P, C.POINTER(BsrView),
                                   C.POINTER(SampleCounts)]
    L.ipc_master_grad.restype = C.c_int
    L.ipc_master_grad.argtypes = [P, P, P, P]
    L.ipc_set_item_capacity.restype = C.c_int
    L.ipc_set_item_capacity.argtypes = [P, C.c_int64]
    L.ipc_master_hess.restype = C.c_int
    L.ipc_master_hess.argtypes = [P, P, P, C.c_int64, P, P, C.POINTER(C.c_int64)]
    L.ipc_ccd_max_step.restype = C.c_int
    L.ipc_ccd_max_step.argtypes = [P, P, P, P, P, C.POINTER(C.c_double), C.POINTER(CcdInfo)]
    L.ipc_contact_pass.restype = C.c_int
    L.ipc_contact_pass.argtypes = [P, P, P, P, P, P, C.POINTER(C.c_double), P, C.POINTER(BsrView),
                                   C.POINTER(C.c_double), C.POINTER(CcdInfo), C.POINTER(SampleCounts)]
    L.ipc_contact_pass_host.restype = C.c_int
    L.ipc_contact_pass_host.argtypes = [P, P, P, P, P, P, P, P, C.POINTER(C.c_double), P, C.POINTER(BsrView),
                                        C.POINTER(C.c_double), C.POINTER(CcdInfo), C.POINTER(SampleCounts)]
    L.ipc_profile.restype = C.c_int
    L.ipc_profile.argtypes = [P, C.c_int32, C.c_int32, P, P, P, C.POINTER(C.c_int32)]
    L.ipc_ws_create.restype = C.c_int
    L.ipc_ws_create.argtypes = [P, C.POINTER(WsParams)]
    L.ipc_ws_features.restype = C.c_int
    L.ipc_ws_features.argtypes = [P, P, P, P, P]
    L.ipc_ws_forward.restype = C.c_int
    L.ipc_ws_forward.argtypes = [P, P, P]
    L.ipc_ws_grads.restype = C.c_int
    L.ipc_ws_grads.argtypes = [P, P, P, P, C.POINTER(C.c_double), P]
    L.ipc_ws_train_step.restype = C.c_int
    L.ipc_ws_train_step.argtypes = [P, P, P, P, C.POINTER(C.c_double)]
    L.ipc_ws_get_params.restype = C.c_int
    L.ipc_ws_get_params.argtypes = [P, P]
    L.ipc_ws_predict.restype = C.c_int
    L.ipc_ws_predict.argtypes = [P, P, P, P, P]
    L.ipc_save.restype = C.c_int
    L.ipc_save.argtypes = [P, C.c_char_p, P, P]
    L.ipc_load.restype = C.c_int
    L.ipc_load.argtypes = [P, C.c_char_p, P, P, C.POINTER(C.c_int64)]
    L.ipc_autotune.restype = C.c_int
    L.ipc_autotune.argtypes = [P, P, P, P, C.c_int32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                               C.POINTER(C.c_double)]
    L.ipc_slave_vertices.restype = C.c_int
    L.ipc_slave_vertices.argtypes = [P, P, C.POINTER(C.c_int64)]
    L.ipc_scatter_slave.restype = C.c_int
    L.ipc_scatter_slave.argtypes = [P, P, P]
    L.ipc_set_launch_shape.restype = C.c_int
    L.ipc_set_launch_shape.argtypes = [P, C.c_int32, C.c_int32]
    L.ipc_newton_step.restype = C.c_int
    L.ipc_newton_step.argtypes = [P, P, P, P, P, C.POINTER(StepStats)]
    L.ipc_set_master_body.restype = C.c_int
    L.ipc_set_master_body.argtypes = [P, C.POINTER(MasterBody)]
    L.ipc_newton_step_joint.restype = C.c_int
    L.ipc_newton_step_joint.argtypes = [P, P, P, P, C.POINTER(StepStats)]
    L.ipc_newton_step_envs.restype = C.c_int
    L.ipc_newton_step_envs.argtypes = [P, P, P, P, P, C.POINTER(StepStats), P]
    L.ipc_dual_map_build.restype = C.c_int
    L.ipc_dual_map_build.argtypes = [P, C.c_int64, P, C.c_int64, P, C.c_int64, P, P, P, P]
    L.ipc_face_clip_samples.restype = C.c_int
    L.ipc_face_clip_samples.argtypes = [P, C.c_int64, P, C.c_int64, P, C.c_int64, P, C.c_int64, P, C.c_int64,
                                        P, P, P]
    L.ipc_dual_map_apply.restype = C.c_int
    L.ipc_dual_map_apply.argtypes = [P, P, C.c_int64, P, P, C.c_int64, P, P]
    _lib = L
    return L


def _dm_check(st):
    if st != 0:
        raise GmcpError(st, lib().ipc_last_error(None).decode())


def dual_map_build(V, T, P, stream=0):
    """ipc_dual_map_build on CUDA tensors: V float64 [nv, 3], T int32
    [nt, 3] (simulation surface), P float64 [np, 3] (visual vertices).
    Returns (tri int32 [np], uvwd float64 [np, 4], dist2 float64 [np])."""
    import torch
    V = V.contiguous(); T = T.contiguous(); P = P.contiguous()
    n = P.shape[0]
    tri = torch.empty(n, dtype=torch.int32, device=P.device)
    uvwd = torch.empty((n, 4), dtype=torch.float64, device=P.device)
    d2 = torch.empty(n, dtype=torch.float64, device=P.device)
    _dm_check(lib().ipc_dual_map_build(_ptr(V), V.shape[0], _ptr(T), T.shape[0], _ptr(P), n, _ptr(tri),
                                       _ptr(uvwd), _ptr(d2), C.c_void_p(stream)))
    return tri, uvwd, d2


def alu_peak(kind, device=0, stream=0):
    """ipc_alu_peak: measured FP32 (kind 0) or FP64 (kind 1) FMA rate, TFLOP/s."""
    out = C.c_double()
    f = lib().ipc_alu_peak
    f.restype = C.c_int
    f.argtypes = [C.c_int32, C.c_int32, C.c_void_p, C.POINTER(C.c_double)]
    _dm_check(f(int(kind), int(device), C.c_void_p(stream), C.byref(out)))
    return out.value


def face_clip_samples(xs, ts, xm, tm, pairs, stream=0):
    """ipc_face_clip_samples on CUDA tensors; returns (samples float64
    [n, 12, 8], count int32 [n])."""
    import torch
    xs, ts, xm, tm, pairs = (a.contiguous() for a in (xs, ts, xm, tm, pairs))
    n = pairs.shape[0]
    smp = torch.zeros((n, 12, 8), dtype=torch.float64, device=xs.device)
    cnt = torch.zeros(n, dtype=torch.int32, device=xs.device)
    _dm_check(lib().ipc_face_clip_samples(_ptr(xs), xs.shape[0], _ptr(ts), ts.shape[0], _ptr(xm), xm.shape[0],
                                          _ptr(tm), tm.shape[0], _ptr(pairs), n, _ptr(smp), _ptr(cnt),
                                          C.c_void_p(stream)))
    return smp, cnt


def dual_map_apply(V, T, tri, uvwd, out=None, stream=0):
    """ipc_dual_map_apply: the visual vertices for the deformed simulation
    vertices V (float64 [nv, 3]); returns out (float64 [np, 3])."""
    import torch
    V = V.contiguous()
    if out is None:
        out = torch.empty((tri.shape[0], 3), dtype=torch.float64, device=V.device)
    _dm_check(lib().ipc_dual_map_apply(_ptr(V), _ptr(T), T.shape[0], _ptr(tri), _ptr(uvwd), tri.shape[0],
                                       _ptr(out), C.c_void_p(stream)))
    return out


def make_params(p: dict, precision="fp64", device=0, stream=0) -> Params:
    q = Params()
    q.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    for k in ("dhat", "kappa", "kappa_edge", "kappa_point", "delta_T", "delta_e", "h", "density",
              "youngs", "poisson", "newton_tol", "pcg_rel_tol", "ccd_slack"):
        setattr(q, k, float(p[k]))
    q.face_rule_level = int(p["face_rule_level"])
    q.gravity = (C.c_double * 3)(*[float(v) for v in p["gravity"]])
    q.max_newton, q.max_pcg = int(p["max_newton"]), int(p["max_pcg"])
    q.max_halvings = int(p["max_halvings"])
    q.ccd_max_iter = int(p["ccd_max_iter"])
    q.dhat_guard = float(p.get("dhat_guard") or 0.0)
    q.kappa_guard = float(p.get("kappa_guard") or 0.0)
    q.device = int(device)
    q.stream = C.c_void_p(int(stream)) if stream else None
    q.use_graphs = int(p.get("use_graphs", 1))
    q.face_sampler = int(p.get("face_sampler", 0))
    return q


def scene_struct(scene):
    """(SceneC, keep-alive dict) of host arrays for ipc_create."""
    k = dict(
        ev=np.ascontiguousarray(scene.env_vert_off, dtype=np.int64),
        et=np.ascontiguousarray(scene.env_tet_off, dtype=np.int64),
        es=np.ascontiguousarray(scene.env_stri_off, dtype=np.int64),
        emv=np.ascontiguousarray(scene.env_mvert_off, dtype=np.int64),
        emt=np.ascontiguousarray(scene.env_mtri_off, dtype=np.int64),
        X=np.ascontiguousarray(scene.X, dtype=np.float64),
        T=np.ascontiguousarray(scene.tets, dtype=np.int32),
        S=np.ascontiguousarray(scene.stris, dtype=np.int32),
        D=np.ascontiguousarray(scene.dirichlet, dtype=np.uint8),
        Y=np.ascontiguousarray(scene.Y0, dtype=np.float64),
        M=np.ascontiguousarray(scene.mtris, dtype=np.int32))
    sc = SceneC()
    sc.n_env = int(len(k["ev"]) - 1)
    sc.env_vert_off, sc.env_tet_off = k["ev"].ctypes.data, k["et"].ctypes.data
    sc.env_stri_off, sc.env_mvert_off = k["es"].ctypes.data, k["emv"].ctypes.data
    sc.env_mtri_off = k["emt"].ctypes.data
    sc.n_vert, sc.n_tet, sc.n_stri = k["X"].shape[0], k["T"].shape[0], k["S"].shape[0]
    sc.n_mvert, sc.n_mtri = k["Y"].shape[0], k["M"].shape[0]
    sc.pad_rest, sc.tets, sc.s_tris = k["X"].ctypes.data, k["T"].ctypes.data, k["S"].ctypes.data
    sc.dirichlet, sc.m_rest, sc.m_tris = k["D"].ctypes.data, k["Y"].ctypes.data, k["M"].ctypes.data
    return sc, k


class _CudaArray:
    """Zero-copy wrapper of context-owned device memory for torch.as_tensor."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


class Context:
    """One libgmcp context over a :class:`scenes.Scene` on ``device``.

    Positions passed to the methods are torch CUDA tensors (or arrays that are
    copied to the device), FP64 contiguous ``[n,3]``.  Work is queued on the
    torch stream current at construction."""

    def __init__(self, scene, precision="fp64", device=0, params: Optional[dict] = None,
                 stream=None):
        import torch
        self.torch = torch
        L = lib()
        p = dict(scene.params)
        if params:
            p.update(params)
        self.params = p
        self.precision = precision
        self.device = torch.device("cuda", device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        sc, self._keep = scene_struct(scene)
        self._prm = make_params(p, precision, device, stream.cuda_stream)
        h = C.c_void_p()
        st = L.ipc_create(C.byref(self._prm), C.byref(sc), C.byref(h))
        if st != 0:
            raise GmcpError(st, L.ipc_last_error(None).decode())
        self.h = h
        self.nv, self.ns, self.nmv = sc.n_vert, sc.n_stri, sc.n_mvert
        self.n_env = int(sc.n_env)
        self.joint = getattr(scene, "mtets", None) is not None
        if self.joint:
            # deformable master: the scene's master body joins the time step
            mt = np.ascontiguousarray(scene.mtets, dtype=np.int32)
            md = getattr(scene, "mdirichlet", None)
            md = np.ascontiguousarray(md if md is not None else np.zeros(self.nmv), dtype=np.uint8)
            self._mbody = (mt, md)
            body = MasterBody(mt.shape[0], mt.ctypes.data, md.ctypes.data, float(p.get("joint_radius", 0.0)))
            self._check(L.ipc_set_master_body(self.h, C.byref(body)))

    def close(self):
        if getattr(self, "h", None):
            lib().ipc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != 0:
            raise GmcpError(st, lib().ipc_last_error(self.h).decode())

    def _as(self, a):
        t = self.torch
        if a is None:
            return None
        if not isinstance(a, t.Tensor):
            a = t.as_tensor(np.asarray(a, dtype=np.float64))
        return a.to(device=self.device, dtype=t.float64).contiguous()

    # -- broad phase -------------------------------------------------------
    def candidates(self, x, xm):
        x, xm = self._as(x), self._as(xm)
        cc = CandCounts()
        self._check(lib().ipc_candidates(self.h, _ptr(x), _ptr(xm), C.byref(cc)))
        return dict(face=cc.face, edge=cc.edge, point=cc.point, max_per_tri=tuple(cc.max_per_tri))

    def candidate_pairs(self, kind: int) -> np.ndarray:
        n = C.c_int64()
        self._check(lib().ipc_candidates_copy(self.h, kind, None, 0, C.byref(n)))
        out = np.zeros((max(n.value, 1), 2), dtype=np.int32)
        self._check(lib().ipc_candidates_copy(self.h, kind, out.ctypes.data, n.value, C.byref(n)))
        return out[: n.value]

    # -- contact pass ------------------------------------------------------
    def barrier_eval(self, x, xm, grad=True, hess=True, counts=True, energy_dev=None, grad_out=None):
        t = self.torch
        x, xm = self._as(x), self._as(xm)
        gdt = t.float32 if self.precision == "mixed" else t.float64
        g = grad_out
        if g is None and grad:
            g = t.empty((self.nv, 3), dtype=gdt, device=self.device)
        e = C.c_double()
        bv = BsrView()
        sc = SampleCounts()
        self._check(lib().ipc_barrier_eval(self.h, _ptr(x), _ptr(xm), _ptr(energy_dev),
                                           None if energy_dev is not None else C.byref(e), _ptr(g),
                                           C.byref(bv) if hess else None,
                                           C.byref(sc) if counts else None))
        out = dict(energy=e.value if energy_dev is None else None, grad=g)
        if counts:
            out["counts"] = dict(face=sc.face, edge=sc.edge, point=sc.point, guard=sc.guard,
                                 face_evaluated=sc.face_evaluated, query_tris=sc.query_tris)
        if hess == "view":
            out["hess"] = bv
        elif hess:
            out["hess"] = self.bsr(bv)
        return out

    def bsr(self, bv: BsrView):
        """Copies of a BSR view as torch tensors (row_ptr, col_idx, vals [nnzb,3,3])."""
        t = self.torch
        rp = t.as_tensor(_CudaArray(bv.row_ptr_dev, (bv.n_rows + 1,), "<i4"), device=self.device).clone()
        ci = t.as_tensor(_CudaArray(bv.col_idx_dev, (bv.nnzb,), "<i4"), device=self.device).clone()
        ts = "<f4" if bv.dtype == 1 else "<f8"
        vals = t.as_tensor(_CudaArray(bv.vals_dev, (bv.nnzb, 3, 3), ts), device=self.device).clone()
        return rp, ci, vals

    def set_item_capacity(self, capacity: int):
        """Item-buffer capacity (ipc_set_item_capacity): smaller item sets take
        the item-parallel kernels, larger ones the warp-per-triangle kernel."""
        self._check(lib().ipc_set_item_capacity(self.h, int(capacity)))

    def master_grad(self, x, xm, out=None):
        """dPsi/dx_m over the master vertices, [n_mvert, 3] FP64 (ipc_master_grad)."""
        t = self.torch
        x, xm = self._as(x), self._as(xm)
        if out is None:
            out = t.empty((self.nmv, 3), dtype=t.float64, device=self.device)
        self._check(lib().ipc_master_grad(self.h, _ptr(x), _ptr(xm), _ptr(out)))
        return out

    def master_hess(self, x, xm, capacity=None):
        """Slave-master and master-master Hessian blocks (ipc_master_hess):
        (ij [n, 2] int32 in the joint numbering, blk [n, 3, 3] FP64), with
        repeated (row, col) entries; grows the arrays once if needed."""
        t = self.torch
        x, xm = self._as(x), self._as(xm)
        cap = int(capacity) if capacity is not None else 1 << 16
        n = C.c_int64()
        while True:
            ij = t.empty((max(cap, 1), 2), dtype=t.int32, device=self.device)
            blk = t.empty((max(cap, 1), 3, 3), dtype=t.float64, device=self.device)
            st = lib().ipc_master_hess(self.h, _ptr(x), _ptr(xm), cap, _ptr(ij), _ptr(blk), C.byref(n))
            if st == 5 and n.value > cap:   # IPC_ERR_CAPACITY
                cap = n.value
                continue
            self._check(st)
            return ij[: n.value], blk[: n.value]

    def ccd_max_step(self, x, dx, xm0, xm1=None):
        x, dx, xm0, xm1 = self._as(x), self._as(dx), self._as(xm0), self._as(xm1)
        a = C.c_double()
        info = CcdInfo()
        self._check(lib().ipc_ccd_max_step(self.h, _ptr(x), _ptr(dx), _ptr(xm0), _ptr(xm1),
                                           C.byref(a), C.byref(info)))
        return dict(alpha=info.alpha, alpha_lin=info.alpha_lin, alpha_accd=info.alpha_accd,
                    n_pt=info.n_pairs_pt, n_ee=info.n_pairs_ee, iter_cap_hit=bool(info.iter_cap_hit),
                    swept_tris=info.swept_tris)

    def contact_pass(self, x, xm0, dx=None, xm1=None, grad=True, hess=True, counts=True,
                     energy_dev=None, grad_out=None, host_alpha=True):
        """ipc_contact_pass: barrier evaluation and step bound sharing one broad
        phase.  hess="view" returns the raw BsrView (no copy)."""
        return self._contact_pass(None, None, x, xm0, dx, xm1, grad, hess, counts, energy_dev, grad_out,
                                  host_alpha)

    def contact_pass_host(self, xs_host, dxs_host, x, dx, xm0, xm1=None, grad=True, hess=True, counts=True,
                          energy_dev=None, grad_out=None, host_alpha=True):
        """ipc_contact_pass_host: the slave vertices' positions xs_host and
        displacements dxs_host (page-locked CPU tensors [n_svert, 3], FP64, in
        slave_vertices() order; dxs_host may be None with dx None) copied in
        and scattered into x and dx inside the pass; outputs as contact_pass."""
        t = self.torch
        for h in (xs_host, dxs_host):
            if h is not None and (h.device.type != "cpu" or h.dtype != t.float64 or not h.is_contiguous()):
                raise ValueError("host inputs must be contiguous FP64 CPU tensors")
        return self._contact_pass(xs_host, dxs_host, x, xm0, dx, xm1, grad, hess, counts, energy_dev, grad_out,
                                  host_alpha)

    def _contact_pass(self, xs_host, dxs_host, x, xm0, dx, xm1, grad, hess, counts, energy_dev, grad_out,
                      host_alpha):
        t = self.torch
        x, xm0, dx, xm1 = self._as(x), self._as(xm0), self._as(dx), self._as(xm1)
        gdt = t.float32 if self.precision == "mixed" else t.float64
        g = grad_out
        if g is None and grad:
            g = t.empty((self.nv, 3), dtype=gdt, device=self.device)
        e = C.c_double()
        bv = BsrView()
        sc = SampleCounts()
        a = C.c_double()
        info = CcdInfo()
        want_a = dx is not None and host_alpha
        outs = (_ptr(energy_dev), None if energy_dev is not None else C.byref(e), _ptr(g),
                C.byref(bv) if hess else None, C.byref(a) if want_a else None,
                C.byref(info) if want_a else None, C.byref(sc) if counts else None)
        if xs_host is None:
            self._check(lib().ipc_contact_pass(self.h, _ptr(x), _ptr(xm0), _ptr(xm1), _ptr(dx), *outs))
        else:
            self._check(lib().ipc_contact_pass_host(
                self.h, C.c_void_p(xs_host.data_ptr()),
                None if dxs_host is None else C.c_void_p(dxs_host.data_ptr()), _ptr(x), _ptr(dx), _ptr(xm0),
                _ptr(xm1), *outs))
        out = dict(energy=e.value if energy_dev is None else None, grad=g)
        if counts:
            out["counts"] = dict(face=sc.face, edge=sc.edge, point=sc.point, guard=sc.guard,
                                 face_evaluated=sc.face_evaluated, query_tris=sc.query_tris)
        if hess == "view":
            out["hess"] = bv
        elif hess:
            out["hess"] = self.bsr(bv)
        if want_a:
            out.update(alpha=info.alpha, alpha_lin=info.alpha_lin, alpha_accd=info.alpha_accd,
                       n_pt=info.n_pairs_pt, n_ee=info.n_pairs_ee, swept_tris=info.swept_tris)
        return out

    # -- profiling ---------------------------------------------------------
    def profile_start(self):
        self._check(lib().ipc_profile(self.h, 1, 0, None, None, None, None))

    def profile_stop(self):
        self._check(lib().ipc_profile(self.h, 0, 0, None, None, None, None))

    def profile_read(self):
        n = C.c_int32()
        K = 64
        names = C.create_string_buffer(32 * K)
        ms = (C.c_double * K)()
        calls = (C.c_int64 * K)()
        self._check(lib().ipc_profile(self.h, 2, K, names, ms, calls, C.byref(n)))
        out = {}
        for i in range(min(n.value, K)):
            nm = names.raw[32 * i:32 * i + 32].split(b"\0")[0].decode()
            out[nm] = dict(ms=ms[i], calls=calls[i])
        return out

    def newton_step(self, x, v, xm_next=None, dx_pred=None):
        """In-place implicit-Euler step on x, v (torch FP64 CUDA tensors [n,3]).

        Returns the step statistics with ``status`` (0, or STEP_INFEASIBLE,
        STEP_NOT_CONVERGED, STEP_LINESEARCH); other failures raise."""
        t = self.torch
        for a in (x, v):
            if not (isinstance(a, t.Tensor) and a.is_cuda and a.dtype == t.float64 and a.is_contiguous()):
                raise TypeError("x and v must be contiguous FP64 CUDA tensors")
        st = StepStats()
        xm_t, dxp_t = self._as(xm_next), self._as(dx_pred)   # alive until the call returns
        r = lib().ipc_newton_step(self.h, _ptr(x), _ptr(v), _ptr(xm_t), _ptr(dxp_t), C.byref(st))
        if r not in (0, STEP_INFEASIBLE, STEP_NOT_CONVERGED, STEP_LINESEARCH):
            self._check(r)
        return self._stats_dict(st, r)

    @staticmethod
    def _stats_dict(st, status):
        return dict(status=status, newton_iters=st.newton_iters, pcg_iters=st.pcg_iters_total,
                    halvings=st.line_search_halvings, residual=st.residual, res0=st.res0,
                    alpha0=st.alpha0, last_alpha=st.last_alpha, energy=st.energy, ms=st.ms_total,
                    pred_used=st.pred_used)

    def newton_step_joint(self, x, v, f_ext=None):
        """In-place step of the pad and the deformable master together
        (ipc_newton_step_joint): x, v are [n_pad + n_master, 3] FP64 CUDA
        tensors; f_ext the external nodal forces (same shape) or None."""
        t = self.torch
        for a in (x, v):
            if not (isinstance(a, t.Tensor) and a.is_cuda and a.dtype == t.float64 and a.is_contiguous()):
                raise TypeError("x and v must be contiguous FP64 CUDA tensors")
        st = StepStats()
        f_t = self._as(f_ext)   # alive until the call returns
        r = lib().ipc_newton_step_joint(self.h, _ptr(x), _ptr(v), _ptr(f_t), C.byref(st))
        if r not in (0, STEP_INFEASIBLE, STEP_NOT_CONVERGED, STEP_LINESEARCH):
            self._check(r)
        return self._stats_dict(st, r)

    def newton_step_envs(self, x, v, xm_next=None, dx_pred=None):
        """The step of every environment (ipc_newton_step_envs): in place on
        x, v; returns (overall status, [per-environment statistics dicts
        with their own ``status``])."""
        t = self.torch
        for a in (x, v):
            if not (isinstance(a, t.Tensor) and a.is_cuda and a.dtype == t.float64 and a.is_contiguous()):
                raise TypeError("x and v must be contiguous FP64 CUDA tensors")
        ne = self.n_env
        st = (StepStats * ne)()
        status = np.zeros(ne, dtype=np.int32)
        xm_t, dxp_t = self._as(xm_next), self._as(dx_pred)   # alive until the call returns
        r = lib().ipc_newton_step_envs(self.h, _ptr(x), _ptr(v), _ptr(xm_t), _ptr(dxp_t), st,
                                       status.ctypes.data)
        if r not in (0, STEP_INFEASIBLE, STEP_NOT_CONVERGED, STEP_LINESEARCH):
            self._check(r)
        return r, [self._stats_dict(st[e], int(status[e])) for e in range(ne)]

    # -- learned warm start -------------------------------------------------
    def ws_create(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, pos_scale=1e-3,
                  disp_scale=1e-5, force_scale=1e-3):
        """Network with the flattened FP32 parameters ``params`` (length
        WS_NPARAM: W1 b1 W2 b2 W3 b3 W4 b4, row-major)."""
        p = np.ascontiguousarray(params, dtype=np.float32).ravel()
        if p.size != WS_NPARAM:
            raise ValueError(f"expected {WS_NPARAM} parameters, got {p.size}")
        self._ws_keep = p
        w = WsParams(p.ctypes.data, lr, beta1, beta2, eps, pos_scale, disp_scale, force_scale)
        self._check(lib().ipc_ws_create(self.h, C.byref(w)))
        self.ws_disp_scale = disp_scale

    def ws_features(self, x, v, xm):
        t = self.torch
        x, v, xm = self._as(x), self._as(v), self._as(xm)
        f = t.empty((self.nv, 32), dtype=t.bfloat16, device=self.device)
        self._check(lib().ipc_ws_features(self.h, _ptr(x), _ptr(v), _ptr(xm), _ptr(f)))
        return f

    def _feats(self, feats):
        t = self.torch
        if feats is None:
            return None
        if feats.dtype != t.bfloat16 or not feats.is_cuda or feats.shape != (self.nv, 32):
            raise TypeError("features must be a CUDA bfloat16 tensor [n_vert, 32]")
        return feats.contiguous()

    def _f32(self, a, shape):
        t = self.torch
        a = t.as_tensor(a).to(device=self.device, dtype=t.float32).contiguous()
        if tuple(a.shape) != shape:
            raise ValueError(f"expected shape {shape}, got {tuple(a.shape)}")
        return a

    def ws_forward(self, feats=None):
        t = self.torch
        f = self._feats(feats)
        y = t.empty((self.nv, 3), dtype=t.float32, device=self.device)
        self._check(lib().ipc_ws_forward(self.h, _ptr(f), _ptr(y)))
        return y

    def ws_grads(self, feats, target, mask):
        f = self._feats(feats)
        tg, mk = self._f32(target, (self.nv, 3)), self._f32(mask, (self.nv,))
        loss = C.c_double()
        g = np.zeros(WS_NPARAM, dtype=np.float32)
        self._check(lib().ipc_ws_grads(self.h, _ptr(f), _ptr(tg), _ptr(mk), C.byref(loss),
                                       g.ctypes.data))
        return loss.value, g

    def ws_train_step(self, feats, target, mask):
        f = self._feats(feats)
        tg, mk = self._f32(target, (self.nv, 3)), self._f32(mask, (self.nv,))
        loss = C.c_double()
        self._check(lib().ipc_ws_train_step(self.h, _ptr(f), _ptr(tg), _ptr(mk), C.byref(loss)))
        return loss.value

    def ws_params(self):
        out = np.zeros(WS_NPARAM, dtype=np.float32)
        self._check(lib().ipc_ws_get_params(self.h, out.ctypes.data))
        return out

    def ws_predict(self, x, v, xm):
        t = self.torch
        x, v, xm = self._as(x), self._as(v), self._as(xm)
        dx = t.empty((self.nv, 3), dtype=t.float64, device=self.device)
        self._check(lib().ipc_ws_predict(self.h, _ptr(x), _ptr(v), _ptr(xm), _ptr(dx)))
        return dx

    def pass_kernels(self):
        """Kernel launches of one graph-replayed ipc_contact_pass (-1: no graph)."""
        f = lib().ipc_contact_pass_kernels
        f.restype = C.c_int
        f.argtypes = [C.c_void_p, C.POINTER(C.c_int64)]
        n = C.c_int64()
        self._check(f(self.h, C.byref(n)))
        return n.value

    # -- checkpoint / resume -------------------------------------------------
    def save(self, path, x, v):
        """ipc_save: snapshot of (x, v), the master pose, the step count and
        the network to the file at path."""
        x, v = self._as(x), self._as(v)
        self._check(lib().ipc_save(self.h, os.fsencode(path), _ptr(x), _ptr(v)))

    def load(self, path, x, v):
        """ipc_load into the CUDA tensors x, v (FP64 [n_vert, 3], written in
        place); returns the snapshot's step count."""
        n = C.c_int64(-1)
        self._check(lib().ipc_load(self.h, os.fsencode(path), _ptr(x), _ptr(v), C.byref(n)))
        return n.value

    # -- launch shapes ------------------------------------------------------
    def autotune(self, x, xm0, dx=None, reps=3):
        """Pick the launch shapes of the contact pass by timing; returns
        (samples blocks/SM, query blocks/SM, best ms)."""
        x, xm0, dx = self._as(x), self._as(xm0), self._as(dx)
        a, b, ms = C.c_int32(), C.c_int32(), C.c_double()
        self._check(lib().ipc_autotune(self.h, _ptr(x), _ptr(xm0), _ptr(dx), int(reps), C.byref(a),
                                       C.byref(b), C.byref(ms)))
        return a.value, b.value, ms.value

    def slave_vertices(self):
        """Ids of the slave (tactile) surface vertices, ascending (numpy int32)."""
        n = C.c_int64()
        self._check(lib().ipc_slave_vertices(self.h, None, C.byref(n)))
        ids = np.zeros(n.value, dtype=np.int32)
        self._check(lib().ipc_slave_vertices(self.h, ids.ctypes.data, C.byref(n)))
        return ids

    def scatter_slave(self, xs, x):
        """x[ids] = xs on the device (xs [n_slave, 3], x [nv, 3], FP64)."""
        xs, x = self._as(xs), self._as(x)
        self._check(lib().ipc_scatter_slave(self.h, _ptr(xs), _ptr(x)))
        return x

    def set_launch_shape(self, samples_bpsm, query_bpsm):
        self._check(lib().ipc_set_launch_shape(self.h, int(samples_bpsm), int(query_bpsm)))
