"""ctypes front end of the FP64 CPU oracle (``gmcp_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  The product library never loads it.
``build()`` compiles the C source with gcc into ``oracle/_build``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "gmcp_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")

_lib = None


def build(force: bool = False, openmp: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", LIB + ".tmp", SRC, "-lm"]
        subprocess.check_call(cmd)
        os.replace(LIB + ".tmp", LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


P = C.c_void_p
D = C.c_double
I = C.c_int
I64 = C.c_int64
dp = C.POINTER(C.c_double)
ip = C.POINTER(C.c_int32)


class ContactResult(C.Structure):
    _fields_ = [("energy", D), ("n_samples", I64 * 4), ("guard_energy", D), ("tri_energy", dp), ("tri_coef", dp),
                ("tri_normal", dp), ("grad", dp), ("nblk", I64), ("blk_ij", ip), ("blk", dp)]


class AccdInfo(C.Structure):
    _fields_ = [("alpha_accd", D), ("n_pt", I64), ("n_ee", I64), ("n_iter_total", I64),
                ("max_iter_hit", I), ("alpha_type", D * 3)]


class Stats(C.Structure):
    _fields_ = [("status", I), ("newton_iters", I), ("pcg_iters_total", I), ("residual", D),
                ("res0", D), ("alpha0", D), ("last_alpha", D), ("energy", D), ("pred_used", I)]


def _declare(L):
    L.orc_hermite.restype = D; L.orc_hermite.argtypes = [D, D]
    L.orc_barrier.restype = None; L.orc_barrier.argtypes = [D, D, dp, dp, dp]
    L.orc_face_rule.restype = I; L.orc_face_rule.argtypes = [I, dp]
    L.orc_scene_create.restype = P
    L.orc_scene_create.argtypes = [I, P, P, P, P, I, P, I, P, I, P, I, P, D, D, D, D, D, D, I]
    L.orc_scene_free.argtypes = [P]
    L.orc_scene_n_medges.restype = I; L.orc_scene_n_medges.argtypes = [P]
    L.orc_scene_medges.argtypes = [P, P]
    L.orc_candidates.restype = I64; L.orc_candidates.argtypes = [P, I, P, P, C.POINTER(ip)]
    L.orc_free.argtypes = [P]
    L.orc_scene_set_all_pairs.argtypes = [P, I]
    L.orc_scene_set_face_clip.argtypes = [P, I]
    L.orc_set_verbose.argtypes = [I]
    L.orc_scene_set_guard.argtypes = [P, D, D]
    L.orc_contact_lagged.argtypes = [P, P, P, P, I, P, P]
    L.orc_contact_eval.restype = C.POINTER(ContactResult)
    L.orc_contact_eval.argtypes = [P, P, P, I, P]
    L.orc_contact_result_free.argtypes = [C.POINTER(ContactResult)]
    L.orc_samples.restype = I64; L.orc_samples.argtypes = [P, P, P, I, P, C.POINTER(dp)]
    L.orc_alpha_lin.restype = D; L.orc_alpha_lin.argtypes = [P, P, P, P, P]
    L.orc_master_grad.argtypes = [P, P, P, I, P, P]
    L.orc_master_hess.restype = I64
    L.orc_master_hess.argtypes = [P, P, P, I, P, I64, P, P]
    L.orc_pt_dist2.restype = D; L.orc_pt_dist2.argtypes = [P, P, P, P]
    L.orc_ee_dist2.restype = D; L.orc_ee_dist2.argtypes = [P, P, P, P]
    L.orc_face_clip_samples.restype = I; L.orc_face_clip_samples.argtypes = [P, P, P]
    L.orc_dual_map_coords.argtypes = [P, P, P, P, P]
    L.orc_dual_map_build.argtypes = [P, P, C.c_int64, P, C.c_int64, P, P, P]
    L.orc_dual_map_apply.argtypes = [P, P, P, P, C.c_int64, P]
    L.orc_surface_min_dist2.restype = D
    L.orc_surface_min_dist2.argtypes = [P, P, C.c_int64, P, P, C.c_int64]
    L.orc_accd.restype = D; L.orc_accd.argtypes = [I, P, P, D, D, I, C.POINTER(I)]
    L.orc_accd_min.restype = D
    L.orc_accd_min.argtypes = [P, P, P, P, P, D, I, C.POINTER(AccdInfo)]
    L.orc_ccd_max_step.restype = D
    L.orc_ccd_max_step.argtypes = [P, P, P, P, P, D, I, dp, dp]
    L.orc_psd_project.argtypes = [I, P]
    L.orc_nh_tet.restype = I; L.orc_nh_tet.argtypes = [P, D, D, D, P, P, dp, P, P]
    L.orc_sim_create.restype = P
    L.orc_sim_create.argtypes = [P, I, P, I, P, P, D, D, D, D, P, D, D, I, I, I, D, I]
    L.orc_sim_create_joint.restype = P
    L.orc_sim_create_joint.argtypes = [P, I, P, I, P, P, I, P, P, D, D, D, D, P, D, D, I, I, I, D, I]
    L.orc_sim_set_fext.argtypes = [P, P]
    L.orc_sim_free.argtypes = [P]
    L.orc_sim_nnzb.restype = I64; L.orc_sim_nnzb.argtypes = [P]
    L.orc_sim_mass.argtypes = [P, P]
    L.orc_sim_set_master.argtypes = [P, P]
    L.orc_newton_step.restype = I
    L.orc_newton_step.argtypes = [P, P, P, P, P, C.POINTER(Stats)]
    L.orc_newton_system.restype = I; L.orc_newton_system.argtypes = [P, P, P, dp, P, P]
    L.orc_sim_pattern.argtypes = [P, P, P]
    L.orc_pcg_solve.restype = I; L.orc_pcg_solve.argtypes = [P, P, P, P, D, I]
    if hasattr(L, "orc_mlp_forward"):
        L.orc_mlp_forward.argtypes = [I, P, P, P]
        L.orc_mlp_loss_grad.restype = D
        L.orc_mlp_loss_grad.argtypes = [I, P, P, P, P]


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------
def hermite(x, delta):
    return lib().orc_hermite(float(x), float(delta))


def barrier(g, eps):
    B, dB, d2B = D(), D(), D()
    lib().orc_barrier(float(g), float(eps), C.byref(B), C.byref(dB), C.byref(d2B))
    return B.value, dB.value, d2B.value


def face_rule(L):
    out = np.zeros((4 ** L, 3))
    n = lib().orc_face_rule(L, out.ctypes.data_as(dp))
    return out[:n]


def pt_dist2(p, t0, t1, t2):
    a = [_f64(v) for v in (p, t0, t1, t2)]
    return lib().orc_pt_dist2(*[_p(v) for v in a])


def surface_min_dist(xa, ta, xb, tb):
    """Brute-force minimum distance between two triangle surfaces (all
    vertex-triangle pairs both ways and all edge pairs)."""
    xa, xb = _f64(xa), _f64(xb)
    ta = np.ascontiguousarray(ta, dtype=np.int32)
    tb = np.ascontiguousarray(tb, dtype=np.int32)
    d2 = lib().orc_surface_min_dist2(xa.ctypes.data, ta.ctypes.data, ta.shape[0],
                                     xb.ctypes.data, tb.ctypes.data, tb.shape[0])
    return float(np.sqrt(max(d2, 0.0)))


def face_clip_samples(xs, xm):
    """Paper-exact face samples of slave triangle xs [3,3] against master
    triangle xm [3,3] (Sec. 4.1: projection, Sutherland-Hodgman clip, fan,
    3-point Gauss per sub-triangle).  Returns [n, 8]: beta_s[3], beta_m[3],
    g, w."""
    xs, xm = _f64(xs).reshape(9), _f64(xm).reshape(9)
    out = np.zeros((12, 8))
    n = lib().orc_face_clip_samples(_p(xs), _p(xm), _p(out))
    return out[:n].copy()


def dual_map_coords(p, v0, v1, v2):
    """(u, v, w, delta) of point p on triangle (v0, v1, v2): Sec. 3.2,
    Eqs. (decomp), (gram)."""
    a = [_f64(q) for q in (p, v0, v1, v2)]
    out = np.zeros(4)
    lib().orc_dual_map_coords(*[_p(q) for q in a], _p(out))
    return out


def dual_map_build(V, T, P):
    """Dual-mesh mapper precomputation, Sec. 3.2 (Eq. bary_proj): for each
    visual vertex the nearest simulation triangle (brute force, ties to the
    lowest index), its (u, v, w, delta) and the squared distance."""
    V, P = _f64(V).reshape(-1, 3), _f64(P).reshape(-1, 3)
    T = np.ascontiguousarray(T, dtype=np.int32).reshape(-1, 3)
    tri = np.zeros(P.shape[0], dtype=np.int32)
    uvwd = np.zeros((P.shape[0], 4))
    d2 = np.zeros(P.shape[0])
    lib().orc_dual_map_build(V.ctypes.data, T.ctypes.data, T.shape[0], P.ctypes.data, P.shape[0],
                             tri.ctypes.data, uvwd.ctypes.data, d2.ctypes.data)
    return tri, uvwd, d2


def dual_map_apply(V, T, tri, uvwd):
    """Per-frame update, Sec. 3.2, Eq. (bary_interp)."""
    V = _f64(V).reshape(-1, 3)
    T = np.ascontiguousarray(T, dtype=np.int32).reshape(-1, 3)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    uvwd = _f64(uvwd).reshape(-1, 4)
    out = np.zeros((tri.shape[0], 3))
    lib().orc_dual_map_apply(V.ctypes.data, T.ctypes.data, tri.ctypes.data, uvwd.ctypes.data, tri.shape[0],
                             out.ctypes.data)
    return out


def ee_dist2(a0, a1, b0, b1):
    a = [_f64(v) for v in (a0, a1, b0, b1)]
    return lib().orc_ee_dist2(*[_p(v) for v in a])


def accd(kind, x4, p4, s=0.1, tc=1.0, max_iter=100000):
    x4, p4 = _f64(x4).reshape(12), _f64(p4).reshape(12)
    it = I()
    t = lib().orc_accd(kind, _p(x4), _p(p4), s, tc, max_iter, C.byref(it))
    return t, it.value


def psd_project(A):
    A = _f64(A).copy()
    lib().orc_psd_project(A.shape[0], _p(A))
    return A


def nh_tet(Dminv, vol, mu, lam, X4, x4):
    """One tet at rest positions X4 and current positions x4 ([4][3])."""
    Dminv, X4, x4 = _f64(Dminv).reshape(9), _f64(X4).reshape(12), _f64(x4).reshape(12)
    psi = D()
    g = np.zeros(12); H = np.zeros((12, 12))
    ok = lib().orc_nh_tet(_p(Dminv), vol, mu, lam, _p(X4), _p(x4), C.byref(psi), _p(g), _p(H))
    return bool(ok), psi.value, g, H


class Scene:
    """Oracle view of a :class:`paper_2605_24339_b300.scenes.Scene`."""

    def __init__(self, sc, params=None):
        p = dict(sc.params)
        if params:
            p.update(params)
        self.params = p
        self.sc = sc
        self._keep = dict(
            ev=np.ascontiguousarray(sc.env_vert_off, dtype=np.int64),
            es=np.ascontiguousarray(sc.env_stri_off, dtype=np.int64),
            emv=np.ascontiguousarray(sc.env_mvert_off, dtype=np.int64),
            emt=np.ascontiguousarray(sc.env_mtri_off, dtype=np.int64),
            X=_f64(sc.X), S=np.ascontiguousarray(sc.stris, dtype=np.int32),
            Y=_f64(sc.Y0), M=np.ascontiguousarray(sc.mtris, dtype=np.int32))
        k = self._keep
        self.h = lib().orc_scene_create(
            sc.n_env, _p(k["ev"]), _p(k["es"]), _p(k["emv"]), _p(k["emt"]),
            sc.X.shape[0], _p(k["X"]), sc.stris.shape[0], _p(k["S"]),
            sc.Y0.shape[0], _p(k["Y"]), sc.mtris.shape[0], _p(k["M"]),
            p["dhat"], p["kappa"], p["kappa_edge"], p["kappa_point"], p["delta_T"],
            p["delta_e"], int(p["face_rule_level"]))
        lib().orc_scene_set_guard(self.h, p.get("dhat_guard", 0.0), p.get("kappa_guard", 0.0))
        lib().orc_scene_set_face_clip(self.h, int(p.get("face_sampler", 0)))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_scene_free(self.h)
            self.h = None

    def medges(self):
        n = lib().orc_scene_n_medges(self.h)
        out = np.zeros((n, 2), dtype=np.int32)
        lib().orc_scene_medges(self.h, _p(out))
        return out

    def candidates(self, kind, x, xm):
        x, xm = _f64(x), _f64(xm)
        ptr = ip()
        n = lib().orc_candidates(self.h, kind, _p(x), _p(xm), C.byref(ptr))
        out = np.zeros((0, 2), dtype=np.int32)
        if n > 0:
            out = np.ctypeslib.as_array(ptr, shape=(2 * n,)).reshape(n, 2).copy()
        lib().orc_free(ptr)
        return out

    def contact(self, x, xm, subset=None):
        x, xm = _f64(x), _f64(xm)
        sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int32)
        r = lib().orc_contact_eval(self.h, _p(x), _p(xm), 0 if sub is None else len(sub), _p(sub))
        R = r.contents
        ns, nv = self.sc.stris.shape[0], self.sc.X.shape[0]
        nb = R.nblk
        out = dict(
            energy=R.energy,
            n_samples=np.array([R.n_samples[0], R.n_samples[1], R.n_samples[2]]),
            n_guard=R.n_samples[3], guard_energy=R.guard_energy,
            tri_energy=np.ctypeslib.as_array(R.tri_energy, shape=(ns,)).copy(),
            tri_coef=np.ctypeslib.as_array(R.tri_coef, shape=(ns, 9)).copy(),
            tri_normal=np.ctypeslib.as_array(R.tri_normal, shape=(ns, 3)).copy(),
            grad=np.ctypeslib.as_array(R.grad, shape=(nv, 3)).copy(),
            blk_ij=np.ctypeslib.as_array(R.blk_ij, shape=(max(nb, 1), 2))[:nb].copy(),
            blk=np.ctypeslib.as_array(R.blk, shape=(max(nb, 1), 3, 3))[:nb].copy())
        lib().orc_contact_result_free(r)
        return out

    def master_grad(self, x, xm, subset=None):
        """dPsi/dx_m over the master vertices with each sample's normal and
        weights held fixed (Sec. 4.3, Eq. gap), [nmv, 3]; subset: only the
        samples of these slave triangles."""
        x, xm = _f64(x), _f64(xm)
        sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int32)
        out = np.zeros((xm.shape[0], 3))
        lib().orc_master_grad(self.h, _p(x), _p(xm), 0 if sub is None else len(sub), _p(sub), _p(out))
        return out

    def master_hess(self, x, xm, subset=None):
        """Slave-master and master-master blocks (Sec. 4.2-4.3), summed over
        repeats: dict (row, col) -> 3x3, master vertex j numbered nv + j."""
        x, xm = _f64(x), _f64(xm)
        sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int32)
        ns = 0 if sub is None else len(sub)
        n = lib().orc_master_hess(self.h, _p(x), _p(xm), ns, _p(sub), 0, None, None)
        ij = np.zeros((max(n, 1), 2), dtype=np.int32)
        blk = np.zeros((max(n, 1), 3, 3))
        lib().orc_master_hess(self.h, _p(x), _p(xm), ns, _p(sub), n, _p(ij), _p(blk))
        out = {}
        for (r, c), b in zip(ij[:n], blk[:n]):
            key = (int(r), int(c))
            out[key] = out.get(key, 0.0) + b
        return out

    def set_all_pairs(self, flag: bool):
        lib().orc_scene_set_all_pairs(self.h, int(bool(flag)))

    def lagged(self, x, xm, dx, alphas):
        x, xm, dx = _f64(x), _f64(xm), _f64(dx)
        al = _f64(alphas)
        out = np.zeros(al.shape[0])
        lib().orc_contact_lagged(self.h, _p(x), _p(xm), _p(dx), al.shape[0], _p(al), _p(out))
        return out

    def samples(self, x, xm, subset=None):
        x, xm = _f64(x), _f64(xm)
        sub = None if subset is None else np.ascontiguousarray(subset, dtype=np.int32)
        ptr = dp()
        n = lib().orc_samples(self.h, _p(x), _p(xm), 0 if sub is None else len(sub), _p(sub),
                              C.byref(ptr))
        out = np.zeros((0, 11))
        if n > 0:
            out = np.ctypeslib.as_array(ptr, shape=(11 * n,)).reshape(n, 11).copy()
        lib().orc_free(ptr)
        return out

    def alpha_lin(self, x, xm, dx, dxm=None):
        a = [_f64(v) if v is not None else None for v in (x, xm, dx, dxm)]
        return lib().orc_alpha_lin(self.h, *[_p(v) for v in a])

    def accd_min(self, x, dx, xm0, dxm=None):
        a = [_f64(v) if v is not None else None for v in (x, dx, xm0, dxm)]
        info = AccdInfo()
        al = lib().orc_accd_min(self.h, *[_p(v) for v in a], self.params["ccd_slack"],
                                int(self.params["ccd_max_iter"]), C.byref(info))
        return al, info

    def ccd_max_step(self, x, dx, xm0, xm1=None):
        a = [_f64(v) if v is not None else None for v in (x, dx, xm0, xm1)]
        al, aa = D(), D()
        r = lib().orc_ccd_max_step(self.h, *[_p(v) for v in a], self.params["ccd_slack"],
                                   int(self.params["ccd_max_iter"]), C.byref(al), C.byref(aa))
        return r, al.value, aa.value


class Sim:
    """Oracle time stepper over a Scene (keeps the master position state)."""

    def __init__(self, scene: Scene):
        self.scene = scene
        sc, p = scene.sc, scene.params
        self._keep = dict(T=np.ascontiguousarray(sc.tets, dtype=np.int32),
                          Dr=np.ascontiguousarray(sc.dirichlet, dtype=np.uint8),
                          g=_f64(p["gravity"]))
        k = self._keep
        self.joint = getattr(sc, "mtets", None) is not None
        if self.joint:
            # deformable master: the system is the pad, then the master body
            k["MT"] = np.ascontiguousarray(sc.mtets, dtype=np.int32)
            md = getattr(sc, "mdirichlet", None)
            k["MD"] = np.ascontiguousarray(md if md is not None else np.zeros(sc.Y0.shape[0]), dtype=np.uint8)
            self.h = lib().orc_sim_create_joint(
                scene.h, sc.X.shape[0], _p(scene._keep["X"]), sc.tets.shape[0], _p(k["T"]), _p(k["Dr"]),
                k["MT"].shape[0], _p(k["MT"]), _p(k["MD"]), p["h"], p["density"], p["youngs"], p["poisson"],
                _p(k["g"]), p["newton_tol"], p["pcg_rel_tol"], int(p["max_newton"]), int(p["max_pcg"]),
                int(p["max_halvings"]), p["ccd_slack"], int(p["ccd_max_iter"]))
            self.nsys = sc.X.shape[0] + sc.Y0.shape[0]
        else:
            self.h = lib().orc_sim_create(
                scene.h, sc.X.shape[0], _p(scene._keep["X"]), sc.tets.shape[0], _p(k["T"]),
                _p(k["Dr"]), p["h"], p["density"], p["youngs"], p["poisson"], _p(k["g"]),
                p["newton_tol"], p["pcg_rel_tol"], int(p["max_newton"]), int(p["max_pcg"]),
                int(p["max_halvings"]), p["ccd_slack"], int(p["ccd_max_iter"]))
            self.nsys = sc.X.shape[0]

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.orc_sim_free(self.h)
            self.h = None

    @property
    def nnzb(self):
        return lib().orc_sim_nnzb(self.h)

    def mass(self):
        out = np.zeros(self.nsys)
        lib().orc_sim_mass(self.h, _p(out))
        return out

    def set_fext(self, f):
        """External nodal forces [nsys, 3] of the joint step."""
        self._keep["F"] = _f64(f).copy()
        lib().orc_sim_set_fext(self.h, _p(self._keep["F"]))

    def set_master(self, xm):
        xm = _f64(xm)
        lib().orc_sim_set_master(self.h, _p(xm))

    def step(self, x, v, xm_next=None, dx_pred=None):
        x, v = _f64(x).copy(), _f64(v).copy()
        a = [_f64(t) if t is not None else None for t in (xm_next, dx_pred)]
        st = Stats()
        lib().orc_newton_step(self.h, _p(x), _p(v), _p(a[0]), _p(a[1]), C.byref(st))
        return x, v, st

    def pattern(self):
        nv = self.nsys
        rp = np.zeros(nv + 1, dtype=np.int32)
        ci = np.zeros(self.nnzb, dtype=np.int32)
        lib().orc_sim_pattern(self.h, _p(rp), _p(ci))
        return rp, ci

    def system(self, x, v):
        x, v = _f64(x), _f64(v)
        E = D()
        G = np.zeros_like(x)
        A = np.zeros((self.nnzb, 3, 3))
        ok = lib().orc_newton_system(self.h, _p(x), _p(v), C.byref(E), _p(G), _p(A))
        return bool(ok), E.value, G, A

    def pcg(self, A, b, tol=1e-12, max_it=100000):
        A, b = _f64(A), _f64(b)
        x = np.zeros_like(b)
        it = lib().orc_pcg_solve(self.h, _p(A), _p(b), _p(x), tol, max_it)
        return x, it
