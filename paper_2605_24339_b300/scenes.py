"""Seeded synthetic workloads for the GMCP contact pass.

This module only builds meshes, seeds and motion scripts.  It contains none of
the contact method's arithmetic (no samples, gaps, barriers, CCD or elasticity),
so that the CPU oracle and the CUDA library can both be fed from it without
sharing any part of the method.

Workloads (all lengths in metres):

* ``tactile_indent``     -- one tetrahedral gel pad (structured slab, 6 tets
  per hex) whose bottom face is the slave (tactile) surface, above a rigid
  icosphere.  Default sizes: 32x32 quads, 16 mm side, 2 mm thick in 4 layers
  (5,445 vertices, 24,576 tets, 2,048 slave triangles), icosphere subdivision
  3 (642 vertices, 1,280 triangles) of radius 5 mm whose apex sits 2*dhat
  below the pad; vertex jitter N(0, 1e-5 m).
* ``gel_on_terrain``     -- a 256x256-quad gel pad (0.1 mm quads, 2 mm thick,
  8 layers: 594,441 vertices, 3,145,728 tets, 131,072 slave triangles) above
  a 316x316-quad height field (199,712 triangles, 20x20 mm) whose height is
  0.5 mm * Perlin(x/2mm, y/2mm).
* ``fingertip_batch``    -- many independent environments, each with several
  square pads of random size around a perturbed convex sphere.

The master (opposing) mesh is kinematic in every workload; the pad's top face
is Dirichlet and carries the scripted press/shear velocity.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

__all__ = [
    "Scene", "splitmix64_stream", "pad_slab", "icosphere", "perlin2",
    "height_field", "tactile_indent", "gel_on_terrain", "gel_dense", "fingertip_batch",
    "drape_on_master", "concat_envs", "patch_test", "top_face_tris",
]

_MASK64 = (1 << 64) - 1


def splitmix64_stream(seed: int, n: int) -> np.ndarray:
    """n outputs of Steele/Lea/Flood's SplitMix64 generator started at ``seed``."""
    out = np.empty(n, dtype=np.uint64)
    s = seed & _MASK64
    for i in range(n):
        s = (s + 0x9E3779B97F4A7C15) & _MASK64
        z = s
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        out[i] = z ^ (z >> 31)
    return out


# ---------------------------------------------------------------------------
# meshes
# ---------------------------------------------------------------------------

# Kuhn (Freudenthal) split of the unit cube into 6 tets along (0,0,0)-(1,1,1):
# one tet per axis permutation; it is conforming between neighbouring cubes.
_PERMS = [(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)]


def pad_slab(nx: int, ny: int, nz: int, dx: float, dz: float,
             origin=(0.0, 0.0, 0.0), with_tets: bool = True):
    """Structured tetrahedral slab.

    Returns ``(X, tets, bottom_tris, top_mask)``: rest positions ``[nv,3]``
    float64, tets ``[nt,4]`` int32 with positive volume, the bottom-face
    triangles ``[2*nx*ny,3]`` int32 oriented so that ``(x1-x0)x(x2-x0)``
    points to -z (out of the slab), and a bool mask of the top-face vertices.
    Vertex (i,j,k) has index ``i + (nx+1)*(j + (ny+1)*k)``; k=0 is the bottom.
    ``with_tets=False`` returns an empty tet array (surface-only workloads).
    """
    ox, oy, oz = origin
    i = np.arange(nx + 1)
    j = np.arange(ny + 1)
    k = np.arange(nz + 1)
    K, J, I = np.meshgrid(k, j, i, indexing="ij")
    X = np.stack([ox + I * dx, oy + J * dx, oz + K * dz], axis=-1).reshape(-1, 3)
    X = X.astype(np.float64)

    def vid(ii, jj, kk):
        return ii + (nx + 1) * (jj + (ny + 1) * kk)

    ci, cj, ck = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()
    tets = [np.zeros((0, 4), dtype=np.int64)]
    for p in (_PERMS if with_tets else []):
        off = np.zeros((4, 3), dtype=np.int64)
        for s in range(1, 4):
            off[s] = off[s - 1]
            off[s, p[s - 1]] += 1
        vs = [vid(ci + off[s, 0], cj + off[s, 1], ck + off[s, 2]) for s in range(4)]
        t = np.stack(vs, axis=1)
        # parity of the permutation decides the orientation
        inv = sum(1 for a in range(3) for b in range(a + 1, 3) if p[a] > p[b])
        if inv % 2 == 1:
            t = t[:, [0, 2, 1, 3]]
        tets.append(t)
    tets = np.concatenate(tets, axis=0).astype(np.int32)

    qi, qj = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    qi, qj = qi.ravel(), qj.ravel()
    v00, v10 = vid(qi, qj, 0), vid(qi + 1, qj, 0)
    v01, v11 = vid(qi, qj + 1, 0), vid(qi + 1, qj + 1, 0)
    # faces of the Kuhn tets on z=0: (00,10,11) and (00,01,11); orient to -z
    t1 = np.stack([v00, v11, v10], axis=1)
    t2 = np.stack([v00, v01, v11], axis=1)
    bottom = np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)
    top = np.zeros(X.shape[0], dtype=bool)
    top[vid(*np.meshgrid(i, j, indexing="ij"), nz).ravel()] = True
    return X, tets, bottom, top


def icosphere(subdiv: int, radius: float, center=(0.0, 0.0, 0.0)):
    """Subdivided icosahedron projected to a sphere; outward triangles."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
             (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in verts]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
             (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
             (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
             (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    for _ in range(subdiv):
        cache = {}
        new_faces = []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = verts[a] + verts[b]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = new_faces
    V = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    F = np.array(faces, dtype=np.int32)
    # make every face outward (the icosahedron list above is already CCW-out,
    # but enforce it against the centre to be safe)
    c = np.asarray(center, dtype=np.float64)
    n = np.cross(V[F[:, 1]] - V[F[:, 0]], V[F[:, 2]] - V[F[:, 0]])
    flip = np.einsum("ij,ij->i", n, V[F].mean(axis=1) - c) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    return V, F


def _perm_table(seed: int) -> np.ndarray:
    """256-entry permutation, Fisher-Yates shuffled by SplitMix64(seed)."""
    r = splitmix64_stream(seed, 256)
    p = np.arange(256, dtype=np.int64)
    for i in range(255, 0, -1):
        jj = int(r[i] % np.uint64(i + 1))
        p[i], p[jj] = p[jj], p[i]
    return np.concatenate([p, p])


def perlin2(x: np.ndarray, y: np.ndarray, perm: np.ndarray) -> np.ndarray:
    """2-D gradient noise after Perlin's 2002 'improved noise': lattice hash via
    the permutation table, 8 unit-ish gradients, quintic fade 6t^5-15t^4+10t^3."""
    xi = np.floor(x).astype(np.int64)
    yi = np.floor(y).astype(np.int64)
    xf, yf = x - xi, y - yi
    xi &= 255
    yi &= 255

    def fade(t):
        return t * t * t * (t * (t * 6 - 15) + 10)

    gx = np.array([1, -1, 1, -1, 1, -1, 0, 0], dtype=np.float64)
    gy = np.array([1, 1, -1, -1, 0, 0, 1, -1], dtype=np.float64)

    def grad(h, dx_, dy_):
        h = h & 7
        return gx[h] * dx_ + gy[h] * dy_
    aa = perm[perm[xi] + yi]
    ab = perm[perm[xi] + yi + 1]
    ba = perm[perm[xi + 1] + yi]
    bb = perm[perm[xi + 1] + yi + 1]
    u, v = fade(xf), fade(yf)
    n00 = grad(aa, xf, yf)
    n10 = grad(ba, xf - 1, yf)
    n01 = grad(ab, xf, yf - 1)
    n11 = grad(bb, xf - 1, yf - 1)
    nx0 = n00 + u * (n10 - n00)
    nx1 = n01 + u * (n11 - n01)
    return nx0 + v * (nx1 - nx0)


def height_field(nq: int, size: float, amp: float, wavelength: float, seed: int,
                 center=(0.0, 0.0)):
    """Open terrain surface z = amp*perlin(x/wl, y/wl) over a square of side
    ``size`` with ``nq`` quads per side; triangles face +z."""
    perm = _perm_table(seed)
    s = np.linspace(-size / 2, size / 2, nq + 1)
    Yg, Xg = np.meshgrid(s + center[1], s + center[0], indexing="ij")
    Z = amp * perlin2(Xg / wavelength + 0.5, Yg / wavelength + 0.5, perm)
    V = np.stack([Xg, Yg, Z], axis=-1).reshape(-1, 3)
    qj, qi = np.meshgrid(np.arange(nq), np.arange(nq), indexing="ij")
    qi, qj = qi.ravel(), qj.ravel()

    def vid(ii, jj):
        return ii + (nq + 1) * jj
    v00, v10, v01, v11 = vid(qi, qj), vid(qi + 1, qj), vid(qi, qj + 1), vid(qi + 1, qj + 1)
    t1 = np.stack([v00, v10, v11], axis=1)    # +z
    t2 = np.stack([v00, v11, v01], axis=1)    # +z
    F = np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)
    return V.astype(np.float64), F


def _fib_hull_sphere(n_pts: int, radius: float, center, rng):
    """Fibonacci-sphere points joined by their convex hull, then a seeded radial
    perturbation of at most 2 %.  The hull is computed by scipy (qhull)."""
    from scipy.spatial import ConvexHull
    k = np.arange(n_pts) + 0.5
    phi = np.arccos(1 - 2 * k / n_pts)
    th = math.pi * (1 + 5 ** 0.5) * k
    P = np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)
    hull = ConvexHull(P)
    F = hull.simplices.astype(np.int32)
    n = np.cross(P[F[:, 1]] - P[F[:, 0]], P[F[:, 2]] - P[F[:, 0]])
    flip = np.einsum("ij,ij->i", n, P[F].mean(axis=1)) < 0
    F[flip] = F[flip][:, [0, 2, 1]]
    r = radius * (1.0 + 0.02 * (rng.random(n_pts) * 2 - 1))
    V = P * r[:, None] + np.asarray(center, dtype=np.float64)
    return V, F


# ---------------------------------------------------------------------------
# scene container
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Scene:
    """A batch of environments, concatenated.  Per-env CSR offsets index the
    concatenated arrays; all indices are global (already offset)."""
    X: np.ndarray            # [nv,3] pad rest positions
    tets: np.ndarray         # [nt,4] int32
    stris: np.ndarray        # [ns,3] int32 slave (tactile) triangles, outward
    dirichlet: np.ndarray    # [nv] uint8
    Y0: np.ndarray           # [nmv,3] master positions at t=0
    mtris: np.ndarray        # [nmt,3] int32 master triangles, outward
    env_vert_off: np.ndarray
    env_tet_off: np.ndarray
    env_stri_off: np.ndarray
    env_mvert_off: np.ndarray
    env_mtri_off: np.ndarray
    # scripted Dirichlet velocity per pad vertex and suggested parameters
    v_dirichlet: np.ndarray  # [nv,3]
    params: dict
    name: str = ""
    n_steps: int = 10
    # deformable master (joint step): tets over the master vertices and
    # their Dirichlet flags; None = a kinematic master
    mtets: Optional[np.ndarray] = None
    mdirichlet: Optional[np.ndarray] = None

    @property
    def n_env(self) -> int:
        return len(self.env_vert_off) - 1

    @property
    def nv(self) -> int:
        return self.X.shape[0]

    @property
    def ns(self) -> int:
        return self.stris.shape[0]


def _single_env(X, tets, stris, dirichlet, Y0, mtris, vdir, params, name, n_steps):
    z = lambda n: np.array([0, n], dtype=np.int64)
    return Scene(X=np.ascontiguousarray(X, dtype=np.float64),
                 tets=np.ascontiguousarray(tets, dtype=np.int32),
                 stris=np.ascontiguousarray(stris, dtype=np.int32),
                 dirichlet=np.ascontiguousarray(dirichlet, dtype=np.uint8),
                 Y0=np.ascontiguousarray(Y0, dtype=np.float64),
                 mtris=np.ascontiguousarray(mtris, dtype=np.int32),
                 env_vert_off=z(X.shape[0]), env_tet_off=z(tets.shape[0]),
                 env_stri_off=z(stris.shape[0]), env_mvert_off=z(Y0.shape[0]),
                 env_mtri_off=z(mtris.shape[0]),
                 v_dirichlet=np.ascontiguousarray(vdir, dtype=np.float64),
                 params=params, name=name, n_steps=n_steps)


def concat_envs(scenes: List[Scene], name: str = "batch") -> Scene:
    """Concatenate single- or multi-env scenes, offsetting indices."""
    Xs, Ts, Ss, Ds, Ys, Ms, Vd = [], [], [], [], [], [], []
    offs = {k: [0] for k in ("v", "t", "s", "mv", "mt")}
    for sc in scenes:
        for e in range(sc.n_env):
            v0, v1 = sc.env_vert_off[e], sc.env_vert_off[e + 1]
            t0, t1 = sc.env_tet_off[e], sc.env_tet_off[e + 1]
            s0, s1 = sc.env_stri_off[e], sc.env_stri_off[e + 1]
            m0, m1 = sc.env_mvert_off[e], sc.env_mvert_off[e + 1]
            q0, q1 = sc.env_mtri_off[e], sc.env_mtri_off[e + 1]
            Xs.append(sc.X[v0:v1]); Vd.append(sc.v_dirichlet[v0:v1])
            Ds.append(sc.dirichlet[v0:v1]); Ys.append(sc.Y0[m0:m1])
            Ts.append(sc.tets[t0:t1] - v0 + offs["v"][-1])
            Ss.append(sc.stris[s0:s1] - v0 + offs["v"][-1])
            Ms.append(sc.mtris[q0:q1] - m0 + offs["mv"][-1])
            offs["v"].append(offs["v"][-1] + (v1 - v0))
            offs["t"].append(offs["t"][-1] + (t1 - t0))
            offs["s"].append(offs["s"][-1] + (s1 - s0))
            offs["mv"].append(offs["mv"][-1] + (m1 - m0))
            offs["mt"].append(offs["mt"][-1] + (q1 - q0))
    a = lambda k: np.array(offs[k], dtype=np.int64)
    return Scene(X=np.concatenate(Xs), tets=np.concatenate(Ts).astype(np.int32),
                 stris=np.concatenate(Ss).astype(np.int32),
                 dirichlet=np.concatenate(Ds), Y0=np.concatenate(Ys),
                 mtris=np.concatenate(Ms).astype(np.int32),
                 env_vert_off=a("v"), env_tet_off=a("t"), env_stri_off=a("s"),
                 env_mvert_off=a("mv"), env_mtri_off=a("mt"),
                 v_dirichlet=np.concatenate(Vd), params=dict(scenes[0].params),
                 name=name, n_steps=scenes[0].n_steps)


def default_params(**kw) -> dict:
    """Physical and solver parameters shared by the workloads (SI units).
    kappa_edge / kappa_point default to kappa*lbar and kappa*lbar^2 (lbar =
    mean slave edge length at rest) and are filled in by the workload."""
    p = dict(dhat=1e-4, kappa=1e5, kappa_edge=None, kappa_point=None,
             delta_T=0.1, delta_e=0.1, face_rule_level=1, h=1e-3,
             density=1100.0, youngs=3e5, poisson=0.45, gravity=(0.0, 0.0, 0.0),
             newton_tol=1e-6, pcg_rel_tol=1e-3, max_newton=50, max_pcg=2000,
             max_halvings=40, ccd_slack=0.1, ccd_max_iter=100000,
             dhat_guard=None, kappa_guard=None)
    p.update(kw)
    return p


def _mean_edge_len(X, F):
    e = np.concatenate([X[F[:, 1]] - X[F[:, 0]], X[F[:, 2]] - X[F[:, 1]],
                        X[F[:, 0]] - X[F[:, 2]]])
    return float(np.linalg.norm(e, axis=1).mean())


def _finish_params(p, X, S):
    lbar = _mean_edge_len(X, S)
    if p.get("kappa_edge") is None:
        p["kappa_edge"] = p["kappa"] * lbar
    if p.get("kappa_point") is None:
        p["kappa_point"] = p["kappa"] * lbar * lbar
    if p.get("dhat_guard") is None:
        p["dhat_guard"] = 0.1 * p["dhat"]
    if p.get("kappa_guard") is None:
        p["kappa_guard"] = 0.0          # primitive guard barrier off by default
    return p


def top_face_tris(nx: int, ny: int, nz: int):
    """Top-face triangles of ``pad_slab(nx, ny, nz, ...)``, oriented so that
    (x1-x0)x(x2-x0) points to +z (out of the slab)."""
    def vid(ii, jj):
        return ii + (nx + 1) * (jj + (ny + 1) * nz)
    F = []
    for i in range(nx):
        for j in range(ny):
            a, b, c, d = vid(i, j), vid(i + 1, j), vid(i + 1, j + 1), vid(i, j + 1)
            F.append((a, b, c))
            F.append((a, c, d))
    return np.asarray(F, dtype=np.int32)


def patch_test(slave_n=(5, 5, 2), master_n=(4, 4, 2), gap=0.002, dhat=1e-3, kappa=1e4, youngs=1000.0,
               poisson=0.0, pressure=10.0, h=1.0, density=1.0, face_rule_level=1, shift=(0.0, 0.0),
               pcg_rel_tol=1e-9):
    """Contact patch test (Sec. 5.1, "Contact patch test"): two elastic blocks
    of 1 x 1 x 0.5, the upper one ``gap`` above the lower one, with
    non-matching structured tet meshes (``slave_n`` and ``master_n`` cells
    along x, y, z).  The upper block is the pad: its bottom face is the slave
    (tactile) surface.  The lower block is a deformable master: its top face
    gives the master triangles, its bottom face is held (Dirichlet).  A
    uniform pressure on the upper block's top face is applied as nodal forces
    (each top triangle's force split evenly over its vertices).  With Poisson
    ratio 0 the exact static state is a uniform stress sigma_zz = -pressure in
    both blocks.  Returns (scene, f_ext) with f_ext [n_pad + n_master, 3];
    ``scene.mtets`` / ``scene.mdirichlet`` describe the master body.
    The upper block is held sideways by its inertia alone, and at kappa =
    1e8 the barrier is ~1e8 times stiffer than that mode: a linear solve to
    a relative residual of 1e-3 (or 1e-6) leaves an error along the free
    mode that the barrier turns back into residual, and Newton stalls near
    5e-5.  Hence the PCG tolerance of 1e-9 (every step of kappa 1e4, 1e6 and
    1e8 then converges to the 1e-6 residual)."""
    sx, sy, sz = slave_n
    mx, my, mz = master_n
    Xm, Tm, _, _ = pad_slab(mx, my, mz, 1.0 / mx, 0.5 / mz, origin=(shift[0], shift[1], 0.0))
    Fm = top_face_tris(mx, my, mz)
    Xs, Ts, Bs, top_s = pad_slab(sx, sy, sz, 1.0 / sx, 0.5 / sz, origin=(0.0, 0.0, 0.5 + gap))
    mdir = (np.abs(Xm[:, 2]) < 1e-12).astype(np.uint8)
    p = default_params(dhat=dhat, kappa=kappa, h=h, density=density, youngs=youngs, poisson=poisson,
                       face_rule_level=face_rule_level, gravity=(0.0, 0.0, 0.0), pcg_rel_tol=pcg_rel_tol)
    p = _finish_params(p, Xs, Bs)
    sc = _single_env(Xs, Ts, Bs, np.zeros(Xs.shape[0], dtype=np.uint8), Xm, Fm, np.zeros_like(Xs), p,
                     "patch_test", 3)
    sc.mtets = np.ascontiguousarray(Tm, dtype=np.int32)
    sc.mdirichlet = mdir
    f = np.zeros((Xs.shape[0] + Xm.shape[0], 3))
    Ft = top_face_tris(sx, sy, sz)
    for tri in Ft:
        P = Xs[tri]
        area = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
        f[tri, 2] -= pressure * area / 3.0
    return sc, f


def tactile_indent(n_quads=32, side=16e-3, nz=4, thick=2e-3, sphere_subdiv=3,
                   radius=5e-3, dhat=1e-4, kappa=1e5, h=1e-3, press=0.3e-3,
                   n_steps=10, jitter=1e-5, seed=1, face_rule_level=1) -> Scene:
    """Soft pad pressed onto a rigid icosphere (single env)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    dx = side / n_quads
    X, tets, bot, top = pad_slab(n_quads, n_quads, nz, dx, thick / nz,
                                 origin=(-side / 2, -side / 2, 0.0))
    Y, F = icosphere(sphere_subdiv, radius, center=(0.0, 0.0, -2 * dhat - radius))
    X = X + rng.normal(0.0, jitter, X.shape)
    Y = Y + rng.normal(0.0, jitter, Y.shape)
    vdir = np.zeros_like(X)
    vdir[top, 2] = -(press + 2 * dhat) / (n_steps * h)
    p = _finish_params(default_params(dhat=dhat, kappa=kappa, h=h,
                                      face_rule_level=face_rule_level), X, bot)
    return _single_env(X, tets, bot, top.astype(np.uint8), Y, F, vdir, p,
                       "tactile_indent", n_steps)


def gel_on_terrain(n_quads=256, dx=1e-4, nz=8, thick=2e-3, terrain_quads=316,
                   terrain_size=20e-3, amp=0.5e-3, wavelength=2e-3, dhat=5e-5,
                   kappa=1e5, h=1e-2, press_speed=0.5e-3, n_steps=50, seed=2,
                   face_rule_level=2) -> Scene:
    """Large gel pad above a Perlin height field (single env).  The pad starts
    2*dhat above the highest terrain vertex; its top face is pressed at
    ``press_speed`` (the first 60 % of the steps) then sheared along +x."""
    side = n_quads * dx
    Y, F = height_field(terrain_quads, terrain_size, amp, wavelength, seed)
    z0 = float(Y[:, 2].max()) + 2 * dhat
    X, tets, bot, top = pad_slab(n_quads, n_quads, nz, dx, thick / nz,
                                 origin=(-side / 2, -side / 2, z0))
    vdir = np.zeros_like(X)
    vdir[top, 2] = -press_speed
    p = _finish_params(default_params(dhat=dhat, kappa=kappa, h=h,
                                      face_rule_level=face_rule_level), X, bot)
    p["shear_after_step"] = int(0.6 * n_steps)
    p["shear_velocity"] = (press_speed, 0.0, 0.0)
    return _single_env(X, tets, bot, top.astype(np.uint8), Y, F, vdir, p,
                       "gel_on_terrain", n_steps)


def gel_dense(n_quads=256, dx=1e-4, nz=8, thick=2e-3, plate_quads=442, plate_size=28e-3,
              amp=0.1e-3, wavelength=2e-3, dhat=5e-5, seed=3, face_rule_level=2, with_tets=True):
    """Contact-dense variant of gel_on_terrain: the same 256x256-quad gel pad
    (131,072 slave triangles x 16 face samples) over a larger, lower Perlin
    plate (442x442 quads over 28x28 mm, 390,728 triangles, amplitude 0.1 mm,
    wavelength 2 mm), so that the pad can be pressed onto it everywhere.
    Returns (scene, x) with x the pad draped fully onto the plate
    (drape_on_master with a depth beyond the plate's relief): every slave
    vertex sits 0.3-0.9 dhat above the plate, so nearly every face sample is
    active."""
    side = n_quads * dx
    Y, F = height_field(plate_quads, plate_size, amp, wavelength, seed)
    z0 = float(Y[:, 2].max()) + 2 * dhat
    X, tets, bot, top = pad_slab(n_quads, n_quads, nz, dx, thick / nz,
                                 origin=(-side / 2, -side / 2, z0), with_tets=with_tets)
    vdir = np.zeros_like(X)
    vdir[top, 2] = -0.5e-3
    p = _finish_params(default_params(dhat=dhat, face_rule_level=face_rule_level, h=1e-2), X, bot)
    sc = _single_env(X, tets, bot, top.astype(np.uint8), Y, F, vdir, p, "gel_dense", 50)
    depth = float(Y[:, 2].max() - Y[:, 2].min()) + 4 * dhat
    return sc, drape_on_master(sc, depth)


def _fingertip_env(e, pads_per_env, quad_range, dx, nz, thick, tri_range, radius, dhat, kappa, h,
                   press_speed, n_steps, seed, face_rule_level, pressed, with_tets):
    """Environment e of fingertip_batch (a function of its arguments only, so
    that environments can be built in worker processes); with ``pressed``
    also the pad positions moved that far toward the object."""
    rng = np.random.Generator(np.random.PCG64(seed + e))
    T = int(rng.integers(tri_range[0], tri_range[1] + 1))
    Y, F = _fib_hull_sphere(T // 2 + 2, radius, (0.0, 0.0, 0.0), rng)
    rmax = float(np.linalg.norm(Y, axis=1).max())
    Xs, Ts, Ss, Ds, Vd, Xq = [], [], [], [], [], []
    nvo = 0
    dirs = _pad_dirs(pads_per_env)
    for k in range(pads_per_env):
        nq = int(rng.integers(quad_range[0], quad_range[1] + 1))
        side = nq * dx
        Xp, tp, bp, topm = pad_slab(nq, nq, nz, dx, thick / nz,
                                    origin=(-side / 2, -side / 2, 0.0), with_tets=with_tets)
        # rotate the pad so its bottom normal (-z) points at the centre
        R = _frame_from_dir(dirs[k])
        Xr = Xp @ R.T
        Xp = Xr + dirs[k] * (rmax + 2 * dhat)
        if pressed is not None:
            Xq.append(Xr + dirs[k] * (rmax + 2 * dhat) - dirs[k] * pressed)
        vd = np.zeros_like(Xp)
        vd[topm] = -dirs[k] * press_speed
        Xs.append(Xp); Ts.append(tp + nvo); Ss.append(bp + nvo)
        Ds.append(topm.astype(np.uint8)); Vd.append(vd)
        nvo += Xp.shape[0]
    X = np.concatenate(Xs)
    S = np.concatenate(Ss)
    p = _finish_params(default_params(dhat=dhat, kappa=kappa, h=h,
                                      face_rule_level=face_rule_level), X, S)
    sc = _single_env(X, np.concatenate(Ts), S, np.concatenate(Ds), Y, F,
                     np.concatenate(Vd), p, f"env{e}", n_steps)
    return sc if pressed is None else (sc, np.concatenate(Xq))


def fingertip_batch(n_env=512, pads_per_env=5, quad_range=(16, 128), dx=0.25e-3,
                    nz=2, thick=0.5e-3, tri_range=(2000, 80000), radius=15e-3,
                    dhat=1e-4, kappa=1e5, h=1e-3, press_speed=0.5e-3,
                    n_steps=100, seed=3, face_rule_level=1, pressed=None,
                    with_tets=True, workers=1):
    """Many independent envs: each has ``pads_per_env`` square pads of side
    U{quad_range} quads facing the centre of a perturbed convex sphere with
    U[tri_range] triangles, 2*dhat away from the sphere's largest radius.
    With ``pressed`` (a distance) returns ``(scene, x)``, x the pads moved
    that far toward their objects (what press_pads gives, without needing
    the tets).  ``workers > 1`` builds the envs in that many worker processes
    (started with spawn); the result does not depend on it."""
    args = (pads_per_env, quad_range, dx, nz, thick, tri_range, radius, dhat, kappa, h,
            press_speed, n_steps, seed, face_rule_level, pressed, with_tets)
    if workers > 1 and n_env > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn")) as ex:
            out = list(ex.map(_fingertip_env, range(n_env), *[[a] * n_env for a in args],
                              chunksize=max(1, n_env // (4 * workers))))
    else:
        out = [_fingertip_env(e, *args) for e in range(n_env)]
    if pressed is None:
        return concat_envs(out, name="fingertip_batch")
    return concat_envs([o[0] for o in out], name="fingertip_batch"), np.concatenate([o[1] for o in out])


def thin_shell(nq: int, side: float, thickness: float):
    """Closed thin plate: the surface of a box of side x side x thickness
    with nq x nq quads on the two large faces and nq x 1 quads on each rim,
    triangulated with outward normals.  Returns (Y [n,3], F [m,3] int32)."""
    i = np.arange(nq + 1)
    I, J = np.meshgrid(i, i, indexing="ij")
    a = side / 2
    Y = []
    for k, z in enumerate((-thickness / 2, thickness / 2)):
        Y.append(np.stack([-a + I.ravel() * side / nq, -a + J.ravel() * side / nq,
                           np.full(I.size, z)], axis=1))
    Y = np.concatenate(Y).astype(np.float64)
    vid = lambda ii, jj, kk: ii + (nq + 1) * (jj + (nq + 1) * kk)
    quads = []
    for kk in (0, 1):                                   # large faces
        for ii in range(nq):
            for jj in range(nq):
                quads.append((vid(ii, jj, kk), vid(ii + 1, jj, kk), vid(ii + 1, jj + 1, kk), vid(ii, jj + 1, kk)))
    for ii in range(nq):                                # rims y = -a, y = +a
        for jj in (0, nq):
            quads.append((vid(ii, jj, 0), vid(ii + 1, jj, 0), vid(ii + 1, jj, 1), vid(ii, jj, 1)))
    for jj in range(nq):                                # rims x = -a, x = +a
        for ii in (0, nq):
            quads.append((vid(ii, jj, 0), vid(ii, jj + 1, 0), vid(ii, jj + 1, 1), vid(ii, jj, 1)))
    F = []
    for q in quads:
        for tri in ((q[0], q[1], q[2]), (q[0], q[2], q[3])):
            p0, p1, p2 = Y[list(tri)]
            n = np.cross(p1 - p0, p2 - p0)
            c = (p0 + p1 + p2) / 3
            F.append(tri if np.dot(n, c) > 0 else (tri[0], tri[2], tri[1]))   # outward (box centred at 0)
    return Y, np.asarray(F, dtype=np.int32)


def ccd_stress(n_env=64, pad_quads=128, pad_dx=0.25e-3, pad_nz=4, shell_quads=100, shell_side=30e-3,
               shell_thickness=1e-3, gap=1e-3, speed=(0.5, 2.0), dhat=1e-4, kappa=1e5, h=1e-3,
               seed=4, face_rule_level=1):
    """CCD / line-search stress: per env, a free pad (no Dirichlet vertices)
    moving at U[speed] m/s toward a closed thin shell from ``gap`` away, the
    whole env at a seeded random rotation.  At 2 m/s and h = 1 ms a step moves
    the pad 2 mm, more than the shell is thick.  Returns (scene, v0)."""
    envs, vs = [], []
    Ys, Fs = thin_shell(shell_quads, shell_side, shell_thickness)
    for e in range(n_env):
        rng = np.random.Generator(np.random.PCG64(seed * 1000 + e))
        side = pad_quads * pad_dx
        X, tets, bot, _ = pad_slab(pad_quads, pad_quads, pad_nz, pad_dx, pad_dx,
                                   origin=(-side / 2, -side / 2, shell_thickness / 2 + gap))
        q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        if np.linalg.det(q) < 0:
            q[:, 0] = -q[:, 0]
        spd = rng.uniform(speed[0], speed[1])
        v = np.zeros_like(X)
        v[:, 2] = -spd
        p = _finish_params(default_params(dhat=dhat, kappa=kappa, h=h, face_rule_level=face_rule_level),
                           X, bot)
        envs.append(_single_env(X @ q.T, tets, bot, np.zeros(X.shape[0], dtype=np.uint8), Ys @ q.T, Fs,
                                np.zeros_like(X), p, f"env{e}", 10))
        vs.append(v @ q.T)
    return concat_envs(envs, name="ccd_stress"), np.concatenate(vs)


def _pad_dirs(n):
    """n unit directions spread over the sphere (outward from the object)."""
    base = [np.array(v, dtype=np.float64) for v in
            [(0, 0, 1), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, -1)]]
    out = []
    for i in range(n):
        d = base[i % 6] + 0.05 * (i // 6)
        out.append(d / np.linalg.norm(d))
    return out


def _frame_from_dir(d):
    """Rotation R with R @ (0,0,1) = d (so the pad's -z bottom faces -d)."""
    z = np.asarray(d, dtype=np.float64)
    a = np.array([1.0, 0.0, 0.0]) if abs(z[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    x = np.cross(a, z); x /= np.linalg.norm(x)
    y = np.cross(z, x)
    return np.stack([x, y, z], axis=1)


def press_pads(scene: Scene, depth: float) -> np.ndarray:
    """A pressed state of a batch of pads: every pad (a connected component of
    the tet mesh) is translated rigidly by ``depth`` along the unit direction
    of its Dirichlet (top) vertices' scripted velocity.  Returns x [nv,3]."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    nv = scene.X.shape[0]
    T = scene.tets
    rows = np.concatenate([T[:, 0], T[:, 0], T[:, 0]])
    cols = np.concatenate([T[:, 1], T[:, 2], T[:, 3]])
    g = coo_matrix((np.ones(rows.shape[0], dtype=np.int8), (rows, cols)), shape=(nv, nv))
    ncomp, lab = connected_components(g, directed=False)
    top = scene.dirichlet.astype(bool)
    vd = scene.v_dirichlet
    nrm = np.linalg.norm(vd, axis=1)
    u = np.zeros((ncomp, 3))
    sel = top & (nrm > 0)
    np.add.at(u, lab[sel], vd[sel] / nrm[sel, None])
    un = np.linalg.norm(u, axis=1)
    u[un > 0] /= un[un > 0, None]
    return scene.X + depth * u[lab]


def drape_on_master(scene: Scene, depth: float, gap_lo: float = 0.3,
                    gap_hi: float = 0.9, seed: int = 7) -> np.ndarray:
    """A pressed, intersection-free pad state for a single-env scene whose
    pad bottom faces -z (terrain or sphere below).

    Each slave-surface vertex is placed at ``max(z - depth, h(x,y) + gap)``:
    ``z`` its rest height, ``h`` the master surface height under it (vertical
    ray cast onto the master triangles) and ``gap ~ dhat*U[gap_lo, gap_hi]``
    drawn per vertex.  Every other pad vertex takes the vertical displacement
    of its nearest surface vertex in xy, blended linearly with height toward
    the top face, which moves down by ``depth``.  Returns x ``[nv,3]``."""
    from scipy.spatial import cKDTree
    rng = np.random.Generator(np.random.PCG64(seed))
    X = scene.X
    dhat = scene.params["dhat"]
    bottom = np.unique(scene.stris)
    zb, ztop = X[bottom, 2].mean(), X[:, 2].max()
    hgt = _surface_height(scene.Y0, scene.mtris, X[bottom, :2])
    gap = dhat * rng.uniform(gap_lo, gap_hi, bottom.shape[0])
    zr = X[bottom, 2]
    target = np.where(np.isfinite(hgt), np.maximum(zr - depth, hgt + gap), zr - depth)
    dz_b = target - zr
    _, nn = cKDTree(X[bottom, :2]).query(X[:, :2])
    s = np.clip((X[:, 2] - zb) / (ztop - zb), 0.0, 1.0)
    x = X.copy()
    x[:, 2] += (1 - s) * dz_b[nn] + s * (-depth)
    x[bottom, 2] = zr + dz_b
    return x


def _surface_height(Y, F, P):
    """Largest z of the master surface on the vertical line through each xy
    point of P (NaN where the line misses every triangle)."""
    tri = Y[F]
    lo = tri[:, :, :2].min(axis=1)
    hi = tri[:, :, :2].max(axis=1)
    cell = max(float(np.median(hi - lo)) * 2.0, 1e-9)
    g0 = np.minimum(P.min(axis=0), lo.min(axis=0)) - cell
    nby = int(np.floor((max(P[:, 1].max(), hi[:, 1].max()) - g0[1]) / cell)) + 2
    c0 = np.floor((lo - g0) / cell).astype(np.int64)
    c1 = np.floor((hi - g0) / cell).astype(np.int64)
    # expand each triangle over the buckets its xy box covers
    nxs = c1[:, 0] - c0[:, 0] + 1
    nys = c1[:, 1] - c0[:, 1] + 1
    cnt = nxs * nys
    tid = np.repeat(np.arange(F.shape[0]), cnt)
    loc = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
    bx = c0[tid, 0] + loc // nys[tid]
    by = c0[tid, 1] + loc % nys[tid]
    tkey = bx * nby + by
    order = np.argsort(tkey, kind="stable")
    tkey, tid = tkey[order], tid[order]
    pc = np.floor((P - g0) / cell).astype(np.int64)
    pkey = pc[:, 0] * nby + pc[:, 1]
    a = np.searchsorted(tkey, pkey, side="left")
    b = np.searchsorted(tkey, pkey, side="right")
    n = b - a
    pid = np.repeat(np.arange(P.shape[0]), n)
    t = tid[np.repeat(a, n) + (np.arange(n.sum()) - np.repeat(np.cumsum(n) - n, n))]
    A, B, C = tri[t, 0], tri[t, 1], tri[t, 2]
    v0, v1 = B[:, :2] - A[:, :2], C[:, :2] - A[:, :2]
    den = v0[:, 0] * v1[:, 1] - v0[:, 1] * v1[:, 0]
    d = P[pid] - A[:, :2]
    ok = np.abs(den) > 1e-300
    den = np.where(ok, den, 1.0)
    u = (d[:, 0] * v1[:, 1] - d[:, 1] * v1[:, 0]) / den
    v = (v0[:, 0] * d[:, 1] - v0[:, 1] * d[:, 0]) / den
    inside = ok & (u >= -1e-12) & (v >= -1e-12) & (u + v <= 1 + 1e-12)
    z = A[:, 2] + u * (B[:, 2] - A[:, 2]) + v * (C[:, 2] - A[:, 2])
    out = np.full(P.shape[0], -np.inf)
    np.maximum.at(out, pid[inside], z[inside])
    out[~np.isfinite(out)] = np.nan
    return out


def crop(scene: Scene, x: np.ndarray, center, half_width: float, margin: float):
    """Contact-only sub-scene of a single-env scene: the slave triangles whose
    centroid (at x) lies in the xy square ``center +- half_width``, their
    vertices, and the master triangles whose xy box meets the square grown by
    ``margin``.  Tets are dropped (the sub-scene serves the contact pass
    only).  Returns ``(sub_scene, x_sub)``."""
    cx, cy = center
    cen = x[scene.stris].mean(axis=1)
    sel = (np.abs(cen[:, 0] - cx) <= half_width) & (np.abs(cen[:, 1] - cy) <= half_width)
    S = scene.stris[sel]
    verts, inv = np.unique(S, return_inverse=True)
    S2 = inv.reshape(-1, 3).astype(np.int32)
    tri = scene.Y0[scene.mtris]
    lo, hi = tri[:, :, :2].min(axis=1), tri[:, :, :2].max(axis=1)
    w = half_width + margin
    msel = (hi[:, 0] >= cx - w) & (lo[:, 0] <= cx + w) & (hi[:, 1] >= cy - w) & (lo[:, 1] <= cy + w)
    M = scene.mtris[msel]
    mverts, minv = np.unique(M, return_inverse=True)
    M2 = minv.reshape(-1, 3).astype(np.int32)
    X2 = scene.X[verts]
    sub = _single_env(X2, np.zeros((0, 4), dtype=np.int32), S2,
                      scene.dirichlet[verts], scene.Y0[mverts], M2, scene.v_dirichlet[verts],
                      dict(scene.params), scene.name + "_crop", scene.n_steps)
    return sub, x[verts].copy()
