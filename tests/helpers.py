"""Small synthetic scenes used by the tests (geometry only)."""
import numpy as np

from paper_2605_24339_b300 import scenes as S


def flat_over_big_triangle(nq=2, dx=1e-3, gap=3e-5, dhat=1e-4, rest_gap=1e-3,
                           kappa=1e5, face_only=True, L=1):
    """A flat pad (bottom at z=0, normal -z) over one large master triangle
    facing +z.  The master sits ``rest_gap`` below at t=0 (Y0) and ``gap``
    below in the returned current configuration xm."""
    X, tets, bot, top = S.pad_slab(nq, nq, 1, dx, dx, origin=(0.0, 0.0, 0.0))
    side = nq * dx
    c = side / 2
    R = 40 * side
    Y0 = np.array([[c - R, c - R, -rest_gap], [c + 2 * R, c - R, -rest_gap],
                   [c - R, c + 2 * R, -rest_gap]])
    F = np.array([[0, 1, 2]], dtype=np.int32)
    p = S.default_params(dhat=dhat, kappa=kappa, face_rule_level=L)
    if face_only:
        p["kappa_edge"] = 0.0
        p["kappa_point"] = 0.0
    p = S._finish_params(p, X, bot)
    sc = S._single_env(X, tets, bot, top.astype(np.uint8), Y0, F, np.zeros_like(X), p,
                       "flat", 1)
    xm = Y0.copy()
    xm[:, 2] = -gap
    return sc, X.copy(), xm


def small_indent(n_quads=8, subdiv=2, press=0.15e-3, seed=1, L=1, dhat=1e-4):
    """Reduced tactile_indent scene plus a draped (pressed) pad state."""
    sc = S.tactile_indent(n_quads=n_quads, side=n_quads * 0.5e-3, nz=2, thick=1e-3,
                          sphere_subdiv=subdiv, radius=2e-3, seed=seed,
                          face_rule_level=L, dhat=dhat)
    x = S.drape_on_master(sc, press, seed=seed + 10)
    return sc, x


def flat_press(nq=4, n_steps=4, pcg_rel_tol=1e-6):
    """Pad (nq x nq x 2 hexes of 0.5 mm, tetrahedralised) whose top face is
    driven down 0.3 mm over ``n_steps`` steps onto one large flat master
    triangle 0.2 mm below (Dirichlet velocity in ``sc.v_dirichlet``)."""
    sc, _, _ = flat_over_big_triangle(nq=nq, dx=0.5e-3, gap=2e-4, rest_gap=2e-4,
                                      face_only=False)
    X, tets, stris, top = S.pad_slab(nq, nq, 2, 0.5e-3, 0.5e-3)
    sc.X, sc.tets, sc.stris = X, tets, stris
    sc.dirichlet = top.astype(np.uint8)
    sc.env_vert_off = np.array([0, sc.X.shape[0]])
    sc.env_tet_off = np.array([0, sc.tets.shape[0]])
    sc.env_stri_off = np.array([0, sc.stris.shape[0]])
    sc.v_dirichlet = np.zeros_like(sc.X)
    sc.v_dirichlet[top, 2] = -3e-4 / (n_steps * sc.params["h"])
    sc.n_steps = n_steps
    sc.params.update(pcg_rel_tol=pcg_rel_tol)
    return sc


def rotation(seed):
    rng = np.random.default_rng(seed)
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def load_golden(name):
    rows = []
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(v) for v in line.split()])
    return np.array(rows)


MM = 1e-3


def one_slave_triangle(Y, F, gap_rest=1e-3, kappa=1e5, kappa_edge=1e2, kappa_point=1e-1,
                       dhat=1e-4, L=1):
    """One tet whose bottom face is the only slave triangle: S0=(0,0,0),
    S1=(0,1,0), S2=(1,0,0) mm, normal -z; a point (x, y) of it has
    beta^s = (1-x-y, y, x).  ``Y`` [n,3] (metres) is the current master, ``F``
    its outward triangles; at rest (Y0) the master sits ``gap_rest`` lower,
    so that 0.9 g_ref > dhat and every sample takes eps = dhat (Eq.
    adaptive_eps).  Returns (scene, x, xm)."""
    X = np.array([[0, 0, 0], [0, 1, 0], [1, 0, 0], [0, 0, 1]], dtype=np.float64) * MM
    tets = np.array([[0, 2, 1, 3]], dtype=np.int32)
    stris = np.array([[0, 1, 2]], dtype=np.int32)
    Y = np.asarray(Y, dtype=np.float64)
    Y0 = Y.copy()
    Y0[:, 2] -= gap_rest
    p = S.default_params(dhat=dhat, kappa=kappa, kappa_edge=kappa_edge, kappa_point=kappa_point,
                         face_rule_level=L)
    p = S._finish_params(p, X, stris)
    dirichlet = np.array([0, 0, 0, 1], dtype=np.uint8)
    sc = S._single_env(X, tets, stris, dirichlet, Y0, np.asarray(F, dtype=np.int32),
                       np.zeros_like(X), p, "one_slave_triangle", 1)
    return sc, X.copy(), Y


def outward_up(Y, F):
    """Orient each triangle of F so that its normal has a positive z part."""
    F = np.array(F, dtype=np.int32)
    for t in F:
        n = np.cross(Y[t[1]] - Y[t[0]], Y[t[2]] - Y[t[0]])
        if n[2] < 0:
            t[1], t[2] = t[2], t[1]
    return F


def spike_master(apex_xy, gap, radius=1.0, depth=10.0):
    """An upward spike: apex at (apex_xy, -gap), three base vertices
    ``radius`` mm away horizontally and ``depth`` mm lower; three faces."""
    ax, ay = apex_xy
    Y = [[ax * MM, ay * MM, -gap]]
    for th in (90.0, 210.0, 330.0):
        r = np.deg2rad(th)
        Y.append([(ax + radius * np.cos(r)) * MM, (ay + radius * np.sin(r)) * MM,
                  -gap - depth * MM])
    Y = np.array(Y)
    return Y, outward_up(Y, [[0, 1, 2], [0, 2, 3], [0, 3, 1]])


def edge_master(gap_a, gap_b):
    """One master triangle whose edge A-B runs along y = 0.25 mm from
    x = -0.01 mm to x = 9.99 mm (A at depth gap_a, B at gap_b); its third
    vertex C = (-0.01, 1.25) mm lies 10 mm below A, so the face rises steeply
    away from A-B and the edges A-C and B-C miss the slave triangle."""
    Y = np.array([[-0.01 * MM, 0.25 * MM, -gap_a], [9.99 * MM, 0.25 * MM, -gap_b],
                  [-0.01 * MM, 1.25 * MM, -gap_a - 10.0 * MM]])
    return Y, outward_up(Y, [[0, 1, 2]])


def face_master(gap):
    """One master triangle parallel to the slave at depth gap:
    M0=(0.18,-1), M1=(2.5,-1), M2=(0.18,2.5) mm."""
    Y = np.array([[0.18, -1.0, 0.0], [2.5, -1.0, 0.0], [0.18, 2.5, 0.0]]) * MM
    Y[:, 2] = -gap
    return Y, outward_up(Y, [[0, 1, 2]])


# -- comparisons of GPU results with the oracle's -------------------------------
def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    d = np.linalg.norm((a - b).ravel())
    n = np.linalg.norm(b.ravel())
    return d / n if n > 0 else d


def bsr_dict(rp, ci, vals):
    rp, ci, vals = rp.cpu().numpy(), ci.cpu().numpy(), vals.cpu().numpy().astype(np.float64)
    out = {}
    for i in range(rp.shape[0] - 1):
        for k in range(rp[i], rp[i + 1]):
            out[(i, int(ci[k]))] = vals[k]
    return out


def hess_rel(gpu_h, orc):
    G = bsr_dict(*gpu_h)
    O = {(int(i), int(j)): b for (i, j), b in zip(orc["blk_ij"], orc["blk"])}
    num = den = 0.0
    for k in set(G) | set(O):
        g = G.get(k, np.zeros((3, 3)))
        o = O.get(k, np.zeros((3, 3)))
        num += np.sum((g - o) ** 2)
        den += np.sum(o ** 2)
    return np.sqrt(num / den) if den > 0 else np.sqrt(num)


def hess_blocks_check(gpu_h, orc, tol, rows=None):
    """Every 3x3 block against the oracle's: ||G - O||_F <= tol ||O||_F, with a
    floor of tol * 1e-9 of the largest block for blocks the oracle does not
    have (the GPU pattern may hold zero blocks).  The contact blocks are sums
    of PSD terms, so no block is a cancelling sum.  rows: only blocks in these
    rows.  Returns the largest per-block relative error."""
    G = bsr_dict(*gpu_h)
    O = {(int(i), int(j)): b for (i, j), b in zip(orc["blk_ij"], orc["blk"])}
    if rows is not None:
        rs = set(int(r) for r in rows)
        G = {k: v for k, v in G.items() if k[0] in rs}
        O = {k: v for k, v in O.items() if k[0] in rs}
    big = max(np.linalg.norm(b) for b in O.values())
    worst = 0.0
    for k in set(G) | set(O):
        g = G.get(k, np.zeros((3, 3)))
        o = O.get(k, np.zeros((3, 3)))
        err = np.linalg.norm(g - o)
        ref = max(np.linalg.norm(o), 1e-9 * big)
        worst = max(worst, err / ref)
        assert err <= tol * ref, (k, err, np.linalg.norm(o))
    return worst


def cauchy_stress(X, T, x, youngs, poisson):
    """Cauchy stress of every tet [nt, 3, 3] for compressible Neo-Hookean
    (the material of the time step): P = mu (F - F^-T) + lam ln J F^-T,
    sigma = P F^T / J."""
    mu = youngs / (2 * (1 + poisson))
    lam = youngs * poisson / ((1 + poisson) * (1 - 2 * poisson))
    Dm = np.stack([X[T[:, k]] - X[T[:, 0]] for k in (1, 2, 3)], axis=2)
    Ds = np.stack([x[T[:, k]] - x[T[:, 0]] for k in (1, 2, 3)], axis=2)
    F = Ds @ np.linalg.inv(Dm)
    J = np.linalg.det(F)
    Fit = np.transpose(np.linalg.inv(F), (0, 2, 1))
    P = mu * (F - Fit) + lam * np.log(J)[:, None, None] * Fit
    return P @ np.transpose(F, (0, 2, 1)) / J[:, None, None]


def patch_report(sc, x):
    """sigma_zz mean, its largest relative error against -pressure and the
    largest other stress component, per block, for a patch-test state x
    (pad vertices, then master vertices)."""
    n = sc.X.shape[0]
    out = {}
    for name, X, T, xs in (("upper", sc.X, sc.tets, x[:n]), ("lower", sc.Y0, sc.mtets, x[n:])):
        sig = cauchy_stress(X, T, xs, sc.params["youngs"], sc.params["poisson"])
        szz = sig[:, 2, 2]
        other = np.abs(sig[:, [0, 1, 0, 0, 1], [0, 1, 1, 2, 2]]).max()
        out[name] = dict(mean=float(szz.mean()), max_rel_err=float(np.abs(szz / -10.0 - 1.0).max()),
                         spurious=float(other))
    return out
