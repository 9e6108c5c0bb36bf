"""GPU dual-mesh mapper (ipc_dual_map_build / ipc_dual_map_apply through the
C ABI) against the oracle's (Sec. 3.2, Eqs. bary_proj, decomp, gram,
bary_interp).

The nearest triangle can tie (a point equidistant from two triangles), so
the unique part is compared exactly: the minimum distance (the two sides
compute it in a different operation order, so within 1e-12 relative, or
1e-12 absolute on a unit-size mesh for points on the surface), the
triangle wherever the runner-up is farther by more than 1e-9 (relative and
absolute), and
otherwise that the GPU's triangle attains the minimum.  The coordinates are
compared with the oracle's for the GPU's triangle (1e-12), and the per-frame
positions with the oracle's update of the same embedding (1e-12 of the
mesh size)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2605_24339_b300 import binding
    binding.lib()
    return binding


def bent_grid(n, seed):
    """n x n grid over [0, 1]^2 with a smooth height field and jittered
    interior vertices; two triangles per quad."""
    rng = np.random.default_rng(seed)
    xs = np.linspace(0.0, 1.0, n + 1)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    V = np.stack([X.ravel(), Y.ravel(), 0.15 * np.sin(4 * X.ravel()) * np.cos(3 * Y.ravel())], 1)
    inner = (X.ravel() > 0) & (X.ravel() < 1) & (Y.ravel() > 0) & (Y.ravel() < 1)
    V[inner, :2] += rng.uniform(-0.2, 0.2, (inner.sum(), 2)) / n
    T = []
    for i in range(n):
        for j in range(n):
            a, b = i * (n + 1) + j, (i + 1) * (n + 1) + j
            T += [[a, b, b + 1], [a, b + 1, a + 1]]
    return V, np.array(T, dtype=np.int32)


def deform(V, t):
    th = 0.4 * t
    R = np.array([[np.cos(th), 0, np.sin(th)], [0, 1, 0], [-np.sin(th), 0, np.cos(th)]])
    W = V.copy()
    W[:, 2] += 0.3 * t * (W[:, 0] - 0.5) ** 2
    return W @ R.T + np.array([0.1, -0.2, 0.05]) * t


def check(B, oracle_mod, V, T, P):
    dev = "cuda"
    Vd = torch.as_tensor(V, device=dev)
    Td = torch.as_tensor(T, device=dev)
    Pd = torch.as_tensor(P, device=dev)
    tri, uvwd, d2 = B.dual_map_build(Vd, Td, Pd)
    tri, uvwd, d2 = tri.cpu().numpy(), uvwd.cpu().numpy(), d2.cpu().numpy()
    otri, ouvwd, od2 = oracle_mod.dual_map_build(V, T, P)
    # distances (not their squares): a point on a vertex gives 0 on one side
    # and a rounding-sized value on the other
    np.testing.assert_allclose(np.sqrt(d2), np.sqrt(od2), rtol=1e-12, atol=1e-12)
    assert ((tri >= 0) & (tri < len(T))).all()
    # the GPU's triangle attains the minimum; where the minimum is clear it is the oracle's
    d2_gpu_tri = np.array([oracle_mod.lib().orc_pt_dist2(*[np.ascontiguousarray(q).ctypes.data for q in
                                                          (P[i], V[T[tri[i], 0]], V[T[tri[i], 1]], V[T[tri[i], 2]])])
                           for i in range(len(P))])
    np.testing.assert_allclose(np.sqrt(d2_gpu_tri), np.sqrt(od2), rtol=1e-12, atol=1e-12)
    ref = np.stack([oracle_mod.dual_map_coords(P[i], *V[T[tri[i]]]) for i in range(len(P))])
    np.testing.assert_allclose(uvwd, ref, rtol=0, atol=1e-12)
    for t in (0.0, 0.5, 1.0):
        W = deform(V, t)
        out = B.dual_map_apply(torch.as_tensor(W, device=dev), Td, torch.as_tensor(tri, device=dev),
                               torch.as_tensor(uvwd, device=dev)).cpu().numpy()
        np.testing.assert_allclose(out, oracle_mod.dual_map_apply(W, T, tri, uvwd), rtol=0, atol=1e-12)
    return tri, otri, od2


@pytest.mark.parametrize("n,npts,seed", [(6, 300, 1), (40, 4000, 2)])
def test_dual_map_matches_oracle(B, oracle_mod, n, npts, seed):
    V, T = bent_grid(n, seed)
    rng = np.random.default_rng(seed + 10)
    P = np.c_[rng.uniform(-0.05, 1.05, (npts, 2)), rng.uniform(-0.3, 0.3, npts)]
    P[: npts // 10] = rng.uniform(-2.0, 3.0, (npts // 10, 3))   # far from the surface, outside the grid
    P[npts // 10: npts // 10 + 20] = V[rng.integers(0, len(V), 20)]   # on vertices
    tri, otri, od2 = check(B, oracle_mod, V, T, P)
    # where the runner-up is clearly farther the triangle itself is unique
    n_clear = 0
    for i in rng.choice(len(P), 200, replace=False):
        d = np.array([oracle_mod.lib().orc_pt_dist2(*[np.ascontiguousarray(q).ctypes.data for q in
                                                     (P[i], V[T[k, 0]], V[T[k, 1]], V[T[k, 2]])])
                      for k in range(len(T))])
        srt = np.sqrt(np.sort(d))
        if srt[1] > srt[0] * (1 + 1e-9) + 1e-9:   # (points on a vertex tie up to rounding)
            assert tri[i] == otri[i]
            n_clear += 1
    assert n_clear > 20


def test_dual_map_undeformed_identity(B):
    V, T = bent_grid(12, 5)
    rng = np.random.default_rng(7)
    P = np.c_[rng.uniform(0, 1, (2000, 2)), rng.uniform(-0.1, 0.1, 2000)]
    Vd, Td = torch.as_tensor(V, device="cuda"), torch.as_tensor(T, device="cuda")
    tri, uvwd, _ = B.dual_map_build(Vd, Td, torch.as_tensor(P, device="cuda"))
    out = B.dual_map_apply(Vd, Td, tri, uvwd).cpu().numpy()
    np.testing.assert_allclose(out, P, rtol=0, atol=1e-12)


def test_dual_map_edge_cases(B, oracle_mod):
    # one triangle; a point above its interior, one beyond a vertex, one on an edge
    V = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    T = np.array([[0, 1, 2]], dtype=np.int32)
    P = np.array([[0.2, 0.3, 0.5], [2.0, -1.0, 0.0], [0.5, 0.5, 0.0]])
    check(B, oracle_mod, V, T, P)
    # no visual vertices
    tri, uvwd, d2 = B.dual_map_build(torch.as_tensor(V, device="cuda"), torch.as_tensor(T, device="cuda"),
                                     torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert tri.numel() == 0
    # a triangle index outside the vertex range is an argument error, not a fault
    with pytest.raises(B.GmcpError):
        B.dual_map_build(torch.as_tensor(V, device="cuda"),
                         torch.as_tensor(np.array([[0, 1, 7]], dtype=np.int32), device="cuda"),
                         torch.as_tensor(P, device="cuda"))
