"""GPU paper-exact face samples (ipc_face_clip_samples through the C ABI)
against the oracle's (Sec. 4.1 "Face samples": projection onto the slave
tangent plane, Sutherland-Hodgman clip, fan triangulation, 3-point Gauss per
sub-triangle; reading R18).  Both sides evaluate the same operations in the
same order with single rounding (the CUDA file is compiled without FMA
contraction), so the sample counts must agree exactly and the samples to
1e-13 on unit-size triangles."""
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


def random_meshes(rng, n):
    """n slave and n master triangles (separate vertices), slaves in z ~ 0,
    masters above with random tilt; a third of the masters contain their
    slave's projection, a third lie inside it."""
    xs = np.c_[rng.uniform(0, 1, (3 * n, 2)), rng.uniform(-0.05, 0.05, 3 * n)]
    xm = np.c_[rng.uniform(0, 1, (3 * n, 2)), rng.uniform(0.05, 0.3, 3 * n)]
    k = n // 3
    c = xs.reshape(n, 3, 3)[:k].mean(1, keepdims=True)
    xm.reshape(n, 3, 3)[:k] = c + 4.0 * (xm.reshape(n, 3, 3)[:k] - xm.reshape(n, 3, 3)[:k].mean(1, keepdims=True))
    c2 = xm.reshape(n, 3, 3)[k:2 * k].mean(1, keepdims=True)
    xs.reshape(n, 3, 3)[k:2 * k] = c2 - np.array([0, 0, 0.2]) + 4.0 * (
        xs.reshape(n, 3, 3)[k:2 * k] - xs.reshape(n, 3, 3)[k:2 * k].mean(1, keepdims=True))
    T = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    return xs, T, xm, T.copy()


@pytest.mark.parametrize("n,seed", [(200, 1), (20000, 2)])
def test_face_clip_matches_oracle(B, oracle_mod, n, seed):
    rng = np.random.default_rng(seed)
    xs, ts, xm, tm = random_meshes(rng, n)
    pairs = np.c_[np.arange(n), np.arange(n)].astype(np.int32)
    pairs = pairs[rng.permutation(n)]
    dev = "cuda"
    smp, cnt = B.face_clip_samples(*(torch.as_tensor(a, device=dev) for a in (xs, ts, xm, tm, pairs)))
    smp, cnt = smp.cpu().numpy(), cnt.cpu().numpy()
    check = range(n) if n <= 2000 else rng.choice(n, 2000, replace=False)
    n_with = 0
    for i in check:
        s, m = pairs[i]
        ref = oracle_mod.face_clip_samples(xs[ts[s]], xm[tm[m]])
        assert cnt[i] == len(ref), (i, cnt[i], len(ref))
        np.testing.assert_allclose(smp[i, :cnt[i]], ref, rtol=0, atol=1e-13)
        n_with += len(ref) > 0
    assert n_with > len(check) // 3


def test_face_clip_edge_cases(B):
    dev = "cuda"
    xs = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0]])
    xm = np.array([[5.0, 5, 1], [6, 5, 1], [5, 6, 1]])     # no overlap
    xv = np.array([[0.0, 0, 1], [1, 0, 1], [0, 0, 2]])     # master plane contains n_s
    T = np.array([[0, 1, 2]], dtype=np.int32)
    for m in (xm, xv):
        smp, cnt = B.face_clip_samples(*(torch.as_tensor(a, device=dev) for a in
                                         (xs, T, m, T, np.array([[0, 0]], dtype=np.int32))))
        assert cnt.item() == 0
    # an index out of range marks its pair with count -1 and leaves the others alone
    pairs = np.array([[0, 0], [0, 3], [-1, 0]], dtype=np.int32)
    smp, cnt = B.face_clip_samples(*(torch.as_tensor(a, device=dev) for a in (xs, T, xs + [0, 0, -1e-3], T, pairs)))
    assert cnt.cpu().tolist()[1:] == [-1, -1] and cnt[0].item() == 3
