"""The Gram step of the recycle update (rbicgstab_update_gram): G = Z^T Z and
H = Z^T W for the FP32 column blocks W = [Y, P, S], Z = [AY, AP, AS] of the
mixed path, on the tensor cores (tcgen05, TF32 pairs) and on CUDA cores,
against the same products formed in FP64 with NumPy from the same FP32
values.  Each entry is checked against the error bound of its kernel's
arithmetic, relative to sum_i |z_i w_i|:

* CUDA cores: FP32 sums of 8 rows, compensated across chunks:
  gamma_8 = 8u / (1 - 8u), u = 2^-24;
* tensor cores: the TF32 split (hi hi' + hi lo' + lo hi' misses at most
  3 * 2^-22 |x x'|) plus FP32 accumulation in TMEM over a chunk of 4 tiles
  x 4 K-steps x 3 products and FP32 sums of the chunks of one CTA:
  3 * 2^-22 + gamma_L, L = 48 + chunks per CTA.

Column scales spread over six decades; n is ragged (not a multiple of the
32-row tile) and spans one partial chunk to many per CTA."""
import numpy as np
import pytest

from paper_1406_2831_gb300 import build as rbuild
from paper_1406_2831_gb300 import rbicgstab as rb

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


def gamma(L):
    return L * U32 / (1 - L * U32)


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    rbuild.build()
    rb.lib()
    return t


def _blocks(torch, n, ky, nit, ns, seed, same_sign=False):
    rng = np.random.default_rng(seed)
    ld = (n + 31) // 32 * 32

    def blk(c):
        a = np.zeros((c, ld), np.float32)
        v = rng.standard_normal((c, n))
        if same_sign:
            v = np.abs(v)
        v *= 10.0 ** rng.uniform(-3, 3, (c, 1))
        a[:, :n] = v
        return a
    host = [blk(ky), blk(ky), blk(nit), blk(nit), blk(ns), blk(ns)]
    dev = [torch.from_numpy(h).cuda() for h in host]
    return host, dev, ld


def _reference(host, n):
    Y, AY, P, AP, S, AS = [h[:, :n].astype(np.float64) for h in host]
    Z = np.vstack([AY, AP, AS])
    W = np.vstack([Y, P, S])
    return Z @ Z.T, Z @ W.T, np.abs(Z) @ np.abs(Z).T, np.abs(Z) @ np.abs(W).T


def _tc_bound(n):
    tiles = (n + 31) // 32
    chunks = (tiles + 3) // 4
    grid = min(152, chunks)
    per_cta = (chunks + grid - 1) // grid
    return 3 * 2.0 ** -22 + gamma(48 + per_cta)


CASES = [
    # n, ky, nit, ns, kcap, scap
    (100_003, 20, 25, 24, 20, 25),     # the benchmark's k = 20, s = 25, a half-step cycle
    (100_003, 0, 25, 25, 20, 25),      # the first cycle of a solve without a space
    (77, 8, 3, 3, 8, 25),              # one partial tile
    (40_000, 30, 25, 25, 30, 25),      # k = 30 (the 27-point workload)
    (2_000_003, 20, 25, 25, 20, 25),   # 128^3-sized columns: many chunks per CTA
]


@pytest.mark.parametrize("case", CASES)
def test_update_gram_both_paths_within_their_bounds(torch, case):
    n, ky, nit, ns, kcap, scap = case
    host, dev, ld = _blocks(torch, n, ky, nit, ns, seed=n + ky)
    G0, H0, AG, AH = _reference(host, n)
    for path, bound in (("cudacore", gamma(8)), ("tensor", _tc_bound(n))):
        G, H = rb.update_gram_n(n, *dev, kcap=kcap, scap=scap, path=path)
        rg = np.max(np.abs(G - G0) / AG)
        rh = np.max(np.abs(H - H0) / AH)
        print(f"{path:8s} n={n} m={ky + nit + ns}: max |err| / sum|zw|  G {rg:.2e}  H {rh:.2e}  (bound {bound:.2e})")
        assert rg <= bound and rh <= bound, (path, rg, rh, bound)
        assert np.array_equal(G, G.T)


def test_update_gram_same_sign_columns(torch):
    """All entries positive: the partial sums grow linearly, the worst case
    for FP32 accumulation."""
    n = 300_007
    host, dev, ld = _blocks(torch, n, 20, 25, 25, seed=5, same_sign=True)
    G0, H0, AG, AH = _reference(host, n)
    G, H = rb.update_gram_n(n, *dev, kcap=20, scap=25, path="tensor")
    rg = np.max(np.abs(G - G0) / AG)
    rh = np.max(np.abs(H - H0) / AH)
    print(f"tensor same-sign n={n}: G {rg:.2e} H {rh:.2e}")
    assert max(rg, rh) <= _tc_bound(n)


def test_update_gram_deterministic(torch):
    n = 250_001
    host, dev, ld = _blocks(torch, n, 20, 25, 25, seed=9)
    G1, H1 = rb.update_gram_n(n, *dev, kcap=20, scap=25, path="tensor")
    G2, H2 = rb.update_gram_n(n, *dev, kcap=20, scap=25, path="tensor")
    assert np.array_equal(G1, G2) and np.array_equal(H1, H2)


def test_update_gram_rejects_layouts_that_do_not_fit(torch):
    host, dev, ld = _blocks(torch, 1000, 8, 8, 8, seed=1)
    with pytest.raises(rb.RbError):
        rb.update_gram_n(1000, *dev, kcap=64, scap=32, path="tensor")
    with pytest.raises(rb.RbError):
        rb.update_gram_n(1000, *dev, kcap=4, scap=25, path="auto")   # ky = 8 > kcap
