"""The benchmark's algorithmic byte and flop counts, rebuilt stream by stream
from the arrays each pass reads and writes (Alg. 2 passes P1-P5, Alg. 1),
at the 128^3 benchmark operator: these are the numerators of the reported
roofline fractions."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

N = 128
n = N ** 3
z = 7 * N ** 3 - 6 * N ** 2      # 7-point stencil with Dirichlet boundary


def _streams(vb, ab, k, R):
    """Bytes per pass as a list of (array, bytes) streams, each touched once."""
    A = [("val", z * ab), ("col", 4 * z), ("row_ptr", 4 * (n + 1))]
    vec = n * vb
    P1 = A + [("p_r gather", R * vec), ("C-hat", k * vec), ("r~0", vec), ("q_raw_r write", R * vec)]
    P2 = [("q_raw_r", R * vec), ("C", k * vec), ("r_r", R * vec), ("q_r write", R * vec), ("s_r write", R * vec)]
    P3 = A + [("s_r gather", R * vec), ("C-hat", k * vec), ("t_raw_r write", R * vec)]
    P4 = [("t_raw_r", R * vec), ("C", k * vec), ("s_r", R * vec), ("r~0", vec), ("t_r write", R * vec)]
    P5 = [(f"{v}_r", R * vec) for v in ("x", "p", "q", "s", "t")] + \
         [(f"{v}_r write", R * vec) for v in ("x", "r", "p")]
    return [sum(b for _, b in P) for P in (P1, P2, P3, P4, P5)]


def test_pass_bytes_match_stream_inventory():
    for vb, ab, k, R in [(4, 4, 20, 4), (8, 8, 20, 1), (4, 4, 20, 2), (8, 8, 8, 4)]:
        assert bench.pass_bytes(n, z, k, vb, ab, R) == _streams(vb, ab, k, R), (vb, ab, k, R)


def test_iteration_totals():
    """A mixed 4-RHS block iteration moves 1.58 GB; an FP64 single-RHS one 2.06 GB."""
    assert abs(sum(bench.pass_bytes(n, z, 20, 4, 4, 4)) / 1e9 - 1.58) < 0.005
    assert abs(sum(bench.pass_bytes(n, z, 20, 8, 8, 1)) / 1e9 - 2.06) < 0.005


def test_pass_flops_counts():
    """Per RHS: an SpMV is 2z, a k-column projection or correction 2nk, a dot
    or axpy 2n."""
    k = 20
    f = bench.pass_flops(n, z, k, 1)
    assert f[0] == 2 * z + 2 * n * k + 2 * n          # A p, C-hat^T q_raw, (r~0, q_raw)
    assert f[1] == 2 * n * k + 2 * n + 2 * n          # C zeta, s = r - alpha q, ||s||^2
    assert f[2] == 2 * z + 2 * n * k                  # A s, C-hat^T t_raw
    assert f[3] == 2 * n * k + 4 * 2 * n              # C gamma, (s,t), (t,t), (r~0,t), (r~0,s)
    assert f[4] == 10 * n                             # x, r, p updates and ||r||^2
    assert bench.pass_flops(n, z, k, 4) == [4 * v for v in f]


def test_rbicg_iteration_model():
    """Alg. 1, FP64, k = 20: two SpMV + projection passes (A with C-hat, A^T
    with C), the corrections of q and q~ with (p~, q), four axpys with three
    dots, two search-direction updates."""
    k, v = 20, 8
    A = (v + 4) * z + 4 * (n + 1)
    b1 = 2 * (A + n * v + k * n * v + n * v)               # matrix, p gather, k columns, z write
    b2 = 2 * k * n * v + 3 * n * v + 2 * n * v             # C, C~, z, z~, p~; q, q~ writes
    b3 = 8 * n * v + 4 * n * v                             # x, x~, r, r~, p, p~, q, q~; 4 writes
    b4 = 4 * n * v + 2 * n * v                             # r, r~, p, p~; 2 writes
    byt, fl = bench.rbicg_iter_bytes_flops(n, z, k)
    assert byt == b1 + b2 + b3 + b4
    assert fl == 2 * (2 * z + 2 * n * k) + (4 * n * k + 2 * n) + (8 * n + 6 * n) + 4 * n
