"""Input generators: valid simple CSR, determinism, the stated sizes."""
import numpy as np
import pytest

import graphgen as gg


def assert_simple_csr(g):
    rp, col = g.rowptr, g.col
    assert rp.dtype == np.int64 and col.dtype == np.int32
    assert rp[0] == 0 and rp[-1] == col.size and np.all(np.diff(rp) >= 0)
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rp))
    assert np.all(col >= 0) and np.all(col < g.n)
    assert not np.any(src == col), "self-loop"
    # strictly ascending within each row (sorted, no duplicates)
    same_row = src[1:] == src[:-1]
    assert np.all(col[1:][same_row] > col[:-1][same_row])
    # symmetric
    fwd = np.sort(src * g.n + col)
    bwd = np.sort(col.astype(np.int64) * g.n + src)
    assert np.array_equal(fwd, bwd)


@pytest.mark.parametrize("make", [
    lambda: gg.erdos_renyi(500, 0.03, seed=3),
    lambda: gg.erdos_renyi(50, 1.0, seed=3),
    lambda: gg.rmat(1 << 12, 20000, seed=2),
    lambda: gg.chung_lu(5000, 2.1, 10.0, 300.0, seed=4),
    lambda: gg.barabasi_albert(800, 5, seed=5),
    lambda: gg.complete_multipartite((3, 4, 5)),
    lambda: gg.from_edges(5, [(0, 1), (1, 0), (2, 2), (3, 4), (3, 4)]),
])
def test_simple_csr(make):
    assert_simple_csr(make())


def test_exact_edge_count_and_determinism():
    a = gg.rmat(1 << 14, 100_000, seed=11)
    b = gg.rmat(1 << 14, 100_000, seed=11)
    c = gg.rmat(1 << 14, 100_000, seed=12)
    assert a.m == 100_000
    assert np.array_equal(a.col, b.col) and np.array_equal(a.rowptr, b.rowptr)
    assert not np.array_equal(a.col, c.col)


def test_er_density():
    g = gg.triangle_er()
    assert g.n == 4096 and abs(g.m - 32768) < 600  # E[m] = C(4096,2) 16/4095 = 32768
    assert_simple_csr(g)


def test_batch_layout():
    b = gg.batch_small(40, nmin=16, nmax=300, seed=3)
    assert b.G == 40 and b.vtx_off[0] == 0 and b.vtx_off[-1] == b.graph.n
    assert_simple_csr(b.graph)
    for i in range(b.G):
        v0, v1 = b.vtx_off[i], b.vtx_off[i + 1]
        assert 16 <= v1 - v0 <= 300
        seg = b.graph.col[b.graph.rowptr[v0]:b.graph.rowptr[v1]]
        assert np.all((seg >= v0) & (seg < v1)), "arc leaves its graph"
        assert_simple_csr(b.part(i))
    assert set(b.kind[::2]) == {0} and set(b.kind[1::2]) == {1}


def test_poisson_stream():
    t, q, g = gg.poisson_stream(20000, 2000.0, 3, 64, seed=1)
    assert np.all(np.diff(t) > 0)
    assert abs(t[-1] - 10.0) < 0.5
    assert set(np.unique(q)) == {0, 1, 2} and g.min() >= 0 and g.max() < 64
