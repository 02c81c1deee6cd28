"""The algorithmic work that bench.py divides by the measured kernel times (the numerators of
its roofline fractions), checked against closed forms of the nested-dissection tree and of
the local solves.  CPU only."""
import bench


def _levels(nodes):
    out = {}
    for ns, nf, lev in nodes:
        out.setdefault(lev, []).append((ns, nf))
    return out


def test_nested_dissection_sizes_of_the_1024_grid():
    # 64 x 64 subdomains of 16^2 cells, P1 on 4-edge segments: 16 DOFs per interface.  Level L
    # halves the subdomain grid L times (4096 / 2^L nodes); its separator is a line of
    # 2^floor(L/2) interfaces; the root separator is a whole line of 64 interfaces.
    lev = _levels(bench.nd_sizes([16] * 64, [16] * 64))
    assert sorted(lev) == list(range(1, 13))
    for L, ns_nf in lev.items():
        assert len(ns_nf) == 4096 >> L
        assert max(ns for ns, _ in ns_nf) == 16 * (1 << (L // 2))
    assert lev[12] == [(1024, 1024)]  # the root: no boundary
    # a level-1 node (two subdomains) in the interior is bounded by 6 interfaces
    assert max(nf for _, nf in lev[1]) == 16 + 6 * 16
    # the two halves of the domain share the root separator as their whole boundary
    assert all(nf == 512 + 1024 for _, nf in lev[11])


def test_interface_sweep_bytes_are_one_read_of_each_block():
    nodes = bench.nd_sizes([16] * 64, [16] * 64)
    (l1b, l1f), (ub, uf), (db, df) = bench.iface_work(nodes)
    # upward: every internal node reads its nsep x nf separator rows once (8 bytes, one
    # multiply-add each) plus its gathered right-hand side and output
    total_up = sum(8.0 * ns * nf + 16.0 * nf for ns, nf, _ in nodes)
    assert l1b + ub == total_up
    assert l1f + uf == sum(2.0 * ns * nf for ns, nf, _ in nodes)
    assert l1b == sum(8.0 * ns * nf + 16.0 * nf for ns, nf, lev in nodes if lev == 1)
    # downward: levels 2 .. 11 read their nsep x nbnd coupling blocks (the root is final after
    # the upward sweep, level 1 is done inside the reconstruction)
    assert db == sum(8.0 * ns * (nf - ns) + 16.0 * ns for ns, nf, lev in nodes if 2 <= lev <= 11)
    assert df == sum(2.0 * ns * (nf - ns) for ns, nf, lev in nodes if 2 <= lev <= 11)
    # the figures the ncu summaries compare the measured DRAM traffic with
    assert round(ub / 1e6, 1) == 307.9 and round(db / 1e6, 1) == 230.1 and round(l1b / 1e6, 1) == 32.4


def test_local_solve_work_per_subdomain():
    # a 16^2 subdomain: factor of b = 16 block rows of 16 x 16, one block solve (2 b a^2
    # multiply-adds), the residual and its stencil
    (mb, mf), (db, df) = bench.local_work([16], [16], 1, True)
    assert mb == 8.0 * 16 * 256 + 80.0 * 256
    assert mf == 4.0 * 16 * 256 + 14.0 * 256
    assert db == 4.0 * 16 * 256 + 80.0 * 256  # float32 factor of the downscaling
    assert df == 4.0 * 16 * 256 + 18.0 * 256
    (mb64, _), (db64, _) = bench.local_work([16] * 4, [16] * 2, 3, False)
    assert mb64 == 3 * 8 * mb and db64 == 3 * 8 * (8.0 * 16 * 256 + 80.0 * 256)
