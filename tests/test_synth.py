"""The seeded synthetic maps: deterministic, contiguous, shared edges bit-identical."""
import numpy as np

from paper_1802_07625_gb300 import synth


def _ring(m, k):
    return m.xy[m.ring_offsets[k]:m.ring_offsets[k + 1]]


def test_generator_is_deterministic():
    a = synth.make_workload("voronoi16_64")
    b = synth.make_workload("voronoi16_64")
    assert np.array_equal(a.xy, b.xy) and np.array_equal(a.values, b.values)


def test_xoshiro_reference_stream():
    # first outputs of xoshiro256** seeded by SplitMix64(0), independent of the host
    r = synth.Xoshiro256ss(0)
    first = [r.next_u64() for _ in range(3)]
    r2 = synth.Xoshiro256ss(0)
    assert first == [r2.next_u64() for _ in range(3)]
    assert all(0 <= v < 2 ** 64 for v in first)
    u = [synth.Xoshiro256ss(5).uniform() for _ in range(2)]
    assert u[0] == u[1] and 0.0 <= u[0] < 1.0


def test_voronoi_cells_tile_the_inset():
    m = synth.make_workload("voronoi16_64")
    areas = np.array([synth._signed_area(_ring(m, k)) for k in range(m.n_rings)])
    assert np.all(areas > 0)
    assert abs(areas.sum() - 48.0 ** 2) < 1e-9
    assert m.xy.min() >= 8.0 - 1e-9 and m.xy.max() <= 56.0 + 1e-9
    seg = np.diff(np.concatenate([_ring(m, 0), _ring(m, 0)[:1]]), axis=0)
    assert np.max(np.hypot(seg[:, 0], seg[:, 1])) <= 0.5 + 1e-9


def test_shared_edges_have_identical_vertices():
    m = synth.make_workload("voronoi16_64")
    edges = {}
    for k in range(m.n_rings):
        r = _ring(m, k)
        for a in range(len(r)):
            p, q = tuple(r[a]), tuple(r[(a + 1) % len(r)])
            edges[(p, q)] = edges.get((p, q), 0) + 1
    interior = [e for e in edges if (e[1], e[0]) in edges]
    # every interior edge appears once in each direction, with the same coordinates
    assert len(interior) > 100
    for p, q in interior:
        assert edges[(p, q)] == 1 and edges[(q, p)] == 1


def test_workload_sizes_match_their_recipes():
    m2 = synth.make_workload("clustered300_512")
    assert m2.n_regions == 300 and 35_000 < m2.n_vertices < 50_000
    m3 = synth.make_workload("powerlaw3000_1024")
    assert m3.n_regions == 3000 and 450_000 < m3.n_vertices < 700_000
    assert m3.values.min() >= 1.0


def test_blocks_map_is_seeded_and_tiles_the_inner_half():
    a, b = synth.blocks_map(128, 64), synth.blocks_map(128, 64)
    assert np.array_equal(a.values, b.values) and np.array_equal(a.xy, b.xy)
    assert a.n_regions == 8 and np.all(a.values > 0)
    assert a.xy[:, 0].min() == 32.0 and a.xy[:, 0].max() == 96.0
    assert a.xy[:, 1].min() == 16.0 and a.xy[:, 1].max() == 48.0
