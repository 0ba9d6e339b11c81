"""The seeded workload recipes (CPU): the uneven batch of 64 systems and the
per-configuration seeds are deterministic, have the stated shapes, and use
only grid edges the library compiles."""
import math

from paper_1601_07159_gb300 import build_lib, synth


def test_batched_draw_recipe():
    a = synth.batched_systems()
    b = synth.batched_systems()
    assert len(a) == 64
    assert [(s.n, s.n_occ) for s in a] == [(s.n, s.n_occ) for s in b]           # seeded
    for s in a:
        assert s.n in (32, 36, 40, 48, 64)
        assert 16 <= s.n_occ <= 128
        assert s.n_bands == (3 * s.n_occ) // 2
        assert math.isclose(s.L / s.n, 20.5 / 48)                                # the 48^3 cell's spacing
        assert s.kernel == "bare"
        assert s.n in build_lib.shape_lists()["f32"][0]
    assert len({s.n for s in a}) == 5                                            # every edge drawn
    pairs = sum(s.n_occ * (s.n_occ + 1) // 2 for s in a)
    assert pairs == 207841                                                       # the unique pair solves of one batched build


def test_seeds_are_distinct_per_config_and_system():
    seeds = {synth.seed_for(c, i) for c in range(1, 6) for i in range(64)}
    assert len(seeds) == 5 * 64
    assert synth.seed_for(2) == 1601071590 + 2000


def test_named_workloads():
    assert (synth.SI64_48.n, synth.SI64_48.n_occ, synth.SI64_48.n_bands) == (48, 128, 192)
    assert synth.SI64_48.kernel == "erfc" and math.isclose(synth.SI64_48.omega, 0.106)
    assert (synth.DIFF_64.n, synth.DIFF_64.n_occ) == (64, 256)
    assert (synth.SI512_96.n, synth.SI512_96.n_occ, synth.SI512_96.n_bands) == (96, 1024, 1536)


def test_odd_radix_first_instances():
    """The FP32 grids compiled a second time with the odd radix first are
    compiled grids whose lengths have a factor 3 or 5 beside a power of two
    (where the two radix orders differ)."""
    lists = build_lib.shape_lists()
    edges, planes = lists["f32_r1"]
    assert set(edges) <= set(lists["f32"][0]) and set(planes) <= set(lists["f32"][1])
    for n in edges:
        assert (n % 3 == 0 or n % 5 == 0) and n % 4 == 0
    units = [u[1] for u in build_lib.units()]
    assert all(f"pair_plane_f32_{n}_{n}_r1.o" in units and f"pair_pencil_f32_{n}_r1.o" in units for n in edges)
