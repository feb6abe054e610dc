"""Input generators: layouts tile the grid, streams are reproducible."""
import numpy as np

from workloads import (get_config, guillotine, layout_stats, lognormal_kc,
                       regular_blocks, splitmix64, uniform01)


def covers_exactly(vps, nx, ny, grid=0):
    cnt = np.zeros((ny, nx), np.int32)
    for g, x0, y0, w, h in vps:
        if g != grid:
            continue
        assert w >= 1 and h >= 1 and x0 + w <= nx and y0 + h <= ny
        cnt[y0:y0 + h, x0:x0 + w] += 1
    return (cnt == 1).all()


def test_splitmix64_published_outputs():
    """First outputs of SplitMix64 seeded with 0 (reference implementation
    by Vigna, splitmix64.c)."""
    got = [int(splitmix64(0, n)) for n in range(3)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_uniform_range():
    u = uniform01(7, np.arange(100000, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def test_regular_blocks_tile():
    assert covers_exactly(regular_blocks(64, 64, 16, 16), 64, 64)
    assert covers_exactly(regular_blocks(100, 37, 32, 32), 100, 37)


def test_guillotine_tiles_with_min_side():
    vps = guillotine(1024, 1024, 4096, 8, 99)
    assert len(vps) == 4096 and covers_exactly(vps, 1024, 1024)
    st = layout_stats(vps)
    assert st["w_min"] >= 8 and st["h_min"] >= 8 and st["area_mean"] == 256.0
    assert vps == guillotine(1024, 1024, 4096, 8, 99)


def test_guillotine_x_alignment():
    vps = guillotine(1024, 1024, 4096, 8, 99, x_align=8)
    assert len(vps) == 4096 and covers_exactly(vps, 1024, 1024)
    assert all(x0 % 8 == 0 and w % 8 == 0 for (_, x0, _, w, _) in vps)
    assert len({w for (_, _, _, w, _) in vps}) > 3 and len({h for (_, _, _, _, h) in vps}) > 10


def test_lognormal_kc_range_and_mean():
    k = lognormal_kc(256, 256, 3, 0)
    assert k.dtype == np.int32 and k.min() >= 1 and k.max() <= 64
    assert 3.5 < k.mean() < 5.5
    assert not np.array_equal(k, lognormal_kc(256, 256, 3, 1))


def test_batch_workload_grids():
    w = get_config("batch64_fp32")
    assert len(w.grids) == 64
    for gi, g in enumerate(w.grids):
        assert 64 <= g.nx <= 512 and g.nx == g.ny and 32 <= g.nz <= 96
        assert 2 <= g.k_in <= 48
        assert covers_exactly(w.vps, g.nx, g.ny, grid=gi)


def test_autotune_split_layout_tiles():
    from paper_1310_4218_gb300.autotune import split_layout
    vps = guillotine(256, 256, 64, 8, 5)
    for f in (1, 2, 3):
        s = split_layout(vps, f)
        assert covers_exactly(s, 256, 256)
        assert len(s) >= len(vps)
    s2 = split_layout(vps, 2)
    assert all(w >= 8 and h >= 8 for (_, _, _, w, h) in s2)


def test_autotune_cache_key_separates_workloads():
    """The autotuner's cache key changes with the dynamics, the layout and the
    re-draw interval, so one workload never reuses another's result."""
    from paper_1310_4218_gb300.autotune import signature, split_layout
    a = get_config("lognormal_fp32_1024x1024x96")
    b = get_config("jacobi_fp32_1024x1024x96")
    ka = signature(a.grids, a.vps, a.kc_epoch_steps)
    assert ka == signature(a.grids, list(reversed(a.vps)), a.kc_epoch_steps)
    assert ka != signature(b.grids, b.vps, b.kc_epoch_steps)
    import dataclasses
    g = a.grids[0]
    assert ka != signature([dataclasses.replace(g, dynamics=1)], a.vps, a.kc_epoch_steps)
    assert ka != signature([dataclasses.replace(g, nu=0.1)], a.vps, a.kc_epoch_steps)
    assert ka != signature(a.grids, split_layout(a.vps, 2), a.kc_epoch_steps)
    assert ka != signature(a.grids, a.vps, 0)


def test_jacobi_workload_is_the_lognormal_one_with_the_jacobi_sweep():
    """Same grid, VPs, k_c arrays and re-draws as the lognormal workload; the
    dynamics phase is the weighted Jacobi sweep (nu = 1/7), no advection."""
    a = get_config("lognormal_fp32_1024x1024x96")
    b = get_config("jacobi_fp32_1024x1024x96")
    ga, gb = a.grids[0], b.grids[0]
    assert b.vps == a.vps and b.steps == a.steps and b.kc_epoch_steps == a.kc_epoch_steps
    assert (gb.nx, gb.ny, gb.nz, gb.r) == (ga.nx, ga.ny, ga.nz, ga.r)
    assert (gb.dynamics, gb.nu) == (1, 1.0 / 7.0) and ga.dynamics == 0
    assert (gb.cx, gb.cy, gb.cz) == (0.0, 0.0, 0.0)
    assert np.array_equal(b.kc_array(0, 1), a.kc_array(0, 1))
