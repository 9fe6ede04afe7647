"""Sorting stage (Sect. 3) and neighbour lists through the C ABI: bucket keys,
bucket starts and the permutation bit-exact against the oracle's binning and
stable counting sort; neighbour sets exact against brute force."""
import math

import numpy as np
import pytest

from helpers import need_gpu, pos_h_of
from paper_1807_08116_gb300 import ics

pytestmark = pytest.mark.gpu


def _ctx(n, cap=None, log2_M=None):
    from paper_1807_08116_gb300 import native as nv
    return nv.Ctx(max(n, 1), cap if cap is not None else max(1024, 200 * n), log2_M=log2_M)


def _sort(ph, grid=None, ctx=None):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    n = len(ph)
    ctx = ctx or _ctx(n)
    x = torch.as_tensor(ph, device="cuda")
    key = torch.empty(n, dtype=torch.int32, device="cuda")
    start = torch.empty(ctx.M + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(n, dtype=torch.int32, device="cuda")
    nv.sph_bin_and_sort(ctx, x, grid=grid, key=key, cell_start=start, perm=perm)
    torch.cuda.synchronize()
    return ctx, key.cpu().numpy(), start.cpu().numpy(), perm.cpu().numpy()


def _lists(ctx, n):
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    start = torch.empty(n + 1, dtype=torch.int32, device="cuda")
    need = nv.sph_build_neighbors(ctx, n, nb_start=start)
    idx = torch.empty(max(need, 1), dtype=torch.int32, device="cuda")
    nv.sph_build_neighbors(ctx, n, nb_start=start, nb_idx=idx)
    torch.cuda.synchronize()
    assert ctx.device_status() == 0
    return start.cpu().numpy(), idx.cpu().numpy()[:need]


def _check_sort(orc, ph, grid, ctx=None):
    ctx, key, start, perm = _sort(ph, grid, ctx)
    _, _, okey = orc.bin_particles(ph, grid)
    assert np.array_equal(key, okey)
    _, ostart, operm = orc.counting_sort(okey, 1 << grid["log2_M"])
    assert np.array_equal(start, ostart)
    assert np.array_equal(perm, operm)
    return ctx, perm


def _row_sets(start, idx, perm, rows):
    """Neighbour sets (original indices) of the given original rows; asserts
    that no row holds a duplicate."""
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm), dtype=perm.dtype)
    out = {}
    for i in rows:
        s = inv[i]
        row = perm[idx[start[s]:start[s + 1]]]
        out[int(i)] = set(row.tolist())
        assert len(out[int(i)]) == len(row), f"duplicate in row {i}"
    return out


def _check_lists(orc, ph, ctx, perm, rows=None):
    n = len(ph)
    start, idx = _lists(ctx, n)
    rows = np.arange(n) if rows is None else np.asarray(rows)
    sets = _row_sets(start, idx, perm, rows)
    ostart, oidx = orc.neighbors(ph, rows=rows)
    for k, i in enumerate(rows):
        ref = set(oidx[ostart[k]:ostart[k + 1]].tolist())
        got = sets[int(i)]
        assert got == ref, f"row {i}: missing {sorted(ref - got)[:5]} extra {sorted(got - ref)[:5]}"
    return start, idx, sets


def _auto_grid(ph, log2_M):
    # the documented automatic grid, restated from its definition
    x0 = [float(np.floor(ph[:, d].min())) - 1.0 for d in range(3)]
    hmin, hmax = float(ph[:, 3].min()), float(ph[:, 3].max())
    l0 = math.ceil(math.log2(hmin))
    nl = min(24, 1 + max(0, math.ceil(math.log2(hmax)) - l0))
    return dict(x0=x0[0], y0=x0[1], z0=x0[2], log2_L0=l0, n_levels=nl, log2_M=log2_M)


def test_single_halo_sort_and_lists(orc):
    d = ics.single_halo(8192, 8192, seed=0)
    ph = pos_h_of(d["r"][:8192], d["h"])
    ctx = _ctx(8192)
    grid = _auto_grid(ph, ctx.log2_M)
    # automatic grid reproduces its definition
    _sort(ph, None, ctx)
    assert ctx.grid() == pytest.approx(grid)
    ctx, perm = _check_sort(orc, ph, grid, ctx)
    start, idx, sets = _check_lists(orc, ph, ctx, perm)
    mean = (start[-1]) / 8192
    print(f"mean neighbours {mean:.1f}")
    assert 40 < mean < 120


def test_explicit_grids_and_levels(orc):
    d = ics.single_halo(4096, 0, seed=3)
    ph = pos_h_of(d["r"], d["h"])
    for grid in (dict(x0=-50.0, y0=-50.0, z0=-50.0, log2_L0=-6, n_levels=12, log2_M=14),
                 dict(x0=-3.0, y0=-7.5, z0=-1.25, log2_L0=-2, n_levels=3, log2_M=12),
                 dict(x0=0.0, y0=0.0, z0=0.0, log2_L0=0, n_levels=1, log2_M=10)):
        ctx = _ctx(4096, log2_M=grid["log2_M"])
        ctx, perm = _check_sort(orc, ph, grid, ctx)
        _check_lists(orc, ph, ctx, perm)


def _adversarial(seed):
    rng = np.random.default_rng(seed)
    L = 0.125
    parts = []
    # on cell faces of the level-0 grid and exact lattice points
    g = np.arange(-4, 5) * L
    x, y, z = np.meshgrid(g, g, g[:4], indexing="ij")
    lat = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    parts.append(pos_h_of(lat, np.full(len(lat), L)))
    # many copies of one position (a long bucket) with equal and different h
    dup = np.tile([[0.3, -0.2, 0.1]], (150, 1))
    parts.append(pos_h_of(dup, rng.choice([L / 2, L, 2 * L], 150)))
    # h spanning 9 octaves
    r = rng.normal(size=(1500, 3))
    parts.append(pos_h_of(r, (L / 4) * 2.0 ** rng.uniform(0, 9, 1500)))
    # far outliers with large h and a tiny-h cluster
    parts.append(pos_h_of(rng.normal(size=(20, 3)) * 40, rng.uniform(5, 30, 20)))
    parts.append(pos_h_of(rng.normal(size=(300, 3)) * 1e-3, np.full(300, 1e-3)))
    ph = np.concatenate(parts).astype(np.float32)
    return ph[rng.permutation(len(ph))]


@pytest.mark.parametrize("seed", [0, 1])
def test_adversarial_inputs(orc, seed):
    ph = _adversarial(seed)
    n = len(ph)
    ctx = _ctx(n, cap=n * n)
    grid = _auto_grid(ph, ctx.log2_M)
    ctx, perm = _check_sort(orc, ph, grid, ctx)
    start, idx, sets = _check_lists(orc, ph, ctx, perm)
    # the relation is symmetric
    for i in range(n):
        for j in sets[i]:
            assert i in sets[j]


def test_two_halo_sampled_and_symmetric(orc):
    d = ics.two_halo(131072, 131072, seed=1)
    ng = d["n_gas"]
    ph = pos_h_of(d["r"][:ng], d["h"])
    ctx = _ctx(ng)
    grid = _auto_grid(ph, ctx.log2_M)
    ctx, perm = _check_sort(orc, ph, grid, ctx)
    rows = np.random.default_rng(2).choice(ng, 400, replace=False)
    start, idx, _ = _check_lists(orc, ph, ctx, perm, rows=rows)
    # symmetry over all rows via sorted pair lists
    s = np.repeat(np.arange(ng), np.diff(start))
    a = np.stack([s, idx], 1)
    b = np.stack([idx, s], 1)
    ka = np.sort(a[:, 0].astype(np.int64) * ng + a[:, 1])
    kb = np.sort(b[:, 0].astype(np.int64) * ng + b[:, 1])
    assert np.array_equal(ka, kb)


def test_large_collision_sampled_rows(orc):
    d = ics.two_halo(1048576, 1048576, seed=2)
    ng = d["n_gas"]
    ph = pos_h_of(d["r"][:ng], d["h"])
    ctx = _ctx(ng, cap=ng * 160)
    grid = _auto_grid(ph, ctx.log2_M)
    ctx, perm = _check_sort(orc, ph, grid, ctx)
    rows = np.random.default_rng(3).choice(ng, 96, replace=False)
    _check_lists(orc, ph, ctx, perm, rows=rows)


def test_lists_are_deterministic():
    torch = need_gpu()
    ph = _adversarial(5)
    n = len(ph)
    ctx, _, _, _ = _sort(ph, ctx=_ctx(n, cap=n * n))
    a = _lists(ctx, len(ph))
    ctx2, _, _, _ = _sort(ph, ctx=_ctx(n, cap=n * n))
    b = _lists(ctx2, len(ph))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_capacity_overflow_is_reported():
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    d = ics.single_halo(4096, 0, seed=1)
    ph = pos_h_of(d["r"], d["h"])
    ctx = _ctx(4096, cap=1000)
    _sort(ph, None, ctx)
    with pytest.raises(nv.SphError) as ex:
        nv.sph_build_neighbors(ctx, 4096)
    assert ex.value.code == nv.SPH_ERR_NB_OVERFLOW
    assert ctx.nb_total() > 1000
    # asynchronous form: the kernel drops what does not fit and raises a flag
    nv.sph_build_neighbors(ctx, 4096, want_needed=False)
    assert ctx.device_status() & nv.SPH_FLAG_NB_OVERFLOW


def test_invalid_arguments_are_rejected():
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    ctx = _ctx(100)
    x = torch.zeros((200, 4), device="cuda")
    with pytest.raises(nv.SphError):
        nv.sph_bin_and_sort(ctx, x)            # more particles than the context holds
    with pytest.raises(nv.SphError):
        nv.sph_bin_and_sort(ctx, x[:50], grid=dict(x0=0, y0=0, z0=0, log2_L0=0, n_levels=40,
                                                   log2_M=ctx.log2_M))
    with pytest.raises(nv.SphError):
        nv.sph_build_neighbors(ctx, 7)         # no sort of 7 particles happened


def test_giant_reverse_segments(orc):
    # three wide particles inside 30000 narrow ones: every narrow particle
    # reaches them from a lower level, so their rows are ~30000 long and are
    # ordered by the chunked bitonic + merge path of the segmented sort
    rng = np.random.default_rng(21)
    small = pos_h_of(rng.uniform(0, 1, size=(30000, 3)), np.full(30000, 0.02))
    big = pos_h_of(np.array([[0.5, 0.5, 0.5], [0.45, 0.5, 0.52], [0.55, 0.48, 0.5]]),
                   np.array([0.8, 0.85, 0.9]))
    ph = np.concatenate([small, big]).astype(np.float32)
    n = len(ph)
    ctx = _ctx(n, cap=n * 200)
    ctx, key, start, perm = _sort(ph, ctx=ctx)
    rows = np.concatenate([np.arange(30000, 30003), rng.choice(30000, 40, replace=False)])
    start, idx, sets = _check_lists(orc, ph, ctx, perm, rows=rows)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(n, dtype=perm.dtype)
    for i in range(30000, 30003):
        s = inv[i]
        row = idx[start[s]:start[s + 1]]
        assert len(row) > 20000
        tail = row[-20000:]          # the reverse part, canonical ascending order
        assert np.all(np.diff(tail) > 0)
    ctx2 = _ctx(n, cap=n * 200)
    _sort(ph, ctx=ctx2)
    s2, i2 = _lists(ctx2, n)
    assert np.array_equal(s2, start) and np.array_equal(i2, idx)


def test_two_pass_fallback_when_scratch_is_small(orc):
    # sparse neighbourhoods and a capacity below 48 entries per row: the build
    # falls back to the count + fill searches; the lists are the same
    rng = np.random.default_rng(61)
    n = 3000
    ph = pos_h_of(rng.uniform(0, 1, size=(n, 3)), np.full(n, 0.03))
    small = _ctx(n, cap=40 * n)
    big = _ctx(n, cap=200 * n)
    _, _, _, perm = _sort(ph, ctx=small)
    a = _lists(small, n)
    _sort(ph, ctx=big)
    b = _lists(big, n)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    _check_lists(orc, ph, small, perm, rows=np.arange(0, n, 7))


def _levels_sorted(orc, ph, grid, perm):
    level, _, _ = orc.bin_particles(ph, grid)
    return level[perm]


@pytest.mark.parametrize("n_wide", [40, 70, 200])
def test_row_layout_own_then_reverse_ascending(orc, n_wide):
    # wide particles among narrow ones get reverse parts of about 20-300
    # entries (both sides of the 32- and 64-entry limits of the per-warp
    # ranking); every row must hold its own-level-and-up part first and its
    # finer-level partners after it in ascending order, and the sets must be
    # the brute-force ones
    rng = np.random.default_rng(31 + n_wide)
    narrow = pos_h_of(rng.uniform(0, 1, size=(6000, 3)), np.full(6000, 0.04))
    wide = pos_h_of(rng.uniform(0.1, 0.9, size=(n_wide, 3)), rng.uniform(0.06, 0.2, n_wide))
    ph = np.concatenate([narrow, wide]).astype(np.float32)
    ph = ph[rng.permutation(len(ph))]
    n = len(ph)
    ctx = _ctx(n)
    grid = _auto_grid(ph, ctx.log2_M)
    ctx, perm = _check_sort(orc, ph, grid, ctx)
    start, idx, _ = _check_lists(orc, ph, ctx, perm)
    lv = _levels_sorted(orc, ph, grid, perm)
    lens = []
    for s in range(n):
        row = idx[start[s]:start[s + 1]]
        finer = lv[row] < lv[s]
        k = int(finer.sum())
        lens.append(k)
        assert not finer[:len(row) - k].any(), f"row {s}: a finer partner before the own part ends"
        assert np.all(np.diff(row[len(row) - k:]) > 0), f"row {s}: reverse part not ascending"
    lens = np.array(lens)
    assert lens.max() > 64 and ((lens > 1) & (lens <= 32)).any() and ((lens > 32) & (lens <= 64)).any()


def test_group_wider_than_one_row_cap_walks_row_by_row(orc):
    # one level of cells of 1/64 and h = 0.994: each row's search box spans
    # 255 cells per axis (16.6M cells, under the 2^24 cap of one row), but
    # two rows 3 cells apart in every axis form one group whose union box
    # spans 258 (17.2M cells, over the cap); the group is then walked row by
    # row, and the lists must still be the brute-force ones, with no flag
    x = np.float32(0.5 / 64)
    ph = np.array([[x, x, x, 0.994], [x + 3 / 64, x + 3 / 64, x + 3 / 64, 0.994]], np.float32)
    grid = dict(x0=-4.0, y0=-4.0, z0=-4.0, log2_L0=-6, n_levels=1, log2_M=10)
    ctx = _ctx(2, log2_M=10)
    ctx, perm = _check_sort(orc, ph, grid, ctx)
    start, idx, sets = _check_lists(orc, ph, ctx, perm)
    assert sets == {0: {1}, 1: {0}}


@pytest.mark.parametrize("batched", [False, True])
def test_one_launch_sort_equals_the_kernel_sequence(orc, batched):
    # the sorting stage as one cooperative launch and as its sequence of
    # kernels: keys, starts, permutation, derived grid and the neighbour
    # lists built from each (which read the bucket, level and occupancy
    # statistics) are bitwise equal, and equal to the oracle's sort
    torch = need_gpu()
    from paper_1807_08116_gb300 import native as nv
    from paper_1807_08116_gb300.sim import assemble_batch
    if batched:
        lst = [ics.two_halo(3000, 100, seed=81), ics.single_halo(5000, 0, seed=82),
               ics.single_halo(700, 50, seed=83)]
        ic, go, do, so = assemble_batch(lst)
        ng = int(ic["n_gas"])
        ph = pos_h_of(ic["r"][:ng], ic["h"])
        batch = nv.Batch(go, do, torch.as_tensor(so, device="cuda"))
    else:
        d = ics.two_halo(40000, 0, seed=84)
        ph = pos_h_of(d["r"], d["h"])
        ng = len(ph)
        batch = None
    out = []
    for fused in (1, 0, 1):
        ctx = _ctx(ng)
        ctx.set_sort_fused(fused)
        if batch is not None:
            nv.sph_ctx_set_batch(ctx, batch)
        _, key, start, perm = _sort(ph, ctx=ctx)
        grid = ctx.grid()
        st, idx = _lists(ctx, ng)
        out.append((key, start, perm, grid, st, idx))
    for a, b in ((out[0], out[1]), (out[2], out[1])):
        for x, y in zip(a, b):
            if isinstance(x, dict):
                assert x == y
            else:
                assert np.array_equal(x, y)
    if not batched:
        _, _, okey = orc.bin_particles(ph, out[0][3])
        _, ostart, operm = orc.counting_sort(okey, 1 << out[0][3]["log2_M"])
        assert np.array_equal(out[0][0], okey)
        assert np.array_equal(out[0][1], ostart)
        assert np.array_equal(out[0][2], operm)
