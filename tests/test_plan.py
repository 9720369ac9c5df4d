"""Host-side schedule of the batched fit (lsefit_plan_build): no GPU needed."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def B():
    from paper_1512_08017_gb300 import _build
    _build.build()
    from paper_1512_08017_gb300 import lsefit
    return lsefit


def build(B, offsets, degree=None, m_max=5, **tuning):
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    S = off.size - 1
    deg = None if degree is None else np.ascontiguousarray(degree, dtype=np.int32)
    tun = B.Tuning()
    for k, v in tuning.items():
        setattr(tun, k, v)
    plan = B.Plan()
    dp = deg.ctypes.data_as(ctypes.c_void_p) if deg is not None else None
    rc = B.lib.lsefit_plan_build(off.ctypes.data_as(ctypes.c_void_p), dp, S, m_max, ctypes.byref(tun), 152,
                                 ctypes.byref(plan), None, 0, None, 0)
    if rc not in (B.OK, B.ERR_WORKSPACE):
        return rc, None, None, None
    bt = np.zeros(max(4 * plan.n_block_tasks, 4), dtype=np.int32)
    wt = np.zeros(max(4 * plan.n_warp_tasks, 4), dtype=np.int32)
    rc = B.lib.lsefit_plan_build(off.ctypes.data_as(ctypes.c_void_p), dp, S, m_max, ctypes.byref(tun), 152,
                                 ctypes.byref(plan), bt.ctypes.data_as(ctypes.c_void_p), plan.n_block_tasks,
                                 wt.ctypes.data_as(ctypes.c_void_p), plan.n_warp_tasks)
    return rc, plan, bt[: 4 * plan.n_block_tasks].reshape(-1, 4), wt[: 4 * plan.n_warp_tasks].reshape(-1, 4)


def test_cover_and_order(B):
    rng = np.random.default_rng(1)
    lens = np.concatenate([[0, 1, 70000, 3], rng.integers(0, 20000, 500)])
    off = np.concatenate([[0], np.cumsum(lens)])
    deg = rng.integers(1, 6, lens.size)
    rc, plan, bt, wt = build(B, off, deg, warp_max_len=4096, chunk_len=8192, task_order=2,
                             schedule=1)
    assert rc == B.OK
    seen = np.zeros(lens.size, dtype=int)
    # block tasks: consecutive chunks of one series, chunk count right, first-task index right
    t = 0
    while t < len(bt):
        s, c, nch, first = bt[t]
        assert c == 0 and first == t and nch == -(-lens[s] // 8192)
        for k in range(nch):
            assert tuple(bt[t + k]) == (s, k, nch, first)
        seen[s] += 1
        t += nch
    assert plan.n_split_series == sum(1 for s in np.unique(bt[:, 0]) if -(-lens[s] // 8192) > 1)
    # block tasks longest first
    firsts = [lens[s] for s, c, _, _ in bt if c == 0]
    assert firsts == sorted(firsts, reverse=True)
    # warp tasks: records, grouped by degree then longest first
    for s, lo, hi, n in wt:
        seen[s] += 1
        assert lens[s] <= 4096
        assert (int(hi) << 32) + (int(lo) & 0xffffffff) == off[s] and n == lens[s]
    keys = [(deg[s], -lens[s]) for s in wt[:, 0]]
    assert keys == sorted(keys)
    assert np.all(seen == 1)
    assert plan.total_points == off[-1] and plan.num_series == lens.size


def test_without_degrees_longest_first(B):
    lens = np.array([5, 100, 7, 100, 3000])
    off = np.concatenate([[0], np.cumsum(lens)])
    rc, plan, bt, wt = build(B, off, warp_max_len=1 << 20)
    assert rc == B.OK and plan.n_block_tasks == 0
    assert list(wt[:, 0]) == [4, 1, 3, 2, 0]  # stable for equal lengths


def test_bad_inputs(B):
    assert build(B, [0, 5, 3])[0] == B.ERR_INVALID_ARG          # decreasing offsets
    assert build(B, [1, 5])[0] == B.ERR_INVALID_ARG             # offsets[0] != 0
    assert build(B, [0, 5], m_max=9)[0] == B.ERR_INVALID_ARG    # degree bound
    rc, plan, _, _ = build(B, [0, 0])                            # one empty series is fine
    assert rc == B.OK and plan.n_warp_tasks == 1


def test_workspace_sizes(B):
    rc, plan, _, _ = build(B, [0, 100, 200000, 200010], warp_max_len=1000, chunk_len=65536)
    assert rc == B.OK
    ws = B.lib.lsefit_batched_workspace_size(ctypes.byref(plan))
    assert ws % 256 == 0 and ws >= 256 + 16 * 3
    assert B.lib.lsefit_backward_workspace_size(ctypes.byref(plan)) > 0
    assert B.lib.lsefit_range_workspace_size(ctypes.byref(plan)) >= 256 + 16 * 3


def test_degree_classes(B):
    """Default schedule: warp tasks by degree class (degrees outside 1..8 first),
    longest first within a class; class_begin and class_points describe them."""
    rng = np.random.default_rng(2)
    lens = rng.integers(0, 70000, 800)
    off = np.concatenate([[0], np.cumsum(lens)])
    deg = rng.integers(1, 6, lens.size)
    deg[:7] = [0, -3, 9, 100, 8, 7, 6]
    rc, plan, bt, wt = build(B, off, deg, warp_max_len=1 << 20)
    assert rc == B.OK and plan.tuning.schedule == 3 and plan.n_block_tasks == 0
    cls = np.where((deg >= 1) & (deg <= 8), deg, 0)
    keys = [(cls[s], -lens[s]) for s in wt[:, 0]]
    assert keys == sorted(keys)
    begin = list(plan.class_begin)
    assert begin[0] == 0 and begin[-1] == plan.n_warp_tasks and begin == sorted(begin)
    for c in range(9):
        members = wt[begin[c]:begin[c + 1], 0]
        assert np.all(cls[members] == c) and members.size == np.count_nonzero(cls == c)
        assert plan.class_points[c] == lens[cls == c].sum()


def test_degree_classes_without_degrees(B):
    lens = np.array([5, 100, 7, 100, 3000])
    off = np.concatenate([[0], np.cumsum(lens)])
    rc, plan, bt, wt = build(B, off, warp_max_len=1 << 20)
    assert rc == B.OK
    assert list(plan.class_begin) == [0] + [5] * 9 and plan.class_points[0] == lens.sum()



def class_blocks(B, plan, grid):
    cb = np.zeros(10, dtype=np.int32)
    rc = B.lib.lsefit_plan_class_blocks(ctypes.byref(plan), grid, cb.ctypes.data_as(ctypes.c_void_p))
    assert rc == B.OK
    return cb


def test_class_blocks_share_the_grid(B):
    """Schedule 3's block sharing (lsefit_plan_class_blocks, the function the fit
    calls): a partition of the grid into one block range per degree class, in
    class order, that gives the blocks to the classes holding points."""
    grid = 152
    rng = np.random.default_rng(3)
    lens = rng.integers(1, 20000, 3000)
    off = np.concatenate([[0], np.cumsum(lens)])
    deg = rng.integers(1, 6, lens.size)
    rc, plan, _, _ = build(B, off, deg, warp_max_len=1 << 20)
    assert rc == B.OK
    cb = class_blocks(B, plan, grid)
    assert cb[0] == 0 and cb[-1] == grid and np.all(np.diff(cb) >= 0)
    counts = np.diff(cb)
    assert counts[0] == 0 and np.all(counts[6:] == 0) and np.all(counts[1:6] > 0)
    # shares follow the points: each class within two blocks of its share of the
    # points times a cost per point that grows with the degree by at most 2.2x
    pts = np.array([plan.class_points[c] for c in range(9)], dtype=float)
    share = pts[1:6] / pts[1:6].sum() * grid
    assert np.all(counts[1:6] >= np.floor(share / 2.2) - 2) and np.all(counts[1:6] <= np.ceil(share * 2.2) + 2)
    # for equal points, a higher degree never gets fewer blocks
    eq = np.concatenate([[0], np.cumsum(np.full(8 * 40, 1000))])
    rc, plan, _, _ = build(B, eq, np.repeat(np.arange(1, 9), 40), m_max=8, warp_max_len=1 << 20)
    cb = class_blocks(B, plan, grid)
    assert np.all(np.diff(np.diff(cb)[1:9]) >= 0) and cb[1] == 0 and cb[9] == grid


def test_class_blocks_single_class_and_invalid_degrees(B):
    grid = 152
    off = np.arange(0, 4097 * 4096, 4096)
    # one degree: every block starts on its class
    rc, plan, _, _ = build(B, off, np.full(4096, 3), m_max=3, warp_max_len=1 << 20)
    assert list(class_blocks(B, plan, grid)) == [0, 0, 0, 0] + [grid] * 6
    # tasks of an invalid degree are only marked: no block starts on class 0 ...
    deg = np.full(4096, 3)
    deg[:2000] = 0
    rc, plan, _, _ = build(B, off, deg, m_max=3, warp_max_len=1 << 20)
    assert plan.class_points[0] == 2000 * 4096
    assert list(class_blocks(B, plan, grid)) == [0, 0, 0, 0] + [grid] * 6
    # ... unless they are all there is: a plan built without degrees shares the
    # grid as one class (before, its total cost was 0 and blocks started on
    # empty classes)
    rc, plan, _, _ = build(B, off, m_max=3, warp_max_len=1 << 20)
    assert plan.class_points[0] == 4096 * 4096
    assert list(class_blocks(B, plan, grid)) == [0] + [grid] * 9
    rc, plan, _, _ = build(B, off, np.zeros(4096), m_max=3, warp_max_len=1 << 20)
    assert list(class_blocks(B, plan, 7)) == [0] + [7] * 9


def test_class_blocks_bad_arguments(B):
    rc, plan, _, _ = build(B, [0, 10, 20], [1, 2])
    cb = np.zeros(10, dtype=np.int32)
    ptr = cb.ctypes.data_as(ctypes.c_void_p)
    assert B.lib.lsefit_plan_class_blocks(ctypes.byref(plan), 0, ptr) == B.ERR_INVALID_ARG
    assert B.lib.lsefit_plan_class_blocks(None, 152, ptr) == B.ERR_INVALID_ARG
    assert B.lib.lsefit_plan_class_blocks(ctypes.byref(plan), 152, None) == B.ERR_INVALID_ARG


def test_plan_records_a_common_warp_task_length(B):
    """warp_task_len: the length every warp task shares (the gradient pass then
    splits their points evenly over its warps), 0 when lengths differ."""
    rc, plan, _, _ = build(B, np.arange(0, 65 * 4096, 4096), m_max=3)
    assert rc == B.OK and plan.warp_task_len == 4096
    rc, plan, _, _ = build(B, [0, 10, 30, 60], m_max=3)
    assert rc == B.OK and plan.warp_task_len == 0
    # series longer than warp_max_len become block tasks and do not count
    rc, plan, _, _ = build(B, [0, 100, 200, 300, 100300], m_max=3, warp_max_len=1000)
    assert rc == B.OK and plan.warp_task_len == 100 and plan.n_block_tasks > 0
    rc, plan, _, _ = build(B, [0], m_max=3)
    assert rc == B.OK and plan.warp_task_len == 0
