"""The library's GPU-free host logic (paper_2504_13750_gb300/csrc/janc_host.h),
driven on the CPU through tests/host_harness.cpp:

* the serving pool allocator: first fit, 256-byte pieces, no overlap,
  merging of free neighbours;
* the admission pass of the continuous-batching server: arrival order with
  skip-ahead past requests the pool cannot hold, the slot limit, the cell
  budget (a request over it is admitted only into an empty active set; later
  requests pass it until it has waited max_skip_s), failed admissions.

(The AMR block lists are built on the device; tests/test_gpu_amr.py checks
them against the AMR oracle's neighbour definition.)"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def hh(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("hh") / "libhost_harness.so")
    subprocess.run([cxx, "-std=c++17", "-O1", "-shared", "-fPIC", os.path.join(HERE, "host_harness.cpp"), "-o", out],
                   check=True)
    lib = ctypes.CDLL(out)
    P = ctypes.c_void_p
    lib.hh_pool.restype = ctypes.c_int
    lib.hh_pool.argtypes = [ctypes.c_longlong, P, ctypes.c_int, P, P, P, P, ctypes.c_int]
    lib.hh_admission.restype = ctypes.c_int
    lib.hh_admission.argtypes = [ctypes.c_int, P, P, P, P, ctypes.c_longlong, ctypes.c_int, ctypes.c_longlong,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong,
                                 P, P, P, P]
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def pool_run(hh, size, ops):
    op = np.asarray(ops, dtype=np.int64)
    out = np.zeros(len(op), dtype=np.int64)
    used = np.zeros(1, dtype=np.int64)
    fo = np.zeros(256, dtype=np.int64)
    fl = np.zeros(256, dtype=np.int64)
    nf = hh.hh_pool(size, _ptr(op), len(op), _ptr(out), _ptr(used), _ptr(fo), _ptr(fl), 256)
    return out, int(used[0]), list(zip(fo[:nf].tolist(), fl[:nf].tolist()))


def test_pool_first_fit_and_merging(hh):
    KB = 1024
    # A = 1000 B (one 1 KiB piece), B = 256, C = 512; free B; a 200 B request
    # takes B's hole (the first fit), a 300 B request does not fit there and
    # goes after C; freeing everything leaves one block
    out, used, free = pool_run(hh, 8 * KB, [1000, 256, 512, -2, 200, 300, -1, -3, -5, -6])
    assert out[:3].tolist() == [0, 1024, 1280]
    assert out[4] == 1024 and out[5] == 1792
    assert used == 0 and free == [(0, 8 * KB)]
    # nothing fits: -1, and the pool is unchanged
    out, used, free = pool_run(hh, 2 * KB, [1500, 1000])
    assert out.tolist() == [0, -1] and used == 1536 and free == [(1536, 512)]


def test_pool_random_operations_keep_pieces_disjoint(hh):
    rng = np.random.default_rng(0)
    size = 1 << 20
    ops, live = [], []
    for i in range(400):
        if live and rng.random() < 0.45:
            j = live.pop(int(rng.integers(len(live))))
            ops.append(-(j + 1))
        else:
            ops.append(int(rng.integers(1, 40000)))
            live.append(i)
    out, used, free = pool_run(hh, size, ops)
    held = {}
    for i, o in enumerate(ops):
        if o > 0 and out[i] >= 0:
            held[i] = (int(out[i]), (o + 255) // 256 * 256)
        elif o < 0:
            held.pop(-o - 1, None)
    pieces = sorted(list(held.values()) + free)
    assert all(off % 256 == 0 for off, _ in pieces)
    # held pieces and free blocks tile [0, size) exactly, and free blocks never touch
    pos = 0
    for off, n in pieces:
        assert off == pos, (off, pos)
        pos += n
    assert pos == size
    assert used == sum(n for _, n in held.values())
    assert all(a + n < b for (a, n), (b, _) in zip(free, free[1:]))


def admission(hh, reqs, *, pool=1 << 30, max_active=64, budget=0, max_skip=0.0, now=0.0, active=(0, 0, 0),
              fail=()):
    n = len(reqs)
    cells = np.array([r[0] for r in reqs], dtype=np.int64)
    fp = np.array([r[1] for r in reqs], dtype=np.int64)
    ts = np.array([r[2] for r in reqs], dtype=np.float64)
    fl = np.array([1 if i in fail else 0 for i in range(n)], dtype=np.int32)
    out = np.zeros(max(n, 1), dtype=np.int32)
    left = np.zeros(max(n, 1), dtype=np.int32)
    nleft = np.zeros(1, dtype=np.int32)
    pused = np.zeros(1, dtype=np.int64)
    na = hh.hh_admission(n, _ptr(cells), _ptr(fp), _ptr(ts), _ptr(fl), pool, max_active, budget, max_skip, now,
                         active[0], active[1], active[2], _ptr(out), _ptr(left), _ptr(nleft), _ptr(pused))
    assert na >= 0
    return out[:na].tolist(), left[:int(nleft[0])].tolist(), int(pused[0])


def test_admission_in_arrival_order_up_to_the_slot_limit(hh):
    reqs = [(1000, 4096, 0.0)] * 5
    adm, left, used = admission(hh, reqs, max_active=3)
    assert adm == [0, 1, 2] and left == [3, 4] and used == 3 * 4096
    # slots already taken count too
    adm, left, _ = admission(hh, reqs, max_active=3, active=(2, 100, 0))
    assert adm == [0] and left == [1, 2, 3, 4]


def test_admission_skips_past_what_the_pool_cannot_hold(hh):
    # 10 KiB pool with 6 KiB in use: the 8 KiB head waits, the 2 KiB one behind it is admitted
    reqs = [(10, 8192, 0.0), (10, 2048, 0.0), (10, 4096, 0.0)]
    adm, left, used = admission(hh, reqs, pool=10 * 1024, active=(1, 10, 6 * 1024))
    assert adm == [1] and left == [0, 2] and used == 8 * 1024


def test_cell_budget_with_aging(hh):
    # 500 cells active, budget 600: the 200-cell head would exceed it
    reqs = [(200, 256, 0.0), (50, 256, 0.5), (60, 256, 0.6)]
    adm, left, _ = admission(hh, reqs, budget=600, max_skip=1.0, now=0.9, active=(1, 500, 256))
    assert adm == [1] and left == [0, 2]          # the head waits, later ones pass it (550 + 60 > 600)
    adm, left, _ = admission(hh, reqs, budget=600, max_skip=1.0, now=1.0, active=(1, 500, 256))
    assert adm == [] and left == [0, 1, 2]        # the head has waited 1 s: nothing passes it any more
    # a request over the budget is admitted into an empty active set, and then blocks the rest
    adm, left, _ = admission(hh, [(1000, 256, 0.0), (50, 256, 0.0)], budget=600, max_skip=5.0, now=1.0)
    assert adm == [0] and left == [1]
    # no budget: everything that fits goes in
    adm, left, _ = admission(hh, reqs, budget=0, active=(1, 500, 256))
    assert adm == [0, 1, 2] and left == []


def test_failed_admission_leaves_the_queue_and_returns_its_piece(hh):
    reqs = [(10, 4096, 0.0), (10, 4096, 0.0), (10, 4096, 0.0)]
    adm, left, used = admission(hh, reqs, fail={1})
    assert adm == [0, 2] and left == [] and used == 2 * 4096
