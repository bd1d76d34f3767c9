"""The serving runtime's GPU-free decisions (csrc/serving_policy.h), on the CPU.

Admission is FIFO: the head of the queue starts when a lane is free, its
maps fit under the memory cap, the running tiles stay within the budget (a
request alone always starts) and no running request shares a depth map with
it in a way that needs ordering (both write one, or one writes what the
other reads; reading the same neighbour is fine). A pushed frame takes a
free slot, else evicts the oldest frame that no request holds. The tile order
of the launches and of the batched and served work lists covers every tile of
a grid exactly once. The headers are built with the host compiler through a
small ctypes shim.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2211_16266_gb300", "csrc")
SHIM = os.path.join(ROOT, "tests", "host", "serving_policy_shim.cpp")

OK, SLOTS, MEMORY, TILES, DEPTH = range(5)


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    so = str(tmp_path_factory.mktemp("policy") / "libserving_policy.so")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-I", CSRC, "-o", so, SHIM])
    L = ctypes.CDLL(so)
    ip = ctypes.POINTER(ctypes.c_int)
    u64 = ctypes.c_ulonglong
    L.sp_tile_budget.argtypes = [ctypes.c_int]
    L.sp_tile_budget.restype = u64
    L.sp_depth_conflict.argtypes = [ctypes.c_int, ip, ctypes.c_int, ip, ip, ip, ctypes.c_int]
    L.sp_admit_block.argtypes = [ctypes.c_int, ctypes.c_int, u64, u64, u64, u64, u64, u64, ctypes.c_int]
    L.sp_ring_pick_slot.argtypes = [ip, ip, ip, ctypes.POINTER(u64), ctypes.c_int]
    L.sp_tile_of_block.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ip, ip]
    L.sp_tile_of_block.restype = None
    return L


def _ints(xs):
    return (ctypes.c_int * max(1, len(xs)))(*xs)


def conflict(L, req, running):
    """req and running entries: (ref, [filter frames])."""
    ref, filters = req
    flat = [f for _, fs in running for f in fs]
    return bool(L.sp_depth_conflict(ref, _ints(filters), len(filters), _ints([r for r, _ in running]),
                                    _ints(flat), _ints([len(fs) for _, fs in running]), len(running)))


def test_depth_conflicts(lib):
    assert not conflict(lib, (4, []), [])
    assert conflict(lib, (4, []), [(4, [])])                      # two writers of frame 4
    assert conflict(lib, (4, [2, 3]), [(3, [])])                  # reads what a running request writes
    assert conflict(lib, (5, []), [(3, [5, 6])])                  # writes what a running request reads
    assert not conflict(lib, (4, [2, 3]), [(5, [2, 3])])          # both read 2 and 3: no ordering needed
    assert not conflict(lib, (4, [2]), [(5, [6]), (7, [])])
    assert conflict(lib, (4, [2]), [(5, [6]), (2, [])])           # any running request counts


def test_admission_conditions(lib):
    base = dict(running=1, max_active=4, bytes_in_use=10, mem_cap=100, running_tiles=50, tile_budget=200)

    def block(bytes_=10, tiles=10, conflict_=0, **kw):
        s = dict(base, **kw)
        return lib.sp_admit_block(s["running"], s["max_active"], s["bytes_in_use"], s["mem_cap"],
                                  s["running_tiles"], s["tile_budget"], bytes_, tiles, conflict_)

    assert block() == OK
    assert block(running=4) == SLOTS
    assert block(bytes_=90) == OK and block(bytes_=91) == MEMORY        # the cap itself still fits
    assert block(tiles=150) == OK and block(tiles=151) == TILES
    assert block(tiles=10_000, running=0, running_tiles=0) == OK        # alone, any size starts
    assert block(conflict_=1) == DEPTH
    assert block(running=4, conflict_=1, bytes_=1000) == SLOTS          # lanes are checked first


def test_tile_budget_is_two_waves_of_six_blocks(lib):
    assert lib.sp_tile_budget(152) == 152 * 12
    assert lib.sp_tile_budget(0) == 12


def _pick(L, slots):
    n = len(slots)
    used, loading, pins = ([s[i] for s in slots] for i in range(3))
    seq = (ctypes.c_ulonglong * n)(*[s[3] for s in slots])
    return L.sp_ring_pick_slot(_ints(used), _ints(loading), _ints(pins), seq, n)


def test_ring_slot_choice(lib):
    # (used, loading, pins, seq)
    assert _pick(lib, [(1, 0, 0, 5), (0, 0, 0, 0), (0, 0, 0, 0)]) == 1           # first free slot
    assert _pick(lib, [(1, 0, 0, 5), (0, 1, 1, 0), (1, 0, 0, 3)]) == 2           # loading slot skipped
    assert _pick(lib, [(1, 0, 0, 5), (1, 0, 2, 1), (1, 0, 0, 3)]) == 2           # oldest unheld frame
    assert _pick(lib, [(1, 0, 1, 5), (1, 0, 2, 1), (0, 1, 1, 0)]) == -1          # every slot held


def test_fifo_admission_simulated(lib):
    """Random arrivals and completions on a 12-frame ring, 4 lanes: requests start
    in arrival order, no two running requests ever share a depth map in a
    conflicting way, lanes, memory and tiles stay within their limits, and every
    request eventually runs."""
    rng = np.random.default_rng(7)
    max_active, cap, budget = 4, 1000, 300
    queue, running, started, submitted = [], [], [], []
    bytes_in_use = tiles_in_use = 0
    next_id = 0
    for step in range(3000):
        if rng.random() < 0.55 and next_id < 800:
            ref = int(rng.integers(0, 12))
            nf = int(rng.integers(0, 4))
            filters = [int(f) for f in rng.choice(12, size=nf, replace=False) if f != ref]
            req = dict(id=next_id, ref=ref, filters=filters, bytes=int(rng.integers(50, 400)),
                       tiles=int(rng.integers(20, 200)))
            queue.append(req)
            submitted.append(next_id)
            next_id += 1
        elif running and rng.random() < 0.6:
            done = running.pop(int(rng.integers(0, len(running))))
            bytes_in_use -= done["bytes"]
            tiles_in_use -= done["tiles"]
        while queue:
            r = queue[0]
            c = conflict(lib, (r["ref"], r["filters"]), [(q["ref"], q["filters"]) for q in running])
            b = lib.sp_admit_block(len(running), max_active, bytes_in_use, cap, tiles_in_use, budget,
                                   r["bytes"], r["tiles"], int(c))
            if b != OK:
                break
            queue.pop(0)
            running.append(r)
            started.append(r["id"])
            bytes_in_use += r["bytes"]
            tiles_in_use += r["tiles"]
            assert len(running) <= max_active and bytes_in_use <= cap
            assert len(running) == 1 or tiles_in_use <= budget
            writes = [q["ref"] for q in running]
            assert len(set(writes)) == len(writes)
            for q in running:
                for p in running:
                    assert p is q or q["ref"] not in p["filters"]
        if step > 2500 and not queue and not running and next_id >= 800:
            break
    # drain: finishing the running requests lets the rest of the queue start
    while queue or running:
        if running:
            done = running.pop(0)
            bytes_in_use -= done["bytes"]
            tiles_in_use -= done["tiles"]
        while queue:
            r = queue[0]
            c = conflict(lib, (r["ref"], r["filters"]), [(q["ref"], q["filters"]) for q in running])
            if lib.sp_admit_block(len(running), max_active, bytes_in_use, cap, tiles_in_use, budget,
                                  r["bytes"], r["tiles"], int(c)) != OK:
                break
            queue.pop(0)
            running.append(r)
            started.append(r["id"])
            bytes_in_use += r["bytes"]
            tiles_in_use += r["tiles"]
        assert queue == [] or running, "a queued request could never start"
    assert started == submitted


def test_tile_order_is_a_bijection_in_strips(lib):
    """Every launch and work list walks a gx x gy tile grid in strips of 8 tile rows,
    column by column, and the rows below the last full strip row by row: each tile
    exactly once (grids of 1..40 x 1..40 tiles and the 1920x960, 3840x1920 and 250x130
    panoramas' grids of 32x8 tiles)."""
    tx, ty = ctypes.c_int(), ctypes.c_int()
    grids = [(gx, gy) for gx in range(1, 41) for gy in range(1, 41)]
    grids += [(60, 120), (120, 240), (8, 17), ((250 + 31) // 32, (130 + 7) // 8)]
    for gx, gy in grids:
        seen = np.zeros((gy, gx), dtype=int)
        order = []
        for L in range(gx * gy):
            lib.sp_tile_of_block(gx, gy, L, ctypes.byref(tx), ctypes.byref(ty))
            assert 0 <= tx.value < gx and 0 <= ty.value < gy, (gx, gy, L)
            seen[ty.value, tx.value] += 1
            order.append((tx.value, ty.value))
        assert np.all(seen == 1), (gx, gy)
        # the first strip: 8 rows of column 0, then of column 1, ...
        if gy >= 8:
            assert order[:8] == [(0, r) for r in range(8)]
            if gx > 1:
                assert order[8] == (1, 0)
