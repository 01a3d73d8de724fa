"""The serving session's arena bookkeeping (paper_2510_15602_gb300/csrc/arena.cuh,
plain host C++) on the CPU: built with g++ behind a small C shim and driven by a
seeded random sequence of allocations and releases, it must agree after every
step with a brute-force model that marks every byte of the arena: alloc returns
the lowest-addressed run of free bytes long enough, largest() is the longest
such run, and the free list holds exactly the maximal free runs (coalesced)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_2510_15602_gb300", "csrc", "arena.cuh")

SHIM = r"""
#include "%s"
#include <stddef.h>
using qfca::Arena;
extern "C" {
void *arena_new(size_t n) { Arena *a = new Arena; a->reset(n); return a; }
void arena_free(void *a) { delete (Arena *)a; }
int arena_alloc(void *a, size_t n, size_t *off) { return ((Arena *)a)->alloc(n, off) ? 1 : 0; }
void arena_release(void *a, size_t off, size_t n) { ((Arena *)a)->release(off, n); }
size_t arena_largest(void *a) { return ((Arena *)a)->largest(); }
int arena_blocks(void *a, size_t *out, int cap) {
    int i = 0;
    for (auto &kv : ((Arena *)a)->free_) {
        if (i < cap) { out[2 * i] = kv.first; out[2 * i + 1] = kv.second; }
        i++;
    }
    return i;
}
}
"""


@pytest.fixture(scope="module")
def lib(tmp_path_factory):
    d = tmp_path_factory.mktemp("arena")
    src = d / "shim.cpp"
    src.write_text(SHIM % HEADER)
    so = d / "libarena.so"
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-fPIC", "-shared", "-o", str(so), str(src)])
    L = ctypes.CDLL(str(so))
    S = ctypes.c_size_t
    L.arena_new.restype = ctypes.c_void_p
    L.arena_new.argtypes = [S]
    L.arena_free.argtypes = [ctypes.c_void_p]
    L.arena_alloc.argtypes = [ctypes.c_void_p, S, ctypes.POINTER(S)]
    L.arena_release.argtypes = [ctypes.c_void_p, S, S]
    L.arena_largest.restype = S
    L.arena_largest.argtypes = [ctypes.c_void_p]
    L.arena_blocks.argtypes = [ctypes.c_void_p, ctypes.POINTER(S), ctypes.c_int]
    return L


def free_runs(used):
    """Maximal runs of free bytes as [(offset, length)]."""
    runs, i, n = [], 0, len(used)
    while i < n:
        if used[i]:
            i += 1
            continue
        j = i
        while j < n and not used[j]:
            j += 1
        runs.append((i, j - i))
        i = j
    return runs


def blocks(L, a):
    buf = (ctypes.c_size_t * 4096)()
    k = L.arena_blocks(a, buf, 2048)
    assert k <= 2048
    return [(buf[2 * i], buf[2 * i + 1]) for i in range(k)]


@pytest.mark.parametrize("size,seed", [(1000, 0), (4096, 1), (257, 2)])
def test_arena_matches_byte_model(lib, size, seed):
    rng = np.random.default_rng(seed)
    a = lib.arena_new(size)
    used = np.zeros(size, bool)
    live = []  # (offset, length) handed out
    try:
        for step in range(3000):
            if live and (rng.random() < 0.45 or len(live) > 40):
                off, n = live.pop(int(rng.integers(len(live))))
                lib.arena_release(a, off, n)
                assert used[off:off + n].all()
                used[off:off + n] = False
            else:
                n = int(rng.integers(1, max(2, size // 6)))
                runs = free_runs(used)
                fit = [o for o, ln in runs if ln >= n]
                off = ctypes.c_size_t(0)
                ok = lib.arena_alloc(a, n, ctypes.byref(off))
                assert bool(ok) == bool(fit), step
                if ok:
                    assert off.value == fit[0], step  # first fit: the lowest-addressed run
                    used[off.value:off.value + n] = True
                    live.append((off.value, n))
            runs = free_runs(used)
            assert blocks(lib, a) == runs, step  # coalesced: exactly the maximal free runs
            assert lib.arena_largest(a) == max([ln for _, ln in runs], default=0), step
        for off, n in live:  # everything returned: one block again
            lib.arena_release(a, off, n)
        assert blocks(lib, a) == [(0, size)]
    finally:
        lib.arena_free(a)
