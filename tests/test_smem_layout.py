"""Shared-memory layout of the compile-time FFT engine (host logic, no GPU).

The kernels keep TB sequences of length N in one [N][TB] buffer with the swizzled
position at(idx, b) of tf_fft_ct.cuh: 64-byte rows are paired across blocks of S rows
(S = the plan's first radix) and the sequence index is XOR-swizzled by the row.  This test
restates that mapping and the Stockham pass index map in Python.  It then checks two
properties for every plan of the menus in tf_ct_kernels.cuh:

* at() is a bijection onto [0, N*TB) (both precisions);
* every pass's loads and stores (16-byte accesses by quarter-warp phases, FP32 tiles)
  need the minimum number of shared-memory wavefronts, i.e. no bank conflicts.

The menus are parsed from the kernel header, so a new plan is covered automatically.
"""
import os
import re
from collections import defaultdict

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_2004_13904_gb300", "csrc", "tf_ct_kernels.cuh")


def _menu(name):
    text = open(HDR).read()
    i = text.index(f"#define {name}(X)")
    j = text.index("\n\n", i)
    return [tuple(int(v) for v in m.split(",")) for m in re.findall(r"X\(([\d,\s]+)\)", text[i:j])]


def _plans():
    out = []
    for name in ("TF_CT_MENU", "TF_CT_MENU_COLS_F32"):
        for entry in _menu(name):
            out.append((name, entry[0], entry[1:]))
    return out


def _tiles(N, radices, dtype):
    """(TB, V, NT) as Tiles / ColTiles choose them."""
    if radices[0] >= 16:
        return 8, 2, 64
    if dtype == "f32":
        return (16 if N <= 96 else 8), 2, (64 if N <= 64 else (128 if N <= 256 else 256))
    return (8 if N <= 96 else 4), 2, 64


def _at(TB, csize, S):
    rows_per_line = max(128 // (TB * csize), 1)

    q = 2 if TB * csize == 64 else 4 if TB * csize == 32 else 1

    def row_of(idx):
        return idx ^ ((idx // S) & (q - 1)) if q > 1 else idx

    def swz(row):
        return ((row // rows_per_line) & (TB // 2 - 1)) << 1 if TB >= 4 else 0

    def at(idx, b):
        row = row_of(idx)
        return row * TB + (b ^ swz(row))
    return at


def _wavefronts(word_addrs, access_bytes):
    per = 128 // access_bytes
    words = access_bytes // 4
    total = 0
    for p in range(0, 32, per):
        banks = defaultdict(set)
        for a in word_addrs[p:p + per]:
            if a is None:
                continue
            for w in range(words):
                banks[(a + w) % 32].add(a + w)
        total += max((len(v) for v in banks.values()), default=0)
    return total


@pytest.mark.parametrize("menu,N,radices", _plans())
@pytest.mark.parametrize("dtype,csize", [("f32", 8), ("f64", 16)])
def test_position_map_is_a_bijection(menu, N, radices, dtype, csize):
    TB, _, _ = _tiles(N, radices, dtype)
    at = _at(TB, csize, radices[0])
    pos = sorted(at(i, b) for i in range(N) for b in range(TB))
    assert pos == list(range(N * TB))


@pytest.mark.parametrize("menu,N,radices", _plans())
def test_fp32_passes_are_bank_conflict_free(menu, N, radices):
    TB, V, NT = _tiles(N, radices, "f32")
    at = _at(TB, 8, radices[0])
    G = TB // V
    Ns = 1
    for R in radices:
        NB = N // R
        total = NB * G
        for w in range(NT // 32):
            for it in range((total + NT - 1) // NT):
                us = [w * 32 + lane + it * NT for lane in range(32)]
                active = sum(u < total for u in us)
                if not active:
                    continue
                for r in range(R):
                    loads, stores = [], []
                    for u in us:
                        if u >= total:
                            loads.append(None)
                            stores.append(None)
                            continue
                        j, b0 = u // G, (u % G) * V
                        k = j % Ns
                        loads.append(2 * at(j + r * NB, b0))
                        stores.append(2 * at((j - k) * R + k + r * Ns, b0))
                    minimum = (active * 16 + 127) // 128
                    assert _wavefronts(loads, 16) == minimum, (N, radices, R, "load")
                    assert _wavefronts(stores, 16) == minimum, (N, radices, R, "store")
        Ns *= R


def test_menus_parsed():
    rows, cols = _menu("TF_CT_MENU"), _menu("TF_CT_MENU_COLS_F32")
    assert (224, 8, 4, 7) in rows and (224, 16, 14) in cols
    assert [e[0] for e in rows] == [e[0] for e in cols]


def test_forward_accumulator_tmem_budget():
    """cols_fwd keeps the layer accumulators of MC model columns in tensor memory for
    single-precision plans on 256-thread CTAs: the last pass's slots (iterations x last
    radix x 4 words) fit the 32 columns given to each model column in each half of the
    CTA's warps, the last pass gives every thread a task (every TMEM access warp-uniform),
    and the shared-memory request lets at most 4 CTAs reside on an SM (228 KB, 1 KB
    reserved per CTA), whose allocations then fit the SM's 512 columns (none waits).
    The kernel's two shared buffers (passes alternate between them) are what the launch
    asks for, so this also checks the request covers the second buffer."""
    text = open(HDR).read()
    col_words = int(re.search(r"kColWords = (\d+);", text).group(1))
    mc = int(re.search(r"#define TF_FWD_MC (\d+)", text).group(1))
    floor = int(re.search(r"constexpr size_t kTmemSmemFloor = (\d+);", text).group(1))
    alloc = 2 * mc * col_words
    assert alloc in (32, 64, 128, 256, 512)          # a power of two, at least 32
    used = 0
    for N, *radices in _menu("TF_CT_MENU_COLS_F32"):
        TB, V, NT = _tiles(N, radices, "f32")
        if NT != 256:
            continue
        R = radices[-1]
        total = (N // R) * (TB // V)
        iters = (total + NT - 1) // NT
        assert total % NT == 0, (N, radices)
        assert iters * R * 4 <= col_words, (N, radices)
        tw = (N - 1 + 1) & ~1
        smem = max((tw + 2 * N * TB) * 8, floor)     # two buffers (ping-pong passes)
        resident = min(233472 // (smem + 1024), 2048 // NT)
        assert resident * alloc <= 512, (N, resident)
        # cols_adj: the data spectrum in the 8 input slots of each thread's first
        # inverse-pass task (at most one per thread, tasks filling whole warps), 64
        # columns per CTA; every column CTA asks for at least the floor, so at most 4
        # (forward or adjoint) share an SM: 4 x 128 columns at most
        R0 = radices[0]
        total0 = (N // R0) * (TB // V)
        assert total0 % 32 == 0 and total0 <= NT and R0 == 8, (N, radices)
        assert min(233472 // (max((tw + 2 * N * TB) * 8, floor) + 1024), 2048 // NT) * 128 <= 512
        used += 1
    assert used >= 3          # 320, 448 and 512


def _pipe_tb():
    text = open(HDR).read()
    return int(re.search(r"#define TF_PIPE_TB (\d+)", text).group(1))


@pytest.mark.parametrize("N,radices", [(e[0], e[1:]) for e in _menu("TF_CT_MENU") if e[0] > 256])
def test_bulk_copy_row_tiles_are_bank_conflict_free(N, radices):
    """The bulk-copy row kernels (lengths above 256) run TF_PIPE_TB sequences on 32 TB
    threads: the position map stays a bijection and every pass moves its 16-byte slots at
    the minimum number of wavefronts.  The first pass of rows_c2r reads each sequence pair's
    rows 2b, 2b + 1 from the copied input tile, whose row r starts at r hs + (64 / RT)(r / 4)
    values (RT = 2 TB rows): its 8-byte loads also need the minimum (two per warp)."""
    TB, V = _pipe_tb(), 2
    NT, RT = 32 * TB, 2 * TB
    at = _at(TB, 8, radices[0])
    assert sorted(at(i, b) for i in range(N) for b in range(TB)) == list(range(N * TB))
    G = TB // V
    Ns = 1
    for R in radices:
        NB = N // R
        total = NB * G
        for w in range(NT // 32):
            for it in range((total + NT - 1) // NT):
                us = [w * 32 + lane + it * NT for lane in range(32)]
                active = sum(u < total for u in us)
                if not active:
                    continue
                for r in range(R):
                    loads, stores = [], []
                    for u in us:
                        if u >= total:
                            loads.append(None)
                            stores.append(None)
                            continue
                        j, b0 = u // G, (u % G) * V
                        k = j % Ns
                        loads.append(2 * at(j + r * NB, b0))
                        stores.append(2 * at((j - k) * R + k + r * Ns, b0))
                    minimum = (active * 16 + 127) // 128
                    assert _wavefronts(loads, 16) == minimum, (N, radices, R, "load")
                    assert _wavefronts(stores, 16) == minimum, (N, radices, R, "store")
        Ns *= R
    hs = ((N // 2 + 1) + 15) // 16 * 16
    in_row = lambda r: r * hs + (64 // RT) * (r // 4)
    R = radices[0]
    NB = N // R
    for w in range((NB * G + 31) // 32):
        us = [w * 32 + lane for lane in range(32) if w * 32 + lane < NB * G]
        for r in range(R):
            for q in range(V):
                for half in range(2):            # row 2b and row 2b + 1
                    addrs = []
                    for u in us:
                        j, b0 = u // G, (u % G) * V
                        idx = j + r * NB
                        k = N - idx if 2 * idx > N else idx
                        addrs.append(2 * (in_row(2 * (b0 + q) + half) + k))
                    addrs += [None] * (32 - len(addrs))
                    minimum = (len(us) * 8 + 127) // 128
                    assert _wavefronts(addrs, 8) == minimum, (N, radices, r, q, half)
