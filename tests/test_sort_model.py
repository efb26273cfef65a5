"""CPU model of the radix sort's scatter step (csrc/sort.cu): each 4,096-
element tile is sorted by digit in shared memory before it is written out.
Warp w of the block owns elements [512 w, 512 w + 512) of the tile (lane l:
512 w + 32 r + l for r = 0..15) and ranks each element among its warp's
earlier elements of the same digit (the __match_any_sync group below the
lane plus the warp's running count); the warps' counts, summed in warp
order, give each warp its first slot per digit in the sorted tile; a tile
slot p of digit d goes to the output slot gbase[d] + (p - lbase[d]).

The model runs those index computations on random keys with many ties and
ragged last tiles and checks that two passes (the lists' 16-bit keys) give
exactly a stable sort, that no shared-memory slot or output slot is written
twice or falls outside its tile, and that the kernel source still states
the steps the model follows."""
import os

import numpy as np
import pytest

K_TILE, WARPS, DIGITS = 4096, 8, 256
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1706_01449_gb300", "csrc",
                   "sort.cu")


def scatter_pass(keys, vals, shift):
    n = len(keys)
    nb = (n + K_TILE - 1) // K_TILE
    digit = (keys >> shift) & 0xFF
    # hist + scan: per (digit, tile) counts, row-exclusive over tiles, digit bases
    hist = np.zeros((DIGITS, nb), np.int64)
    for b in range(nb):
        np.add.at(hist[:, b], digit[b * K_TILE:(b + 1) * K_TILE], 1)
    dbase = np.concatenate([[0], np.cumsum(hist.sum(1))[:-1]])
    rowpre = np.concatenate([np.zeros((DIGITS, 1), np.int64), np.cumsum(hist, 1)[:, :-1]], 1)
    k_out = np.full(n, -1, np.int64)
    v_out = np.full(n, -1, np.int64)
    for b in range(nb):
        lo, ln = b * K_TILE, min(K_TILE, n - b * K_TILE)
        cnt = np.zeros((WARPS, DIGITS), np.int64)
        rank = np.zeros(K_TILE, np.int64)
        for w in range(WARPS):
            for r in range(16):
                idx = [w * 512 + 32 * r + l for l in range(32)]
                ds = [int(digit[lo + i]) if i < ln else DIGITS for i in idx]  # dead lanes: a digit of their own
                for l, i in enumerate(idx):
                    if i < ln:
                        below = sum(1 for l2 in range(l) if ds[l2] == ds[l])  # popc(peers & lanes below)
                        rank[i] = cnt[w][ds[l]] + below
                for d in set(x for x in ds if x != DIGITS):
                    cnt[w][d] += ds.count(d)
        tc = cnt.sum(0)
        lbase = np.concatenate([[0], np.cumsum(tc)[:-1]])
        gbase = dbase + rowpre[:, b]
        wbase = np.zeros((WARPS, DIGITS), np.int64)
        run = lbase.copy()
        for w in range(WARPS):
            wbase[w] = run
            run = run + cnt[w]
        skeys = np.full(K_TILE, -1, np.int64)
        sidx = np.full(K_TILE, -1, np.int64)
        for i in range(ln):
            pos = wbase[i // 512][digit[lo + i]] + rank[i]
            assert 0 <= pos < ln and skeys[pos] == -1
            skeys[pos], sidx[pos] = keys[lo + i], i
        for p in range(ln):
            d = (skeys[p] >> shift) & 0xFF
            q = gbase[d] + (p - lbase[d])
            assert 0 <= q < n and k_out[q] == -1
            k_out[q], v_out[q] = skeys[p], vals[lo + sidx[p]]
    return k_out, v_out


@pytest.mark.parametrize("n", [1, 4095, 4096, 9000, 12289])
def test_two_passes_are_a_stable_sort(n):
    rng = np.random.default_rng(n)
    keys = rng.integers(0, 2 ** 16, n).astype(np.int64)
    keys[::5] = keys[0]  # many equal keys
    keys[1::7] &= 0xFF00  # many equal low digits
    vals = np.arange(n)
    k, v = keys, vals
    for shift in (0, 8):
        k, v = scatter_pass(k, v, shift)
    order = np.argsort(keys, kind="stable")
    assert (k == keys[order]).all() and (v == vals[order]).all()


def test_model_matches_the_kernel_source():
    src = open(SRC).read()
    assert "constexpr int kPerWarp = kTile / kScatterWarps;  // 512" in src
    assert "const int i = w * kPerWarp + 32 * r + lane;" in src
    assert "srank[r][threadIdx.x] = (uint16_t)(before + __popc(below));" in src
    assert "const uint32_t pos = cnt[w][(key[r] >> shift) & 0xFFu] + srank[r][threadIdx.x];" in src
    assert "const int64_t q = off + (int64_t)(gbase[dd] + ((uint32_t)p - lbase[dd]));" in src
    assert "vals_out[q] = vals_in[off + lo + sidx[p]];" in src
