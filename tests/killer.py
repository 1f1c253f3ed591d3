"""An adversarial ("killer") input for the GPU sort's sampled pivots (Section V.B's
worst case against Section V.C's randomised samples), used by the depth-guard tests.

The sampler is seeded and deterministic, so an adversary that knows the seed can
compute every sample position.  This one also models where the partition kernel puts
every element in the deterministic look-back reservation mode, and so follows the
largest segment down the levels.  It assigns values lazily (McIlroy's "antiquicksort"
idea): every element starts undecided and larger than every decided one; at each level
the undecided elements the pivot sample reads get the smallest values still free, so
the sampled median sits among the segment's smallest elements and the large child
loses only a few dozen elements per level.  The undecided elements get the remaining
values, shuffled, at the end.

Test-side only: it models the CUDA path (sample positions, tile geometry, staging
order) and is neither part of the product nor shared with the oracle.  The GPU test
checks the model itself against the pivot kernel's reported sample positions.
"""
from __future__ import annotations

import numpy as np

M64 = (1 << 64) - 1


def _mix64(z: int) -> int:
    """SplitMix64 finaliser (the published constants)."""
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def sample_positions(b: int, e: int, samples: int, seed: int) -> list[int]:
    """Positions the pivot kernel samples in segment [b, e): stratum k of S strata,
    offset by a seeded hash with multiply-shift range reduction (segments < 2^32)."""
    m = e - b
    S = min(samples, 63, m)
    if S % 2 == 0:
        S -= 1
    S = max(S, 1)
    q, r = m // S, m % S
    out = []
    for k in range(S):
        a0 = q * k + (r * k) // S
        a1 = q * (k + 1) + (r * (k + 1)) // S
        w = a1 - a0
        z = _mix64((seed ^ ((b * 0x9E3779B97F4A7C15) & M64) ^ ((e * 0xC2B2AE3D27D4EB4F) & M64)
                    ^ (((k + 1) * 0x165667B19E3779F9) & M64)) & M64)
        out.append(b + a0 + (((z >> 32) * w) >> 32))
    return out


def partition_layout(ids: np.ndarray, b: int, e: int, cls: np.ndarray, block: int,
                     items: int, vec: int, vec_off: int = 0):
    """Model of one look-back-mode partition of segment [b, e) whose positions hold the
    element ids `ids` (len e - b); cls[id] is -1 (< p), 0 (= p) or +1 (> p).  Tiles of
    block * items elements start at the vector boundary at or below b; thread t of a
    tile holds vectors k * block + t; a thread's < p keys are staged in key order after
    those of lower threads (permuted by lane & (lowest set bit of items) - 1 when all its
    keys go to one run), > p keys from the back; tile runs follow in tile order, < p from
    b upward, > p from e downward.  Returns (ids of the < p child, ids of the > p child)."""
    tile = block * items
    s0 = b - ((b + vec_off) & (vec - 1))
    nt = (e - s0 + tile - 1) // tile
    i = np.arange(items)
    th = np.arange(block)
    k, j = i // vec, i % vec
    pos = (s0 + np.arange(nt)[:, None, None] * tile
           + (k[None, None, :] * block + th[None, :, None]) * vec + j[None, None, :])
    valid = (pos >= b) & (pos < e)
    idx = np.where(valid, pos - b, 0)
    c = np.where(valid, cls[ids[idx]], 0)
    lt, gt = valid & (c < 0), valid & (c > 0)
    clt, cgt = lt.sum(2), gt.sum(2)
    tex_lt, tex_gt = np.cumsum(clt, 1) - clt, np.cumsum(cgt, 1) - cgt
    rk_lt = np.cumsum(lt, 2) - lt
    rk_gt = np.cumsum(gt, 2) - gt
    krot = (items & -items) - 1
    perm = i[None, None, :] ^ ((th & 31) & krot)[None, :, None]
    slot_lt = tex_lt[..., None] + np.where((clt == items)[..., None], perm, rk_lt)
    x_gt = tex_gt[..., None] + np.where((cgt == items)[..., None], perm, rk_gt)
    tlt, tgt = clt.sum(1), cgt.sum(1)
    ex_lt, ex_gt = np.cumsum(tlt) - tlt, np.cumsum(tgt) - tgt
    nlt, ngt = int(tlt.sum()), int(tgt.sum())
    left = np.empty(nlt, dtype=ids.dtype)
    right = np.empty(ngt, dtype=ids.dtype)
    left[(ex_lt[:, None, None] + slot_lt)[lt]] = ids[idx[lt]]
    right[(ngt - 1 - (ex_gt[:, None, None] + x_gt))[gt]] = ids[idx[gt]]
    return left, right


def killer_int32(n: int, seed: int, samples: int = 31, block: int = 192, items: int = 24,
                 small: int = 4096, levels: int | None = None, shuffle_seed: int = 7):
    """int32 keys (a permutation of -n/2 .. n/2 - 1) on which the look-back-mode sort
    with this sampler seed, sample count, partition shape (block x items, 16-byte
    vectors) and on-chip threshold keeps one segment above the threshold for `levels`
    levels (default: the whole array's depth bound 2 ceil(log2(n + 1)) + 8).  Returns
    (keys, the modelled sizes of the large segment level by level)."""
    vec = 4
    if levels is None:
        lg = 1
        while (1 << lg) < n + 1:
            lg += 1
        levels = 2 * lg + 8
    val = np.full(n, -1, dtype=np.int64)          # -1: undecided (larger than all decided)
    nxt = 0                                       # smallest value still free
    ids = np.arange(n, dtype=np.int64)            # element at each position of the segment
    b, e = 0, n
    sizes = []
    for _ in range(levels):
        if e - b <= small:
            break
        sizes.append(e - b)
        pos = sample_positions(b, e, samples, seed)
        sid = ids[np.array(pos) - b]
        for x in sid:                             # the samples read undecided: decide small
            if val[x] < 0:
                val[x] = nxt
                nxt += 1
        sv = np.sort(val[sid])
        p = sv[(len(sv) - 1) // 2]
        v = val[ids]
        cls = np.zeros(n, dtype=np.int8)
        cls[ids] = np.where(v < 0, 1, np.sign(v - p)).astype(np.int8)
        left, right = partition_layout(ids, b, e, cls, block, items, vec)
        ids = right
        b, e = e - len(right), e
    rest = np.flatnonzero(val < 0)
    val[rest] = nxt + np.random.default_rng(shuffle_seed).permutation(len(rest))
    return (val - n // 2).astype(np.int32), sizes
