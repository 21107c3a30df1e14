"""The repair rule of the speculative BCPFW kernel (solve_spec.cu), modelled on
the host: for every interleaving its barriers allow, the repaired LMO equals
the exact one (the LMO of Sec. 3.1, eq. 7: argmin of grad_ij = C_ij + q_j over
j, ties to the smallest j).

What the kernel guarantees about the residual q each party reads, as versions
(version k = q after the first k block updates of the epoch; a pairwise step,
Alg. A.3, changes q in the two columns j*, v only):
  - producers take their segment minima for update u with every column at some
    version in [ver, u], ver = max(u - 4, 0) (they wait until update u - 5 is
    applied), each column independently (reads race with the chain's stores);
  - with three chain warps in rotation, the chain warp of u prepares after its
    own update u - 3 (so every column is at version >= u - 2), with the updates
    u - 2, u - 1 possibly half applied; the last-change marks of u - 4 and
    u - 3 are visible, those of u - 2 and u - 1 may or may not be; after the
    hand-over of u - 2 every column is at version >= u - 1; after that of
    u - 1 at version u;
  - with one chain warp, it prepares update u after applying u - 1 itself:
    every column is at version u and every mark is visible; there is no
    hand-over;
  - with the split chain, a preparer takes update u once u - 4 is published
    (every column at version >= u - 3; the marks of u - 4 and earlier
    visible, those of u - 3 .. u - 1 may or may not be), and the decider,
    which applied u - 3 .. u - 1 itself, merges their columns at version u.
The atom warp takes the away vertex (Alg. A.3: the atom with the largest
gradient) at versions in [ver, u] as well; the chain takes it again when one of
the row's atom columns changed since ver. The model draws all of these at
random (with many exact ties in C + q), runs the chain's steps in the kernel's
order and compares with the exact LMO and away vertex.
"""
import os
import re

import numpy as np
import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2103_05857_gb300",
                   "csrc", "solve_spec.cu")


def _kernel_source():
    with open(SRC) as fh:
        return fh.read()


LAG = int(re.search(r"constexpr int kSpecLag = (\d+);", _kernel_source()).group(1))  # producers' lead
# the chain-warp counts the kernel is built for
CHAINS = tuple(int(v) for v in re.search(r"static_assert\(CH == (\d+) \|\| CH == (\d+),",
                                         _kernel_source()).groups())


def _min(keys):
    return min(keys) if keys else (np.inf, 1 << 30)


def _chain_lmo(rng, u, C, q0, dec, deltas, nseg, atoms, CHAIN, drop=None):
    """The kernel's LMO and away vertex for update u under one random
    interleaving, with CHAIN chain warps (1 or 3) or the split chain
    ("split"). `drop` leaves one repair out (a planted mistake): "stale" (no
    segment recompute), "history" (no columns of the updates the preparing
    warp knows are published), "c3", "c2" or "c1" (no merge of the columns
    of u-3, u-2 or u-1), "atoms" (the atom warp's away statistics always
    kept)."""
    if CHAIN == "split":
        return _split_lmo(rng, u, C, q0, dec, deltas, nseg, atoms, drop)
    n = len(C)
    seg_of = (np.arange(n) // 4) % nseg  # quads interleaved over the producer warps

    def value(j, k):  # grad at column j with q at version k
        return C[j] + q0[j] + sum(deltas[w][j] for w in range(k) if dec[w] is not None and j in dec[w])

    ver = u - LAG if u > LAG else 0
    # atom warp: away vertex (largest gradient over the row's atoms, ties to
    # the smallest column) with every atom column at a version in [ver, u]
    away = min((-value(j, int(rng.integers(ver, u + 1))), j) for j in atoms)[1]
    # producers: per column a version in [ver, u]
    cand = {}
    for s in range(nseg):
        cols = np.nonzero(seg_of == s)[0]
        if len(cols) == 0:  # (the kernel pads: such a segment never wins)
            continue
        vals = [(value(j, int(rng.integers(ver, u + 1))), int(j)) for j in cols]
        cand[s] = min(vals)
    # prepare: after the warp's own update u - CHAIN (and the wait for u - CHAIN - 1
    # within it): marks up to u - CHAIN visible, the later ones maybe; every
    # column at a version in [u - CHAIN + 1, u]
    lo = max(u - CHAIN + 1, 0)
    visible = {w for w in range(u) if w <= u - CHAIN or rng.random() < 0.5}

    def lastmod(j):
        ws = [w for w in range(u) if w in visible and dec[w] is not None and j in dec[w]]
        return max(ws) if ws else -1

    def prep_value(j):
        return value(j, int(rng.integers(lo, u + 1)))

    keys = []
    for s in cand:
        val, cj = cand[s]
        if lastmod(cj) >= ver and drop != "stale":  # stale segment: recomputed now
            cols = np.nonzero(seg_of == s)[0]
            keys.append(min((prep_value(j), int(j)) for j in cols))
        else:
            keys.append((val, cj))
    for w in range(u - CHAIN, u - LAG - 1, -1):  # columns of the updates before the hand-over
        if w >= ver and w >= 0 and dec[w] is not None and drop != "history":
            keys.extend((prep_value(c), c) for c in dec[w])
    olddirty = any(lastmod(j) >= ver for j in atoms)
    fk, js = _min(keys)
    pj = js
    # hand-over 1: update u-2 is applied, u-1 may be half applied
    c2 = dec[u - 2] if CHAIN == 3 and u >= 2 and dec[u - 2] is not None and drop != "c2" else ()
    redo = pj in c2
    for c in c2:
        k = value(c, int(rng.integers(max(u - 1, 0), u + 1)))
        if (k, c) < (fk, js):
            fk, js = k, c
    pj2 = js
    # hand-over 2: update u-1 is applied, every column at version u
    c1 = dec[u - 1] if CHAIN == 3 and u >= 1 and dec[u - 1] is not None and drop != "c1" else ()
    redo = redo or pj2 in c1
    if redo:
        fk, js = min((value(j, u), j) for j in range(n))
    else:
        for c in c1:
            k = value(c, u)
            if (k, c) < (fk, js):
                fk, js = k, c
    # away statistics: taken again when an atom column changed since ver
    hit = any(j in c1 or j in c2 for j in atoms)
    if (olddirty or hit) and drop != "atoms":
        away = min((-value(j, u), j) for j in atoms)[1]
    return js, away, value


def _split_lmo(rng, u, C, q0, dec, deltas, nseg, atoms, drop=None):
    """The split chain: the preparer of u starts once u - 4 is published; the
    decider merges the columns of u - 3, u - 2, u - 1 at the current
    residual and takes the full LMO when the prepared minimum sits on one of
    them."""
    n = len(C)
    seg_of = (np.arange(n) // 4) % nseg

    def value(j, k):
        return C[j] + q0[j] + sum(deltas[w][j] for w in range(k) if dec[w] is not None and j in dec[w])

    ver = u - LAG if u > LAG else 0
    away = min((-value(j, int(rng.integers(ver, u + 1))), j) for j in atoms)[1]
    cand = {}
    for s in range(nseg):
        cols = np.nonzero(seg_of == s)[0]
        if len(cols) == 0:
            continue
        cand[s] = min((value(j, int(rng.integers(ver, u + 1))), int(j)) for j in cols)
    lo = max(u - 3, 0)
    visible = {w for w in range(u) if w <= u - 4 or rng.random() < 0.5}

    def lastmod(j):
        ws = [w for w in range(u) if w in visible and dec[w] is not None and j in dec[w]]
        return max(ws) if ws else -1

    def prep_value(j):
        return value(j, int(rng.integers(lo, u + 1)))

    keys = []
    for s in cand:
        val, cj = cand[s]
        if lastmod(cj) >= ver and drop != "stale":
            cols = np.nonzero(seg_of == s)[0]
            keys.append(min((prep_value(j), int(j)) for j in cols))
        else:
            keys.append((val, cj))
    for w in range(u - 4, u - LAG - 1, -1):
        if w >= ver and w >= 0 and dec[w] is not None and drop != "history":
            keys.extend((prep_value(c), c) for c in dec[w])
    olddirty = any(lastmod(j) >= ver for j in atoms)
    pk, pj = _min(keys)
    merged = []
    for back, name in ((3, "c3"), (2, "c2"), (1, "c1")):
        w = u - back
        if w >= 0 and dec[w] is not None and drop != name:
            merged.extend(dec[w])
    if pj in merged:
        fk, js = min((value(j, u), j) for j in range(n))
    else:
        fk, js = min([(pk, pj)] + [(value(c, u), c) for c in merged])
    if (olddirty or any(j in merged for j in atoms)) and drop != "atoms":
        away = min((-value(j, u), j) for j in atoms)[1]
    return js, away, value


def _mismatches(seed, trials, chain, drop=None):
    rng = np.random.default_rng(seed)
    bad = 0
    for _ in range(trials):
        n = int(rng.integers(8, 72))
        nseg = int(rng.integers(1, 5))
        u = int(rng.integers(0, 14))
        # small integers: many exact ties between columns
        C = rng.integers(0, 6, n).astype(float)
        q0 = rng.integers(-3, 4, n).astype(float)
        dec, deltas = [], []
        for w in range(u):
            if rng.random() < 0.8:
                a, b = (int(v) for v in rng.choice(n, 2, replace=False))
                dec.append((a, b))
                d = np.zeros(n)
                d[a] = float(rng.integers(1, 4))    # mass moved onto j*: its q grows
                d[b] = -float(rng.integers(1, 4))   # and off v: its q drops
                deltas.append(d)
            else:
                dec.append(None)
                deltas.append(np.zeros(n))
        atoms = [int(j) for j in rng.choice(n, int(rng.integers(1, 6)), replace=False)]
        js, away, value = _chain_lmo(rng, u, C, q0, dec, deltas, nseg, atoms, chain, drop)
        exact = min((value(j, u), j) for j in range(n))[1]
        exact_away = min((-value(j, u), j) for j in atoms)[1]
        bad += (js != exact) or (away != exact_away)
    return bad


def test_model_follows_the_kernel_constants():
    """The kernel is built for one chain warp or three in rotation; with
    three the hand-over takes the columns of u-2 and u-1, the other changed
    columns are the ones of u-CHAIN .. u-LAG."""
    assert CHAINS == (1, 3) and LAG >= max(CHAINS)
    with open(SRC) as fh:
        src = fh.read()
    # the split chain's preparer waits for update u - 4, the decider merges u-3 .. u-1
    assert "const int p4 = u - 4;" in src and "c3[2]" in src


@pytest.mark.parametrize("chain", [1, 3, "split"])
def test_speculative_repair_gives_the_exact_lmo(chain):
    assert _mismatches(2103, 4000, chain) == 0


@pytest.mark.parametrize("chain", [1, 3, "split"])
def test_each_repair_is_needed(chain):
    """Leaving out any one repair makes the model return wrong LMOs on the
    same kind of draws, so the test above has something to catch."""
    drops = {3: ("stale", "history", "c2", "c1", "atoms"), 1: ("stale", "history", "atoms"),
             "split": ("stale", "history", "c3", "c2", "c1", "atoms")}[chain]
    for drop in drops:
        assert _mismatches(7, 1500, chain, drop) > 0, drop
