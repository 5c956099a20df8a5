"""Pins of the mesh-generation oracle (Sec. 3.1, Eq. ref_crit): Morton keys
against a string interleaving of the bits, refinement closed forms, a per-cell
brute force, and the host mesh generator's refinement of a base level."""
import itertools

import numpy as np
import pytest

from oracle.meshgen import morton_key, morton_sorted, refine_level
from paper_1911_10228_gb300.inputs import box_coords, cell_centres, refine_mesh, torus


def _key_by_strings(x, y, z):
    bx, by, bz = (format(v + (1 << 20), "021b") for v in (x, y, z))
    return int("".join(a + b + c for a, b, c in zip(bx, by, bz)), 2)


def test_morton_key_is_the_bit_interleaving():
    rng = np.random.default_rng(0)
    for x, y, z in rng.integers(-(1 << 19), 1 << 19, size=(200, 3)).tolist() + [[0, 0, 0], [-1, -1, -1]]:
        assert morton_key(x, y, z) == _key_by_strings(x, y, z)


def test_morton_order_of_a_cube_and_across_zero():
    cube = [tuple(c) for c in itertools.product((0, 1), repeat=3)]
    assert [tuple(c) for c in morton_sorted(reversed(cube)).tolist()] == cube   # z fastest, then y, then x
    # monotone along each axis, negative coordinates first
    assert morton_key(-1, 0, 0) < morton_key(0, 0, 0) < morton_key(1, 0, 0)
    assert morton_key(0, 0, -5) < morton_key(0, 0, 3)


def _field(n, N=4, seed=0):
    return np.random.default_rng(seed).standard_normal((n, N, N, N))


def test_zero_source_and_threshold_edges():
    c = box_coords(2)
    flags, ch, buf = refine_level(c, np.zeros((8, 4, 4, 4)), 0.1)
    assert not flags.any() and len(ch) == 0 and len(buf) == 0
    f = np.zeros((8, 4, 4, 4))
    f[3, 1, 2, 3] = 1.0
    f[5, 0, 0, 0] = -0.5
    assert refine_level(c, f, 1.0)[0].sum() == 0                     # strict: the maximum never exceeds itself
    assert refine_level(c, f, 0.5)[0].tolist() == [0, 0, 0, 1, 0, 0, 0, 0]   # |-0.5| is not > 0.5 * 1
    assert refine_level(c, f, 0.4999)[0].tolist() == [0, 0, 0, 1, 0, 1, 0, 0]


def test_single_block_closed_forms():
    flags, ch, buf = refine_level([[3, -2, 7]], _field(1), 0.5)
    assert flags.tolist() == [True]
    assert {tuple(v) for v in ch.tolist()} == {(6 + a, -4 + b, 14 + d) for a in (0, 1) for b in (0, 1) for d in (0, 1)}
    assert len(buf) == 26 and {tuple(v) for v in buf.tolist()} == {
        (3 + a, -2 + b, 7 + d) for a in (-1, 0, 1) for b in (-1, 0, 1) for d in (-1, 0, 1) if (a, b, d) != (0, 0, 0)}
    # two face-adjacent refined blocks: the union of two 3^3 neighbourhoods minus the pair
    flags, ch, buf = refine_level([[0, 0, 0], [1, 0, 0]], np.ones((2, 4, 4, 4)), 0.5)
    assert flags.all() and len(ch) == 16 and len(buf) == 4 * 3 * 3 - 2
    # the centre of a full 3^3 level: its neighbours exist, nothing to add
    c = box_coords(3)
    f = np.zeros((27, 4, 4, 4))
    f[13] = 1.0
    flags, ch, buf = refine_level(c, f, 0.5)
    assert flags.sum() == 1 and flags[13] and len(ch) == 8 and len(buf) == 0
    for lst in (ch, buf):
        keys = [morton_key(*v) for v in lst.tolist()]
        assert keys == sorted(keys) and len(set(keys)) == len(keys)


def test_brute_force_on_random_levels():
    rng = np.random.default_rng(5)
    for trial in range(6):
        box = box_coords(5) + rng.integers(-20, 20, size=3)
        c = box[rng.choice(len(box), size=int(rng.integers(1, 60)), replace=False)]
        f = rng.standard_normal((len(c), 4, 4, 4)) * rng.uniform(0, 3, size=(len(c), 1, 1, 1))
        rel = float(rng.uniform(0.1, 0.9))
        flags, ch, buf = refine_level(c, f, rel)
        # per-cell test of the criterion
        thr = rel * np.abs(f).max()
        want = np.array([any(abs(v) > thr for v in blk.ravel()) for blk in f])
        assert flags.tolist() == want.tolist()
        # buffer by scanning the bounding box for cells adjacent to a refined block
        ref = {tuple(v) for v, w in zip(c.tolist(), want) if w}
        lvl = {tuple(v) for v in c.tolist()}
        lo, hi = c.min(axis=0) - 1, c.max(axis=0) + 1
        scan = set()
        for x in range(lo[0], hi[0] + 1):
            for y in range(lo[1], hi[1] + 1):
                for z in range(lo[2], hi[2] + 1):
                    if (x, y, z) in lvl:
                        continue
                    if any(max(abs(x - r[0]), abs(y - r[1]), abs(z - r[2])) == 1 for r in ref):
                        scan.add((x, y, z))
        assert {tuple(v) for v in buf.tolist()} == scan
        assert {tuple(v) for v in ch.tolist()} == {(2 * r[0] + a, 2 * r[1] + b, 2 * r[2] + d)
                                                  for r in ref for a in (0, 1) for b in (0, 1) for d in (0, 1)}


@pytest.mark.parametrize("thr", [1e-3, 0.3])
def test_matches_the_host_generator_on_a_base_level(thr):
    """The host mesh generator refines a base level by the same criterion and
    closes it with the same buffer (a base level has no coarser level)."""
    N, h0 = 4, 1.0 / 24
    src = lambda x: torus(x, (0.5, 0.5, 0.5), 0.25, 0.05)
    base = box_coords(6)
    prob = refine_mesh(src, base, N, h0, 2, thr)
    f = src(cell_centres(base, N, h0))
    flags, ch, buf = refine_level(base, f, thr)
    assert {tuple(v) for v in ch.tolist()} == {tuple(v) for v in np.asarray(prob.coords[1]).tolist()}
    added = {tuple(v) for v in np.asarray(prob.coords[0]).tolist()} - {tuple(v) for v in base.tolist()}
    assert {tuple(v) for v in buf.tolist()} == added
