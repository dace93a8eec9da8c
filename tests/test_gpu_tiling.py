"""Tile shapes never change results: every vertex sums its element
contributions in the same order whatever the block rows, z-chunk or tile
class (wide 32-column tiles, narrow 8-column tiles for the leftover columns).
Operator applies and whole V-cycles under hand-set and autotuned shapes are
compared bit for bit with the default shape, and the autotuner's cache file
is checked to reproduce its choices."""
import pytest
import torch

from synth import random_vector, sphere_sinkers

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2511_13109_gb300")
DEV = torch.device("cuda:0")

MODES = (1, 2, 3, 4)  # residual, first / later Chebyshev step, pre-smoothing step


def _ctx(N, prec):
    p = sphere_sinkers(N, 4, 0.11, 0.02, 1e4, seed=77)
    c = pkg.Context(N, None, prec, device=DEV)
    c.prepare(torch.from_numpy(p.eta).to(DEV), 10.0)
    return c


def _shapes(prec):
    rows = (8, 12, 16) if prec == pkg.MIXED else (8,)
    return [(by, z) for by in rows for z in (0, 1, 3, 7)]


# N = 16: finest level has 32 cubes per axis (one wide and one narrow strip);
# N = 24: 48 cubes per axis (one wide strip and three narrow ones)
@pytest.mark.parametrize("N", [16, 24])
@pytest.mark.parametrize("prec", [pkg.FP64, pkg.MIXED])
def test_apply_independent_of_tile_shape(N, prec):
    c = _ctx(N, prec)
    dtype = pkg.F32 if prec == pkg.MIXED else pkg.F64
    td = torch.float32 if prec == pkg.MIXED else torch.float64
    for level in range(2, c.L + 1):
        x = torch.from_numpy(random_vector(3 * c.V[level], 3 + level)).to(DEV).to(td)
        ref = c.apply(level, x, dtype=dtype).clone()
        for by, z in _shapes(prec):
            c.set_tile_config(level, 0, by, z)
            y = c.apply(level, x, dtype=dtype)
            assert torch.equal(y, ref), (level, by, z)
        c.set_tile_config(level, 0, 8, 0)


@pytest.mark.parametrize("prec", [pkg.FP64, pkg.MIXED])
def test_vcycle_independent_of_tile_shape(prec):
    c = _ctx(16, prec)
    r = torch.from_numpy(random_vector(3 * c.V[c.L], 11)).to(DEV)
    ref = c.vcycle(r).clone()
    for i, (by, z) in enumerate(_shapes(prec)):
        for level in range(2, c.L + 1):
            for m in MODES:
                # vary the shape across levels and modes as well
                by_l = _shapes(prec)[(i + level + m) % len(_shapes(prec))][0]
                c.set_tile_config(level, m, by_l, z)
        z_out = c.vcycle(r)
        assert torch.equal(z_out, ref), (by, z)


def test_autotune_cache_round_trip(tmp_path):
    cache = str(tmp_path / "tiles.txt")
    c = _ctx(16, pkg.MIXED)
    r = torch.from_numpy(random_vector(3 * c.V[c.L], 5)).to(DEV)
    ref = c.vcycle(r).clone()
    tuned = c.autotune(2, cache)
    assert set(tuned) == {(l, m) for l in range(2, c.L + 1) for m in MODES}
    assert all(by in (8, 12, 16) and z >= 0 for by, z in tuned.values())
    assert torch.equal(c.vcycle(r), ref)
    # a second context reads the same choices back from the cache file
    c2 = _ctx(16, pkg.MIXED)
    assert c2.autotune(2, cache) == tuned
    assert torch.equal(c2.vcycle(r), ref)
