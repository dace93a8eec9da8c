"""Host-side tiling of the stencil kernels (agca_stencil_tiles): the wide and
narrow tiles partition every vertex plane, and the z-chunks partition the
vertex planes, for every grid size the library accepts and every tile shape.
The kernels' results do not depend on the shape (checked bit for bit on the
GPU); this checks the ownership the kernels rely on, on the CPU."""
import numpy as np
import pytest

from paper_2511_13109_gb300 import agca


def _owned(n, by, zch):
    g = agca.stencil_tiles(n, by, zch)
    nv = n + 1
    cnt = np.zeros((nv, nv), dtype=np.int32)
    # wide tiles: 32 x by threads, own columns x0 .. x0 + 30, rows y0 .. y0 + by - 2
    for t in range(g["gxw"] * g["gyw"]):
        x0, y0 = (t % g["gxw"]) * 31, (t // g["gxw"]) * (by - 1)
        cnt[y0:min(y0 + by - 1, nv), x0:min(x0 + 31, nv)] += 1
    # narrow tiles: 8 x 4by threads, own columns x0 .. x0 + 6, rows y0 .. y0 + 4by - 2
    byn = 4 * by
    for u in range(g["gxn"] * g["gyn"]):
        x0, y0 = g["x0n"] + (u % g["gxn"]) * 7, (u // g["gxn"]) * (byn - 1)
        cnt[y0:min(y0 + byn - 1, nv), x0:min(x0 + 7, nv)] += 1
    return g, cnt


@pytest.mark.parametrize("by", [8, 12, 16])
def test_tiles_partition_every_plane(by):
    for n in list(range(2, 130)) + [192, 256, 384, 512, 1024]:
        for zch in (0, 1, 3, 7, 64, 5000):
            g, cnt = _owned(n, by, zch)
            assert (cnt == 1).all(), (n, by, zch)
            nv = n + 1
            assert 1 <= g["zch"] <= nv and g["gz"] * g["zch"] >= nv > (g["gz"] - 1) * g["zch"], (n, zch, g)
            if zch > 0:
                assert g["zch"] == min(zch, nv)
            # the narrow strips only take columns the wide strips leave
            assert g["x0n"] == 31 * g["gxw"] and (g["gxn"] == 0 or g["x0n"] < nv)


def test_tiles_reject_bad_arguments():
    for args in ((0, 8, 0), (1025, 8, 0), (64, 10, 0), (64, 8, -1)):
        with pytest.raises(agca.AgcaError):
            agca.stencil_tiles(*args)
