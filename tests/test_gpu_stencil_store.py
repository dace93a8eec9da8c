"""Stencil storage of the stored-Galerkin part of the coarse operators
(Remark 5, Eq. 5.8) against the oracle: the touched vertices (vertices of
flagged elements) bit-exact and numbered in ascending order, every touched
interior vertex's 15 x 3 x 3 couplings to 1e-12 of the oracle's assembly of
the flagged elements' matrices, and the levels' applies (DCA part matrix-free
plus stencils) to 1e-12 (FP64) / 1e-5 (FP32)."""
import numpy as np
import pytest
import torch

from oracle import agca as oagca
from synth import random_vector, sphere_sinkers

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2511_13109_gb300")
DEV = torch.device("cuda:0")


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_stencils_match_oracle(prec):
    N, L = 8, 3
    p = sphere_sinkers(N, 3, 0.15, 0.02, 1e4)
    H = oagca.Hierarchy(N, L, p.eta, 10.0)
    c = pkg.Context(N, L, pkg.FP64 if prec == "fp64" else pkg.MIXED, device=DEV)
    c.prepare(torch.from_numpy(p.eta).to(DEV), 10.0)
    for l in range(1, L):
        m = H.mesh[l]
        assert len(H.flist[l]) > 0
        touched = np.zeros(m.nv, dtype=bool)
        touched[m.tets[H.flist[l]].ravel()] = True
        sidx = c.level_data(l, pkg.FIELD_SIDX).cpu().numpy()
        assert np.array_equal(sidx >= 0, touched)
        assert np.array_equal(sidx[touched], np.arange(touched.sum()))
        info = c.level_info(l)
        assert info.n_stencil == touched.sum()
        got = c.level_data(l, pkg.FIELD_STENCIL).cpu().numpy().reshape(-1, 15, 3, 3)
        ref = oagca.stencil_blocks(H, l, oagca.flagged_operator(H, l))
        inner = m.interior
        n1 = m.n + 1
        scale = np.abs(ref).max()
        for o, d in enumerate(oagca.KUHN_OFFSETS):
            nb = m.ijk + d
            ok = ((nb >= 1) & (nb <= m.n - 1)).all(axis=1)   # interior neighbour: the Dirichlet mask keeps it
            rows = np.nonzero(touched & inner & ok)[0]
            diff = np.abs(got[sidx[rows], o] - ref[rows, o]).max() if len(rows) else 0.0
            assert diff <= 1e-12 * scale, (l, o, diff)
        assert n1 ** 3 == m.nv
    for l in range(1, L + 1):
        x = random_vector(3 * c.V[l], 80 + l)
        if prec == "fp64":
            y = c.apply(l, torch.from_numpy(x).to(DEV)).cpu().numpy()
            ref = H.A[l] @ (x * H.mask[l])
            assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max(), l
        else:
            x32 = x.astype(np.float32)
            y = c.apply(l, torch.from_numpy(x32).to(DEV), dtype=pkg.F32).cpu().numpy().astype(np.float64)
            ref = H.A[l] @ (x32.astype(np.float64) * H.mask[l])
            assert np.abs(y - ref).max() <= 1e-5 * np.abs(ref).max(), l
