"""Batched solves (agca_batch_*): problems of uneven sizes in one lockstep
MINRES with persistent stencil launches, against the same problems solved one
by one and against the oracle."""
import numpy as np
import pytest
import torch

from oracle import agca as oagca
from oracle import stokes as ostokes
from synth import batch_problems, random_vector, sphere_sinkers

pytestmark = pytest.mark.gpu

pkg = pytest.importorskip("paper_2511_13109_gb300")
DEV = torch.device("cuda:0")


def _problems():
    # uneven sizes and depths (levels 2, 3, 3, 2), different sphere fields
    out = []
    for k, (N, dr) in enumerate(((4, 1e2), (8, 1e4), (6, 1e3), (4, 1e6))):
        out.append(sphere_sinkers(N, 1 + k, 0.12 + 0.02 * k, 0.03, dr, seed=100 + k))
    return out


@pytest.fixture(scope="module", params=[pkg.FP64, pkg.MIXED])
def batch(request):
    probs = _problems()
    s = torch.cuda.Stream(device=DEV)
    with torch.cuda.stream(s):
        b = pkg.Batch([p.N for p in probs], request.param, device=DEV, stream=s)
        b.prepare([torch.from_numpy(p.eta).to(DEV) for p in probs], 10.0)
    s.synchronize()
    return request.param, probs, b, s


def test_batched_vcycle_equals_single(batch):
    prec, probs, b, s = batch
    with torch.cuda.stream(s):
        rs = [torch.from_numpy(random_vector(3 * c.V[c.L], 5 + i)).to(DEV) for i, c in enumerate(b.contexts)]
        zs = b.vcycle(rs)
        for i, p in enumerate(probs):
            c = pkg.Context(p.N, b.contexts[i].L, prec, device=DEV)
            c.prepare(torch.from_numpy(p.eta).to(DEV), 10.0)
            ref = c.vcycle(rs[i])
            torch.cuda.synchronize()
            assert torch.equal(zs[i], ref), i
    s.synchronize()


def test_batched_solve(batch):
    prec, probs, b, s = batch
    with torch.cuda.stream(s):
        bs = [b.load_vector(i, torch.from_numpy(p.fbar.ravel()).to(DEV)) for i, p in enumerate(probs)]
        xs, its, rel = b.solve(bs, 1e-11, 20000)
    s.synchronize()
    assert all(r <= 1e-11 for r in rel), rel
    for i, p in enumerate(probs):
        L = b.contexts[i].L
        H = oagca.Hierarchy(p.N, L, p.eta, 10.0)
        S = ostokes.Stokes(H)
        xd = S.direct(bs[i].cpu().numpy())
        xg = xs[i].cpu().numpy()
        assert np.linalg.norm(xg - xd) <= 1e-8 * np.linalg.norm(xd), (i, its[i], rel[i])


def test_batched_zero_rhs_problem(batch):
    """A problem with b = 0 is skipped (x = 0) while the others converge."""
    prec, probs, b, s = batch
    with torch.cuda.stream(s):
        bs = [b.load_vector(i, torch.from_numpy(p.fbar.ravel()).to(DEV)) for i, p in enumerate(probs)]
        bs[2].zero_()
        xs, its, rel = b.solve(bs, 1e-9, 20000)
    s.synchronize()
    assert its[2] == 0 and float(xs[2].abs().max()) == 0.0
    assert all(rel[i] <= 1e-9 for i in (0, 1, 3))


def test_batch_config_generator_sizes():
    """The 24-problem batch recipe: sizes 32/48/64, 8 of each, seeded."""
    params = batch_problems(generate=False)
    assert sorted(p["N"] for p in params) == [32] * 8 + [48] * 8 + [64] * 8
    assert all(0.05 <= p["radius"] <= 0.15 for p in params)
    assert {int(round(np.log10(p["dr"]))) for p in params} <= {2, 3, 4, 5, 6}
    assert [pkg.default_levels(N) for N in (32, 48, 64)] == [5, 5, 6]
