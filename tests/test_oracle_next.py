"""Pins of the oracle's parts for the next rows: the three P0 projections of
the coarse coefficient (arithmetic, harmonic, geometric mean, Sec. 3.2 /
Fig. 6), the paper's gradient-norm flag rule (Eq. 2.8) and its outer solver
(FGMRES with the block-triangular preconditioner of Eq. 4.1 and the
diag(A)-BFBT of Eq. 4.2), each checked against closed forms and invariants
that do not reuse the oracle's formulas."""
import itertools

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla
import pytest

from oracle import agca
from oracle.mesh import PERMS, Mesh, children_n


def test_projections_of_two_valued_children():
    a, b = 3.0, 7000.0
    for pos in itertools.combinations(range(8), 4):  # every arrangement of 4 a's and 4 b's
        c = np.full(8, b)
        c[list(pos)] = a
        assert agca.coarse_mean(c, "arithmetic") == pytest.approx((a + b) / 2, rel=1e-15)
        assert agca.coarse_mean(c, "harmonic") == pytest.approx(2 * a * b / (a + b), rel=1e-15)
        assert agca.coarse_mean(c, "geometric") == pytest.approx(np.sqrt(a * b), rel=1e-15)
    c = np.full(8, 0.37)
    assert agca.coarse_mean(c, "arithmetic") == 0.37
    for p in ("harmonic", "geometric"):
        assert agca.coarse_mean(c, p) == pytest.approx(0.37, rel=2e-16)
    with pytest.raises(ValueError):
        agca.coarse_mean(c, "median")


@pytest.mark.parametrize("projection", agca.PROJECTIONS)
def test_projection_equals_mean_over_finest_descendants(projection):
    """The recursion over levels equals the same mean taken over all finest
    descendants at once (equal weights), and HM <= GM <= AM."""
    N, L = 4, 3
    eta = np.exp(np.random.default_rng(3).normal(0.0, 2.0, 6 * (2 * N) ** 3))
    mean, mx, mn, _ = agca.flag_hierarchy(N, L, eta, 10.0, projection)
    nL = 2 * N
    desc = np.arange(len(eta))[:, None]  # finest descendants of each level-L element
    for l in range(L - 1, 0, -1):
        desc = desc[children_n(nL >> (L - l))].reshape(6 * (nL >> (L - l)) ** 3, -1)
        v = eta[desc]
        want = {"arithmetic": v.mean(axis=1), "harmonic": 1.0 / (1.0 / v).mean(axis=1),
                "geometric": np.exp(np.log(v).mean(axis=1))}[projection]
        assert np.allclose(mean[l], want, rtol=1e-13, atol=0)
        assert (mean[l] <= mx[l] * (1 + 1e-14)).all() and (mean[l] >= mn[l] * (1 - 1e-14)).all()
    am = agca.flag_hierarchy(N, L, eta, 10.0, "arithmetic")[0]
    gm = agca.flag_hierarchy(N, L, eta, 10.0, "geometric")[0]
    hm = agca.flag_hierarchy(N, L, eta, 10.0, "harmonic")[0]
    for l in range(1, L):
        assert (hm[l] <= gm[l] * (1 + 1e-13)).all() and (gm[l] <= am[l] * (1 + 1e-13)).all()


@pytest.mark.parametrize("projection", ["harmonic", "geometric"])
def test_dca_equals_gca_for_constant_viscosity_any_projection(projection):
    """Sec. 2.1: for a constant coefficient the rediscretised and Galerkin
    coarse operators coincide; every projection of a constant is the constant."""
    N, L = 2, 2
    eta = np.full(6 * (2 * N) ** 3, 4.5)
    h_dca = agca.Hierarchy(N, L, eta, nu=1e30, projection=projection)   # nothing flagged
    h_gca = agca.Hierarchy(N, L, eta, nu=-1.0, projection=projection)   # everything flagged
    A, B = h_dca.A[1].toarray(), h_gca.A[1].toarray()
    assert np.abs(A - B).max() <= 1e-12 * np.abs(A).max()


def test_gradient_norm_of_linear_field():
    """The P1 interpolant of a linear function is the function: its gradient
    is the constant vector on every element."""
    n = 6
    m = Mesh(n)
    a = np.array([3.0, -40.0, 12.5])
    eta_v = m.coords @ a + 2.0
    g = agca.gradient_norms(m, eta_v)
    assert np.allclose(g, np.linalg.norm(a), rtol=1e-12, atol=0)
    N, L = n // 2, 2
    _, flags = agca.gradient_flags(N, L, eta_v, 0.99 * np.linalg.norm(a))
    assert flags[1].all()
    _, flags = agca.gradient_flags(N, L, eta_v, 1.01 * np.linalg.norm(a))
    assert not flags[1].any()


def test_gradient_norm_from_kuhn_path_differences():
    """On a Kuhn tetrahedron with path permutation p the P1 gradient has
    component p[k] equal to the difference of the nodal values along the
    k-th path edge divided by h (the edges are axis-parallel)."""
    n = 4
    m = Mesh(n)
    eta_v = np.random.default_rng(5).uniform(0.5, 2.0, m.nv)
    g = np.zeros((m.ne, 3))
    for e in range(m.ne):
        p = PERMS[e % 6]
        v = m.tets[e]
        for k in range(3):
            g[e, p[k]] = (eta_v[v[k + 1]] - eta_v[v[k]]) * n
    assert np.allclose(agca.gradient_norms(m, eta_v), np.linalg.norm(g, axis=1), rtol=1e-12, atol=0)


def test_gradient_flags_of_a_step():
    """Nodal values 1 left of x = 1/2 and 1000 from it on: only the cubes of
    the column just left of the step have vertices on both sides (each of
    their tetrahedra joins the cube origin to the opposite corner), with
    gradient norm 999 n; every coarse element covering that column is
    flagged, no other."""
    N, L = 4, 3
    nL = 2 * N
    m = Mesh(nL)
    eta_v = np.where(m.ijk[:, 0] < nL // 2, 1.0, 1000.0)
    gmax, flags = agca.gradient_flags(N, L, eta_v, 10.0)
    col = (np.arange(m.ne) // 6) % nL
    crossing = col == nL // 2 - 1
    assert np.allclose(gmax[L][crossing], 999.0 * nL, rtol=1e-12) and not gmax[L][~crossing].any()
    for l in range(1, L):
        nl = nL >> (L - l)
        ccol = (np.arange(6 * nl ** 3) // 6) % nl
        want = ccol == (nL // 2 - 1) >> (L - l)
        assert np.array_equal(flags[l], want)
        assert flags[l].sum() == 6 * nl * nl


# ---- the paper's outer solver (Sec. 4): FGMRES + block-triangular + BFBT ----
@pytest.fixture(scope="module")
def stokes_small():
    from oracle import stokes as ostokes
    from synth import sphere_sinkers

    p = sphere_sinkers(2, 2, 0.2, 0.05, 1e3)
    H = agca.Hierarchy(2, 2, p.eta, 10.0)
    S = ostokes.Stokes(H)
    return p, S


def test_bfbt_is_exact_for_a_diagonal_velocity_block(stokes_small):
    """With A replaced by W = diag(A) the Schur complement B W^-1 B^T is Z
    itself, and Z^-1 (B W^-1 W W^-1 B^T) Z^-1 = Z^-1 (Eq. 4.2)."""
    from oracle.fgmres import BlockTriangular

    _, S = stokes_small
    Q = BlockTriangular(S)
    W = sp.diags(np.where(S.mask > 0, 1.0 / np.where(Q.winv > 0, Q.winv, 1.0), 0.0))
    Qd = BlockTriangular(S, A_bfbt=W)
    x = np.random.default_rng(4).normal(size=S.np_)
    x -= x.mean()
    assert np.allclose(Qd.bfbt(Qd.Z @ x), x, rtol=0, atol=1e-10 * np.abs(x).max())
    # the default BFBT differs from Z^-1 (A is not diagonal) but is symmetric
    y = np.random.default_rng(5).normal(size=S.np_)
    y -= y.mean()
    assert abs(Q.bfbt(x) @ y - x @ Q.bfbt(y)) <= 1e-10 * np.linalg.norm(Q.bfbt(x)) * np.linalg.norm(y)


def test_exact_block_triangular_fgmres_converges_in_two_steps(stokes_small):
    """With A~ = A and S~ = S = B A^-1 B^T exact, K Q^-1 = [[I, 0], [B A^-1, I]]
    has (K Q^-1 - I)^2 = 0, so FGMRES reaches the solution in two steps.  A
    missing or sign-flipped coupling term A~^-1 B^T S~^-1 takes three (the
    sign of the Schur block alone is not seen: -S~ and +S~ both give a
    degree-2 minimal polynomial)."""
    from oracle.fgmres import BlockTriangular, solve

    p, S = stokes_small
    iv = np.nonzero(S.mask > 0)[0]
    lu = spla.splu(S.A[iv][:, iv].tocsc())

    def a_exact(r):
        z = np.zeros_like(r)
        z[iv] = lu.solve(r[iv])
        return z

    Bi = S.B[:, iv].toarray()
    Sd = Bi @ lu.solve(Bi.T)
    Spinv = np.linalg.pinv(Sd, rcond=1e-12)

    def s_exact(rp):
        return Spinv @ (rp - rp.mean())

    b = S.rhs(p.fbar)
    x, its = solve(S, b, rtol=1e-10, precond=BlockTriangular(S, a_inv=a_exact, s_inv=s_exact))
    assert its <= 2
    x_ref = S.direct(b)
    assert np.abs(x - x_ref).max() <= 1e-8 * np.abs(x_ref).max()


def test_fgmres_vcycle_bfbt_matches_direct_solve(stokes_small):
    from oracle.fgmres import solve

    p, S = stokes_small
    b = S.rhs(p.fbar)
    x, its = solve(S, b, rtol=1e-11)
    x_ref = S.direct(b)
    assert its > 2
    assert np.linalg.norm(b - S.K(x)) <= 1.01e-11 * np.linalg.norm(b)
    assert np.abs(x - x_ref).max() <= 1e-8 * np.abs(x_ref).max()


def test_z_couples_pressure_vertices_two_kuhn_offsets_apart():
    """Z = B W^-1 B^T (the BFBT operator of Eq. 4.2) couples pressure vertex
    i with j exactly when j - i is a sum of two Kuhn offsets (a pressure hat
    and a velocity hat overlap only inside one pressure cell): 65 distinct
    offsets in [-2, 2]^3, every one of them present at an interior vertex, so
    per-vertex stencils over those 65 offsets hold Z, and mod-5 colour
    probing separates them."""
    from oracle import stokes as ostokes
    from oracle.fgmres import BlockTriangular
    from synth import sphere_sinkers

    N = 6
    p = sphere_sinkers(N, 2, 0.2, 0.05, 1e3, seed=9)
    S = ostokes.Stokes(agca.Hierarchy(N, 2, p.eta, 10.0))
    Z = BlockTriangular(S).Z.tocoo()
    nv = N + 1
    tol = 1e-13 * np.abs(Z.data).max()
    ijk = lambda v: np.stack([v % nv, (v // nv) % nv, v // (nv * nv)], axis=-1)
    keep = np.abs(Z.data) > tol
    d = ijk(Z.col[keep]) - ijk(Z.row[keep])
    offsets = set(map(tuple, d))
    kuhn = [(0, 0, 0)] + [s * np.array(e) for e in ((1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 0, 1),
                                                      (0, 1, 1), (1, 1, 1)) for s in (1, -1)]
    pairs = {tuple(np.add(a, b)) for a in kuhn for b in kuhn}
    assert len(pairs) == 65
    assert offsets == pairs
    # the centre vertex (3, 3, 3) couples with all 65
    c = 3 + nv * (3 + nv * 3)
    assert len(set(map(tuple, d[Z.row[keep] == c]))) == 65
    assert np.abs(d).max() <= 2


# ---- stencil storage of the coarse operators (Remark 5) ----
def test_agca_rows_fit_the_15_point_kuhn_stencil():
    """Every level's AGCA operator, with DCA and stored Galerkin elements
    mixed, couples a vertex only with itself and its 14 Kuhn neighbours, so
    per-vertex 15-offset stencils hold it exactly: the stencils rebuild the
    matrix (nonzero count included) and apply as the matrix does."""
    from synth import sphere_sinkers

    p = sphere_sinkers(4, 3, 0.15, 0.02, 1e4)
    H = agca.Hierarchy(4, 3, p.eta, 10.0)
    assert sum(len(H.flist[l]) for l in (1, 2)) > 0
    for l in (1, 2, 3):
        blocks = agca.stencil_blocks(H, l)
        nnz_stencil = np.count_nonzero(blocks)
        assert nnz_stencil == H.A[l].count_nonzero(), l  # nothing outside the 15 offsets
        x = np.random.default_rng(l).normal(size=3 * H.mesh[l].nv)
        y = agca.stencil_apply(H, l, blocks, x)
        assert np.allclose(y, H.A[l] @ x, rtol=0, atol=1e-12 * np.abs(H.A[l] @ x).max()), l
    assert len(agca.KUHN_OFFSETS) == 15 and len({tuple(o) for o in agca.KUHN_OFFSETS}) == 15


# ---- coarse coefficients evaluated on the coarse grid (Eq. 2.5, Sec. 3.2) ----
def test_level_coefficient_override():
    """Overriding a coarse level's DCA coefficient with the values the
    children's projection gives changes nothing; with every element DCA
    (no flags) the level operator is the assembly of the rediscretised
    element matrices of the given coefficient."""
    from oracle import fem
    from synth import sphere_sinkers

    p = sphere_sinkers(4, 3, 0.15, 0.02, 1e4)
    H = agca.Hierarchy(4, 3, p.eta, 10.0)
    H2 = agca.Hierarchy(4, 3, p.eta, 10.0, level_coef={1: H.mean[1].copy(), 2: H.mean[2].copy()})
    for l in (1, 2, 3):
        assert (H.A[l] != H2.A[l]).nnz == 0
    rng = np.random.default_rng(3)
    c = {l: np.exp(rng.normal(size=H.mesh[l].ne)) for l in (1, 2)}
    Hd = agca.Hierarchy(4, 3, p.eta, 1e300, level_coef=c)
    for l in (1, 2):
        m = Hd.mesh[l]
        A = fem.assemble(m, fem.element_matrices(m, c[l]))
        ref = fem.mask_matrix(A, Hd.mask[l], Hd.mask[l])
        assert abs(Hd.A[l] - ref).max() <= 1e-13 * abs(ref).max()
    # flags keep the finest descendants' extremes
    assert all(np.array_equal(Hd.flags[l], H.mx[l] > 1e300 * H.mn[l]) for l in (1, 2))


def test_analytic_level_coefficients_of_quadratic_field_equal_the_projection():
    """The 4-point rule integrates quadratics exactly, and a parent's mean is
    the average of its 8 equal-volume children's means: for a quadratic
    field the analytic coarse coefficients equal the arithmetic projection."""
    import torch

    from synth import field_problem, level_coefficients

    def fn(x):
        v = 1.0 + x[..., 0] ** 2 + 2.0 * x[..., 1] * x[..., 2] + 0.5 * x[..., 2]
        return v, torch.zeros_like(v)

    N, L = 4, 3
    p = field_problem(N, fn)
    mean, _, _, _ = agca.flag_hierarchy(N, L, p.eta, 10.0)
    lc = level_coefficients(fn, N, L, "analytic")
    for l in (1, 2):
        assert np.abs(lc[l] - mean[l]).max() <= 1e-14 * np.abs(mean[l]).max()


def test_p1_means_of_linear_field_are_exact_means():
    import torch

    from synth import field_problem, p1_element_means

    def fn(x):
        v = 2.0 + 3.0 * x[..., 0] - x[..., 1] + 0.25 * x[..., 2]
        return v, torch.zeros_like(v)

    p = field_problem(3, fn)
    assert np.abs(p1_element_means(6, fn) - p.eta).max() <= 1e-14 * np.abs(p.eta).max()


def test_tanh_cube_tends_to_the_unaligned_cube():
    """eta_3 (Eq. 3.7 profiles) approaches eta_2 away from the cube faces as
    omega grows; eta_1 is the aligned cube of cfg0."""
    import torch

    from synth import C_UA, cube_field

    pts = torch.tensor([[C_UA, C_UA, C_UA], [0.1, 0.2, 0.9], [C_UA + 0.1, C_UA - 0.1, C_UA], [0.5, 0.5, 0.5]],
                       dtype=torch.float64)
    e2, f2 = cube_field("unaligned", 1e6)(pts)
    e3, _ = cube_field("tanh", 1e6, omega=1e3)(pts)
    assert torch.allclose(e3, e2, rtol=1e-9)
    assert float(e2[0]) == 1e3 and float(e2[1]) == 1e-3 and float(f2[0]) == -1.0
    e1, _ = cube_field("aligned", 1e6)(pts)
    assert float(e1[3]) == 1e3 and float(e1[1]) == 1e-3


def test_flagged_stencils_plus_dca_part_rebuild_the_level_operator():
    """Remark 5's storage for AGCA: per-vertex 15-offset stencils of the
    flagged elements' Galerkin matrices only, plus the matrix-free DCA part of
    the unflagged elements, apply as the level operator; the stencils are
    nonzero only at vertices of flagged elements."""
    from oracle import fem
    from synth import sphere_sinkers

    p = sphere_sinkers(4, 3, 0.15, 0.02, 1e4)
    H = agca.Hierarchy(4, 3, p.eta, 10.0)
    for l in (1, 2):
        m = H.mesh[l]
        assert len(H.flist[l]) > 0
        S = agca.stencil_blocks(H, l, agca.flagged_operator(H, l))
        unflagged = np.setdiff1d(np.arange(m.ne), H.flist[l])
        Ad = fem.mask_matrix(fem.assemble(m, fem.element_matrices(m, H.mean[l][unflagged], unflagged), unflagged),
                             H.mask[l], H.mask[l])
        x = np.random.default_rng(l).normal(size=3 * m.nv)
        y = agca.stencil_apply(H, l, S, x) + Ad @ x
        ref = H.A[l] @ x
        assert np.abs(y - ref).max() <= 1e-12 * np.abs(ref).max()
        touched = np.zeros(m.nv, dtype=bool)
        touched[m.tets[H.flist[l]].ravel()] = True
        assert np.abs(S[~touched]).max() == 0.0
        assert np.abs(S[touched & m.interior]).max(axis=(1, 2, 3)).min() > 0.0
