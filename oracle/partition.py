"""Domain decomposition of the AGCA V-cycle and the MINRES Stokes solve over
z-slabs, one rank per slab: the parallel layout of the paper (processes own
sub-domains; Remark 1: the local Galerkin products need no communication;
Sec. 5), written as a plain CPU reference that ranks run under
torch.distributed (gloo).  Test infrastructure, like the rest of oracle/.

Partition.  Level l has n_l = n_L / 2^(L-l) cubes per axis; the n_1 cube
layers of the coarsest level are split into R contiguous ranges [a_r, b_r),
and rank r owns the cube layers [a_r 2^(l-1), b_r 2^(l-1)) of every level:
slab boundaries lie on coarsest-cube faces, so the 8 children of an element
always belong to its rank.  Rank r stores the vertex planes z0..z1 of its
slab; the planes z0 (r > 0) and z1 (r < R-1) are interface planes that it
shares with its neighbours.

Communication (all of it):
  * operator apply (and the diagonal, the Stokes blocks B, B^T, the load
    vector and the lumped pressure mass): each rank sums its own elements'
    contributions, then the two ranks of an interface plane exchange their
    partial sums of that plane and add them (both get the same values:
    floating-point addition commutes);
  * restriction P^T r: each fine vertex is counted by exactly one rank (its
    owner: the lower slab owns a shared plane's dot-product share, see
    `owned`), then the coarse interface planes are summed as above;
  * prolongation: none (a fine vertex's coarse neighbours lie in its slab);
  * inner products and the pressure mean: an all-reduce of one scalar;
  * coarsest level: the local dense matrices and right-hand sides are summed
    over all ranks and every rank solves the same Cholesky system.
Flags, viscosity means and stored Galerkin matrices are computed by each
rank from its own elements' viscosity only.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import fem
from .agca import coarse_mean, splitmix64
from .mesh import Mesh, children_n, local_interpolation, prolongation
from .stokes import minres


class SlabComm:
    """One rank's exchanges: interface-plane sums with the neighbouring slabs
    (point-to-point) and sums over all ranks (all-reduce).  dist =
    torch.distributed with an initialised process group, or None for one
    rank (no communication)."""

    def __init__(self, dist=None):
        self.dist = dist
        self.rank = dist.get_rank() if dist is not None else 0
        self.world = dist.get_world_size() if dist is not None else 1

    def interface_sum(self, lo, hi):
        """lo / hi: this rank's partial values on its lower / upper interface
        plane (None where the slab ends at the domain boundary); returns them
        summed with the neighbours' partial values of the same planes."""
        if self.world == 1:
            return lo, hi
        import torch

        reqs, recv = [], {}
        for key, plane, peer in (("lo", lo, self.rank - 1), ("hi", hi, self.rank + 1)):
            if plane is None:
                continue
            t = torch.from_numpy(np.ascontiguousarray(plane, dtype=np.float64))
            r = torch.empty_like(t)
            reqs.append(self.dist.isend(t, peer))
            reqs.append(self.dist.irecv(r, peer))
            recv[key] = r
        for q in reqs:
            q.wait()
        out_lo = lo + recv["lo"].numpy() if lo is not None else None
        out_hi = hi + recv["hi"].numpy() if hi is not None else None
        return out_lo, out_hi

    def allreduce(self, a):
        if self.world == 1:
            return a
        import torch

        t = torch.from_numpy(np.array(a, dtype=np.float64, ndmin=1))
        self.dist.all_reduce(t)
        out = t.numpy()
        return out if np.ndim(a) else float(out[0])


def slab_layers(n1: int, rank: int, world: int):
    """Coarsest cube layers [a, b) of a rank."""
    if world > n1:
        raise ValueError(f"{world} ranks for {n1} coarsest cube layers")
    return rank * n1 // world, (rank + 1) * n1 // world


class SlabLevel:
    """Index bookkeeping of one level on one slab."""

    def __init__(self, n: int, z0: int, z1: int):
        self.n, self.z0, self.z1 = n, z0, z1
        self.m = n + 1
        self.plane = self.m * self.m
        self.nv = self.plane * (z1 - z0 + 1)          # local vertices: planes z0..z1
        self.v0 = self.plane * z0                     # global id of local vertex 0
        self.e0, self.e1 = 6 * n * n * z0, 6 * n * n * z1  # global ids of the slab's elements
        self.elems = np.arange(self.e0, self.e1)

    def local_dofs(self, gdofs, nv_global):
        """Global SoA DoF ids c * V + v -> local c * V_loc + (v - v0)."""
        c, v = np.divmod(gdofs, nv_global)
        return c * self.nv + (v - self.v0)

    def vertex_slice(self):
        return slice(self.v0, self.v0 + self.nv)


class SlabHierarchy:
    """The AGCA hierarchy of one slab (same method and parameters as
    oracle.agca.Hierarchy, arithmetic P0 coefficient projection)."""

    def __init__(self, N: int, L: int, eta_slab: np.ndarray, nu: float, comm: SlabComm,
                 cheb_lo: float = 0.1, cheb_hi: float = 1.1, cheb_degree: int = 2, power_iters: int = 20):
        nL = 2 * N
        self.N, self.L, self.nu, self.comm = N, L, nu, comm
        self.cheb_lo, self.cheb_hi, self.cheb_degree, self.power_iters = cheb_lo, cheb_hi, cheb_degree, power_iters
        n = {l: nL >> (L - l) for l in range(1, L + 1)}
        a, b = slab_layers(n[1], comm.rank, comm.world)
        self.lv = {l: SlabLevel(n[l], a << (l - 1), b << (l - 1)) for l in range(1, L + 1)}
        self.mesh = {l: Mesh(n[l]) for l in range(1, L + 1)}  # geometry of the whole level
        # children of the slab's elements, as local element ids of the next finer level
        self.ch_global = {l: children_n(n[l]) for l in range(1, L)}
        self.ch = {l: self.ch_global[l][self.lv[l].elems] - self.lv[l + 1].e0 for l in range(1, L)}
        for l in range(1, L):
            assert self.ch[l].min() >= 0 and self.ch[l].max() < len(self.lv[l + 1].elems), \
                "children must stay in the slab"
        eta = np.asarray(eta_slab, dtype=np.float64)
        assert eta.shape == (len(self.lv[L].elems),)
        # viscosity hierarchy, flags and stored Galerkin matrices: slab-local (Remark 1)
        self.mean, self.mx, self.mn, self.flags = {L: eta}, {L: eta}, {L: eta}, {}
        for l in range(L - 1, 0, -1):
            k = self.ch[l]
            self.mean[l] = coarse_mean(self.mean[l + 1][k])
            self.mx[l] = self.mx[l + 1][k].max(axis=1)
            self.mn[l] = self.mn[l + 1][k].min(axis=1)
            self.flags[l] = self.mx[l] > nu * self.mn[l]
        self.flist = {l: np.nonzero(self.flags[l])[0] for l in range(1, L)}
        self.findex = {}
        for l in range(1, L):
            idx = np.full(len(self.lv[l].elems), -1, dtype=np.int64)
            idx[self.flist[l]] = np.arange(len(self.flist[l]))
            self.findex[l] = idx
        self.gca = {}
        for l in range(L - 1, 0, -1):
            self.gca[l] = self._galerkin(l, self.flist[l])
        self._build_operators()

    # ---- element matrices (the oracle's formulas on the slab's elements) ----
    def _child_matrices(self, l, kids):
        shape = kids.shape
        kids = kids.ravel()
        fl = self.lv[l + 1]
        C = fem.element_matrices(self.mesh[l + 1], self.mean[l + 1][kids], kids + fl.e0)
        if l + 1 < self.L:
            fi = self.findex[l + 1][kids]
            sel = fi >= 0
            C[sel] = self.gca[l + 1][fi[sel]]
        return C.reshape(shape + (12, 12))

    def _galerkin(self, l, elems):
        if len(elems) == 0:
            return np.zeros((0, 12, 12))
        p = local_interpolation(self.mesh[l], self.mesh[l + 1], self.ch_global[l], elems + self.lv[l].e0)
        P12 = np.zeros(p.shape[:2] + (12, 12))
        for c in range(3):
            P12[:, :, 4 * c:4 * c + 4, 4 * c:4 * c + 4] = p
        C = self._child_matrices(l, self.ch[l][elems])
        return np.einsum("fkia,fkij,fkjb->fab", P12, C, P12)

    def level_element_matrices(self, l):
        lv = self.lv[l]
        A = fem.element_matrices(self.mesh[l], self.mean[l], lv.elems)
        if l < self.L and len(self.flist[l]):
            A[self.flist[l]] = self.gca[l]
        return A

    # ---- slab operators ------------------------------------------------------
    def _assemble(self, l, mats):
        lv, m = self.lv[l], self.mesh[l]
        dofs = lv.local_dofs(fem.element_dofs(m, lv.elems), m.nv)
        rows = np.repeat(dofs, 12, axis=1).ravel()
        cols = np.tile(dofs, (1, 12)).ravel()
        n = 3 * lv.nv
        return sp.coo_matrix((mats.ravel(), (rows, cols)), shape=(n, n)).tocsr()

    def _build_operators(self):
        L = self.L
        self.A, self.P, self.D, self.invD, self.lam, self.mask, self.own = {}, {}, {}, {}, {}, {}, {}
        for l in range(1, L + 1):
            lv, m = self.lv[l], self.mesh[l]
            self.mask[l] = np.tile(m.interior[lv.vertex_slice()].astype(np.float64), 3)
            own = np.ones(lv.nv)
            if self.comm.rank < self.comm.world - 1:
                own[-lv.plane:] = 0.0  # the upper interface plane's share belongs to the next slab
            self.own[l] = np.tile(own, 3)
            A = self._assemble(l, self.level_element_matrices(l))
            self.A[l] = fem.mask_matrix(A, self.mask[l], self.mask[l])
            self.D[l] = self.interface(l, self.A[l].diagonal())
            inv = np.zeros_like(self.D[l])
            inv[self.mask[l] > 0] = 1.0 / self.D[l][self.mask[l] > 0]
            self.invD[l] = inv
        for l in range(1, L):
            lc, lf = self.lv[l], self.lv[l + 1]
            Pg = prolongation(self.mesh[l], self.mesh[l + 1])[lf.vertex_slice()]
            outside = Pg[:, :lc.v0].nnz + Pg[:, lc.v0 + lc.nv:].nnz
            assert outside == 0, "a slab's fine vertices interpolate from its own coarse vertices"
            Ps = Pg[:, lc.vertex_slice()]
            P = sp.block_diag([Ps, Ps, Ps]).tocsr()
            self.P[l] = fem.mask_matrix(P, self.mask[l + 1], self.mask[l])
        for l in range(2, L + 1):
            self.lam[l] = self.power_lambda(l)
        self._coarse_setup()

    def interface(self, l, y):
        """Sum the partial values of the interface planes with the neighbours."""
        lv = self.lv[l]
        Y = y.reshape(3, lv.nv)
        lo = Y[:, :lv.plane].copy() if self.comm.rank > 0 else None
        hi = Y[:, -lv.plane:].copy() if self.comm.rank < self.comm.world - 1 else None
        lo, hi = self.comm.interface_sum(lo, hi)
        Y = Y.copy()
        if lo is not None:
            Y[:, :lv.plane] = lo
        if hi is not None:
            Y[:, -lv.plane:] = hi
        return Y.ravel()

    def apply(self, l, x):
        return self.interface(l, self.A[l] @ x)

    def dot(self, l, x, y):
        return self.comm.allreduce(float(np.dot(self.own[l] * x, y)))

    def restrict(self, l, r):
        """P^T r from level l to l - 1."""
        return self.interface(l - 1, self.P[l - 1].T @ (self.own[l] * r))

    def prolong(self, l, e):
        """P e from level l - 1 to l (no exchange)."""
        return self.P[l - 1] @ e

    def start_vector(self, l):
        lv, m = self.lv[l], self.mesh[l]
        v = np.arange(lv.v0, lv.v0 + lv.nv)
        gidx = np.concatenate([c * m.nv + v for c in range(3)])
        u = (splitmix64(gidx) >> np.uint64(11)).astype(np.float64) * 2.0 ** -53
        return 2.0 * u - 1.0

    def power_lambda(self, l):
        v = self.start_vector(l) * self.mask[l]
        for _ in range(self.power_iters):
            w = self.invD[l] * self.apply(l, v)
            v = w / np.sqrt(self.dot(l, w, w))
        return self.dot(l, v, self.apply(l, v)) / self.dot(l, v, self.D[l] * v)

    def chebyshev(self, l, b, x):
        a, bb = self.cheb_lo * self.lam[l], self.cheb_hi * self.lam[l]
        theta, delta = 0.5 * (bb + a), 0.5 * (bb - a)
        sigma = theta / delta
        rho = 1.0 / sigma
        invD = self.invD[l]
        r = b - self.apply(l, x)
        d = invD * r / theta
        x = x + d
        for _ in range(1, self.cheb_degree):
            rho_new = 1.0 / (2.0 * sigma - rho)
            r = b - self.apply(l, x)
            d = rho_new * rho * d + (2.0 * rho_new / delta) * (invD * r)
            x = x + d
            rho = rho_new
        return x

    def _coarse_setup(self):
        """The coarsest operator summed over all ranks (dense, global
        numbering) and factored redundantly on every rank."""
        lv, m = self.lv[1], self.mesh[1]
        nglob = 3 * m.nv
        self.coarse_gidx = np.concatenate([c * m.nv + np.arange(lv.v0, lv.v0 + lv.nv) for c in range(3)])
        A = self.A[1].tocoo()
        dense = np.zeros((nglob, nglob))
        np.add.at(dense, (self.coarse_gidx[A.row], self.coarse_gidx[A.col]), A.data)
        dense = self.comm.allreduce(dense.ravel()).reshape(nglob, nglob)
        mask = fem.velocity_mask(m)
        self.coarse_idx = np.nonzero(mask > 0)[0]
        self.coarse_factor = sla.cho_factor(dense[self.coarse_idx][:, self.coarse_idx], lower=True)
        self.coarse_nglob = nglob

    def coarse_solve(self, b):
        g = np.zeros(self.coarse_nglob)
        g[self.coarse_gidx] = self.own[1] * b
        g = self.comm.allreduce(g)
        z = np.zeros(self.coarse_nglob)
        z[self.coarse_idx] = sla.cho_solve(self.coarse_factor, g[self.coarse_idx])
        return z[self.coarse_gidx]

    def vcycle(self, b, l=None):
        if l is None:
            l = self.L
        if l == 1:
            return self.coarse_solve(b)
        x = self.chebyshev(l, b, np.zeros_like(b))
        r = b - self.apply(l, x)
        ec = self.vcycle(self.restrict(l, r), l - 1)
        x = x + self.prolong(l, ec)
        return self.chebyshev(l, b, x)


class SlabStokes:
    """The Stokes system of oracle.stokes.Stokes on one slab: velocity on
    level L, pressure on level L-1 (the P1-iso-P2 / P1 pair, Eq. 3.3),
    preconditioner blockdiag(V-cycle, mean-free lumped 1/eta mass)."""

    def __init__(self, hier: SlabHierarchy):
        self.h = h = hier
        L = h.L
        self.lu, self.lp = h.lv[L], h.lv[L - 1]
        vm, pm = h.mesh[L], h.mesh[L - 1]
        self.vm, self.pm = vm, pm
        ch = h.ch_global[L - 1]
        parent = np.empty(vm.ne, dtype=np.int64)
        parent[ch.ravel()] = np.repeat(np.arange(pm.ne), 8)
        D = fem.divergence(pm, vm, parent, elems=self.lu.elems)[self.lp.vertex_slice()].tocsc()
        # velocity columns in the slab's local numbering
        gcols = np.concatenate([c * vm.nv + np.arange(self.lu.v0, self.lu.v0 + self.lu.nv) for c in range(3)])
        D = D[:, gcols]
        self.mask = h.mask[L]
        self.B = -(D @ sp.diags(self.mask)).tocsr()
        self.BT = self.B.T.tocsr()
        M = fem.pressure_mass_lumped(pm, h.mean[L], h.ch[L - 1], elems=self.lp.elems)
        self.Mp = self.pinterface(M[self.lp.vertex_slice()])
        ownp = np.ones(self.lp.nv)
        if h.comm.rank < h.comm.world - 1:
            ownp[-self.lp.plane:] = 0.0
        self.ownp = ownp
        self.nu_ = 3 * self.lu.nv
        self.np_ = self.lp.nv
        self.np_global = pm.nv

    def pinterface(self, p):
        lp = self.lp
        lo = p[:lp.plane].copy() if self.h.comm.rank > 0 else None
        hi = p[-lp.plane:].copy() if self.h.comm.rank < self.h.comm.world - 1 else None
        lo, hi = self.h.comm.interface_sum(lo, hi)
        p = p.copy()
        if lo is not None:
            p[:lp.plane] = lo
        if hi is not None:
            p[-lp.plane:] = hi
        return p

    def split(self, x):
        return x[:self.nu_], x[self.nu_:]

    def K(self, x):
        u, p = self.split(x)
        yu = self.h.interface(self.h.L, self.h.A[self.h.L] @ u + self.BT @ p)
        yp = self.pinterface(self.B @ u)
        return np.concatenate([yu, yp])

    def dot(self, x, y):
        own = np.concatenate([self.h.own[self.h.L], self.ownp])
        return self.h.comm.allreduce(float(np.dot(own * x, y)))

    def project(self, p):
        mean = self.h.comm.allreduce(float(np.dot(self.ownp, p))) / self.np_global
        return p - mean

    def precondition(self, r):
        ru, rp = self.split(r)
        zu = self.h.vcycle(ru)
        zp = self.project(self.project(rp) / self.Mp)
        return np.concatenate([zu, zp])

    def rhs(self, fbar_slab):
        b = fem.load_vector(self.vm, fbar_slab, elems=self.lu.elems)
        bu = np.concatenate([b[c * self.vm.nv:(c + 1) * self.vm.nv][self.lu.vertex_slice()] for c in range(3)])
        return np.concatenate([self.h.interface(self.h.L, bu), np.zeros(self.np_)])

    def minres(self, b, rtol, maxit):
        return minres(self.K, self.precondition, b, rtol, maxit, dot=self.dot)
