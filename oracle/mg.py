"""Geometric h-multigrid components (oracle; test infrastructure).

Sec. 3.3 of the paper: the pressure Poisson problem is solved by CG
preconditioned with one multigrid V-cycle per iteration; smoothing is a
Chebyshev polynomial of degree 5 (pre and post) with smoothing range 20 built
on the matrix diagonal; the coarse-grid solver is also Chebyshev with a fixed
number of iterations; the transfers are matrix-free.  The paper defers the
transfer and level details to other work, so this oracle takes the readings:
  * levels are h-levels n, n/2, ..., n_coarse, each re-discretised with the
    SIPG form of the same degree and tau = (k+1)^2 / h_level;
  * prolongation is the exact embedding of a coarse cell polynomial into its
    8 children (evaluation at the children's LGL nodes); restriction is its
    transpose;
  * Chebyshev follows Saad, Iterative Methods for Sparse Linear Systems,
    2nd ed., Algorithm 12.1, preconditioned with the inverse diagonal, on the
    interval [lambda_max / range, lambda_max]; "degree m" means m updates of x.
"""
import numpy as np

from . import dg, rules


class Transfer:
    """Embedding of the coarse space (mesh n/2) into the fine space (mesh n)."""

    def __init__(self, coarse_space, fine_space):
        self.cs, self.fs = coarse_space, fine_space
        mc, mf = coarse_space.mesh, fine_space.mesh
        assert all(nf == 2 * nc for nf, nc in zip(mf.n, mc.n))
        nodes = fine_space.nodes
        P1 = [rules.lagrange(coarse_space.nodes, 0.5 * (c + nodes))[0] for c in (0, 1)]
        self.P = {}
        for cz in (0, 1):
            for cy in (0, 1):
                for cx in (0, 1):
                    self.P[(cx, cy, cz)] = dg.tensor3(P1[cx], P1[cy], P1[cz])
        ijk = mf.ijk
        self.parent = mc.elem(ijk[0] // 2, ijk[1] // 2, ijk[2] // 2)
        self.child = np.stack([ijk[0] % 2, ijk[1] % 2, ijk[2] % 2])

    def prolongate(self, Xc):
        Xf = np.empty((self.fs.mesh.E, self.fs.ndofs_cell))
        for key, P in self.P.items():
            sel = np.all(self.child == np.array(key)[:, None], axis=0)
            Xf[sel] = Xc[self.parent[sel]] @ P.T
        return Xf

    def restrict(self, Xf):
        Xc = np.zeros((self.cs.mesh.E, self.cs.ndofs_cell))
        for key, P in self.P.items():
            sel = np.all(self.child == np.array(key)[:, None], axis=0)
            np.add.at(Xc, self.parent[sel], Xf[sel] @ P)
        return Xc


def chebyshev(apply_A, inv_diag, b, x0, lam_max, smoothing_range, degree):
    """Jacobi-preconditioned Chebyshev iteration (Saad, Alg. 12.1) on
    [lam_max / smoothing_range, lam_max]; `degree` updates of x.  x0=None means
    a zero initial guess (no matrix-vector product for the first residual)."""
    lam_min = lam_max / smoothing_range
    theta = 0.5 * (lam_max + lam_min)
    delta = 0.5 * (lam_max - lam_min)
    sigma = theta / delta
    rho = 1.0 / sigma
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - apply_A(x)
    d = inv_diag * r / theta
    for it in range(degree):
        x = x + d
        if it == degree - 1:
            break
        r = r - apply_A(d)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * inv_diag * r
        rho = rho_new
    return x


class Hierarchy:
    """Levels of the SIPG Laplacian on meshes n, n/2, ..., coarse_n (all
    directions halved together)."""

    def __init__(self, mesh, k, coarse_n=2, penalty_factor=1.0):
        self.levels = []
        n = list(mesh.n)
        meshes = [mesh]
        while all(v % 2 == 0 and v // 2 >= coarse_n for v in n):
            n = [v // 2 for v in n]
            meshes.append(dg.Mesh(n, mesh.lo, mesh.hi))
        meshes.reverse()                       # level 0 = coarsest
        for m in meshes:
            s = dg.Space(m, k)
            L = dg.Laplace(s, penalty_factor)
            self.levels.append({"space": s, "op": L, "inv_diag": 1.0 / L.diagonal()})
        self.transfers = [Transfer(self.levels[i]["space"], self.levels[i + 1]["space"])
                          for i in range(len(self.levels) - 1)]

    def vcycle(self, b, lam_max, degree=5, smoothing_range=20.0, coarse_iters=None,
               level=None):
        """One V-cycle applied to b; lam_max is a list per level (coarsest
        first) so that the oracle and the device use the same intervals."""
        if level is None:
            level = len(self.levels) - 1
        lv = self.levels[level]
        A = lv["op"].apply
        if level == 0:
            it = coarse_iters if coarse_iters is not None else degree
            return chebyshev(A, lv["inv_diag"], b, None, lam_max[0], smoothing_range, it)
        x = chebyshev(A, lv["inv_diag"], b, None, lam_max[level], smoothing_range, degree)
        r = b - A(x)
        T = self.transfers[level - 1]
        ec = self.vcycle(T.restrict(r), lam_max, degree, smoothing_range, coarse_iters,
                         level - 1)
        x = x + T.prolongate(ec)
        return chebyshev(A, lv["inv_diag"], b, x, lam_max[level], smoothing_range, degree)
