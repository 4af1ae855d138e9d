"""DG operators assembled from explicit element and face matrices (oracle).

Test infrastructure only; see the package docstring.

Paper references (arXiv:1802.01439):
  Sec. 3.2  function spaces (mixed degrees k_u = k, k_p = k - 1), LGL nodal
            tensor-product basis, Gauss quadrature exact on affine cells with
            3/2 over-integration of the convective term, average and jump
            operators, and the weak forms m, c (local Lax-Friedrichs flux),
            g, d (central fluxes), v and l (symmetric interior penalty).
  Sec. 3.3  matrix forms M, C, L, D, G, V of the dual-splitting substeps.
  Sec. 4    Taylor-Green vortex on the periodic cube [-pi, pi]^3.

Mesh and vector layout: a uniform periodic Cartesian mesh of nx*ny*nz hexes,
element id e = i + nx*(j + ny*l).  A scalar DG vector is an array (E, N^3) with
local node id I = ix + N*(iy + N*iz) (x fastest); a vector field is
(3, E, N^3).  This is the flat layout [comp][elem][z][y][x].

Readings of the paper used here (it leaves them open):
  * penalty tau = penalty_factor * (k+1)^2 / h_a on faces normal to axis a;
  * Gauss rule with k+1 points for m, l, v and with k_u+1 points for d and g;
    floor(3(k+1)/2) points for c; faces use the same 1D counts;
  * the LLF term max(|u-.n|, |u+.n|) [[u]].n equals max(...) (u- - u+);
  * face orientation: the face (e, axis a) joins e- = e and e+ = its periodic
    +a neighbour, n = +e_a.
"""
import numpy as np

from . import rules

PI = np.pi


class Mesh:
    """Uniform periodic Cartesian mesh of the box [lo, hi] (Sec. 4: (2^l)^d
    elements on [-pi, pi]^3; any n per direction is allowed here)."""

    def __init__(self, n, lo=(-PI, -PI, -PI), hi=(PI, PI, PI), dtype=np.float64):
        """dtype: the precision of every table and product (np.float64; or
        np.longdouble for an extended-precision evaluation of the same
        discrete operators: lo and hi stay the given doubles)."""
        if np.isscalar(n):
            n = (n, n, n)
        self.n = tuple(int(v) for v in n)
        self.dtype = np.dtype(dtype)
        self.lo = np.array(lo, dtype=np.float64).astype(dtype)
        self.hi = np.array(hi, dtype=np.float64).astype(dtype)
        self.h = (self.hi - self.lo) / np.array(self.n, dtype=dtype)
        self.E = self.n[0] * self.n[1] * self.n[2]
        e = np.arange(self.E)
        self.ijk = np.stack([e % self.n[0], (e // self.n[0]) % self.n[1],
                             e // (self.n[0] * self.n[1])])

    @property
    def volume(self):
        return float(np.prod(self.hi - self.lo))

    def elem(self, i, j, l):
        nx, ny, nz = self.n
        return (i % nx) + nx * ((j % ny) + ny * (l % nz))

    def neighbor(self, axis, sign):
        """Periodic neighbour of every element along `axis` in direction
        `sign` (+1 or -1)."""
        idx = [self.ijk[0].copy(), self.ijk[1].copy(), self.ijk[2].copy()]
        idx[axis] = idx[axis] + sign
        return self.elem(*idx)


def tensor3(Ax, Ay, Az):
    """3D tensor-product table T[q, I] = Ax[qx, ix] Ay[qy, iy] Az[qz, iz] with
    x-fastest flattening of both q and I."""
    return np.kron(Az, np.kron(Ay, Ax))


class Space:
    """Scalar DG space of tensor degree k on `mesh` with LGL nodal basis."""

    def __init__(self, mesh, k):
        self.mesh = mesh
        self.k = int(k)
        self.N = self.k + 1
        self.dtype = mesh.dtype
        self.nodes = rules.lgl_nodes(self.k, self.dtype)
        self.ndofs_cell = self.N ** 3
        self.size = mesh.E * self.ndofs_cell

    def node_coords(self):
        """Physical coordinates (3, E, N^3) of every nodal DoF."""
        m = self.mesh
        N = self.N
        I = np.arange(N ** 3)
        loc = np.stack([I % N, (I // N) % N, I // (N * N)])
        X = np.empty((3, m.E, N ** 3))
        for a in range(3):
            X[a] = m.lo[a] + (m.ijk[a][:, None] + self.nodes[loc[a]][None, :]) * m.h[a]
        return X

    def interpolate(self, f):
        """Nodal interpolation of f(x, y, z) -> array (or tuple of arrays)."""
        X = self.node_coords()
        return np.asarray(f(X[0], X[1], X[2]))


# ----------------------------------------------------------------------------
# Quadrature tables of one space at n_q Gauss points per direction.
# ----------------------------------------------------------------------------
class _Tables:
    def __init__(self, space, nq):
        dt = space.dtype
        self.g, self.w = rules.gauss(nq, dt)
        self.V, self.D = rules.lagrange(space.nodes, self.g, dt)      # (nq, N)
        self.V0, self.D0 = rules.lagrange(space.nodes, [0.0], dt)      # (1, N)
        self.V1, self.D1 = rules.lagrange(space.nodes, [1.0], dt)


def _cell_tables(space, nq):
    """Phi (Q^3, N^3), physical gradients dPhi[a] (Q^3, N^3), weights W (Q^3)
    including the Jacobian determinant h_x h_y h_z."""
    t = _Tables(space, nq)
    h = space.mesh.h
    Phi = tensor3(t.V, t.V, t.V)
    dPhi = [tensor3(t.D, t.V, t.V) / h[0], tensor3(t.V, t.D, t.V) / h[1],
            tensor3(t.V, t.V, t.D) / h[2]]
    W = np.kron(t.w, np.kron(t.w, t.w)) * np.prod(h)
    return Phi, dPhi, W


def _face_tables(space, nq, axis, side):
    """Trace tables on the face normal to `axis` at xi_axis = side (0 or 1):
    values (Q^2, N^3), physical normal derivative d/dx_axis (Q^2, N^3) and
    face weights (Q^2) including the face area element."""
    t = _Tables(space, nq)
    h = space.mesh.h
    Vend = t.V1 if side == 1 else t.V0
    Dend = t.D1 if side == 1 else t.D0
    Tv = [t.V, t.V, t.V]
    Td = [t.V, t.V, t.V]
    Tv[axis] = Vend
    Td[axis] = Dend / h[axis]
    val = tensor3(*Tv)
    der = tensor3(*Td)
    wt = [t.w, t.w, t.w]
    wt[axis] = np.ones(1, dtype=space.dtype)
    area = np.prod([h[a] for a in range(3) if a != axis])
    wf = np.kron(wt[2], np.kron(wt[1], wt[0])) * area
    return val, der, wf


def _apply_cell(A, X):
    return X @ A.T


# ----------------------------------------------------------------------------
# Mass and inverse mass: m_h^e(v, u) = (v, u)_Omega_e, Sec. 3.2; the inverse
# is block diagonal and applied exactly, Sec. 3.3.
# ----------------------------------------------------------------------------
class Mass:
    def __init__(self, space):
        self.space = space
        Phi, _, W = _cell_tables(space, space.N)
        self.Me = Phi.T @ (W[:, None] * Phi)

    def apply(self, X):
        """X: (..., E, N^3) -> M X."""
        return X @ self.Me.T

    def apply_inverse(self, X):
        """Dense LU solve with the element mass matrix, cell by cell."""
        X = np.asarray(X)
        flat = X.reshape(-1, X.shape[-1])
        Y = np.linalg.solve(self.Me, flat.T).T
        return Y.reshape(X.shape)


# ----------------------------------------------------------------------------
# SIPG Laplace l_h^e (Sec. 3.2).  Summing the element-boundary terms of both
# neighbours gives, per interior face F with n = n^- and d_n = d/dx_axis:
#   a_F(q, p) = int_F -{d_n q}[p] - [q]{d_n p} + tau [q][p],
#   [p] = p^- - p^+, {d_n p} = (d_n p^- + d_n p^+)/2.
# ----------------------------------------------------------------------------
class Laplace:
    def __init__(self, space, penalty_factor=1.0, coefficient=1.0):
        self.space = space
        nq = space.N
        Phi, dPhi, W = _cell_tables(space, nq)
        self.Ke = coefficient * sum(dP.T @ (W[:, None] * dP) for dP in dPhi)
        self.blocks = []
        for axis in range(3):
            tau = penalty_factor * (space.k + 1) ** 2 / space.mesh.h[axis]
            vm, dm, wf = _face_tables(space, nq, axis, 1)   # e- at xi = 1
            vp, dp, _ = _face_tables(space, nq, axis, 0)    # e+ at xi = 0
            jump = {"-": vm, "+": -vp}
            avgd = {"-": 0.5 * dm, "+": 0.5 * dp}
            B = {}
            for s in "-+":
                for t in "-+":
                    B[s + t] = coefficient * (
                        -avgd[s].T @ (wf[:, None] * jump[t])
                        - jump[s].T @ (wf[:, None] * avgd[t])
                        + tau * jump[s].T @ (wf[:, None] * jump[t]))
            self.blocks.append(B)

    def apply(self, X):
        """X: (E, N^3) or (ncomp, E, N^3)."""
        X = np.asarray(X, dtype=self.space.dtype)
        if X.ndim == 3:
            return np.stack([self.apply(x) for x in X])
        m = self.space.mesh
        Y = _apply_cell(self.Ke, X)
        for axis in range(3):
            B = self.blocks[axis]
            em = np.arange(m.E)
            ep = m.neighbor(axis, +1)
            Y[em] += X[em] @ B["--"].T + X[ep] @ B["-+"].T
            # every element is the '+' side of exactly one face per axis
            Y[ep] += X[em] @ B["+-"].T + X[ep] @ B["++"].T
        return Y

    def diagonal(self):
        """Diagonal of the assembled matrix, (E, N^3)."""
        m = self.space.mesh
        d = np.diag(self.Ke).copy()
        for axis in range(3):
            B = self.blocks[axis]
            d = d + np.diag(B["--"]) + np.diag(B["++"])
            if m.n[axis] == 1:       # the cell is its own neighbour
                d = d + np.diag(B["-+"]) + np.diag(B["+-"])
        return np.tile(d, (m.E, 1))

    def matrix(self):
        """Dense global matrix (small meshes only)."""
        n = self.space.size
        E, nd = self.space.mesh.E, self.space.ndofs_cell
        A = np.empty((n, n))
        for j in range(n):
            x = np.zeros(n)
            x[j] = 1.0
            A[:, j] = self.apply(x.reshape(E, nd)).ravel()
        return A


class Viscous(Laplace):
    """Viscous SIPG term v_h^e with the Laplace formulation F_v = nu grad u
    (Sec. 3.2): nu times the scalar SIPG form, applied per velocity component
    (no coupling between components)."""

    def __init__(self, space, nu, penalty_factor=1.0):
        super().__init__(space, penalty_factor, coefficient=nu)


class Helmholtz:
    """(mass_factor * M + V) of the viscous substep, Sec. 3.3."""

    def __init__(self, space, nu, mass_factor, penalty_factor=1.0):
        self.M = Mass(space)
        self.V = Viscous(space, nu, penalty_factor)
        self.mass_factor = mass_factor

    def apply(self, X):
        return self.mass_factor * self.M.apply(X) + self.V.apply(X)


# ----------------------------------------------------------------------------
# Velocity divergence d_h^e(q, u) = -(grad q, u)_e + (q, {{u}}.n)_de and
# pressure gradient g_h^e(v, p) = -(div v, p)_e + (v, {{p}} n)_de with central
# fluxes (Sec. 3.2).  Both use k_u + 1 Gauss points.  They are assembled
# independently so that D^T = -G is a genuine check.
# ----------------------------------------------------------------------------
class Divergence:
    def __init__(self, space_u, space_p):
        assert space_u.mesh is space_p.mesh
        self.su, self.sp = space_u, space_p
        nq = space_u.N
        Phu, _, W = _cell_tables(space_u, nq)
        Php, dPhp, _ = _cell_tables(space_p, nq)
        # cell: y_p = - sum_a dPhp_a^T W (Phu u_a)
        self.cell = [-(dPhp[a].T @ (W[:, None] * Phu)) for a in range(3)]
        self.faces = []
        for axis in range(3):
            vum, _, wf = _face_tables(space_u, nq, axis, 1)
            vup, _, _ = _face_tables(space_u, nq, axis, 0)
            vpm, _, _ = _face_tables(space_p, nq, axis, 1)
            vpp, _, _ = _face_tables(space_p, nq, axis, 0)
            # [q]{{u}}.n with [q] = q- - q+, {{u_a}} = (u_a- + u_a+)/2
            self.faces.append({
                "--": 0.5 * vpm.T @ (wf[:, None] * vum),
                "-+": 0.5 * vpm.T @ (wf[:, None] * vup),
                "+-": -0.5 * vpp.T @ (wf[:, None] * vum),
                "++": -0.5 * vpp.T @ (wf[:, None] * vup)})

    def apply(self, U):
        """U: (3, E, Nu^3) -> (E, Np^3)."""
        m = self.su.mesh
        Y = sum(U[a] @ self.cell[a].T for a in range(3))
        em = np.arange(m.E)
        for axis in range(3):
            F = self.faces[axis]
            ep = m.neighbor(axis, +1)
            ua = U[axis]
            Y[em] += ua[em] @ F["--"].T + ua[ep] @ F["-+"].T
            Y[ep] += ua[em] @ F["+-"].T + ua[ep] @ F["++"].T
        return Y


class Gradient:
    def __init__(self, space_u, space_p):
        self.su, self.sp = space_u, space_p
        nq = space_u.N
        Phu, dPhu, W = _cell_tables(space_u, nq)
        Php, _, _ = _cell_tables(space_p, nq)
        # cell: y_a = - dPhu_a^T W (Php p)
        self.cell = [-(dPhu[a].T @ (W[:, None] * Php)) for a in range(3)]
        self.faces = []
        for axis in range(3):
            vum, _, wf = _face_tables(space_u, nq, axis, 1)
            vup, _, _ = _face_tables(space_u, nq, axis, 0)
            vpm, _, _ = _face_tables(space_p, nq, axis, 1)
            vpp, _, _ = _face_tables(space_p, nq, axis, 0)
            # [v].n {{p}}: only the normal component of v couples
            self.faces.append({
                "--": 0.5 * vum.T @ (wf[:, None] * vpm),
                "-+": 0.5 * vum.T @ (wf[:, None] * vpp),
                "+-": -0.5 * vup.T @ (wf[:, None] * vpm),
                "++": -0.5 * vup.T @ (wf[:, None] * vpp)})

    def apply(self, P):
        """P: (E, Np^3) -> (3, E, Nu^3)."""
        m = self.su.mesh
        Y = np.stack([P @ self.cell[a].T for a in range(3)])
        em = np.arange(m.E)
        for axis in range(3):
            F = self.faces[axis]
            ep = m.neighbor(axis, +1)
            Y[axis][em] += P[em] @ F["--"].T + P[ep] @ F["-+"].T
            Y[axis][ep] += P[em] @ F["+-"].T + P[ep] @ F["++"].T
        return Y


# ----------------------------------------------------------------------------
# Convective term c_h^e(v, u) = -(grad v, u (x) u)_e
#   + (v, ({{u (x) u}} + max(|u^-.n|, |u^+.n|) [[u]]) . n)_de   (Sec. 3.2)
# evaluated pointwise at nq_conv^3 cell and nq_conv^2 face Gauss points
# (3/2 over-integration).  Returns the weak form C(U) (not M^-1 C).
# ----------------------------------------------------------------------------
class Convective:
    def __init__(self, space, nq=None):
        self.space = space
        self.nq = nq if nq is not None else (3 * (space.k + 1)) // 2
        self.Phi, self.dPhi, self.W = _cell_tables(space, self.nq)
        self.face = []
        for axis in range(3):
            vm, _, wf = _face_tables(space, self.nq, axis, 1)
            vp, _, _ = _face_tables(space, self.nq, axis, 0)
            self.face.append((vm, vp, wf))

    def apply(self, U, cells=None):
        """U: (3, E, N^3) -> C(U): (3, E, N^3).  With `cells` (a list of cell
        ids) only the rows of those cells are computed (the others stay zero):
        their cell terms and the faces that touch them, in the same
        arithmetic."""
        m = self.space.mesh
        U = np.asarray(U, dtype=self.space.dtype)
        sel = np.arange(m.E) if cells is None else np.asarray(cells)
        uq = np.stack([U[c][sel] @ self.Phi.T for c in range(3)])  # (3, |sel|, Q^3)
        Y = np.zeros_like(U)
        for c in range(3):
            for d in range(3):
                F = uq[c] * uq[d] * self.W[None, :]
                Y[c][sel] -= F @ self.dPhi[d]
        for axis in range(3):
            vm, vp, wf = self.face[axis]
            em = np.arange(m.E)
            ep = m.neighbor(axis, +1)
            if cells is not None:       # faces with a selected cell on either side
                keep = np.isin(em, sel) | np.isin(ep, sel)
                em, ep = em[keep], ep[keep]
            um = np.stack([U[c][em] @ vm.T for c in range(3)])     # (3, faces, Q^2)
            up = np.stack([U[c][ep] @ vp.T for c in range(3)])
            unm, unp = um[axis], up[axis]
            lam = np.maximum(np.abs(unm), np.abs(unp))
            for c in range(3):
                Fs = (um[c] * unm + up[c] * unp) / 2 + lam * (um[c] - up[c])
                Fs = Fs * wf[None, :]
                np.add.at(Y[c], em, Fs @ vm)
                np.subtract.at(Y[c], ep, Fs @ vp)
        if cells is not None:
            out = np.zeros_like(Y)
            out[:, sel] = Y[:, sel]
            Y = out
        return Y


    def magnitude(self, U):
        """The sums of apply() over the absolute values of every factor and
        term: |C(U)| <= magnitude(U) elementwise, and magnitude(U) times the
        unit roundoff and the length of the summation chains bounds the
        rounding error of any evaluation order (a running error bound in the
        sense of Higham, Accuracy and Stability of Numerical Algorithms,
        Sec. 3.3).  The weak form nearly cancels for smooth fields, so this
        is the scale against which two evaluations can be compared."""
        m = self.space.mesh
        A = np.abs(np.asarray(U, dtype=np.float64))
        aPhi, adPhi = np.abs(self.Phi), [np.abs(t) for t in self.dPhi]
        uq = np.stack([A[c] @ aPhi.T for c in range(3)])
        Y = np.zeros_like(A)
        for c in range(3):
            for d in range(3):
                Y[c] += (uq[c] * uq[d] * self.W[None, :]) @ adPhi[d]
        em = np.arange(m.E)
        for axis in range(3):
            vm, vp, wf = self.face[axis]
            ep = m.neighbor(axis, +1)
            um = np.stack([A[c][em] @ np.abs(vm).T for c in range(3)])
            up = np.stack([A[c][ep] @ np.abs(vp).T for c in range(3)])
            lam = np.maximum(um[axis], up[axis])
            for c in range(3):
                Fs = (0.5 * (um[c] * um[axis] + up[c] * up[axis]) + lam * (um[c] + up[c])) * wf[None, :]
                Y[c][em] += Fs @ np.abs(vm)
                Y[c][ep] += Fs @ np.abs(vp)
        return Y

    def vjp(self, U, Wt):
        """Vector-Jacobian product (dC/dU)^T Wt, written out pointwise.

        Cell: with g_cd(q) = sum_i Wt_c,i d_d phi_i(q), the cell part of
        <Wt, C(U)> is -sum_q W sum_cd g_cd u_c u_d, whose derivative in u_e(q)
        is -W sum_d (g_ed + g_de) u_d; it is tested with phi_j.
        Face: <Wt, face part> = sum wf sum_c (Wt^-_c - Wt^+_c) F*_c; the
        derivative of F* in u^- and u^+ follows from the product rule, with
        d|s|/ds = sign(s) and d max(a, b) sent to the larger argument (half to
        each on a tie)."""
        m = self.space.mesh
        U = np.asarray(U, dtype=np.float64)
        Wt = np.asarray(Wt, dtype=np.float64)
        uq = [U[c] @ self.Phi.T for c in range(3)]
        g = [[Wt[c] @ self.dPhi[d].T for d in range(3)] for c in range(3)]
        G = np.zeros_like(U)
        for e in range(3):
            ge = -self.W[None, :] * sum((g[e][d] + g[d][e]) * uq[d] for d in range(3))
            G[e] += ge @ self.Phi
        em = np.arange(m.E)
        for axis in range(3):
            vm, vp, wf = self.face[axis]
            ep = m.neighbor(axis, +1)
            um = [U[c][em] @ vm.T for c in range(3)]
            up = [U[c][ep] @ vp.T for c in range(3)]
            jw = [Wt[c][em] @ vm.T - Wt[c][ep] @ vp.T for c in range(3)]
            unm, unp = um[axis], up[axis]
            am, ap = np.abs(unm), np.abs(unp)
            lam = np.maximum(am, ap)
            sm = np.where(am > ap, np.sign(unm), np.where(am == ap, 0.5 * np.sign(unm), 0.0))
            sp = np.where(ap > am, np.sign(unp), np.where(am == ap, 0.5 * np.sign(unp), 0.0))
            jw_um = sum(jw[c] * um[c] for c in range(3))
            jw_up = sum(jw[c] * up[c] for c in range(3))
            jw_du = sum(jw[c] * (um[c] - up[c]) for c in range(3))
            for e in range(3):
                gm = 0.5 * jw[e] * unm + lam * jw[e]
                gp = 0.5 * jw[e] * unp - lam * jw[e]
                if e == axis:
                    gm = gm + 0.5 * jw_um + sm * jw_du
                    gp = gp + 0.5 * jw_up + sp * jw_du
                G[e][em] += (gm * wf[None, :]) @ vm
                G[e][ep] += (gp * wf[None, :]) @ vp
        return G


# ----------------------------------------------------------------------------
# Projection substep with divergence and continuity penalty terms (Sec. 3.2,
# the terms a_D and a_C of the projection step, and the matrix form
# M + A_D + A_C of Sec. 3.3):
#   a_D(v, u) = (div v, tau_D div u)_e,
#   tau_D = zeta_D ||u_ex||_e h / (k_u + 1) dt,
#   a_C(v, u) = sum over interior faces of (v.n, {{tau_C}} [u].n),
#   tau_C = zeta_C ||u_ex||_e dt,
# with ||u_ex||_e the element-wise volume average of the Euclidean norm of
# the extrapolated velocity and h = V_e^(1/3).  Summed over both cells of a
# face the continuity term is int {{tau_C}} (v- - v+).n (u- - u+).n.
# ----------------------------------------------------------------------------
def velocity_norm_average(space, U):
    """(1/V_e) int_e |u| dx per cell, Gauss rule with k+1 points."""
    Phi, _, W = _cell_tables(space, space.N)
    speed = np.sqrt(sum((U[c] @ Phi.T) ** 2 for c in range(3)))
    return (speed * W[None, :]).sum(axis=1) / np.prod(space.mesh.h)


def penalty_parameters(space, U_ex, dt, zeta_d=1.0, zeta_c=1.0):
    nrm = velocity_norm_average(space, U_ex)
    h_eff = np.prod(space.mesh.h) ** (1.0 / 3.0)
    return zeta_d * nrm * h_eff / (space.k + 1) * dt, zeta_c * nrm * dt


class Projection:
    """M + A_D + A_C on a velocity field (3, E, N^3) with per-cell tau_D and
    tau_C (arrays of length E)."""

    def __init__(self, space, tau_d, tau_c):
        self.space = space
        self.tau_d = np.asarray(tau_d, dtype=np.float64)
        self.tau_c = np.asarray(tau_c, dtype=np.float64)
        Phi, dPhi, W = _cell_tables(space, space.N)
        self.Me = Phi.T @ (W[:, None] * Phi)
        self.AD = [[dPhi[b].T @ (W[:, None] * dPhi[a]) for a in range(3)] for b in range(3)]
        self.faces = []
        for axis in range(3):
            vm, _, wf = _face_tables(space, space.N, axis, 1)
            vp, _, _ = _face_tables(space, space.N, axis, 0)
            self.faces.append({"--": vm.T @ (wf[:, None] * vm), "-+": -(vm.T @ (wf[:, None] * vp)),
                               "+-": -(vp.T @ (wf[:, None] * vm)), "++": vp.T @ (wf[:, None] * vp)})

    def apply(self, U, terms="MDC"):
        """(M + A_D + A_C) U, or the sum of the terms named in `terms` (a
        string of "M", "D", "C")."""
        m = self.space.mesh
        U = np.asarray(U, dtype=np.float64)
        Y = np.stack([U[c] @ self.Me.T for c in range(3)]) if "M" in terms else np.zeros_like(U)
        if "D" in terms:
            for b in range(3):
                for a in range(3):
                    Y[b] += self.tau_d[:, None] * (U[a] @ self.AD[b][a].T)
        if "C" not in terms:
            return Y
        em = np.arange(m.E)
        for a in range(3):
            B = self.faces[a]
            ep = m.neighbor(a, +1)
            tc = 0.5 * (self.tau_c[em] + self.tau_c[ep])
            Y[a][em] += tc[:, None] * (U[a][em] @ B["--"].T + U[a][ep] @ B["-+"].T)
            Y[a][ep] += tc[:, None] * (U[a][em] @ B["+-"].T + U[a][ep] @ B["++"].T)
        return Y


# ----------------------------------------------------------------------------
# Diagnostics of Sec. 4.2: kinetic energy and dissipation rate, with the
# element-wise (broken) gradient and k_u + 1 Gauss points.
# ----------------------------------------------------------------------------
def kinetic_energy(space, U):
    Phi, _, W = _cell_tables(space, space.N)
    tot = sum(np.sum((U[c] @ Phi.T) ** 2 * W[None, :]) for c in range(3))
    return 0.5 * tot / space.mesh.volume


def dissipation_rate(space, U, nu):
    _, dPhi, W = _cell_tables(space, space.N)
    tot = 0.0
    for c in range(3):
        for d in range(3):
            tot += np.sum((U[c] @ dPhi[d].T) ** 2 * W[None, :])
    return nu * tot / space.mesh.volume


def dissipation_gradient(space, U, nu):
    """d eps / d U = (2 nu / V) K U per component, K the broken stiffness."""
    _, dPhi, W = _cell_tables(space, space.N)
    K = sum(dP.T @ (W[:, None] * dP) for dP in dPhi)
    return 2.0 * nu / space.mesh.volume * np.stack([U[c] @ K.T for c in range(3)])


def taylor_green(x, y, z):
    """Taylor-Green initial velocity with U0 = L = 1 (Sec. 4)."""
    return (np.sin(x) * np.cos(y) * np.cos(z),
            -np.cos(x) * np.sin(y) * np.cos(z),
            np.zeros_like(x))
