"""Matrix-free GLL spectral-element Poisson/Helmholtz operator (FP64, CPU).

Sec. 5.1: the global operator is never formed.  Its action is the local
element operator applied on each element by GLL quadrature, followed by a
gather-scatter that sums the contributions of nodes shared between elements.
Eq. VelocityEqn gives the Helmholtz form (L + c I) u = f, Eq. PressureEqn the
Poisson form L p = g; here both are A = K + lam * M with K the stiffness
(weak Laplacian) and M the GLL (diagonal) mass matrix, lam = 0 for Poisson.

Domain: the unit box [0,1]^3 split into ex*ey*ez axis-aligned boxes of sides
hx = 1/ex, hy = 1/ey, hz = 1/ez.  Global nodes are numbered
g = ix + nx*(iy + ny*iz), nx = p*ex + 1 (x fastest).  All six faces carry
homogeneous Dirichlet conditions: boundary entries of the input are ignored
(treated as 0) and boundary rows of the output are 0.

This is written element by element in the general "D^T G D" form with an
explicit scatter-add, on purpose: it shares no structure with the GPU kernel.
"""
import numpy as np

from .gll import gll_nodes_weights, gll_derivative


class SemOperator:
    def __init__(self, ex, ey, ez, p, lam=0.0):
        self.ex, self.ey, self.ez, self.p = int(ex), int(ey), int(ez), int(p)
        self.lam = float(lam)
        self.nx, self.ny, self.nz = p * ex + 1, p * ey + 1, p * ez + 1
        self.n = self.nx * self.ny * self.nz
        self.hx, self.hy, self.hz = 1.0 / ex, 1.0 / ey, 1.0 / ez
        self.xi, self.w = gll_nodes_weights(p)
        self.D = gll_derivative(p)
        q = p + 1
        # gather map: element e=(kx,ky,kz), local (i,j,k) -> global index.
        ke = np.arange(ez)[:, None, None, None, None, None]
        je = np.arange(ey)[None, :, None, None, None, None]
        ie = np.arange(ex)[None, None, :, None, None, None]
        k = np.arange(q)[None, None, None, :, None, None]
        j = np.arange(q)[None, None, None, None, :, None]
        i = np.arange(q)[None, None, None, None, None, :]
        gz, gy, gx = p * ke + k, p * je + j, p * ie + i
        self.gidx = (gx + self.nx * (gy + self.ny * gz)).reshape(ex * ey * ez, q, q, q)
        # element arrays are indexed [e, k(z), j(y), i(x)].
        w = self.w
        self.W3 = w[:, None, None] * w[None, :, None] * w[None, None, :]  # [k, j, i]
        self.J = self.hx * self.hy * self.hz / 8.0     # |dx/dxi|
        # G_rr = J * (dxi_r/dx_r)^2; the metric is diagonal for boxes.
        self.Gx = self.J * (2.0 / self.hx) ** 2
        self.Gy = self.J * (2.0 / self.hy) ** 2
        self.Gz = self.J * (2.0 / self.hz) ** 2
        mask = np.ones((self.nz, self.ny, self.nx), dtype=bool)
        mask[0, :, :] = mask[-1, :, :] = False
        mask[:, 0, :] = mask[:, -1, :] = False
        mask[:, :, 0] = mask[:, :, -1] = False
        self.interior = mask.reshape(-1)

    # ------------------------------------------------------------------ geometry
    def coords_1d(self):
        """Global 1D node coordinates in x, y and z (GLL nodes mapped per element)."""
        out = []
        for ne, h in ((self.ex, self.hx), (self.ey, self.hy), (self.ez, self.hz)):
            c = np.empty(self.p * ne + 1)
            for e in range(ne):
                c[e * self.p:(e + 1) * self.p + 1] = e * h + 0.5 * (self.xi + 1.0) * h
            out.append(c)
        return out

    # ------------------------------------------------------------------ operator
    def local_apply(self, U):
        """Local operator on element arrays U[b, e, k, j, i] (Sec. 5.1).

        Gradient by D along each reference direction, scaling by the diagonal
        metric times the quadrature weight, then D^T; plus lam * J * W u.
        """
        D = self.D
        ux = np.einsum('il,bekjl->bekji', D, U)
        uy = np.einsum('jl,bekli->bekji', D, U)
        uz = np.einsum('kl,belji->bekji', D, U)
        W3 = self.W3
        vx, vy, vz = self.Gx * W3 * ux, self.Gy * W3 * uy, self.Gz * W3 * uz
        Y = (np.einsum('li,bekjl->bekji', D, vx)
             + np.einsum('lj,bekli->bekji', D, vy)
             + np.einsum('lk,belji->bekji', D, vz))
        if self.lam != 0.0:
            Y = Y + self.lam * self.J * W3 * U
        return Y

    def apply(self, x, mask=True):
        """y = A x: gather to elements, local operator, scatter-add, mask."""
        x = np.asarray(x, dtype=np.float64)
        single = x.ndim == 1
        X = x[None, :] if single else x
        if mask:
            X = X * self.interior
        U = X[:, self.gidx]
        Y = self.local_apply(U)
        y = np.zeros_like(X)
        nb = X.shape[0]
        for b in range(nb):   # explicit gather-scatter (sum over shared nodes)
            np.add.at(y[b], self.gidx.reshape(-1), Y[b].reshape(-1))
        if mask:
            y = y * self.interior
        return y[0] if single else y

    def diagonal(self):
        """diag(A); 1 on the masked (Dirichlet) nodes, which the PCG ignores.

        Local diagonal of the element operator at node (i,j,k):
        sum_l D_li^2 Gx W_{k,j,l} + sum_l D_lj^2 Gy W_{k,l,i}
        + sum_l D_lk^2 Gz W_{l,j,i} + lam J W_{k,j,i}, then scatter-added.
        """
        D2 = self.D ** 2
        W3 = self.W3
        dx = self.Gx * np.einsum('li,kjl->kji', D2, W3)
        dy = self.Gy * np.einsum('lj,kli->kji', D2, W3)
        dz = self.Gz * np.einsum('lk,lji->kji', D2, W3)
        dl = dx + dy + dz + self.lam * self.J * W3
        d = np.zeros(self.n)
        nel = self.gidx.shape[0]
        np.add.at(d, self.gidx.reshape(-1), np.broadcast_to(dl, (nel,) + dl.shape).reshape(-1))
        d[~self.interior] = 1.0
        return d

    def dense(self, mask=True):
        """Dense assembled matrix by applying A to every unit vector (tiny meshes)."""
        n = self.n
        A = np.zeros((n, n))
        for c0 in range(0, n, 256):
            c1 = min(n, c0 + 256)
            E = np.zeros((c1 - c0, n))
            E[np.arange(c1 - c0), np.arange(c0, c1)] = 1.0
            A[:, c0:c1] = self.apply(E, mask=mask).T
        return A
