"""Independent numerical reference for the oracle pins (numpy / scipy only).

Nothing here is imported by the oracle or by the product package.  The
Dubiner basis is evaluated from its collapsed-coordinate definition with
scipy's Jacobi and Legendre polynomials (a route different from the oracle's
monomial expansion), integrals use Gauss rules from numpy, and the weak form
of Eq. (8) is evaluated pointwise by brute-force quadrature.
"""
from __future__ import annotations

import numpy as np
from scipy.special import eval_jacobi, eval_legendre

KMAX = 15
K_OF_P = (1, 3, 6, 10, 15)
DEG = np.array([0, 1, 1, 2, 2, 2, 3, 3, 3, 3, 4, 4, 4, 4, 4])
MODES = [(d - b, b) for d in range(5) for b in range(d + 1)]  # (a, b), ordered by degree then b


def brute_force_adjacency(tri):
    """(nbr, nbk) [ne,3]: edge k of triangle e joins the two vertices other
    than vertex k; two triangles are neighbours across an edge with the same
    two vertices, nbk the neighbour's local index of it; -1 on the boundary.
    Raises on an edge of more than two triangles."""
    ne = len(tri)
    nbr = np.full((ne, 3), -1, np.int64)
    nbk = np.full((ne, 3), -1, np.int64)
    sides = {}
    for e in range(ne):
        for k in range(3):
            key = tuple(sorted((int(tri[e][(k + 1) % 3]), int(tri[e][(k + 2) % 3]))))
            sides.setdefault(key, []).append((e, k))
    for s in sides.values():
        if len(s) > 2:
            raise ValueError("non-manifold edge")
        if len(s) == 2:
            (a, ka), (b, kb) = s
            nbr[a, ka], nbk[a, ka], nbr[b, kb], nbk[b, kb] = b, kb, a, ka
    return nbr, nbk


def _dleg(n, x):
    # d/dx P_n = n (x P_n - P_{n-1}) / (x^2 - 1), via the Jacobi derivative identity instead:
    # d/dx P_n^{(0,0)} = (n+1)/2 P_{n-1}^{(1,1)}
    if n == 0:
        return np.zeros_like(x)
    return 0.5 * (n + 1) * eval_jacobi(n - 1, 1.0, 1.0, x)


def _djac(n, al, x):
    if n == 0:
        return np.zeros_like(x)
    return 0.5 * (n + al + 1) * eval_jacobi(n - 1, al + 1.0, 1.0, x)


def basis(x, y):
    """phi[i], dphi/dx[i], dphi/dy[i] at points (x, y) with y < 1; shape [15, ...]."""
    x = np.asarray(x, dtype=float)
    y = np.asarray(y, dtype=float)
    m = 1.0 - y
    eta1 = (2.0 * x + y - 1.0) / m
    eta2 = 2.0 * y - 1.0
    v = np.zeros((KMAX,) + x.shape)
    vx = np.zeros_like(v)
    vy = np.zeros_like(v)
    for i, (a, b) in enumerate(MODES):
        N = np.sqrt(2.0 * (2 * a + 1) * (a + b + 1))
        La, dLa = eval_legendre(a, eta1), _dleg(a, eta1)
        Jb, dJb = eval_jacobi(b, 2.0 * a + 1.0, 0.0, eta2), _djac(b, 2.0 * a + 1.0, eta2)
        v[i] = N * La * m ** a * Jb
        # d eta1/dx = 2/m, d eta1/dy = 2x/m^2, d m/dy = -1, d eta2/dy = 2
        vx[i] = N * dLa * 2.0 * m ** (a - 1) * Jb if a >= 1 else 0.0
        t1 = dLa * 2.0 * x * m ** (a - 2) if a >= 1 else 0.0
        t2 = -a * La * m ** (a - 1) if a >= 1 else 0.0
        vy[i] = N * ((t1 + t2) * Jb + La * m ** a * 2.0 * dJb)
    return v, vx, vy


def gauss01(n):
    z, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (z + 1.0), 0.5 * w


def tri_rule(n):
    """Collapsed n x n Gauss rule on the reference triangle (exact to degree 2n-2)."""
    s, w = gauss01(n)
    U, Vv = np.meshgrid(s, s, indexing="ij")
    W = np.outer(w, w) * (1.0 - Vv)
    return (U * (1.0 - Vv)).ravel(), Vv.ravel(), W.ravel()


EDGE = {0: (np.array([1.0, 0.0]), np.array([-1.0, 1.0])),
        1: (np.array([0.0, 1.0]), np.array([0.0, -1.0])),
        2: (np.array([0.0, 0.0]), np.array([1.0, 0.0]))}


def edge_points(k, s):
    p0, d = EDGE[k]
    return p0[0] + d[0] * s, p0[1] + d[1] * s


# ----------------------------------------------------------------------
# brute-force weak form on small meshes
# ----------------------------------------------------------------------
class Tri:
    def __init__(self, xy, tri):
        self.xy = np.asarray(xy, float)
        t = np.array(tri, dtype=np.int64)
        for e in range(len(t)):
            a, b, c = self.xy[t[e]]
            if (b[0] - a[0]) * (c[1] - a[1]) - (c[0] - a[0]) * (b[1] - a[1]) < 0:
                t[e, [1, 2]] = t[e, [2, 1]]
        self.tri = t
        self.ne = len(t)
        self.J = np.zeros((self.ne, 2, 2))
        for e in range(self.ne):
            v0, v1, v2 = self.xy[t[e]]
            self.J[e] = np.column_stack([v1 - v0, v2 - v0])
        self.det = np.linalg.det(self.J)
        self.s = np.sqrt(self.det)
        self.area = 0.5 * self.det
        edges = {}
        for e in range(self.ne):
            for k in range(3):
                a, b = t[e, (k + 1) % 3], t[e, (k + 2) % 3]
                edges.setdefault((min(a, b), max(a, b)), []).append((e, k))
        self.nb = -np.ones((self.ne, 3), np.int64)
        for lst in edges.values():
            if len(lst) == 2:
                (e1, k1), (e2, k2) = lst
                self.nb[e1, k1] = e2
                self.nb[e2, k2] = e1

    def to_ref(self, e, x, y):
        v0 = self.xy[self.tri[e, 0]]
        Ji = np.linalg.inv(self.J[e])
        d = np.stack([x - v0[0], y - v0[1]])
        r = Ji @ d.reshape(2, -1)
        return r[0].reshape(np.shape(x)), r[1].reshape(np.shape(x))

    def to_phys(self, e, xh, yh):
        v0 = self.xy[self.tri[e, 0]]
        J = self.J[e]
        return v0[0] + J[0, 0] * xh + J[0, 1] * yh, v0[1] + J[1, 0] * xh + J[1, 1] * yh

    def phys_basis(self, e, x, y):
        """phi_{e,i}, grad at physical points (orthonormal on Omega_e)."""
        xh, yh = self.to_ref(e, x, y)
        v, vx, vy = basis(xh, yh)
        Ji = np.linalg.inv(self.J[e])
        gx = vx * Ji[0, 0] + vy * Ji[1, 0]
        gy = vx * Ji[0, 1] + vy * Ji[1, 1]
        return v / self.s[e], gx / self.s[e], gy / self.s[e]

    def hb_at(self, e, hv, x, y):
        xh, yh = self.to_ref(e, x, y)
        h = hv[self.tri[e]]
        return h[0] * (1 - xh - yh) + h[1] * xh + h[2] * yh

    def grad_hb(self, e, hv):
        h = hv[self.tri[e]]
        Ji = np.linalg.inv(self.J[e])
        g = np.array([h[1] - h[0], h[2] - h[0]])
        return g @ Ji


def brute_force_rhs(msh: Tri, hv, orders, c, u, g, bc_open=None, xi_hat=0.0, nq=12, fric_lin=0.0, fric_quad=0.0,
                    f_c=0.0):
    """Evaluate Eq. (8) with the LF flux by quadrature of the pointwise fields.

    c[3,15,ne], u[2,15,ne] (same u_Delta as the scheme).  Edges without a
    neighbour are land (mirror state) unless listed in bc_open as (e, k).
    Source r of Eq. (5): g xi grad h_b, bottom friction -tau u with tau =
    fric_lin H + fric_quad |u| evaluated from the element means of H and u
    (Sect. 3), Coriolis f_c (V, -U)."""
    bc_open = set(bc_open or [])
    ne = msh.ne
    K = [K_OF_P[p] for p in orders]
    rhs = np.zeros((3, KMAX, ne))
    xh, yh, wq = tri_rule(nq)
    sg, wg = gauss01(nq)

    def fields(e, x, y):
        ph, _, _ = msh.phys_basis(e, x, y)
        k = K[e]
        xi = np.tensordot(c[0, :k, e], ph[:k], 1)
        U = np.tensordot(c[1, :k, e], ph[:k], 1)
        V = np.tensordot(c[2, :k, e], ph[:k], 1)
        uu = np.tensordot(u[0, :k, e], ph[:k], 1)
        vv = np.tensordot(u[1, :k, e], ph[:k], 1)
        return xi, U, V, uu, vv

    for e in range(ne):
        k = K[e]
        x, y = msh.to_phys(e, xh, yh)
        w = wq * msh.det[e]
        ph, gx, gy = msh.phys_basis(e, x, y)
        xi, U, V, uu, vv = fields(e, x, y)
        hb = msh.hb_at(e, hv, x, y)
        P = g * xi * (0.5 * xi + hb)
        A = [(U, V), (U * uu + P, U * vv), (V * uu, V * vv + P)]
        dh = msh.grad_hb(e, hv)
        # element means by quadrature of the pointwise fields
        Hm = np.sum(w * (xi + hb)) / msh.area[e]
        um, vm = np.sum(w * uu) / msh.area[e], np.sum(w * vv) / msh.area[e]
        tau = fric_lin * Hm + fric_quad * np.hypot(um, vm)
        r = [np.zeros(0), g * xi * dh[0] - tau * uu + f_c * V, g * xi * dh[1] - tau * vv - f_c * U]
        for q in range(k):
            for f in range(3):
                val = np.sum(w * (A[f][0] * gx[q] + A[f][1] * gy[q]))
                if f > 0:
                    val += np.sum(w * r[f] * ph[q])
                rhs[f, q, e] += val
        # edges
        for kk in range(3):
            a = msh.xy[msh.tri[e, (kk + 1) % 3]]
            b = msh.xy[msh.tri[e, (kk + 2) % 3]]
            L = np.hypot(*(b - a))
            nx, ny = (b[1] - a[1]) / L, -(b[0] - a[0]) / L
            xe = a[0] + (b[0] - a[0]) * sg
            ye = a[1] + (b[1] - a[1]) * sg
            mid = 0.5 * (a + b)
            xi, U, V, uu, vv = fields(e, xe, ye)
            hb = msh.hb_at(e, hv, xe, ye)
            hmid = msh.hb_at(e, hv, np.array([mid[0]]), np.array([mid[1]]))[0]
            ra = 1.0 / np.sqrt(msh.area[e])
            ub_a = np.array([u[0, 0, e], u[1, 0, e]]) * ra
            Ha = c[0, 0, e] * ra + hmid
            n = msh.nb[e, kk]
            if n >= 0:
                xo, Uo, Vo, uo, vo = fields(n, xe, ye)
                rb = 1.0 / np.sqrt(msh.area[n])
                ub_b = np.array([u[0, 0, n], u[1, 0, n]]) * rb
                Hb = c[0, 0, n] * rb + hmid
            elif (e, kk) in bc_open:
                xo = np.full_like(xi, xi_hat); Uo, Vo, uo, vo = U, V, uu, vv
                ub_b = ub_a
                Hb = xi_hat + hmid
            else:
                qn = U * nx + V * ny
                wn = uu * nx + vv * ny
                xo, Uo, Vo = xi, U - 2 * qn * nx, V - 2 * qn * ny
                uo, vo = uu - 2 * wn * nx, vv - 2 * wn * ny
                ub_b = ub_a - 2 * (ub_a @ [nx, ny]) * np.array([nx, ny])
                Hb = Ha
            lam = max(abs(ub_a @ [nx, ny]), abs(ub_b @ [nx, ny])) + max(np.sqrt(g * Ha), np.sqrt(g * Hb))

            def An(xi_, U_, V_, u_, v_):
                P_ = g * xi_ * (0.5 * xi_ + hb)
                un = u_ * nx + v_ * ny
                return (U_ * nx + V_ * ny, U_ * un + P_ * nx, V_ * un + P_ * ny)

            Fa = An(xi, U, V, uu, vv)
            Fb = An(xo, Uo, Vo, uo, vo)
            ca = (xi, U, V)
            cb = (xo, Uo, Vo)
            phe, _, _ = msh.phys_basis(e, xe, ye)
            for f in range(3):
                Fh = 0.5 * (Fa[f] + Fb[f] + lam * (ca[f] - cb[f]))
                for q in range(k):
                    rhs[f, q, e] -= L * np.sum(wg * Fh * phe[q])
    return rhs


def solve_u(msh: Tri, hv, orders, c, nq=12):
    """Truncated auxiliary system of Sect. 3 assembled by quadrature:
    M[i,j] = int (sum_{n < K(max deg)} xi_n phi_n + h_b, truncated) phi_i phi_j."""
    xh, yh, wq = tri_rule(nq)
    u = np.zeros((2, KMAX, msh.ne))
    for e in range(msh.ne):
        k = K_OF_P[orders[e]]
        x, y = msh.to_phys(e, xh, yh)
        w = wq * msh.det[e]
        ph, _, _ = msh.phys_basis(e, x, y)
        hb = msh.hb_at(e, hv, x, y)
        # modal h_b (exact: h_b is P1)
        hbm = np.array([np.sum(w * hb * ph[i]) for i in range(3)])
        M = np.zeros((k, k))
        for i in range(k):
            for j in range(k):
                d = max(DEG[i], DEG[j])
                kt = K_OF_P[d]
                H = np.zeros_like(x)
                for nn in range(kt):
                    Hn = (c[0, nn, e] if nn < k else 0.0) + (hbm[nn] if nn < 3 else 0.0)
                    H = H + Hn * ph[nn]
                M[i, j] = np.sum(w * H * ph[i] * ph[j])
        u[0, :k, e] = np.linalg.solve(M, c[1, :k, e])
        u[1, :k, e] = np.linalg.solve(M, c[2, :k, e])
    return u
