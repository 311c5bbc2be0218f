"""Energy, gradient and Hessian of the implicit-Euler incremental potential (Sec. 3).

E(x) = sum_v m_v/(2h^2) |x_v - z_v|^2 + sum_e V_e Psi(F_e)            (Eq. 1, Sec. 3)

Psi is the stable Neo-Hookean energy cited in the Table 1 caption. The paper gives no
formula; the form used here (reading R1) is the rest-stable one

    Psi(F) = mu/2 (tr F^T F - 3) - mu (J - 1) + lam'/2 (J - 1)^2,   lam' = lam + mu,

whose linearisation at F = I is linear elasticity with Lame parameters (mu, lam).
Plain numpy, FP64, vectorised over elements only.

Test infrastructure: only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs use this module; the CUDA path never imports it.
"""
from __future__ import annotations

import numpy as np

# --------------------------------------------------------------------------- material


def lame(E, nu):
    """Lame parameters from Young's modulus and Poisson ratio; returns (mu, lam' = lam+mu)."""
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    mu = E / (2.0 * (1.0 + nu))
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    return mu, lam + mu


def cofactor(F):
    """cof F = dJ/dF (J = det F): columns are cross products of the other two columns."""
    c0, c1, c2 = F[..., :, 0], F[..., :, 1], F[..., :, 2]
    return np.stack([np.cross(c1, c2), np.cross(c2, c0), np.cross(c0, c1)], axis=-1)


def snh_psi(F, mu, lp):
    J = np.linalg.det(F)
    return 0.5 * mu * (np.einsum("...ij,...ij->...", F, F) - 3.0) - mu * (J - 1.0) \
        + 0.5 * lp * (J - 1.0) ** 2


def snh_P(F, mu, lp):
    """First Piola stress dPsi/dF = mu F + (lam'(J-1) - mu) cof F."""
    mu = np.asarray(mu, dtype=np.float64)
    lp = np.asarray(lp, dtype=np.float64)
    J = np.linalg.det(F)
    s = lp * (J - 1.0) - mu
    return mu[..., None, None] * F + s[..., None, None] * cofactor(F)


_EPS = np.zeros((3, 3, 3))
_EPS[0, 1, 2] = _EPS[1, 2, 0] = _EPS[2, 0, 1] = 1.0
_EPS[0, 2, 1] = _EPS[2, 1, 0] = _EPS[1, 0, 2] = -1.0


def det_hessian(F):
    """d^2 J / dF_ij dF_kl = eps_ikm eps_jln F_mn, as a 9x9 in row-major (3i+j) order."""
    H = np.einsum("ikm,jln,...mn->...ijkl", _EPS, _EPS, F)
    return H.reshape(F.shape[:-2] + (9, 9))


def snh_dPdF(F, mu, lp):
    """dP/dF (9x9, index 3i+j) = mu I + lam' g g^T + (lam'(J-1) - mu) d^2J/dF^2."""
    J = np.linalg.det(F)
    g = cofactor(F).reshape(F.shape[:-2] + (9,))
    s = lp * (J - 1.0) - mu
    mu = np.asarray(mu)
    lp = np.asarray(lp)
    return (mu[..., None, None] * np.eye(9) + lp[..., None, None] * g[..., :, None] * g[..., None, :]
            + s[..., None, None] * det_hessian(F))


def psd_clamp(A):
    """Symmetric eigen-decomposition with negative eigenvalues clamped to zero (R7)."""
    w, Q = np.linalg.eigh(0.5 * (A + np.swapaxes(A, -1, -2)))
    return np.einsum("...ik,...k,...jk->...ij", Q, np.maximum(w, 0.0), Q)


# --------------------------------------------------------------------------- mesh


class Mesh:
    """Rest-shape quantities of a tet mesh (Sec. 3): D_m^{-1}, volumes, lumped masses.

    b_1..b_3 are the rows of B = D_m^{-1} (D_m columns are X_k - X_0), b_0 = -sum b_k,
    so F = sum_a x_a b_a^T. Lumped mass m_v = sum over incident tets of rho V_e / 4.
    """

    def __init__(self, X, tets, youngs, poisson, density, pinned):
        self.X = np.asarray(X, dtype=np.float64)
        self.tets = np.asarray(tets, dtype=np.int64)
        T = self.tets.shape[0]
        V = self.X.shape[0]
        Dm = np.stack([self.X[self.tets[:, k]] - self.X[self.tets[:, 0]] for k in (1, 2, 3)], axis=-1)
        det = np.linalg.det(Dm)
        if T and det.min() <= 0:
            raise ValueError("non-positive tet volume")
        self.vol = det / 6.0
        B = np.linalg.inv(Dm) if T else np.zeros((0, 3, 3))
        self.b = np.empty((T, 4, 3))
        self.b[:, 1:, :] = B
        self.b[:, 0, :] = -B.sum(axis=1)
        self.youngs = np.asarray(youngs, dtype=np.float64)
        self.poisson = np.asarray(poisson, dtype=np.float64)
        self.mu, self.lp = lame(youngs, poisson)
        self.rho = np.asarray(density, dtype=np.float64)
        self.mass = np.zeros(V)
        np.add.at(self.mass, self.tets.ravel(), np.repeat(self.rho * self.vol / 4.0, 4))
        self.pinned = np.asarray(pinned).astype(bool)
        self.free = np.nonzero(~self.pinned)[0]
        self.dof_of = -np.ones(V, dtype=np.int64)
        self.dof_of[self.free] = np.arange(self.free.size)
        # body = connected component of the tet graph (for per-body precompute)
        parent = np.arange(V)

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a
        for t in self.tets:
            r0 = find(t[0])
            for v in t[1:]:
                r = find(v)
                if r != r0:
                    parent[r] = r0
        roots = np.array([find(v) for v in range(V)])
        # bodies are numbered by their smallest vertex index (caller order)
        first = {}
        for v in range(V):
            first.setdefault(int(roots[v]), len(first))
        self.body_of_vertex = np.array([first[int(r)] for r in roots], dtype=np.int64)
        self.n_bodies = len(first)
        self.body_of_tet = self.body_of_vertex[self.tets[:, 0]] if T else np.zeros(0, int)
        self.contact = None   # oracle.contact.Contact when the IPC barrier is on (Sec. 7)
        self.rc = 0.0         # candidate radius of the step truncation

    def enable_contact(self, planes, dhat, kappa, rc=None, use_penalty=False, friction_mu=0.0,
                       friction_eps_v=1e-3):
        from . import contact
        self.contact = contact.Contact(self.tets, self.X, planes, dhat, kappa, self.pinned, use_penalty,
                                       friction_mu, friction_eps_v)
        self.rc = 2.0 * dhat if rc is None else float(rc)
        return self

    @property
    def V(self):
        return self.X.shape[0]

    @property
    def T(self):
        return self.tets.shape[0]

    def D(self):
        """Per-element 9x12 map from x_e = [x_0; x_1; x_2; x_3] to vec(F) (3i+j)."""
        T = self.T
        D = np.zeros((T, 9, 12))
        for a in range(4):
            for i in range(3):
                D[:, 3 * i:3 * i + 3, 3 * a + i] = self.b[:, a, :]
        return D


def deformation_gradient(mesh: Mesh, x):
    """F_e = sum_a x_a b_a^T for every element."""
    xe = x[mesh.tets]  # (T,4,3)
    return np.einsum("tai,taj->tij", xe, mesh.b)


# --------------------------------------------------------------------------- energy


def inertia_target(x_t, v_t, h, gravity):
    """z = x_t + h v_t + h^2 M^{-1} f_ext with f_ext = M g (Sec. 3)."""
    return x_t + h * v_t + h * h * np.asarray(gravity)[None, :]


def energy(mesh: Mesh, x, z, h):
    """E(x) over free vertices' inertia plus all elements' elastic energy (Eq. 1)."""
    F = deformation_gradient(mesh, x)
    el = float(np.sum(mesh.vol * snh_psi(F, mesh.mu, mesh.lp)))
    d = (x - z)[mesh.free]
    e = el + float(np.sum(0.5 * mesh.mass[mesh.free] / h ** 2 * np.sum(d * d, axis=1)))
    if mesh.contact is not None:
        e += mesh.contact.energy(x, mesh.contact.pairs(x, mesh.contact.dhat))
        e += mesh.contact.friction_energy(x)
    return e


def vertex_gradient(mesh: Mesh, x, z, h):
    """Assembled gradient g_v (V,3); rows of pinned vertices are zero (not DOFs)."""
    F = deformation_gradient(mesh, x)
    P = snh_P(F, mesh.mu, mesh.lp)
    ge = mesh.vol[:, None, None] * np.einsum("tij,taj->tai", P, mesh.b)
    g = np.zeros_like(x)
    np.add.at(g, mesh.tets.ravel(), ge.reshape(-1, 3))
    g += mesh.mass[:, None] / h ** 2 * (x - z)
    if mesh.contact is not None:
        gb, _ = mesh.contact.vertex_terms(x, mesh.contact.pairs(x, mesh.contact.dhat), mesh.V)
        g += gb
        g += mesh.contact.friction_terms(x, mesh.V)[0]
    g[mesh.pinned] = 0.0
    return g


def element_dPdF(mesh: Mesh, x, psd=False):
    F = deformation_gradient(mesh, x)
    A = snh_dPdF(F, mesh.mu, mesh.lp)
    return psd_clamp(A) if psd else A


def element_hessians(mesh: Mesh, x, h, psd=False, inertia=True):
    """12x12 Hessian of E_hat_e = V_e Psi(F_e) + sum_{a in e} (rho V_e/4)/(2h^2)|x_a - z_a|^2.

    Summed over elements (free rows only) this is the Hessian of E exactly.
    """
    A = element_dPdF(mesh, x, psd)
    D = mesh.D()
    He = mesh.vol[:, None, None] * np.einsum("tpi,tpq,tqj->tij", D, A, D)
    if inertia:
        He += (mesh.rho * mesh.vol / 4.0 / h ** 2)[:, None, None] * np.eye(12)[None]
    return He


def vertex_diag_blocks(mesh: Mesh, x, h):
    """H_vv (V,3,3): inertia m_v/h^2 I plus the incident elements' diagonal 3x3 blocks."""
    He = element_hessians(mesh, x, h, psd=False, inertia=False)
    Hd = np.zeros((mesh.V, 3, 3))
    for a in range(4):
        np.add.at(Hd, mesh.tets[:, a], He[:, 3 * a:3 * a + 3, 3 * a:3 * a + 3])
    Hd += (mesh.mass / h ** 2)[:, None, None] * np.eye(3)[None]
    if mesh.contact is not None:
        _, Hb = mesh.contact.vertex_terms(x, mesh.contact.pairs(x, mesh.contact.dhat), mesh.V)
        Hd += Hb
        Hd += mesh.contact.friction_terms(x, mesh.V)[1]
    return Hd


def global_hessian(mesh: Mesh, x, h, psd=False, dense=True):
    """Hessian of E over free DOFs (3 per free vertex), assembled from element blocks."""
    import scipy.sparse as sp
    He = element_hessians(mesh, x, h, psd=psd, inertia=False)
    n = 3 * mesh.free.size
    dofs = np.repeat(3 * mesh.dof_of[mesh.tets], 3, axis=1) + np.tile(np.arange(3), 4)[None, :]
    rows = np.broadcast_to(dofs[:, :, None], He.shape)
    cols = np.broadcast_to(dofs[:, None, :], He.shape)
    ok = (rows >= 0) & (cols >= 0)
    H = sp.coo_matrix((He[ok], (rows[ok], cols[ok])), shape=(n, n)).tocsr()
    H = H + sp.diags(np.repeat(mesh.mass[mesh.free] / h ** 2, 3))
    return H.toarray() if dense else H.tocsc()


def free_vector(mesh: Mesh, g):
    return g[mesh.free].reshape(-1)


def energy_change(mesh: Mesh, x, z, h, d, alphas):
    """E(x + a d) - E(x) for each a, without the cancellation of a plain difference.

    Per element, with G = a dF (dF = sum_a d_a b_a^T):
      det(F + G) - det F = cof(F):G + F:cof(G) + det G                 (exact for 3x3)
      Psi(F+G) - Psi(F) = mu/2 (2 F:G + G:G) - mu dJ + lam'/2 dJ (dJ + 2 (J - 1))
    and per free vertex m/(2h^2) (2 a d.(x - z) + a^2 |d|^2).
    """
    F = deformation_gradient(mesh, x)
    dd = d.copy()
    dd[mesh.pinned] = 0.0
    dF = deformation_gradient(mesh, dd)
    C = cofactor(F)
    cdF = cofactor(dF)
    J = np.linalg.det(F)
    FdF = np.einsum("tij,tij->t", F, dF)
    dFdF = np.einsum("tij,tij->t", dF, dF)
    CdF = np.einsum("tij,tij->t", C, dF)
    FcdF = np.einsum("tij,tij->t", F, cdF)
    detdF = np.linalg.det(dF)
    fr = mesh.free
    de = np.sum(dd[fr] * (x - z)[fr], axis=1)
    d2 = np.sum(dd[fr] * dd[fr], axis=1)
    out = []
    for a in alphas:
        dJ = a * CdF + a * a * FcdF + a ** 3 * detdF
        dpsi = 0.5 * mesh.mu * (2 * a * FdF + a * a * dFdF) - mesh.mu * dJ + 0.5 * mesh.lp * dJ * (dJ + 2 * (J - 1))
        dine = 0.5 * mesh.mass[fr] / h ** 2 * (2 * a * de + a * a * d2)
        out.append(float(np.sum(mesh.vol * dpsi) + np.sum(dine)))
    return out
