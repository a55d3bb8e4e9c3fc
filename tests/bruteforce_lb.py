"""Definition-level binary-fluid D3Q19 step, independent of the oracle.

Written from the model's definitions rather than from its expanded formulas,
so that it can pin the oracle on tiny lattices:

* chemical potential mu = dF/dphi of the discrete free energy
  F = sum_x [A/2 phi^2 + B/4 phi^4 + kappa/2 sum_a (phi(x+e_a) - phi(x))^2],
  taken numerically by complex step, one site at a time;
* pressure from thermodynamics, P = (phi mu - psi) I + kappa grad phi grad phi
  with psi the local free-energy density (central-difference gradient);
* equilibria as the unique member of span{w_i, w_i c_i, w_i Q_i} whose
  zeroth, first and second moments equal (rho, j, rho cs2 I + P + j j/rho)
  for f and (phi, phi u, Gamma mu I + phi u u) for g, found by a linear solve;
* streaming through an explicit permutation of site indices.

O(N^2) per step: for lattices of a few hundred sites only.
"""
from __future__ import annotations

import numpy as np

# rest, 6 faces, 12 edges: a different order from the oracle's enumeration
VEL = np.array([
    [0, 0, 0],
    [1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
    [1, 1, 0], [-1, -1, 0], [1, -1, 0], [-1, 1, 0],
    [1, 0, 1], [-1, 0, -1], [1, 0, -1], [-1, 0, 1],
    [0, 1, 1], [0, -1, -1], [0, 1, -1], [0, -1, 1]])
_C2 = (VEL ** 2).sum(1)
W = np.select([_C2 == 0, _C2 == 1, _C2 == 2], [1 / 3, 1 / 18, 1 / 36])
CS2 = 1.0 / 3.0
_PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def _basis():
    """Columns: w_i * {1, c_a, Q_ab (a<=b)}; rows: moments {1, c_a, c_a c_b}."""
    cols = [W.copy()]
    for a in range(3):
        cols.append(W * VEL[:, a])
    for a, b in _PAIRS:
        cols.append(W * (VEL[:, a] * VEL[:, b] - (CS2 if a == b else 0.0)))
    Bm = np.array(cols).T                      # [19, 10]
    rows = [np.ones(19)] + [VEL[:, a].astype(float) for a in range(3)]
    rows += [(VEL[:, a] * VEL[:, b]).astype(float) for a, b in _PAIRS]
    Mom = np.array(rows)                        # [10, 19]
    return Bm, Mom


_BM, _MOM = _basis()
_SYS = _MOM @ _BM                               # [10, 10]


def equilibrium_from_moments(m0, m1, m2):
    """m0 [N], m1 [3,N], m2 [3,3,N] -> distribution [19,N]."""
    rhs = [m0] + [m1[a] for a in range(3)] + [m2[a, b] for a, b in _PAIRS]
    coef = np.linalg.solve(_SYS, np.array(rhs))
    return _BM @ coef


def _free_energy(phi3, A, B, kappa):
    e = A / 2 * phi3 ** 2 + B / 4 * phi3 ** 4
    for ax in range(3):
        d = np.roll(phi3, -1, axis=ax) - phi3
        e = e + kappa / 2 * d ** 2
    return e.sum()


def chemical_potential(phi3, A, B, kappa, h=1e-30):
    """mu(x) = dF/dphi(x) by complex step on the discrete free energy."""
    mu = np.zeros(phi3.size)
    flat = phi3.reshape(-1).astype(complex)
    for s in range(flat.size):
        p = flat.copy()
        p[s] += 1j * h
        mu[s] = _free_energy(p.reshape(phi3.shape), A, B, kappa).imag / h
    return mu.reshape(phi3.shape)


def _central_grad(phi3):
    # arrays are [z, y, x]; axis 2 is x
    return [(np.roll(phi3, -1, axis=2 - a) - np.roll(phi3, 1, axis=2 - a)) / 2 for a in range(3)]


def _perm(dims):
    nx, ny, nz = dims
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    x, y, z = x.reshape(-1), y.reshape(-1), z.reshape(-1)
    P = np.zeros((19, nx * ny * nz), dtype=np.int64)
    for i, c in enumerate(VEL):
        P[i] = (x + c[0]) % nx + nx * (((y + c[1]) % ny) + ny * ((z + c[2]) % nz))
    return P


def equilibria(dims, prm, rho, j, phi):
    nx, ny, nz = dims
    A, B, kappa, gam = prm["A"], prm["B"], prm["kappa"], prm["gamma"]
    phi3 = phi.reshape(nz, ny, nx)
    mu = chemical_potential(phi3, A, B, kappa).reshape(-1)
    grad = [g.reshape(-1) for g in _central_grad(phi3)]
    psi = A / 2 * phi ** 2 + B / 4 * phi ** 4 + kappa / 2 * sum(g ** 2 for g in grad)
    n = phi.size
    u = j / rho
    P = np.zeros((3, 3, n))
    for a in range(3):
        P[a, a] += phi * mu - psi
        for b in range(3):
            P[a, b] += kappa * grad[a] * grad[b]
    m2f = P + np.einsum("an,bn->abn", j, j) / rho
    for a in range(3):
        m2f[a, a] += rho * CS2
    m2g = phi * np.einsum("an,bn->abn", u, u)
    for a in range(3):
        m2g[a, a] += gam * mu
    feq = equilibrium_from_moments(rho, j, m2f)
    geq = equilibrium_from_moments(phi, phi * u, m2g)
    return feq, geq


def step(dims, prm, f, g, nsteps=1):
    """f, g [19,N] in VEL order (post-streaming state); returns new arrays."""
    perm = _perm(dims)
    f = np.array(f, dtype=float)
    g = np.array(g, dtype=float)
    for _ in range(nsteps):
        rho = f.sum(0)
        j = VEL.T.astype(float) @ f
        phi = g.sum(0)
        feq, geq = equilibria(dims, prm, rho, j, phi)
        fs = f - (f - feq) / prm["tau"]
        gs = g - (g - geq) / prm["tau_g"]
        fn = np.empty_like(f)
        gn = np.empty_like(g)
        for i in range(19):
            fn[i, perm[i]] = fs[i]
            gn[i, perm[i]] = gs[i]
        f, g = fn, gn
    return f, g


def map_order(c_from, c_to):
    """Index array m with c_to[m[k]] == c_from[k] ... returns m: to-index of each from-row."""
    idx = []
    for c in c_from:
        hits = np.where((c_to == c).all(1))[0]
        assert len(hits) == 1
        idx.append(int(hits[0]))
    return np.array(idx)
