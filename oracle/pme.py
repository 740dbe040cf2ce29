"""FP64 smooth particle-mesh Ewald (Essmann et al. 1995), the PME of Sec. 2.1.2.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper builds the B-splines from their recursive definition and carries
the reciprocal sum with an FFT; this module does the same, step by step:

  1. fractional coordinates u_d = K_d x_d / L_d (positions wrapped into [0, L));
  2. cardinal B-spline weights by the recursion
       M_2(u) = 1 - |u - 1|  on [0, 2],
       M_n(u) = u/(n-1) M_{n-1}(u) + (n-u)/(n-1) M_{n-1}(u-1),
     derivative M_n'(u) = M_{n-1}(u) - M_{n-1}(u-1);
     atom i touches grid points (floor(u_d) - j) mod K_d, j = 0..n-1,
     with weight M_n(u_d - floor(u_d) + j);
  3. charge grid Q(k) = sum_i q_i prod_d M_n(...);
  4. E = ke/(2 pi V) sum_{m != 0} exp(-pi^2 |m|^2/alpha^2)/|m|^2 B(m) |FFT(Q)(m)|^2,
     B(m) = prod_d |b_d(m_d)|^2,
     |b_d(m)|^2 = 1 / |sum_{k=0}^{n-2} M_n(k+1) exp(2 pi i m k / K_d)|^2;
  5. phi = inverse DFT (unnormalised) of G(m) FFT(Q)(m), G = 2 x the energy kernel,
     so that E = 1/2 sum_k Q(k) phi(k) and F_i = -sum_k dQ(k)/dx_i phi(k).

No exclusion correction and no self term here: those belong to the real-space
part (oracle.nonbonded).
"""
import numpy as np


def bspline(n, u):
    """Cardinal B-spline M_n(u) by the recursive definition (vectorised over u)."""
    u = np.asarray(u, dtype=np.float64)
    if n == 2:
        return np.where((u >= 0.0) & (u <= 2.0), 1.0 - np.abs(u - 1.0), 0.0)
    return u / (n - 1) * bspline(n - 1, u) + (n - u) / (n - 1) * bspline(n - 1, u - 1.0)


def dbspline(n, u):
    """dM_n/du = M_{n-1}(u) - M_{n-1}(u - 1)."""
    return bspline(n - 1, u) - bspline(n - 1, u - 1.0)


def d2bspline(n, u):
    """d^2 M_n/du^2 = M_{n-2}(u) - 2 M_{n-2}(u - 1) + M_{n-2}(u - 2) (the derivative rule twice)."""
    return bspline(n - 2, u) - 2.0 * bspline(n - 2, u - 1.0) + bspline(n - 2, u - 2.0)


def bspline_moduli(n, K):
    """|b(m)|^2 for m = 0..K-1 (Essmann Eq. 4.4 modulus)."""
    m = np.arange(K)
    k = np.arange(n - 1)
    w = bspline(n, k + 1.0)
    s = (w[None, :] * np.exp(2j * np.pi * m[:, None] * k[None, :] / K)).sum(axis=1)
    return 1.0 / np.abs(s) ** 2


def _weights(x, box, K, n):
    """Per atom and axis: grid indices (N,3,n), weights (N,3,n), dweights/dx (N,3,n)."""
    L = np.asarray(box, dtype=np.float64)
    xw = x - L * np.floor(x / L)
    u = xw / L * K
    fl = np.floor(u)
    fr = u - fl
    j = np.arange(n)
    idx = (fl[:, :, None].astype(np.int64) - j[None, None, :]) % K[None, :, None]
    t = fr[:, :, None] + j[None, None, :]
    w = bspline(n, t)
    dw = dbspline(n, t) * (K / L)[None, :, None]
    return idx, w, dw


def _weights2(x, box, K, n):
    """As _weights, plus second derivatives d^2 weights / dx^2 (N,3,n)."""
    L = np.asarray(box, dtype=np.float64)
    xw = x - L * np.floor(x / L)
    u = xw / L * K
    fl = np.floor(u)
    fr = u - fl
    j = np.arange(n)
    idx = (fl[:, :, None].astype(np.int64) - j[None, None, :]) % K[None, :, None]
    t = fr[:, :, None] + j[None, None, :]
    s = (K / L)[None, :, None]
    return idx, bspline(n, t), dbspline(n, t) * s, d2bspline(n, t) * s * s


def _green(K, L, alpha, ke, n):
    V = float(np.prod(L))
    m = [np.fft.fftfreq(int(K[d])) * K[d] / L[d] for d in range(3)]
    m2 = m[0][:, None, None] ** 2 + m[1][None, :, None] ** 2 + m[2][None, None, :] ** 2
    B = (bspline_moduli(n, int(K[0]))[:, None, None] * bspline_moduli(n, int(K[1]))[None, :, None]
         * bspline_moduli(n, int(K[2]))[None, None, :])
    with np.errstate(divide="ignore", invalid="ignore"):
        G = ke / (np.pi * V) * np.exp(-np.pi ** 2 * m2 / alpha ** 2) / m2 * B
    G[0, 0, 0] = 0.0
    return G


def pme_force_vjp(x, q, box, alpha, ke, K, lam, order=4):
    """Vector-Jacobian product of the reciprocal-space forces (the NEXT row of the force
    VJP): with F_i = -q_i sum_k grad theta_i(k) phi(k), phi = C Q (C the symmetric
    convolution of step 5), returns gx_j = d(lam . F)/dx_j and gq_j = d(lam . F)/dq_j:

      lam . F = -<psi, phi>,  psi(k) = sum_i q_i lam_i . grad theta_i(k)
      gx_j = -q_j sum_k (Hess theta_j(k) lam_j) phi(k) - q_j sum_k grad theta_j(k) chi(k)
      gq_j = -sum_k (lam_j . grad theta_j(k)) phi(k) - sum_k theta_j(k) chi(k),  chi = C psi.
    """
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64).reshape(-1, 3)
    L = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    K = np.broadcast_to(np.asarray(K, dtype=np.int64), (3,)).copy()
    n = order
    idx, w, dw, d2w = _weights2(x, L, K, n)
    G = _green(K, L, alpha, ke, n)
    scale = float(np.prod(K))

    def conv(M):
        return np.real(np.fft.ifftn(G * np.fft.fftn(M))) * scale
    Q = np.zeros(tuple(K))
    psi = np.zeros(tuple(K))
    N = x.shape[0]
    for a in range(n):
        for b in range(n):
            for c in range(n):
                ii = (idx[:, 0, a], idx[:, 1, b], idx[:, 2, c])
                th = w[:, 0, a] * w[:, 1, b] * w[:, 2, c]
                gth = np.stack([dw[:, 0, a] * w[:, 1, b] * w[:, 2, c], w[:, 0, a] * dw[:, 1, b] * w[:, 2, c],
                                w[:, 0, a] * w[:, 1, b] * dw[:, 2, c]], axis=1)
                np.add.at(Q, ii, q * th)
                np.add.at(psi, ii, q * np.sum(lam * gth, axis=1))
    phi = conv(Q)
    chi = conv(psi)
    gx = np.zeros((N, 3))
    gq = np.zeros(N)
    for a in range(n):
        for b in range(n):
            for c in range(n):
                ii = (idx[:, 0, a], idx[:, 1, b], idx[:, 2, c])
                p, h = phi[ii], chi[ii]
                W = [w[:, 0, a], w[:, 1, b], w[:, 2, c]]
                D = [dw[:, 0, a], dw[:, 1, b], dw[:, 2, c]]
                D2 = [d2w[:, 0, a], d2w[:, 1, b], d2w[:, 2, c]]
                th = W[0] * W[1] * W[2]
                gth = np.stack([D[0] * W[1] * W[2], W[0] * D[1] * W[2], W[0] * W[1] * D[2]], axis=1)
                H = np.empty((N, 3, 3))
                for d in range(3):
                    for e in range(3):
                        f = [W[0], W[1], W[2]]
                        if d == e:
                            f[d] = D2[d]
                        else:
                            f[d] = D[d]
                            f[e] = D[e]
                        H[:, d, e] = f[0] * f[1] * f[2]
                gx -= q[:, None] * (np.einsum("nde,ne->nd", H, lam) * p[:, None] + gth * h[:, None])
                gq -= np.sum(lam * gth, axis=1) * p + th * h
    return gx, gq


def pme(x, q, box, alpha, ke, K, order=4, return_grid=False):
    """Reciprocal-space energy and forces by smooth PME, FP64."""
    x = np.asarray(x, dtype=np.float64).reshape(-1, 3)
    q = np.asarray(q, dtype=np.float64)
    L = np.broadcast_to(np.asarray(box, dtype=np.float64), (3,))
    K = np.broadcast_to(np.asarray(K, dtype=np.int64), (3,)).copy()
    V = float(np.prod(L))
    n = order
    idx, w, dw = _weights(x, L, K, n)
    Q = np.zeros(tuple(K))
    N = x.shape[0]
    for a in range(n):
        for b in range(n):
            for c in range(n):
                np.add.at(Q, (idx[:, 0, a], idx[:, 1, b], idx[:, 2, c]), q * w[:, 0, a] * w[:, 1, b] * w[:, 2, c])
    Qh = np.fft.fftn(Q)
    m = [np.fft.fftfreq(int(K[d])) * K[d] / L[d] for d in range(3)]
    m2 = m[0][:, None, None] ** 2 + m[1][None, :, None] ** 2 + m[2][None, None, :] ** 2
    B = (bspline_moduli(n, int(K[0]))[:, None, None] * bspline_moduli(n, int(K[1]))[None, :, None]
         * bspline_moduli(n, int(K[2]))[None, None, :])
    with np.errstate(divide="ignore", invalid="ignore"):
        G = ke / (np.pi * V) * np.exp(-np.pi ** 2 * m2 / alpha ** 2) / m2 * B
    G[0, 0, 0] = 0.0
    E = 0.5 * float(np.sum(G * np.abs(Qh) ** 2))
    phi = np.real(np.fft.ifftn(G * Qh)) * float(np.prod(K))
    F = np.zeros((N, 3))
    for a in range(n):
        for b in range(n):
            for c in range(n):
                p = phi[idx[:, 0, a], idx[:, 1, b], idx[:, 2, c]]
                F[:, 0] -= q * dw[:, 0, a] * w[:, 1, b] * w[:, 2, c] * p
                F[:, 1] -= q * w[:, 0, a] * dw[:, 1, b] * w[:, 2, c] * p
                F[:, 2] -= q * w[:, 0, a] * w[:, 1, b] * dw[:, 2, c] * p
    if return_grid:
        return E, F, Q, phi
    return E, F


def mesh_size(alpha, box_len, delta):
    """n_mesh = 2 alpha d / (3 delta^(1/5)) (Sec. 2.1.2)."""
    return 2.0 * alpha * box_len / (3.0 * delta ** 0.2)
