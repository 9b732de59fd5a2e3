"""The discrete Lippmann-Schwinger operator, dense and matrix-free.  FP64, NumPy/SciPy.

Test infrastructure: part of the CPU oracle (see ``oracle/__init__.py``).

Definitions (Sec. 2-3; readings listed where the paper is silent):

* strain (Eq. 18): engineering Voigt strain e1..e6 (e4 = 2 e23, e5 = 2 e13,
  e6 = 2 e12, Eq. 17) from central differences (f(i+1) - f(i-1)) / 2h; on the
  first and last node of an axis the first-order one-sided difference
  (the paper asks only for "forward or backward" there);
* contrast stress (Eq. 11): sigma_J = sum_K dC_JK e_K, used as a symmetric
  tensor sigma_jk (sigma_23 = sigma_32 = sigma_4 and so on, no factor 2);
* contrast source: q_j = sum_k D_k sigma_jk + w^2 drho u_j, where D_k is the
  central difference on the zero-extended grid.  q lives on the nodes
  [-1, n]^3 (one node beyond the model on each side);
* scattered field (Eq. 8 after partial integration): u_s(x) = sum_x'
  T(x - x') q(x'), T the kernel table of ``green.kernel_table``;
* operator (Eqs. 19-21): A u = u - u_s restricted to the model's nodes.

``dense_matrix`` builds A entry by entry from these sums (no FFT);
``apply_fft`` evaluates the same operator in the form of Eq. 21: FFTs on the
2n-periodic grid, the spectrum of T, and the derivative D_k applied as the
factor i kappa_k with kappa_k = sin(k_k h) / h.

Sampled-H form (Eq. 21 with H taken literally): the derivative of Eq. 9 is not a difference
but the analytic dG of Appendix A sampled on the grid (``green.h_table``):
u_s,i(x) = sum_x' [sum_J H_iJ(x - x') sigma_J(x') + w^2 sum_j T_ij(x - x') drho u_j(x')] over
the model's nodes x'; ``apply_direct_h`` sums this directly, ``FFTOperator(form="h")`` by FFT.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import green as _green

# Voigt index -> tensor pair (0-based), order 11, 22, 33, 23, 13, 12 (Eq. 17)
VOIGT = ((0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1))
# tensor pair -> Voigt index
T2V = ((0, 5, 4), (5, 1, 3), (4, 3, 2))

_TRIU = [(I, J) for I in range(6) for J in range(I, 6)]


def unpack_contrast(dC21):
    """21 upper-triangle planes -> symmetric (6, 6, ...) Voigt contrast."""
    C = np.zeros((6, 6) + dC21.shape[1:], dtype=np.float64)
    for k, (I, J) in enumerate(_TRIU):
        C[I, J] = dC21[k]
        C[J, I] = dC21[k]
    return C


# ----------------------------------------------------------------------------
# array (matrix-free) pieces
# ----------------------------------------------------------------------------

def _d_axis(f, axis, h):
    """Eq. 18 derivative along one array axis: central inside, one-sided at the ends."""
    f = np.moveaxis(f, axis, 0)
    d = np.empty_like(f)
    d[1:-1] = (f[2:] - f[:-2]) / (2.0 * h)
    d[0] = (f[1] - f[0]) / h
    d[-1] = (f[-1] - f[-2]) / h
    return np.moveaxis(d, 0, axis)


def _axis_of(a):
    """Coordinate a (0=x, 1=y, 2=z) -> array axis of a (nz, ny, nx) field."""
    return 2 - a


def strain(u, h):
    """Voigt strain (6, nz, ny, nx) of a displacement field u (3, nz, ny, nx)  (Eqs. 17-18)."""
    du = lambda c, a: _d_axis(u[c], _axis_of(a), h)  # noqa: E731   d u_c / d x_a
    return np.stack([
        du(0, 0),
        du(1, 1),
        du(2, 2),
        du(1, 2) + du(2, 1),
        du(0, 2) + du(2, 0),
        du(0, 1) + du(1, 0),
    ])


def stress(dC21, eps):
    """Contrast stress sigma_J = sum_K dC_JK eps_K  (Eq. 11)."""
    C = unpack_contrast(dC21)
    return np.einsum("JK...,K...->J...", C, eps)


def contrast_source(u, dC21, drho, h, omega):
    """q_j on the extended nodes [-1, n]^3: sum_k D_k sigma_jk + w^2 drho u_j.

    Returns (3, nz+2, ny+2, nx+2); array index p corresponds to node p - 1.
    """
    sig = stress(dC21, strain(u, h))
    nz, ny, nx = u.shape[1:]
    # sigma zero-extended by two nodes on each side so that D can be taken on [-1, n]
    S = np.zeros((6, nz + 4, ny + 4, nx + 4), dtype=np.complex128)
    S[:, 2:-2, 2:-2, 2:-2] = sig
    q = np.zeros((3, nz + 2, ny + 2, nx + 2), dtype=np.complex128)
    for j in range(3):
        for k in range(3):
            s = S[T2V[j][k]]
            ax = _axis_of(k)
            hi = [slice(1, -1)] * 3
            lo = [slice(1, -1)] * 3
            hi[ax] = slice(2, None)
            lo[ax] = slice(0, -2)
            q[j] += (s[tuple(hi)] - s[tuple(lo)]) / (2.0 * h)
    q[:, 1:-1, 1:-1, 1:-1] += omega ** 2 * drho * u
    return q


def scatter_direct(q, table, n):
    """u_s(x) = sum_{x' in [-1,n]^3} T(x - x') q(x')  by brute-force summation (small n only)."""
    nx, ny, nz = n
    us = np.zeros((3, nz, ny, nx), dtype=np.complex128)
    ext = [np.arange(-1, m + 1) for m in (nz, ny, nx)]
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                mz = (z - ext[0]) % (2 * nz)
                my = (y - ext[1]) % (2 * ny)
                mx = (x - ext[2]) % (2 * nx)
                Tloc = table[:, :, mz[:, None, None], my[None, :, None], mx[None, None, :]]
                us[:, z, y, x] = np.einsum("ijabc,jabc->i", Tloc, q)
    return us


def apply_direct(u, medium, omega, mode="exact"):
    """A u by direct summation (no FFT), for small grids."""
    T = _green.kernel_table(medium.n, medium.h, omega, medium.lam0, medium.mu0, medium.rho0, mode)
    q = contrast_source(u, medium.dC, medium.drho, medium.h, omega)
    return u - scatter_direct(q, T, medium.n)


def scatter_direct_h(sig, w, htab, table, n):
    """Sampled-H scattered field by brute-force summation over the model's nodes (small n only):
    u_s,i(x) = sum_x' sum_J H_iJ(x - x') sig_J(x') + sum_j T_ij(x - x') w_j(x')."""
    nx, ny, nz = n
    us = np.zeros((3, nz, ny, nx), dtype=np.complex128)
    src = [np.arange(m) for m in (nz, ny, nx)]
    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                mz = (z - src[0]) % (2 * nz)
                my = (y - src[1]) % (2 * ny)
                mx = (x - src[2]) % (2 * nx)
                sel = (mz[:, None, None], my[None, :, None], mx[None, None, :])
                Hloc = htab[:, :, sel[0], sel[1], sel[2]]
                Tloc = table[:, :, sel[0], sel[1], sel[2]]
                us[:, z, y, x] = np.einsum("iJabc,Jabc->i", Hloc, sig) + np.einsum("ijabc,jabc->i", Tloc, w)
    return us


def apply_direct_h(u, medium, omega, mode="exact"):
    """A u of the sampled-H form by direct summation (no FFT), for small grids."""
    args = (medium.n, medium.h, omega, medium.lam0, medium.mu0, medium.rho0, mode)
    H = _green.h_table(*args)
    T = _green.kernel_table(*args)
    sig = stress(medium.dC, strain(u, medium.h))
    return u - scatter_direct_h(sig, omega ** 2 * medium.drho * u, H, T, medium.n)


class FFTOperator:
    """A u evaluated as in Eq. 21 on the 2n-periodic grid.

    sigma-hat = FFT(pad sigma), w-hat = FFT(pad(drho u)),
    q-hat_j = sum_k i kappa_k sigma-hat_jk + w^2 w-hat_j,
    u_s = crop IFFT(T-hat q-hat), A u = u - u_s.

    workers: None (default) transforms with numpy.fft on one thread; an integer k transforms
    with scipy.fft on k threads (the same discrete Fourier transform; used to time the oracle on
    all of a machine's cores).  It may be changed after construction.
    """

    def __init__(self, medium, omega, mode="exact", form="fd", workers=None):
        if form not in ("fd", "h"):
            raise ValueError(form)
        self.workers = workers
        self.m = medium
        self.omega = float(omega)
        self.n = medium.n
        self.form = form
        nx, ny, nz = medium.n
        self.P = (2 * nz, 2 * ny, 2 * nx)
        T = _green.kernel_table(medium.n, medium.h, omega, medium.lam0, medium.mu0, medium.rho0, mode)
        self.That = np.fft.fftn(T, axes=(-3, -2, -1))
        if form == "h":
            H = _green.h_table(medium.n, medium.h, omega, medium.lam0, medium.mu0, medium.rho0, mode)
            self.Hhat = np.fft.fftn(H, axes=(-3, -2, -1))
        h = medium.h
        kap = []
        for a, L in enumerate((2 * nx, 2 * ny, 2 * nz)):
            m = np.arange(L)
            kap.append(np.sin(2.0 * np.pi * m / L) / h)
        # kappa as broadcastable arrays over (z, y, x)
        self.kappa = (kap[0][None, None, :], kap[1][None, :, None], kap[2][:, None, None])

    def _fftn(self, a):
        if self.workers is None:
            return np.fft.fftn(a, axes=(-3, -2, -1))
        import scipy.fft
        return scipy.fft.fftn(a, axes=(-3, -2, -1), workers=self.workers)

    def _ifftn(self, a):
        if self.workers is None:
            return np.fft.ifftn(a, axes=(-3, -2, -1))
        import scipy.fft
        return scipy.fft.ifftn(a, axes=(-3, -2, -1), workers=self.workers)

    def _pad(self, f):
        nx, ny, nz = self.n
        F = np.zeros(f.shape[:-3] + self.P, dtype=np.complex128)
        F[..., :nz, :ny, :nx] = f
        return F

    def _crop(self, F):
        nx, ny, nz = self.n
        return F[..., :nz, :ny, :nx]

    def scattered(self, u):
        m = self.m
        sig = stress(m.dC, strain(u, m.h))
        sh = self._fftn(self._pad(sig))
        wh = self._fftn(self._pad(m.drho * u))
        if self.form == "h":
            # Eq. 21: u-hat_i = sum_J H-hat_iJ sigma-hat_J + w^2 sum_j T-hat_ij w-hat_j
            uh = (np.einsum("iJ...,J...->i...", self.Hhat, sh)
                  + self.omega ** 2 * np.einsum("ij...,j...->i...", self.That, wh))
            return self._crop(self._ifftn(uh))
        qh = self.omega ** 2 * wh
        for j in range(3):
            for k in range(3):
                qh[j] = qh[j] + 1j * self.kappa[k] * sh[T2V[j][k]]
        uh = np.einsum("ij...,j...->i...", self.That, qh)
        return self._crop(self._ifftn(uh))

    def apply(self, u):
        return u - self.scattered(u)

    def adjoint(self, w):
        """A^H w: the transposes of the steps of ``apply`` in reverse order.

        With the kernel symmetric (T_ij(m) = T_ji(m) = T_ij(-m)), the
        adjoint convolution uses conj(T-hat); the derivative factor i kappa
        becomes its conjugate -i kappa; the stress and strain maps become the
        transposes of the (real) contrast matrix and strain operator.
        """
        if self.form != "fd":
            raise NotImplementedError("adjoint of the sampled-H form")
        m = self.m
        wh = np.fft.fftn(self._pad(w), axes=(-3, -2, -1))
        zh = np.einsum("ij...,i...->j...", np.conj(self.That), wh)
        # adjoint of the Voigt divergence: tau_J = sum_{(j,k) -> J} conj(i kappa_k) z_j
        tau_h = np.zeros((6,) + self.P, dtype=np.complex128)
        for j in range(3):
            for k in range(3):
                tau_h[T2V[j][k]] += -1j * self.kappa[k] * zh[j]
        tau = self._crop(np.fft.ifftn(tau_h, axes=(-3, -2, -1)))
        z = self._crop(np.fft.ifftn(zh, axes=(-3, -2, -1)))
        C = unpack_contrast(m.dC)
        ctau = np.einsum("JK...,J...->K...", C, tau)
        back = strain_transpose(ctau, m.h) + self.omega ** 2 * m.drho * z
        return w - back


def strain_transpose(t, h):
    """Transpose of ``strain``: (6, nz, ny, nx) -> (3, nz, ny, nx), via the sparse strain matrix."""
    nz, ny, nx = t.shape[1:]
    E = strain_matrix((nx, ny, nz), h)
    return (E.T @ t.reshape(-1)).reshape(3, nz, ny, nx)


# ----------------------------------------------------------------------------
# explicit matrices (dense oracle)
# ----------------------------------------------------------------------------

def _d1(n, h):
    """1-D Eq. 18 derivative matrix (n x n): central inside, one-sided at both ends."""
    D = sp.lil_matrix((n, n))
    for i in range(n):
        if i == 0:
            D[0, 0], D[0, 1] = -1.0 / h, 1.0 / h
        elif i == n - 1:
            D[i, i - 1], D[i, i] = -1.0 / h, 1.0 / h
        else:
            D[i, i - 1], D[i, i + 1] = -0.5 / h, 0.5 / h
    return D.tocsr()


def _dext(n, h):
    """1-D central difference from nodes [0, n) to nodes [-1, n] of a zero-extended field ((n+2) x n)."""
    D = sp.lil_matrix((n + 2, n))
    for p in range(-1, n + 1):
        if 0 <= p + 1 < n:
            D[p + 1, p + 1] += 0.5 / h
        if 0 <= p - 1 < n:
            D[p + 1, p - 1] -= 0.5 / h
    return D.tocsr()


def _embed(n):
    """1-D embedding of nodes [0, n) into [-1, n] ((n+2) x n)."""
    E = sp.lil_matrix((n + 2, n))
    for i in range(n):
        E[i + 1, i] = 1.0
    return E.tocsr()


def _kron3(Mz, My, Mx):
    return sp.kron(Mz, sp.kron(My, Mx)).tocsr()


def strain_matrix(n, h):
    """Sparse (6 N, 3 N) matrix of ``strain`` (N = nx ny nz, layout [comp][z][y][x])."""
    nx, ny, nz = n
    I = [sp.identity(nx), sp.identity(ny), sp.identity(nz)]
    D = [_d1(nx, h), _d1(ny, h), _d1(nz, h)]

    def d(a):  # derivative along coordinate a on the full grid
        ops = [I[2], I[1], I[0]]
        ops[2 - a] = D[a]
        return _kron3(*ops)

    Z = None
    blocks = [[d(0), Z, Z],
              [Z, d(1), Z],
              [Z, Z, d(2)],
              [Z, d(2), d(1)],
              [d(2), Z, d(0)],
              [d(1), d(0), Z]]
    return sp.bmat(blocks, format="csr")


def divergence_matrix(n, h):
    """Sparse (3 M, 6 N) matrix sigma (Voigt, model nodes) -> sum_k D_k sigma_jk on [-1, n]^3 (M = prod(n+2))."""
    nx, ny, nz = n
    Em = [_embed(nx), _embed(ny), _embed(nz)]
    De = [_dext(nx, h), _dext(ny, h), _dext(nz, h)]

    def d(a):
        ops = [Em[2], Em[1], Em[0]]
        ops[2 - a] = De[a]
        return _kron3(*ops)

    blocks = [[None] * 6 for _ in range(3)]
    for j in range(3):
        for k in range(3):
            J = T2V[j][k]
            blocks[j][J] = d(k) if blocks[j][J] is None else blocks[j][J] + d(k)
    # bmat needs each block column to have a known width: fill empty blocks with zeros
    M = (nx + 2) * (ny + 2) * (nz + 2)
    N = nx * ny * nz
    for j in range(3):
        for J in range(6):
            if blocks[j][J] is None:
                blocks[j][J] = sp.csr_matrix((M, N))
    return sp.bmat(blocks, format="csr")


def embed_matrix(n):
    nx, ny, nz = n
    return _kron3(_embed(nz), _embed(ny), _embed(nx))


def kernel_matrix(n, table):
    """Dense (3 N, 3 M) matrix of u_s(x) = sum_{x' in [-1,n]^3} T(x - x') q(x')."""
    nx, ny, nz = n
    Z, Y, X = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    Ze, Ye, Xe = np.meshgrid(np.arange(-1, nz + 1), np.arange(-1, ny + 1), np.arange(-1, nx + 1), indexing="ij")
    dz = (Z.reshape(-1)[:, None] - Ze.reshape(-1)[None, :]) % (2 * nz)
    dy = (Y.reshape(-1)[:, None] - Ye.reshape(-1)[None, :]) % (2 * ny)
    dx = (X.reshape(-1)[:, None] - Xe.reshape(-1)[None, :]) % (2 * nx)
    N, M = dz.shape
    K = np.zeros((3, N, 3, M), dtype=np.complex128)
    for i in range(3):
        for j in range(3):
            K[i, :, j, :] = table[i, j][dz, dy, dx]
    return K.reshape(3 * N, 3 * M)


def dense_matrix(medium, omega, mode="exact"):
    """The LS operator A as an explicit dense (3N x 3N) complex matrix (no FFT).

    A = I - K_T (Dv C E + w^2 Emb drho), with E the strain matrix, C the
    per-voxel Voigt contrast, Dv the extended divergence, Emb the embedding
    of model nodes in [-1, n]^3 and K_T the direct-sum kernel matrix.
    """
    n = medium.n
    nx, ny, nz = n
    N = nx * ny * nz
    h = medium.h
    E = strain_matrix(n, h)
    C = unpack_contrast(medium.dC).reshape(6, 6, N)
    Cm = sp.bmat([[sp.diags(C[I, J]) for J in range(6)] for I in range(6)], format="csr")
    Dv = divergence_matrix(n, h)
    Emb = embed_matrix(n)
    R = sp.block_diag([Emb @ sp.diags(medium.drho.reshape(-1))] * 3, format="csr")
    W = (Dv @ Cm @ E + omega ** 2 * R).toarray()
    T = _green.kernel_table(n, h, omega, medium.lam0, medium.mu0, medium.rho0, mode)
    K = kernel_matrix(n, T)
    return np.eye(3 * N, dtype=np.complex128) - K @ W


def apply_at_points(u, medium, omega, points, mode="exact"):
    """(A u)(x) at a few nodes x by direct summation over the extended grid; any grid size.

    points: iterable of node indices (ix, iy, iz).  Returns an array (len(points), 3) complex.
    The contrast source q is formed on the whole extended grid [-1, n]^3 (as in
    ``contrast_source``); each output then sums T(x - x') q(x') over x' with the kernel of
    ``green.kernel_table`` evaluated at exactly the offsets needed.
    """
    nx, ny, nz = medium.n
    h = medium.h
    q = contrast_source(u, medium.dC, medium.drho, h, omega)
    ext = [np.arange(-1, m + 1) for m in (nx, ny, nz)]
    out = []
    for ix, iy, iz in points:
        MZ, MY, MX = np.meshgrid(iz - ext[2], iy - ext[1], ix - ext[0], indexing="ij")
        nyq = (np.abs(MX) >= nx) | (np.abs(MY) >= ny) | (np.abs(MZ) >= nz)
        self_ = (MX == 0) & (MY == 0) & (MZ == 0)
        off = np.stack([MX, MY, MZ], axis=-1).astype(np.float64) * h
        off[nyq | self_] = h  # placeholder, overwritten below
        T = _green.green(off, omega, medium.lam0, medium.mu0, medium.rho0, mode) * h ** 3
        T[nyq] = 0.0
        T[self_] = _green.self_cell(h, omega, medium.lam0, medium.mu0, medium.rho0)
        us = np.einsum("zyxij,jzyx->i", T, q)
        out.append(u[:, iz, iy, ix] - us)
    return np.array(out)


def kernel_adjoint_ext(lam, medium, omega, mode="exact"):
    """z = K_T^H lam on the extended nodes [-1, n]^3: z(p) = sum_x conj(T(x - p)) lam(x).

    By FFT on the 2n-periodic grid: lam placed at its nodes, multiplied by conj(T-hat)
    (T is even and symmetric), read back at the extended nodes p mod 2n.
    Returns (3, nz+2, ny+2, nx+2); index p holds node p - 1.
    """
    nx, ny, nz = medium.n
    T = _green.kernel_table(medium.n, medium.h, omega, medium.lam0, medium.mu0, medium.rho0, mode)
    That = np.fft.fftn(T, axes=(-3, -2, -1))
    P = (2 * nz, 2 * ny, 2 * nx)
    Lp = np.zeros((3,) + P, dtype=np.complex128)
    Lp[:, :nz, :ny, :nx] = lam
    zh = np.einsum("ij...,i...->j...", np.conj(That), np.fft.fftn(Lp, axes=(-3, -2, -1)))
    zper = np.fft.ifftn(zh, axes=(-3, -2, -1))
    iz = np.arange(-1, nz + 1) % (2 * nz)
    iy = np.arange(-1, ny + 1) % (2 * ny)
    ix = np.arange(-1, nx + 1) % (2 * nx)
    return zper[:, iz[:, None, None], iy[None, :, None], ix[None, None, :]]


def contrast_gradient(u, lam, medium, omega, mode="exact"):
    """Gradients of Re<lam, K_T (Dv dC eps(u) + w^2 Emb drho u)> with respect to the 21 packed
    contrast planes and the density contrast (the discrete adjoint of Eqs. 8 and 11).

    tau = Dv^T z (Voigt, model nodes) with z = K_T^H lam; for packed entry (I, J):
    Re(conj(tau_I) eps_J) (+ Re(conj(tau_J) eps_I) when I != J); density: w^2 Re(sum_j conj(z_j) u_j).
    Returns (gC (21, nz, ny, nx), grho (nz, ny, nx)).
    """
    nx, ny, nz = medium.n
    z = kernel_adjoint_ext(lam, medium, omega, mode)
    Dv = divergence_matrix(medium.n, medium.h)
    tau = (Dv.T @ z.reshape(-1)).reshape(6, nz, ny, nx)
    eps = strain(u, medium.h)
    gC = np.zeros((21, nz, ny, nx))
    for k, (I, J) in enumerate(_TRIU):
        g = np.real(np.conj(tau[I]) * eps[J])
        if I != J:
            g = g + np.real(np.conj(tau[J]) * eps[I])
        gC[k] = g
    zin = z[:, 1:-1, 1:-1, 1:-1]
    grho = omega ** 2 * np.real(np.sum(np.conj(zin) * u, axis=0))
    return gC, grho


def taper_weight(n, h, width):
    """Absorbing-boundary weight of Eq. 25 on the model's nodes, shape (nz, ny, nx).

    Reading of Eq. 25: inside a boundary layer of `width` nodes the contrast sources are
    multiplied by 1 - exp(-l^2 / (N_a h^2)) for each axis a whose layer contains the node, with
    l the distance from the node to the model's outer boundary node plane along that axis and
    N_a the number of nodes along it; outside the layer the factor is 1.  width = 0: no taper.
    """
    out = np.ones(tuple(reversed(n)))
    if width <= 0:
        return out
    factors = []
    for a, N in enumerate(n):
        k = np.arange(N)
        dist = np.minimum(k, N - 1 - k)
        f = np.where(dist < width, 1.0 - np.exp(-(dist * h) ** 2 / (N * h * h)), 1.0)
        factors.append(f)
    return factors[2][:, None, None] * factors[1][None, :, None] * factors[0][None, None, :]


def tapered(medium, width):
    """The medium with its contrasts weighted by ``taper_weight`` (Eq. 25)."""
    import copy
    w = taper_weight(medium.n, medium.h, width)
    m = copy.copy(medium)
    m.dC = medium.dC * w[None]
    m.drho = medium.drho * w
    return m
