"""Plain CPU FP64 oracle: 2.5D kinematic dynamo, IMEX Runge-Kutta fine and coarse
propagators, Parareal, growth rates.

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` import this module.  The CUDA library never calls it, and it
shares no code with the CUDA path (its only shared dependency is ``kd_inputs``, which
draws the seeded inputs and holds none of the method's arithmetic).

Everything is float64 / complex128, written as the plain definitions of the paper's
method with numpy.fft as the only library step (numpy's pocketfft, single-threaded).

Conventions (Sec. 2, Eq. 1 with the monochromatic ansatz B = b(x, y, t) exp(i kz z)):
  * periodic grid x_j = 2 pi j / n in both directions;
  * b_hat(k) = n^-2 sum_x b(x) exp(-i k.x),  b(x) = sum_k b_hat(k) exp(+i k.x);
  * d/dx <-> i kx, d/dy <-> i ky, d/dz <-> i kz, so nabla_k = (d_x, d_y, i kz);
  * arrays are [..., component, ky, kx], FFT index order;
  * dealiasing keeps the square |kx|, |ky| <= n // 3; the state is zero outside it.

The in-plane coordinates are (x, y) with the invariant direction z for both flows.
The paper writes the Galloway-Proctor flow in the (y, z) plane with kx; the cyclic
relabelling (paper y, z, x) -> (x, y, z) maps it onto the stream-function form used
here, and the paper's kx becomes kz.

Parity: pinned by the tests in tests/test_oracle_*.py (closed forms, the paper's
printed component equations, pure-diffusion decay, divergence, linearity, IMEX order,
Parareal finite termination, eigenvalue / Floquet growth rates and Table 1).
"""
import math

import numpy as np

from kd_inputs import fft_wavenumbers

ROBERTS, GALLOWAY_PROCTOR, NO_FLOW = 0, 1, 2
GP_AMPLITUDE = math.sqrt(1.5)   # C = B = sqrt(3/2), omega = 1 (Sec. 2.2)


class Problem:
    """The initial-value problem of Sec. 2: flow, grid side n, kz and Rm."""

    def __init__(self, flow, n, kz, Rm):
        self.flow, self.n, self.kz, self.Rm = int(flow), int(n), float(kz), float(Rm)

    def with_grid(self, n):
        return Problem(self.flow, n, self.kz, self.Rm)


# --------------------------------------------------------------------------- grid
def kept_mask(n):
    """Dealiased set |kx|, |ky| <= n // 3 (2/3 rule) on the FFT-ordered grid."""
    k = np.abs(fft_wavenumbers(n))
    K = n // 3
    return (k[:, None] <= K) & (k[None, :] <= K)


def wavevector(n, kz):
    """(kx, ky, kz) broadcast to [n][n] (rows ky, columns kx)."""
    k = fft_wavenumbers(n)
    kx = np.broadcast_to(k[None, :], (n, n))
    ky = np.broadcast_to(k[:, None], (n, n))
    return kx, ky, np.full((n, n), float(kz))


def grid_points(n):
    """Collocation points x_j = 2 pi j / n (Sec. 4: periodic box of side 2 pi)."""
    return 2.0 * np.pi * np.arange(n) / n


def to_physical(bh):
    """b(x) = sum_k b_hat(k) exp(i k.x) over the last two axes."""
    n = bh.shape[-1]
    return np.fft.ifft2(bh, axes=(-2, -1)) * (n * n)


def to_spectral(b):
    """b_hat(k) = n^-2 sum_x b(x) exp(-i k.x) over the last two axes."""
    n = b.shape[-1]
    return np.fft.fft2(b, axes=(-2, -1)) / (n * n)


# -------------------------------------------------------------------------- flows
def velocity(flow, n, t):
    """Prescribed flow u(x, y, t) on the grid, real [3][n][n] (rows y, columns x).

    Both flows are u = (d_y psi, -d_x psi, psi):
      Roberts (Sec. 2.1, A = B = 1, C = 0): psi = cos x + sin y, so
        u = (cos y, sin x, cos x + sin y);
      Galloway-Proctor CP (Sec. 2.2, omega = 1, C = B = sqrt(3/2)), relabelled:
        psi = sqrt(3/2) (cos(x + cos t) + sin(y + sin t)).
    """
    x = grid_points(n)[None, :]
    y = grid_points(n)[:, None]
    u = np.zeros((3, n, n))
    if flow == ROBERTS:
        u[0] = np.cos(y) + 0.0 * x
        u[1] = np.sin(x) + 0.0 * y
        u[2] = np.cos(x) + np.sin(y)
    elif flow == GALLOWAY_PROCTOR:
        a, sx, sy = GP_AMPLITUDE, math.cos(t), math.sin(t)
        u[0] = a * np.cos(y + sy) + 0.0 * x
        u[1] = a * np.sin(x + sx) + 0.0 * y
        u[2] = a * (np.cos(x + sx) + np.sin(y + sy))
    return u


def velocity_modes(flow, t):
    """Fourier coefficients u_hat(q) of the flow, keyed by q = (qx, qy).

    Written out from the flow's definition with cos a = (e^{ia} + e^{-ia}) / 2 and
    sin a = (e^{ia} - e^{-ia}) / 2i; only q in {(+-1, 0), (0, +-1)} are nonzero.
    """
    if flow == NO_FLOW:
        return {}
    if flow == ROBERTS:
        a, px, py = 1.0, 0.0, 0.0
    else:
        a, px, py = GP_AMPLITUDE, math.cos(t), math.sin(t)
    ex, ey = np.exp(1j * px), np.exp(1j * py)
    z = 0.0 + 0.0j
    return {
        # u_x = a cos(y + py)
        # u_y = a sin(x + px)
        # u_z = a cos(x + px) + a sin(y + py)
        (1, 0): np.array([z, a * ex / 2j, a * ex / 2]),
        (-1, 0): np.array([z, -a * np.conj(ex) / 2j, a * np.conj(ex) / 2]),
        (0, 1): np.array([a * ey / 2, z, a * ey / 2j]),
        (0, -1): np.array([a * np.conj(ey) / 2, z, -a * np.conj(ey) / 2j]),
    }


# ---------------------------------------------------------------------- operators
def cross(a, b):
    """a x b over the component axis (-3)."""
    return np.stack([a[..., 1, :, :] * b[..., 2, :, :] - a[..., 2, :, :] * b[..., 1, :, :],
                     a[..., 2, :, :] * b[..., 0, :, :] - a[..., 0, :, :] * b[..., 2, :, :],
                     a[..., 0, :, :] * b[..., 1, :, :] - a[..., 1, :, :] * b[..., 0, :, :]],
                    axis=-3)


def curl_k(wh, kz):
    """Spectral curl i k3 x w_hat with k3 = (kx, ky, kz) (nabla_k of Sec. 2)."""
    n = wh.shape[-1]
    kx, ky, kzz = wavevector(n, kz)
    return 1j * np.stack([ky * wh[..., 2, :, :] - kzz * wh[..., 1, :, :],
                          kzz * wh[..., 0, :, :] - kx * wh[..., 2, :, :],
                          kx * wh[..., 1, :, :] - ky * wh[..., 0, :, :]], axis=-3)


def divergence_k(bh, kz):
    """nabla_k . b in spectral space: i (kx bx + ky by + kz bz)."""
    n = bh.shape[-1]
    kx, ky, kzz = wavevector(n, kz)
    return 1j * (kx * bh[..., 0, :, :] + ky * bh[..., 1, :, :] + kzz * bh[..., 2, :, :])


def diffusion_rate(prob):
    """lambda(k) = (kx^2 + ky^2 + kz^2) / Rm: Rm^-1 (nabla^2 - kz^2) b = -lambda b_hat."""
    kx, ky, kz = wavevector(prob.n, prob.kz)
    return (kx * kx + ky * ky + kz * kz) / prob.Rm


def rhs_fft(bh, prob, t, mask=None):
    """Explicit term nabla_k x (u x b) by the pseudo-spectral route (Sec. 4):
    inverse FFT, pointwise u x b on the grid, forward FFT, dealias, spectral curl.
    `mask` replaces the 2/3 set by another mode set (alias-free while its largest
    |k| + 1 < n/2, since u has only |q| = 1 modes)."""
    if mask is None:
        mask = kept_mask(prob.n)
    b = to_physical(bh * mask)
    w = cross(velocity(prob.flow, prob.n, t), b)
    return curl_k(to_spectral(w) * mask, prob.kz) * mask


def rhs_conv(bh, prob, t):
    """The same explicit term as an exact spectral convolution:
    w_hat(k) = sum_q u_hat(q) x b_hat(k - q) over the four modes of u, then dealias
    and curl.  Because u has |q| <= 1 and n // 3 + 1 < n / 2, the pseudo-spectral
    product has no aliasing and both routes agree to round-off."""
    n = bh.shape[-1]
    K = n // 3
    mask = kept_mask(n)
    idx = np.arange(-K - 1, K + 2) % n            # centred rows/cols |k| <= K + 1
    src = (bh * mask)[..., idx[:, None], idx[None, :]]
    wc = np.zeros_like(src)
    m = 2 * K + 3
    for (qx, qy), uq in velocity_modes(prob.flow, t).items():
        shifted = np.zeros_like(src)                 # shifted(k) = b_hat(k - q)
        shifted[..., max(qy, 0):m + min(qy, 0), max(qx, 0):m + min(qx, 0)] = \
            src[..., max(-qy, 0):m + min(-qy, 0), max(-qx, 0):m + min(-qx, 0)]
        ub = np.broadcast_to(uq.reshape((3, 1, 1)), shifted.shape)
        wc = wc + cross(ub, shifted)
    wh = np.zeros_like(bh)
    wh[..., idx[:, None], idx[None, :]] = wc
    return curl_k(wh * mask, prob.kz) * mask


# --------------------------------------------------------------------- timesteppers
def _tableau(c, A, H):
    return {"c": np.array(c, dtype=np.float64), "A": np.array(A, dtype=np.float64),
            "H": np.array(H, dtype=np.float64), "stages": len(c) - 1}


# IMEX Runge-Kutta schemes of Ascher, Ruuth & Spiteri (1997), named RK111, RK222 and
# RK443 in Sec. 4: (s+1) x (s+1) tableaux, row i defines stage i; A is the implicit
# (diffusion) tableau, H the explicit one; c are the stage times.
RK111 = _tableau([0.0, 1.0], [[0, 0], [0, 1]], [[0, 0], [1, 0]])
_g = (2.0 - math.sqrt(2.0)) / 2.0
_d = 1.0 - 1.0 / (2.0 * _g)
RK222 = _tableau([0.0, _g, 1.0],
                 [[0, 0, 0], [0, _g, 0], [0, 1 - _g, _g]],
                 [[0, 0, 0], [_g, 0, 0], [_d, 1 - _d, 0]])
RK443 = _tableau([0.0, 1 / 2, 2 / 3, 1 / 2, 1.0],
                 [[0, 0, 0, 0, 0],
                  [0, 1 / 2, 0, 0, 0],
                  [0, 1 / 6, 1 / 2, 0, 0],
                  [0, -1 / 2, 1 / 2, 1 / 2, 0],
                  [0, 3 / 2, -3 / 2, 1 / 2, 1 / 2]],
                 [[0, 0, 0, 0, 0],
                  [1 / 2, 0, 0, 0, 0],
                  [11 / 18, 1 / 18, 0, 0, 0],
                  [5 / 6, -5 / 6, 1 / 2, 0, 0],
                  [1 / 4, 7 / 4, 3 / 4, -7 / 4, 0]])


def imex_step(x0, t, dt, explicit, lam, tab=RK443):
    """One IMEX Runge-Kutta step (Sec. 4: advection and stretching explicit,
    diffusion implicit).  With the diagonal implicit operator L = lambda(k):

        X_i = (X_0 + dt sum_{j<i} H_ij F_j - dt sum_{j<i} A_ij L X_j) / (1 + dt A_ii L),
        F_j = explicit(X_j, t + c_j dt),

    and the step returns X_s (the schemes are stiffly accurate)."""
    c, A, H, s = tab["c"], tab["A"], tab["H"], tab["stages"]
    X = [x0]
    F = []
    for i in range(1, s + 1):
        F.append(explicit(X[i - 1], t + c[i - 1] * dt))
        acc = x0.copy()
        for j in range(i):
            if H[i, j] != 0.0:
                acc = acc + dt * H[i, j] * F[j]
            if A[i, j] != 0.0:
                acc = acc - dt * A[i, j] * lam * X[j]
        X.append(acc / (1.0 + dt * A[i, i] * lam))
    return X[s]


def propagate(bh, prob, t0, dt, nsteps, tab=RK443, explicit=None, mask=None):
    """nsteps IMEX steps of size dt from absolute time t0 (step s starts at t0 + s dt).
    This is the fine propagator F of Sec. 3 when run on the fine grid with dt = delta t.
    `mask` (optional) keeps the state on another mode set than the 2/3 square."""
    lam = diffusion_rate(prob)
    if mask is None:
        mask = kept_mask(prob.n)
    if explicit is None:
        explicit = lambda v, p, tt: rhs_fft(v, p, tt, mask)
    x = bh * mask
    for s in range(nsteps):
        x = imex_step(x, t0 + s * dt, dt, lambda v, tt: explicit(v, prob, tt), lam, tab)
    return x


# ---------------------------------------------------- restriction / prolongation
def restrict(bh, n_c):
    """Fourier restriction to the coarse grid: keep |kx|, |ky| <= n_c // 3 (Sec. 4,
    set_scales resampling); coefficients are grid independent in this normalisation."""
    n = bh.shape[-1]
    Kc = n_c // 3
    k = np.arange(-Kc, Kc + 1)
    out = np.zeros(bh.shape[:-2] + (n_c, n_c), dtype=bh.dtype)
    out[..., (k % n_c)[:, None], (k % n_c)[None, :]] = bh[..., (k % n)[:, None], (k % n)[None, :]]
    return out


def prolong(bh_c, n):
    """Fourier interpolation to the fine grid: zero-pad the coarse spectrum."""
    n_c = bh_c.shape[-1]
    Kc = n_c // 3
    k = np.arange(-Kc, Kc + 1)
    out = np.zeros(bh_c.shape[:-2] + (n, n), dtype=bh_c.dtype)
    out[..., (k % n)[:, None], (k % n)[None, :]] = bh_c[..., (k % n_c)[:, None], (k % n_c)[None, :]]
    return out


def coarse_propagate(bh, prob, n_c, t0, dt_c, nsteps_c, tab=RK443):
    """Classical coarse propagator G (Sec. 3.2 / Sec. 5.2): restrict to the n_c grid,
    take nsteps_c steps of size dt_c with the same equations, prolong back."""
    xc = restrict(bh, n_c)
    xc = propagate(xc, prob.with_grid(n_c), t0, dt_c, nsteps_c, tab)
    return prolong(xc, prob.n)


# ----------------------------------------------------------------------- parareal
def l2(v):
    return float(np.sqrt(np.sum(np.abs(v) ** 2)))


def parareal(u0, fine_op, coarse_op, n_slices, k_max, tol, keep_iterates=False):
    """Parareal (Sec. 3, Eq. 8; Algorithms of Sec. 4.1).

    fine_op(u, n) and coarse_op(u, n) propagate a state across slice n, from t_n to
    t_{n+1}.  Iterate k = 0 is the serial coarse sweep.  Iteration k + 1 evaluates
    the update as  U_{n+1} = F(U^k_n) + (G(U^{k+1}_n) - G(U^k_n)),  with the fine
    values of all slices computed first (the parallel step) and the coarse values
    of the previous sweep kept.  It stops when the defect of Eq. 9,
      sigma = ||U^k_N - U^{k-1}_N|| / ||U^k_N||,
    is <= tol, or after k_max iterations.  Returns the slice states U_0..U_N, the
    iteration count k_con and the defect history (and every iterate if asked)."""
    U = [u0.copy()]
    G = []
    for n in range(n_slices):                       # initial coarse run
        G.append(coarse_op(U[n], n))
        U.append(G[n].copy())
    iterates = [[u.copy() for u in U]] if keep_iterates else None
    sigmas = []
    k_con = k_max
    for k in range(1, k_max + 1):
        Fv = [fine_op(U[n], n) for n in range(n_slices)]     # parallel step
        last_prev = U[n_slices].copy()
        for n in range(n_slices):                             # serial step
            g = coarse_op(U[n], n)
            U[n + 1] = Fv[n] + (g - G[n])
            G[n] = g
        sigma = l2(U[n_slices] - last_prev) / l2(U[n_slices])
        sigmas.append(sigma)
        if keep_iterates:
            iterates.append([u.copy() for u in U])
        if sigma <= tol:
            k_con = k
            break
    return {"U": U, "k_con": k_con, "sigma": sigmas, "iterates": iterates}


def serial_fine(u0, fine_op, n_slices):
    """The serial fine solution at the slice boundaries: U_{n+1} = F(U_n)."""
    U = [u0.copy()]
    for n in range(n_slices):
        U.append(fine_op(U[n], n))
    return U


def speedup_model(k_con, n_slices, rc_over_rf):
    """Estimated Parareal speedup, Eq. 10: s = [(1 + k/N_p) R_c/R_f + k/N_p]^-1."""
    return 1.0 / ((1.0 + k_con / n_slices) * rc_over_rf + k_con / n_slices)


# -------------------------------------------------------------------- growth rates
def energy(bh):
    """Magnetic energy in spectral norm: E = sum_{c,k} |b_hat_c(k)|^2."""
    return float(np.sum(np.abs(bh) ** 2))


def growth_rate(times, energies, fit_from):
    """Amplitude growth rate: least-squares slope of (1/2) ln E(t) over t >= fit_from
    (Sec. 2: kinematic solutions grow or decay exponentially; Table 1 'Growth Rate')."""
    t = np.asarray(times, dtype=np.float64)
    y = 0.5 * np.log(np.asarray(energies, dtype=np.float64))
    sel = t >= fit_from - 1e-12
    t, y = t[sel], y[sel]
    tm, ym = t.mean(), y.mean()
    return float(np.sum((t - tm) * (y - ym)) / np.sum((t - tm) ** 2))


def kept_index(n):
    """Wavenumbers of the dealiased set in a fixed order (ky major, kx minor)."""
    K = n // 3
    k = np.arange(-K, K + 1)
    return [(int(qx), int(qy)) for qy in k for qx in k]


def linear_operator(prob, t=0.0):
    """Sparse matrix of the truncated spectral operator b_hat -> d b_hat / dt on the
    dealiased set (3 components x (2K+1)^2 modes, component-major), built from the
    convolution form: i [k3]_x [u_hat(q)]_x couples mode k - q to mode k, and the
    diagonal holds -lambda(k).  For the steady Roberts flow its leading eigenvalue is
    the growth rate (Sec. 1: steady u gives an eigenvalue problem)."""
    import scipy.sparse as sp
    n = prob.n
    K = n // 3
    modes = kept_index(n)
    M = len(modes)
    pos = {m: i for i, m in enumerate(modes)}
    rows, cols, vals = [], [], []

    def skew(a):
        return np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]], dtype=complex)

    uq = velocity_modes(prob.flow, t)
    for (kx, ky), i in pos.items():
        k3 = np.array([kx, ky, prob.kz], dtype=float)
        ck = 1j * skew(k3)
        lam = (kx * kx + ky * ky + prob.kz ** 2) / prob.Rm
        for c in range(3):
            rows.append(c * M + i)
            cols.append(c * M + i)
            vals.append(-lam)
        for (qx, qy), u in uq.items():
            src = (kx - qx, ky - qy)
            if abs(src[0]) > K or abs(src[1]) > K:
                continue
            j = pos[src]
            blk = ck @ skew(u)
            for a in range(3):
                for b in range(3):
                    if blk[a, b] != 0:
                        rows.append(a * M + i)
                        cols.append(b * M + j)
                        vals.append(blk[a, b])
    return sp.csr_matrix((vals, (rows, cols)), shape=(3 * M, 3 * M), dtype=complex)


def to_kept_vector(bh):
    """Field [3][n][n] -> vector in linear_operator's ordering."""
    n = bh.shape[-1]
    idx = [(qy % n, qx % n) for (qx, qy) in kept_index(n)]
    iy = np.array([a for a, _ in idx])
    ix = np.array([b for _, b in idx])
    return np.concatenate([bh[c][iy, ix] for c in range(3)])


# ----------------------------------------------------------- learned coarse propagator
# A complex-linear map W on the mode set kx, ky in [-m/2, m/2) x 3 components (a coarse
# propagator in the sense of Sec. 3.2), fitted to pairs (x, R F P x) of the fine
# propagator.  Vectors on the set have the layout [3][m][m] (component, ky, kx).
def learned_mask(n, m):
    """Mode set kx, ky in [-m/2, m/2) on the FFT-ordered n x n grid."""
    k = fft_wavenumbers(n)
    inset = (k >= -(m // 2)) & (k < m - m // 2)
    return inset[:, None] & inset[None, :]


def learned_restrict(bh, m):
    """Field [..., 3, n, n] -> learned vector [..., 3 m m] (flattened [3][m][m])."""
    n = bh.shape[-1]
    k = np.arange(-(m // 2), m - m // 2) % n
    v = bh[..., k[:, None], k[None, :]]
    return v.reshape(v.shape[:-3] + (3 * m * m,))


def learned_prolong(x, m, n):
    """Learned vector [..., 3 m m] -> field [..., 3, n, n] (zero outside the set)."""
    k = np.arange(-(m // 2), m - m // 2) % n
    out = np.zeros(x.shape[:-1] + (3, n, n), dtype=complex)
    out[..., k[:, None], k[None, :]] = x.reshape(x.shape[:-1] + (3, m, m))
    return out


def learned_loss_grad(W, X, Y, W0, wd):
    """Training objective of the learned operator and its gradient:
        L = (1/m) sum_i |W x_i - y_i|^2 + wd |W - W0|_F^2,
        dL/dRe W + i dL/dIm W = (2/m) sum_i r_i x_i^H + 2 wd (W - W0),  r_i = W x_i - y_i.
    X, Y: [m, nc] (rows are pairs); W, W0: [nc, nc] complex."""
    m = X.shape[0]
    R = X @ W.T - Y
    D = W - W0
    loss = float(np.sum(np.abs(R) ** 2) / m + wd * np.sum(np.abs(D) ** 2))
    grad = (2.0 / m) * (R.T @ np.conj(X)) + 2.0 * wd * D
    return loss, grad


def learned_ridge(X, Y, W0, wd):
    """Minimiser of learned_loss_grad's objective (its gradient vanishes):
        W (X^T conj(X) / m + wd I) = Y^T conj(X) / m + wd W0."""
    m, nc = X.shape
    A = X.T @ np.conj(X) / m + wd * np.eye(nc)
    B = Y.T @ np.conj(X) / m + wd * W0
    return np.linalg.solve(A.T, B.T).T


def learned_minnorm(X, Y, W0):
    """The smallest change of W0 (Frobenius norm) for which W x_i = y_i for every pair:
        W = W0 + (Y^T - W0 X^T) pinv(X^T),
    X, Y: [m, nc] (rows are pairs).  With fewer pairs than unknowns of a row it is the
    limit of learned_ridge as wd -> 0 (learned_ridge itself needs wd > 0 there)."""
    return W0 + (Y.T - W0 @ X.T) @ np.linalg.pinv(X.T)


def learned_exact_map(prob, m, t0, dt, nsteps):
    """The fine propagator's map on the learned set, R F P, column by column (one fine
    propagation of every unit vector; tiny sets only)."""
    nc = 3 * m * m
    E = np.eye(nc, dtype=complex)
    out = propagate(learned_prolong(E, m, prob.n), prob, t0, dt, nsteps)
    return learned_restrict(out, m).T
