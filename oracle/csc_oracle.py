"""FP64 CPU oracle for dual-domain convolutional sparse coding (Affara, Ghanem & Wonka, arXiv 1709.09479).

TEST INFRASTRUCTURE ONLY. Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import or call this module. The CUDA product path never does, and this module
imports nothing from it: the two share no kernels, helpers, tables or constants.

Everything is plain float64 NumPy/SciPy, written to be checked against the paper by eye. Where the
method has a closed form it is written out; where it iterates, the paper's steps run in the paper's
order. Library FFTs (``scipy.fft``) stand in for the unnormalised DFT F. Its inverse carries 1/D.

Conventions (readings of points the paper leaves open):
* Arrays: images x (N, J, *dims), filters d (K, J, *fs), codes / ADMM state (N, K, *dims).
  ``dims`` is (H, W) or (T, H, W). Codes are shared across the J channels (Sec. 3.3).
* Convolution is circular on the image grid (Sec. 3, start): (d*z)(p) = sum_q d(q) z(p-q).
  Filter tap a along an axis of support f sits at offset a - (f-1)//2, wrapped around.
* D z = sum_k d_k * z_k (Eq. 2). D^T lam is the correlation (d ⋆ lam)(p) = sum_q d(q) lam(p+q).
* The l1 weight is beta (Eq. 1). rho is the ADMM step of Eq. "Inference_solution".

Parity pins for every function are in tests/test_oracle_*.py. The entry points:
``code_admm`` (v-state form) and ``code_admm_textbook`` (the three-variable update of Sec. 3.2);
``learn_paper`` (Sec. 3.2, learning: gamma by CG, d recovery, mu fixed point, final projection);
``csc_alternate`` (Algorithm 1); ``objective`` (Eq. 1); ``duality_gap``; ``fista_code``;
``unrolled_loss_and_grad`` (adjoint of T unrolled coding iterations, not in the paper);
``code_admm_symmetric`` and ``code_admm_dct`` (reflected image boundaries: the DCT variant the paper
mentions at the start of Sec. 3).
"""
from __future__ import annotations

import numpy as np
import scipy.fft as sfft

#: threads handed to scipy.fft (-1: all host cores)
WORKERS = -1

#: lower bound on the multipliers mu_k. Where a filter's norm constraint is inactive, the update
#: mu <- mu ||d|| of Eq. mu_update drives mu_k to 0 geometrically, and the gamma system of
#: Eq. Learning_gamma then has condition number ~ 1/mu_k. At 1e-8 the float64 CG still resolves it,
#: and the bias it leaves in d_k (relative 2 mu_k) sits far below any parity tolerance.
MU_FLOOR = 1e-8


# --------------------------------------------------------------------------------------------
# Grid helpers: DFT, filter support S / S^T (Sec. 3.1 "S projects the filter onto its support")
# --------------------------------------------------------------------------------------------

def _axes(nd):
    return tuple(range(-nd, 0))


def rdft(a, nd):
    """Unnormalised real-to-half-spectrum DFT over the last ``nd`` axes."""
    return sfft.rfftn(a, axes=_axes(nd), workers=WORKERS)


def irdft(A, dims):
    """Inverse of ``rdft`` (carries the 1/D factor)."""
    return sfft.irfftn(A, s=tuple(dims), axes=_axes(len(dims)), workers=WORKERS)


def pad_support(d, dims):
    """S^T: put the taps of d (..., *fs) on the grid ``dims``, tap a at offset a-(f-1)//2, wrapped."""
    nd = len(dims)
    fs = d.shape[-nd:]
    out = np.zeros(d.shape[:-nd] + tuple(dims))
    out[(Ellipsis,) + tuple(slice(0, f) for f in fs)] = d
    return np.roll(out, shift=[-((f - 1) // 2) for f in fs], axis=_axes(nd))


def crop_support(a, fs):
    """S: read the support taps (..., *fs) out of a grid array (..., *dims)."""
    nd = len(fs)
    rolled = np.roll(a, shift=[(f - 1) // 2 for f in fs], axis=_axes(nd))
    return rolled[(Ellipsis,) + tuple(slice(0, f) for f in fs)].copy()


def filter_spectra(d, dims):
    """d_hat_{kj} = F(S^T d_{kj}), shape (K, J, *half-spectrum). Sec. 3.2: D_k = F diag(d_hat_k) F^H."""
    return rdft(pad_support(d, dims), len(dims))


# --------------------------------------------------------------------------------------------
# The operators D and D^T (Eq. 2) and the objective (Eq. 1)
# --------------------------------------------------------------------------------------------

def synthesize(d, z):
    """D z: (N, J, *dims) with (Dz)_{nj} = sum_k d_{kj} * z_{nk} (circular convolution, Eq. 1)."""
    dims = z.shape[2:]
    nd = len(dims)
    dh = filter_spectra(d, dims)                     # (K, J, *O)
    zh = rdft(z, nd)                                 # (N, K, *O)
    return irdft(np.einsum("kj...,nk...->nj...", dh, zh), dims)


def correlate(d, lam):
    """D^T lam: (N, K, *dims) with (D^T lam)_{nk} = sum_j d_{kj} ⋆ lam_{nj} (adjoint of ``synthesize``)."""
    dims = lam.shape[2:]
    nd = len(dims)
    dh = filter_spectra(d, dims)
    lh = rdft(lam, nd)
    return irdft(np.einsum("kj...,nj...->nk...", np.conj(dh), lh), dims)


def objective(x, d, z, beta):
    """Eq. 1 summed over images: 1/2 ||x - sum_k d_k * z_k||^2 + beta * sum ||z_k||_1."""
    r = x - synthesize(d, z)
    return 0.5 * float(np.sum(r * r)) + beta * float(np.sum(np.abs(z)))


# --------------------------------------------------------------------------------------------
# Symmetric boundary: the DCT variant mentioned at the start of Sec. 3
# --------------------------------------------------------------------------------------------

def symmetric_extend(a):
    """Half-sample symmetric extension of the last two axes, (..., H, W) -> (..., 2H, 2W):
    rows H..2H-1 repeat rows H-1..0 and columns likewise. Circular convolution on the extension is
    convolution with reflected boundaries on the image."""
    a = np.concatenate([a, a[..., ::-1, :]], axis=-2)
    return np.concatenate([a, a[..., :, ::-1]], axis=-1)


def code_admm_symmetric(x, d, beta, rho, iters, v0=None):
    """Coding with reflected (symmetric) image boundaries: the dual ADMM of ``code_admm`` on the
    symmetric extension of the images (2H x 2W), whose circular boundary is the image's reflection.
    Returns (v, z) on the extended grid (N, K, 2H, 2W)."""
    return code_admm(symmetric_extend(x), d, beta, rho, iters, v0)


def dct_eigenvalues(d, dims):
    """delta_k(u, v) = sum_(a, b) d_k(a, b) cos(pi u a / H) cos(pi v b / W) over the centred tap offsets
    (a, b): for a filter symmetric about its centre, d(-a, -b) = d(a, b), convolution with reflected
    boundaries is diagonal in the type-II DCT with these eigenvalues. d (K, fh, fw) -> (K, H, W)."""
    H, W = dims
    K, fh, fw = d.shape
    oa = np.arange(fh) - (fh - 1) // 2
    ob = np.arange(fw) - (fw - 1) // 2
    ca = np.cos(np.pi * np.outer(np.arange(H), oa) / H)     # (H, fh)
    cb = np.cos(np.pi * np.outer(np.arange(W), ob) / W)     # (W, fw)
    return np.einsum("ua,kab,vb->kuv", ca, d, cb)


def code_admm_dct(x, d, beta, rho, iters):
    """The dual ADMM of Eq. Inference_solution with the type-II DCT in place of the DFT (grey images,
    filters symmetric about their centre): D_k = C^T diag(delta_k) C with C the orthonormal 2-D DCT,
    so the lambda system is diagonal with entries sum_k delta_k^2 + 1/rho. x (N, 1, H, W),
    d (K, 1, fh, fw). Returns (v, z), each (N, K, H, W)."""
    dims = x.shape[2:]
    N, K = x.shape[0], d.shape[0]
    delta = dct_eigenvalues(d[:, 0], dims)                           # (K, H, W)
    C = lambda a: sfft.dctn(a, type=2, axes=(-2, -1), norm="ortho")
    Ci = lambda a: sfft.idctn(a, type=2, axes=(-2, -1), norm="ortho")
    xc = C(x[:, 0])                                                  # (N, H, W)
    denom = np.sum(delta ** 2, axis=0) + 1.0 / rho
    v = np.zeros((N, K) + tuple(dims))
    for _ in range(iters):
        c = np.clip(v, -beta, beta)
        u = 2.0 * c - v
        r = np.einsum("kuv,nkuv->nuv", delta, C(u)) - xc / rho
        lam = r / denom
        w = Ci(delta[None] * lam[:, None])
        v = w - (c - v)
    z = rho * (np.clip(v, -beta, beta) - v)
    return v, z


# --------------------------------------------------------------------------------------------
# Coding subproblem in the dual (Sec. 3.2, Eqs. Inference_Dual / Inference_ADMM / Inference_solution)
# --------------------------------------------------------------------------------------------

def gram_per_frequency(dh):
    """A(w) = sum_k d_hat_{:k}(w) d_hat_{:k}(w)^H, the J x J blocks of D D^T in Fourier (Sec. 3.2, 3.3).

    Returns (*O, J, J) complex."""
    A = np.einsum("kj...,ki...->...ji", dh, np.conj(dh))
    return A


def solve_per_frequency(dh, rho, rhat):
    """lam_hat(w) = (A(w) + I/rho)^{-1} r_hat(w) for every frequency (the lambda-update of
    Eq. Inference_solution; block diagonal with D blocks of J x J, Sec. 3.3).

    rhat: (N, J, *O) -> (N, J, *O)."""
    J = dh.shape[1]
    if J == 1:
        denom = np.sum(np.abs(dh[:, 0]) ** 2, axis=0) + 1.0 / rho      # (*O)
        return rhat / denom
    A = gram_per_frequency(dh) + np.eye(J) / rho                      # (*O, J, J)
    r = np.moveaxis(rhat, 1, -1)[..., None]                           # (N, *O, J, 1)
    lam = np.linalg.solve(A[None], r)[..., 0]
    return np.moveaxis(lam, -1, 1)


def code_admm(x, d, beta, rho, iters, v0=None):
    """Dual ADMM of Eq. Inference_solution, carried in the single state v = D^T lam - z/rho.

    With v = D^T lam^{i+1} - z^i/rho the theta-update is theta = clamp(v) and the multiplier update is
    z = z^i + rho (theta - D^T lam) = rho (clamp(v) - v). The next lambda right-hand side
    D theta + D z / rho - x/rho equals D u - x/rho with u = 2 clamp(v) - v. v = 0 is z = theta = 0.

    x (N,J,*dims), d (K,J,*fs). Returns (v, z), each (N, K, *dims).
    """
    dims = x.shape[2:]
    nd = len(dims)
    N, K = x.shape[0], d.shape[0]
    dh = filter_spectra(d, dims)
    xh = rdft(x, nd)
    v = np.zeros((N, K) + tuple(dims)) if v0 is None else np.array(v0, dtype=np.float64)
    for _ in range(iters):
        c = np.clip(v, -beta, beta)
        u = 2.0 * c - v
        rhat = np.einsum("kj...,nk...->nj...", dh, rdft(u, nd)) - xh / rho
        lamhat = solve_per_frequency(dh, rho, rhat)
        w = irdft(np.einsum("kj...,nj...->nk...", np.conj(dh), lamhat), dims)   # D^T lam
        v = w - (c - v)
    z = rho * (np.clip(v, -beta, beta) - v)
    return v, z


def code_admm_textbook(x, d, beta, rho, iters, z0=None, theta0=None):
    """The three updates of Eq. Inference_solution exactly as printed (lambda, theta, z).

    lam   = (D D^T + I/rho)^{-1} (D theta + D z / rho - x / rho)
    theta = Pi_C(D^T lam - z / rho),  C = {||theta||_inf <= beta}
    z     = z + rho (theta - D^T lam)
    Returns (z, theta, lam)."""
    dims = x.shape[2:]
    nd = len(dims)
    N, K = x.shape[0], d.shape[0]
    dh = filter_spectra(d, dims)
    z = np.zeros((N, K) + tuple(dims)) if z0 is None else np.array(z0, dtype=np.float64)
    theta = np.zeros_like(z) if theta0 is None else np.array(theta0, dtype=np.float64)
    lam = None
    for _ in range(iters):
        rhs = synthesize(d, theta) + synthesize(d, z) / rho - x / rho
        lam = irdft(solve_per_frequency(dh, rho, rdft(rhs, nd)), dims)
        dtl = correlate(d, lam)
        theta = np.clip(dtl - z / rho, -beta, beta)
        z = z + rho * (theta - dtl)
    return z, theta, lam


def duality_gap(x, d, z, beta):
    """Primal value (Eq. 2) minus the dual value of a feasible point (Eq. Inference_Dual).

    The dual point is the residual lam = D z - x scaled into {||D^T lam||_inf <= beta}.
    The dual objective to maximise is -(1/2 lam^T lam + lam^T x). Returns (gap, primal)."""
    r = synthesize(d, z) - x
    primal = 0.5 * float(np.sum(r * r)) + beta * float(np.sum(np.abs(z)))
    dtr = correlate(d, r)
    m = float(np.max(np.abs(dtr)))
    lam = r * (min(1.0, beta / m) if m > 0 else 1.0)
    dual = -(0.5 * float(np.sum(lam * lam)) + float(np.sum(lam * x)))
    return primal - dual, primal


def lipschitz(d, dims):
    """max over frequencies of the largest eigenvalue of A(w), the Lipschitz constant of the
    gradient of 1/2||x - Dz||^2 (the spectrum of D^T D equals that of D D^T)."""
    dh = filter_spectra(d, dims)
    A = gram_per_frequency(dh)
    return float(np.max(np.linalg.eigvalsh(A)))


def fista_code(x, d, beta, iters, z0=None):
    """Accelerated proximal gradient (FISTA) on Eq. 2, step 1/L with the exact Lipschitz constant.

    Independent of the dual ADMM; used only as a pin for it."""
    dims = x.shape[2:]
    L = lipschitz(d, dims)
    N, K = x.shape[0], d.shape[0]
    z = np.zeros((N, K) + tuple(dims)) if z0 is None else np.array(z0, dtype=np.float64)
    y = z.copy()
    t = 1.0
    for _ in range(iters):
        g = correlate(d, synthesize(d, y) - x)
        a = y - g / L
        znew = np.sign(a) * np.maximum(np.abs(a) - beta / L, 0.0)
        tnew = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
        y = znew + ((t - 1.0) / tnew) * (znew - z)
        z, t = znew, tnew
    return z


# --------------------------------------------------------------------------------------------
# Learning subproblem in the dual (Sec. 3.2, Eqs. Learning_* and mu_update)
# --------------------------------------------------------------------------------------------

def conjugate_gradient(apply, b, x0, tol, maxit):
    """Plain CG on a symmetric positive definite operator, stopping at ||r|| <= tol ||b||.

    Returns (x, iterations)."""
    x = np.array(x0, dtype=np.float64)
    r = b - apply(x)
    p = r.copy()
    rr = float(np.sum(r * r))
    bn = float(np.sqrt(np.sum(b * b)))
    it = 0
    while np.sqrt(rr) > tol * bn and it < maxit:
        Ap = apply(p)
        alpha = rr / float(np.sum(p * Ap))
        x = x + alpha * p
        r = r - alpha * Ap
        rr_new = float(np.sum(r * r))
        p = r + (rr_new / rr) * p
        rr = rr_new
        it += 1
    return x, it


class LearningOperators:
    """Z_k and Z_k^T for codes z (N, K, *dims), applied through the DFT (Sec. 3.2, learning).

    (Z_k e)_n = z_{nk} * e (one grid map e per filter, convolved with every image's code);
    (Z_k^T g) = sum_n z_{nk} ⋆ g_n (correlation summed over images; d is shared by all images)."""

    def __init__(self, z):
        self.dims = z.shape[2:]
        self.nd = len(self.dims)
        self.zh = rdft(z, self.nd)                      # (N, K, *O)

    def ZT(self, g):
        """g (N, *dims) -> (K, *dims)."""
        gh = rdft(g, self.nd)
        return irdft(np.einsum("nk...,n...->k...", np.conj(self.zh), gh), self.dims)

    def Z(self, e):
        """e (K, *dims) -> (N, *dims)."""
        eh = rdft(e, self.nd)
        return irdft(np.einsum("nk...,k...->n...", self.zh, eh), self.dims)


def learn_paper(x, z, d, mu, gamma, steps, cg_tol=1e-12, cg_max=500):
    """``steps`` learning steps of Sec. 3.2, then the unit-norm projection.

    One step, for every channel j (the TCSC learning separates along J, Sec. 3.3):
      gamma_j = -(I + sum_k Z_k S^T S Z_k^T / (2 mu_k))^{-1} x_j      (Eq. Learning_gamma; CG, warm start)
      d_{kj}  = -S Z_k^T gamma_j / (2 mu_k)                            (Eq. Learning_Solution)
    and then mu_k <- mu_k ||d_k||_2 over all channels and taps        (Eq. mu_update).
    A filter whose codes are all zero has S Z_k^T gamma = 0: it keeps its d_k and mu_k. mu is floored
    at MU_FLOOR. After the last step d_k <- d_k / max(1, ||d_k||) (the constraint of Eq. 1).

    x (N,J,*dims), z (N,K,*dims), d (K,J,*fs), mu (K,), gamma (N,J,*dims) warm start.
    Returns (d, mu, gamma, cg_iterations list)."""
    K, J = d.shape[0], d.shape[1]
    fs = d.shape[2:]
    ops = LearningOperators(z)
    d = np.array(d, dtype=np.float64)
    mu = np.array(mu, dtype=np.float64)
    gamma = np.array(gamma, dtype=np.float64)
    active = np.array([np.any(z[:, k] != 0) for k in range(K)])
    iters = []
    for _ in range(steps):
        scale = 1.0 / (2.0 * mu)

        def apply(g):
            e = pad_support(crop_support(ops.ZT(g), fs), ops.dims) * scale.reshape((K,) + (1,) * ops.nd)
            return g + ops.Z(e)

        dnew = np.empty_like(d)
        for j in range(J):
            gamma[:, j], it = conjugate_gradient(apply, -x[:, j], gamma[:, j], cg_tol, cg_max)
            iters.append(it)
            dnew[:, j] = -crop_support(ops.ZT(gamma[:, j]), fs) * scale.reshape((K,) + (1,) * len(fs))
        for k in range(K):
            if not active[k]:
                continue
            d[k] = dnew[k]
            mu[k] = max(mu[k] * float(np.sqrt(np.sum(d[k] ** 2))), MU_FLOOR)
    return project_unit_ball(d), mu, gamma, iters


def project_unit_ball(d):
    """d_k <- d_k / max(1, ||d_k||_2), norm over all channels and taps of filter k (Eq. 1 constraint)."""
    K = d.shape[0]
    n = np.sqrt((d.reshape(K, -1) ** 2).sum(axis=1))
    return d / np.maximum(1.0, n).reshape((K,) + (1,) * (d.ndim - 1))


def learn_normal_equations(x, z, d_shape, mu):
    """Minimiser of Eq. Learning_new for fixed mu by a dense solve of its normal equations
    (S Z^T Z S^T + 2 diag(mu)) d = S Z^T x, built column by column. Small instances only; a pin
    for the dual gamma route of ``learn_paper``. Returns d of shape d_shape = (K, J, *fs)."""
    K, J = d_shape[0], d_shape[1]
    fs = tuple(d_shape[2:])
    ops = LearningOperators(z)
    m = int(np.prod(fs))
    n_unk = K * m
    M = np.zeros((n_unk, n_unk))
    for col in range(n_unk):
        e = np.zeros((K,) + fs)
        e.reshape(-1)[col] = 1.0
        y = ops.Z(pad_support(e, ops.dims))                     # Z S^T e   (N, *dims)
        M[:, col] = crop_support(ops.ZT(y), fs).reshape(-1)     # S Z^T Z S^T e
    M += np.diag(np.repeat(2.0 * np.asarray(mu, dtype=np.float64), m))
    d = np.empty((K, J) + fs)
    for j in range(J):
        rhs = crop_support(ops.ZT(x[:, j]), fs).reshape(-1)
        d[:, j] = np.linalg.solve(M, rhs).reshape((K,) + fs)
    return d


# --------------------------------------------------------------------------------------------
# Alternating minimisation (Algorithm 1)
# --------------------------------------------------------------------------------------------

def csc_alternate(x, d0, beta, rho, n_outer, n_code, n_learn, cg_tol=1e-12, cg_max=500, log=None):
    """Algorithm 1: z, theta = 0 and mu_k = 1/2 at the start, then n_outer rounds of
    {n_code dual-ADMM coding iterations (warm-started ADMM state); n_learn learning steps
    (warm-started gamma) followed by the unit-norm projection}.

    Returns dict(d, z, v, mu, gamma, history) where history holds the objective (Eq. 1) after each
    coding and each learning half-step."""
    N, J = x.shape[0], x.shape[1]
    K = d0.shape[0]
    dims = x.shape[2:]
    d = np.array(d0, dtype=np.float64)
    v = np.zeros((N, K) + tuple(dims))
    mu = np.full(K, 0.5)
    gamma = np.zeros((N, J) + tuple(dims))
    history = []
    z = None
    for o in range(n_outer):
        v, z = code_admm(x, d, beta, rho, n_code, v)
        f_code = objective(x, d, z, beta)
        d, mu, gamma, its = learn_paper(x, z, d, mu, gamma, n_learn, cg_tol, cg_max)
        f_learn = objective(x, d, z, beta)
        history.append({"outer": o, "f_code": f_code, "f_learn": f_learn, "cg_iters": its})
        if log is not None:
            log(history[-1])
    return {"d": d, "z": z, "v": v, "mu": mu, "gamma": gamma, "history": history}


# --------------------------------------------------------------------------------------------
# Reverse mode through T unrolled coding iterations (not in the paper)
# --------------------------------------------------------------------------------------------

def _G(a, b, fs):
    """G(a, b)(q) = sum_p b(p) a(p - q) on the filter support: S F^{-1}(conj(F a) F b)."""
    dims = a.shape[-len(fs):]
    nd = len(fs)
    return crop_support(irdft(np.conj(rdft(a, nd)) * rdft(b, nd), dims), fs)


def unrolled_loss_and_grad(x, d, y, beta, rho, T, v0=None):
    """Loss L = mean((D z_T - y)^2) over all N*J*prod(dims) elements, where z_T is the code after T
    iterations of ``code_admm`` from v0 (default 0), and its gradient with respect to x and d.

    Forward, per iteration: c = clamp(v), m = 1[|v| < beta], u = 2c - v, r = D u - x/rho,
    lam = P r with P = (D D^T + I/rho)^{-1}, w = D^T lam, v' = w - c + v.
    Reverse, given vbar' = dL/dv':
      lambar = D vbar';  rbar = P lambar;  ubar = D^T rbar;  xbar -= rbar / rho
      vbar   = (1 - m) vbar' + (2m - 1) ubar
      dbar_{kj} += G(vbar'_k, lam_j) + G(u_k, rbar_j) - G(w_k, rbar_j) - G(ubar_k, lam_j)
    (the last two terms are the derivative of P with respect to d). Seed: e = (2/M)(D z_T - y),
    zbar = D^T e, vbar_T = rho (m_T - 1) zbar, dbar_{kj} += G(z_{T,k}, e_j).
    Returns (loss, gx (N,J,*dims), gd (K,J,*fs))."""
    dims = x.shape[2:]
    nd = len(dims)
    K, J = d.shape[0], d.shape[1]
    fs = d.shape[2:]
    N = x.shape[0]
    dh = filter_spectra(d, dims)
    xh = rdft(x, nd)

    def D(a):      # (N,K,*dims) -> (N,J,*dims)
        return irdft(np.einsum("kj...,nk...->nj...", dh, rdft(a, nd)), dims)

    def DT(a):     # (N,J,*dims) -> (N,K,*dims)
        return irdft(np.einsum("kj...,nj...->nk...", np.conj(dh), rdft(a, nd)), dims)

    def P(a):      # (N,J,*dims) -> (N,J,*dims)
        return irdft(solve_per_frequency(dh, rho, rdft(a, nd)), dims)

    v = np.zeros((N, K) + tuple(dims)) if v0 is None else np.array(v0, dtype=np.float64)
    tape = []
    for _ in range(T):
        c = np.clip(v, -beta, beta)
        u = 2.0 * c - v
        r = irdft(np.einsum("kj...,nk...->nj...", dh, rdft(u, nd)) - xh / rho, dims)
        lam = P(r)
        w = DT(lam)
        tape.append((v, u, lam, w))
        v = w - c + v
    zT = rho * (np.clip(v, -beta, beta) - v)
    resid = D(zT) - y
    M = resid.size
    loss = float(np.sum(resid * resid)) / M
    e = (2.0 / M) * resid
    gd = np.zeros(d.shape)
    gx = np.zeros(x.shape)
    for k in range(K):
        for j in range(J):
            gd[k, j] = sum(_G(zT[n, k], e[n, j], fs) for n in range(N))
    mT = (np.abs(v) < beta).astype(np.float64)
    vbar = rho * (mT - 1.0) * DT(e)
    for (vt, u, lam, w) in reversed(tape):
        m = (np.abs(vt) < beta).astype(np.float64)
        lambar = D(vbar)
        rbar = P(lambar)
        ubar = DT(rbar)
        gx -= rbar / rho
        for k in range(K):
            for j in range(J):
                gd[k, j] += sum(_G(vbar[n, k], lam[n, j], fs) + _G(u[n, k], rbar[n, j], fs)
                                - _G(w[n, k], rbar[n, j], fs) - _G(ubar[n, k], lam[n, j], fs)
                                for n in range(N))
        vbar = (1.0 - m) * vbar + (2.0 * m - 1.0) * ubar
    return loss, gx, gd
