"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names the part of the paper it pins and the independent fact it uses:
dense textbook matrices, closed forms, finite differences, exact recovery, a dense
normal-equation solve, conjugate-gradient identities and the qualitative ordering of
Table 3 (SR beats multi-image interpolation).
"""
import math

import numpy as np
import pytest

import gen
from tests import dense_model as dm


def _asym_psf(seed, size=5):
    r = np.random.default_rng(seed).uniform(0.1, 1.0, size=(size, size))
    return r / r.sum()


# ------------------------------------------------------------------ operator A_k (Eq. 1)

@pytest.mark.parametrize("f,shifts", [
    (2, [(0.0, 0.0), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5)]),
    (3, gen.third_pixel_shifts()[:5]),
    (2, [(1.5, 0.0), (0.0, 1.0), (-0.5, 0.5)]),    # shifts beyond one LR px and negative
])
def test_forward_equals_dense_DBM(orc, f, shifts):
    """Eq. 1: the oracle's A_k equals the product of the textbook D, B, M_k, column by
    column; an asymmetric PSF catches a flipped convolution."""
    h = w = 4 if f == 2 else 3
    psf = _asym_psf(7)
    P = orc.Problem(h, w, f, shifts, psf)
    A = dm.system_matrices(h, w, f, shifts, psf)
    n = P.H * P.W
    for k in range(P.K):
        cols = np.stack([P.forward(k, np.eye(n)[c].reshape(P.H, P.W)).ravel() for c in range(n)], axis=1)
        np.testing.assert_allclose(cols, A[k], rtol=0, atol=1e-15)


def test_adjoint_equals_dense_transpose(orc):
    """A_k^T: the oracle's adjoint equals the transpose of the dense product."""
    h = w = 4
    shifts = [(0.0, 0.0), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5)]
    psf = _asym_psf(8, 3)
    P = orc.Problem(h, w, 2, shifts, psf)
    A = dm.system_matrices(h, w, 2, shifts, psf)
    m = h * w
    for k in range(P.K):
        cols = np.stack([P.adjoint(k, np.eye(m)[c].reshape(h, w)).ravel() for c in range(m)], axis=1)
        np.testing.assert_allclose(cols, A[k].T, rtol=0, atol=1e-15)


@pytest.mark.parametrize("f", [2, 3])
def test_adjoint_identity(orc, f):
    """<A_k x, e> = <x, A_k^T e> on random inputs at a size the dense test does not reach."""
    h, w = 21, 17
    P = orc.Problem(h, w, f, gen.phase_shifts(f), gen.gaussian_psf(5, 0.7))
    x = gen.random_field((P.H, P.W), 1)
    for k in range(P.K):
        e = gen.random_field((h, w), 10 + k)
        lhs = float(np.sum(P.forward(k, x) * e))
        rhs = float(np.sum(x * P.adjoint(k, e)))
        assert abs(lhs - rhs) <= 1e-13 * np.linalg.norm(x) * np.linalg.norm(e)


def test_shift_add_is_multi_image_interpolation(orc):
    """Sec. 4.1.1: with a delta PSF and all f^2 phases, inserting every LR sample at its HR
    position recovers the HR image exactly; the dense formula agrees elsewhere too."""
    for f in (2, 3):
        h, w = 6, 5
        P = orc.Problem(h, w, f, gen.phase_shifts(f), np.ones((1, 1)))
        xt = gen.phantom(P.H, P.W, 3)
        y = P.forward_all(xt)
        np.testing.assert_array_equal(P.shift_add(y), xt)
    # partial and repeated coverage: dense M^T D^T formula, zero where uncovered, the mean
    # where two frames sample the same HR pixel
    h = w = 4
    shifts = [(0.0, 0.0), (0.5, 0.5), (0.0, 0.0)]
    P = orc.Problem(h, w, 2, shifts, np.ones((1, 1)))
    y = gen.random_field((3, h, w), 4)
    D = dm.decimation(h, w, 2)
    num = np.zeros(P.H * P.W)
    cnt = np.zeros(P.H * P.W)
    for k, (dx, dy) in enumerate(shifts):
        MT = dm.motion(P.H, P.W, int(2 * dy), int(2 * dx)).T
        num += MT @ D.T @ y[k].ravel()
        cnt += MT @ D.T @ np.ones(h * w)
    ref = np.where(cnt > 0, num / np.maximum(cnt, 1), 0.0)
    np.testing.assert_allclose(P.shift_add(y).ravel(), ref, atol=1e-15)


# ------------------------------------------------------------------ BTV prior (Eq. 8)

def _psi(t, eps):
    return math.sqrt(t * t + eps * eps) - eps


@pytest.mark.parametrize("eps", [1e-3, 0.1, 0.0])
def test_btv_closed_forms(orc, eps):
    """Eq. 8 closed forms: constant image -> 0; ramp x = s*v -> every pair has t = -s dx;
    checkerboard (+-c) -> t = +-2c exactly when dx + dy is odd."""
    h, w, f, wb, alpha = 5, 6, 2, 3, 0.4
    P = orc.Problem(h, w, f, gen.half_pixel_shifts(), np.ones((1, 1)), lam=1.0,
                    btv_alpha=alpha, btv_w=wb, eps=eps)
    H, W = P.H, P.W
    assert P.reg_value(np.full((H, W), 2.5)) == 0.0
    assert np.all(P.reg_grad(np.full((H, W), 2.5)) == 0.0)
    s = 0.37
    ramp = s * np.tile(np.arange(W, dtype=np.float64), (H, 1))
    want = sum(alpha ** (dx + dy) * (H - dy) * (W - dx) * _psi(s * dx, eps)
               for dy in range(wb) for dx in range(wb) if (dx, dy) != (0, 0))
    assert P.reg_value(ramp) == pytest.approx(want, rel=1e-13)
    c = 0.8
    chk = c * (-1.0) ** np.add.outer(np.arange(H), np.arange(W))
    want = sum(alpha ** (dx + dy) * (H - dy) * (W - dx) * _psi(2 * c, eps)
               for dy in range(wb) for dx in range(wb) if (dx + dy) % 2 == 1)
    assert P.reg_value(chk) == pytest.approx(want, rel=1e-13)


def test_btv_gradient_translation_invariance(orc):
    """R(x + c) = R(x) for every constant c, so the gradient sums to zero; on a ramp every
    interior pixel (two pixels or more from each border) has zero gradient."""
    P = orc.Problem(6, 7, 2, gen.half_pixel_shifts(), np.ones((1, 1)), lam=1.0)
    x = gen.random_field((P.H, P.W), 5)
    assert abs(P.reg_grad(x).sum()) < 1e-12
    ramp = 0.3 * np.tile(np.arange(P.W, dtype=np.float64), (P.H, 1))
    g = P.reg_grad(ramp)
    assert np.all(np.abs(g[2:-2, 2:-2]) < 1e-15)


def test_tikhonov_prior(orc):
    P = orc.Problem(4, 4, 2, gen.half_pixel_shifts(), np.ones((1, 1)), reg=orc.REG_TIKHONOV)
    x = gen.random_field((8, 8), 6)
    assert P.reg_value(x) == pytest.approx(float(np.sum(x * x)), rel=1e-14)
    np.testing.assert_allclose(P.reg_grad(x), 2 * x, rtol=1e-15)


# ------------------------------------------------------------------ derivatives of J (Eq. 9)

def _small_problem(orc, eps, seed=0, lam=0.3):
    P = orc.Problem(7, 6, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.6), lam=lam, eps=eps)
    y = gen.random_field((P.K, P.h, P.w), seed + 1, 0, 2)
    return P, y


def _distinct_levels(P, seed):
    """Image whose pixel values are distinct multiples of 0.01 (every BTV pair |t| >= 0.01)."""
    n = P.H * P.W
    perm = np.random.default_rng(seed).permutation(n)
    return (0.01 * perm).reshape(P.H, P.W)


@pytest.mark.parametrize("eps,tol", [(0.1, 1e-7), (1e-3, 2e-5)])
def test_gradient_central_differences(orc, eps, tol):
    """grad J against central differences of J (every coordinate)."""
    P, y = _small_problem(orc, eps)
    x = _distinct_levels(P, 3)
    J0, g = P.gradient(x, y)
    assert J0 == pytest.approx(P.objective(x, y), rel=1e-14)
    hstep = 1e-6
    fd = np.empty_like(x)
    for i in range(P.H):
        for j in range(P.W):
            xp = x.copy(); xp[i, j] += hstep
            xm = x.copy(); xm[i, j] -= hstep
            fd[i, j] = (P.objective(xp, y) - P.objective(xm, y)) / (2 * hstep)
    assert np.linalg.norm(fd - g) <= tol * np.linalg.norm(g)


@pytest.mark.parametrize("eps", [0.1, 1e-3])
def test_hessvec_and_curvature_central_differences(orc, eps):
    """H(x) p against central differences of the gradient; p.H p in closed form agrees."""
    P, y = _small_problem(orc, eps)
    x = _distinct_levels(P, 4)
    p = gen.random_field((P.H, P.W), 9)
    hstep = 1e-7 if eps == 0.1 else 1e-9
    _, gp = P.gradient(x + hstep * p, y)
    _, gm = P.gradient(x - hstep * p, y)
    fd = (gp - gm) / (2 * hstep)
    hv = P.hessvec(x, p)
    assert np.linalg.norm(fd - hv) <= 1e-6 * np.linalg.norm(hv)
    assert P.curvature(x, p) == pytest.approx(float(np.sum(p * hv)), rel=1e-12)
    # the curvature's data part alone is 2 sum ||A_k p||^2 (lambda = 0 problem)
    P0 = orc.Problem(7, 6, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.6), lam=0.0, eps=eps)
    assert P0.curvature(x, p) == pytest.approx(2 * sum(np.sum(P0.forward(k, p) ** 2) for k in range(4)), rel=1e-13)


# ------------------------------------------------------------------ SCG (Sec. 3.1, Alg. 1)

@pytest.mark.parametrize("f", [2, 3])
def test_scg_exact_recovery(orc, f):
    """Delta PSF, every phase sampled, lambda = 0, noise-free: sum_k A_k^T A_k = I, J is
    ||x - x_true||^2 with Hessian 2I, and SCG reaches x_true within 5 iterations."""
    h, w = 16, 12
    P = orc.Problem(h, w, f, gen.phase_shifts(f), np.ones((1, 1)), lam=0.0)
    xt = gen.phantom(P.H, P.W, 11)
    y = P.forward_all(xt)
    x, tr = P.scg(y, np.zeros_like(xt), 5)
    assert np.linalg.norm(x - xt) <= 1e-10 * np.linalg.norm(xt)
    assert np.all(tr["accept"] == 1)


def _cholesky_solve(A, b):
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        s = A[j, j] - np.dot(L[j, :j], L[j, :j])
        L[j, j] = math.sqrt(s)
        for i in range(j + 1, n):
            L[i, j] = (A[i, j] - np.dot(L[i, :j], L[j, :j])) / L[j, j]
    z = np.zeros(n)
    for i in range(n):
        z[i] = (b[i] - np.dot(L[i, :i], z[:i])) / L[i, i]
    x = np.zeros(n)
    for i in reversed(range(n)):
        x[i] = (z[i] - np.dot(L[i + 1:, i], x[i + 1:])) / L[i, i]
    return x


def test_scg_tikhonov_normal_equations(orc):
    """Tikhonov prior R = ||x||^2: the SCG iterate converges to the solution of the dense
    normal equations (sum_k A_k^T A_k + lambda I) x = sum_k A_k^T y_k, built from the
    textbook matrices and solved by Cholesky (checked against numpy.linalg.solve)."""
    h = w = 8
    f, lam = 2, 0.05
    shifts = gen.half_pixel_shifts()
    psf = gen.gaussian_psf(5, 0.8)
    P = orc.Problem(h, w, f, shifts, psf, lam=lam, reg=orc.REG_TIKHONOV)
    xt = gen.phantom(P.H, P.W, 12)
    y = P.forward_all(xt) + gen.gaussian_noise((4, h, w), 0.01, 13)
    A = dm.system_matrices(h, w, f, shifts, psf)
    N = sum(a.T @ a for a in A) + lam * np.eye(P.H * P.W)
    rhs = sum(a.T @ y[k].ravel() for k, a in enumerate(A))
    xs = _cholesky_solve(N, rhs)
    np.testing.assert_allclose(xs, np.linalg.solve(N, rhs), rtol=1e-10, atol=1e-12)
    # SCG accepts a step by comparing J before and after it (Delta), so once the decrease
    # falls below the FP64 resolution of J the run stalls: near the minimum J changes with
    # the square of the error, which caps the reachable relative error near
    # sqrt(2.2e-16) ~ 1.5e-8.  The tolerance is 5e-8, a few times that floor.
    x, tr = P.scg(y, np.zeros((P.H, P.W)), 60)
    assert np.linalg.norm(x.ravel() - xs) <= 5e-8 * np.linalg.norm(xs)


def test_scg_quadratic_identities(orc):
    """On a quadratic J the SCG step is an exact line search damped by lambda|p|^2:
    every step is accepted with Delta = 2 - p.H p / delta in [1, 2), Moller's lambda is
    divided by 4 at each step, consecutive gradients are orthogonal (r_{k+1} . p_k = 0 up
    to the damping) and the objective falls monotonically."""
    h = w = 8
    P = orc.Problem(h, w, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.8), lam=0.05,
                    reg=orc.REG_TIKHONOV)
    xt = gen.phantom(P.H, P.W, 14)
    y = P.forward_all(xt) + gen.gaussian_noise((4, h, w), 0.01, 15)
    x, tr = P.scg(y, np.zeros((P.H, P.W)), 12)
    assert np.all(tr["accept"] == 1)
    # Delta = 2 - p.H p / delta tends to 1 as Moller's lambda shrinks; E - J(x + alpha p) is
    # then a difference of nearly equal FP64 numbers, hence the 1e-6 slack below 1
    assert np.all(tr["Delta"] >= 1.0 - 1e-6) and np.all(tr["Delta"] < 2.0)
    np.testing.assert_allclose(tr["lam"], 1e-6 / 4.0 ** np.arange(1, 13), rtol=1e-12)
    assert np.all(np.diff(tr["E"]) < 0)
    # quadratic model: E - J(x + alpha p) = alpha mu - alpha^2 (p.H p) / 2, p.H p = delta - lam_k |p|^2
    lam_k = 1e-6 / 4.0 ** np.arange(0, 12)
    pHp = tr["delta"] - lam_k * tr["pn2"]
    drop = tr["alpha"] * tr["mu"] - 0.5 * tr["alpha"] ** 2 * pHp
    big = drop > 1e-6 * tr["E"]     # decreases well above the FP64 resolution of E
    assert big.sum() >= 4
    np.testing.assert_allclose((tr["E"] - tr["J_trial"])[big], drop[big], rtol=1e-7)


def test_scg_orthogonality_on_quadratic(orc):
    """r_{k+1} . p_k = 0 after an exact line search: check it by re-running k steps."""
    h = w = 6
    P = orc.Problem(h, w, 2, gen.half_pixel_shifts(), gen.gaussian_psf(3, 0.8), lam=0.1,
                    reg=orc.REG_TIKHONOV)
    y = gen.random_field((4, h, w), 16, 0, 1)
    x0 = np.zeros((P.H, P.W))
    x1, _ = P.scg(y, x0, 1)
    _, g0 = P.gradient(x0, y)
    _, g1 = P.gradient(x1, y)
    # p_1 = r_1 = -g0; after the first step -g1 is orthogonal to p_1 up to lambda_1 = 1e-6
    assert abs(np.sum(g1 * g0)) <= 1e-5 * np.sum(g0 * g0)


def _tiny(orc, seed=0, lam=0.01, eps=1e-3):
    P = orc.Problem(64, 64, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), lam=lam, eps=eps)
    xt = gen.phantom(128, 128, gen.CONFIG_SEEDS["tiny"] + seed)
    y = P.forward_all(xt) + gen.gaussian_noise((4, 64, 64), 0.01, gen.CONFIG_SEEDS["tiny"] + 100 + seed)
    return P, xt, y


def test_scg_btv_monotone_and_rejections_consistent(orc):
    """The accepted objective never rises; a step is rejected exactly when the trial
    objective is above the current one (delta > 0 on this convex problem)."""
    P, xt, y = _tiny(orc)
    x, tr = P.scg(y, P.shift_add(y), 50)
    acc = tr["accept"] == 1
    assert np.all(tr["delta"] > 0)
    assert np.all((tr["J_trial"] <= tr["E"]) == acc)
    E_next = np.where(acc, tr["J_trial"], tr["E"])
    assert np.all(np.diff(np.concatenate([tr["E"][:1], E_next])) <= 0)
    assert P.objective(x, y) == pytest.approx(E_next[-1], rel=1e-14)


def _rejecting_btv_problem(orc):
    """A BTV problem whose SCG run rejects several steps, the first one among them."""
    h = 32
    P = orc.Problem(h, h, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), lam=0.05, eps=1e-3)
    xt = gen.phantom(2 * h, 2 * h, 2)
    y = P.forward_all(xt) + gen.gaussian_noise((4, h, h), 0.01, 102)
    return P, y


def test_scg_scale_increase_after_rejection(orc):
    """Moller's steps 3, 7 and 8 after a rejected step k: x, p and mu stay, lambda_bar = lambda_k
    and lambda rises by delta_k (1 - Delta_k) / |p_k|^2, so the next attempt along p_k has the
    curvature delta_{k+1} = delta_k + (lambda_{k+1} - lambda_bar) |p_k|^2 = delta_k (2 - Delta_k)
    and the step alpha_{k+1} = alpha_k / (2 - Delta_k): a smaller step after every failure."""
    P, y = _rejecting_btv_problem(orc)
    x, tr = P.scg(y, P.shift_add(y), 20)
    rej = np.where(tr["accept"][:-1] == 0)[0]
    assert len(rej) >= 3 and rej[0] == 0
    for k in rej:
        D = tr["Delta"][k]
        assert D < 0
        assert tr["delta"][k + 1] == pytest.approx(tr["delta"][k] * (2.0 - D), rel=1e-12)
        assert tr["alpha"][k + 1] == pytest.approx(tr["alpha"][k] / (2.0 - D), rel=1e-12)
        assert tr["mu"][k + 1] == tr["mu"][k] and tr["pn2"][k + 1] == tr["pn2"][k]
        assert tr["E"][k + 1] == tr["E"][k]


def test_scg_fresh_direction_curvature(orc):
    """Every first attempt along a direction p_k (k = 0, or after an accepted step) uses
    delta_k = p_k.H(x_k) p_k + lambda_{k-1} |p_k|^2 (step 2, then step 3 with lambda_bar = 0):
    x_k and p_k are read off the iterates (p_k = (x_{j+1} - x_j) / alpha_j at the first accepted
    j >= k) and H from the independently pinned curvature.  The negative-curvature branch of
    step 4 never runs here (it would change delta); it cannot on a convex J with lambda > 0."""
    P, y = _rejecting_btv_problem(orc)
    x0 = P.shift_add(y)
    n = 16
    _, tr = P.scg(y, x0, n)
    acc = tr["accept"]
    iterates = [P.scg(y, x0, k)[0] for k in range(n + 1)]
    checked = 0
    for k in range(n):
        if not (k == 0 or acc[k - 1] == 1):
            continue
        later = [j for j in range(k, n) if acc[j] == 1]
        if not later:
            continue
        j = later[0]
        p = (iterates[j + 1] - iterates[j]) / tr["alpha"][j]
        if k == 0:
            np.testing.assert_allclose(p, -P.gradient(x0, y)[1], rtol=0, atol=1e-9 * np.abs(p).max())
        lam_prev = 1e-6 if k == 0 else tr["lam"][k - 1]
        want = P.curvature(iterates[k], p) + lam_prev * float(np.sum(p * p))
        assert tr["delta"][k] == pytest.approx(want, rel=1e-9), k
        assert tr["pn2"][k] == pytest.approx(float(np.sum(p * p)), rel=1e-9), k
        assert tr["delta"][k] > 0
        checked += 1
    assert checked >= 8


def test_scg_fd_mode_matches_exact_curvature(orc):
    """Moller's finite-difference s_k and its sigma -> 0 limit H p give the same run up
    to O(sigma) on a smooth prior."""
    P, xt, y = _tiny(orc, eps=0.1)
    x0 = P.shift_add(y)
    xa, ta = P.scg(y, x0, 10, orc.HV_EXACT)
    xb, tb = P.scg(y, x0, 10, orc.HV_FD)
    assert np.array_equal(ta["accept"], tb["accept"])
    np.testing.assert_allclose(tb["delta"], ta["delta"], rtol=1e-4)
    assert np.linalg.norm(xa - xb) <= 1e-5 * np.linalg.norm(xa)


def test_sr_beats_multi_image_interpolation(orc):
    """Table 3 ordering (not its values): the SCG reconstruction has a higher PSNR than
    multi-image interpolation against the ground truth."""
    P, xt, y = _tiny(orc)
    x0 = P.shift_add(y)
    x, _ = P.scg(y, x0, 50)

    def psnr(a):
        return 10 * np.log10(4.0 ** 2 / np.mean((a - xt) ** 2))
    assert psnr(x) > psnr(x0) + 1.0


def test_log_convert_closed_form(orc):
    I0 = 40000.0
    c = np.array([40000, 1, 0, 14715, 65535], dtype=np.uint16)
    y = orc.log_convert(c, I0)
    want = [0.0, math.log(I0), math.log(I0), math.log(I0 / 14715), math.log(I0 / 65535)]
    np.testing.assert_allclose(y, want, rtol=0, atol=1e-14)


def test_objective_equals_dense_residual(orc):
    """Eq. 9 with p = 2: J(x) = sum_k ||A_k x - y_k||^2 + lambda R(x), the data term from the
    dense textbook matrices and R from the ramp closed form (x a ramp along columns)."""
    h, w, f, lam, eps = 4, 5, 2, 0.7, 1e-3
    shifts = gen.half_pixel_shifts()
    psf = _asym_psf(21, 3)
    P = orc.Problem(h, w, f, shifts, psf, lam=lam, eps=eps)
    A = dm.system_matrices(h, w, f, shifts, psf)
    s = 0.21
    x = s * np.tile(np.arange(P.W, dtype=np.float64), (P.H, 1))
    y = gen.random_field((4, h, w), 22)
    data = sum(float(np.sum((A[k] @ x.ravel() - y[k].ravel()) ** 2)) for k in range(4))
    reg = sum(0.4 ** (dx + dy) * (P.H - dy) * (P.W - dx) * _psi(s * dx, eps)
              for dy in range(3) for dx in range(3) if (dx, dy) != (0, 0))
    assert P.objective(x, y) == pytest.approx(data + lam * reg, rel=1e-13)


def test_scg_direction_update_from_iterates(orc):
    """Moller's update p_2 = r_2 + beta_1 p_1, beta_1 = (|r_2|^2 - r_2.r_1) / mu_1, read off
    the iterates: x_2 - x_1 = alpha_2 p_2 with r_k = -grad J(x_k) from the gradient."""
    P, xt, y = _tiny(orc, eps=0.05)
    x0 = P.shift_add(y)
    x1, t1 = P.scg(y, x0, 1)
    x2, t2 = P.scg(y, x0, 2)
    assert t2["accept"][0] == 1 and t2["accept"][1] == 1
    _, g0 = P.gradient(x0, y)
    _, g1 = P.gradient(x1, y)
    r1, r2 = -g0, -g1
    p1 = r1
    beta = (np.sum(r2 * r2) - np.sum(r2 * r1)) / t2["mu"][0]
    p2 = r2 + beta * p1
    np.testing.assert_allclose(x2 - x1, t2["alpha"][1] * p2, rtol=0, atol=1e-12 * np.abs(x2 - x1).max() + 1e-15)
    assert t2["mu"][1] == pytest.approx(float(np.sum(p2 * r2)), rel=1e-12)


def test_oracle_matches_committed_golden_trace(orc):
    """Regression: the oracle reproduces the committed tiny-workload SCG trace, written by
    tests/golden/make_golden.py (oracle only)."""
    import json
    import os
    from tests.golden.make_golden import tiny_problem
    ref = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tiny_scg_trace.json")))
    P, xt, y = tiny_problem()
    x, tr = P.scg(y, P.shift_add(y), 50)
    for k, v in ref["trace"].items():
        np.testing.assert_allclose(tr[k], v, rtol=1e-9, atol=1e-300, err_msg=k)
    assert P.objective(x, y) == pytest.approx(ref["J_final"], rel=1e-12)


# ------------------------------------------------------- L1 data term (Sec. 3.1, reading 1)

def _l1_problem(orc, data_eps, lam=0.3, eps=0.1):
    P = orc.Problem(7, 6, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.6), lam=lam, eps=eps,
                    data_norm=orc.NORM_L1, data_eps=data_eps)
    y = gen.random_field((P.K, P.h, P.w), 31, 0, 2)
    return P, y


def test_l1_objective_equals_dense_residual(orc):
    """J(x) = sum_k sum_i psi_d((A_k x - y_k)_i) + lambda R(x), the residual from the dense
    textbook matrices and R from the ramp closed form."""
    h, w, f, lam, eps, data_eps = 4, 5, 2, 0.7, 1e-3, 0.05
    shifts = gen.half_pixel_shifts()
    psf = _asym_psf(21, 3)
    P = orc.Problem(h, w, f, shifts, psf, lam=lam, eps=eps, data_norm=orc.NORM_L1, data_eps=data_eps)
    A = dm.system_matrices(h, w, f, shifts, psf)
    s = 0.21
    x = s * np.tile(np.arange(P.W, dtype=np.float64), (P.H, 1))
    y = gen.random_field((4, h, w), 22)
    data = sum(_psi(float(t), data_eps) for k in range(4) for t in A[k] @ x.ravel() - y[k].ravel())
    reg = sum(0.4 ** (dx + dy) * (P.H - dy) * (P.W - dx) * _psi(s * dx, eps)
              for dy in range(3) for dx in range(3) if (dx, dy) != (0, 0))
    assert P.objective(x, y) == pytest.approx(data + lam * reg, rel=1e-13)


@pytest.mark.parametrize("data_eps,tol", [(0.1, 1e-7), (1e-2, 1e-6)])
def test_l1_gradient_central_differences(orc, data_eps, tol):
    """grad J = sum_k A_k^T psi_d'(A_k x - y_k) + lambda grad R against central differences."""
    P, y = _l1_problem(orc, data_eps)
    x = _distinct_levels(P, 3)
    J0, g = P.gradient(x, y)
    assert J0 == pytest.approx(P.objective(x, y), rel=1e-14)
    hstep = 1e-6
    fd = np.empty_like(x)
    for i in range(P.H):
        for j in range(P.W):
            xp = x.copy(); xp[i, j] += hstep
            xm = x.copy(); xm[i, j] -= hstep
            fd[i, j] = (P.objective(xp, y) - P.objective(xm, y)) / (2 * hstep)
    assert np.linalg.norm(fd - g) <= tol * np.linalg.norm(g)


@pytest.mark.parametrize("data_eps", [0.1, 1e-2])
def test_l1_hessvec_and_curvature_central_differences(orc, data_eps):
    """H(x) p = sum_k A_k^T diag(psi_d'') A_k p + lambda H_R p against central differences of
    the gradient; the closed-form curvature equals p.H p."""
    P, y = _l1_problem(orc, data_eps)
    x = _distinct_levels(P, 4)
    p = gen.random_field((P.H, P.W), 9)
    hstep = 1e-7
    _, gp = P.gradient(x + hstep * p, y)
    _, gm = P.gradient(x - hstep * p, y)
    fd = (gp - gm) / (2 * hstep)
    hv = P.hessvec(x, p, y)
    assert np.linalg.norm(fd - hv) <= 2e-6 * np.linalg.norm(hv)
    assert P.curvature(x, p, y) == pytest.approx(float(np.sum(p * hv)), rel=1e-12)


def test_l1_tends_to_scaled_l2(orc):
    """psi_d(t) = t^2 / (2 eps_d) + O(t^4 / eps_d^3): with a large eps_d the L1 data term, its
    gradient and its curvature are the (independently pinned) L2 ones divided by 2 eps_d."""
    big = 1e4
    common = dict(lam=0.0, eps=0.1)
    P1 = orc.Problem(7, 6, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.6), data_norm=orc.NORM_L1,
                     data_eps=big, **common)
    P2 = orc.Problem(7, 6, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.6), **common)
    y = gen.random_field((4, 7, 6), 41, 0, 2)
    x = gen.random_field((14, 12), 42, 0, 2)
    p = gen.random_field((14, 12), 43)
    J1, g1 = P1.gradient(x, y)
    J2, g2 = P2.gradient(x, y)
    assert 2 * big * J1 == pytest.approx(J2, rel=1e-7)
    assert np.linalg.norm(2 * big * g1 - g2) <= 1e-7 * np.linalg.norm(g2)
    assert 2 * big * P1.curvature(x, p, y) == pytest.approx(P2.curvature(x, p), rel=1e-7)


def test_l1_scg_monotone_and_rejections_consistent(orc):
    """SCG on the L1 objective: the accepted objective never rises, rejections are exactly
    the steps whose trial objective is above the current one."""
    P = orc.Problem(32, 32, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), lam=0.01, eps=1e-3,
                    data_norm=orc.NORM_L1, data_eps=0.01)
    xt = gen.phantom(64, 64, 7)
    y = P.forward_all(xt) + gen.gaussian_noise((4, 32, 32), 0.01, 8)
    x, tr = P.scg(y, P.shift_add(y), 40)
    acc = tr["accept"] == 1
    assert np.all(tr["delta"] > 0)
    assert np.all((tr["J_trial"] <= tr["E"]) == acc)
    E_next = np.where(acc, tr["J_trial"], tr["E"])
    assert np.all(np.diff(np.concatenate([tr["E"][:1], E_next])) <= 0)
    assert E_next[-1] < 0.5 * tr["E"][0]
    with pytest.raises(ValueError):
        orc.Problem(4, 4, 2, gen.half_pixel_shifts(), gen.gaussian_psf(5, 0.5), data_norm=orc.NORM_L1,
                    data_eps=0.0)


# ------------------------------------------------------------------ binning D (Sec. 4.1.1)

@pytest.mark.parametrize("f,shifts", [
    (2, [(0.0, 0.0), (0.5, 0.0), (0.0, 0.5), (0.5, 0.5)]),
    (3, gen.third_pixel_shifts()[:4]),
    (2, [(0.5, 0.0), (0.0, 0.5), (-0.5, 0.0), (0.0, -0.5)]),   # the synthetic study's four directions
])
def test_binned_forward_and_adjoint_equal_dense(orc, f, shifts):
    """Binning D (the mean of each f x f block, Sec. 4.1.1): the oracle's A_k and A_k^T equal
    the textbook product D_bin B M_k and its transpose; an asymmetric PSF catches a flipped
    block offset."""
    h = w = 4 if f == 2 else 3
    psf = _asym_psf(17, 3)
    P = orc.Problem(h, w, f, shifts, psf, decimation=orc.DECIM_BIN)
    A = dm.system_matrices(h, w, f, shifts, psf, binned=True)
    n, m = P.H * P.W, h * w
    for k in range(P.K):
        cols = np.stack([P.forward(k, np.eye(n)[c].reshape(P.H, P.W)).ravel() for c in range(n)], axis=1)
        np.testing.assert_allclose(cols, A[k], rtol=0, atol=1e-15)
        cols = np.stack([P.adjoint(k, np.eye(m)[c].reshape(h, w)).ravel() for c in range(m)], axis=1)
        np.testing.assert_allclose(cols, A[k].T, rtol=0, atol=1e-15)


@pytest.mark.parametrize("f", [2, 3])
def test_binning_is_the_block_mean(orc, f):
    """With a delta PSF and no shift, A x is the mean of each f x f block of x (numpy's
    reshape-and-mean), at a size the dense test does not reach."""
    h, w = 13, 9
    P = orc.Problem(h, w, f, [(0.0, 0.0)], np.ones((1, 1)), decimation=orc.DECIM_BIN)
    x = gen.random_field((P.H, P.W), 21)
    ref = x.reshape(h, f, w, f).mean(axis=(1, 3))
    np.testing.assert_allclose(P.forward(0, x), ref, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("norm", ["l2", "l1"])
def test_binned_gradient_central_differences(orc, norm):
    """grad J with binning against central differences of J (every coordinate), for both
    data terms."""
    kw = dict(data_norm=orc.NORM_L1, data_eps=0.05) if norm == "l1" else {}
    P = orc.Problem(5, 4, 2, gen.half_pixel_shifts(), gen.gaussian_psf(3, 0.6), lam=0.01, eps=0.1,
                    decimation=orc.DECIM_BIN, **kw)
    y = gen.random_field((4, 5, 4), 51, 0, 2)
    x = _distinct_levels(P, 5)
    J0, g = P.gradient(x, y)
    hstep = 1e-6
    fd = np.empty_like(x)
    for i in range(P.H):
        for j in range(P.W):
            xp = x.copy(); xp[i, j] += hstep
            xm = x.copy(); xm[i, j] -= hstep
            fd[i, j] = (P.objective(xp, y) - P.objective(xm, y)) / (2 * hstep)
    assert np.linalg.norm(fd - g) <= 1e-7 * np.linalg.norm(g)
    with pytest.raises(ValueError):
        orc.Problem(4, 4, 2, gen.half_pixel_shifts(), gen.gaussian_psf(3, 0.5), decimation=2)


# ------------------------------------------------------------------ non-integer shifts (bilinear M_k)

FRAC_SHIFTS = [(0.0, 0.0), (0.6, 0.1), (0.15, 0.55), (-0.3, 0.85)]


@pytest.mark.parametrize("binned", [False, True])
def test_bilinear_forward_and_adjoint_equal_dense(orc, binned):
    """Non-integer HR shifts (reading: bilinear M_k): the oracle's A_k and A_k^T equal the
    textbook D B M_k built from a dense bilinear interpolation matrix, and its transpose."""
    h = w = 4
    psf = _asym_psf(23, 3)
    kw = dict(decimation=orc.DECIM_BIN) if binned else {}
    P = orc.Problem(h, w, 2, FRAC_SHIFTS, psf, **kw)
    A = dm.system_matrices(h, w, 2, FRAC_SHIFTS, psf, binned=binned)
    n, m = P.H * P.W, h * w
    for k in range(P.K):
        cols = np.stack([P.forward(k, np.eye(n)[c].reshape(P.H, P.W)).ravel() for c in range(n)], axis=1)
        np.testing.assert_allclose(cols, A[k], rtol=0, atol=1e-15)
        cols = np.stack([P.adjoint(k, np.eye(m)[c].reshape(h, w)).ravel() for c in range(m)], axis=1)
        np.testing.assert_allclose(cols, A[k].T, rtol=0, atol=1e-15)


def test_half_pixel_shift_is_the_mean_of_two_translations(orc):
    """A shift of n + 1/2 HR px is the mean of the translations by n and n + 1, exactly, at a
    size the dense test does not reach (the integer ones are pinned by the dense D B M)."""
    h, w, f = 9, 11, 2
    psf = gen.gaussian_psf(5, 0.7)
    x = gen.random_field((f * h, f * w), 61)
    Ph = orc.Problem(h, w, f, [(0.75, 0.25)], psf)          # HR shift (0.5, 1.5)
    P0 = orc.Problem(h, w, f, [(0.5, 0.0), (0.5, 0.5), (1.0, 0.0), (1.0, 0.5)], psf)
    ref = 0.25 * sum(P0.forward(k, x) for k in range(4))
    np.testing.assert_allclose(Ph.forward(0, x), ref, rtol=1e-14, atol=1e-14)


def test_bilinear_shift_add_closed_form(orc):
    """f = 1, one frame shifted by half a pixel along x: each sample is spread half and half
    over its two neighbouring HR pixels, so x0 is the mean of the two samples there (one at the
    first column)."""
    h, w = 5, 7
    y = gen.random_field((1, h, w), 62)
    P = orc.Problem(h, w, 1, [(0.5, 0.0)], np.ones((1, 1)))
    ref = np.empty((h, w))
    ref[:, 0] = y[0, :, 0]
    ref[:, 1:] = 0.5 * (y[0, :, 1:] + y[0, :, :-1])
    np.testing.assert_allclose(P.shift_add(y), ref, rtol=1e-15)


@pytest.mark.parametrize("norm", ["l2", "l1"])
def test_bilinear_gradient_central_differences(orc, norm):
    kw = dict(data_norm=orc.NORM_L1, data_eps=0.05) if norm == "l1" else {}
    P = orc.Problem(5, 4, 2, FRAC_SHIFTS, gen.gaussian_psf(3, 0.6), lam=0.01, eps=0.1, **kw)
    y = gen.random_field((4, 5, 4), 63, 0, 2)
    x = _distinct_levels(P, 6)
    J0, g = P.gradient(x, y)
    hstep = 1e-6
    fd = np.empty_like(x)
    for i in range(P.H):
        for j in range(P.W):
            xp = x.copy(); xp[i, j] += hstep
            xm = x.copy(); xm[i, j] -= hstep
            fd[i, j] = (P.objective(xp, y) - P.objective(xm, y)) / (2 * hstep)
    assert np.linalg.norm(fd - g) <= 1e-7 * np.linalg.norm(g)


@pytest.mark.parametrize("seed", range(12))
def test_random_options_forward_equals_dense(orc, seed):
    """Seeded random models (factor 1-3, 1-5 frames with integer or non-integer shifts of
    either sign, PSF 1/3/5 with random asymmetric taps, point or binning D): the oracle's A_k
    and A_k^T equal the dense textbook product and its transpose."""
    rng = np.random.default_rng(5000 + seed)
    f = int(rng.integers(1, 4))
    h, w = (int(v) for v in rng.integers(1, 5, size=2))
    K = int(rng.integers(1, 6))
    frac = bool(rng.integers(0, 2))
    shifts = []
    for _ in range(K):
        t = rng.integers(-f, 2 * f, size=2).astype(np.float64)
        if frac:
            t = t + rng.uniform(0, 1, size=2)
        shifts.append((t[0] / f, t[1] / f))
    size = int(rng.choice([1, 3, 5]))
    psf = rng.uniform(0.1, 1.0, size=(size, size))
    binned = bool(rng.integers(0, 2))
    P = orc.Problem(h, w, f, shifts, psf, **(dict(decimation=orc.DECIM_BIN) if binned else {}))
    A = dm.system_matrices(h, w, f, shifts, psf, binned=binned)
    n, m = P.H * P.W, h * w
    for k in range(P.K):
        cols = np.stack([P.forward(k, np.eye(n)[c].reshape(P.H, P.W)).ravel() for c in range(n)], axis=1)
        np.testing.assert_allclose(cols, A[k], rtol=0, atol=1e-14)
        cols = np.stack([P.adjoint(k, np.eye(m)[c].reshape(h, w)).ravel() for c in range(m)], axis=1)
        np.testing.assert_allclose(cols, A[k].T, rtol=0, atol=1e-14)
