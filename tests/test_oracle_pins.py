"""Pins for the FP64 oracle: each test checks an oracle routine against
something other than itself -- a dense brute-force contraction, a closed form,
a library solver, an identity stated in the paper, finite differences -- so
that a dropped term, a wrong index or a transposed operand fails."""
import numpy as np
import pytest

import oracle
import synth
from conftest import small_problem


def dense(dims, idx, vals):
    T = np.zeros(dims)
    T[tuple(idx)] = vals
    return T


def rand_case(rng, dims=(5, 6, 4), density=0.45, R=3):
    mask = rng.random(dims) < density
    coords = np.nonzero(mask)
    order = rng.permutation(len(coords[0]))          # unsorted input order
    idx = [np.ascontiguousarray(c[order].astype(np.int32)) for c in coords]
    A = [rng.standard_normal((I, R)) for I in dims]
    s = rng.standard_normal(len(order))
    return idx, A, s


# ------------------------------------------------------------ pattern (Sec. 3.4)
def test_counting_sort_is_stable_argsort(rng):
    key = rng.integers(0, 17, size=1000).astype(np.int32)
    perm, row_ptr = oracle.counting_sort(key, 20)
    assert np.array_equal(perm, np.argsort(key, kind="stable"))
    assert np.array_equal(row_ptr, np.concatenate([[0], np.cumsum(np.bincount(key, minlength=20))]))
    assert row_ptr[-1] == 1000


def test_counting_sort_empty_and_range():
    perm, row_ptr = oracle.counting_sort(np.zeros(0, np.int32), 3)
    assert perm.size == 0 and list(row_ptr) == [0, 0, 0, 0]
    with pytest.raises(oracle.OracleError):
        oracle.counting_sort(np.array([0, 3], np.int32), 3)


# ------------------------------------------------------------ TTTP (Sec. 3.3)
def test_tttp_brute_force_dense(rng):
    dims = (5, 6, 4)
    idx, A, s = rand_case(rng, dims)
    M = np.einsum("ir,jr,kr->ijk", *A)
    S = dense(dims, idx, s)
    X = S * M                                              # Omega-hat masked by S
    x = oracle.tttp(dims, idx, s, A)
    np.testing.assert_allclose(x, X[tuple(idx)], rtol=1e-13, atol=1e-13)
    # pattern-only call (s = 1)
    x1 = oracle.tttp(dims, idx, None, A)
    np.testing.assert_allclose(x1, M[tuple(idx)], rtol=1e-13, atol=1e-13)


def test_tttp_skips_missing_factor(rng):
    dims = (5, 6, 4)
    idx, A, s = rand_case(rng, dims)
    x = oracle.tttp(dims, idx, s, [A[0], None, A[2]])
    ref = s * np.einsum("er,er->e", A[0][idx[0]], A[2][idx[2]])
    np.testing.assert_allclose(x, ref, rtol=1e-13, atol=1e-13)
    with pytest.raises(oracle.OracleError):
        oracle.tttp(dims, idx, s, [None, None, None])


def test_tttp_order2_is_sddmm(rng):
    """N = 2: TTTP is the SDDMM S .* (U V^T) (Sec. 3.3)."""
    dims = (7, 9)
    mask = rng.random(dims) < 0.5
    I, J = np.nonzero(mask)
    idx = [I.astype(np.int32), J.astype(np.int32)]
    U, V = rng.standard_normal((7, 4)), rng.standard_normal((9, 4))
    s = rng.standard_normal(len(I))
    x = oracle.tttp(dims, idx, s, [U, V])
    np.testing.assert_allclose(x, (dense(dims, idx, s) * (U @ V.T))[I, J], rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------ MTTKRP (Sec. 3.2)
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_mttkrp_matricized_khatri_rao(rng, mode):
    dims = (5, 6, 4)
    idx, A, s = rand_case(rng, dims)
    T = dense(dims, idx, s)
    others = [n for n in range(3) if n != mode]
    # T_(mode) times the Khatri-Rao product of the other two factors
    Tm = np.moveaxis(T, mode, 0).reshape(dims[mode], -1)
    KR = np.einsum("ar,br->abr", A[others[0]], A[others[1]]).reshape(-1, A[0].shape[1])
    np.testing.assert_allclose(oracle.mttkrp(dims, idx, s, A, mode), Tm @ KR, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------ Solve Factor (Sec. 3.4)
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_solve_factor_dense_normal_equations(rng, mode):
    dims = (5, 6, 4)
    idx, A, s = rand_case(rng, dims, density=0.6)
    w = np.abs(s) + 0.1                                     # positive weights
    lam = 0.3
    rhs = rng.standard_normal((dims[mode], 3))
    out, status, rc = oracle.solve_factor(dims, idx, w, A, mode, rhs, lam)
    assert rc == 0 and not status.any()
    W = dense(dims, idx, w)
    o = [n for n in range(3) if n != mode]
    Wm = np.moveaxis(W, mode, 0)
    # g^(i)_rs = sum_{jk} a_jr b_kr w_ijk a_js b_ks  (Sec. 2.2, written densely)
    G = np.einsum("ijk,jr,kr,js,ks->irs", Wm, A[o[0]], A[o[1]], A[o[0]], A[o[1]])
    for i in range(dims[mode]):
        ref = np.linalg.solve(G[i] + lam * np.eye(3), rhs[i])
        np.testing.assert_allclose(out[i], ref, rtol=1e-12, atol=1e-12)


def test_solve_factor_zeroes_row_gradient():
    """ALS step (Sec. 2.2): after Solve Factor with rhs = MTTKRP(T), the
    Table 1 gradient of the regularized least-squares objective in that factor
    vanishes."""
    dims = (20, 18, 15)
    idx, planted, t = small_problem(dims, 900, 4, seed=7, noise=0.1)
    A = synth.init_factors(dims, 4, seed=7)
    lam = 0.05
    for mode in range(3):
        rhs = oracle.mttkrp(dims, idx, t, A, mode)
        A[mode], _, rc = oracle.solve_factor(dims, idx, None, A, mode, rhs, lam)
        assert rc == 0
        _, g = oracle.loss_grad(dims, idx, t, A, "ls", lam)
        scale = np.abs(rhs).max() + 1.0
        assert np.abs(g[mode]).max() < 1e-10 * scale


def test_solve_factor_full_omega_is_cp_als(rng):
    """Every entry observed: G_i = (V^T V) * (W^T W) for all i (textbook CP-ALS)."""
    dims = (4, 5, 3)
    coords = np.indices(dims).reshape(3, -1)
    order = rng.permutation(coords.shape[1])
    idx = [coords[n][order].astype(np.int32) for n in range(3)]
    A = [rng.standard_normal((I, 2)) for I in dims]
    rhs = rng.standard_normal((dims[0], 2))
    out, _, _ = oracle.solve_factor(dims, idx, None, A, 0, rhs, 0.0)
    G = (A[1].T @ A[1]) * (A[2].T @ A[2])
    np.testing.assert_allclose(out, np.linalg.solve(G, rhs.T).T, rtol=1e-12, atol=1e-12)


def test_solve_factor_rank1_is_ccd_update(rng):
    """R = 1: the ALS row solve equals the coordinate-descent update
    sum v w t / (lambda + sum v^2 w^2) (Sec. 2.3)."""
    dims = (6, 7, 5)
    idx, A, s = rand_case(rng, dims, R=1)
    lam = 0.2
    num = np.zeros(dims[0])
    den = np.zeros(dims[0])
    vw = A[1][idx[1], 0] * A[2][idx[2], 0]
    np.add.at(num, idx[0], vw * s)
    np.add.at(den, idx[0], vw * vw)
    rhs = oracle.mttkrp(dims, idx, s, A, 0)
    out, _, _ = oracle.solve_factor(dims, idx, None, A, 0, rhs, lam)
    np.testing.assert_allclose(out[:, 0], num / (lam + den), rtol=1e-12, atol=1e-14)


def test_solve_factor_empty_row_and_not_spd():
    dims = (4, 3, 3)
    idx = [np.array([0, 0, 2], np.int32), np.array([0, 1, 2], np.int32), np.array([1, 2, 0], np.int32)]
    A = [np.ones((I, 2)) for I in dims]
    rhs = np.arange(8, dtype=np.float64).reshape(4, 2)
    out, st, rc = oracle.solve_factor(dims, idx, None, A, 0, rhs, 0.5)
    assert rc == 0
    np.testing.assert_allclose(out[1], rhs[1] / 0.5)       # empty row: a_i = M_i / lambda
    np.testing.assert_allclose(out[3], rhs[3] / 0.5)
    prev = np.full((4, 2), 7.0)
    # lambda < 0: the rank-1 Grams minus 0.1 I and the empty rows are indefinite
    out, st, rc = oracle.solve_factor(dims, idx, None, A, 0, rhs, -0.1, out=prev)
    assert rc == oracle.ERR_NOT_SPD
    assert list(st) == [1, 1, 1, 1]
    np.testing.assert_array_equal(out, prev)               # rows not written


# ------------------------------------------------------------ ALS (Sec. 2.2)
def test_als_loss_identity():
    """Sec. 2.2: sum (t-m)^2 = sum t^2 + sum_i u_i^T G_i u_i - 2 sum u_ir p_ir."""
    dims = (12, 10, 9)
    idx, _, t = small_problem(dims, 400, 3, seed=3, noise=0.2)
    A = synth.init_factors(dims, 3, seed=3)
    m = oracle.tttp(dims, idx, None, A)
    direct = np.sum((t - m) ** 2)
    P = oracle.mttkrp(dims, idx, t, A, 0)
    Om = dense(dims, idx, np.ones(len(t)))
    G = np.einsum("ijk,jr,kr,js,ks->irs", Om, A[1], A[2], A[1], A[2])
    ident = np.sum(t ** 2) + np.einsum("ir,irs,is->", A[0], G, A[0]) - 2 * np.sum(A[0] * P)
    assert abs(direct - ident) < 1e-10 * direct


def test_als_monotone():
    """ALS is exact block minimization (block Gauss-Seidel, Appendix A): the
    objective never increases."""
    dims = (25, 20, 22)
    idx, _, t = small_problem(dims, 1500, 4, seed=11, noise=0.5)
    A = synth.init_factors(dims, 4, seed=11)
    lam = 1e-2
    f = oracle.objective(dims, idx, t, A, "ls", lam)
    for _ in range(8):
        for d in range(3):
            rhs = oracle.mttkrp(dims, idx, t, A, d)
            A[d], _, _ = oracle.solve_factor(dims, idx, None, A, d, rhs, lam)
            f_new = oracle.objective(dims, idx, t, A, "ls", lam)
            assert f_new <= f * (1 + 1e-12)
            f = f_new


def test_als_recovers_planted_low_rank():
    """A noiseless planted rank-3 tensor is completed: held-out entries match."""
    dims = (30, 30, 30)
    R = 3
    idx_all = synth.distinct_coords(dims, 6000, ("uniform",) * 3, 21)
    planted = synth.factor_matrices(dims, R, "normal", 21)
    m_all = oracle.model_entries(dims, idx_all, planted)
    train = [c[:5000] for c in idx_all]
    test = [c[5000:] for c in idx_all]
    t = m_all[:5000]
    best = np.inf
    for seed in range(3):
        A = synth.init_factors(dims, R, seed=100 + seed)
        for _ in range(300):
            A = oracle.als_sweep(dims, train, t, A, 1e-9)
        pred = oracle.model_entries(dims, test, A)
        rmse = np.sqrt(np.mean((pred - m_all[5000:]) ** 2))
        best = min(best, rmse / np.sqrt(np.mean(m_all ** 2)))
        if best < 1e-4:
            break
    assert best < 1e-4


# ------------------------------------------------------------ losses and gradient (Table 1)
@pytest.mark.parametrize("loss", ["ls", "poisson_log", "poisson_id"])
def test_loss_derivatives_by_differences(loss, rng):
    t = rng.integers(0, 6, size=50).astype(np.float64)
    m = rng.uniform(0.3, 2.0, size=50)
    h = 1e-5
    phi, d1, d2 = oracle.loss_terms(loss, t, m)
    pp, d1p, _ = oracle.loss_terms(loss, t, m + h)
    pm, d1m, _ = oracle.loss_terms(loss, t, m - h)
    np.testing.assert_allclose(d1, (pp - pm) / (2 * h), rtol=1e-7, atol=1e-8)
    np.testing.assert_allclose(d2, (d1p - d1m) / (2 * h), rtol=1e-7, atol=1e-8)


def test_loss_closed_forms():
    t = np.array([3.0, 0.0])
    m = np.array([1.0, 2.0])
    phi, _, _ = oracle.loss_terms("ls", t, m)
    assert list(phi) == [4.0, 4.0]
    phi, _, _ = oracle.loss_terms("poisson_log", t, m)
    np.testing.assert_allclose(phi, [np.e - 3.0, np.e ** 2])
    phi, _, _ = oracle.loss_terms("poisson_id", t, m)
    np.testing.assert_allclose(phi, [1.0, 2.0])
    with pytest.raises(oracle.OracleError) as e:
        oracle.loss_terms("poisson_id", t, np.array([1.0, 0.0]))
    assert e.value.rc == oracle.ERR_DOMAIN


@pytest.mark.parametrize("loss", ["ls", "poisson_log", "poisson_id"])
def test_gradient_central_differences(loss):
    dims = (6, 5, 4)
    R = 3
    if loss == "ls":
        idx, planted, t = small_problem(dims, 60, R, seed=5, noise=0.3)
        A = synth.init_factors(dims, R, seed=5)
    else:
        idx, planted, t = small_problem(dims, 60, R, seed=5, factor="uniform01", recipe="poisson")
        A = synth.perturb(planted, seed=5)
        if loss == "poisson_log":
            A = [0.5 * a for a in A]
    lam = 0.1
    f0, g = oracle.loss_grad(dims, idx, t, A, loss, lam)
    for d in range(3):
        for (i, r) in [(0, 0), (dims[d] - 1, R - 1), (2, 1)]:
            h = 1e-6 * max(1.0, abs(A[d][i, r]))
            Ap = [a.copy() for a in A]
            Am = [a.copy() for a in A]
            Ap[d][i, r] += h
            Am[d][i, r] -= h
            fd = (oracle.objective(dims, idx, t, Ap, loss, lam)
                  - oracle.objective(dims, idx, t, Am, loss, lam)) / (2 * h)
            assert abs(fd - g[d][i, r]) <= 1e-6 * max(1.0, abs(fd))


# ------------------------------------------------------------ Gauss-Newton (Sec. 2.5)
def explicit_jacobian(dims, idx, A):
    """J[e, (p, l, r)] = d m_e / d a^(p)_{l r} = delta_{i_p(e) l} prod_{n != p} a^(n)_{i_n(e) r}."""
    R = A[0].shape[1]
    m = len(idx[0])
    offs = np.concatenate([[0], np.cumsum([I * R for I in dims])])
    J = np.zeros((m, offs[-1]))
    for e in range(m):
        for p in range(3):
            h = np.ones(R)
            for n in range(3):
                if n != p:
                    h = h * A[n][idx[n][e]]
            J[e, offs[p] + idx[p][e] * R: offs[p] + (idx[p][e] + 1) * R] = h
    return J, offs


def flat(blocks):
    return np.concatenate([b.ravel() for b in blocks])


def unflat(v, dims, R):
    out, o = [], 0
    for I in dims:
        out.append(v[o:o + I * R].reshape(I, R))
        o += I * R
    return out


@pytest.mark.parametrize("loss", ["ls", "poisson_log"])
def test_ggn_matvec_explicit(loss, rng):
    dims = (5, 4, 3)
    R = 2
    idx, planted, t = small_problem(dims, 30, R, seed=9, factor="uniform01",
                                    recipe="poisson" if loss != "ls" else "noise", noise=0.1)
    A = synth.perturb(planted, seed=9)
    lam = 0.07
    J, _ = explicit_jacobian(dims, idx, A)
    _, _, d2 = oracle.loss_terms(loss, t, oracle.model_entries(dims, idx, A))
    H = J.T @ (d2[:, None] * J) + 2 * lam * np.eye(J.shape[1])
    x = [rng.standard_normal((I, R)) for I in dims]
    y = oracle.ggn_matvec(dims, idx, t, A, loss, lam, x)
    np.testing.assert_allclose(flat(y), H @ flat(x), rtol=1e-12, atol=1e-12)
    # symmetric and positive definite
    x2 = [rng.standard_normal((I, R)) for I in dims]
    y2 = oracle.ggn_matvec(dims, idx, t, A, loss, lam, x2)
    assert abs(flat(x) @ flat(y2) - flat(x2) @ flat(y)) < 1e-12 * np.abs(flat(y)).sum()
    assert flat(x) @ flat(y) > 0


def test_ggn_equals_hessian_at_exact_fit(rng):
    """At an exact least-squares fit (phi' = 0) Gauss-Newton is Newton: the
    matvec equals the finite-difference Hessian-vector product."""
    dims = (5, 4, 6)
    R = 2
    idx, planted, t = small_problem(dims, 40, R, seed=13, recipe="exact")
    lam = 0.0
    x = [rng.standard_normal((I, R)) for I in dims]
    y = oracle.ggn_matvec(dims, idx, t, planted, "ls", lam, x)
    h = 1e-5
    _, gp = oracle.loss_grad(dims, idx, t, [a + h * v for a, v in zip(planted, x)], "ls", lam)
    _, gm = oracle.loss_grad(dims, idx, t, [a - h * v for a, v in zip(planted, x)], "ls", lam)
    fd = (flat(gp) - flat(gm)) / (2 * h)
    np.testing.assert_allclose(flat(y), fd, rtol=1e-6, atol=1e-7 * np.abs(fd).max())


@pytest.mark.parametrize("precondition", [True, False])
def test_pcg_reaches_dense_solve(precondition, rng):
    """PCG on n unknowns reaches the dense solution after n iterations."""
    dims = (4, 3, 3)
    R = 2
    idx, planted, t = small_problem(dims, 20, R, seed=17, noise=0.1)
    A = synth.perturb(planted, seed=17)
    lam = 0.5
    J, _ = explicit_jacobian(dims, idx, A)
    H = 2 * J.T @ J + 2 * lam * np.eye(J.shape[1])
    b = [rng.standard_normal((I, R)) for I in dims]
    n = J.shape[1]
    x = oracle.pcg(dims, idx, t, A, "ls", lam, b, n, precondition)
    np.testing.assert_allclose(flat(x), np.linalg.solve(H, flat(b)), rtol=1e-8, atol=1e-9)


def test_precond_is_block_diagonal_inverse(rng):
    dims = (4, 3, 5)
    R = 2
    idx, planted, t = small_problem(dims, 25, R, seed=19, noise=0.1)
    A = synth.perturb(planted, seed=19)
    lam = 0.3
    J, offs = explicit_jacobian(dims, idx, A)
    H = 2 * J.T @ J + 2 * lam * np.eye(J.shape[1])
    r = [rng.standard_normal((I, R)) for I in dims]
    z = flat(oracle.precond_apply(dims, idx, t, A, "ls", lam, r))
    fr = flat(r)
    for p in range(3):
        for l in range(dims[p]):
            sl = slice(offs[p] + l * R, offs[p] + (l + 1) * R)
            np.testing.assert_allclose(z[sl], np.linalg.solve(H[sl, sl], fr[sl]), rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------ general-loss ALS (Sec. 2.2)
def test_newton_als_ls_one_step_is_als_solve(rng):
    """For least squares the block objective is quadratic, so one Newton step
    from any starting factor lands on the block minimizer, which is the ALS
    solve (G_i + lambda I) a_i = sum_e h_e t_e (Sec. 2.2) -- here by dense
    normal equations per row."""
    dims = (7, 6, 5)
    idx, A, _ = rand_case(rng, dims, density=0.6, R=3)
    t = rng.standard_normal(len(idx[0]))
    lam = 0.3
    for mode in range(3):
        got, taken = oracle.newton_als_mode(dims, idx, t, A, mode, "ls", lam, inner_iters=1)
        assert taken == 1
        o1, o2 = [d for d in range(3) if d != mode]
        for i in range(dims[mode]):
            sel = idx[mode] == i
            H = A[o1][idx[o1][sel]] * A[o2][idx[o2][sel]]
            want = np.linalg.solve(H.T @ H + lam * np.eye(3), H.T @ t[sel])
            np.testing.assert_allclose(got[mode][i], want, rtol=1e-10, atol=1e-12)
        for d in range(3):
            if d != mode:
                np.testing.assert_array_equal(got[d], A[d])


def test_newton_als_poisson_reaches_block_stationarity():
    """Poisson with the log link (Sec. 5.7): each row problem is convex, so the
    Newton iterations drive the gradient of the objective with respect to the
    factor being updated (pinned by finite differences above) to zero."""
    dims = (15, 12, 10)
    idx, planted, _ = small_problem(dims, 700, 3, seed=5, factor="uniform01", recipe="poisson")
    model = oracle.model_entries(dims, idx, planted)
    t = synth.observe(model, "poisson", 5)
    A = [0.7 * a for a in synth.perturb(planted, 5)]
    lam = 0.1
    _, g0 = oracle.loss_grad(dims, idx, t, A, "poisson_log", lam)
    A1, taken = oracle.newton_als_mode(dims, idx, t, A, 0, "poisson_log", lam, inner_iters=40,
                                       tol=1e-14)
    _, g1 = oracle.loss_grad(dims, idx, t, A1, "poisson_log", lam)
    assert np.linalg.norm(g1[0]) <= 1e-9 * np.linalg.norm(g0[0])
    assert taken >= 2


def test_newton_als_poisson_descends():
    """A general-loss ALS sweep with the paper's inner tolerances (1e-3, at most
    5 Newton steps) does not increase the Poisson objective."""
    dims = (20, 18, 16)
    idx, planted, _ = small_problem(dims, 1500, 4, seed=8, factor="uniform01", recipe="poisson")
    t = synth.observe(oracle.model_entries(dims, idx, planted), "poisson", 8)
    A = [0.8 * a for a in synth.perturb(planted, 8)]
    lam = 0.1
    f = oracle.objective(dims, idx, t, A, "poisson_log", lam)
    for _ in range(3):
        A = oracle.newton_als_sweep(dims, idx, t, A, "poisson_log", lam)
        f_new = oracle.objective(dims, idx, t, A, "poisson_log", lam)
        assert f_new <= f * (1 + 1e-12)
        f = f_new


# ------------------------------------------------------------ full Newton product (Sec. 2.5)
@pytest.mark.parametrize("loss", ["ls", "poisson_log"])
def test_newton_matvec_is_gradient_difference(loss, rng):
    """The full Hessian-vector product equals the central difference of the
    gradient (pinned above) along x, away from an exact fit (phi' != 0)."""
    dims = (9, 8, 7)
    R = 3
    idx, planted, _ = small_problem(dims, 250, R, seed=31, factor="uniform01", recipe="poisson")
    t = synth.observe(oracle.model_entries(dims, idx, planted), "poisson", 31)
    A = [0.9 * a for a in synth.perturb(planted, 31)]
    x = [rng.standard_normal((I, R)) for I in dims]
    lam = 0.05
    eps = 1e-5
    _, gp = oracle.loss_grad(dims, idx, t, [a + eps * v for a, v in zip(A, x)], loss, lam)
    _, gm = oracle.loss_grad(dims, idx, t, [a - eps * v for a, v in zip(A, x)], loss, lam)
    y = oracle.newton_matvec(dims, idx, t, A, loss, lam, x)
    for d in range(3):
        fd = (gp[d] - gm[d]) / (2 * eps)
        assert np.linalg.norm(y[d] - fd) <= 1e-7 * np.linalg.norm(fd)
    # and it differs from the Gauss-Newton product (the phi' term is present)
    g = oracle.ggn_matvec(dims, idx, t, A, loss, lam, x)
    assert sum(np.linalg.norm(a - b) for a, b in zip(y, g)) > 1e-3 * sum(np.linalg.norm(b) for b in g)


def test_newton_matvec_symmetric(rng):
    dims = (8, 7, 6)
    idx, planted, t = small_problem(dims, 200, 3, seed=33, noise=0.3)
    A = synth.init_factors(dims, 3, seed=33)
    x = [rng.standard_normal((I, 3)) for I in dims]
    z = [rng.standard_normal((I, 3)) for I in dims]
    hx = oracle.newton_matvec(dims, idx, t, A, "ls", 0.1, x)
    hz = oracle.newton_matvec(dims, idx, t, A, "ls", 0.1, z)
    a = sum(np.vdot(u, v) for u, v in zip(z, hx))
    b = sum(np.vdot(u, v) for u, v in zip(hz, x))
    assert abs(a - b) <= 1e-11 * abs(a)


# ------------------------------------------------------------ coordinate minimization (Sec. 2.3)
def test_ccd_rank1_is_als_rank1():
    """Sec. 2.3: for least squares a coordinate step is a rank-1 ALS step, so
    with R = 1 a CCD++ sweep equals an ALS sweep."""
    dims = (14, 12, 10)
    idx, _, t = small_problem(dims, 600, 2, seed=41, noise=0.2)
    A = synth.init_factors(dims, 1, seed=41)
    c = oracle.ccd_sweep(dims, idx, t, A, 0.3)
    a = oracle.als_sweep(dims, idx, t, A, 0.3)
    for d in range(3):
        np.testing.assert_allclose(c[d], a[d], rtol=1e-11, atol=1e-13)


def test_ccd_each_coordinate_is_minimized(rng):
    """Each column update is the exact minimizer of the LS objective along that
    column, row by row: the partial derivatives of f (Table 1 gradient, pinned
    by differences above) in column r of the factor just updated vanish."""
    dims = (9, 8, 7)
    idx, _, t = small_problem(dims, 300, 3, seed=43, noise=0.3)
    A = synth.init_factors(dims, 3, seed=43)
    lam = 0.2
    out = oracle.ccd_sweep(dims, idx, t, A, lam)
    # the last update of the sweep is column R-1 of the last factor: its partial
    # derivatives are zero at the returned point (f uses lambda on ||A||^2 with the
    # factor-2 convention of Table 1: grad = 2 sum h (m - t) + 2 lambda a)
    _, g = oracle.loss_grad(dims, idx, t, out, "ls", lam)
    G = np.abs(g[2][:, -1]).max()
    assert G <= 1e-10 * np.abs(g[0]).max()


def test_ccd_monotone():
    dims = (20, 18, 16)
    idx, _, t = small_problem(dims, 1200, 4, seed=45, noise=0.5)
    A = synth.init_factors(dims, 4, seed=45)
    lam = 0.05
    f = oracle.objective(dims, idx, t, A, "ls", lam)
    for _ in range(4):
        A = oracle.ccd_sweep(dims, idx, t, A, lam)
        f_new = oracle.objective(dims, idx, t, A, "ls", lam)
        assert f_new <= f * (1 + 1e-12)
        f = f_new


# ------------------------------------------- coordinate minimization, general loss (Sec. 2.3)
def _poisson_small(dims, nnz, R, seed):
    idx, planted, t = small_problem(dims, nnz, R, seed, factor="uniform01", recipe="poisson")
    return idx, t, [0.8 * a for a in planted]


def test_ccd_newton_ls_one_step_is_ccd():
    """Sec. 2.3: for least squares one Newton step per column is the CCD++
    update (pinned above), and a second step finds nothing left to do."""
    dims = (14, 12, 10)
    idx, _, t = small_problem(dims, 700, 3, seed=51, noise=0.2)
    A = synth.init_factors(dims, 3, seed=51)
    ref = oracle.ccd_sweep(dims, idx, t, A, 0.3)
    one, steps = oracle.ccd_newton_sweep(dims, idx, t, A, "ls", 0.3, inner_iters=1)
    assert (steps == 1).all()
    two, steps2 = oracle.ccd_newton_sweep(dims, idx, t, A, "ls", 0.3, inner_iters=5, tol=1e-6)
    assert (steps2 == 2).all()
    for d in range(3):
        np.testing.assert_allclose(one[d], ref[d], rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(two[d], ref[d], rtol=1e-11, atol=1e-13)


def test_ccd_newton_step_is_the_coordinate_newton_step():
    """One step on column r = 0 of A^(0) is, for every row i, -f'/f'' of the
    objective along u_i0, with both derivatives taken by central differences
    of the objective itself (the first update of the sweep)."""
    dims = (7, 6, 5)
    idx, t, A = _poisson_small(dims, 150, 2, seed=53)
    lam = 0.4
    out, _ = oracle.ccd_newton_sweep(dims, idx, t, A, "poisson_log", lam, inner_iters=1)
    got = out[0][:, 0] - A[0][:, 0]
    h = 1e-4
    for i in range(dims[0]):
        def f(delta):
            B = [a.copy() for a in A]
            B[0][i, 0] += delta
            return oracle.objective(dims, idx, t, B, "poisson_log", lam)
        f0, fp, fm = f(0.0), f(h), f(-h)
        d1 = (fp - fm) / (2 * h)
        d2 = (fp - 2 * f0 + fm) / (h * h)
        assert abs(got[i] - (-d1 / d2)) <= 1e-5 * max(1.0, abs(d1 / d2)), i


def test_ccd_newton_converges_to_column_stationarity():
    """With many steps each column reaches its minimizer: the gradient (Table 1,
    pinned above) in the last updated column vanishes at the end of the sweep."""
    dims = (9, 8, 7)
    idx, t, A = _poisson_small(dims, 300, 3, seed=55)
    lam = 1.0
    out, steps = oracle.ccd_newton_sweep(dims, idx, t, A, "poisson_log", lam, inner_iters=60,
                                         tol=1e-13)
    assert steps.max() < 60
    _, g = oracle.loss_grad(dims, idx, t, out, "poisson_log", lam)
    assert np.abs(g[2][:, -1]).max() <= 1e-9 * np.abs(g[0]).max()


def test_ccd_newton_poisson_monotone():
    """Columns minimized exactly (convex in each coordinate for the log link)
    make every sweep non-increasing; lambda = 1 as for coordinate minimization
    in Sec. 5.7."""
    dims = (16, 14, 12)
    idx, t, A = _poisson_small(dims, 900, 4, seed=57)
    lam = 1.0
    f = oracle.objective(dims, idx, t, A, "poisson_log", lam)
    for _ in range(3):
        A, _ = oracle.ccd_newton_sweep(dims, idx, t, A, "poisson_log", lam, inner_iters=40,
                                       tol=1e-12)
        f_new = oracle.objective(dims, idx, t, A, "poisson_log", lam)
        assert f_new <= f * (1 + 1e-12)
        f = f_new


def test_oracle_index_dtype_does_not_matter():
    """Index arrays of any integer type are converted for the C code; the
    converted copies must live through the call (int64 indices once read
    freed memory), so int64 and int32 inputs give identical results."""
    rng = np.random.default_rng(77)
    dims, R, m = (300, 200, 100), 4, 3000
    i64 = [rng.integers(0, I, m) for I in dims]
    i32 = [c.astype(np.int32) for c in i64]
    t = rng.standard_normal(m)
    A = [rng.standard_normal((I, R)) for I in dims]
    x = [rng.standard_normal((I, R)) for I in dims]
    for _ in range(3):     # repeated, so freed copies would be reused
        assert np.array_equal(oracle.tttp(dims, i64, t, A), oracle.tttp(dims, i32, t, A))
        for d in range(3):
            assert np.array_equal(oracle.mttkrp(dims, i64, t, A, d), oracle.mttkrp(dims, i32, t, A, d))
            rhs = rng.standard_normal((dims[d], R))
            a = oracle.solve_factor(dims, i64, None, A, d, rhs, 0.1)[0]
            b = oracle.solve_factor(dims, i32, None, A, d, rhs, 0.1)[0]
            assert np.array_equal(a, b)
        f1, g1 = oracle.loss_grad(dims, i64, t, A, "ls", 0.1)
        f2, g2 = oracle.loss_grad(dims, i32, t, A, "ls", 0.1)
        assert f1 == f2 and all(np.array_equal(u, v) for u, v in zip(g1, g2))
        y1 = oracle.ggn_matvec(dims, i64, t, A, "ls", 0.1, x)
        y2 = oracle.ggn_matvec(dims, i32, t, A, "ls", 0.1, x)
        assert all(np.array_equal(u, v) for u, v in zip(y1, y2))


# ---------------------------------------------------------------- OpenMP build
def test_openmp_build_is_bit_identical():
    """The OpenMP build of the oracle (the timed CPU baseline) only splits
    independent loops; every routine must give bit-identical results to the
    plain build, which the pins above check against the mathematics."""
    dims = (37, 29, 23)
    idx, planted, t = small_problem(dims, 3000, 4, 91, noise=0.05)
    A = [a * 1.03 for a in planted]
    rng = np.random.default_rng(5)
    x = [rng.standard_normal(a.shape) for a in A]
    s = rng.uniform(0.5, 1.5, len(t))

    def run():
        out = [oracle.tttp(dims, idx, t, A), oracle.tttp(dims, idx, None, [A[0], None, A[2]])]
        for d in range(3):
            out.append(oracle.mttkrp(dims, idx, s, A, d))
            rhs = oracle.mttkrp(dims, idx, t, A, d)
            out.append(oracle.solve_factor(dims, idx, s, A, d, rhs, 0.05)[0])
        for loss in ("ls", "poisson_log"):
            f, g = oracle.loss_grad(dims, idx, t, A, loss, 0.1)
            out += [np.array([f])] + g
            out += oracle.ggn_matvec(dims, idx, t, A, loss, 0.1, x)
        out += oracle.ggn_step(dims, idx, t, A, "ls", 0.1, 4)
        return out

    oracle.set_parallel(False)
    plain = run()
    try:
        assert oracle.set_parallel(True, 4) == 4
        par = run()
    finally:
        oracle.set_parallel(False)
    assert len(plain) == len(par)
    for a, b in zip(plain, par):
        assert np.array_equal(a, b)
