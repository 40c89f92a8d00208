"""Pins of the oracle's M-rPIE iteration (Eqs. 5-7): exact fixed point on
consistent data, closed forms on constant inputs, the M-ePIE special case,
step-size-zero invariance, equality of the update numerators with an
independently pinned gradient, and group-order invariance."""
import numpy as np
import pytest

from oracle import grad, model, rpie


def consistent_problem(W=16, M=2, n=3, step=6, seed=0):
    rng = np.random.default_rng(seed)
    H = (n - 1) * step + W + 4
    O = (0.5 + 0.5 * rng.random((H, H))) * np.exp(1j * rng.uniform(-1, 1, (H, H)))
    P = rng.normal(size=(M, W, W)) + 1j * rng.normal(size=(M, W, W))
    iy, ix = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    pos = np.stack([2.0 + step * iy.ravel(), 2.0 + step * ix.ravel()], 1)
    I = model.model_intensities(O, P, pos)
    return O, P, pos, I


def test_fixed_point_on_consistent_data():
    O, P, pos, I = consistent_problem()
    st = rpie.State.create(O, P, pos)
    err = rpie.iterate(st, I, rpie.RPIEParams(gamma=0.1, beta=1.0, eps=0.0, reg_eps=0.0))
    assert err < 1e-26
    np.testing.assert_allclose(st.O, O, atol=1e-13)
    np.testing.assert_allclose(st.P, P, atol=1e-12 * np.abs(P).max())


def test_zero_step_sizes_change_nothing():
    O, P, pos, I = consistent_problem(seed=1)
    I = I * 1.7 + 3.0
    st = rpie.State.create(O, P, pos)
    rpie.iterate(st, I, rpie.RPIEParams(alpha_O=0.0, alpha_P=0.0))
    np.testing.assert_array_equal(st.O, O)
    np.testing.assert_array_equal(st.P, P)


def test_closed_form_constant_probe_and_object():
    # P = p, o = a constant, I = I0 at the zero frequency only: every other
    # frequency of Psi is zero, so the constrained wave is the constant
    # kappa p a with kappa = sqrt(I0) / (|p a| W + eps).  The object update
    # gives o' = a (1 + alpha_O (kappa - 1)) and, with beta = 0, the probe
    # update gives P' = p (1 + alpha_P (kappa - 1)).
    W, p, a, I0, eps = 8, 1.3 * np.exp(0.4j), 0.6 * np.exp(-0.9j), 50.0, 1e-8
    O = np.full((W, W), a)
    P = np.full((1, W, W), p)
    I = np.zeros((1, W, W))
    I[0, W // 2, W // 2] = I0
    kappa = np.sqrt(I0) / (abs(p * a) * W + eps)
    for aO in (1.0, 0.5):
        st = rpie.State.create(O, P, np.zeros((1, 2)))
        rpie.iterate(st, I, rpie.RPIEParams(alpha_O=aO, alpha_P=0.0, gamma=0.3, eps=eps, reg_eps=0.0))
        np.testing.assert_allclose(st.O, a * (1 + aO * (kappa - 1)), rtol=1e-13)
    st = rpie.State.create(O, P, np.zeros((1, 2)))
    rpie.iterate(st, I, rpie.RPIEParams(alpha_O=0.0, alpha_P=0.8, beta=0.0, eps=eps, reg_eps=0.0))
    np.testing.assert_allclose(st.P, p * (1 + 0.8 * (kappa - 1)), rtol=1e-13)


def test_single_mode_beta_gamma_one_is_textbook_epie():
    rng = np.random.default_rng(4)
    W = 16
    O = rng.normal(size=(20, 20)) + 1j * rng.normal(size=(20, 20))
    P = rng.normal(size=(1, W, W)) + 1j * rng.normal(size=(1, W, W))
    I = rng.uniform(0, 5, size=(1, W, W))
    pos = np.array([[2.0, 3.0]])
    st = rpie.State.create(O, P, pos)
    rpie.iterate(st, I, rpie.RPIEParams(alpha_O=0.7, alpha_P=0.9, beta=1.0, gamma=1.0, eps=0.0, reg_eps=0.0))
    # ePIE (Maiden & Rodenburg 2009), written with an explicit DFT matrix
    n = np.arange(W)
    Fm = np.exp(-2j * np.pi * np.outer(n, n) / W) / np.sqrt(W)
    o = O[2:2 + W, 3:3 + W]
    psi = P[0] * o
    Psi = Fm @ psi @ Fm.T
    sqI = np.sqrt(model.from_detector(I[0]))
    psi_c = Fm.conj().T @ (sqI * np.exp(1j * np.angle(Psi))) @ Fm.conj()
    o_new = o + 0.7 * np.conj(P[0]) * (psi_c - psi) / np.max(np.abs(P[0]) ** 2)
    P_new = P[0] + 0.9 * np.conj(o) * (psi_c - psi) / np.max(np.abs(o) ** 2)
    np.testing.assert_allclose(st.O[2:2 + W, 3:3 + W], o_new, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(st.P[0], P_new, rtol=1e-12, atol=1e-12)


def test_update_numerators_are_minus_half_the_gradient():
    # With eps = 0 the object numerator sum_p D_p conj(P_p) equals -1/2 of the
    # gradient of the amplitude loss with respect to the crop, and the probe
    # numerator D_p conj(o) equals -1/2 of dL/dP_p (single position).  The
    # gradient itself is pinned by finite differences in test_oracle_grad.
    rng = np.random.default_rng(7)
    W, M = 16, 2
    O = rng.normal(size=(24, 24)) + 1j * rng.normal(size=(24, 24))
    P = rng.normal(size=(M, W, W)) + 1j * rng.normal(size=(M, W, W))
    I = rng.uniform(0, 20, size=(1, W, W))
    pos = np.array([[3.0, 5.0]])
    _, gO, gP, _ = grad.loss_and_grad(O, P, pos, I, delta=0.0)
    Pmax = np.max(np.sum(np.abs(P) ** 2, 0))
    st = rpie.State.create(O, P, pos)
    rpie.iterate(st, I, rpie.RPIEParams(alpha_O=1.0, alpha_P=1.0, beta=1.0, gamma=1.0, eps=0.0, reg_eps=0.0))
    num_o = (st.O - O)[3:3 + W, 5:5 + W] * Pmax
    np.testing.assert_allclose(num_o, -0.5 * gO[3:3 + W, 5:5 + W], rtol=1e-10, atol=1e-10)
    omax = np.max(np.abs(O[3:3 + W, 5:5 + W]) ** 2)
    np.testing.assert_allclose((st.P - P) * omax, -0.5 * gP, rtol=1e-10, atol=1e-10)


def test_group_members_commute_and_sequential_mode():
    O, P, pos, I = consistent_problem(n=4, step=17, seed=3)   # all boxes disjoint
    I = I * 1.3
    prm = rpie.RPIEParams(update_probe=False)
    a = rpie.State.create(O, P, pos)
    rpie.iterate(a, I, prm)
    b = rpie.State.create(O, P, pos)
    rpie.iterate(b, I, prm, groups=[np.random.default_rng(0).permutation(len(pos))])
    np.testing.assert_allclose(a.O, b.O, atol=1e-14)
    # with the probe update on, the order of the summed numerators only rounds
    prm = rpie.RPIEParams()
    a = rpie.State.create(O, P, pos)
    rpie.iterate(a, I, prm)
    b = rpie.State.create(O, P, pos)
    rpie.iterate(b, I, prm, groups=[np.arange(len(pos))[::-1]])
    np.testing.assert_allclose(a.P, b.P, rtol=1e-12, atol=1e-12 * np.abs(P).max())
    # a group of one position is Eq. 5 exactly: max_group=1 == one group per position
    a = rpie.State.create(O, P, pos)
    rpie.iterate(a, I, rpie.RPIEParams(max_group=1))
    b = rpie.State.create(O, P, pos)
    rpie.iterate(b, I, prm, groups=[np.array([j]) for j in range(len(pos))])
    np.testing.assert_array_equal(a.O, b.O)
    np.testing.assert_array_equal(a.P, b.P)


def test_constraint_fixes_modulus_and_keeps_mode_ratios():
    # After one iteration with alpha=1, gamma=0 on a single position with a
    # probe of constant |sum P|^2, the new model intensity equals I exactly.
    rng = np.random.default_rng(9)
    W, M = 16, 2
    q = np.exp(1j * rng.uniform(-np.pi, np.pi, (M, W, W)))
    P = q / np.sqrt(M)                       # sum_p |P_p|^2 = 1 everywhere
    O = np.exp(1j * rng.uniform(-1, 1, (W, W)))
    I = rng.uniform(1, 10, size=(1, W, W))
    st = rpie.State.create(O, P, np.zeros((1, 2)))
    rpie.iterate(st, I, rpie.RPIEParams(alpha_O=1.0, alpha_P=0.0, gamma=0.0, eps=0.0, reg_eps=0.0))
    # o' = sum_p psi'_p conj(P_p): with M modes this is a projection, so check
    # the constrained waves directly instead
    psi = P * O[None]
    Psi = model.F(psi)
    S = np.sum(np.abs(Psi) ** 2, 0)
    sqI = np.sqrt(model.from_detector(I[0]))
    Psi_c = Psi * sqI / np.sqrt(S)
    np.testing.assert_allclose(np.sum(np.abs(Psi_c) ** 2, 0), model.from_detector(I[0]), rtol=1e-12)
    np.testing.assert_allclose(Psi_c[0] / Psi_c[1], Psi[0] / Psi[1], rtol=1e-12)
    D = model.Finv(Psi_c) - psi
    np.testing.assert_allclose(st.O, O + np.sum(D * np.conj(P), 0), rtol=1e-12, atol=1e-12)


def test_error_decreases_on_noise_free_data_with_true_probe():
    O, P, pos, I = consistent_problem(W=16, M=1, n=4, step=4, seed=11)
    st = rpie.State.create(np.ones_like(O), P, pos)
    errs = rpie.run(st, I, rpie.RPIEParams(update_probe=False, eps=1e-6), 20)
    assert errs[-1] < 0.2 * errs[0]
    assert all(b <= a * 1.05 for a, b in zip(errs, errs[1:]))
