"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: Gaussian moments (the quadrature
property the paper requires of the lattice, Sec. 5), Maxwellian moments of the equilibrium (Eqs. 8,
9, 15), the algebra of the projection (Eq. 19), exact conservation laws, the Chapman-Enskog viscosity
nu = theta (tau - 1/2) (Sec. 6, "tau = mu/p = nu/theta"), the quasi-steady Couette closed form, the
Stokes second problem (Eq. 4), the lattice free-molecular force (Sec. 4.1, Eq. 13), and the
Galilean equivalence of the moving-wall (lab) and body-force (body) frames.  The
closed forms are written out here from the mathematics, not taken from the oracle.
"""
import math

import numpy as np
import pytest

import oracle as orc


def gauss_moment_1d(p, mean=0.0, var=1.0):
    """E[X^p] for X ~ N(mean, var), from the binomial expansion and the central moments
    E[Z^k] = (k-1)!! for even k."""
    tot = 0.0
    for k in range(0, p + 1, 2):
        dfact = math.prod(range(k - 1, 0, -2)) if k else 1
        tot += math.comb(p, k) * mean ** (p - k) * var ** (k / 2) * dfact
    return tot


# ------------------------------------------------------------------------------------------------
# lattice tables (Appendix A; textbook D2Q9)
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("Q,degree", [(37, 9), (9, 5)])
def test_lattice_integrates_gaussian_moments(Q, degree):
    c, w, th = orc.lattice(Q)
    assert len(w) == Q and abs(w.sum() - 1.0) < 1e-14
    for p in range(degree + 1):
        for q in range(degree + 1 - p):
            s = float(np.sum(w * c[:, 0] ** p * c[:, 1] ** q))
            exact = gauss_moment_1d(p, 0.0, th) * gauss_moment_1d(q, 0.0, th)
            assert abs(s - exact) < 2e-12 * max(1.0, abs(exact)), (p, q, s, exact)
    # one degree higher is not integrated: the table is the degree-`degree` rule, not a finer one
    p = degree + 1
    s = float(np.sum(w * c[:, 0] ** p)) if p % 2 == 0 else float(np.sum(w * c[:, 0] ** (p + 1)))
    pe = p if p % 2 == 0 else p + 1
    assert abs(s - gauss_moment_1d(pe, 0.0, th)) > 1e-6


def test_d2q37_theta_and_shells():
    c, w, th = orc.lattice(37)
    # Table footnote: lattice speed c = 1.19697977039307 sqrt(theta); with c = 1 lattice unit
    assert abs(1.0 / math.sqrt(th) - 1.19697977039307) < 1e-14
    speeds = sorted(set(int(x * x + y * y) for x, y in c))
    assert speeds == [0, 1, 2, 4, 5, 8, 9, 10]
    counts = {s: int(sum(1 for x, y in c if x * x + y * y == s)) for s in speeds}
    assert counts == {0: 1, 1: 4, 2: 4, 4: 4, 5: 8, 8: 4, 9: 4, 10: 8}


# ------------------------------------------------------------------------------------------------
# equilibrium (Eq. 15 and its 4th-order continuation) against the Maxwellian (Eqs. 8, 9)
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("Q,order", [(37, 2), (37, 4), (9, 2)])
def test_equilibrium_matches_maxwellian_moments(Q, order):
    c, w, th = orc.lattice(Q)
    rng = np.random.default_rng(15)
    for _ in range(20):
        rho = rng.uniform(0.9, 1.1)
        ux, uy = rng.uniform(-0.1, 0.1, 2)
        feq = orc.equilibrium(Q, order, rho, ux, uy)
        for p in range(order + 1):
            for q in range(order + 1 - p):
                s = float(np.sum(feq * c[:, 0] ** p * c[:, 1] ** q))
                exact = rho * gauss_moment_1d(p, ux, th) * gauss_moment_1d(q, uy, th)
                assert abs(s - exact) < 1e-13 * max(1.0, abs(exact)), (p, q, s, exact)


def test_equilibrium_orders_differ_at_third_moment():
    # H2 misses the Maxwellian's third moment by rho u^3 terms; H4 gets it (a dropped H3 term fails)
    c, w, th = orc.lattice(37)
    rho, ux, uy = 1.0, 0.08, -0.03
    exact = rho * gauss_moment_1d(3, ux, th)
    m2 = float(np.sum(orc.equilibrium(37, 2, rho, ux, uy) * c[:, 0] ** 3))
    m4 = float(np.sum(orc.equilibrium(37, 4, rho, ux, uy) * c[:, 0] ** 3))
    assert abs(m4 - exact) < 1e-14
    assert abs(m2 - exact) > 1e-5


# ------------------------------------------------------------------------------------------------
# projected non-equilibrium part (Eq. 19)
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("Q", [37, 9])
def test_projection_is_the_hermite_projection(Q):
    c, w, th = orc.lattice(Q)
    rng = np.random.default_rng(19)
    feq = orc.equilibrium(Q, 2, 1.02, 0.03, -0.05)
    fadv = feq + 1e-3 * w * rng.standard_normal(Q)
    fne = orc.project(Q, fadv, feq)
    d = fadv - feq
    # same moments of degree <= 2 as f^adv - f^eq ...
    for p, q in [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]:
        m = lambda g: float(np.sum(g * c[:, 0] ** p * c[:, 1] ** q))
        assert abs(m(fne) - (m(d) if (p, q) != (0, 0) else 0.0)) < 1e-16 + 1e-13 * abs(m(d)), (p, q)
    # ... and fne / w is a polynomial of degree <= 2 in c (it lies in H^2)
    basis = np.stack([np.ones(Q), c[:, 0], c[:, 1], c[:, 0] ** 2, c[:, 0] * c[:, 1], c[:, 1] ** 2], 1)
    coef, *_ = np.linalg.lstsq(basis, fne / w, rcond=None)
    assert np.max(np.abs(basis @ coef - fne / w)) < 1e-14


# ------------------------------------------------------------------------------------------------
# body-force source (Guo-type, half-force velocity): its moments, and the moments of one node's
# collision with the force on.  The closed forms follow from the lattice's Gaussian moments,
# sum w c_a c_b = theta d_ab and sum w c_a c_b c_c c_d = theta^2 (d_ab d_cd + d_ac d_bd + d_ad d_bc)
# (exact for both lattices): for S_i = k w_i [c.F/theta + ((c.u)(c.F) - theta u.F)/theta^2],
#   sum S = 0,   sum S c = k F,   sum S c c = k (u F + F u),   k = 1 - 1/(2 tau).
# A flipped sign or a wrong factor on either term of S fails one of these.
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("Q", [37, 9])
def test_force_source_moments(Q):
    c, w, th = orc.lattice(Q)
    rng = np.random.default_rng(23)
    for _ in range(25):
        tau = rng.uniform(0.55, 5.0)
        ux, uy, Fx, Fy = rng.uniform(-0.05, 0.05, 4)
        S = orc.source(Q, tau, ux, uy, Fx, Fy)
        k = 1.0 - 0.5 / tau
        u, F = np.array([ux, uy]), np.array([Fx, Fy])
        scale = np.abs(F).max()
        assert abs(S.sum()) < 1e-15 * scale
        first = np.array([np.sum(S * c[:, a]) for a in (0, 1)])
        assert np.abs(first - k * F).max() < 1e-14 * scale
        second = np.array([[np.sum(S * c[:, a] * c[:, b]) for b in (0, 1)] for a in (0, 1)])
        exact = k * (np.outer(u, F) + np.outer(F, u))
        assert np.abs(second - exact).max() < 1e-14 * scale, (second, exact)


@pytest.mark.parametrize("Q,order,coll", [(37, 2, orc.COLL_REG), (37, 4, orc.COLL_REG), (37, 4, orc.COLL_BGK),
                                          (9, 2, orc.COLL_REG), (9, 2, orc.COLL_BGK)])
def test_collision_with_body_force_moments(Q, order, coll):
    """One node's collision at random (rho, j, Pi) and force F = rho g x: with the half-force velocity
    u = (j + F/2)/rho,
      mass:      sum f* = rho;
      momentum:  sum f* c = j + F  (the source adds (1 - 1/2tau) F, the retained first moment
                 (1 - 1/tau) J^ne with J^ne = -F/2 the rest: exact growth by F per step);
      stress (regularized): sum f* c c = rho theta I + rho u u + (1 - 1/tau)(Pi - rho theta I - rho u u)
                 + (1 - 1/(2 tau))(u F + F u).
    The projection's first Hermite moment is also checked directly: sum fne c = J^ne = -F/2."""
    c, w, th = orc.lattice(Q)
    rng = np.random.default_rng(29)
    for _ in range(20):
        tau = rng.uniform(0.55, 4.0)
        rho = rng.uniform(0.95, 1.05)
        feq0 = orc.equilibrium(Q, 2, rho, *rng.uniform(-0.03, 0.03, 2))
        fadv = feq0 + 2e-3 * w * rng.standard_normal(Q)
        gx = rng.uniform(-1e-3, 1e-3)
        rho = fadv.sum()
        j = np.array([np.sum(fadv * c[:, 0]), np.sum(fadv * c[:, 1])])
        F = np.array([rho * gx, 0.0])
        u = (j + 0.5 * F) / rho
        fout = orc.collide(Q, order, coll, tau, fadv, gx)
        assert abs(fout.sum() - rho) < 1e-14 * rho
        jout = np.array([np.sum(fout * c[:, 0]), np.sum(fout * c[:, 1])])
        assert np.abs(jout - (j + F)).max() < 1e-15 * rho, (jout, j + F)
        # the projection keeps J^ne = sum (f^adv - f^eq) c = j - rho u = -F/2
        feq = orc.equilibrium(Q, order, rho, *u)
        fne = orc.project(Q, fadv, feq)
        Jne = np.array([np.sum(fne * c[:, 0]), np.sum(fne * c[:, 1])])
        assert np.abs(Jne + 0.5 * F).max() < 1e-15 * rho
        if coll == orc.COLL_REG:
            Pi = np.array([[np.sum(fadv * c[:, a] * c[:, b]) for b in (0, 1)] for a in (0, 1)])
            Peq = rho * th * np.eye(2) + rho * np.outer(u, u)
            exact = Peq + (1 - 1 / tau) * (Pi - Peq) + (1 - 0.5 / tau) * (np.outer(u, F) + np.outer(F, u))
            Pout = np.array([[np.sum(fout * c[:, a] * c[:, b]) for b in (0, 1)] for a in (0, 1)])
            assert np.abs(Pout - exact).max() < 1e-14 * rho, (Pout, exact)


# ------------------------------------------------------------------------------------------------
# conservation laws of the whole step
# ------------------------------------------------------------------------------------------------

def _perturbed(Q, nx, ny, label, seed, amp=1e-3):
    c, w, th = orc.lattice(Q)
    rng = np.random.default_rng(seed)
    f = orc.rest_state(Q, nx, ny) * (1.0 + amp * rng.standard_normal((ny, nx, Q)))
    f[label != 0] = orc.rest_state(Q, nx, ny)[label != 0]
    return f


def _mass_momentum(Q, f, label):
    c, _, _ = orc.lattice(Q)
    fl = f[label == 0]
    return fl.sum(), (fl * c[:, 0]).sum(), (fl * c[:, 1]).sum()


CASES = [(9, 2, orc.COLL_BGK), (9, 2, orc.COLL_REG), (37, 2, orc.COLL_REG), (37, 4, orc.COLL_REG),
         (37, 4, orc.COLL_BGK)]


@pytest.mark.parametrize("Q,order,coll", CASES)
def test_periodic_box_conserves_mass_and_momentum(Q, order, coll):
    nx, ny = 11, 9
    lab = np.zeros((ny, nx), np.uint8)
    f = _perturbed(Q, nx, ny, lab, 1)
    m0 = _mass_momentum(Q, f, lab)
    f, F = orc.run(Q, lab, 0.7, 0.1, 0.0, 25, eq_order=order, collision=coll, f=f)
    m1 = _mass_momentum(Q, f, lab)
    assert abs(m1[0] - m0[0]) < 1e-13 * m0[0]
    assert abs(m1[1] - m0[1]) < 1e-13 * m0[0] and abs(m1[2] - m0[2]) < 1e-13 * m0[0]
    assert np.all(F == 0.0)


@pytest.mark.parametrize("Q,order,coll", CASES)
def test_static_walls_conserve_mass(Q, order, coll):
    nx, ny = 24, 20
    lab = orc.geometry_beam(nx, ny, 6, 5)
    f = _perturbed(Q, nx, ny, lab, 2)
    m0 = _mass_momentum(Q, f, lab)
    f, F = orc.run(Q, lab, 0.9, 0.1, 0.0, 20, eq_order=order, collision=coll, f=f)
    m1 = _mass_momentum(Q, f, lab)
    assert abs(m1[0] - m0[0]) < 1e-13 * m0[0]


@pytest.mark.parametrize("Q,order,coll", CASES)
def test_momentum_balance_with_body_force_and_body(Q, order, coll):
    """P_fluid(n+1) - P_fluid(n) = M g(n+1/2) - F_n exactly: the body force adds M g per step and the
    momentum-exchange force is exactly what the fluid gives to the body."""
    nx, ny = 26, 22
    lab = orc.geometry_beam(nx, ny, 7, 6)
    f = _perturbed(Q, nx, ny, lab, 3)
    tau, omega, u0, n0, N = 0.85, 0.21, 2e-3, 5, 12
    prev = _mass_momentum(Q, f, lab)
    M = prev[0]
    f_now = f
    for k in range(N):
        f_now, F = orc.run(Q, lab, tau, omega, u0, 1, eq_order=order, collision=coll, drive=orc.DRIVE_BODY,
                           f=f_now, n0=n0 + k)
        cur = _mass_momentum(Q, f_now, lab)
        g = u0 * omega * math.cos(omega * (n0 + k + 0.5))
        assert abs(cur[0] - M) < 1e-13 * M
        assert abs((cur[1] - prev[1]) - (M * g - F[0, 0])) < 2e-14 * M
        assert abs((cur[2] - prev[2]) - (0.0 - F[0, 1])) < 2e-14 * M
        prev = cur


# ------------------------------------------------------------------------------------------------
# viscosity: shear-wave decay rate -> nu = theta (tau - 1/2)
# ------------------------------------------------------------------------------------------------

def _shear_decay_nu(Q, order, coll, tau, L, steps=400, skip=40):
    c, w, th = orc.lattice(Q)
    k = 2 * math.pi / L
    y = np.arange(L)
    U = 1e-4
    f = np.zeros((L, 1, Q))
    for j in range(L):
        f[j, 0] = orc.equilibrium(Q, order, 1.0, U * math.sin(k * j), 0.0)
    lab = np.zeros((L, 1), np.uint8)
    amps = []
    for n in range(steps):
        f, _ = orc.run(Q, lab, tau, 0.1, 0.0, 1, eq_order=order, collision=coll, f=f, n0=n)
        ux = (f[:, 0, :] * c[:, 0]).sum(1) / f[:, 0, :].sum(1)
        amps.append(2.0 / L * float(np.sum(ux * np.sin(k * y))))
    a = np.log(np.array(amps[skip:]))
    slope = np.polyfit(np.arange(len(a)), a, 1)[0]
    return -slope / k ** 2, th * (tau - 0.5)


@pytest.mark.parametrize("Q,order,coll,tau", [(9, 2, orc.COLL_BGK, 0.8), (9, 2, orc.COLL_REG, 0.7),
                                              (37, 2, orc.COLL_REG, 0.8), (37, 4, orc.COLL_REG, 0.65)])
def test_shear_wave_viscosity(Q, order, coll, tau):
    # nu(k) = nu (1 + O(k^2)): two wavelengths, Richardson extrapolation to k -> 0
    n1, nu = _shear_decay_nu(Q, order, coll, tau, 32)
    n2, _ = _shear_decay_nu(Q, order, coll, tau, 64)
    extrap = n2 + (n2 - n1) / 3.0
    assert abs(n2 - nu) < 1e-2 * nu
    assert abs(extrap - nu) < 1e-4 * nu, (n1, n2, extrap, nu)


# ------------------------------------------------------------------------------------------------
# moving wall + force: quasi-steady Couette flow (D2Q9 half-way bounce-back is exact for Couette)
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("coll", [orc.COLL_BGK, orc.COLL_REG])
def test_quasi_steady_couette_force(coll):
    """Plate (1 row) and static top wall (1 row) H = ny - 2 nodes apart (half-way walls).  For a slow
    wall velocity U(t) the wall shear is rho (-nu U/H - U' H/3) per unit length, up to O(w^2 H^4/nu^2)."""
    nx, H, tau = 3, 8, 0.8
    ny = H + 2
    nu = (tau - 0.5) / 3.0
    omega, u0, N = 2 * math.pi / 100000, 1e-3, 3000
    lab = orc.geometry_plate(9, nx, ny)
    _, F = orc.run(9, lab, tau, omega, u0, N, collision=coll, drive=orc.DRIVE_WALL)
    for n in (N - 200, N - 1):
        t = n + 0.5
        U = u0 * math.sin(omega * t)
        dU = u0 * omega * math.cos(omega * t)
        expect = nx * (-nu * U / H - dU * H / 3.0)
        assert abs(F[n, 0] - expect) < 2e-4 * abs(expect), (F[n, 0], expect)


# ------------------------------------------------------------------------------------------------
# Stokes' second problem (Eq. 4): wall force -rho U0 sqrt(nu w/2)(sin + cos) per unit area
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("Q,coll,in_tol,q_tol", [(9, orc.COLL_BGK, 0.01, 0.01), (9, orc.COLL_REG, 0.01, 0.01),
                                                  (37, orc.COLL_REG, 0.01, 0.03)])
def test_stokes_second_problem(Q, coll, in_tol, q_tol):
    """D2Q37: node-return bounce-back puts the wall of each shell at a different distance, which moves
    the inertial (quadrature) part by a few percent; the dissipative part stays within 1%."""
    c, w, th = orc.lattice(Q)
    nx, ny, tau, P = 2, 200, 0.8, 1000
    omega, u0 = 2 * math.pi / P, 1e-3
    nu = th * (tau - 0.5)
    lab = orc.geometry_plate(Q, nx, ny)
    _, F = orc.run(Q, lab, tau, omega, u0, 4 * P, collision=coll, drive=orc.DRIVE_WALL)
    Fin, Fq = orc.in_phase_quadrature(F[:, 0], omega, orc.DRIVE_WALL, skip=2 * P)
    expect = -u0 * math.sqrt(nu * omega / 2.0) * nx
    assert abs(Fin / expect - 1) < in_tol and abs(Fq / expect - 1) < q_tol, (Fin, Fq, expect)
    assert abs(math.atan2(Fq, Fin) - math.pi * 5 / 4 + 2 * math.pi) < 0.02
    # Eq. 20 for the plate: gamma_bar = sqrt(tau omega) with tau = nu / theta
    gb = orc.gamma_bar(Fin, u0, 1.0, th, nx)
    assert abs(gb / math.sqrt(nu / th * omega) - 1) < in_tol


# ------------------------------------------------------------------------------------------------
# free-molecular limit (Sec. 4.1): collisionless gas against bounce-back walls
# ------------------------------------------------------------------------------------------------

def _lattice_sums(Q):
    c, w, th = orc.lattice(Q)
    inc = c[:, 1] > 0            # populations that hit a wall lying below them (reversed: |c_n|)
    S_nt = float(np.sum(w[inc] * c[inc, 1] * c[inc, 0] ** 2))
    S_3 = float(np.sum(w[inc] * c[inc, 1] ** 3))
    return S_nt, S_3, th


@pytest.mark.parametrize("Q", [37, 9])
def test_free_molecular_tangential_plate(Q):
    """Until reflected particles return, a collisionless gas at rest sends w_i rho0 onto the plate along
    every link; bounce-back then gives exactly F_x = -(2 rho0 U_w / theta) S_nt per unit length with
    S_nt = sum_{c_n<0} w |c_n| c_t^2 (the lattice form of the BB free-molecular force, Eq. 13 with
    F^BB = 2 F^DS)."""
    S_nt, _, th = _lattice_sums(Q)
    nx, ny = 5, 60
    omega, u0 = 0.05, 1e-3
    lab = orc.geometry_plate(Q, nx, ny)
    _, F = orc.run(Q, lab, 1e15, omega, u0, 8, collision=orc.COLL_BGK, drive=orc.DRIVE_WALL)
    for n in range(8):
        U = u0 * math.sin(omega * (n + 0.5))
        assert abs(F[n, 0] - (-2.0 * U / th * S_nt * nx)) < 1e-12 * abs(U) * nx
    if Q == 37:
        # continuum BB value for comparison: sum -> int_{v_n<0} |v_n| v_t^2 f_M = theta^{3/2}/sqrt(2 pi)
        assert abs(S_nt / (th ** 1.5 / math.sqrt(2 * math.pi)) - 1) < 0.15


def test_free_molecular_normal_wall():
    """Wall moving along its normal: F_x = -n_y (rho0 theta + (2 rho0 U/theta) S_3) per row, with
    S_3 = sum_{c_n<0} w |c_n|^3 -> sqrt(2/pi) theta^{3/2} in the continuum (Eq. 13: sqrt(32/pi) L_y
    rho sqrt(theta) u for BB on the two faces normal to the motion)."""
    Q = 37
    _, S_3, th = _lattice_sums(Q)   # symmetric in x <-> y
    nx, ny = 60, 4
    lab = np.zeros((ny, nx), np.uint8)
    lab[:, :3] = 1
    lab[:, nx - 3:] = 2
    omega, u0 = 0.05, 1e-3
    _, F = orc.run(Q, lab, 1e15, omega, u0, 8, collision=orc.COLL_BGK, drive=orc.DRIVE_WALL)
    for n in range(8):
        U = u0 * math.sin(omega * (n + 0.5))
        expect = -ny * (th + 2.0 * U / th * S_3)
        assert abs(F[n, 0] - expect) < 1e-12 * ny
    assert abs(S_3 / (math.sqrt(2 / math.pi) * th ** 1.5) - 1) < 0.02


# ------------------------------------------------------------------------------------------------
# post-processing
# ------------------------------------------------------------------------------------------------

def test_fit_recovers_sinusoid():
    omega = 2 * math.pi / 37.0
    t = np.arange(500) + 0.5
    F = 0.3 * np.sin(omega * t) - 0.7 * np.cos(omega * t) + 0.05
    A, B, C = orc.fit_force(F, omega)
    assert abs(A - 0.3) < 1e-12 and abs(B + 0.7) < 1e-12 and abs(C - 0.05) < 1e-12
    Fin, Fq = orc.in_phase_quadrature(F, omega, orc.DRIVE_BODY)
    assert abs(Fin + 0.3) < 1e-12 and abs(Fq - 0.7) < 1e-12


def test_params_from_tau_omega():
    # tau*omega = (tau_LB - 1/2) omega; Stokes layer of 4 nodes or 128 steps per period
    tl, om, P = orc.params_from_tau_omega(37, 0.01)
    th = 1 / 1.19697977039307 ** 2
    assert P == math.ceil(8 * math.pi / math.sqrt(2 * th * 0.01)) == 213
    assert abs((tl - 0.5) * om - 0.01) < 1e-15 and abs(om - 2 * math.pi / 213) < 1e-15
    for to in (1.0, 10.0, 100.0):
        tl, om, P = orc.params_from_tau_omega(37, to)
        assert P == 128 and abs((tl - 0.5) * om - to) < 1e-12 * to
    tl, om, P = orc.params_from_tau_omega(9, 1e-3)
    assert P == math.ceil(8 * math.pi / math.sqrt(2 / 3 * 1e-3))


# ------------------------------------------------------------------------------------------------
# diffuse-scattering walls (Eq. 11)
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("Q,order,coll", CASES)
def test_diffuse_walls_conserve_mass_and_balance_momentum(Q, order, coll):
    nx, ny = 26, 22
    lab = orc.geometry_beam(nx, ny, 7, 6)
    lab[0, :] = 2                                     # a static wall row as well
    if Q == 37:
        lab[:3, :] = 2
    f = _perturbed(Q, nx, ny, lab, 4)
    tau, omega, u0, n0 = 0.85, 0.21, 2e-3, 3
    prev = _mass_momentum(Q, f, lab)
    M = prev[0]
    f1, F = orc.run(Q, lab, tau, omega, u0, 1, eq_order=order, collision=coll, drive=orc.DRIVE_BODY, f=f, n0=n0,
                    wall=orc.WALL_DS)
    cur = _mass_momentum(Q, f1, lab)
    assert abs(cur[0] - M) < 1e-13 * M
    # the static wall row takes momentum too: only a body-only box gives the exact balance below
    lab2 = orc.geometry_beam(nx, ny, 7, 6)
    f = _perturbed(Q, nx, ny, lab2, 5)
    prev = _mass_momentum(Q, f, lab2)
    f1, F = orc.run(Q, lab2, tau, omega, u0, 1, eq_order=order, collision=coll, drive=orc.DRIVE_BODY, f=f, n0=n0,
                    wall=orc.WALL_DS)
    cur = _mass_momentum(Q, f1, lab2)
    g = u0 * omega * math.cos(omega * (n0 + 0.5))
    assert abs((cur[1] - prev[1]) - (prev[0] * g - F[0, 0])) < 2e-14 * prev[0]
    assert abs((cur[2] - prev[2]) - (0.0 - F[0, 1])) < 2e-14 * prev[0]


@pytest.mark.parametrize("Q", [37, 9])
def test_free_molecular_diffuse_plate_is_half_bounce_back(Q):
    """Sec. 4.1: F^BB = 2 F^DS in free-molecular flow.  Collisionless gas at rest on a tangential
    plate: the diffuse wall returns w_i rho_w (1 + c_i.U/theta + O(U^2)) with rho_w = rho0 (1 + O(U^2)),
    so F_x = -(rho0 U / theta) S_nt per unit length, half the bounce-back value."""
    S_nt, _, th = _lattice_sums(Q)
    nx, ny, omega, u0 = 5, 60, 0.05, 1e-3
    lab = orc.geometry_plate(Q, nx, ny)
    _, F_ds = orc.run(Q, lab, 1e15, omega, u0, 8, collision=orc.COLL_BGK, drive=orc.DRIVE_WALL, wall=orc.WALL_DS)
    _, F_bb = orc.run(Q, lab, 1e15, omega, u0, 8, collision=orc.COLL_BGK, drive=orc.DRIVE_WALL, wall=orc.WALL_BB)
    for n in range(8):
        U = u0 * math.sin(omega * (n + 0.5))
        expect = -U / th * S_nt * nx
        # O(U^2) from rho_w, and FP64 sums of link terms of size w rho0
        assert abs(F_ds[n, 0] - expect) < 1e-6 * abs(expect) + 1e-12 * u0 * nx
        assert abs(F_bb[n, 0] - 2.0 * expect) < 1e-12 * u0 * nx


def test_diffuse_slip_reduction_goes_from_continuum_to_free_molecular():
    """Slip of a diffuse wall lowers the damping, from no effect in the continuum limit (tau*omega
    -> 0, no slip) monotonically down to about the free-molecular ratio 1/2 (F^BB = 2 F^DS, pinned
    exactly above).  D2Q37-H2 plate, gamma_bar(DS)/gamma_bar(BB) at tau*omega = 0.01, 0.1, 1
    (0.975, 0.836, 0.471).  (The paper prints a reduction of 0 - 0.4 over its cases; for this
    discretization the plate at tau*omega = 1 shows a reduction of 0.53, recorded as a discrepancy
    in the design notes.)"""
    Q, nx, ny = 37, 2, 120
    lab = orc.geometry_plate(Q, nx, ny)
    ratios = []
    for to in (0.01, 0.1, 1.0):
        tau, omega, P = orc.params_from_tau_omega(Q, to)
        res = {}
        for wall in (orc.WALL_BB, orc.WALL_DS):
            _, F = orc.run(Q, lab, tau, omega, 1e-3, 4 * P, collision=orc.COLL_REG, drive=orc.DRIVE_WALL, wall=wall)
            res[wall], _ = orc.in_phase_quadrature(F[:, 0], omega, orc.DRIVE_WALL, skip=2 * P)
        ratios.append(res[orc.WALL_DS] / res[orc.WALL_BB])
    assert ratios[0] > 0.95
    assert ratios[0] > ratios[1] > ratios[2] > 0.4, ratios


# ------------------------------------------------------------------------------------------------
# lab frame (moving wall, Sec. 6) against body frame (body force): Galilean equivalence
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("tau_omega", [0.1, 1.0, 10.0])
def test_lab_and_body_frames_agree_up_to_half_a_step(tau_omega):
    """Two independent mechanisms drive the same flow.  In a periodic box, u_B = u_L - V with the
    same periodic pressure turns the linear Stokes problem of a body moving with V(t) into the one of
    a fixed body in fluid pushed by the force density -rho dV/dt, so the force on the body is the
    same function of time (no Froude-Krylov term: the uniform force takes the place of the pressure
    ramp that an unbounded domain would need).  On the lattice the body-frame momentum exchange of
    step n carries the populations collided at step n - 1/2 against n + 1/2 for the moving-wall
    term, so the two histories match after a half-step time shift, i.e. a rotation of (F_in, F_q)
    by omega/2.  The unshifted quadrature differs by about omega/2 of the amplitude (> 1e-2 here), so
    a wrong wall term, drive sign or force stamp fails this pin."""
    Q, n, b = 37, 64, 8
    tau, om, P = orc.params_from_tau_omega(Q, tau_omega)
    lab = orc.geometry_beam(n, n, b, b)
    fits = {}
    for drive in (orc.DRIVE_WALL, orc.DRIVE_BODY):
        _, F = orc.run(Q, lab, tau, om, 1e-3, 6 * P, eq_order=4, drive=drive, nthreads=orc.max_threads())
        fits[drive] = orc.in_phase_quadrature(F[:, 0], om, drive, skip=3 * P)
    li, lq = fits[orc.DRIVE_WALL]
    bi, bq = fits[orc.DRIVE_BODY]
    amp = math.hypot(li, lq)
    c, s = math.cos(om / 2), math.sin(om / 2)
    assert abs(lq - bq) > 1e-2 * amp
    assert abs(li - (bi * c - bq * s)) < 3e-4 * amp
    assert abs(lq - (bq * c + bi * s)) < 3e-4 * amp
