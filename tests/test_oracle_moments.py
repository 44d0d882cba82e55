"""Pins of the FP64 oracle's per-cell discrete functions (CPU only).

Each check is a moment condition the paper fixes, evaluated by brute force over
the discrete velocities on random seeded macros:
  * f^eq, F (Sec. III A, Eqs. 24-25): zeroth/first/second moments.
  * g^eq, G (Sec. III B, Eqs. 29-31): the moments that Eq. (32) inverts for
    u and p, and the momentum flux p I + rho u u.
  * h^eq, H, H~ (Sec. III C, Eqs. 35-36): the appendix's moment conditions
    (Chapman-Enskog analysis), for both D2Q5 and D2Q9 scalar lattices.
  * the implicit scalar moments of Eq. (37): residual of the 2x2 system.
"""
import numpy as np
import pytest

import oracle

CS2 = 1.0 / 3.0
CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1], dtype=float)
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1], dtype=float)


def random_cells(seed, n=25):
    g = np.random.Generator(np.random.PCG64(seed))
    for _ in range(n):
        cell = {k: float(g.normal(0.0, 0.3)) for k in oracle.CELL_INPUTS}
        cell["phi"] = float(g.uniform(-0.05, 1.05))
        cell["c1"] = float(g.uniform(0.0, 2.0))
        cell["c2"] = float(g.uniform(0.0, 2.0))
        cell["ux"], cell["uy"] = (float(v) for v in g.normal(0.0, 0.05, 2))
        yield cell


def random_params(seed, q):
    g = np.random.Generator(np.random.PCG64(seed + 1000))
    return dict(scalar_q=q, W=float(g.uniform(3, 6)), M=0.01, sigma=float(g.uniform(0.001, 0.05)),
                rho1=float(g.uniform(0.5, 2.0)), rho2=float(g.uniform(0.001, 0.5)),
                mu1=0.1, mu2=0.05, D1=float(g.uniform(0.01, 0.3)), D2=float(g.uniform(0.001, 0.3)),
                Keq=float(g.uniform(0.2, 5.0)), A=float(g.uniform(0.0, 1.0)),
                gx=float(g.normal(0, 1e-3)), gy=float(g.normal(0, 1e-3)), g_rho_ref=0.7,
                Fx=float(g.normal(0, 1e-4)), Fy=float(g.normal(0, 1e-4)))


def moments(a, q=9):
    a = np.asarray(a)[:q]
    cx, cy = CX[:q], CY[:q]
    return (a.sum(), np.array([(cx * a).sum(), (cy * a).sum()]),
            np.array([[(cx * cx * a).sum(), (cx * cy * a).sum()],
                      [(cy * cx * a).sum(), (cy * cy * a).sum()]]))


def normal(c):
    n = np.hypot(c["dphix"], c["dphiy"])
    return np.array([c["dphix"], c["dphiy"]]) / (n + 1e-4)


def derived(p, c):
    """Continuum quantities the moment conditions refer to (Eqs. 4-6, 18)."""
    phi = c["phi"]
    # rho of Eq. (6) at phi clipped to the physical range [0, 1]
    rho = min(max(phi, 0.0), 1.0) * (p["rho1"] - p["rho2"]) + p["rho2"]
    beta, k = 12 * p["sigma"] / p["W"], 1.5 * p["sigma"] * p["W"]
    mu_phi = 4 * beta * phi * (phi - 1) * (phi - 0.5) - k * c["lap"]
    G = (rho - p["g_rho_ref"]) * np.array([p["gx"], p["gy"]]) + np.array([p["Fx"], p["Fy"]])
    F = mu_phi * np.array([c["dphix"], c["dphiy"]]) + G
    Dm = p["D1"] * p["D2"] / (p["Keq"] * p["D1"] * (1 - phi) + p["D2"] * phi)
    S1 = p["A"] * Dm * (p["Keq"] * c["c2"] * phi - c["c1"] * (1 - phi))
    flux = (c["dphix"] * (c["dc1x"] + p["Keq"] * c["dc2x"])
            + c["dphiy"] * (c["dc1y"] + p["Keq"] * c["dc2y"]))
    return rho, F, Dm, S1, flux


TOL = 1e-13


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_phase_field_equilibrium_and_source_moments(seed):
    p = random_params(seed, 5)
    for c in random_cells(seed):
        o = oracle.cell_functions(p, c)
        u = np.array([c["ux"], c["uy"]])
        m0, m1, m2 = moments(o["feq"])
        assert m0 == pytest.approx(c["phi"], abs=TOL)
        assert np.allclose(m1, c["phi"] * u, atol=TOL, rtol=0)
        assert np.allclose(m2, CS2 * c["phi"] * np.eye(2), atol=TOL, rtol=0)
        m0, m1, _ = moments(o["F"])
        target = (np.array([c["dtpux"], c["dtpuy"]])
                  + CS2 * 4 * c["phi"] * (1 - c["phi"]) / p["W"] * normal(c))
        assert abs(m0) < TOL
        assert np.allclose(m1, target, atol=TOL, rtol=0)


@pytest.mark.parametrize("seed", [4, 5, 6])
def test_flow_equilibrium_and_force_moments(seed):
    p = random_params(seed, 5)
    for c in random_cells(seed):
        o = oracle.cell_functions(p, c)
        rho, F, *_ = derived(p, c)
        u = np.array([c["ux"], c["uy"]])
        m0, m1, m2 = moments(o["geq"])
        assert abs(m0) < TOL
        assert np.allclose(m1, rho * u, atol=TOL, rtol=0)
        assert np.allclose(m2, c["p"] * np.eye(2) + rho * np.outer(u, u), atol=TOL, rtol=0)
        # Eq. (32b) inverts sum_{i != 0} g_i = p (1 - w0)/cs^2 - rho s_0(u)
        w0 = 4.0 / 9.0
        s0 = w0 * (-(u @ u) / (2 * CS2))
        assert o["geq"][1:].sum() == pytest.approx(c["p"] * (1 - w0) / CS2 - rho * s0, abs=TOL)
        m0, m1, _ = moments(o["G"])
        grad = np.array([c["dphix"], c["dphiy"]])
        assert m0 == pytest.approx((p["rho1"] - p["rho2"]) * (u @ grad), abs=TOL)
        assert np.allclose(m1, F, atol=TOL, rtol=0)
        assert o["G"][0] == 0.0


@pytest.mark.parametrize("q", [5, 9])
@pytest.mark.parametrize("seed", [7, 8])
def test_scalar_moments_match_the_appendix(q, seed):
    p = random_params(seed, q)
    for c in random_cells(seed):
        o = oracle.cell_functions(p, c)
        rho, F, Dm, S1, flux = derived(p, c)
        u = np.array([c["ux"], c["uy"]])
        n = normal(c)
        for k, ck in ((1, c["c1"]), (2, c["c2"])):
            m0, m1, m2 = moments(o["h%deq" % k], q)
            assert m0 == pytest.approx(ck, abs=TOL)
            assert np.allclose(m1, ck * u, atol=TOL, rtol=0)
            assert np.allclose(m2, CS2 * ck * np.eye(2), atol=TOL, rtol=0)
            assert np.all(o["h%deq" % k][q:] == 0.0)
        m0, m1, _ = moments(o["H1"], q)
        assert m0 == pytest.approx(S1, abs=TOL)
        assert np.allclose(m1, np.array([c["dtc1ux"], c["dtc1uy"]])
                           + CS2 * 4 * (1 - c["phi"]) * c["c1"] / p["W"] * n, atol=TOL, rtol=0)
        m0, m1, _ = moments(o["H2"], q)
        assert m0 == pytest.approx(-S1, abs=TOL)
        assert np.allclose(m1, np.array([c["dtc2ux"], c["dtc2uy"]])
                           - CS2 * 4 * c["phi"] * c["c2"] / p["W"] * n, atol=TOL, rtol=0)
        m0, m1, _ = moments(o["Ht1"], q)
        assert m0 == pytest.approx(-Dm * flux, abs=TOL)
        assert np.allclose(m1, 0.0, atol=TOL)
        m0, m1, _ = moments(o["Ht2"], q)
        assert m0 == pytest.approx(Dm * flux, abs=TOL)


def test_implicit_scalar_solve_satisfies_eq37():
    g = np.random.Generator(np.random.PCG64(11))
    for _ in range(200):
        p = dict(D1=float(g.uniform(0.01, 0.3)), D2=float(g.uniform(0.001, 0.3)),
                 Keq=float(g.uniform(0.05, 20)), A=float(g.uniform(0, 5)))
        phi, P1, P2 = float(g.uniform(-0.02, 1.02)), float(g.uniform(0, 3)), float(g.uniform(0, 3))
        c1, c2 = oracle.solve_scalars(p, phi, P1, P2)
        Dm = p["D1"] * p["D2"] / (p["Keq"] * p["D1"] * (1 - phi) + p["D2"] * phi)
        S = p["A"] * Dm * (p["Keq"] * c2 * phi - c1 * (1 - phi))
        assert c1 == pytest.approx(P1 + 0.5 * S, abs=1e-13)
        assert c2 == pytest.approx(P2 - 0.5 * S, abs=1e-13)
        assert c1 + c2 == pytest.approx(P1 + P2, abs=1e-13)


def test_relaxation_times_follow_eqs_27_38():
    s = oracle.OracleSim(dict(nx=2, ny=2, M=0.01, D1=0.1, D2=0.001))
    tf, t1, t2 = s.taus()
    assert tf == pytest.approx(0.53, abs=1e-15)
    assert t1 == pytest.approx(0.8, abs=1e-15)
    assert t2 == pytest.approx(0.503, abs=1e-15)


def test_invalid_parameters_are_rejected():
    for bad in (dict(D1=0.0), dict(M=-1.0), dict(rho2=0.0), dict(scalar_q=7), dict(nx=0)):
        with pytest.raises(ValueError):
            oracle.OracleSim(dict(dict(nx=4, ny=4), **bad))


def test_restart_from_macros_returns_them():
    """init_macros puts every population at its equilibrium (Eqs. 24, 29-30, 35);
    with phi uniform and no force the moments of Eqs. (26), (32), (37) must give
    back the six fields exactly (to rounding), whatever u, p, c1, c2 are."""
    import oracle
    nx, ny = 7, 5
    g = np.random.default_rng(11)
    params = dict(nx=nx, ny=ny, sigma=0.01, rho1=1.0, rho2=0.2, mu1=0.1, mu2=0.05,
                  D1=0.1, D2=0.02, Keq=2.0, A=0.3)
    s = oracle.OracleSim(params)
    phi = np.full((ny, nx), 0.3)
    ux, uy = 0.05 * g.standard_normal((2, ny, nx))
    p = 1e-3 * g.standard_normal((ny, nx))
    c1, c2 = g.uniform(0.1, 1.0, (2, ny, nx))
    s.init_macros(phi, ux, uy, p, c1, c2)
    f = s.fields()
    for name, want in (("phi", phi), ("ux", ux), ("uy", uy), ("p", p), ("c1", c1), ("c2", c2)):
        np.testing.assert_allclose(f[name], want, rtol=1e-12, atol=1e-15, err_msg=name)
