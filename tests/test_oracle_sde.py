"""Pins of the oracle's particle SDE updates against closed forms.

Eq. Lagrangian-velocity: with frozen homogeneous statistics each velocity
component is an Ornstein-Uhlenbeck process; its Euler-Maruyama discretisation
has a closed-form variance recursion and, for a non-diagonal G_ij, the
discrete Lyapunov recursion R_{n+1} = (I + G dt) R_n (I + G dt)^T + C0 eps dt I.
Eq. frequency-model: with S_omega = 0 and fixed <omega> = Om the stationary law
is Gamma(1/C4, C4 Om) (Fokker-Planck of the square-root diffusion).
Eq. IECM: with one bin (IEM) psi - <psi> shrinks by exactly (1 - r) per step.
"""
import numpy as np
import pytest

from oracle import oracle as orc

NF = 22  # per-particle field vector of the oracle's SDE routine


def fields(n, **kw):
    F = np.zeros((n, NF))
    names = dict(U=0, V=1, Om=2, C0eps=3, G11=4, G12=5, G21=6, G22=7, G33=8, Fx=9, Fy=10,
                 Ux=11, Uy=12, Vx=13, Vy=14, lapU=15, lapV=16, Som=17, tm=18, cm=19)
    F[:, names["tm"]] = 1e300
    F[:, names["Om"]] = 1.0
    for k, v in kw.items():
        F[:, names[k]] = v
    return F


def state(n, **kw):
    s = {k: np.zeros(n) for k in ("u", "v", "w", "om", "psi")}
    s["om"][:] = 1.0
    for k, v in kw.items():
        s[k] = np.array(v, dtype=float) * np.ones(n)
    return s


def run(params, dt, F, s, nsteps, rng):
    n = F.shape[0]
    for _ in range(nsteps):
        z = rng.standard_normal((n, 8))
        s = orc.sde(params, dt, F, z, s)
    return s


def test_ou_discrete_variance_recursion():
    p = orc.default_params(nu=0.0)
    a, c, dt, n = 2.0, 0.5, 0.05, 100000
    F = fields(n, G11=-a, G22=-a, G33=-a, C0eps=c)
    s = state(n)
    rng = np.random.default_rng(1)
    var, q = 0.0, (1 - a * dt) ** 2
    for k in (1, 1, 3, 55):
        s = run(p, dt, F, s, k, rng)
        for _ in range(k):
            var = q * var + c * dt
        for comp in ("u", "v", "w"):
            se = var * np.sqrt(2.0 / n)
            assert abs(s[comp].var() - var) < 5 * se, (comp, s[comp].var(), var)
    vstar = c * dt / (1 - q)
    assert abs(var - vstar) / vstar < 1e-4
    # the discrete fixed point differs from the continuous c/(2a) by much more than the noise
    assert abs(vstar - c / (2 * a)) > 8 * vstar * np.sqrt(2.0 / n)


def test_ou_continuous_limit():
    p = orc.default_params(nu=0.0)
    a, c, dt, n = 2.0, 0.5, 0.002, 20000
    F = fields(n, G11=-a, G22=-a, G33=-a, C0eps=c)
    s = run(p, dt, F, state(n), 2000, np.random.default_rng(2))
    target = c / (2 * a)
    for comp in ("u", "v", "w"):
        assert abs(s[comp].var() - target) < 5 * target * np.sqrt(2.0 / n) + 2 * a * dt * target


def test_anisotropic_lyapunov_recursion():
    p = orc.default_params(nu=0.0)
    G = np.array([[-1.3, 0.7, 0.0], [-0.4, -0.9, 0.0], [0.0, 0.0, -1.6]])
    c, dt, n = 0.3, 0.04, 200000
    Um = np.array([0.3, -0.1, 0.0])
    F = fields(n, U=Um[0], V=Um[1], G11=G[0, 0], G12=G[0, 1], G21=G[1, 0], G22=G[1, 1],
               G33=G[2, 2], C0eps=c)
    rng = np.random.default_rng(3)
    m = np.array([0.2, 0.1, -0.05])
    Lc = np.array([[0.3, 0, 0], [0.1, 0.2, 0], [0.05, -0.02, 0.25]])
    U0 = Um + m + rng.standard_normal((n, 3)) @ Lc.T
    s = dict(u=U0[:, 0].copy(), v=U0[:, 1].copy(), w=U0[:, 2].copy(), om=np.ones(n), psi=np.zeros(n))
    R = Lc @ Lc.T
    A = np.eye(3) + G * dt
    At = np.eye(3) + G.T * dt
    Rt, mt = R.copy(), m.copy()
    for _ in range(12):
        s = orc.sde(p, dt, F, rng.standard_normal((n, 8)), s)
        m = A @ m
        R = A @ R @ A.T + c * dt * np.eye(3)
        mt = At @ mt
        Rt = At @ Rt @ At.T + c * dt * np.eye(3)
    U = np.stack([s["u"], s["v"], s["w"]], axis=1)
    emp_m = U.mean(axis=0) - Um
    emp_R = np.cov(U.T, bias=True)
    se_m = np.sqrt(np.diag(R) / n)
    assert np.all(np.abs(emp_m - m) < 5 * se_m), (emp_m, m)
    se_R = np.sqrt((np.outer(np.diag(R), np.diag(R)) + R ** 2) / n)
    assert np.all(np.abs(emp_R - R) < 5 * se_R), (emp_R, R)
    # the transposed drift matrix is rejected by the same statistics
    assert np.any(np.abs(emp_R - Rt) > 10 * se_R) or np.any(np.abs(emp_m - mt) > 10 * se_m)


def test_frequency_stationary_gamma():
    p = orc.default_params()
    C3, C4 = p["C3"], p["C4"]
    Om, dt, n = 1.0, 0.002, 20000
    F = fields(n, Om=Om, Som=0.0)
    s = run(p, dt, F, state(n, om=Om), 1500, np.random.default_rng(4))
    om = s["om"]
    shape, scale = 1 / C4, C4 * Om
    mean, var = shape * scale, shape * scale ** 2
    assert abs(om.mean() - mean) < 5 * np.sqrt(var / n) + C3 * Om * dt * mean
    mu4 = 3 * shape * (shape + 2) * scale ** 4
    se_var = np.sqrt((mu4 - var ** 2) / n)
    assert abs(om.var() - var) < 5 * se_var + 2 * C3 * Om * dt * var
    skew = np.mean((om - om.mean()) ** 3) / om.std() ** 3
    assert abs(skew - 2 / np.sqrt(shape)) < 0.2


def test_frequency_drift_terms():
    p = orc.default_params()
    C3 = p["C3"]
    Om, Som, dt, n, om0 = 1.0, 0.7, 0.01, 50000, 2.0
    F = fields(n, Om=Om, Som=Som)
    s = run(p, dt, F, state(n, om=om0), 1, np.random.default_rng(5))
    want = om0 - C3 * Om * (om0 - Om) * dt - Som * Om * om0 * dt
    sd = np.sqrt(2 * C3 * p["C4"] * Om ** 2 * om0 * dt)
    assert abs(s["om"].mean() - want) < 5 * sd / np.sqrt(n)
    assert abs(s["om"].var() - sd ** 2) < 5 * sd ** 2 * np.sqrt(2 / n)


@pytest.mark.parametrize("mix_exp", [0, 1])
def test_iem_exact_decay(mix_exp):
    p = orc.default_params(mix_exp=mix_exp)
    n, dt, tm = 1000, 0.01, 0.05
    rng = np.random.default_rng(6)
    psi = rng.random(n)
    m = psi.mean()
    F = fields(n, tm=tm, cm=m)
    s = state(n)
    s["psi"] = psi.copy()
    out = orc.sde(p, dt, F, rng.standard_normal((n, 8)), s)
    r = (1 - np.exp(-dt / tm)) if mix_exp else dt / tm
    assert np.max(np.abs((out["psi"] - m) - (1 - r) * (psi - m))) < 1e-15
    assert abs(out["psi"].mean() - m) < 1e-15


def test_iecm_variance_between_iem_rate_and_none():
    p = orc.default_params(nb1=2, nb2=2, nb3=2)
    n, dt, tm = 4000, 0.02, 0.05
    rng = np.random.default_rng(8)
    u, v, w = rng.standard_normal((3, n))
    psi = 1 / (1 + np.exp(-2 * u)) + 0.1 * rng.random(n)  # correlated with U
    ids = rng.permutation(n).astype(np.uint32)
    b = orc.bins(p, u, v, w, ids)
    cm = np.array([psi[b == k].mean() for k in range(8)])
    F = fields(n, tm=tm)
    F[:, 19] = cm[b]
    s = state(n)
    s["psi"] = psi.copy()
    out = orc.sde(p, dt, F, np.zeros((n, 8)), s)
    r = dt / tm
    v0, v1 = psi.var(), out["psi"].var()
    assert (1 - r) ** 2 * v0 < v1 < v0
    assert abs(out["psi"].sum() - psi.sum()) < 1e-10
