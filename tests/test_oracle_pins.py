"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, an exact identity of the model, a finite-difference gradient of the
Hamiltonian as printed (Eq. a2), a printed number (tests/golden), or a
statistical law (OU variance, free-draining centre-of-mass diffusion,
equipartition).  A plausible slip in the oracle -- a dropped term, a wrong
sign or index, a transposed operand -- fails at least one of them.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from golden_values import PAPER
from inputs import jittered_rods
from oracle import oracle as O

NU, TSTAR = PAPER["nu"], PAPER["Tstar"]


def closed_zeta(M, nu=NU):
    th = np.arange(M) * np.pi / M
    return 4.0 * nu * (1.0 - np.cos(th)) ** 2


# ---------------------------------------------------------------- transforms

@pytest.mark.parametrize("M", [2, 5, 64, 256])
def test_phi_orthonormal(M):
    """Eq. c2: the mode transform is orthogonal (with phi_{n,0} = 1/sqrt(N+1))."""
    phi = O.Model(M).tables()["phi"]
    assert np.abs(phi.T @ phi - np.eye(M)).max() < 1e-13
    assert np.abs(phi @ phi.T - np.eye(M)).max() < 1e-13


@pytest.mark.parametrize("M", [5, 64])
def test_transforms_are_inverse_pair(M):
    """Eq. c1: beads -> modes -> beads is the identity."""
    m = O.Model(M)
    r = jittered_rods(1, M, seed=3)[0]
    assert np.abs(m.modes_to_beads(m.beads_to_modes(r)) - r).max() < 1e-11


@pytest.mark.parametrize("M", [7, 64, 255])
def test_hamiltonian_in_mode_form(M):
    """Eqs. c6, c9, c10: H' = 1/2 sum zeta^l_p |R_p|^2 - L_c + N/2, where H' is
    the bead-form Hamiltonian of Eq. a2 (scaled by lambda d^2)."""
    m = O.Model(M)
    t = m.tables()
    for seed in range(3):
        r = jittered_rods(1, M, jitter=0.8, seed=seed)[0]
        R = r @ t["phi"]                                    # R_p = sum_n r_n phi_{n,p}
        Lc = np.linalg.norm(np.diff(r, axis=1), axis=0).sum()
        mode_form = 0.5 * np.sum(t["zl"][None, :] * R * R) - Lc + 0.5 * (M - 1)
        assert m.energy(r) == pytest.approx(mode_form, rel=1e-11, abs=1e-9)


@pytest.mark.parametrize("M", [6, 64])
def test_chi_orthogonality(M):
    """Eq. e6: sum_n chi_{n,p} chi_{n,q} = [2 sin(p pi / 2(N+1))]^2 delta_pq."""
    chi = O.Model(M).tables()["chi"]
    s = (2.0 * np.sin(np.arange(M) * np.pi / (2 * M))) ** 2
    assert np.abs(chi.T @ chi - np.diag(s)).max() < 1e-13


@pytest.mark.parametrize("M", [4, 64, 512])
def test_zeta_closed_form(M):
    """Eq. e9 equals 4 nu (1 - cos theta_p)^2 (algebra of Eqs. c9, e9)."""
    z = O.Model(M).tables()["zeta"]
    ref = closed_zeta(M)
    assert np.allclose(z, ref, rtol=1e-9, atol=1e-15)


# ---------------------------------------------------------------- forces

def _fd_grad_modes(m, R, eps=1e-5):
    """Central finite differences of H'(phi R) with respect to every R_p^alpha."""
    g = np.zeros_like(R)
    for a in range(3):
        for p in range(m.M):
            Rp = R.copy(); Rp[a, p] += eps
            Rm = R.copy(); Rm[a, p] -= eps
            g[a, p] = (m.energy(m.modes_to_beads(Rp)) - m.energy(m.modes_to_beads(Rm))) / (2 * eps)
    return g


@pytest.mark.parametrize("M", [5, 16])
def test_delta_H_is_gradient_remainder(M):
    """Eq. e10 is exact: -dH'/dR_p = -zeta_p R_p + DeltaH_p (DeltaH from Eq. e11)."""
    m = O.Model(M)
    t = m.tables()
    for seed in range(2):
        r = jittered_rods(1, M, jitter=0.6, seed=10 + seed)[0]
        R = m.beads_to_modes(r)
        grad = _fd_grad_modes(m, R)
        rhs = -t["zeta"][None, :] * R + m.delta_H(r)
        assert np.abs(-grad - rhs).max() < 2e-7
        assert np.abs(m.delta_H(r)[:, 0]).max() < 1e-12     # chi_{n,0} = 0


@pytest.mark.parametrize("M", [5, 16])
def test_full_force_is_gradient(M):
    """Eq. b3: the Euler force is -dH'/dr_n of Eq. a2 (finite differences)."""
    m = O.Model(M)
    r = jittered_rods(1, M, jitter=0.6, seed=21)[0]
    F = m.full_force(r)
    eps = 1e-5
    for a in range(3):
        for n in range(M):
            rp = r.copy(); rp[a, n] += eps
            rm = r.copy(); rm[a, n] -= eps
            g = (m.energy(rp) - m.energy(rm)) / (2 * eps)
            assert F[a, n] == pytest.approx(-g, abs=2e-7)
    assert np.abs(F.sum(axis=1)).max() < 1e-12            # internal forces sum to zero


# ---------------------------------------------------------------- update coefficients

def test_h_limits():
    """Eq. f3 (h -> dtau for slow modes) and Eq. f4 (h -> e^{-zeta dtau}/(zeta^l - zeta)
    for modes with zeta^l dtau large)."""
    M = 512
    small = O.Model(M, dtau=0.01).tables()
    assert small["h"][1] == pytest.approx(0.01, rel=1e-6)
    big = O.Model(M, dtau=100.0).tables()
    p = np.arange(200, M)
    ref = np.exp(-big["zeta"][p] * 100.0) / (big["zl"][p] - big["zeta"][p])
    assert np.allclose(big["h"][p], ref, rtol=1e-12)


@pytest.mark.parametrize("M,dtau", [(64, 10.0), (256, 100.0)])
def test_h_is_quadrature_of_d5_under_f1(M, dtau):
    """Eq. f2 = the integral of Eq. d5 with DeltaH(t') = DeltaH e^{-zeta^l t'} (Eq. f1),
    evaluated by adaptive quadrature."""
    t = O.Model(M, dtau=dtau).tables()
    for p in (1, 2, 7, M // 2, M - 1):
        z, zl = t["zeta"][p], t["zl"][p]
        val, _ = integrate.quad(lambda s: math.exp(z * (s - dtau)) * math.exp(-zl * s), 0.0, dtau,
                                epsabs=0, epsrel=1e-12, limit=200)
        assert t["h"][p] == pytest.approx(val, rel=1e-8)


def test_ou_decay_closed_form():
    """Eq. d3 without coupling or noise: R_p(k dtau) = exp(-zeta_p k dtau) R_p(0)."""
    M, dtau, k = 32, 3.0, 7
    m = O.Model(M, Tstar=0.0, dtau=dtau)
    R0 = m.beads_to_modes(jittered_rods(1, M, seed=4)[0])
    R = m.run_modes(R0[None], seed=1, jobs=[0], step0=0, nsteps=k, coupling=False)[0]
    ref = np.exp(-closed_zeta(M) * k * dtau)[None, :] * R0
    assert np.abs(R - ref).max() < 1e-10 * np.abs(R0).max()


def test_ou_variance_any_step():
    """Eqs. d3, d6 are exact for any step when DeltaH = 0 (the OU process):
    from R = 0, Var R_p after k steps = T* (1 - e^{-2 zeta_p k dtau}) / zeta_p,
    and Var R_0 = 2 T* k dtau; modes stay uncorrelated."""
    M, dtau, k, C = 8, 40.0, 3, 4000
    m = O.Model(M, dtau=dtau)
    R = m.run_modes(np.zeros((C, 3, M)), seed=7, jobs=np.arange(C), step0=0, nsteps=k,
                    coupling=False)
    z = closed_zeta(M)
    var = R.var(axis=(0, 1))
    ref = np.empty(M)
    ref[0] = 2 * TSTAR * k * dtau
    ref[1:] = TSTAR * (1 - np.exp(-2 * z[1:] * k * dtau)) / z[1:]
    tol = 4.5 * math.sqrt(2.0 / (3 * C))
    assert np.all(np.abs(var / ref - 1) < tol), var / ref
    X = R.transpose(0, 1, 2).reshape(-1, M) / np.sqrt(ref)[None, :]
    corr = np.corrcoef(X.T) - np.eye(M)
    assert np.abs(corr).max() < 4.5 / math.sqrt(3 * C)


# ---------------------------------------------------------------- dynamics laws

def test_com_free_draining_diffusion():
    """Sec. 7B: the centre of mass diffuses with D = kT/((N+1) xi), i.e. T*/(N+1)
    in scaled units, exactly for the coupled dynamics and any step."""
    M, dtau, k, C = 16, 5.0, 6, 3000
    m = O.Model(M, dtau=dtau)
    R0 = np.stack([m.equilibrium_start(3, j) for j in range(C)])
    R = m.run_modes(R0, seed=3, jobs=np.arange(C), step0=0, nsteps=k)
    dcm = (R[:, :, 0] - R0[:, :, 0]) / math.sqrt(M)           # r_cm = R_0 / sqrt(N+1)
    msd = np.mean(np.sum(dcm ** 2, axis=1))
    ref = 6 * TSTAR * k * dtau / M
    assert msd == pytest.approx(ref, rel=4.5 * math.sqrt(2.0 / (3 * C)))


def test_euler_com_free_draining_diffusion():
    """Same law for the bead-position Euler scheme (Eqs. b3-b5)."""
    M, dtau, k, C = 12, 0.05, 40, 2000
    m = O.Model(M, dtau=dtau)
    r0 = jittered_rods(C, M, seed=5)
    r = m.run_euler(r0, seed=5, jobs=np.arange(C), step0=0, nsteps=k)
    dcm = r.mean(axis=2) - r0.mean(axis=2)
    msd = np.mean(np.sum(dcm ** 2, axis=1))
    assert msd == pytest.approx(6 * TSTAR * k * dtau / M, rel=4.5 * math.sqrt(2.0 / (3 * C)))


def test_generalised_equipartition_fast_modes():
    """Boltzmann weight exp(-H'/T*) implies <R_p^a dH'/dR_p^a> = T* for every p, a;
    with dH'/dR_p = zeta_p R_p - DeltaH_p (Eq. e10).  Checked on modes that
    equilibrate within the run, at a small step."""
    M, dtau, C, nsteps, every = 16, 0.05, 32, 3000, 20
    m = O.Model(M, dtau=dtau)
    t = m.tables()
    R = np.stack([m.equilibrium_start(11, j) for j in range(C)])
    R = m.run_modes(R, seed=11, jobs=np.arange(C), step0=0, nsteps=400)
    acc, cnt = np.zeros(M), 0
    step = 400
    for _ in range(nsteps // every):
        R = m.run_modes(R, seed=11, jobs=np.arange(C), step0=step, nsteps=every)
        step += every
        for c in range(C):
            dH = m.delta_H(m.modes_to_beads(R[c]))
            acc += np.mean(R[c] * (t["zeta"][None, :] * R[c] - dH), axis=0)
            cnt += 1
    ratio = (acc / cnt)[4:] / TSTAR
    assert abs(ratio.mean() - 1) < 0.03, ratio
    assert np.all(np.abs(ratio - 1) < 0.12), ratio


def test_euler_stability_limit():
    """Sec. 3A: the default Euler scheme is safe at dtau = 0.1 and unstable at
    dtau ~ 0.3 (noise switched off, perturbed ground state)."""
    M = 64
    for dtau, stable in ((PAPER["euler_dtau_safe"], True), (PAPER["euler_dtau_unstable"], False)):
        m = O.Model(M, Tstar=0.0, dtau=dtau)
        l0 = m.ground_bonds()
        r = np.zeros((3, M))
        r[0, 1:] = np.cumsum(l0)
        e_ground = m.energy(r)
        r += 1e-3 * jittered_rods(1, M, spacing=0.0, jitter=1.0, seed=8)[0]
        e0 = m.energy(r) - e_ground
        r = m.run_euler(r[None], seed=0, jobs=[0], step0=0, nsteps=3000)[0]
        e = m.energy(r) - e_ground
        if stable:
            assert np.isfinite(e) and e < 1e-3 * e0      # the perturbation relaxes
        else:
            assert not np.isfinite(e) or e > 1e3 * e0    # the perturbation grows
    # at the printed "unstable" value the linear stability bound 2/max zeta^l is crossed
    zl = O.Model(M).tables()["zl"]
    assert 2.0 / zl.max() < PAPER["euler_dtau_unstable"] < 2.0 / zl.max() + 0.01


def test_euler_and_mode_paths_converge():
    """Eq. e10 is an exact rewrite of Eq. b3, so with the same Brownian path the
    mode integrator and the Euler scheme converge to the same trajectory as
    dtau -> 0; their gap shrinks linearly (both are first order here)."""
    M, T = 16, 0.064
    levels = [8e-3, 4e-3, 2e-3, 1e-3]
    nfine = int(round(T / levels[-1]))
    rng = np.random.default_rng(123)
    zf = rng.normal(size=(nfine, 3, M))          # Brownian increments at the finest level
    r0 = jittered_rods(1, M, jitter=0.2, seed=9)[0]
    gaps = []
    for dt in levels:
        k = int(round(dt / levels[-1]))
        z = zf.reshape(nfine // k, k, 3, M).sum(axis=1) / math.sqrt(k)
        m = O.Model(M, dtau=dt)
        re = r0.copy()
        R = m.beads_to_modes(r0)
        for s in range(z.shape[0]):
            re = m.euler_step_z(re, z[s])
            R = m.mode_step_z(R, z[s])
        gaps.append(np.abs(m.modes_to_beads(R) - re).max())
    gaps = np.array(gaps)
    assert gaps[-1] < 2e-3
    rates = gaps[1:] / gaps[:-1]
    assert np.all((rates > 0.35) & (rates < 0.7)), gaps


def test_shear_converges_to_exact_linear_flow():
    """Eq. btum in mode space (coupling and noise off): x_p' = -zeta x_p + g y_p,
    y_p' = -zeta y_p has the exact solution x(t) = e^{-zeta t} (x0 + g y0 t).
    The centre of mass is advected exactly: x_cm += g y_cm dtau."""
    M, g, T = 16, 0.05, 4.0
    r0 = jittered_rods(1, M, seed=12)[0]
    z = closed_zeta(M)
    for dt in (0.01,):
        m = O.Model(M, Tstar=0.0, dtau=dt)
        R0 = m.beads_to_modes(r0)
        R = R0.copy()
        for _ in range(int(round(T / dt))):
            R = m.mode_step_z(R, np.zeros((3, M)), shear=g, coupling=False)
        ref_x = np.exp(-z * T) * (R0[0] + g * R0[1] * T)
        assert np.abs(R[0] - ref_x).max() < 2e-3 * np.abs(R0).max()
        assert R[0, 0] == pytest.approx(R0[0, 0] + g * R0[1, 0] * T, rel=1e-12, abs=1e-12)


# ---------------------------------------------------------------- starts and statics

@pytest.mark.parametrize("M", [64, 512])
def test_ground_state_rod(M):
    """Straight-rod minimum of Eq. a2: zero gradient, bulk bond b = 1/(1-2 nu)
    (Eq. a3; printed as approx 3.3 in Sec. 2A)."""
    m = O.Model(M)
    l0 = m.ground_bonds()
    r = np.zeros((3, M))
    r[0, 1:] = np.cumsum(l0)
    assert np.abs(m.full_force(r)).max() < 1e-12
    assert l0[M // 2] == pytest.approx(1 / (1 - 2 * NU), rel=1e-9)
    assert round(l0[M // 2], 1) == PAPER["b_approx"]


def test_equilibrium_start_statistics():
    """The starting sampler: centre of mass at the origin, bulk bonds ~ b, and the
    tangent correlation decays as exp(-s/l_p) with l_p = b^2 nu / T* bonds
    (Eq. a3, printed as approx 114 bp), within 5%."""
    M, C = 256, 300
    m = O.Model(M)
    b = 1 / (1 - 2 * NU)
    lp = b * b * NU / TSTAR
    assert round(lp) == PAPER["lp_bp_approx"]
    corr = np.zeros(41)
    lens = []
    for j in range(C):
        R = m.equilibrium_start(2, j)
        assert np.abs(R[:, 0]).max() == 0.0
        r = m.modes_to_beads(R)
        assert np.abs(r.mean(axis=1)).max() < 1e-10
        u = np.diff(r, axis=1)
        L = np.linalg.norm(u, axis=0)
        lens.append(L[20:-20])
        t = u / L
        for s in range(41):
            corr[s] += np.mean(np.sum(t[:, 20:M - 61] * t[:, 20 + s:M - 61 + s], axis=0))
    corr /= C
    assert np.mean(np.concatenate(lens)) == pytest.approx(b, rel=0.01)
    s = np.arange(41)
    assert np.all(np.abs(corr / np.exp(-s / lp) - 1) < 0.05)


# ---------------------------------------------------------------- random numbers

def test_uniforms_exact_and_open():
    """u = (floor(x/2^9) + 1/2)/2^23 lies strictly inside (0,1) and is exact in FP32."""
    for x in (0, 1, 511, 512, 2**31, 2**32 - 1):
        u = O.u01(x)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u


def test_philox_is_keyed_and_counter_sensitive():
    a = O.philox4x32_10([0, 0, 0, 0], [0, 0])
    assert not np.array_equal(a, O.philox4x32_10([1, 0, 0, 0], [0, 0]))
    assert not np.array_equal(a, O.philox4x32_10([0, 0, 0, 0], [1, 0]))
    assert not np.array_equal(a, O.philox4x32_10([0, 0, 0, 1], [0, 0]))


def test_bead_normals_statistics():
    """The noise of Eq. b5: iid N(0,1) over beads, axes, steps and chains."""
    M = 256
    z = np.concatenate([O.bead_normals(1, j, s, 0, M).ravel()
                        for j in range(4) for s in range(40)])
    assert abs(z.mean()) < 4.5 / math.sqrt(z.size)
    assert abs(z.var() - 1) < 4.5 * math.sqrt(2.0 / z.size)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    zz = np.stack([O.bead_normals(1, 0, s, 0, M) for s in range(200)])   # [s][3][M]
    X = zz.transpose(1, 0, 2).reshape(3, -1)
    c = np.corrcoef(X)
    assert np.abs(c - np.eye(3)).max() < 4.5 / math.sqrt(X.shape[1])
    lag = np.corrcoef(zz[:-1].ravel(), zz[1:].ravel())[0, 1]
    assert abs(lag) < 4.5 / math.sqrt(zz[1:].size)


def test_bead_normals_use_every_box_muller_value_once():
    """Four normals per Philox call, each used by exactly one (bead, axis).

    Flattened in the order k = 3n + alpha, the normals of a step follow the
    calls' words: the two values of a Box-Muller pair share their radius, so
    z_{2i}^2 + z_{2i+1}^2 = -2 ln u(word 4c or 4c + 2) of call c exactly, and
    no two (bead, axis) slots hold the same value (a slot mapped twice, or a
    call index shifted by one, would repeat values or break the pairing)."""
    for M in (7, 64, 65, 256):
        z = O.bead_normals(3, 11, 5, 0, M)           # [3][M]
        k = z.T.ravel()                              # k = 3 n + alpha
        assert np.unique(k).size == k.size
        for c in range(len(k) // 4):
            w = O.philox4x32_10([5, 0, c, 0], [3, 11])
            for pair in range(2):
                r2 = k[4 * c + 2 * pair] ** 2 + k[4 * c + 2 * pair + 1] ** 2
                assert r2 == pytest.approx(-2.0 * math.log(O.u01(int(w[2 * pair]))), rel=1e-12)
        # lag correlation along k over many steps: the pairs are uncorrelated
        zz = np.stack([O.bead_normals(3, 11, s, 0, M).T.ravel() for s in range(400)])
        for lag in (1, 2, 3, 4):
            r = np.corrcoef(zz[:, :-lag].ravel(), zz[:, lag:].ravel())[0, 1]
            assert abs(r) < 4.5 / math.sqrt(zz[:, lag:].size)


# ---------------------------------------------------------------- Monte Carlo (Sec. 5A)

def _two_bond_quadrature(T, nu, n=1500):
    """<|L|^2>, <|u_1|^2>, <|r_1 - r_cm|^2> of a 3-bead chain under exp(-H'/T*),
    by direct quadrature over the bond lengths l1, l2 and the bond angle.

    H' = 1/2 (l1-1)^2 + 1/2 (l2-1)^2 - nu l1 l2 c (Eq. a2 with N = 2), volume
    element l1^2 l2^2 dl1 dl2 dc; the c-integral is done in closed form:
    int e^{kc} dc = 2 sinh(k)/k and <c> = coth(k) - 1/k, k = nu l1 l2 / T*.
    L = u1 + u2 and r_1 - r_cm = (u1 - u2)/3."""
    l = np.linspace(1e-4, 3.0 + 14.0 * math.sqrt(T), n)
    L1, L2 = np.meshgrid(l, l, indexing="ij")
    k = nu * L1 * L2 / T
    logw = (2 * np.log(L1) + 2 * np.log(L2) - (0.5 * (L1 - 1) ** 2 + 0.5 * (L2 - 1) ** 2) / T
            + k - np.log(k) + np.log1p(-np.exp(-2 * k)))
    w = np.exp(logw - logw.max())
    c = 1.0 / np.tanh(k) - 1.0 / k
    Z = w.sum()
    return np.array([(w * (L1 ** 2 + L2 ** 2 + 2 * L1 * L2 * c)).sum() / Z,
                     (w * L1 ** 2).sum() / Z,
                     (w * (L1 ** 2 + L2 ** 2 - 2 * L1 * L2 * c)).sum() / Z / 9.0])


@pytest.mark.parametrize("T,nu", [(TSTAR, NU), (0.3, 0.2)])
def test_mc_samples_boltzmann_two_bonds(T, nu):
    """The mode-space Metropolis sampler (Sec. 5A) on a 3-bead chain reproduces
    averages of the Boltzmann weight of Eq. a2 computed by quadrature in bond
    coordinates, which share nothing with the mode machinery (chi, phi, steps)."""
    m = O.Model(3, Tstar=T, nu=nu)
    C = 32
    r = np.zeros((3, 3))
    r[0] = [-1.5, 0.0, 1.5]
    R = np.repeat(m.beads_to_modes(r)[None], C, axis=0)
    step, R = m.mc_tuned_steps(R, 7, np.arange(C))
    R, acc, obs = m.run_mc(R, 7, np.arange(C), 0, 20000, step, sample=True)
    per = obs[:, :3] / obs[:, 3:4]
    mean, se = per.mean(axis=0), per.std(axis=0, ddof=1) / math.sqrt(C)
    q = _two_bond_quadrature(T, nu)
    assert np.all(np.abs(mean - q) < 4.5 * se + 1e-12), (mean, q, se)
    assert np.all(np.abs(mean / q - 1) < 0.01), (mean, q)
    rate = acc[:, 1:].sum() / (3.0 * 20000 * C * 2)
    assert 0.25 < rate < 0.55


def test_mc_generalised_equipartition():
    """MC samples obey <R_p^a dH'/dR_p^a> = T* for every internal mode, the
    identity of any Boltzmann sampler, with dH'/dR_p = zeta_p R_p - DeltaH_p
    (Eq. e10) evaluated independently of the sampler's energy routine."""
    M, C = 12, 32
    m = O.Model(M)
    t = m.tables()
    R = np.stack([m.equilibrium_start(3, j) for j in range(C)])
    step, R = m.mc_tuned_steps(R, 3, np.arange(C))
    acc, cnt = np.zeros(M), 0
    for k in range(100):
        R, _, _ = m.run_mc(R, 3, np.arange(C), 100 * k, 100, step)
        for c in range(C):
            dH = m.delta_H(m.modes_to_beads(R[c]))
            acc += np.mean(R[c] * (t["zeta"][None, :] * R[c] - dH), axis=0)
            cnt += 1
    ratio = (acc / cnt)[1:] / TSTAR
    assert abs(ratio.mean() - 1) < 0.04, ratio
    # p = 1 relaxes slowest and its estimator has the largest variance: mean only
    assert np.all(np.abs(ratio[1:] - 1) < 0.12), ratio


@pytest.mark.parametrize("M", [5, 64])
def test_bond_path_equals_bead_path(M):
    """Eq. e11 two ways: the oracle's DeltaH = chi^T v (bond path) equals the
    bead-space stencil f_n = v_n - v_{n+1} (v_0 = v_{N+1} = 0) projected with
    phi^T (bead path), since sum_n phi_{n,p} (v_n - v_{n+1}) = sum_n chi_{n,p} v_n."""
    m = O.Model(M)
    phi = m.tables()["phi"]
    r = jittered_rods(1, M, seed=21)[0]
    u = np.diff(r, axis=1)
    s = 1.0 / np.linalg.norm(u, axis=0) - (1.0 - 2.0 * NU)
    v = np.zeros((3, M + 1))
    v[:, 1:M] = u * s
    f = v[:, :M] - v[:, 1:]
    bead_path = f @ phi
    assert np.abs(m.delta_H(r) - bead_path).max() < 1e-12 * max(1.0, np.abs(bead_path).max())


def test_stored_monte_carlo_reference_is_the_oracles():
    """tests/golden/mc_reference.txt (the Monte Carlo benchmark the step-size
    scans compare with) holds what the oracle's sampler gives: the 64-bead row
    is recomputed here with the writer's settings and must agree to the stored
    digits (the sampler is deterministic: Philox-keyed proposals)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "mc_reference.txt")
    row = next(line.split() for line in open(path) if line.split() and line.split()[0] == "64")
    stored = np.array([float(x) for x in row[1:7]])
    M, Cm = 64, 64
    m = O.Model(M, dtau=10.0)
    R = np.stack([m.equilibrium_start(9, j) for j in range(Cm)])
    step, R = m.mc_tuned_steps(R, 9, np.arange(Cm))
    R, _, _ = m.run_mc(R, 9, np.arange(Cm), 0, 4000, step)
    R, _, obs = m.run_mc(R, 9, np.arange(Cm), 4000, 20000, step, sample=True)
    per = obs[:, :3] / obs[:, 3:4]
    mine = np.concatenate([per.mean(axis=0), per.std(axis=0, ddof=1) / math.sqrt(Cm)])
    assert np.allclose(mine, stored, rtol=1e-9, atol=0)


# ---------------------------------------------------------------- mode-keyed noise (Eq. c4)

def test_mode_normals_statistics_and_key():
    """The mode-keyed noise: iid N(0,1) over modes, axes, steps and chains, and a
    stream of its own (Philox tag 2), so it shares no value with the bead noise
    of the same key and step."""
    M = 256
    Z = np.concatenate([O.mode_normals(1, j, s, M).ravel() for j in range(4) for s in range(40)])
    assert abs(Z.mean()) < 4.5 / math.sqrt(Z.size)
    assert abs(Z.var() - 1) < 4.5 * math.sqrt(2.0 / Z.size)
    assert stats.kstest(Z, "norm").pvalue > 1e-4
    assert np.array_equal(O.mode_normals(3, 5, 7, 64), O.bead_normals(3, 5, 7, 2, 64))
    assert not np.intersect1d(O.mode_normals(3, 5, 7, 64).ravel(), O.bead_normals(3, 5, 7, 0, 64).ravel()).size


def test_mode_keyed_step_is_the_bead_step_with_projected_noise():
    """Eq. c4 makes the bead noise enter only through Z = phi^T z.  A step with
    the mode noise Z given equals the bead-noise step with z = phi Z (phi
    orthonormal, so phi^T phi Z = Z): the mode-keyed variant integrates the same
    dynamics, with shear and coupling, on the same trajectory."""
    for M in (5, 64):
        m = O.Model(M, dtau=10.0)
        R0 = m.equilibrium_start(2, 0)
        Z = O.mode_normals(2, 0, 0, M)
        z = m.modes_to_beads(Z)                 # phi Z, per axis (Eq. c1)
        for shear, coupling in ((0.0, True), (0.3, True), (0.0, False)):
            a = m.mode_step_Zm(R0, Z, shear=shear, coupling=coupling)
            b = m.mode_step_z(R0, z, shear=shear, coupling=coupling)
            assert np.abs(a - b).max() < 1e-12 * (1 + np.abs(b).max()), (M, shear, coupling)


def test_mode_keyed_ou_variance_and_com_diffusion():
    """With mode-keyed noise the OU law of Eqs. d3, d6 (DeltaH = 0) holds for
    any step, and the centre of mass diffuses freely with D = T*/(N+1) (Sec. 7B),
    as with bead noise."""
    M, dtau, k, C = 8, 40.0, 3, 4000
    m = O.Model(M, dtau=dtau)
    R = m.run_modes(np.zeros((C, 3, M)), seed=7, jobs=np.arange(C), step0=0, nsteps=k, coupling=False,
                    mode_noise=True)
    z = closed_zeta(M)
    ref = np.empty(M)
    ref[0] = 2 * TSTAR * k * dtau
    ref[1:] = TSTAR * (1 - np.exp(-2 * z[1:] * k * dtau)) / z[1:]
    var = R.var(axis=(0, 1))
    assert np.all(np.abs(var / ref - 1) < 4.5 * math.sqrt(2.0 / (3 * C))), var / ref
    M, dtau, k, C = 16, 5.0, 6, 3000
    m = O.Model(M, dtau=dtau)
    R0 = np.stack([m.equilibrium_start(3, j) for j in range(C)])
    R = m.run_modes(R0, seed=3, jobs=np.arange(C), step0=0, nsteps=k, mode_noise=True)
    dcm = (R[:, :, 0] - R0[:, :, 0]) / math.sqrt(M)
    msd = np.mean(np.sum(dcm ** 2, axis=1))
    assert msd == pytest.approx(6 * TSTAR * k * dtau / M, rel=4.5 * math.sqrt(2.0 / (3 * C)))
