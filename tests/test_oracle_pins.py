"""Pins of the FP64 CPU oracle against facts that do not come from the oracle.

Each test names what fixes the expected value: published known-answer vectors,
closed forms, exact invariants of the Wilson action and of Haar measure, the
strong- and weak-coupling limits, or brute force on a single link.  A plausible
mistake anywhere in the oracle (a dropped staple term, a wrong sign or index in
the SU(2) embedding, a transposed product, a wrong action normalisation) fails
at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cplx(U):
    return oracle.as_complex(U)


def su3_defects(U):
    M = cplx(U).reshape(-1, 3, 3)
    eye = np.eye(3)
    unit = np.abs(np.einsum("nki,nkj->nij", M.conj(), M) - eye).max()
    det = np.abs(np.linalg.det(M) - 1.0).max()
    return unit, det


# --------------------------------------------------------------------------
# Philox4x32-10 and the uniform maps
# --------------------------------------------------------------------------

def test_philox_known_answers():
    rows = 0
    with open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            w = [int(x, 16) for x in line.split()]
            assert oracle.philox4x32_10(w[0:4], w[4:6]) == w[6:10]
            rows += 1
    assert rows == 3


def test_philox_counter_sensitivity():
    # a bijection of the counter for fixed key: distinct counters, distinct blocks
    seen = set()
    for i in range(2000):
        seen.add(tuple(oracle.philox4x32_10([i, i % 7, 3, 0], [11, 0])))
    assert len(seen) == 2000
    # each key word matters
    a = oracle.philox4x32_10([1, 2, 3, 4], [5, 6])
    assert a != oracle.philox4x32_10([1, 2, 3, 4], [5, 7])
    assert a != oracle.philox4x32_10([1, 2, 3, 4], [4, 6])


def test_uniform_map_extremes_and_bins():
    # the 52-bit map is centred in its bin: the extremes are exactly 2^-53 and 1-2^-53
    assert oracle.u01_f64(0, 0) == 2.0 ** -53
    assert oracle.u01_f64(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    assert oracle.u01_f32(0) == 2.0 ** -24
    assert oracle.u01_f32(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    # the low 12 bits of the second word and the low 9 bits of the single word are dropped
    assert oracle.u01_f64(5, 0xABC) == oracle.u01_f64(5, 0)
    assert oracle.u01_f32(0x1FF) == oracle.u01_f32(0)
    # centred bins: u * 2^53 (resp. 2^24) is an odd integer, and exact in float32 for the f32 map
    rng = np.random.default_rng(3)
    for a, b in rng.integers(0, 2 ** 32, size=(200, 2)):
        u = oracle.u01_f64(int(a), int(b))
        m = u * 2.0 ** 53
        assert m == math.floor(m) and int(m) % 2 == 1 and 0.0 < u < 1.0
        v = oracle.u01_f32(int(a))
        assert float(np.float32(v)) == v and int(v * 2.0 ** 24) % 2 == 1


# --------------------------------------------------------------------------
# start configurations and the plaquette
# --------------------------------------------------------------------------

def test_cold_start_is_identity_and_plaquette_one():
    L = (4, 4, 4, 6)
    U = oracle.cold_start(L)
    M = cplx(U)
    assert np.array_equal(M, np.broadcast_to(np.eye(3), M.shape))
    assert oracle.plaquette(L, U) == 1.0


def test_odd_extent_rejected():
    with pytest.raises(ValueError):
        oracle.cold_start((4, 4, 4, 5))


def abelian_config(L, n0, n2):
    """U_1(x) = diag(e^{iB x0}, e^{-iB x0}, 1), U_3(x) = diag(e^{iC x2}, e^{-iC x2}, 1), others 1."""
    U = oracle.cold_start(L)
    B = 2 * math.pi * n0 / L[0]
    C = 2 * math.pi * n2 / L[2]
    x0 = np.arange(L[0])
    x2 = np.arange(L[2])
    ph1 = B * x0[None, None, None, :]
    ph3 = C * x2[None, :, None, None]
    for mu, ph in ((1, ph1), (3, ph3)):
        ph = np.broadcast_to(ph, (L[3], L[2], L[1], L[0]))
        U[..., mu, 0, 0, 0] = np.cos(ph)
        U[..., mu, 0, 0, 1] = np.sin(ph)
        U[..., mu, 1, 1, 0] = np.cos(ph)
        U[..., mu, 1, 1, 1] = -np.sin(ph)
    return U, B, C


def test_plaquette_closed_form_abelian_field():
    # constant field B in the (0,1) plane and C in the (2,3) plane; the other
    # four planes are flat: P = (4 + (2cos B + 1)/3 + (2cos C + 1)/3) / 6
    L = (6, 4, 8, 4)
    U, B, C = abelian_config(L, 1, 3)
    expect = (4.0 + (2 * math.cos(B) + 1) / 3 + (2 * math.cos(C) + 1) / 3) / 6.0
    assert abs(oracle.plaquette(L, U) - expect) < 1e-14


def test_hot_start_is_haar_su3():
    L = (8, 8, 8, 8)
    U = oracle.hot_start(L, 7)
    unit, det = su3_defects(U)
    assert unit < 1e-14 and det < 1e-14
    tr = np.trace(cplx(U).reshape(-1, 3, 3), axis1=1, axis2=2)
    n = tr.size
    # Haar SU(3): <Tr U> = 0, <|Tr U|^2> = 1, <|Tr U|^4> = 2, <(Tr U)^3> = 1
    # (the last is 0 on U(3): it pins the det = 1 completion of the third row)
    assert abs(tr.mean()) < 4 * math.sqrt(1.0 / n)
    assert abs((abs(tr) ** 2).mean() - 1.0) < 4 * math.sqrt(1.0 / n)
    assert abs((abs(tr) ** 4).mean() - 2.0) < 4 * math.sqrt(22.0 / n)
    assert abs((tr ** 3).mean() - 1.0) < 4 * math.sqrt(7.0 / n)
    # plaquette of a Haar configuration: 0 within its fluctuation 1/sqrt(18 * 6V)
    assert abs(oracle.plaquette(L, U)) < 4 / math.sqrt(18 * 6 * np.prod(L))


def test_plaquette_gauge_invariant():
    L = (4, 6, 4, 4)
    U = oracle.hot_start(L, 12)
    oracle.sweep(L, 5.7, 3, 0, 2, U)
    p0 = oracle.plaquette(L, U)
    oracle.gauge_transform(L, 99, U)
    p1 = oracle.plaquette(L, U)
    assert abs(p1 - p0) < 1e-13
    unit, det = su3_defects(U)
    assert unit < 1e-13 and det < 1e-13


def test_plaquette_translation_invariant():
    L = (4, 6, 4, 8)
    U = oracle.hot_start(L, 5)
    p0 = oracle.plaquette(L, U)
    for axis in range(4):  # lattice axis x_axis is array axis 3 - axis
        V = np.ascontiguousarray(np.roll(U, 1, axis=3 - axis))
        assert abs(oracle.plaquette(L, V) - p0) < 1e-13


# --------------------------------------------------------------------------
# the staple: brute force against the action
# --------------------------------------------------------------------------

def site_index(L, x):
    return x[0] + L[0] * (x[1] + L[1] * (x[2] + L[2] * x[3]))


@pytest.mark.parametrize("mu", [0, 1, 2, 3])
def test_staple_is_action_derivative(mu):
    # The Wilson action's dependence on one link is -(beta/3) Re Tr(U A): replacing
    # U_mu(x) by W changes sum_P (1/3) Re Tr U_P by (1/3) Re Tr((W - U) A).
    L = (4, 4, 6, 4)
    V = np.prod(L)
    U = oracle.hot_start(L, 21)
    W = oracle.hot_start(L, 22)
    rng = np.random.default_rng(mu)
    for _ in range(3):
        x = [int(rng.integers(0, L[i])) for i in range(4)]
        s = site_index(L, x)
        A = cplx(oracle.staple(L, U, s, mu))
        total0 = oracle.plaquette(L, U) * 6 * V
        U2 = U.copy()
        U2[x[3], x[2], x[1], x[0], mu] = W[x[3], x[2], x[1], x[0], mu]
        total1 = oracle.plaquette(L, U2) * 6 * V
        u = cplx(U[x[3], x[2], x[1], x[0], mu])
        w = cplx(W[x[3], x[2], x[1], x[0], mu])
        pred = np.real(np.trace((w - u) @ A)) / 3.0
        assert abs((total1 - total0) - pred) < 1e-11


def test_staple_translation_covariant():
    # shifting the configuration shifts the staple (checks the periodic wrap)
    L = (4, 6, 4, 4)
    U = oracle.hot_start(L, 8)
    for axis in range(4):
        Ush = np.ascontiguousarray(np.roll(U, 1, axis=3 - axis))
        for x in ([0, 0, 0, 0], [3, 5, 3, 3], [1, 2, 3, 0]):
            y = list(x)
            y[axis] = (y[axis] + 1) % L[axis]
            for mu in range(4):
                a = oracle.staple(L, U, site_index(L, x), mu)
                b = oracle.staple(L, Ush, site_index(L, y), mu)
                assert np.abs(a - b).max() < 1e-13


# --------------------------------------------------------------------------
# the update
# --------------------------------------------------------------------------

def test_updates_stay_in_su3():
    L = (4, 4, 4, 4)
    U = oracle.hot_start(L, 1)
    for t in range(3):
        for mu in range(4):
            for p in range(2):
                oracle.half_sweep(L, 5.7, 1, t, mu, p, U)
                unit, det = su3_defects(U)
                assert unit < 1e-13 and det < 1e-13


def test_half_sweep_touches_only_its_links():
    L = (4, 4, 4, 4)
    U = oracle.hot_start(L, 2)
    U0 = U.copy()
    oracle.half_sweep(L, 5.7, 4, 0, 2, 1, U)
    x = np.indices((L[3], L[2], L[1], L[0]))
    par = (x.sum(axis=0) % 2).astype(bool)
    changed = np.any(U != U0, axis=(5, 6, 7))
    assert not changed[..., [0, 1, 3]].any()
    assert not changed[~par, 2].any()
    assert changed[par, 2].mean() > 0.99


def test_site_order_within_half_sweep_irrelevant():
    # checkerboard independence: links of one (mu, parity) never enter each other's staples
    L = (4, 6, 4, 4)
    U = oracle.hot_start(L, 3)
    for mu in range(4):
        for p in range(2):
            a = U.copy()
            b = U.copy()
            oracle.half_sweep(L, 5.7, 9, 5, mu, p, a, reverse=False)
            oracle.half_sweep(L, 5.7, 9, 5, mu, p, b, reverse=True)
            assert np.array_equal(a, b)


def test_resume_equals_continuous():
    L = (4, 4, 4, 4)
    a = oracle.hot_start(L, 3)
    b = a.copy()
    oracle.sweep(L, 5.7, 17, 0, 4, a)
    oracle.sweep(L, 5.7, 17, 0, 2, b)
    oracle.sweep(L, 5.7, 17, 2, 2, b)
    assert np.array_equal(a, b)


def test_tiny_lattice_extent_two():
    L = (2, 2, 2, 2)
    U = oracle.hot_start(L, 1)
    (acc, prop), plaq = oracle.sweep(L, 5.7, 1, 0, 3, U)
    unit, det = su3_defects(U)
    assert unit < 1e-13 and det < 1e-13 and prop == 3 * 4 * 16 * 3


# --------------------------------------------------------------------------
# the Kennedy-Pendleton sampler
# --------------------------------------------------------------------------

def kp_target_bin_probs(alpha, edges):
    from scipy import integrate
    f = lambda a: math.sqrt(max(0.0, 1.0 - a * a)) * math.exp(alpha * (a - 1.0))
    probs = np.array([integrate.quad(f, lo, hi, limit=200)[0] for lo, hi in zip(edges[:-1], edges[1:])])
    return probs / probs.sum()


def kp_acceptance_exact(alpha):
    # proposal delta ~ Gamma(3/2, rate alpha); accepted with probability sqrt(1 - delta/2) on delta < 2
    from scipy import integrate
    g = lambda d: math.sqrt(1.0 - d / 2.0) * alpha ** 1.5 / math.gamma(1.5) * math.sqrt(d) * math.exp(-alpha * d)
    return integrate.quad(g, 0.0, 2.0, limit=200)[0]


@pytest.mark.parametrize("alpha", [0.5, 2.0, 8.0, 20.0])
def test_kp_a0_distribution_chisquare(alpha):
    from scipy import stats
    n = 1_000_000
    q, acc = oracle.kp_draws(alpha, 1234 + int(alpha * 10), n)
    a0 = q[acc, 0]
    # bins with roughly equal target mass
    lo = -1.0 if alpha < 4 else max(-1.0, 1.0 - 12.0 / alpha)
    edges = np.linspace(lo, 1.0, 41)
    edges[0] = -1.0  # the first bin also holds the far tail
    probs = kp_target_bin_probs(alpha, edges)
    keep = probs * a0.size > 20
    counts, _ = np.histogram(a0, bins=edges)
    assert counts.sum() == a0.size
    chi2 = (((counts - probs * a0.size) ** 2) / (probs * a0.size))[keep].sum()
    dof = keep.sum() - 1
    assert stats.chi2.sf(chi2, dof) > 1e-4, (chi2, dof)
    # acceptance of the one-hit proposal against its exact value
    pacc = kp_acceptance_exact(alpha)
    assert abs(acc.mean() - pacc) < 5 * math.sqrt(pacc * (1 - pacc) / n)
    # isotropic direction: <a_i> = 0, <a_i^2> = (1 - <a0^2>)/3, |a| = 1
    qa = q[acc]
    assert np.abs((qa ** 2).sum(axis=1) - 1.0).max() < 1e-13
    m2 = (1.0 - (a0 ** 2).mean()) / 3.0
    for i in (1, 2, 3):
        assert abs(qa[:, i].mean()) < 5 * math.sqrt(m2 / a0.size)
        assert abs((qa[:, i] ** 2).mean() - m2) < 5 * math.sqrt(2 * m2 * m2 / a0.size) + 1e-4


# --------------------------------------------------------------------------
# equilibrium: single link, strong and weak coupling
# --------------------------------------------------------------------------

def haar_su3_numpy(rng, n):
    """Haar SU(3) samples from the QR decomposition of complex Gaussian matrices (Mezzadri 2007)."""
    Z = (rng.standard_normal((n, 3, 3)) + 1j * rng.standard_normal((n, 3, 3))) / math.sqrt(2)
    Q, R = np.linalg.qr(Z)
    d = np.diagonal(R, axis1=1, axis2=2)
    Q = Q * (d / np.abs(d))[:, None, :]
    det = np.linalg.det(Q)
    return Q / (det ** (1.0 / 3.0))[:, None, None]


@pytest.mark.parametrize("f32", [False, True])
def test_single_link_heatbath_equilibrium(f32):
    # All links but one frozen: the chain of one-link updates must sample
    # exp((beta/3) Re Tr(U A)) dHaar(U).  Its mean of f = Re Tr(U A)/3 is compared
    # with brute-force Haar Monte Carlo reweighted by the same weight.
    L = (4, 4, 4, 4)
    beta = 2.0
    U = oracle.hot_start(L, 31, f32=f32)
    x = (1, 2, 0, 3)
    mu = 1
    s = site_index(L, x)
    A = cplx(oracle.staple(L, U, s, mu, f32=f32))
    n = 20000
    f = np.empty(n)
    for t in range(n):
        oracle.update_links(L, beta, 77, t, mu, [s], U, f32=f32)
        u = cplx(U[x[3], x[2], x[1], x[0], mu])
        f[t] = np.real(np.trace(u @ A)) / 3.0
    # binned error of the chain
    nb = 40
    bins = f[: (n // nb) * nb].reshape(nb, -1).mean(axis=1)
    chain, chain_err = bins.mean(), bins.std(ddof=1) / math.sqrt(nb)
    rng = np.random.default_rng(5)
    H = haar_su3_numpy(rng, 2_000_000)
    g = np.real(np.einsum("nij,ji->n", H, A)) / 3.0
    w = np.exp(beta * (g - g.max()))
    exact = (g * w).sum() / w.sum()
    exact_err = math.sqrt((((g - exact) * w) ** 2).sum()) / w.sum()
    assert abs(chain - exact) < 4.5 * math.hypot(chain_err, exact_err), (chain, chain_err, exact, exact_err)
    # and the links stay in SU(3) (to rounding of the storage precision)
    unit, det = su3_defects(U)
    assert unit < (2e-7 if f32 else 1e-13)


@pytest.mark.parametrize("beta", [0.1, 0.2])
def test_strong_coupling_plaquette(beta):
    # <P> = beta/18 + beta^2/216 + O(beta^3) (one-plaquette character expansion of SU(3))
    L = (6, 6, 6, 6)
    U = oracle.hot_start(L, 40)
    _, plaq = oracle.sweep(L, beta, 41, 0, 320, U)
    p = plaq[20:]
    nb = 20
    bins = p.reshape(nb, -1).mean(axis=1)
    mean, err = bins.mean(), bins.std(ddof=1) / math.sqrt(nb)
    expect = beta / 18 + beta ** 2 / 216
    assert abs(mean - expect) < 4 * err + 2 * beta ** 3 / 1000, (mean, err, expect)


@pytest.mark.parametrize("beta", [50.0, 100.0])
def test_weak_coupling_plaquette(beta):
    # equipartition over the 3(V-1)(N^2-1) non-gauge Gaussian modes: 1 - <P> = (2/beta)(1 - 1/V)
    L = (4, 4, 4, 4)
    V = np.prod(L)
    U = oracle.cold_start(L)
    _, plaq = oracle.sweep(L, beta, 50, 0, 300, U)
    one_minus = 1.0 - plaq[60:].mean()
    expect = 2.0 / beta * (1.0 - 1.0 / V)
    assert abs(one_minus / expect - 1.0) < 0.03, (one_minus, expect)


def test_one_hit_acceptance_near_paper_value():
    # Soft check: the paper quotes 97.2% one-hit acceptance at beta = 5.7 for its
    # sampler (Sec. 2.1); the KP one-hit acceptance after thermalisation is close.
    L = (6, 6, 6, 6)
    U = oracle.hot_start(L, 60)
    oracle.sweep(L, 5.7, 61, 0, 60, U)
    (acc, prop), _ = oracle.sweep(L, 5.7, 61, 60, 20, U)
    rate = acc / prop
    assert 0.95 < rate < 0.99, rate


# --------------------------------------------------------------------------
# repeat-until-accepted heatbath (the non-MPI program's sampler, Sec. 2.1)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("alpha", [0.5, 8.0])
def test_kp_repeat_until_accepted(alpha):
    # every draw accepted; a0 still follows sqrt(1-a0^2) e^{alpha a0}; the
    # number of proposals is geometric with mean 1/p_acc
    from scipy import stats
    n = 400_000
    q, acc, tries = oracle.kp_draws(alpha, 99, n, max_tries=64, with_tries=True)
    assert acc.all()
    a0 = q[:, 0]
    lo = -1.0 if alpha < 4 else max(-1.0, 1.0 - 12.0 / alpha)
    edges = np.linspace(lo, 1.0, 31)
    edges[0] = -1.0
    probs = kp_target_bin_probs(alpha, edges)
    counts, _ = np.histogram(a0, bins=edges)
    keep = probs * n > 20
    chi2 = (((counts - probs * n) ** 2) / (probs * n))[keep].sum()
    assert stats.chi2.sf(chi2, keep.sum() - 1) > 1e-4, chi2
    p = kp_acceptance_exact(alpha)
    mean_tries = tries / n
    sd = math.sqrt((1 - p) / p ** 2 / n)
    assert abs(mean_tries - 1 / p) < 5 * sd, (mean_tries, 1 / p)


def test_single_link_equilibrium_repeat_until_accepted():
    L = (4, 4, 4, 4)
    beta = 2.0
    U = oracle.hot_start(L, 31)
    x = (1, 2, 0, 3)
    mu = 1
    s = site_index(L, x)
    A = cplx(oracle.staple(L, U, s, mu))
    n = 20000
    f = np.empty(n)
    prop = acc = 0
    for t in range(n):
        acc_t, prop_t = oracle.update_links(L, beta, 78, t, mu, [s], U, max_tries=64)
        acc += acc_t
        prop += prop_t
        u = cplx(U[x[3], x[2], x[1], x[0], mu])
        f[t] = np.real(np.trace(u @ A)) / 3.0
    bins = f.reshape(40, -1).mean(axis=1)
    chain, chain_err = bins.mean(), bins.std(ddof=1) / math.sqrt(40)
    rng = np.random.default_rng(6)
    H = haar_su3_numpy(rng, 2_000_000)
    g = np.real(np.einsum("nij,ji->n", H, A)) / 3.0
    w = np.exp(beta * (g - g.max()))
    exact = (g * w).sum() / w.sum()
    exact_err = math.sqrt((((g - exact) * w) ** 2).sum()) / w.sum()
    assert abs(chain - exact) < 4.5 * math.hypot(chain_err, exact_err), (chain, chain_err, exact, exact_err)
    assert acc >= 0.9999 * 3 * n and prop > 3 * n  # nearly every subgroup accepted, after redraws


def test_one_try_is_the_one_hit_heatbath():
    L = (4, 4, 4, 4)
    a = oracle.hot_start(L, 3)
    b = a.copy()
    sa = oracle.sweep(L, 5.7, 17, 0, 2, a)
    sb = oracle.sweep(L, 5.7, 17, 0, 2, b, max_tries=1)
    assert np.array_equal(a, b) and sa[0] == sb[0]
    c = a.copy()
    (acc, prop), _ = oracle.sweep(L, 5.7, 17, 2, 2, c, max_tries=8)
    assert acc == 2 * 4 * 256 * 3 and prop > acc  # every subgroup accepted, after some retries
