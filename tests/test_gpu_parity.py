"""Parity of the CUDA path (called through the C ABI) with the FP64 CPU oracle.

Every oracle input is produced by the oracle itself (its hot/cold start) or by
the seeded recipes below; no expected value comes from the CUDA path.

Tolerances:
  FP64 path: link by link <= 1e-12 after one half-sweep and after one full
    sweep (same config, same Philox key): both sides run the same FP64
    arithmetic; they differ only by FMA contraction and libm-vs-CUDA
    transcendental rounding (~1e-16 relative per operation, a few hundred
    operations per update).
  FP32-mixed path vs the oracle's FP64 reading of it (same FP32 uniforms,
    storage rounded to FP32 after an FP64 Gram-Schmidt): link by link
    <= 5e-5.  FP32 rounding of the staple (6 paths of 3 products of O(1)
    entries) and of the heatbath gives ~1e-6; the bound leaves headroom for
    the larger |A| of cold-ish configurations.  A one-hit accept decision may
    differ from the oracle's only where the oracle's decision margin is within
    FP32 rounding of the threshold (|margin| < 1e-4); such flips are counted
    and bounded.
"""
import math
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
import paper_0904_1179_gb300 as su3
from paper_0904_1179_gb300 import build as su3_build

pytestmark = pytest.mark.gpu

BETA = 5.7
F64_TOL = 1e-12
F32_TOL = 5e-5
F32_MARGIN = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    su3_build.build()
    oracle.build()


def parity_mask(L):
    x = np.indices((L[3], L[2], L[1], L[0]))
    return (x.sum(axis=0) % 2).astype(bool)


def site_list(L, parity):
    """Canonical indices of the sites of one parity, in canonical order."""
    mask = parity_mask(L).reshape(-1)
    s = np.arange(mask.size)
    return s[mask == bool(parity)]


def flat_links(U):
    return U.reshape(-1, 4, 3, 3, 2)


def su3_defects(U):
    M = (U[..., 0] + 1j * U[..., 1]).reshape(-1, 3, 3)
    unit = np.abs(np.einsum("nki,nkj->nij", M.conj(), M) - np.eye(3)).max()
    det = np.abs(np.linalg.det(M) - 1.0).max()
    return unit, det


# (10, 14, 6, 12): ragged block tails; on a 152-SM GB300 it is above the four-lane
# size limit for FP64 and below it for FP32, so both kernel forms meet it
DIMS_SMALL = [(4, 4, 4, 4), (8, 8, 8, 8), (8, 8, 8, 16), (6, 4, 10, 8), (2, 2, 2, 2), (10, 14, 6, 12)]


# ---------------------------------------------------------------------------
# start configurations, layout, plaquette
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [su3.SU3_FP64, su3.SU3_FP32_MIXED])
def test_cold_start(prec):
    L = (4, 6, 4, 8)
    with su3.Lattice(L, BETA, 1, start=su3.SU3_COLD, precision=prec) as lat:
        U = lat.get_links()
        assert np.array_equal(U, oracle.cold_start(L))
        assert lat.plaquette() == 1.0


@pytest.mark.parametrize("L", [(4, 4, 4, 4), (8, 8, 8, 16), (6, 4, 10, 8)])
def test_hot_start_matches_oracle(L):
    with su3.Lattice(L, BETA, 7, start=su3.SU3_HOT, precision=su3.SU3_FP64) as lat:
        G = lat.get_links()
    O = oracle.hot_start(L, 7)
    assert np.abs(G - O).max() < 1e-13
    with su3.Lattice(L, BETA, 7, start=su3.SU3_HOT, precision=su3.SU3_FP32_MIXED) as lat:
        G = lat.get_links()
    O = oracle.hot_start(L, 7, f32=True)
    # rows 0,1 are the FP32 roundings of the same FP64 numbers: equal, or one
    # float ulp apart where the FP64 values straddle a rounding boundary
    d = np.abs(G - O)
    assert d.max() < 2.5e-7
    assert (d[..., :2, :, :] == 0).mean() > 0.999


@pytest.mark.parametrize("prec", [su3.SU3_FP64, su3.SU3_FP32_MIXED])
def test_links_roundtrip_exact(prec):
    L = (6, 4, 10, 8)
    f32 = prec == su3.SU3_FP32_MIXED
    O = oracle.hot_start(L, 3, f32=f32)
    with su3.Lattice(L, BETA, 1, start=su3.SU3_COLD, precision=prec) as lat:
        lat.set_links(O)
        assert np.array_equal(lat.get_links(), O)


def test_fp32_set_rounds_and_rebuilds_row2():
    L = (4, 4, 4, 4)
    O = oracle.hot_start(L, 3)
    with su3.Lattice(L, BETA, 1, start=su3.SU3_COLD, precision=su3.SU3_FP32_MIXED) as lat:
        lat.set_links(O)
        G = lat.get_links()
    assert np.array_equal(G[..., :2, :, :], O[..., :2, :, :].astype(np.float32).astype(np.float64))
    assert np.abs(G - O).max() < 3e-7


@pytest.mark.parametrize("L", DIMS_SMALL)
def test_plaquette_matches_oracle(L):
    O = oracle.hot_start(L, 11)
    oracle.sweep(L, BETA, 5, 0, 3, O)
    with su3.Lattice(L, BETA, 1, start=su3.SU3_COLD) as lat:
        lat.set_links(O)
        assert abs(lat.plaquette() - oracle.plaquette(L, O)) < 1e-13
    Of = oracle.hot_start(L, 11, f32=True)
    oracle.sweep(L, BETA, 5, 0, 3, Of, f32=True)
    with su3.Lattice(L, BETA, 1, start=su3.SU3_COLD, precision=su3.SU3_FP32_MIXED) as lat:
        lat.set_links(Of)
        assert abs(lat.plaquette() - oracle.plaquette(L, Of, f32=True)) < 2e-6


# ---------------------------------------------------------------------------
# the FP64 sweep
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", DIMS_SMALL)
def test_fp64_half_sweeps_match_oracle(L):
    seed, t = 19, 3
    U0 = oracle.hot_start(L, 5)
    oracle.sweep(L, BETA, 8, 0, 1, U0)
    pm = parity_mask(L)
    with su3.Lattice(L, BETA, seed, start=su3.SU3_COLD) as lat:
        for mu in range(4):
            for p in range(2):
                lat.set_links(U0)
                lat.sweep_count = t
                lat.half_sweep(mu, p)
                G = lat.get_links()
                O = U0.copy()
                oracle.half_sweep(L, BETA, seed, t, mu, p, O)
                assert np.abs(G - O).max() < F64_TOL, (mu, p, np.abs(G - O).max())
                # only the links of (mu, p) changed
                other = np.ones((L[3], L[2], L[1], L[0], 4), dtype=bool)
                other[pm == bool(p), mu] = False
                assert np.array_equal(G[other], U0[other])


@pytest.mark.parametrize("L", DIMS_SMALL)
def test_fp64_sweep_matches_oracle(L):
    seed = 23
    U0 = oracle.hot_start(L, 6)
    O = U0.copy()
    (acc, prop), plaq = oracle.sweep(L, BETA, seed, 0, 2, O)
    with su3.Lattice(L, BETA, seed, start=su3.SU3_COLD) as lat:
        lat.set_links(U0)
        lat.set_stats(True)
        lat.sweep(2)
        G = lat.get_links()
        assert lat.sweep_count == 2
        assert np.abs(G - O).max() < F64_TOL
        assert lat.stats() == (acc, prop)
        assert abs(lat.plaquette() - plaq[-1]) < 1e-13


@pytest.mark.parametrize("beta", [0.2, 50.0])
def test_extreme_couplings_match_oracle(beta):
    # strong coupling (alpha ~ 0.1: the Kennedy-Pendleton proposal is often
    # rejected) and weak coupling (alpha ~ 100): one sweep link by link (FP64)
    # and one half-sweep against the oracle's FP32 reading
    L = (4, 4, 4, 6)
    U0 = oracle.hot_start(L, 8)
    O = U0.copy()
    stats, _ = oracle.sweep(L, beta, 12, 0, 1, O)
    with su3.Lattice(L, beta, 12, start=su3.SU3_COLD) as lat:
        lat.set_links(U0)
        lat.set_stats(True)
        lat.sweep(1)
        assert np.abs(lat.get_links() - O).max() < F64_TOL
        assert lat.stats() == stats
    U32 = oracle.hot_start(L, 8, f32=True)
    with su3.Lattice(L, beta, 12, start=su3.SU3_COLD, precision=su3.SU3_FP32_MIXED) as lat:
        lat.set_links(U32)
        lat.half_sweep(1, 0)
        G = flat_links(lat.get_links())
        sites = site_list(L, 0)
        Of, marg = oracle.updated_links(L, beta, 12, 0, 1, sites, U32, f32=True, with_margins=True)
        d = np.abs(G[sites, 1] - Of).max(axis=(1, 2, 3))
        bad = d > F32_TOL
        assert bad.sum() <= 1 and (not bad.any() or (np.nanmin(np.abs(marg[bad]), axis=1) < F32_MARGIN).all())


def test_fp64_cold_start_chain_config0():
    # 4^4, beta 5.7, cold start, Philox seed 1, 20 sweeps, plaquette after each sweep
    L = (4, 4, 4, 4)
    O = oracle.cold_start(L)
    _, plaq = oracle.sweep(L, BETA, 1, 0, 20, O)
    with su3.Lattice(L, BETA, 1, start=su3.SU3_COLD) as lat:
        gp = []
        for _ in range(20):
            lat.sweep(1)
            gp.append(lat.plaquette())
        assert np.abs(lat.get_links() - O).max() < F64_TOL
    assert np.abs(np.array(gp) - plaq).max() < 1e-13


def test_graph_replay_equals_eager_half_sweeps():
    L = (8, 8, 8, 16)
    for prec in (su3.SU3_FP64, su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT):
        with su3.Lattice(L, BETA, 4, start=su3.SU3_HOT, precision=prec) as a, \
                su3.Lattice(L, BETA, 4, start=su3.SU3_HOT, precision=prec) as b:
            a.sweep(3)
            for t in range(3):
                for mu in range(4):
                    for p in range(2):
                        b.half_sweep(mu, p)
                b.sweep_count = t + 1
            assert np.array_equal(a.get_links(), b.get_links())


@pytest.mark.parametrize("prec", [su3.SU3_FP64, su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT])
def test_block_size_does_not_change_results(prec):
    L = (6, 4, 10, 8)
    ref = None
    for threads in (32, 64, 96, 128, 256):
        with su3.Lattice(L, BETA, 9, start=su3.SU3_HOT, precision=prec) as lat:
            lat.set_block_size(threads)
            lat.sweep(2)
            U = lat.get_links()
        if ref is None:
            ref = U
        assert np.array_equal(U, ref), threads


@pytest.mark.parametrize("prec", [su3.SU3_FP64, su3.SU3_FP32_MIXED])
def test_resume_from_checkpoint(prec):
    L = (8, 8, 8, 8)
    with su3.Lattice(L, BETA, 31, start=su3.SU3_HOT, precision=prec) as a:
        a.sweep(4)
        ref = a.get_links()
    with su3.Lattice(L, BETA, 31, start=su3.SU3_HOT, precision=prec) as b:
        b.sweep(2)
        ck = b.get_links()
        n = b.sweep_count
    with su3.Lattice(L, BETA, 31, start=su3.SU3_COLD, precision=prec) as c:
        c.set_links(ck)
        c.sweep_count = n
        c.sweep(2)
        assert np.array_equal(c.get_links(), ref)


# ---------------------------------------------------------------------------
# the FP32-mixed sweep
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT])
@pytest.mark.parametrize("L", [(4, 4, 4, 4), (8, 8, 8, 8), (6, 4, 10, 8), (10, 14, 6, 12)])
def test_fp32_half_sweeps_match_oracle_reading(L, prec):
    seed, t = 29, 5
    U0 = oracle.hot_start(L, 7, f32=True)
    oracle.sweep(L, BETA, 2, 0, 2, U0, f32=True)
    pm = parity_mask(L)
    flips = 0
    total = 0
    worst = 0.0
    with su3.Lattice(L, BETA, seed, start=su3.SU3_COLD, precision=prec) as lat:
        for mu in range(4):
            for p in range(2):
                lat.set_links(U0)
                lat.sweep_count = t
                lat.half_sweep(mu, p)
                G = flat_links(lat.get_links())
                sites = site_list(L, p)
                O, marg = oracle.updated_links(L, BETA, seed, t, mu, sites, U0, f32=True, with_margins=True)
                d = np.abs(G[sites, mu] - O).max(axis=(1, 2, 3))
                bad = d > F32_TOL
                if bad.any():
                    m = np.nanmin(np.abs(marg[bad]), axis=1)
                    assert (m < F32_MARGIN).all(), (mu, p, d[bad], m)
                flips += int(bad.sum())
                total += sites.size
                worst = max(worst, float(d[~bad].max()))
                other = np.ones((L[3], L[2], L[1], L[0], 4), dtype=bool)
                other[pm == bool(p), mu] = False
                assert np.array_equal(lat.get_links()[other], U0[other])
    assert flips <= max(2, total // 2000), (flips, total)
    print("fp32 (precision %d) half-sweeps %s: worst |dU| %.2e, flips %d of %d" % (prec, L, worst, flips, total))


# The same lattice updated by the four-lane kernel and by the one-thread kernel
# (one thread per link pair where L3 is a multiple of 4, per link otherwise),
# each checked against the oracle's FP32 reading, and against each other: both
# add the staple in the same order and round every step identically.
@pytest.mark.parametrize("prec", [su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT])
@pytest.mark.parametrize("L", [(8, 8, 8, 8), (6, 4, 10, 8), (10, 14, 6, 10)])
def test_fp32_four_lane_and_one_lane_kernels_match_oracle_reading(L, prec):
    seed, t = 41, 3
    U0 = oracle.hot_start(L, 9, f32=True)
    oracle.sweep(L, BETA, 4, 0, 1, U0, f32=True)
    flips = total = 0
    with su3.Lattice(L, BETA, seed, start=su3.SU3_COLD, precision=prec) as lat:
        for mu in range(4):
            for p in range(2):
                got = {}
                for lanes in (4, 1):
                    lat.set_lanes(lanes)
                    lat.set_links(U0)
                    lat.sweep_count = t
                    lat.half_sweep(mu, p)
                    got[lanes] = lat.get_links()
                assert np.array_equal(got[4], got[1]), (mu, p)
                sites = site_list(L, p)
                O, marg = oracle.updated_links(L, BETA, seed, t, mu, sites, U0, f32=True, with_margins=True)
                d = np.abs(flat_links(got[1])[sites, mu] - O).max(axis=(1, 2, 3))
                bad = d > F32_TOL
                if bad.any():
                    assert (np.nanmin(np.abs(marg[bad]), axis=1) < F32_MARGIN).all(), (mu, p, d[bad])
                flips += int(bad.sum())
                total += sites.size
        lat.set_lanes(0)
    assert flips <= max(2, total // 2000), (flips, total)


def test_lanes_setting_validated():
    with su3.Lattice((4, 4, 4, 4), BETA, 1, start=su3.SU3_COLD) as lat:
        for bad in (-1, 2, 3, 8):
            with pytest.raises(su3.Su3Error):
                lat.set_lanes(bad)
        lat.set_lanes(4)
        lat.set_lanes(0)
    with su3.Batch([(4, 4, 4, 4)], [BETA], [1], start=su3.SU3_COLD) as b:
        with pytest.raises(su3.Su3Error):
            su3.su3_set_lanes(b.handle, 1)


# The FP32 fused plaquette (taken inside the odd-site updates of mu = 1, 2, 3)
# against the oracle's plaquette of the configuration the sweep produced, in
# the oracle's FP32 reading (row 2 rebuilt from the stored rows): the bound is
# the FP32 rounding of the staple terms, ~1e-7 per plaquette.
@pytest.mark.parametrize("prec", [su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT])
@pytest.mark.parametrize("L", [(8, 8, 8, 16), (6, 4, 10, 6), (4, 4, 4, 4)])
def test_fp32_fused_plaquette_matches_oracle(L, prec):
    U0 = oracle.hot_start(L, 13, f32=True)
    with su3.Lattice(L, BETA, 6, start=su3.SU3_COLD, precision=prec) as lat:
        lat.set_links(U0)
        for _ in range(3):
            got = lat.sweep_measured(1)[0]
            ref = oracle.plaquette(L, lat.get_links(), f32=True)
            assert abs(got - ref) < 2e-6, (got, ref)


@pytest.mark.parametrize("prec", [su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT])
def test_fp32_far_from_unitary_takes_full_gram_schmidt(prec):
    # the links being updated have rows 0 and 1 stretched by 2 % and 1.5 %
    # (their staples, from the other links, stay in SU(3)): the
    # reunitarisation's norm errors exceed 1e-3, so every updated link goes
    # through the full FP64 Gram-Schmidt branch; the result is still the
    # oracle's FP32 reading, and unitary to FP32 rounding
    L = (4, 4, 4, 8)
    U0 = oracle.hot_start(L, 17, f32=True)
    pm = parity_mask(L)
    seed, t = 31, 2
    with su3.Lattice(L, BETA, seed, start=su3.SU3_COLD, precision=prec) as lat:
        for mu, p in ((0, 0), (2, 1)):
            U1 = U0.copy()
            sel = U1[pm == bool(p), mu]
            sel[:, 0] *= 1.02
            sel[:, 1] *= 0.985
            U1[pm == bool(p), mu] = sel
            U1 = U1.astype(np.float32).astype(np.float64)
            lat.set_links(U1)
            lat.sweep_count = t
            lat.half_sweep(mu, p)
            G = flat_links(lat.get_links())
            sites = site_list(L, p)
            O, marg = oracle.updated_links(L, BETA, seed, t, mu, sites, U1, f32=True, with_margins=True)
            d = np.abs(G[sites, mu] - O).max(axis=(1, 2, 3))
            bad = d > F32_TOL
            assert bad.sum() <= 1, (bad.sum(), d.max())
            assert not bad.any() or (np.nanmin(np.abs(marg[bad]), axis=1) < F32_MARGIN).all()
            unit, det = su3_defects(G[sites, mu])
            assert unit < 5e-7 and det < 5e-7, (unit, det)


def test_fp32_links_stay_su3_and_float():
    L = (8, 8, 8, 8)
    with su3.Lattice(L, BETA, 3, start=su3.SU3_HOT, precision=su3.SU3_FP32_MIXED) as lat:
        lat.sweep(10)
        U = lat.get_links()
    rows = U[..., :2, :, :]
    assert np.array_equal(rows, rows.astype(np.float32).astype(np.float64))
    unit, det = su3_defects(U)
    assert unit < 5e-7 and det < 5e-7


# ---------------------------------------------------------------------------
# full-size lattice (32^4, the benchmark's workload), sampled against the oracle
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("prec", [su3.SU3_FP64, su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT])
def test_full_size_32x4_sampled(prec):
    L = (32, 32, 32, 32)
    f32 = prec != su3.SU3_FP64
    seed = 7
    U0 = oracle.hot_start(L, seed, f32=f32)
    rng = np.random.default_rng(1)
    with su3.Lattice(L, BETA, seed, start=su3.SU3_HOT, precision=prec) as lat:
        G0 = lat.get_links()
        # GPU hot start = oracle hot start (Gram-Schmidt of Gaussian rows amplifies
        # rounding by 1/|r1 - proj|, ~100 for the worst of 4.2M links)
        assert np.abs(G0 - U0).max() < (2.5e-7 if f32 else 1e-13)
        lat.set_links(U0)
        for mu, p in ((0, 0), (3, 1)):
            lat.set_links(U0)
            lat.half_sweep(mu, p)
            G = flat_links(lat.get_links())
            sites = rng.choice(site_list(L, p), size=1500, replace=False)
            O, marg = oracle.updated_links(L, BETA, seed, 0, mu, sites, U0, f32=f32, with_margins=True)
            d = np.abs(G[sites, mu] - O).max(axis=(1, 2, 3))
            if f32:
                bad = d > F32_TOL
                assert bad.sum() <= 2
                if bad.any():
                    assert (np.nanmin(np.abs(marg[bad]), axis=1) < F32_MARGIN).all()
            else:
                assert d.max() < F64_TOL
        # the graphed sweep at full size equals eight eager half-sweeps, and keeps SU(3)
        lat.set_links(U0)
        lat.sweep_count = 0
        lat.sweep(1)
        A = lat.get_links()
        lat.set_links(U0)
        lat.sweep_count = 0
        for mu in range(4):
            for p in range(2):
                lat.half_sweep(mu, p)
        B = lat.get_links()
        assert np.array_equal(A, B)
        sample = flat_links(A)[rng.choice(np.prod(L), size=20000, replace=False)]
        unit, det = su3_defects(sample)
        assert unit < (5e-7 if f32 else 1e-13) and det < (5e-7 if f32 else 1e-13)


def tiled_config(tile, reps, seed, f32):
    """An oracle hot start on a small lattice, repeated periodically: a seeded
    non-trivial configuration of a large lattice without generating every
    link.  Neighbour wraps of the large lattice still meet different links."""
    Ut = oracle.hot_start(tile, seed, f32=f32)
    return np.ascontiguousarray(np.tile(Ut, (reps, reps, reps, reps, 1, 1, 1, 1)))


@pytest.mark.parametrize("L,beta,tile", [((48, 48, 48, 48), 5.7, (12, 12, 12, 12)),
                                         ((64, 64, 64, 64), 6.0, (8, 8, 8, 8))])
def test_large_lattices_sampled(L, beta, tile):
    # the precision study's 48^4 and the large-lattice 64^4 workloads at full
    # size: sampled updated links of two half-sweeps against the oracle
    reps = L[0] // tile[0]
    rng = np.random.default_rng(5)
    for prec in (su3.SU3_FP64, su3.SU3_FP32_MIXED):
        f32 = prec != su3.SU3_FP64
        U0 = tiled_config(tile, reps, 21, f32)
        with su3.Lattice(L, beta, 7, start=su3.SU3_COLD, precision=prec) as lat:
            for mu, p in ((2, 1), (3, 0)):
                lat.set_links(U0)
                lat.sweep_count = 5
                lat.half_sweep(mu, p)
                G = flat_links(lat.get_links())
                # sites on the wrap of every direction, and random ones
                edge = [s for s in (0, np.prod(L) - 1, L[0] - 1, L[0] * L[1] * L[2] * (L[3] - 1))
                        if (lambda x: sum(x) % 2)(np.unravel_index(s, L[::-1])) == p]
                sites = np.concatenate([edge, rng.choice(site_list(L, p), size=300, replace=False)]).astype(np.int64)
                O, marg = oracle.updated_links(L, beta, 7, 5, mu, sites, U0, f32=f32, with_margins=True)
                d = np.abs(G[sites, mu] - O).max(axis=(1, 2, 3))
                if f32:
                    bad = d > F32_TOL
                    assert bad.sum() <= 1
                    if bad.any():
                        assert (np.nanmin(np.abs(marg[bad]), axis=1) < F32_MARGIN).all()
                else:
                    assert d.max() < F64_TOL, d.max()
                del G
        del U0


# ---------------------------------------------------------------------------
# statistical agreement over long chains
# ---------------------------------------------------------------------------

def binned(x, nb=20):
    x = np.asarray(x)
    b = x[: (x.size // nb) * nb].reshape(nb, -1).mean(axis=1)
    return b.mean(), b.std(ddof=1) / math.sqrt(nb)


def test_fp64_chain_agrees_with_oracle_chain():
    # independent chains (different seeds), 6^4 at beta 5.7, binned means within 3 sigma
    L = (6, 6, 6, 6)
    O = oracle.hot_start(L, 100)
    _, po = oracle.sweep(L, BETA, 101, 0, 600, O)
    with su3.Lattice(L, BETA, 202, start=su3.SU3_HOT) as lat:
        lat.sweep(100)
        pg = []
        for _ in range(2000):
            lat.sweep(1)
            pg.append(lat.plaquette())
    mo, eo = binned(po[100:])
    mg, eg = binned(pg)
    assert abs(mo - mg) < 3 * math.hypot(eo, eg), (mo, eo, mg, eg)


def test_fp32_chain_agrees_with_fp64_chain():
    L = (8, 8, 8, 8)
    res = {}
    for prec in (su3.SU3_FP64, su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT):
        with su3.Lattice(L, BETA, 300 + prec, start=su3.SU3_HOT, precision=prec) as lat:
            lat.sweep(200)
            p = []
            for _ in range(2000):
                lat.sweep(1)
                p.append(lat.plaquette())
        res[prec] = binned(p)
    (m64, e64), (m32, e32), (me, ee) = res[su3.SU3_FP64], res[su3.SU3_FP32_MIXED], res[su3.SU3_FP32_EFT]
    assert abs(m64 - m32) < 3 * math.hypot(e64, e32), res
    assert abs(m64 - me) < 3 * math.hypot(e64, ee), res
    print("plaquette 8^4 beta 5.7: FP64 %.6f(%d)  FP32-mixed %.6f(%d)  FP32-EFT %.6f(%d)"
          % (m64, round(e64 * 1e6), m32, round(e32 * 1e6), me, round(ee * 1e6)))


def test_acceptance_rate_reported():
    L = (8, 8, 8, 8)
    with su3.Lattice(L, BETA, 5, start=su3.SU3_HOT) as lat:
        lat.sweep(100)
        lat.set_stats(True)
        lat.sweep(20)
        acc, prop = lat.stats()
    rate = acc / prop
    assert prop == 20 * 4 * np.prod(L) * 3
    assert 0.95 < rate < 0.99
    print("one-hit acceptance at beta 5.7: %.4f (paper: 0.972)" % rate)


# ---------------------------------------------------------------------------
# the oracle's Philox against cuRAND's (a third-party implementation)
# ---------------------------------------------------------------------------

CURAND_PROBE = r"""
#include <cstdio>
#include <curand_philox4x32_x.h>
__global__ void k(const uint4* c, const uint2* key, uint4* o, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = curand_Philox4x32_10(c[i], key[i]);
}
int main() {
  const int n = 256;
  uint4 hc[n]; uint2 hk[n]; uint4 ho[n];
  unsigned s = 12345u;
  for (int i = 0; i < n; ++i) {
    unsigned w[6];
    for (int j = 0; j < 6; ++j) { s = s * 1664525u + 1013904223u; w[j] = s; }
    hc[i] = make_uint4(w[0], w[1], w[2], w[3]); hk[i] = make_uint2(w[4], w[5]);
  }
  uint4 *dc, *dout; uint2* dk;
  cudaMalloc(&dc, sizeof hc); cudaMalloc(&dk, sizeof hk); cudaMalloc(&dout, sizeof ho);
  cudaMemcpy(dc, hc, sizeof hc, cudaMemcpyHostToDevice);
  cudaMemcpy(dk, hk, sizeof hk, cudaMemcpyHostToDevice);
  k<<<(n + 127) / 128, 128>>>(dc, dk, dout, n);
  if (cudaMemcpy(ho, dout, sizeof ho, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  for (int i = 0; i < n; ++i)
    printf("%u %u %u %u %u %u %u %u %u %u\n", hc[i].x, hc[i].y, hc[i].z, hc[i].w, hk[i].x, hk[i].y,
           ho[i].x, ho[i].y, ho[i].z, ho[i].w);
  return 0;
}
"""


def test_philox_matches_curand():
    nvcc = su3_build.nvcc()
    d = tempfile.mkdtemp()
    try:
        src = os.path.join(d, "probe.cu")
        exe = os.path.join(d, "probe")
        open(src, "w").write(CURAND_PROBE)
        subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe, src], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
        rows = [list(map(int, ln.split())) for ln in out if ln.strip()]
        assert len(rows) == 256
        for r in rows:
            assert oracle.philox4x32_10(r[0:4], r[4:6]) == r[6:10]
    finally:
        shutil.rmtree(d)


# ---------------------------------------------------------------------------
# repeat-until-accepted heatbath (max_tries > 1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 10, 8)])
def test_fp64_repeat_until_accepted_matches_oracle(L):
    seed, tries = 41, 8
    U0 = oracle.hot_start(L, 12)
    for mu, p in ((0, 0), (3, 1)):
        with su3.Lattice(L, BETA, seed, start=su3.SU3_COLD) as lat:
            lat.set_heatbath(tries)
            lat.set_links(U0)
            lat.sweep_count = 2
            lat.set_stats(True)
            lat.half_sweep(mu, p)
            G = lat.get_links()
            gstats = lat.stats()
        O = U0.copy()
        ostats = oracle.half_sweep(L, BETA, seed, 2, mu, p, O, max_tries=tries)
        assert np.abs(G - O).max() < F64_TOL
        assert gstats == ostats and ostats[1] > ostats[0]
    # a full sweep
    O = U0.copy()
    ostats, _ = oracle.sweep(L, BETA, seed, 0, 1, O, max_tries=tries)
    with su3.Lattice(L, BETA, seed, start=su3.SU3_COLD) as lat:
        lat.set_heatbath(tries)
        lat.set_links(U0)
        lat.set_stats(True)
        lat.sweep(1)
        assert np.abs(lat.get_links() - O).max() < F64_TOL
        assert lat.stats() == ostats


@pytest.mark.parametrize("prec", [su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT])
def test_fp32_repeat_until_accepted_matches_oracle_reading(prec):
    L = (8, 8, 8, 8)
    seed, t, tries = 43, 3, 8
    U0 = oracle.hot_start(L, 9, f32=True)
    with su3.Lattice(L, BETA, seed, start=su3.SU3_COLD, precision=prec) as lat:
        lat.set_heatbath(tries)
        for mu, p in ((1, 0), (2, 1)):
            lat.set_links(U0)
            lat.sweep_count = t
            lat.half_sweep(mu, p)
            G = flat_links(lat.get_links())
            sites = site_list(L, p)
            O, marg = oracle.updated_links(L, BETA, seed, t, mu, sites, U0, f32=True, with_margins=True,
                                           max_tries=tries)
            d = np.abs(G[sites, mu] - O).max(axis=(1, 2, 3))
            assert (d > F32_TOL).sum() <= 2, d.max()


def test_heatbath_setting_validated():
    with su3.Lattice((4, 4, 4, 4), BETA, 1, start=su3.SU3_COLD) as lat:
        for bad in (0, -3, (1 << 20) + 1):
            with pytest.raises(su3.Su3Error):
                lat.set_heatbath(bad)
        lat.set_heatbath(1)


# ---------------------------------------------------------------------------
# plaquette fused into the sweep (su3_sweep_measured)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("L", [(4, 4, 4, 4), (6, 4, 10, 8), (2, 2, 2, 2)])
def test_fp64_fused_plaquette_matches_oracle(L):
    # per-sweep plaquettes of the updated configuration, against the oracle's
    # separate plaquette pass after each sweep
    seed, n = 17, 4
    U0 = oracle.hot_start(L, 5)
    O = U0.copy()
    _, plaq = oracle.sweep(L, BETA, seed, 0, n, O)
    with su3.Lattice(L, BETA, seed, start=su3.SU3_COLD) as lat:
        lat.set_links(U0)
        got = lat.sweep_measured(n)
        assert lat.sweep_count == n
        assert np.abs(lat.get_links() - O).max() < F64_TOL
        assert abs(lat.plaquette() - got[-1]) < 1e-14
    assert np.abs(got - plaq).max() < 1e-13


@pytest.mark.parametrize("prec", [su3.SU3_FP64, su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT])
def test_fused_plaquette_same_chain_as_sweep(prec):
    # the measuring sweep updates exactly like su3_sweep; its plaquette equals
    # su3_plaquette of the same configuration up to summation order (FP64) or
    # the FP32 staple rounding (~1e-7 per plaquette, averaged over the lattice)
    L = (8, 8, 8, 16)
    tol = 1e-13 if prec == su3.SU3_FP64 else 2e-6
    with su3.Lattice(L, BETA, 3, start=su3.SU3_HOT, precision=prec) as a, \
            su3.Lattice(L, BETA, 3, start=su3.SU3_HOT, precision=prec) as b:
        ref = []
        for _ in range(3):
            a.sweep(1)
            ref.append(a.plaquette())
        got = b.sweep_measured(3)
        assert np.array_equal(a.get_links(), b.get_links())
        assert np.abs(got - np.array(ref)).max() < tol
        b.set_block_size(64)  # partials are re-sized with the block size
        a.sweep(1)
        got2 = b.sweep_measured(1)
        assert np.array_equal(a.get_links(), b.get_links())
        assert abs(got2[0] - a.plaquette()) < tol


def test_fused_plaquette_ring_wraps_and_needs_stats_off():
    L = (4, 4, 4, 4)
    n = 4100  # more than one ring of per-sweep results
    with su3.Lattice(L, BETA, 8, start=su3.SU3_HOT) as a, su3.Lattice(L, BETA, 8, start=su3.SU3_HOT) as b:
        got = a.sweep_measured(n)
        b.sweep(n - 5)
        ref = []
        for _ in range(5):
            b.sweep(1)
            ref.append(b.plaquette())
        assert np.abs(got[-5:] - np.array(ref)).max() < 1e-13
        assert np.all(np.isfinite(got)) and np.all(np.abs(got) <= 1.0)
        assert len(a.sweep_measured(0)) == 0
        a.set_stats(True)
        with pytest.raises(su3.Su3Error):
            a.sweep_measured(1)
        a.set_stats(False)
        a.sweep_measured(1)
        with pytest.raises(su3.Su3Error):
            su3.su3_sweep_measured(a.handle, -1)


# ---------------------------------------------------------------------------
# the paper's Table 1 workloads in full: 8^4 x 512, 12^4 x 101, 16^4 x 32,
# 32^4 x 2 sweeps, FP64, beta 5.7, hot start from seed 7.
#
# Two chains that share every random number but differ by rounding do not
# stay together forever: at beta 5.7 a 1e-15 difference grows about 2x per
# sweep (the oracle against itself with one entry changed by 1e-15 reaches
# 1e-10 after 15 sweeps, 1e-4 after 65, and an accept decision flips near
# sweep 74, after which the chains are unrelated samples of the same
# distribution).  So: per-sweep plaquettes to 1e-12 over the first 8 sweeps,
# every link of the 32^4 column after its 2 sweeps to 1e-12, and the 8^4
# chain's equilibrium plaquette and acceptance statistically.
# ---------------------------------------------------------------------------

def _binned(x, nb):
    x = np.asarray(x)[: len(x) // nb * nb].reshape(nb, -1).mean(axis=1)
    return x.mean(), x.std(ddof=1) / math.sqrt(nb)


def test_table1_chains_match_oracle():
    import concurrent.futures as cf
    import multiprocessing as mp
    from paper_0904_1179_gb300.workloads import TABLE1, HEADLINE_SEED
    horizon = 8
    # the four oracle chains run at once (spawned processes, one thread each)
    with cf.ProcessPoolExecutor(max_workers=len(TABLE1), mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(oracle.hot_chain, L, BETA, HEADLINE_SEED, n) for L, n in TABLE1]
        gpu = []
        for L, n in TABLE1:
            with su3.Lattice(L, BETA, HEADLINE_SEED, start=su3.SU3_HOT) as lat:
                plaq = lat.sweep_measured(n)
                gpu.append((lat.get_links() if n <= horizon else None, plaq))
        ref = [f.result() for f in futs]
    for (L, n), (G, gp), (O, op, _, _) in zip(TABLE1, gpu, ref):
        k = min(n, horizon)
        assert np.abs(gp[:k] - op[:k]).max() < 1e-12, (L, np.abs(gp[:k] - op[:k]).max())
        if G is not None:
            assert np.abs(G - O).max() < 1e-12, (L, np.abs(G - O).max())
    # 8^4 x 512: equilibrium plaquette after 112 thermalisation sweeps, 20 bins
    g_mean, g_err = _binned(gpu[0][1][112:], 20)
    o_mean, o_err = _binned(ref[0][1][112:], 20)
    assert abs(g_mean - o_mean) < 4 * math.hypot(g_err, o_err), (g_mean, g_err, o_mean, o_err)


