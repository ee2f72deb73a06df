"""The paper's domain decomposition emulated on one GPU (Sec. 2.1, Tables 1-2).

A decomposed lattice must reproduce the undivided lattice bit for bit: every
link update runs the same arithmetic on the same neighbours with the same
Philox numbers (keyed by the global site); the decomposition only changes
where links are stored and adds the boundary exchange.  So the reference here
is the single-lattice path, itself pinned to the oracle by test_gpu_parity.py,
plus one direct comparison with the oracle.
"""
import numpy as np
import pytest

import oracle
import paper_0904_1179_gb300 as su3
from paper_0904_1179_gb300 import build as su3_build

pytestmark = pytest.mark.gpu

BETA = 5.7
PRECS = [su3.SU3_FP64, su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT]
# (ndmpi, mpifactor, lbcex)
DECOMPS = [(1, 2, 1), (2, 2, 1), (3, 2, 1), (4, 2, 1), (1, 1, 1), (4, 1, 1), (2, 4, 1), (1, 1, 0)]


@pytest.fixture(scope="module", autouse=True)
def built():
    su3_build.build()
    oracle.build()


def run(L, prec, decomp, seed=5, sweeps=2):
    with su3.Lattice(L, BETA, seed, start=su3.SU3_HOT, precision=prec, decomp=decomp) as lat:
        lat.set_stats(True)
        lat.sweep(sweeps)
        return lat.get_links(), lat.stats(), lat.plaquette()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("decomp", DECOMPS)
def test_decomposed_sweep_bitwise_equals_plain(prec, decomp):
    L = (8, 8, 8, 8)
    ref = run(L, prec, None)
    got = run(L, prec, decomp)
    assert np.array_equal(got[0], ref[0])
    assert got[1] == ref[1]
    assert got[2] == ref[2]


@pytest.mark.parametrize("decomp", [(2, 2, 1), (4, 2, 1), (3, 2, 1)])
def test_uneven_extents(decomp):
    # sublattices (4, 2, 6, 4): the thinnest legal slab, and unequal extents
    L = (8, 4, 12, 8)
    for prec in (su3.SU3_FP64, su3.SU3_FP32_MIXED):
        assert np.array_equal(run(L, prec, decomp)[0], run(L, prec, None)[0])


def test_decomposed_matches_oracle():
    L = (4, 8, 4, 4)
    U0 = oracle.hot_start(L, 3)
    O = U0.copy()
    stats, plaq = oracle.sweep(L, BETA, 9, 0, 2, O)
    with su3.Lattice(L, BETA, 9, start=su3.SU3_COLD, decomp=(2, 2, 1)) as lat:
        lat.set_links(U0)
        lat.set_stats(True)
        lat.sweep(2)
        assert np.abs(lat.get_links() - O).max() < 1e-12
        assert lat.stats() == stats
        assert abs(lat.plaquette() - plaq[-1]) < 1e-13


@pytest.mark.parametrize("prec", [su3.SU3_FP64, su3.SU3_FP32_MIXED])
def test_half_sweeps_set_get_and_block_size(prec):
    L = (8, 8, 8, 8)
    with su3.Lattice(L, BETA, 6, start=su3.SU3_HOT, precision=prec) as a, \
            su3.Lattice(L, BETA, 6, start=su3.SU3_HOT, precision=prec, decomp=(3, 2, 1)) as b:
        # eager half-sweeps
        for mu in range(4):
            for p in range(2):
                a.half_sweep(mu, p)
                b.half_sweep(mu, p)
        assert np.array_equal(a.get_links(), b.get_links())
        # gather, keep sweeping from the sublattices
        a.sweep_count = b.sweep_count = 1
        a.sweep(1)
        b.sweep(1)
        assert np.array_equal(a.get_links(), b.get_links())
        # set a new configuration: scattered into the sublattices, ghosts refilled
        U = oracle.hot_start(L, 77, f32=prec != su3.SU3_FP64)
        a.set_links(U)
        b.set_links(U)
        b.set_block_size(64)
        a.sweep(2)
        b.sweep(2)
        assert np.array_equal(a.get_links(), b.get_links())
        assert a.plaquette() == b.plaquette()


def _halo_sites(L, nd, nf):
    """Ghost cells a sublattice's staples read: the faces of every cut
    direction and the edges x + a - b of every ordered pair of cut directions."""
    l = [L[d] // nf if d < nd else L[d] for d in range(4)]
    vol = int(np.prod(l))
    faces = sum(2 * vol // l[d] for d in range(nd))
    edges = sum(vol // (l[a] * l[b]) for a in range(nd) for b in range(nd) if a != b)
    return (faces + edges) * nf ** nd


@pytest.mark.parametrize("decomp", DECOMPS)
def test_decomp_info(decomp):
    L = (8, 8, 12, 8)
    with su3.Lattice(L, BETA, 1, start=su3.SU3_COLD, decomp=decomp) as lat:
        nd, nf, ex, nsub, halo = lat.decomp_info()
        assert (nd, nf, ex) == decomp and nsub == nf ** nd
        # every ghost cell is refreshed for its 4 directions once per sweep
        assert halo == (4 * _halo_sites(L, nd, nf) if ex else 0)
    with su3.Lattice(L, BETA, 1, start=su3.SU3_COLD) as lat:
        assert lat.decomp_info() == (0, 1, 0, 1, 0)


def test_bad_arguments():
    L = (8, 8, 12, 8)
    for nd, nf, ex in [(0, 2, 1), (5, 2, 1), (1, 0, 1), (1, 2, 0), (3, 4, 1), (2, 3, 1), (1, 2, 2)]:
        with pytest.raises(su3.Su3Error):
            su3.su3_decomp_create(*L, BETA, 1, su3.SU3_COLD, su3.SU3_FP64, nd, nf, ex)
    with su3.Lattice(L, BETA, 1, start=su3.SU3_COLD, decomp=(2, 2, 1)) as lat:
        with pytest.raises(su3.Su3Error):
            lat.set_lanes(1)
        lat.set_stats(True)
        with pytest.raises(su3.Su3Error):
            lat.sweep_measured(1)
        lat.set_stats(False)
        lat.sweep(1)


# The fused plaquette and the repeat-until-accepted heatbath on decomposed
# lattices: the same chain and the same per-sweep plaquettes as the undivided
# lattice, bit for bit (the sublattice kernels run the same update code on
# the same neighbours and random numbers, and the per-block partial sums of
# the plaquette are added in a fixed order -- different blocks than the
# undivided kernel's, so the plaquettes agree to summation order).
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("decomp", [(2, 2, 1), (4, 2, 1), (1, 1, 0)])
def test_decomposed_measured_sweep_and_repeat_heatbath(prec, decomp):
    L = (8, 8, 8, 8)
    tol = 1e-13 if prec == su3.SU3_FP64 else 2e-6
    for max_tries in (1, 6):
        with su3.Lattice(L, BETA, 12, start=su3.SU3_HOT, precision=prec) as a, \
                su3.Lattice(L, BETA, 12, start=su3.SU3_HOT, precision=prec, decomp=decomp) as b:
            a.set_heatbath(max_tries)
            b.set_heatbath(max_tries)
            pa = a.sweep_measured(3)
            pb = b.sweep_measured(3)
            assert np.array_equal(a.get_links(), b.get_links())
            assert np.abs(pa - pb).max() < 1e-13
            assert abs(pb[-1] - b.plaquette()) < tol
            a.set_stats(True)
            b.set_stats(True)
            a.sweep(1)
            b.sweep(1)
            assert a.stats() == b.stats()
            assert np.array_equal(a.get_links(), b.get_links())


def test_decomposed_measured_and_repeat_match_oracle():
    L = (4, 8, 4, 4)
    U0 = oracle.hot_start(L, 3)
    for max_tries in (1, 5):
        O = U0.copy()
        stats, plaq = oracle.sweep(L, BETA, 9, 0, 2, O, max_tries=max_tries)
        with su3.Lattice(L, BETA, 9, start=su3.SU3_COLD, decomp=(2, 2, 1)) as lat:
            lat.set_links(U0)
            lat.set_heatbath(max_tries)
            got = lat.sweep_measured(2)
            assert np.abs(lat.get_links() - O).max() < 1e-12
            assert np.abs(got - plaq).max() < 1e-13


def test_full_size_32x4_sixteen_sublattices():
    # the 32^4 column of Table 1 cut like its np = 16 row (ndmpi 4, mpifactor 2)
    L = (32, 32, 32, 32)
    with su3.Lattice(L, BETA, 7, start=su3.SU3_HOT) as a:
        a.sweep(2)
        ref, pa = a.get_links(), a.plaquette()
    with su3.Lattice(L, BETA, 7, start=su3.SU3_HOT, decomp=(4, 2, 1)) as b:
        b.sweep(2)
        assert np.array_equal(b.get_links(), ref)
        assert b.plaquette() == pa
