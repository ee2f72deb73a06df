"""The persistent sweeps (su3_set_schedule: one kernel per sweep, or one per
direction; FP64 one per direction) against the eight half-sweep kernels and
against the oracle.

The persistent kernel applies the per-link update of the half-sweep kernels to
the same inputs: a tile of a half-sweep starts only after the previous
half-sweep has finished every tile whose links its staples read or whose
staples read its links.  Its results are therefore compared bit for bit with
the eight-kernel schedule (itself pinned to the oracle half-sweep by
half-sweep in test_gpu_parity.py), and one full sweep also goes to the
oracle's FP32 reading directly.
"""
import numpy as np
import pytest

import oracle
import paper_0904_1179_gb300 as su3
from paper_0904_1179_gb300 import build as su3_build

pytestmark = pytest.mark.gpu

BETA = 5.7
F32_TOL = 5e-5
PRECS = [su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT]


@pytest.fixture(scope="module", autouse=True)
def built():
    su3_build.build()
    oracle.build()


SCHEDS = [su3.SU3_SCHED_PERSISTENT, su3.SU3_SCHED_PER_DIRECTION, su3.SU3_SCHED_CHAINED]


def pair(L, prec, seed, lanes=0, threads=0, schedule=su3.SU3_SCHED_PERSISTENT):
    """Two identical lattices, the first on a persistent schedule, the second on eight kernels."""
    a = su3.Lattice(L, BETA, seed, start=su3.SU3_HOT, precision=prec)
    b = su3.Lattice(L, BETA, seed, start=su3.SU3_HOT, precision=prec)
    for lat in (a, b):
        if lanes:
            lat.set_lanes(lanes)
        if threads:
            lat.set_block_size(threads)
    a.set_schedule(schedule)
    b.set_schedule(su3.SU3_SCHED_PHASES)
    assert a.schedule == schedule
    assert b.schedule == su3.SU3_SCHED_PHASES
    return a, b


# 8^4 (one lane per pair forced; 4 layers of 8 tiles of 32), 12^3 x 16
# (8 layers of 27 tiles of 32), 16^4 (8 layers of 32 tiles of 64), 32^4 (the
# bench lattice: 16 layers of 128 tiles of 128).
@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("L,lanes", [((8, 8, 8, 8), 1), ((12, 12, 12, 16), 0), ((16, 16, 16, 16), 0),
                                     ((32, 32, 32, 32), 0)])
def test_persistent_sweep_equals_eight_kernels(L, lanes, prec, sched):
    a, b = pair(L, prec, 21, lanes=lanes, schedule=sched)
    with a, b:
        for lat in (a, b):
            lat.set_stats(True)
            lat.sweep(3)
            lat.status()
        assert np.array_equal(a.get_links(), b.get_links())
        assert a.stats() == b.stats()
        assert a.sweep_count == b.sweep_count == 3


# FP64, one launch per direction: 8^3 x 4 (4 layers of 2 tiles of 128),
# 12^3 x 8 (8 layers of 864 sites: 27 tiles of 32), 16^4, 32^4 (the bench
# lattice: 32 layers of 128 tiles of 128); one thread per link (the
# four-lane form of the smallest lattices is switched off).
@pytest.mark.parametrize("sched", [su3.SU3_SCHED_PER_DIRECTION, su3.SU3_SCHED_CHAINED])
@pytest.mark.parametrize("L,threads", [((8, 8, 8, 4), 128), ((12, 12, 12, 8), 32), ((16, 16, 16, 16), 0),
                                       ((32, 32, 32, 32), 0)])
def test_fp64_per_direction_equals_eight_kernels(L, threads, sched):
    a, b = pair(L, su3.SU3_FP64, 23, lanes=1, threads=threads, schedule=sched)
    with a, b:
        for lat in (a, b):
            lat.set_stats(True)
            lat.sweep(3)
            lat.status()
        assert np.array_equal(a.get_links(), b.get_links())
        assert a.stats() == b.stats()


def test_fp64_per_direction_matches_oracle():
    L = (8, 8, 8, 8)
    with su3.Lattice(L, BETA, 31, start=su3.SU3_HOT, precision=su3.SU3_FP64) as lat:
        lat.set_lanes(1)
        lat.set_block_size(64)
        lat.set_schedule(su3.SU3_SCHED_PER_DIRECTION)
        U0 = lat.get_links()
        lat.sweep(1)
        U1 = lat.get_links()
    oracle.sweep(L, BETA, 31, 0, 1, U0)  # in place: sweep t = 0 of the same chain
    assert np.abs(U1 - U0).max() < 1e-12


@pytest.mark.parametrize("prec", PRECS)
def test_persistent_block_sizes(prec):
    L = (16, 16, 16, 16)
    ref = None
    for threads in (32, 64, 128, 256):
        a, b = pair(L, prec, 5, threads=threads)
        with a, b:
            a.sweep(2)
            b.sweep(2)
            Ua = a.get_links()
            assert np.array_equal(Ua, b.get_links()), threads
        if ref is None:
            ref = Ua
        assert np.array_equal(Ua, ref), threads


# Measuring sweeps run the eight half-sweep kernels whatever the schedule;
# persistent and measuring sweeps interleaved give the same chain.
@pytest.mark.parametrize("prec", PRECS)
def test_persistent_and_measured_sweeps_interleave(prec):
    L = (16, 16, 16, 16)
    a, b = pair(L, prec, 8)
    with a, b:
        for lat in (a, b):
            lat.sweep(2)
        pa = a.sweep_measured(3)
        pb = b.sweep_measured(3)
        for lat in (a, b):
            lat.sweep(1)
        assert np.array_equal(pa, pb)
        assert np.array_equal(a.get_links(), b.get_links())
        assert a.sweep_count == b.sweep_count == 6


@pytest.mark.parametrize("sched", SCHEDS)
@pytest.mark.parametrize("prec", PRECS)
def test_persistent_repeat_until_accepted_equals_eight_kernels(prec, sched):
    L = (12, 12, 12, 16)
    a, b = pair(L, prec, 14, schedule=sched)
    with a, b:
        for lat in (a, b):
            lat.set_heatbath(8)
            lat.set_stats(True)
            lat.sweep(2)
        assert np.array_equal(a.get_links(), b.get_links())
        assert a.stats() == b.stats()


# One full persistent sweep against the oracle's FP32 reading.  A one-hit
# decision taken within FP32 rounding of its threshold may flip (see the
# half-sweep tests); inside a full sweep such a flip also moves the later
# updates that read the flipped link, a few dozen links at most, so all but a
# small fraction of links must agree to 5e-5.
@pytest.mark.parametrize("prec", PRECS)
def test_persistent_sweep_matches_oracle_reading(prec):
    L = (8, 8, 8, 8)
    seed, t = 33, 4
    U0 = oracle.hot_start(L, 19, f32=True)
    oracle.sweep(L, BETA, 6, 0, 1, U0, f32=True)
    O = U0.copy()
    oracle.sweep(L, BETA, seed, t, 1, O, f32=True)
    with su3.Lattice(L, BETA, seed, start=su3.SU3_COLD, precision=prec) as lat:
        lat.set_lanes(1)
        lat.set_schedule(su3.SU3_SCHED_PERSISTENT)
        lat.set_links(U0)
        lat.sweep_count = t
        lat.sweep(1)
        G = lat.get_links()
    d = np.abs(G - O).max(axis=(-1, -2, -3))
    off = int((d > F32_TOL).sum())
    assert off <= d.size // 100, (off, d.size)
    print("persistent FP32 sweep (precision %d) vs oracle: worst |dU| %.2e over %d links, %d beyond 5e-5"
          % (prec, float(np.sort(d.ravel())[d.size - off - 1]), d.size, off))


def test_automatic_schedule_follows_the_waves():
    # 16^4: 0.2 waves per half-sweep and 24^3 x 16: 0.7, eight launches;
    # 24^4: 1.1, 32^4: 3.4 and 32^3 x 64: 6.7, the chained half-sweep
    # launches (waves on a GPU of 152 SMs)
    for L, sched in (((16, 16, 16, 16), su3.SU3_SCHED_PHASES), ((24, 24, 24, 16), su3.SU3_SCHED_PHASES),
                     ((24, 24, 24, 24), su3.SU3_SCHED_CHAINED), ((32, 32, 32, 32), su3.SU3_SCHED_CHAINED),
                     ((32, 32, 32, 64), su3.SU3_SCHED_CHAINED)):
        with su3.Lattice(L, BETA, 1, precision=su3.SU3_FP32_MIXED) as lat:
            assert lat.schedule == sched, L
    # FP64 (384 links per SM in flight): 16^4 0.6 waves, 24^4 2.8, 32^4 9.0
    for L, sched in (((16, 16, 16, 16), su3.SU3_SCHED_PHASES), ((24, 24, 24, 24), su3.SU3_SCHED_PER_DIRECTION),
                     ((32, 32, 32, 32), su3.SU3_SCHED_PHASES)):
        with su3.Lattice(L, BETA, 1, precision=su3.SU3_FP64) as lat:
            assert lat.schedule == sched, L


def test_schedule_applies_where_documented():
    # a layer that is not a whole number of blocks (10 x 20 x 20 = 4000
    # pairs, 128 threads), a lattice below 4 layers (L3 = 4), the four-lane
    # kernel: the eight kernels, and both persistent schedules are refused
    for L, prec in (((20, 20, 20, 16), su3.SU3_FP32_MIXED), ((16, 16, 16, 4), su3.SU3_FP32_MIXED),
                    ((8, 8, 8, 8), su3.SU3_FP32_EFT), ((8, 8, 8, 8), su3.SU3_FP64)):
        with su3.Lattice(L, BETA, 1, precision=prec) as lat:
            assert lat.schedule == su3.SU3_SCHED_PHASES, L
            for sched in SCHEDS:
                with pytest.raises(su3.Su3Error) as e:
                    lat.set_schedule(sched)
                assert e.value.code == su3.SU3_EINVAL
    # FP64: per direction or chained half-sweeps, not one launch per sweep
    with su3.Lattice((16, 16, 16, 16), BETA, 1, precision=su3.SU3_FP64) as lat:
        with pytest.raises(su3.Su3Error) as e:
            lat.set_schedule(su3.SU3_SCHED_PERSISTENT)
        assert e.value.code == su3.SU3_EINVAL
        for sched in (su3.SU3_SCHED_PER_DIRECTION, su3.SU3_SCHED_CHAINED):
            lat.set_schedule(sched)
            assert lat.schedule == sched
    with su3.Lattice((16, 16, 16, 16), BETA, 1, precision=su3.SU3_FP32_MIXED) as lat:
        with pytest.raises(su3.Su3Error):
            lat.set_schedule(7)
        lat.set_schedule(su3.SU3_SCHED_PHASES)
        assert lat.schedule == su3.SU3_SCHED_PHASES
        lat.set_schedule(su3.SU3_SCHED_PERSISTENT)
        assert lat.schedule == su3.SU3_SCHED_PERSISTENT
        lat.set_schedule(su3.SU3_SCHED_PER_DIRECTION)
        assert lat.schedule == su3.SU3_SCHED_PER_DIRECTION
        lat.set_schedule(su3.SU3_SCHED_AUTO)
        assert lat.schedule == su3.SU3_SCHED_PHASES  # a fraction of a wave per half-sweep
        with pytest.raises(su3.Su3Error):
            lat.debug(0.0)
    with su3.Batch([(8, 8, 8, 8)], [BETA], [1]) as bt:
        with pytest.raises(su3.Su3Error):
            su3.su3_set_schedule(bt.handle, su3.SU3_SCHED_PHASES)


# Fault detection without a fault: a work item that never reports completion
# makes the waits on it run out (0.2 s), the sweep stops, su3_status reports
# SU3_ETIMEOUT once, and the context keeps working.  Item 0 is the first tile
# of phase 0 (mu = 0, even sites), waited on inside the launch; item 128 (the
# lattice's 16^4 / 4 / 128 = 128 tiles per phase) the first tile of phase 1
# (mu = 0, odd sites), which in the per-direction form is waited on only by
# the next launch, the programmatic dependent launch of mu = 1.
# The chained half-sweep launches number each launch's tiles by block index:
# item 0 is the first tile of every half-sweep, and the wait on it lies in the
# next launch.  FP64: 16^4 / 2 / 128 = 256 tiles per phase, so item 256 is the
# first of phase 1.
@pytest.mark.parametrize("sched,prec,item", [(su3.SU3_SCHED_PERSISTENT, su3.SU3_FP32_MIXED, 0),
                                             (su3.SU3_SCHED_PERSISTENT, su3.SU3_FP32_MIXED, 128),
                                             (su3.SU3_SCHED_PER_DIRECTION, su3.SU3_FP32_MIXED, 0),
                                             (su3.SU3_SCHED_PER_DIRECTION, su3.SU3_FP32_MIXED, 128),
                                             (su3.SU3_SCHED_CHAINED, su3.SU3_FP32_MIXED, 0),
                                             (su3.SU3_SCHED_PER_DIRECTION, su3.SU3_FP64, 0),
                                             (su3.SU3_SCHED_PER_DIRECTION, su3.SU3_FP64, 256),
                                             (su3.SU3_SCHED_CHAINED, su3.SU3_FP64, 0)])
def test_withheld_tile_times_out_without_fault(sched, prec, item):
    L = (16, 16, 16, 16)
    with su3.Lattice(L, BETA, 2, precision=prec) as lat:
        lat.set_block_size(128)
        lat.set_schedule(sched)
        assert lat.schedule == sched
        lat.debug(0.2, withhold_item=item)
        lat.sweep(1)
        with pytest.raises(su3.Su3Error) as e:
            lat.status()
        assert e.value.code == su3.SU3_ETIMEOUT
        lat.status()  # cleared
        lat.debug(2.0, withhold_item=-1)
        lat.sweep(2)
        lat.status()
        assert 0.0 < lat.plaquette() < 1.0
