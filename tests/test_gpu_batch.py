"""The batched sweep: many replicas of uneven extents, beta and seed in one
persistent, graph-captured launch per sweep.

Parity: each replica of a batch equals the same lattice run alone (bit for
bit: same update code, same Philox counters keyed by the replica's seed), and
the FP64 batch equals the FP64 oracle link by link to 1e-12.  The dispatch
configuration (tile size, blocks per SM, L2 window) and autotuning change
nothing in the results.  Fault detection: a withheld arrival makes the
bounded waits run out and the call report SU3_ETIMEOUT, with the GPU context
still usable.
"""
import numpy as np
import pytest

import oracle
import paper_0904_1179_gb300 as su3
from paper_0904_1179_gb300 import build as su3_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    su3_build.build()
    oracle.build()


# a small uneven mix: ragged tiles, different extents per direction, different beta
MIX = [(4, 4, 4, 4), (6, 4, 10, 8), (8, 8, 8, 8), (2, 2, 2, 2), (4, 6, 4, 8), (8, 8, 8, 16), (4, 4, 4, 4)]
BETAS = [5.7, 5.5, 6.0, 5.9, 5.6, 6.2, 5.8]
SEEDS = [1000 + r for r in range(len(MIX))]


def config_batch():
    """The 96-replica batch of the benchmark (32x 8^4, 32x 12^4, 16x 16^4, 16x 8^3x16)."""
    from paper_0904_1179_gb300.workloads import batch_96
    return batch_96()


@pytest.mark.parametrize("prec", [su3.SU3_FP64, su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT])
def test_replicas_equal_single_lattices(prec):
    with su3.Batch(MIX, BETAS, SEEDS, start=su3.SU3_HOT, precision=prec) as b:
        b.sweep(3)
        plaq = b.plaquettes()
        assert b.sweep_count == 3
        for r, L in enumerate(MIX):
            with su3.Lattice(L, BETAS[r], SEEDS[r], start=su3.SU3_HOT, precision=prec) as lat:
                lat.sweep(3)
                assert np.array_equal(b.get_links(r), lat.get_links()), r
                assert plaq[r] == lat.plaquette()


def test_fp64_batch_matches_oracle():
    with su3.Batch(MIX, BETAS, SEEDS, start=su3.SU3_COLD, precision=su3.SU3_FP64) as b:
        starts = []
        for r, L in enumerate(MIX):
            U = oracle.hot_start(L, 50 + r)
            b.set_links(r, U)
            starts.append(U)
        b.sweep(2)
        for r, L in enumerate(MIX):
            O = starts[r].copy()
            oracle.sweep(L, BETAS[r], SEEDS[r], 0, 2, O)
            assert np.abs(b.get_links(r) - O).max() < 1e-12, r


@pytest.mark.parametrize("prec", [su3.SU3_FP64, su3.SU3_FP32_MIXED])
def test_dispatch_config_does_not_change_results(prec):
    ref = None
    for threads, bps, window in [(128, 0, 0), (32, 1, 1), (64, 2, 3), (256, 1, 2), (96, 3, 0)]:
        with su3.Batch(MIX, BETAS, SEEDS, start=su3.SU3_HOT, precision=prec) as b:
            b.config(threads, bps, window)
            b.sweep(2)
            got = [b.get_links(r) for r in range(len(MIX))]
        if ref is None:
            ref = got
        for r in range(len(MIX)):
            assert np.array_equal(got[r], ref[r]), (threads, bps, window, r)


def test_autotune_keeps_the_chain_and_is_remembered():
    dims, betas, seeds = config_batch()
    dims, betas, seeds = dims[::8], betas[::8], seeds[::8]  # 12 replicas of the same mix
    with su3.Batch(dims, betas, seeds, start=su3.SU3_HOT) as a:
        a.sweep(1)
        before = [a.get_links(r) for r in range(a.n)]
        cfg = a.autotune()
        assert a.sweep_count == 1
        for r in range(a.n):
            assert np.array_equal(a.get_links(r), before[r])
        a.sweep(2)
        tuned = [a.get_links(r) for r in range(a.n)]
        assert a.get_config() == cfg
    with su3.Batch(dims, betas, seeds, start=su3.SU3_HOT) as b:
        assert b.get_config() == cfg  # remembered for the same replica set
        b.config(128, 0, 0)
        b.sweep(3)
        for r in range(b.n):
            assert np.array_equal(b.get_links(r), tuned[r])


def test_config_batch_runs_and_stays_su3():
    dims, betas, seeds = config_batch()
    with su3.Batch(dims, betas, seeds, start=su3.SU3_HOT) as b:
        b.sweep(5)
        p = np.array(b.plaquettes())
        assert np.all((p > 0.2) & (p < 0.7))
        for r in (0, 40, 70, 90):
            U = b.get_links(r)
            M = (U[..., 0] + 1j * U[..., 1]).reshape(-1, 3, 3)
            assert np.abs(np.einsum("nki,nkj->nij", M.conj(), M) - np.eye(3)).max() < 5e-7


# The sweep runs four launches, one per direction; launch mu numbers its
# items from 0, phase 2 mu of every replica first (window = all replicas).
# Item 0 is the first tile of phase 0 of replica 0, waited on inside launch
# 0; the item after all phase-0 tiles is the first tile of phase 1 of
# replica 0, waited on only by phase 2 in the next launch, a programmatic
# dependent launch.
@pytest.mark.parametrize("cross_launch", [False, True])
def test_withheld_arrival_times_out_without_fault(cross_launch):
    threads = 64
    first_phase1 = sum(-(-(int(np.prod(L)) // 2) // threads) for L in MIX)
    with su3.Batch(MIX, BETAS, SEEDS, start=su3.SU3_HOT) as b:
        b.config(threads, 0, 0)
        b.debug(0.2, withhold_item=first_phase1 if cross_launch else 0)
        b.sweep(1)
        with pytest.raises(su3.Su3Error) as e:
            b.status()
        assert e.value.code == su3.SU3_ETIMEOUT
        b.status()  # the status was cleared; the context still works
        b.debug(2.0, withhold_item=-1)
        b.sweep(1)
        b.status()
        assert len(b.plaquettes()) == len(MIX)
    with su3.Lattice((4, 4, 4, 4), 5.7, 1, start=su3.SU3_COLD) as lat:
        lat.sweep(1)
        assert 0.0 < lat.plaquette() < 1.0


def test_single_calls_reject_batch_handles():
    with su3.Batch(MIX[:2], BETAS[:2], SEEDS[:2]) as b:
        with pytest.raises(su3.Su3Error):
            su3.su3_sweep(b.handle, 1)
        with pytest.raises(su3.Su3Error):
            su3.su3_plaquette(b.handle)
        out = np.empty(su3.links_shape(MIX[0]), dtype=np.float64)
        with pytest.raises(su3.Su3Error):
            su3.su3_batch_links_get(b.handle, 5, out)


def test_batch_repeat_until_accepted_equals_single_lattices():
    with su3.Batch(MIX, BETAS, SEEDS, start=su3.SU3_HOT, precision=su3.SU3_FP32_MIXED) as b:
        b.set_heatbath(4)
        b.sweep(2)
        for r, L in enumerate(MIX):
            with su3.Lattice(L, BETAS[r], SEEDS[r], start=su3.SU3_HOT, precision=su3.SU3_FP32_MIXED) as lat:
                lat.set_heatbath(4)
                lat.sweep(2)
                assert np.array_equal(b.get_links(r), lat.get_links()), r


# More replicas than the kernel parameters carry (200): the descriptors are
# read from global memory; each replica still equals the lattice run alone.
@pytest.mark.parametrize("prec", [su3.SU3_FP32_MIXED, su3.SU3_FP64])
def test_batch_beyond_parameter_descriptors(prec):
    n = 203
    dims = [MIX[r % len(MIX)] for r in range(n)]
    betas = [BETAS[r % len(BETAS)] for r in range(n)]
    seeds = [5000 + r for r in range(n)]
    with su3.Batch(dims, betas, seeds, start=su3.SU3_HOT, precision=prec) as b:
        b.sweep(2)
        b.status()
        for r in (0, 101, 202):
            with su3.Lattice(dims[r], betas[r], seeds[r], start=su3.SU3_HOT, precision=prec) as lat:
                lat.sweep(2)
                assert np.array_equal(b.get_links(r), lat.get_links()), r
