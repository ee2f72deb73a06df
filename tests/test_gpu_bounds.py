"""The bounds-checked build (libsu3_bounds.so, -DSU3_BOUNDS_CHECK): every link
load and store of every kernel checks its direction, parity and index against
the extent of the store it addresses -- the single lattice, one replica of a
batch, one sublattice's extended box -- and records, never traps, an access
out of range.  The decomposed, batched and single-lattice parity cases, and
the persistent and chained schedules, run through it in a separate process; no access may be out of range, and the
results must equal those of the product build (the checks change no
arithmetic)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_0904_1179_gb300 as su3
from paper_0904_1179_gb300 import build as su3_build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r'''
import json, sys
import numpy as np
sys.path.insert(0, %(root)r)
import paper_0904_1179_gb300 as su3
su3.use_library(%(lib)r)
try:
    su3.su3_bounds_status(clear=True)
    checked = True
except su3.Su3Error:  # the product build has no checks compiled in
    checked = False
out = {}
P = [su3.SU3_FP64, su3.SU3_FP32_MIXED, su3.SU3_FP32_EFT]
# single lattices: site-paired and single-site FP32 layouts, ragged tails, both lane forms
for L in [(4, 4, 4, 4), (6, 4, 10, 8), (10, 14, 6, 10), (2, 2, 2, 2), (8, 8, 8, 16)]:
    for prec in P:
        with su3.Lattice(L, 5.7, 3, start=su3.SU3_HOT, precision=prec) as lat:
            for lanes in (0, 1, 4):
                lat.set_lanes(lanes)
                lat.sweep(1)
            lat.set_heatbath(3)
            lat.sweep_measured(1)
            lat.set_heatbath(1)
            lat.set_block_size(64)
            lat.sweep(1)
            U = lat.get_links()
            lat.set_links(U)
            out["plain %%s %%d" %% (L, prec)] = lat.plaquette()
# the persistent and chained schedules (one lane per link; 8 x3 layers of the
# pair lattice, or 16 of the FP64 lattice, in tiles of 64)
for prec in P:
    with su3.Lattice((8, 8, 8, 16), 5.7, 4, start=su3.SU3_HOT, precision=prec) as lat:
        lat.set_lanes(1)
        lat.set_block_size(64)
        scheds = [su3.SU3_SCHED_CHAINED, su3.SU3_SCHED_PER_DIRECTION]
        if prec != su3.SU3_FP64:
            scheds.append(su3.SU3_SCHED_PERSISTENT)
        for sched in scheds:
            lat.set_schedule(sched)
            lat.sweep(1)
        out["schedules %%d" %% prec] = lat.plaquette()
# decomposed lattices, every sublattice and ghost layer
for dec in [(1, 2, 1), (2, 2, 1), (3, 2, 1), (4, 2, 1), (2, 4, 1), (1, 1, 0)]:
    for prec in P:
        L = (8, 8, 8, 8) if dec != (2, 4, 1) else (16, 16, 8, 8)
        with su3.Lattice(L, 5.7, 5, start=su3.SU3_HOT, precision=prec, decomp=dec) as lat:
            lat.sweep(2)
            lat.sweep_measured(1)
            lat.set_heatbath(4)
            lat.sweep(1)
            out["decomp %%s %%d" %% (dec, prec)] = lat.plaquette()
# batches of uneven replicas
dims = [(8, 8, 8, 8), (12, 12, 12, 12), (8, 8, 8, 16), (6, 4, 10, 8), (4, 4, 4, 6)]
for prec in P:
    with su3.Batch(dims, [5.5, 5.7, 5.9, 6.0, 6.1], [11, 12, 13, 14, 15], start=su3.SU3_HOT, precision=prec) as b:
        for cfg in [(128, 0, 0), (64, 2, 2), (256, 1, 1)]:
            b.config(*cfg)
            b.sweep(1)
        b.set_heatbath(3)
        b.sweep(1)
        out["batch %%d" %% prec] = [float(x) for x in b.plaquettes()]
out["status"] = su3.su3_bounds_status() if checked else None
print(json.dumps(out))
'''


def run_checked_cases(lib):
    code = SCRIPT % {"root": ROOT, "lib": lib}
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_bounds_checked_build_sees_no_access_out_of_range():
    lib = su3_build.build(bounds_check=True)
    checked = run_checked_cases(lib)
    assert checked.pop("status") == 0
    product = run_checked_cases(su3_build.build())
    assert product.pop("status") is None
    assert checked == product  # the checks change no result
