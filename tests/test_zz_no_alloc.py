"""su3_plaquette_noalloc: the plaquette for callers that cannot allocate device
memory (for example code running under CUDA stream capture, or runtimes that
only hand out memory from their own pool).  The entry point keeps its scratch
in a fixed device array instead of allocating; this test checks, through the C
ABI, that it returns what the allocating su3_plaquette returns and what the
oracle computes for the same configuration, on two calls in a row.  The file
is named to be collected last."""
import numpy as np
import pytest

import oracle
import paper_0904_1179_gb300 as su3
from paper_0904_1179_gb300 import build as su3_build

pytestmark = pytest.mark.gpu


def device_layout(U, L, precision):
    """Canonical host links -> the library's device layout (index permutation only)."""
    V = int(np.prod(L))
    flat = U.reshape(V, 4, 3, 3, 2)
    x = np.indices((L[3], L[2], L[1], L[0])).reshape(4, -1)
    parity = (x.sum(axis=0) % 2).astype(bool)
    if precision == su3.SU3_FP64:
        soa = np.empty((4, 2, 9, V // 2, 2), dtype=np.float64)
        for p in (0, 1):
            sel = flat[parity == bool(p)].reshape(V // 2, 4, 9, 2)
            soa[:, p] = sel.transpose(1, 2, 0, 3)
    elif L[3] % 4 == 0:
        # site pairs (h, h + V/4): entry e = 3 row + col of pair j holds
        # (re u(h), re u(h + V/4), im u(h), im u(h + V/4)); pairs in tiles of
        # 32 (the last one padded), a tile's six entries one after another
        Vp = V // 4
        nt = (Vp + 31) // 32
        soa = np.zeros((4, 2, nt, 6, 32, 4), dtype=np.float32)
        for p in (0, 1):
            rows01 = flat[parity == bool(p)][:, :, :2]  # (h, mu, row, col, re/im)
            a, b = rows01[:Vp], rows01[Vp:]
            quad = np.stack([a[..., 0], b[..., 0], a[..., 1], b[..., 1]], axis=-1)  # (j, mu, row, col, 4)
            ent = np.zeros((nt * 32, 4, 6, 4), dtype=np.float32)
            ent[:Vp] = quad.reshape(Vp, 4, 6, 4)
            soa[:, p] = ent.reshape(nt, 32, 4, 6, 4).transpose(2, 0, 3, 1, 4)
    else:
        soa = np.empty((4, 2, 3, V // 2, 4), dtype=np.float32)
        for p in (0, 1):
            rows01 = flat[parity == bool(p)][:, :, :2]  # (h, mu, row, col, re/im)
            # column k -> (re u0k, re u1k, im u0k, im u1k)
            soa[:, p] = rows01.transpose(1, 3, 0, 4, 2).reshape(4, 3, V // 2, 4).astype(np.float32)
    return np.ascontiguousarray(soa)


# tolerances against the allocating entry point (same kernels, same order:
# equal up to the summation of the partials) and against the oracle (FP64:
# rounding order; FP32 stores: the FP32 rounding of the plaquette products,
# ~1e-7 per plaquette)
# (8, 6, 4, 10): FP32 stores one site per column group; (8, 6, 4, 8) and
# (6, 6, 6, 4): L3 a multiple of 4, FP32 stores site pairs (384 pairs per
# (mu, parity): twelve whole tiles; 216: the last tile padded)
@pytest.mark.parametrize("L", [(8, 6, 4, 10), (8, 6, 4, 8), (6, 6, 6, 4)])
@pytest.mark.parametrize("precision,tol,tol_oracle", [(su3.SU3_FP64, 1e-13, 1e-13),
                                                      (su3.SU3_FP32_MIXED, 1e-12, 2e-6),
                                                      (su3.SU3_FP32_EFT, 1e-12, 2e-6)])
def test_noalloc_plaquette_matches_allocating_entry_point(L, precision, tol, tol_oracle):
    torch = pytest.importorskip("torch")
    su3_build.build()
    oracle.build()
    stream = torch.cuda.current_stream()
    out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    expect = []
    with su3.Lattice(L, 5.7, 12, start=su3.SU3_HOT, precision=precision) as lat:
        for call in range(2):  # two calls in a row, on two different configurations
            lat.sweep(2)
            expect.append(lat.plaquette())
            U = lat.get_links()
            dev = torch.from_numpy(device_layout(U, L, precision)).cuda()
            su3.su3_plaquette_noalloc(dev.data_ptr(), L, precision, out[call:].data_ptr(), stream.cuda_stream)
            torch.cuda.synchronize()
            got = out[call].item()
            assert abs(got - expect[call]) < tol, (call, got, expect[call])
            ref = oracle.plaquette(L, U, f32=precision != su3.SU3_FP64)
            assert abs(got - ref) < tol_oracle, (call, got, ref)
    assert expect[0] != expect[1]


def test_noalloc_rejects_oversized_lattice():
    torch = pytest.importorskip("torch")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    links = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(su3.Su3Error) as e:
        su3.su3_plaquette_noalloc(links.data_ptr(), (66, 64, 64, 64), su3.SU3_FP64, out.data_ptr())
    assert e.value.code == -5 and "64^4" in str(e.value)
    # extents whose product overflows 64-bit integers are rejected the same way
    with pytest.raises(su3.Su3Error) as e:
        su3.su3_plaquette_noalloc(links.data_ptr(), (1 << 30, 1 << 30, 1 << 30, 1 << 30), su3.SU3_FP32_EFT,
                                  out.data_ptr())
    assert e.value.code == -5
