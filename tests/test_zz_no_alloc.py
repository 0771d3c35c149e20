"""The allocation-free count (kc_count_dag_noalloc) against kc_count.

kc_count_dag_noalloc serves callers that cannot allocate device memory when
they count (their own pool allocator holds the GPU's memory, or allocation
would stall a latency-bound loop): its scratch is a fixed array inside the
library and the caller passes the DAG in device memory.  Counts are exact
integers, so the bar is equality with the existing entry point, on two calls
in a row (the array keeps the previous call's contents, which must not leak
into the next result).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
from paper_2502_00317_gb300 import graphgen as gg
from paper_2502_00317_gb300 import kclique as kc

pytestmark = pytest.mark.gpu


def _device_dag(ctx, h):
    import torch

    _, _, orow, ocol = ctx.export_dag(h)
    d_orow = torch.from_numpy(orow.astype(np.uint64).view(np.int64)).cuda()
    d_ocol = torch.from_numpy(np.ascontiguousarray(ocol, dtype=np.uint32).view(np.int32)).cuda()
    if d_ocol.numel() == 0:
        d_ocol = torch.zeros(1, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    return d_orow, d_ocol


def test_noalloc_count_matches_kc_count():
    # 200,000 vertices: more than one binning pass of 131,072 roots
    graphs = [gg.chung_lu_planted(n=200_000, n_cliques=100, seed=3), gg.complete(40), gg.er_gnp(400, 0.3, 12)]
    with kc.Context(0) as ctx:
        for g in graphs:
            h = ctx.upload_host(g.n, g.rowptr, g.col)
            d_orow, d_ocol = _device_dag(ctx, h)
            for k in (1, 2, 3, 4, 5, 6, 7):
                want = ctx.count(h, k)
                first = kc.kc_count_dag_noalloc(g.n, d_orow, d_ocol, k)
                second = kc.kc_count_dag_noalloc(g.n, d_orow, d_ocol, k)
                assert first == second == want, (g.n, k, first, second, want)
            ctx.free(h)
    assert kc.kc_count_dag_noalloc(40, *_complete_dag(40), 5) == oracle.binom(40, 5)


def _complete_dag(n):
    import torch

    orow = np.array([n * r - r * (r + 1) // 2 for r in range(n + 1)], dtype=np.uint64)
    ocol = np.concatenate([np.arange(r + 1, n, dtype=np.uint32) for r in range(n)])
    return (torch.from_numpy(orow.view(np.int64)).cuda(), torch.from_numpy(ocol.view(np.int32)).cuda())


def test_noalloc_limits_and_invalid_dag():
    # out-degree 299 > 256: refused, nothing counted
    with pytest.raises(kc.KcError) as e:
        kc.kc_count_dag_noalloc(300, *_complete_dag(300), 4)
    assert e.value.status == kc.KC_E_UNSUPPORTED
    # an entry outside [row + 1, n): refused by the device-side check
    import torch

    orow = torch.tensor([0, 2, 3, 3], dtype=torch.int64, device="cuda")
    ocol = torch.tensor([1, 9, 2], dtype=torch.int32, device="cuda")
    with pytest.raises(kc.KcError) as e:
        kc.kc_count_dag_noalloc(3, orow, ocol, 3)
    assert e.value.status == kc.KC_E_INVALID_GRAPH
    with pytest.raises(kc.KcError) as e:
        kc.kc_count_dag_noalloc(3, orow, ocol, 0)
    assert e.value.status == kc.KC_E_INVALID_ARG
    # still usable afterwards, twice in a row
    assert kc.kc_count_dag_noalloc(40, *_complete_dag(40), 6) == oracle.binom(40, 6)
    assert kc.kc_count_dag_noalloc(40, *_complete_dag(40), 6) == oracle.binom(40, 6)
