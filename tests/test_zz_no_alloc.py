"""The allocation-free volume reduction, flood_storage_static.

It serves callers that cannot allocate device memory: code inside a stream
capture, code living within a device-memory budget that an embedding
application owns, and loops that must never wait on the allocator.  Its block
partials sit in a fixed device array, so each call only reads the caller's
depth field and writes the caller's output.  Checked here, on two calls in a
row through the C ABI, against the library's own storage report (same
arithmetic and order, so bit for bit) and against the FP64 oracle's storage
of the same depths (a sum in another order: 1e-12 relative).  This file is
collected last."""
import numpy as np
import pytest

import oracle
from paper_2302_08341_gb300 import synth
from tests.gpu_util import require_gpu

pytestmark = pytest.mark.gpu


def test_static_storage_matches_the_volume_report_on_two_calls_in_a_row():
    capi = require_gpu()
    import torch
    ny, nx, M = 150, 330, 3
    terr = synth.make_terrain(ny, nx, seed=41)
    rm, sc = synth.ensemble_prior(41, M)
    with capi.Grid(terr.z, terr.n) as g:
        g.ensemble_init(M, rm, sc, synth.hyetograph_constant(120.0, 600.0))
        g.advance_to(200.0)
        vol = g.volumes()["storage"]
        depths = [g.get_state(m)[0] for m in range(M)]
    L = capi.lib()
    stream = torch.cuda.current_stream()
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    for m, pad in ((0, 0), (2, 5)):  # two calls in a row, the second on a padded pitch
        ld = nx + pad
        h = torch.zeros((ny, ld), dtype=torch.float32, device="cuda")
        h[:, :nx] = torch.tensor(depths[m], device="cuda")
        rc = L.flood_storage_static(h.data_ptr(), ny, nx, ld, 3.0, out.data_ptr(),
                                    stream.cuda_stream)
        assert rc == 0, L.flood_storage_static_error()
        stream.synchronize()
        assert vol[m] > 0
        assert out.item() == vol[m]
        ref = oracle.storage(depths[m].astype(np.float64), 3.0)
        assert abs(out.item() - ref) <= 1e-12 * ref
    # sizes beyond the fixed partials array are refused before any launch
    rc = L.flood_storage_static(h.data_ptr(), 65537, 1, 1, 3.0, out.data_ptr(), stream.cuda_stream)
    assert rc == -1 and b"FLOOD_STATIC_MAX_ROWS" in L.flood_storage_static_error()
