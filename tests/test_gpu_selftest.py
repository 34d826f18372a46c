"""The bounded-wait failure path, exercised on purpose and safely: a wait on
a barrier nothing arrives at must give up after its limit, the workspace
status must read CR_ETIMEOUT, and the context must stay usable (a merge
afterwards is still exact)."""
import numpy as np
import pytest
import torch

import oracle
import paper_1303_4312_gb300 as cr
from paper_1303_4312_gb300 import _lib

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_reports():
    lib = _lib.load()
    ws = torch.zeros(256, dtype=torch.uint8, device="cuda")
    elapsed = torch.zeros(1, dtype=torch.int64, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    limit = 1_000_000                                    # 1 ms
    assert lib.cr_selftest_bounded_wait(ws.data_ptr(), ws.numel(), limit, elapsed.data_ptr(),
                                        s) == 0
    with pytest.raises(cr.CorankError) as e:
        cr.workspace_status(ws)
    assert e.value.name == "CR_ETIMEOUT"
    ns = int(elapsed.item())
    assert limit <= ns < 50 * limit, ns
    # the context is still usable
    rng = np.random.default_rng(500)
    A = np.sort(rng.integers(0, 100, 50000)).astype(np.int32)
    B = np.sort(rng.integers(0, 100, 40000)).astype(np.int32)
    C = cr.merge(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda())
    torch.cuda.synchronize()
    assert np.array_equal(C.cpu().numpy(), oracle.merge(A, B)[0])
