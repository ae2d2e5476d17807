"""spm_assemble_csc_static: assembly for callers that cannot allocate.

spm_assemble_csc needs a device workspace from its caller.  A caller that is
not allowed to allocate device memory -- code living inside a host
application that owns every device allocation and passes it only inputs and
outputs, or a loop that must not allocate once running -- has no way to
provide one.  spm_assemble_csc_static runs the same assembly on a scratch
array that is compiled into the library, so the call allocates nothing.

These tests call it through the C ABI twice in a row, on inputs of different
sizes and modes (the second call finds the first call's leftovers in the
shared scratch), and compare each result with spm_assemble_csc on the same
inputs.  Sizes too large for the scratch must be refused before any launch.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import workloads
from tests.gpu_helpers import to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()


def _static_call(d, mode):
    """Outputs come from the test (it may allocate); the call under test does not."""
    import paper_1805_03380_gb300 as spm
    rows, cols, vals = to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"])
    m = rows.numel()
    dev = vals.device
    col_ptr = torch.full((d["shape"][1] + 1,), -7, dtype=torch.int64, device=dev)
    row_idx = torch.full((max(m, 1),), -7, dtype=torch.int32, device=dev)
    out_vals = torch.full((max(m, 1),), 123.0, dtype=vals.dtype, device=dev)
    d_nnz = torch.full((1,), -1, dtype=torch.int64, device=dev)
    d_status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    spm.spm_assemble_csc_static(d["shape"][0], d["shape"][1], rows, cols, vals, None, mode, 0, col_ptr, row_idx,
                                out_vals, d_nnz, None, d_status)
    torch.cuda.synchronize()
    assert int(d_status.item()) == 0
    k = int(d_nnz.item())
    return col_ptr.cpu().numpy(), row_idx[:k].cpu().numpy(), out_vals[:k].cpu().numpy()


def _regular_call(d, mode):
    import paper_1805_03380_gb300 as spm
    A = spm.assemble_csc(to_dev(d["rows"]), to_dev(d["cols"]), to_dev(d["vals"]), d["shape"], mode=mode)
    return A.col_ptr.cpu().numpy(), A.row_idx.cpu().numpy(), A.vals.cpu().numpy()


def _compare(got, want, dtype):
    # the same kernels on the same input: the same bytes
    np.testing.assert_array_equal(got[0], want[0])
    np.testing.assert_array_equal(got[1], want[1])
    assert got[2].dtype == want[2].dtype == dtype
    assert got[2].tobytes() == want[2].tobytes()


def test_static_scratch_matches_workspace_call_twice_in_a_row():
    first = workloads.zipf_batch(m=300_001, n=20_000, seed=workloads.SEED_BASE + 90)
    second = workloads.last_write_1000()
    for d, mode in ((first, "sum"), (second, "set")):
        _compare(_static_call(d, mode), _regular_call(d, mode), np.asarray(d["vals"]).dtype)


def test_static_scratch_refuses_sizes_beyond_its_capacity():
    import paper_1805_03380_gb300 as spm
    dev = torch.device("cuda")
    m = 4_000_000  # needs about 80 MB of workspace, more than the 32 MiB scratch
    rows = torch.zeros(m, dtype=torch.int32, device=dev)
    vals = torch.zeros(m, dtype=torch.float64, device=dev)
    col_ptr = torch.zeros(11, dtype=torch.int64, device=dev)
    d_nnz = torch.zeros(1, dtype=torch.int64, device=dev)
    d_status = torch.zeros(1, dtype=torch.int32, device=dev)
    with pytest.raises(spm.SpmError) as e:
        spm.spm_assemble_csc_static(10, 10, rows, rows, vals, None, "sum", 0, col_ptr, rows, vals, d_nnz, None,
                                    d_status)
    assert e.value.code == 3
