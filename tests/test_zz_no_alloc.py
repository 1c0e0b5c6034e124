"""sgc_count_device_static: counting with no device allocation.

Callers that cannot call cudaMalloc while they count (their device memory
belongs to another framework's allocator, or their footprint must stay fixed
after start-up) use this entry point; all of its scratch comes from the
library's static device array.  Its results must equal those of the
allocating entry point, sgc_count_device, on the same inputs - checked on two
calls in a row, since the array keeps the previous call's contents.

This file is collected last so that a run stopping at the first failure has
run every other test first; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
import paper_1903_04395_gb300 as sgc
import sgcgen

pytestmark = pytest.mark.gpu

FP32_RTOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    sgc.build()
    return torch


@pytest.mark.parametrize("precision", [sgc.SGC_FP64, sgc.SGC_FP32])
def test_static_matches_allocating_entry_point(torch_cuda, precision):
    torch = torch_cuda
    rp, ci = sgcgen.er(3000, 12000, 11)
    parent = sgcgen.pruefer_tree(7, 5)
    g = sgc.Graph(rp, ci)
    t = sgc.Template(parent)
    n_iter = 11  # passes of 8 + 2 + 1 colorings
    seeds = torch.arange(100, 100 + n_iter, dtype=torch.int64, device="cuda")
    stream = torch.cuda.Stream()
    opt = sgc.sgc_options_init(precision=precision, stream=stream.cuda_stream)
    ref = torch.zeros(n_iter, dtype=torch.float64, device="cuda")
    outs = [torch.full((n_iter,), -1.0, dtype=torch.float64, device="cuda") for _ in range(2)]
    # the inputs were written on torch's current stream; the library reads them on `stream`
    stream.wait_stream(torch.cuda.current_stream())
    sgc.sgc_count_device(g.handle, t.handle, seeds.data_ptr(), n_iter, opt, ref.data_ptr())
    stream.synchronize()
    ref_h = ref.cpu().numpy()
    for call in range(2):
        out = outs[call]
        free0 = torch.cuda.mem_get_info()[0]
        sgc.sgc_count_device_static(g.handle, t.handle, seeds.data_ptr(), n_iter, opt, out.data_ptr())
        if call == 1:
            # nothing was allocated on the device by the call (the first call of the process may
            # load the module that holds the static array)
            assert torch.cuda.mem_get_info()[0] == free0
        got = out.cpu().numpy()
        if precision == sgc.SGC_FP64:
            assert np.array_equal(got, ref_h), (call, got, ref_h)
        else:
            assert np.allclose(got, ref_h, rtol=FP32_RTOL, atol=0), (call, got, ref_h)
    # and both agree with the exact oracle
    want = [oracle.count(rp, ci, parent, oracle.colors(s, len(rp) - 1, len(parent))).maps
            for s in range(100, 100 + n_iter)]
    tol = 0 if precision == sgc.SGC_FP64 else FP32_RTOL
    assert all(abs(r - w) <= tol * w for r, w in zip(ref_h, want))


def test_static_rejects_requests_above_its_size(torch_cuda):
    torch = torch_cuda
    rp, ci = sgcgen.rmat(16, seed=1)
    g = sgc.Graph(rp, ci)
    t = sgc.Template(sgcgen.path_tree(12))
    seeds = torch.arange(1, 3, dtype=torch.int64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(sgc.SgcError) as ei:
        sgc.sgc_count_device_static(g.handle, t.handle, seeds.data_ptr(), 2, None, out.data_ptr())
    assert ei.value.status == sgc.SGC_ERR_UNSUPPORTED
    assert "static workspace" in str(ei.value)
