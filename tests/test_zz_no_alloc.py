"""The evaluation entry point that allocates no device memory.

Some callers cannot call cudaMalloc (a plug-in whose process gives all free
device memory to another allocator, code under a fixed device-memory budget,
a latency-critical loop that cannot take an allocation's implicit
synchronisation). mocd_evaluate_noalloc serves them with a fixed scratch array
compiled into the library. This test calls it through the C ABI on device
buffers and checks it against the allocating entry point mocd_evaluate, bit
for bit, on two calls in a row (the second with a different size, so stale
scratch from the first call would show up), and against the CPU oracle."""
import numpy as np
import pytest

import oracle
import paper_2506_01752_gb300 as mocd
import synth

pytestmark = pytest.mark.gpu


def _node_major(lab):
    count, n = lab.shape
    W = (count + 3) // 4 * 4
    out = np.zeros((n, W), dtype=np.int32)
    out[:, :count] = lab.T
    return out


def test_noalloc_matches_evaluate_on_two_calls():
    import torch

    mocd.build.build()
    mocd.load()
    dev = torch.device("cuda", 0)
    rp, ci, _ = synth.workload("lfr-40k", seed=0)
    n = rp.size - 1
    d_rp = torch.from_numpy(rp.astype(np.int32)).to(dev)
    d_ci = torch.from_numpy(ci).to(dev)
    ctx = mocd.graph_upload(rp, ci)
    try:
        cases = [(100, 1, None), (37, 2, 500)]  # 100 x 40,000 = 4.0M cells: within the limit
        free_before = None
        for call, (count, seed, nd) in enumerate(cases):
            lab = synth.random_labels(n, count, seed, n_distinct=nd)
            d_lab = torch.from_numpy(_node_major(lab)).to(dev)
            d_intra = torch.full((count,), -1, dtype=torch.int64, device=dev)
            d_sumsq = torch.full((count,), -1, dtype=torch.int64, device=dev)
            torch.cuda.synchronize()
            if call == 1:
                free_before = torch.cuda.mem_get_info(dev)[0]
            stream = torch.cuda.current_stream(dev)
            mocd.evaluate_noalloc(d_rp.data_ptr(), d_ci.data_ptr(), n, d_lab.data_ptr(), count,
                                  d_intra.data_ptr(), d_sumsq.data_ptr(), stream)
            torch.cuda.synchronize()
            if call == 1:
                assert torch.cuda.mem_get_info(dev)[0] == free_before  # nothing allocated
            ref_intra, ref_sumsq = mocd.evaluate(ctx, lab)
            assert np.array_equal(d_intra.cpu().numpy(), ref_intra)
            assert np.array_equal(d_sumsq.cpu().numpy(), ref_sumsq)
            # and directly against the CPU oracle's exact objectives
            orc_intra, orc_sumsq = oracle.objectives(rp, ci, lab)
            assert np.array_equal(d_intra.cpu().numpy(), orc_intra)
            assert np.array_equal(d_sumsq.cpu().numpy(), orc_sumsq)
    finally:
        mocd.destroy(ctx)


def test_noalloc_rejects_sizes_beyond_the_scratch():
    import torch

    mocd.load()
    dev = torch.device("cuda", 0)
    n = mocd.NOALLOC_MAX_CELLS // 100 + 1
    dummy = torch.zeros(16, dtype=torch.int64, device=dev)
    with pytest.raises(mocd.MocdError) as e:
        mocd.evaluate_noalloc(dummy.data_ptr(), dummy.data_ptr(), n, dummy.data_ptr(), 100,
                              dummy.data_ptr(), dummy.data_ptr())
    assert e.value.status == -10
    with pytest.raises(mocd.MocdError) as e:
        mocd.evaluate_noalloc(dummy.data_ptr(), dummy.data_ptr(), 10, dummy.data_ptr(), 129,
                              dummy.data_ptr(), dummy.data_ptr())
    assert e.value.status == -1
