"""Out-of-core ingest: windows streamed from host memory in batches, two in
flight, give every window's quantities and the time sum of all windows
exactly as the oracle."""
import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("batch_packets,pinned", [(1 << 16, False), (200000, True), (1 << 22, False)])
def test_stream_equals_oracle(batch_packets, pinned):
    from paper_2510_14050_gb300 import stream, synth
    w = synth.generate(5, sizes=[70000, 0, 5000, 131072, 1, 90000, 40000, 300000, 12345, 65536, 8192],
                       first_window=21)
    src, dst = w.src, w.dst
    if pinned:
        src = torch.from_numpy(w.src.view(np.int32)).pin_memory()
        dst = torch.from_numpy(w.dst.view(np.int32)).pin_memory()
    res = stream.stream_windows(src, dst, w.offsets, batch_packets=batch_packets)
    try:
        assert res.batches == len(stream.plan_batches(w.offsets, batch_packets))
        for i in range(w.nwin):
            exp = oracle.window_quantities(*w.window(i))
            assert dict(zip(oracle.QUANTITY_NAMES, (int(v) for v in res.quantities[i]))) == exp, f"window {i}"
        exp_sum = oracle.sum_matrices([oracle.traffic_matrix(*w.window(i)) for i in range(w.nwin)])
        for x, y in zip(res.sum.to_numpy(), exp_sum):
            assert np.array_equal(x, y)
        assert res.sum.quantities() == oracle.network_quantities(exp_sum)
    finally:
        res.sum.free()
