"""The roofline ceilings measured on the GPU (smcrt_microbench): FP32 FMA
throughput and int64 atomic rates, through the C-ABI."""
import pytest

import paper_2112_08035_gb300 as smc

pytestmark = pytest.mark.gpu


def test_microbench_ceilings_plausible():
    import torch
    m = smc.microbench(0)
    props = torch.cuda.get_device_properties(0)
    # 128 FP32 lanes per SM, an FMA = 2 flops, clocks between 0.8 and 2.2 GHz
    lo = props.multi_processor_count * 128 * 2 * 0.8e9
    hi = props.multi_processor_count * 128 * 2 * 2.2e9
    assert lo < m["fp32_flops"] < hi, m
    # atomics: scattered targets at least 1e9 per second, 32 hot ones 1e8
    assert m["atomics_distinct_per_s"] > 1e9 and m["atomics_hot_per_s"] > 1e8, m


def test_microbench_rejects_small_scratch():
    import ctypes as C
    import torch
    buf = torch.empty(1024, dtype=torch.int64, device="cuda")
    f, a, h = C.c_double(), C.c_double(), C.c_double()
    rc = smc.lib().smcrt_microbench(0, C.c_void_p(buf.data_ptr()), 8192, C.byref(f), C.byref(a), C.byref(h))
    assert rc == smc.ERR_BAD_ARG
