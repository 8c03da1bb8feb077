"""The FP32 FMA-rate measurement behind the compositing kernels' ALU roofline: it counts what it runs
(8 chains x 16 FMAs x iterations per thread, FMA = 2 operations), scales linearly with the work, and
lands below the nominal issue rate (SMs x 128 lanes x 2 x 2.1 GHz) and above a third of it (the SM clock
under load can sit well below its maximum)."""
import pytest

pytestmark = pytest.mark.gpu


def test_fma_rate_is_counted_and_plausible(dv):
    import torch
    props = torch.cuda.get_device_properties(0)
    f1, ms1 = dv.dv_measure_fp32_fma(0, 2048, 10)
    f2, ms2 = dv.dv_measure_fp32_fma(0, 4096, 10)
    assert f2 == pytest.approx(2 * f1)
    n_blocks = props.multi_processor_count * 8
    assert f1 == pytest.approx(2.0 * 8 * 16 * 2048 * n_blocks * 256 * 10)
    rate = f2 / (ms2 * 1e-3)
    nominal = props.multi_processor_count * 128 * 2 * 2.1e9   # 2.1 GHz: at or above this part's maximum SM clock
    assert nominal / 3 < rate < 1.05 * nominal, (rate / 1e12, nominal / 1e12)
    assert ms2 > ms1
