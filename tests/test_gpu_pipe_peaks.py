"""The pipe microbenchmarks behind the roofline denominators: rates that a
GB300-class device can reach (between a fifth and one and a half times the
nominal issue rate at its maximum clock: FP32 FMA 128 and the XU 16 lane
operations a clock per SM), and the expected ordering of the pipes."""
import pytest

pytestmark = pytest.mark.gpu


def test_pipe_rates_are_plausible():
    import torch
    from paper_2508_05773_gb300 import build as native_build
    native_build.build()
    import paper_2508_05773_gb300 as pkg
    pkg.load()
    props = torch.cuda.get_device_properties(0)
    sms = props.multi_processor_count
    clk_hz = 2.07e9  # upper bound of the SM clock on this class of device
    fma, t = pkg.brmppi_measure_pipe(pkg.PIPE_FMA, 20000)
    xu, _ = pkg.brmppi_measure_pipe(pkg.PIPE_XU, 4000)
    imad, _ = pkg.brmppi_measure_pipe(pkg.PIPE_IMAD, 10000)
    nominal_fma = 128 * sms * clk_hz
    assert 0.2 * nominal_fma < fma < 1.5 * nominal_fma, (fma, nominal_fma)
    assert 0.2 * 16 * sms * clk_hz < xu < 1.5 * 16 * sms * clk_hz, xu
    assert xu < fma and imad <= 1.05 * fma
    assert t > 0
    with pytest.raises(pkg.BrmppiError):
        pkg.brmppi_measure_pipe(7, 10)
