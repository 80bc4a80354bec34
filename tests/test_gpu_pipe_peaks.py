"""vegas_pipe_peak: each measured pipe rate is positive and, per SM and clock,
inside the band the B300's unit counts allow (a 4-scheduler SM issues at most
128 lane-operations per clock; the float FMA pipes deliver up to 128, the
special-function unit and the shared-memory pipe far fewer), and argument
errors are refused."""
import pytest

import paper_2002_12921_b300 as V

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def peaks():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    V.lib()
    return V.binding.pipe_peaks()


# (lowest plausible, highest possible) lane-operations per SM per clock
BANDS = {"ffma": (64, 130), "dfma": (0.1, 70), "ex2": (4, 40), "product": (8, 70),
         "imad": (16, 130), "lds": (16, 40), "atoms_u32": (4, 40), "atoms_f32": (1, 40)}


@pytest.mark.parametrize("name", V.binding.PIPES)
def test_peak_per_sm_per_clock_is_plausible(peaks, name):
    p = peaks[name]
    assert 500 < p["sm_mhz"] < 2200, p
    lo, hi = BANDS[name]
    assert lo <= p["per_sm_per_clk"] <= hi, (name, p)


def test_float_atomics_are_not_faster_than_integer_ones(peaks):
    assert peaks["atoms_f32"]["per_s"] <= 1.1 * peaks["atoms_u32"]["per_s"]


def test_bad_arguments_are_refused():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    scratch = torch.zeros(64, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    for op, nbytes in ((len(V.binding.PIPES), 64), (-1, 64), (0, 8)):
        with pytest.raises(V.VegasError) as e:
            V.binding.vegas_pipe_peak(op, 0, scratch.data_ptr(), nbytes, st)
        assert e.value.status == V.VEGAS_EINVAL
