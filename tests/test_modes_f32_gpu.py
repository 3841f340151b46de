"""FP32 state input and output (sfp_set_modes_f32, SFP_OBS_MODES_F32): the same
packed [3][M_c] layout as the FP64 calls at half the host bytes.  The FP32 and
mixed paths keep R_p (p >= 1) in FP32, so their values pass through unchanged;
R_0 = sqrt(M) r_cm goes through the FP64 centre of mass."""
import numpy as np
import pytest

import paper_1411_3487_gb300 as sfp
from oracle import oracle as O
from paper_1411_3487_gb300 import build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def chains(lengths, dtau=10.0):
    return [{"n_beads": M, "dtau": dtau, "job_id": 70 + c} for c, M in enumerate(lengths)]


def starts(lengths, seed=3):
    return [O.Model(M, dtau=10.0).equilibrium_start(seed, 70 + c) for c, M in enumerate(lengths)]


def pinned_f32(n):
    torch = pytest.importorskip("torch")
    return torch.empty(n, dtype=torch.float32, pin_memory=True).numpy()


@pytest.mark.parametrize("precision", [sfp.SFP_MIXED_BF16, sfp.SFP_FP32, sfp.SFP_FP32_SIMT])
@pytest.mark.parametrize("lengths", [[128] * 5, [64, 100, 128, 64, 512, 100]], ids=["one_group", "mixed"])
def test_f32_round_trip_matches_the_fp64_calls(precision, lengths):
    """set_modes_f32 then SFP_OBS_MODES: p >= 1 bit-exact to the FP32 input, R_0
    within FP64 rounding of it; SFP_OBS_MODES_F32 equals the FP32 rounding of
    SFP_OBS_MODES bit for bit."""
    R = starts(lengths)
    R32 = [r.astype(np.float32) for r in R]
    b = sfp.Batch(chains(lengths), seed=1, precision=precision)
    b.set_modes(R32)
    G = b.modes()
    G32 = b.observe(sfp.SFP_OBS_MODES_F32)
    if not isinstance(G, list):
        G, G32 = list(G), list(G32)
    for g, g32, r in zip(G, G32, R32):
        assert g32.dtype == np.float32
        np.testing.assert_array_equal(g[:, 1:], r[:, 1:].astype(np.float64))
        np.testing.assert_allclose(g[:, 0], r[:, 0].astype(np.float64), rtol=1e-14, atol=1e-300)
        np.testing.assert_array_equal(g32, g.astype(np.float32))
    b.close()


@pytest.mark.parametrize("precision", [sfp.SFP_MIXED_BF16, sfp.SFP_FP32])
def test_steps_from_an_f32_start_equal_steps_from_the_same_values_in_fp64(precision):
    """The state a step sees is the same whichever call set it: 40 fused steps
    from set_modes_f32 and from set_modes of the same (FP32-exact) values agree
    bit for bit."""
    lengths = [256] * 9
    R32 = np.stack(starts(lengths)).astype(np.float32)
    out = []
    for f32 in (True, False):
        b = sfp.Batch(chains(lengths), seed=2, precision=precision)
        b.set_modes(R32 if f32 else R32.astype(np.float64))
        b.step(40)
        out.append(b.modes())
        b.close()
    np.testing.assert_array_equal(out[0], out[1])


def test_pinned_buffers_are_read_and_written_in_place():
    """Page-locked caller buffers with one length group: the load kernel reads
    the FP32 input directly and the store kernel writes the FP32 output
    directly; same values as pageable buffers."""
    lengths = [128] * 33
    R32 = np.stack(starts(lengths)).astype(np.float32)
    n = R32.size
    hin, hout = pinned_f32(n), pinned_f32(n)
    hin[:] = R32.ravel()
    b = sfp.Batch(chains(lengths), seed=4, precision=sfp.SFP_MIXED_BF16)
    L = sfp._lib.load()
    sfp._lib.check(L.sfp_set_modes_f32(b._h, hin.ctypes.data, n))
    sfp._lib.check(L.sfp_step(b._h, 7))
    sfp._lib.check(L.sfp_observe(b._h, sfp.SFP_OBS_MODES_F32, hout.ctypes.data, n * 4))
    ref = b.observe(sfp.SFP_OBS_MODES_F32)
    np.testing.assert_array_equal(hout.reshape(ref.shape), ref)
    b.set_modes(R32)
    b.set_step(0)   # set_modes leaves the step counters (Philox keys) at 7
    b.step(7)
    np.testing.assert_array_equal(b.observe(sfp.SFP_OBS_MODES_F32), ref)
    b.close()


def test_fp64_state_takes_f32_input_rounded():
    """SFP_FP64 keeps FP64 state: set_modes_f32 widens the FP32 values exactly."""
    lengths = [100, 64]
    R32 = [r.astype(np.float32) for r in starts(lengths)]
    b = sfp.Batch(chains(lengths), seed=1, precision=sfp.SFP_FP64)
    b.set_modes(R32)
    for g, r in zip(b.modes(), R32):
        np.testing.assert_array_equal(g[:, 1:], r[:, 1:].astype(np.float64))
    b.close()


def test_f32_calls_reject_short_buffers():
    lengths = [64] * 3
    b = sfp.Batch(chains(lengths), seed=1, precision=sfp.SFP_FP32)
    L = sfp._lib.load()
    n = 3 * sum(lengths)
    a = np.zeros(n, dtype=np.float32)
    assert L.sfp_set_modes_f32(b._h, a.ctypes.data, n - 1) == sfp._lib.SFP_EINVAL
    assert L.sfp_set_modes_f32(b._h, None, n) == sfp._lib.SFP_EINVAL
    assert L.sfp_observe(b._h, sfp.SFP_OBS_MODES_F32, a.ctypes.data, n * 4 - 1) == sfp._lib.SFP_EINVAL
    assert L.sfp_observe(b._h, sfp.SFP_OBS_MODES_F32, a.ctypes.data, n * 4) == sfp._lib.SFP_OK
    b.close()
