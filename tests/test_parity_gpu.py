"""Parity of the CUDA path with the FP64 oracle, through the C ABI.

Same seeded inputs on both sides (oracle equilibrium starts, or neutral jittered
rods from tests/inputs.py), same Philox noise keys.  Tolerances:
  * Philox words: bit-exact.
  * Trajectories (the mode state, p >= 1): per chain ||R_gpu - R_ref|| / ||R_ref||
    <= 1e-5 for FP32 after up to 1000 steps; <= 1e-9 for FP64.
  * Single stages after one step (diagnostics): absolute on bond vectors and
    projected noise, relative on the force; the tensor-core path is looser
    there because its FP32 accumulation in TMEM rounds less finely than FMA.
"""
import math

import numpy as np
import pytest

import paper_1411_3487_gb300 as sfp
from golden_values import shear_tau
from inputs import jittered_rods
from oracle import oracle as O
from paper_1411_3487_gb300 import _lib, build

pytestmark = pytest.mark.gpu

TSTAR, NU = 0.034, 0.35
TOL = {sfp.SFP_FP32_SIMT: 1e-5, sfp.SFP_FP32: 1e-5, sfp.SFP_MIXED_BF16: 1e-5, sfp.SFP_FP64: 1e-9}
# A "precision" parameter is (precision, kernel path): the SFP_FP32 and
# SFP_MIXED_BF16 paths run fused (one kernel per step, M = 64/128/256/512;
# a 512-bead tile on a cluster of two CTAs) by default, or staged.
SIMT = pytest.param((sfp.SFP_FP32_SIMT, sfp.SFP_PATH_STAGED), id="simt")
TC = pytest.param((sfp.SFP_FP32, sfp.SFP_PATH_FUSED), id="tcgen05")
TCS = pytest.param((sfp.SFP_FP32, sfp.SFP_PATH_STAGED), id="tcgen05_staged")
F64 = pytest.param((sfp.SFP_FP64, sfp.SFP_PATH_STAGED), id="fp64")
BF = pytest.param((sfp.SFP_MIXED_BF16, sfp.SFP_PATH_FUSED), id="bf16")
BFS = pytest.param((sfp.SFP_MIXED_BF16, sfp.SFP_PATH_STAGED), id="bf16_staged")
PRECISIONS = [SIMT, TC, TCS, F64, BF, BFS]


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def rel_err(A, B):
    """Per-chain relative L2 error over the internal modes p >= 1."""
    A = np.asarray(A)[:, :, 1:]
    B = np.asarray(B)[:, :, 1:]
    return np.linalg.norm((A - B).reshape(len(A), -1), axis=1) / np.linalg.norm(B.reshape(len(B), -1), axis=1)


def starts(M, C, seed=1, dtau=1.0):
    m = O.Model(M, dtau=dtau)
    return np.stack([m.equilibrium_start(seed, j) for j in range(C)])


def make_batch(M, C, dtau, precision, seed=1, shear=0.0):
    precision, path = precision if isinstance(precision, tuple) else (precision, sfp.SFP_PATH_FUSED)
    b = sfp.Batch([{"n_beads": M, "dtau": dtau, "shear_rate_per_s": shear}] * C, seed=seed,
                  precision=precision)
    b.set_path(path)
    return b


def test_philox_bit_exact():
    for seed, job, step, tag in ((0, 0, 0, 0), (1, 7, 123456789012, 0), (0xFFFFFFFF, 3, 2**40 + 5, 1)):
        g = sfp.philox_words(seed, job, step, tag, 1000)
        for i in (0, 1, 31, 500, 999):
            ref = O.philox4x32_10([step & 0xFFFFFFFF, step >> 32, i, tag], [seed, job])
            assert np.array_equal(g[i], ref)


@pytest.mark.parametrize("precision", [SIMT, TCS, F64])
@pytest.mark.parametrize("M,C,dtau", [(256, 37, 100.0), (64, 45, 10.0), (67, 5, 10.0), (512, 3, 100.0)])
def test_each_stage_one_step(precision, M, C, dtau):
    """a1 inverse transform, a2 force, a3 noise, a4 forward transform, a5 update."""
    precision, _ = precision
    m = O.Model(M, dtau=dtau)
    t = m.tables()
    R0 = starts(M, C, dtau=dtau)
    b = make_batch(M, C, dtau, (precision, sfp.SFP_PATH_STAGED))
    b.set_modes(R0)
    b.step(1)
    fp64 = precision == sfp.SFP_FP64
    tc = precision == sfp.SFP_FP32
    # a1: bond vectors u_n = r_n - r_{n-1} = sum_p chi_{n,p} R_p (Eq. e5), slot 0 = 0
    r_ref = np.stack([m.modes_to_beads(x) for x in R0])
    u_ref = np.zeros_like(r_ref)
    u_ref[:, :, 1:] = np.diff(r_ref, axis=2)
    u_gpu = b.probe(sfp.SFP_PROBE_BONDS)
    assert np.abs(u_gpu - u_ref).max() <= (1e-11 if fp64 else 2e-4 if tc else 2e-5)
    # a3: bead noise of step 0
    z_ref = np.stack([O.bead_normals(1, j, 0, 0, M) for j in range(C)])
    assert np.abs(b.probe(sfp.SFP_PROBE_NOISE) - z_ref).max() <= (1e-13 if fp64 else 4e-6)
    # a2 + a4: the bond forces v_n (index 0 holds 0) and DeltaH = chi^T v (Eq. e11);
    # chi^T of the GPU's own v must give the oracle's DeltaH as well
    dH_ref = np.stack([m.delta_H(x) for x in r_ref])
    dH_gpu = b.probe(sfp.SFP_PROBE_DH)
    v_gpu = b.probe(sfp.SFP_PROBE_FORCE)
    assert np.all(v_gpu[:, :, 0] == 0)
    dH_of_v = np.einsum("np,can->cap", t["chi"], v_gpu[:, :, 1:])     # oracle chi: row n - 1 is bond n
    ftol = 1e-9 if fp64 else 2e-3
    assert np.all(rel_err(dH_gpu, dH_ref) < ftol)
    assert np.all(rel_err(dH_of_v, dH_ref) < ftol)
    # a4: projected noise Z = phi^T z
    Z_ref = np.einsum("np,can->cap", t["phi"], z_ref)
    assert np.abs(b.probe(sfp.SFP_PROBE_ZMODE) - Z_ref).max() <= (1e-12 if fp64 else 1e-4 if tc else 2e-5)
    # a5: the state after one step
    R1 = m.run_modes(R0, 1, np.arange(C), 0, 1)
    assert np.all(rel_err(b.modes(), R1) < TOL[precision])
    assert np.all(b.observe(sfp.SFP_OBS_STEP) == 1)


@pytest.mark.parametrize("precision", [SIMT, TC, TCS])
def test_trajectory_256bp_fp32(precision):
    """4096 x 256-bp workload, 32-chain subset: 1000 steps at dtau = 100 (15.9 ps)."""
    M, C, dtau = 256, 32, 100.0
    m = O.Model(M, dtau=dtau)
    R = starts(M, C, dtau=dtau)
    b = make_batch(M, C, dtau, precision)
    b.set_modes(R)
    done = 0
    for mark in (1, 10, 100, 1000):
        R = m.run_modes(R, 1, np.arange(C), done, mark - done)
        b.step(mark - done)
        done = mark
        G = b.modes()
        e = rel_err(G, R)
        assert e.max() < TOL[precision[0]], (mark, e.max())
        # centre of mass (FP64 accumulator, FP32 noise projection)
        dcm = np.abs(G[:, :, 0] - R[:, :, 0]).max() / math.sqrt(M)
        assert dcm < 1e-5 * math.sqrt(6 * TSTAR * dtau * mark / M) + 1e-9


def test_trajectory_64bp_fp64_full_config():
    """Single 64-bp chain, FP64, dtau = 10 (1.59 ps), 2e4 steps, seed 1."""
    M, dtau, n = 64, 10.0, 20000
    m = O.Model(M, dtau=dtau)
    R = starts(M, 1, dtau=dtau)
    b = make_batch(M, 1, dtau, sfp.SFP_FP64)
    b.set_modes(R)
    b.step(n)
    Rref = m.run_modes(R, 1, [0], 0, n)
    assert rel_err(b.modes(), Rref).max() < TOL[sfp.SFP_FP64]
    assert abs(b.modes()[0, 0, 0] - Rref[0, 0, 0]) < 1e-9


@pytest.mark.parametrize("precision", PRECISIONS)
@pytest.mark.parametrize("M,C", [(3, 4), (5, 1), (67, 5), (130, 45), (33, 300), (64, 43), (128, 85),
                                 (256, 84), (512, 45)])
def test_ragged_and_tiny_shapes(precision, M, C):
    dtau = 5.0
    m = O.Model(M, dtau=dtau)
    r0 = jittered_rods(C, M, seed=M)
    R = np.stack([m.beads_to_modes(x) for x in r0])
    b = make_batch(M, C, dtau, precision)
    b.set_modes(R)
    b.step(50)
    Rref = m.run_modes(R, 1, np.arange(C), 0, 50)
    assert rel_err(b.modes(), Rref).max() < TOL[precision[0]]


@pytest.mark.parametrize("precision", PRECISIONS)
def test_uneven_batch_with_shear(precision):
    """Lengths 64/128/256/512 with their Table 1 steps, mixed shear, one batch."""
    lengths = [64, 128, 256, 512, 64, 256, 128, 512, 256]
    dt = {64: 10.0, 128: 50.0, 256: 100.0, 512: 100.0}
    rates = [0.0, 1.54e8, 0.0, 1e8, 5e7, 0.0, 0.0, 1.54e8, 1e6]
    chains = [{"n_beads": M, "dtau": dt[M], "shear_rate_per_s": s, "job_id": 100 + i}
              for i, (M, s) in enumerate(zip(lengths, rates))]
    b = sfp.Batch(chains, seed=5, precision=precision[0])
    b.set_path(precision[1])
    starts_ = [O.Model(M, dtau=dt[M]).equilibrium_start(5, 100 + i) for i, M in enumerate(lengths)]
    b.set_modes(starts_)
    b.step(120)
    G = b.modes()
    for i, M in enumerate(lengths):
        m = O.Model(M, dtau=dt[M])
        ref = m.run_modes(starts_[i][None], 5, [100 + i], 0, 120, shear=shear_tau(rates[i]))
        assert rel_err(G[i][None], ref)[0] < TOL[precision[0]], i


@pytest.mark.parametrize("precision", [SIMT, F64])
def test_init_equilibrium_matches_oracle_sampler(precision):
    for M, C in ((64, 5), (256, 7), (512, 2)):
        b = make_batch(M, C, 10.0, precision, seed=9)
        b.init_equilibrium(0)
        m = O.Model(M)
        ref = np.stack([m.equilibrium_start(9, j) for j in range(C)])
        G = b.modes()
        assert rel_err(G, ref).max() < (1e-12 if precision[0] == sfp.SFP_FP64 else 1e-6)
        assert np.all(G[:, :, 0] == 0)
        assert np.all(b.observe(sfp.SFP_OBS_STEP) == 0)


@pytest.mark.parametrize("precision", PRECISIONS)
def test_checkpoint_resume_is_bit_exact(precision):
    M, C = 128, 20
    b = make_batch(M, C, 50.0, precision)
    b.init_equilibrium(5)
    blob = b.save()
    b.step(30)
    A = b.modes()
    b.load(blob)
    b.step(30)
    assert np.array_equal(b.modes(), A)
    assert np.all(b.observe(sfp.SFP_OBS_STEP) == 35)


def test_positions_round_trip_and_shape_observables():
    M, C = 256, 6
    d = sfp.derive()
    m = O.Model(M, dtau=100.0)
    R = starts(M, C)
    R[:, :, 0] = np.array([1.0, -2.0, 3.0]) * math.sqrt(M)         # off-origin centre of mass
    pos_nm = np.stack([m.modes_to_beads(x) for x in R]) * d["d_nm"]
    b = make_batch(M, C, 100.0, sfp.SFP_FP64)
    b.set_positions(pos_nm)
    assert rel_err(b.modes(), R).max() < 1e-12
    assert np.abs(b.positions_nm() - pos_nm).max() < 1e-10
    assert np.allclose(b.observe(sfp.SFP_OBS_COM), np.array([1.0, -2.0, 3.0]) * d["d_nm"])
    shape = b.observe(sfp.SFP_OBS_SHAPE)
    for c in range(C):
        ref = m.observables(R[c])
        assert shape[c, :3] == pytest.approx(ref[:3] * d["d_nm"] ** 2, rel=1e-10)


@pytest.mark.parametrize("precision", [SIMT, TC, TCS, BF])
def test_full_size_256bp_sampled(precision):
    """The 4096 x 256-bp workload at full size, in the benchmark's launch
    configuration; six sampled chains recomputed by the oracle."""
    M, C, dtau, n = 256, 4096, 100.0, 20
    b = make_batch(M, C, dtau, precision)
    b.init_equilibrium(0)
    R0 = b.modes()
    b.step(n)
    G = b.modes()
    m = O.Model(M, dtau=dtau)
    pick = np.array([0, 1, 777, 2048, 4000, 4095])
    ref = m.run_modes(R0[pick], 1, pick, 0, n)
    assert rel_err(G[pick], ref).max() < TOL[precision[0]]
    # a law that holds at any size: centre-of-mass diffusion D = T*/(N+1)
    dcm = (G[:, :, 0] - R0[:, :, 0]) / math.sqrt(M)
    msd = np.mean(np.sum(dcm ** 2, axis=1))
    assert msd == pytest.approx(6 * TSTAR * dtau * n / M, rel=4.5 * math.sqrt(2 / (3 * C)))


def test_budget_and_errors():
    with pytest.raises(sfp.SfpError) as e:
        sfp.Batch([{"n_beads": 256, "dtau": 100.0}] * 64, hbm_budget_bytes=100_000,
                  precision=sfp.SFP_FP32_SIMT)
    assert e.value.code == _lib.SFP_ENOMEM
    b = make_batch(64, 3, 10.0, sfp.SFP_FP32_SIMT)
    with pytest.raises(sfp.SfpError):
        b.probe(sfp.SFP_PROBE_DH)                 # no step yet
    with pytest.raises(sfp.SfpError):
        b.step(-1)


@pytest.mark.parametrize("precision", [SIMT, TC, BF])
def test_nonfinite_state_is_reported(precision):
    M, C = 64, 4
    b = make_batch(M, C, 10.0, precision)
    R = starts(M, C)
    R[2, 1, 5] = np.nan
    b.set_modes(R)
    b.step(1)
    with pytest.raises(sfp.SfpError) as e:
        b.modes()
    assert e.value.code == _lib.SFP_ENONFINITE


def test_fused_and_staged_paths_agree():
    """The one-kernel step and the per-stage kernels compute the same step
    (Eq. e11 as chi^T v in both), so their trajectories agree to FP32
    rounding; probes refuse a fused step."""
    M, C, dtau = 128, 90, 50.0
    R = starts(M, C, dtau=dtau)
    out = []
    for path in (sfp.SFP_PATH_FUSED, sfp.SFP_PATH_STAGED):
        b = make_batch(M, C, dtau, (sfp.SFP_FP32, path))
        b.set_modes(R)
        b.step(200)
        out.append(b.modes())
        if path == sfp.SFP_PATH_FUSED:
            with pytest.raises(sfp.SfpError):
                b.probe(sfp.SFP_PROBE_DH)
    assert rel_err(out[0], out[1]).max() < 1e-5
    dcm = np.abs(out[0][:, :, 0] - out[1][:, :, 0]).max() / math.sqrt(M)
    assert dcm < 1e-5 * math.sqrt(6 * TSTAR * dtau * 200 / M)


@pytest.mark.parametrize("prec", [sfp.SFP_FP32, sfp.SFP_MIXED_BF16], ids=["tf32", "bf16"])
@pytest.mark.parametrize("M,C", [(256, 50), (64, 100), (128, 301), (512, 85)])
def test_fused_multi_step_launch_is_bit_exact(M, C, prec):
    """sfp_step(n) runs n steps in one fused launch; chains are independent, so
    it must reproduce n launches of one step bit for bit (and the oracle)."""
    dtau = 50.0
    R = starts(M, C, dtau=dtau)
    out = []
    for split in (False, True):
        b = make_batch(M, C, dtau, (prec, sfp.SFP_PATH_FUSED))
        b.set_modes(R)
        if split:
            for _ in range(37):
                b.step(1)
        else:
            b.step(37)
        out.append(b.modes())
        assert np.all(b.observe(sfp.SFP_OBS_STEP) == 37)
    assert np.array_equal(out[0], out[1])
    ref = O.Model(M, dtau=dtau).run_modes(R, 1, np.arange(C), 0, 37)
    assert rel_err(out[0], ref).max() < TOL[prec]


@pytest.mark.parametrize("M,C", [(256, 40), (512, 6), (64, 45)])
def test_bf16_transforms_against_the_oracle(M, C):
    """SFP_MIXED_BF16: the staged transforms with a three-pass BF16 hi/lo split
    (about 16 bits per product).  One step's stages and a 100-step trajectory
    against the oracle, with bounds from that precision: bonds are sums of
    terms up to ~1e2 d, so ~1e-3 absolute; the state relative error ~1e-4."""
    dtau = {64: 10.0, 256: 100.0, 512: 100.0}[M]
    m = O.Model(M, dtau=dtau)
    R0 = starts(M, C, dtau=dtau)
    b = make_batch(M, C, dtau, (sfp.SFP_MIXED_BF16, sfp.SFP_PATH_STAGED))
    b.set_modes(R0)
    b.step(1)
    r_ref = np.stack([m.modes_to_beads(x) for x in R0])
    u_ref = np.zeros_like(r_ref)
    u_ref[:, :, 1:] = np.diff(r_ref, axis=2)
    assert np.abs(b.probe(sfp.SFP_PROBE_BONDS) - u_ref).max() < 1e-2
    z_ref = np.stack([O.bead_normals(1, j, 0, 0, M) for j in range(C)])
    Z_ref = np.einsum("np,can->cap", m.tables()["phi"], z_ref)
    assert np.abs(b.probe(sfp.SFP_PROBE_ZMODE) - Z_ref).max() < 1e-3
    b.step(99)
    ref = m.run_modes(R0, 1, np.arange(C), 0, 100)
    e = rel_err(b.modes(), ref)
    print("bf16", M, "trajectory error after 100 steps", e.max())
    assert e.max() < 1e-3


@pytest.mark.parametrize("M,C", [(256, 50), (128, 90), (64, 100)])
def test_bf16_fused_step_against_the_oracle(M, C):
    """SFP_MIXED_BF16 on the one-kernel step (kind::f16 MMAs on BF16 hi/lo
    operands, the R tile split in the kernel): 1000 steps against the oracle.
    A three-pass BF16 product carries ~17 bits, so the per-step error is a few
    1e-7 of the state and the 1000-step bound is the FP32 one, 1e-5, for the
    fused kernel and for the staged kernels (both form DeltaH = chi^T v)."""
    dtau = {64: 10.0, 128: 50.0, 256: 100.0}[M]
    m = O.Model(M, dtau=dtau)
    R = starts(M, C, dtau=dtau)
    fused = make_batch(M, C, dtau, (sfp.SFP_MIXED_BF16, sfp.SFP_PATH_FUSED))
    staged = make_batch(M, C, dtau, (sfp.SFP_MIXED_BF16, sfp.SFP_PATH_STAGED))
    fused.set_modes(R)
    staged.set_modes(R)
    done = 0
    for mark in (1, 100, 1000):
        R = m.run_modes(R, 1, np.arange(C), done, mark - done)
        fused.step(mark - done)
        staged.step(mark - done)
        done = mark
        G = fused.modes()
        e = rel_err(G, R)
        print("bf16 fused", M, "step", mark, "error", e.max())
        assert e.max() < 1e-5, (mark, e.max())
        es = rel_err(staged.modes(), R)
        print("bf16 staged", M, "step", mark, "error", es.max())
        assert es.max() < 1e-5, (mark, es.max())
        dcm = np.abs(G[:, :, 0] - R[:, :, 0]).max() / math.sqrt(M)
        assert dcm < 1e-5 * math.sqrt(6 * TSTAR * dtau * mark / M) + 1e-9
    assert np.all(fused.observe(sfp.SFP_OBS_STEP) == 1000)
    with pytest.raises(sfp.SfpError):
        fused.probe(sfp.SFP_PROBE_DH)


def test_fp64_one_kernel_per_chain_against_the_oracle():
    """SFP_FP64 on SFP_PATH_FUSED: one CUDA-core kernel per chunk of steps, a CTA
    per chain with its state in shared memory.  Mixed lengths (3, 67 and the
    paper's four), mixed shear: 150 steps in one call equal 150 calls of one
    step bit for bit, match the oracle to 1e-9 and the staged FP64 kernels to
    1e-11; probes refuse the fused step."""
    lengths = [3, 64, 67, 128, 256, 512, 64]
    dt = {3: 5.0, 64: 10.0, 67: 10.0, 128: 50.0, 256: 100.0, 512: 100.0}
    rates = [0.0, 1.54e8, 0.0, 5e7, 0.0, 1e8, 0.0]
    chains = [{"n_beads": M, "dtau": dt[M], "shear_rate_per_s": r, "job_id": 300 + i}
              for i, (M, r) in enumerate(zip(lengths, rates))]
    starts_ = [O.Model(M, dtau=dt[M]).equilibrium_start(4, 300 + i) for i, M in enumerate(lengths)]
    out = []
    for path, split in ((sfp.SFP_PATH_FUSED, False), (sfp.SFP_PATH_FUSED, True), (sfp.SFP_PATH_STAGED, False)):
        b = sfp.Batch(chains, seed=4, precision=sfp.SFP_FP64)
        b.set_path(path)
        b.set_modes(starts_)
        if split:
            for _ in range(150):
                b.step(1)
        else:
            b.step(150)
        out.append(b.modes())
        assert np.all(b.observe(sfp.SFP_OBS_STEP) == 150)
        if path == sfp.SFP_PATH_FUSED:
            with pytest.raises(sfp.SfpError):
                b.probe(sfp.SFP_PROBE_DH)
        b.close()
    for i, M in enumerate(lengths):
        assert np.array_equal(out[0][i], out[1][i]), i
        ref = O.Model(M, dtau=dt[M]).run_modes(starts_[i][None], 4, [300 + i], 0, 150, shear=shear_tau(rates[i]))
        assert rel_err(out[0][i][None], ref)[0] < 1e-9, (i, rel_err(out[0][i][None], ref)[0])
        assert rel_err(out[0][i][None], out[2][i][None])[0] < 1e-11, i
        assert abs(out[0][i][0, 0] - ref[0, 0, 0]) < 1e-9 * math.sqrt(M)


@pytest.mark.parametrize("M,C", [(256, 50), (512, 12), (100, 7)])
def test_bf16_two_pass_against_the_oracle(M, C):
    """SFP_MIXED_BF16_2: two passes (A_lo B_hi + A_hi B_hi), the tables rounded
    to BF16 (8 bits), so every transform carries ~2^-9 relative error.  The
    fused kernel rounds its stacked table [h chi; w phi] and the staged kernels
    chi^T and phi^T, so the two differ by that rounding (measured 1-2e-4 after
    200 steps) and each stays within 1e-3 of the FP64 oracle over 200 steps
    (measured 1-2e-4); lengths without tensor-core transforms (100 beads) run
    FP32 CUDA-core transforms.  The errors are printed."""
    dtau = 100.0 if M >= 256 else 10.0
    m = O.Model(M, dtau=dtau)
    R = starts(M, C, dtau=dtau)
    out = []
    for path in (sfp.SFP_PATH_FUSED, sfp.SFP_PATH_STAGED):
        b = make_batch(M, C, dtau, (sfp.SFP_MIXED_BF16_2, path))
        b.set_modes(R)
        b.step(200)
        out.append(b.modes())
        b.close()
    ref = m.run_modes(R, 1, np.arange(C), 0, 200)
    e_f, e_s = rel_err(out[0], ref).max(), rel_err(out[1], ref).max()
    print("bf16x2", M, "error after 200 steps: fused", e_f, "staged", e_s, "fused vs staged",
          rel_err(out[0], out[1]).max())
    assert e_f < 1e-3 and e_s < 1e-3
    assert rel_err(out[0], out[1]).max() < 1e-3


@pytest.mark.parametrize("M", [64, 512])
def test_pipeline_wait_timeout_is_reported(monkeypatch, M):
    """Bounded waits: with SFP_TEST_STALL=1 the fused kernel's MMA thread first
    waits on a barrier that nothing arrives at.  That wait gives up after its
    1 s limit, raises the timeout bit and the abort flag, every other wait of
    the CTA gives up too, and the kernel returns: the step reports
    SFP_ETIMEDOUT, the state is left as it was, and the GPU context stays
    usable for the next batch.  At 512 beads both CTAs of each cluster stall
    and meet at the cluster barrier before they leave."""
    C, dtau = 8, {64: 10.0, 512: 100.0}[M]
    R = starts(M, C, dtau=dtau)
    b = make_batch(M, C, dtau, (sfp.SFP_MIXED_BF16, sfp.SFP_PATH_FUSED))
    b.set_modes(R)
    monkeypatch.setenv("SFP_TEST_STALL", "1")
    b.step(1)
    with pytest.raises(sfp.SfpError) as e:
        b.modes()
    assert e.value.code == _lib.SFP_ETIMEDOUT
    monkeypatch.delenv("SFP_TEST_STALL")
    b.close()
    b2 = make_batch(M, C, dtau, (sfp.SFP_MIXED_BF16, sfp.SFP_PATH_FUSED))
    b2.set_modes(R)
    b2.step(5)
    ref = O.Model(M, dtau=dtau).run_modes(R, 1, np.arange(C), 0, 5)
    assert rel_err(b2.modes(), ref).max() < TOL[sfp.SFP_MIXED_BF16]


@pytest.mark.parametrize("prec", [sfp.SFP_FP32, sfp.SFP_MIXED_BF16], ids=["tf32", "bf16"])
def test_fused_512bp_pair_against_the_oracle(prec):
    """512-bead chains on the fused step: each tile runs on a cluster of two
    CTAs, one per half of the bonds and modes, which exchange every A operand
    block.  1000 steps against the oracle at the FP32 bound, on 82 chains
    (default tile: 4 chains, 21 tiles, the last one with 2) and the centre of
    mass carried by the first CTA of each pair."""
    M, C, dtau = 512, 82, 100.0
    m = O.Model(M, dtau=dtau)
    R = starts(M, C, dtau=dtau)
    b = make_batch(M, C, dtau, (prec, sfp.SFP_PATH_FUSED))
    b.set_modes(R)
    done = 0
    for mark in (1, 100, 1000):
        R = m.run_modes(R, 1, np.arange(C), done, mark - done)
        b.step(mark - done)
        done = mark
        G = b.modes()
        e = rel_err(G, R)
        print("fused 512", prec, "step", mark, "error", e.max())
        assert e.max() < TOL[prec], (mark, e.max())
        dcm = np.abs(G[:, :, 0] - R[:, :, 0]).max() / math.sqrt(M)
        assert dcm < 1e-5 * math.sqrt(6 * TSTAR * dtau * mark / M) + 1e-9
    assert np.all(b.observe(sfp.SFP_OBS_STEP) == 1000)


@pytest.mark.parametrize("prec", [sfp.SFP_FP32, sfp.SFP_MIXED_BF16], ids=["tf32", "bf16"])
def test_full_size_512bp_sampled(prec):
    """The 16384 x 512-bp mixed-precision workload at full size on the fused
    step (456 clusters of two CTAs: six waves of tiles of 36 chains); six sampled chains
    recomputed by the oracle, and free-draining centre-of-mass diffusion over
    all chains."""
    M, C, dtau, n = 512, 16384, 100.0, 20
    b = make_batch(M, C, dtau, (prec, sfp.SFP_PATH_FUSED))
    b.init_equilibrium(0)
    R0 = b.modes()
    b.step(n)
    G = b.modes()
    m = O.Model(M, dtau=dtau)
    pick = np.array([0, 1, 35, 36, 9999, 16383])
    ref = m.run_modes(R0[pick], 1, pick, 0, n)
    assert rel_err(G[pick], ref).max() < TOL[prec]
    dcm = (G[:, :, 0] - R0[:, :, 0]) / math.sqrt(M)
    msd = np.mean(np.sum(dcm ** 2, axis=1))
    assert msd == pytest.approx(6 * TSTAR * dtau * n / M, rel=4.5 * math.sqrt(2 / (3 * C)))


def test_page_locked_and_pageable_buffers_agree():
    """sfp_set_modes and the SFP_OBS_MODES read of sfp_observe take a
    page-locked host buffer straight from the GPU (no staging copy) and a
    pageable one through a copy: both give the same state, bit for bit."""
    import ctypes as ct
    import torch
    M, C, dtau = 256, 40, 100.0
    R = starts(M, C, dtau=dtau)
    n = R.size
    out = []
    for pinned in (False, True):
        b = make_batch(M, C, dtau, (sfp.SFP_MIXED_BF16, sfp.SFP_PATH_FUSED))
        if pinned:
            hin = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
            hout = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        else:
            hin, hout = np.empty(n), np.empty(n)
        hin[:] = R.ravel()
        L = _lib.load()
        _lib.check(L.sfp_set_modes(b._h, hin.ctypes.data, n))
        _lib.check(L.sfp_step(b._h, 7))
        _lib.check(L.sfp_observe(b._h, sfp.SFP_OBS_MODES, hout.ctypes.data, n * 8))
        out.append(hout.reshape(R.shape).copy())
        b.close()
    assert np.array_equal(out[0], out[1])
    ref = O.Model(M, dtau=dtau).run_modes(R, 1, np.arange(C), 0, 7)
    assert rel_err(out[1], ref).max() < TOL[sfp.SFP_MIXED_BF16]
