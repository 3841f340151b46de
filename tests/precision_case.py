"""Per-observable error of a GPU precision against the FP64 oracle (shared by
tests/test_precision_gpu.py and bench.py --workload precision).

GPU: the whole batch (e.g. 16384 x 512 bp) runs with sampling every `every`
steps; the oracle reruns the first `sub` chains from the same starts and noise
keys and accumulates the same sums (Sec. 5B observables i-iii, mode power,
centre-of-mass windows at lags of 1 and 10 samples).  Each error is
|GPU - oracle| / |oracle| of the subset's sums (max over chains, modes or lags)."""
import numpy as np

# d = a (1 - 2 nu) in nm from the printed dsDNA values (a = 0.33 nm, nu = 0.35,
# Sec. 2A): the oracle's sums are scaled to nm^2 with it, not with the library's
D_NM = 0.33 * (1.0 - 2.0 * 0.35)


def errors(sfp, O, precision, M=512, C=16384, dtau=100.0, steps=2000, every=20, sub=32, seed=1):
    b = sfp.Batch([{"n_beads": M, "dtau": dtau}] * C, seed=seed, precision=precision)
    b.init_equilibrium(0)
    R0 = b.modes()[:sub].copy() if precision == sfp.SFP_FP64 else None
    m = O.Model(M, dtau=dtau)
    R = np.stack([m.equilibrium_start(seed, j) for j in range(sub)])
    if R0 is not None:
        assert np.abs(R0 - R).max() < 1e-8 * np.abs(R).max()
    # start the GPU subset from the oracle's FP64 starts so only the dynamics differ
    full = b.modes()
    full[:sub] = R
    b.set_modes(full)
    b.set_sampling(every)
    b.step(steps)
    g_shape = b.observe(sfp.SFP_OBS_ACCUM)[:sub]
    g_pow = b.observe(sfp.SFP_OBS_MODE_POWER)[:sub]
    g_msd = b.observe(sfp.SFP_OBS_COM_MSD)[:sub]
    g_fin = b.modes()[:sub]
    b.close()
    d2 = D_NM ** 2
    shape = np.zeros((sub, 4))
    power = np.zeros((sub, 3, M))
    msd = np.zeros((sub, 4, 2))
    snap = np.zeros((sub, 4, 3))
    nsamp = steps // every + 1
    for k in range(nsamp):
        if k:
            R = m.run_modes(R, seed, np.arange(sub), every * (k - 1), every)
        for c in range(sub):
            o = m.observables(R[c])
            shape[c] += [o[0], o[1], o[2], 1.0]
            power[c] += R[c] ** 2
            for i, lag in enumerate((1, 10, 100, 1000)):
                if k % lag == 0:
                    if k:
                        msd[c, i] += [np.sum((o[3:6] - snap[c, i]) ** 2), 1.0]
                    snap[c, i] = o[3:6]

    def rel(a, b):
        return float(np.max(np.abs(a - b) / np.abs(b)))

    fin = R
    traj = np.linalg.norm((g_fin - fin)[:, :, 1:].reshape(sub, -1), axis=1) / \
        np.linalg.norm(fin[:, :, 1:].reshape(sub, -1), axis=1)
    return {
        "L2": rel(g_shape[:, 0], shape[:, 0] * d2),
        "u_mid2": rel(g_shape[:, 1], shape[:, 1] * d2),
        "r_mid2": rel(g_shape[:, 2], shape[:, 2] * d2),
        "mode_power": rel(g_pow[:, :, 1:].sum(axis=(1, 2)), power[:, :, 1:].sum(axis=(1, 2))),
        "mode_power_worst_mode": rel(g_pow[:, :, 1:].sum(axis=1), power[:, :, 1:].sum(axis=1)),
        "com_msd_lag1": rel(g_msd[:, 0, 0], msd[:, 0, 0] * d2),
        "com_msd_lag10": rel(g_msd[:, 1, 0], msd[:, 1, 0] * d2),
        "trajectory": float(traj.max()),
        "chains": C, "beads": M, "steps": steps, "sample_every": every, "oracle_subset": sub,
    }
