"""Error metrics and tolerances used by the GPU parity tests.

Readings of the tolerances (the paper gives none; see the design notes):
* plain FP32 path, 1e-6 relative: MSD per lag |d(tau)| / MSD_ref(tau) for
  tau >= 1 and MSD(0) == 0 exactly; correlations |d(tau)| / |C_ref(0)|.
* tensor-core split path, 1e-5 relative: MSD |d(tau)| / MSD_ref(tau_max),
  correlations |d(tau)| / |C_ref(0)|, at every tau.
"""
import numpy as np

PLAIN_TOL = 1e-6
TC_TOL = 1e-5


def msd_rel_per_lag(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    if got.shape[0] == 1:
        return 0.0
    return float(np.max(np.abs(got[1:] - ref[1:]) / np.abs(ref[1:])))


def rel_to(got, ref, scale):
    return float(np.max(np.abs(np.asarray(got, np.float64) - np.asarray(ref, np.float64))) / abs(scale))


def check_plain_msd(got, ref, tol=PLAIN_TOL, what="msd"):
    got = np.asarray(got)
    assert got[0] == 0.0, f"{what}: MSD(0) = {got[0]!r}, want exactly 0"
    err = msd_rel_per_lag(got, ref)
    assert err <= tol, f"{what}: max relative error per lag {err:.3e} > {tol:.0e}"
    return err


def check_acf(got, ref, tol, what="acf"):
    err = rel_to(got, ref, ref[0])
    assert err <= tol, f"{what}: max error / C(0) {err:.3e} > {tol:.0e}"
    return err


def check_tc_msd(got, ref, tol=TC_TOL, what="msd", tau_max_ref=None):
    scale = ref[-1] if tau_max_ref is None else tau_max_ref
    err = rel_to(got, ref, scale)
    assert err <= tol, f"{what}: max error / MSD(tau_max) {err:.3e} > {tol:.0e}"
    return err
