"""Shared pieces of the GPU parity tests: side-by-side runs of the CUDA path
(through the C ABI) and the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

from oracle import afqmc as O


def wrap_phase(d):
    return (d + np.pi) % (2 * np.pi) - np.pi


def rel_err(a, b, floor=1.0):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(floor, float(np.max(np.abs(b)))))


def compare_state(gpu, orc, *, rtol, walkers=None, label=""):
    """Per-walker weights, log-overlaps and orbitals of the GPU context
    against an OracleRun whose walker_ids are `walkers` (default all)."""
    st = gpu.walkers()
    idx = np.arange(gpu.n_walkers) if walkers is None else np.asarray(walkers)
    w_g, lo_g = st["weight"][idx], st["logO"][idx]
    w_o, lo_o = orc.weight, orc.logO
    scale = max(1e-300, float(np.max(np.abs(w_o))))
    ew = float(np.max(np.abs(w_g - w_o))) / scale
    live = w_o > 0
    elr = float(np.max(np.abs((lo_g - lo_o).real)[live] / np.maximum(1.0, np.abs(lo_o.real[live])))) if live.any() else 0.0
    eli = float(np.max(np.abs(wrap_phase((lo_g - lo_o).imag))[live])) if live.any() else 0.0
    ephi = 0.0
    for a, b in ((st["Phi_up"][idx], orc.Phi_up), (st["Phi_dn"][idx], orc.Phi_dn)):
        if b.shape[2] == 0:
            continue
        n = np.max(np.abs(b), axis=(1, 2))
        ephi = max(ephi, float(np.max(np.max(np.abs(a - b), axis=(1, 2))[live] / n[live])) if live.any() else 0.0)
    assert ew <= rtol, f"{label} weights rel err {ew:.3e}"
    assert elr <= rtol, f"{label} log|O| err {elr:.3e}"
    assert eli <= rtol * 10, f"{label} arg O err {eli:.3e}"
    assert ephi <= rtol * 10, f"{label} orbitals rel err {ephi:.3e}"
    return dict(weight=ew, logO_re=elr, logO_im=eli, phi=ephi)


def compare_energy(gpu, orc, *, rtol, walkers=None, label=""):
    e_g, _ = gpu.afqmc_local_energy()
    idx = np.arange(gpu.n_walkers) if walkers is None else np.asarray(walkers)
    e_o = orc.local_energies()
    live = orc.weight > 0
    err = float(np.max(np.abs(e_g[idx] - e_o)[live])) / max(1.0, float(np.max(np.abs(e_o))))
    assert err <= rtol, f"{label} local energy rel err {err:.3e}"
    return err


def compare_green(gpu, orc, walker_pos, walker_id, *, rtol, label=""):
    Gu_g, Gd_g = gpu.afqmc_green(int(walker_id))
    _, Gu, Gd, _ = O.mixed_green(orc.trial, orc.Phi_up[walker_pos:walker_pos + 1],
                                 orc.Phi_dn[walker_pos:walker_pos + 1])
    err = max(rel_err(Gu_g, Gu[0]), rel_err(Gd_g, Gd[0]) if orc.Phi_dn.shape[2] else 0.0)
    assert err <= rtol, f"{label} Green's function rel err {err:.3e}"
    return err
