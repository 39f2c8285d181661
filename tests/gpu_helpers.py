"""Shared pieces of the GPU parity tests: side-by-side runs of the CUDA path
(through the C ABI) and the FP64 oracle on the same seeded inputs.

Every quantity is held to the bar per walker:
* weights: |w_gpu - w_orc| / w_orc for each walker the oracle keeps alive,
  and a walker the oracle killed is killed on the GPU too (and vice versa);
* overlaps: |ln O_gpu - ln O_orc| (the phase wrapped to (-pi, pi]), which is
  the relative error of the complex overlap O itself;
* orbitals and Green's functions: max |a - b| / max |b| per walker;
* local energies: |E_gpu - E_orc| / max(1 Ha, |E_orc|) per walker;
* when the whole population is followed, the log of the weight scale the
  combs divided out.
"""
from __future__ import annotations

import numpy as np

from oracle import afqmc as O


def wrap_phase(d):
    return (d + np.pi) % (2 * np.pi) - np.pi


def rel_err(a, b, floor=1.0):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(floor, float(np.max(np.abs(b)))))


def _per_walker_rel(a, b):
    """max over walkers of max|a_w - b_w| / max|b_w|."""
    if a.size == 0:
        return 0.0
    num = np.max(np.abs(a - b).reshape(a.shape[0], -1), axis=1)
    den = np.max(np.abs(b).reshape(b.shape[0], -1), axis=1)
    return float(np.max(num / np.maximum(den, 1e-300)))


def compare_green_all(gpu, orc, idx, live, *, rtol, label=""):
    """Green's functions of every live sampled walker (both spins)."""
    pos = np.nonzero(live)[0]
    if pos.size == 0:
        return 0.0
    _, Gu, Gd, _ = O.mixed_green(orc.trial, orc.Phi_up[pos], orc.Phi_dn[pos])
    err = 0.0
    for k, p in enumerate(pos):
        gu, gd = gpu.afqmc_green(int(idx[p]))
        err = max(err, rel_err(gu, Gu[k]))
        if orc.Phi_dn.shape[2]:
            err = max(err, rel_err(gd, Gd[k]))
    assert err <= rtol, f"{label} Green's function rel err {err:.3e}"
    return err


def compare_state(gpu, orc, *, rtol, walkers=None, label="", green=True):
    """Per-walker weights, overlaps, orbitals and (green=True) Green's
    functions of the GPU context against an OracleRun whose walker_ids are
    `walkers` (default all)."""
    st = gpu.walkers()
    idx = np.arange(gpu.n_walkers) if walkers is None else np.asarray(walkers)
    w_g, lo_g = st["weight"][idx], st["logO"][idx]
    w_o, lo_o = orc.weight, orc.logO
    live = w_o > 0
    killed_g = ~(w_g > 0)
    assert np.array_equal(killed_g, ~live), (
        f"{label} killed walkers differ: gpu {np.nonzero(killed_g)[0]}, "
        f"oracle {np.nonzero(~live)[0]}")
    ew = float(np.max(np.abs(w_g - w_o)[live] / w_o[live])) if live.any() else 0.0
    d = lo_g - lo_o
    dl = np.abs(d.real + 1j * wrap_phase(d.imag))
    elo = float(np.max(dl[live])) if live.any() else 0.0
    ephi = 0.0
    for a, b in ((st["Phi_up"][idx], orc.Phi_up), (st["Phi_dn"][idx], orc.Phi_dn)):
        if b.shape[2] == 0:
            continue
        ephi = max(ephi, _per_walker_rel(a[live], b[live]))
    assert ew <= rtol, f"{label} weights per-walker rel err {ew:.3e}"
    assert elo <= rtol, f"{label} overlap rel err |d ln O| {elo:.3e}"
    assert ephi <= rtol, f"{label} orbitals rel err {ephi:.3e}"
    out = dict(weight=ew, overlap=elo, phi=ephi)
    if green:
        out["green"] = compare_green_all(gpu, orc, idx, live, rtol=rtol, label=label)
    return out


def compare_energy(gpu, orc, *, rtol, walkers=None, label=""):
    """Per-walker local energies, relative to max(1 Ha, |E|)."""
    e_g, _ = gpu.afqmc_local_energy()
    idx = np.arange(gpu.n_walkers) if walkers is None else np.asarray(walkers)
    e_o = orc.local_energies()
    live = orc.weight > 0
    if not live.any():
        return 0.0
    err = float(np.max((np.abs(e_g[idx] - e_o) / np.maximum(1.0, np.abs(e_o)))[live]))
    assert err <= rtol, f"{label} local energy rel err {err:.3e}"
    return err


def compare_green(gpu, orc, walker_pos, walker_id, *, rtol, label=""):
    Gu_g, Gd_g = gpu.afqmc_green(int(walker_id))
    _, Gu, Gd, _ = O.mixed_green(orc.trial, orc.Phi_up[walker_pos:walker_pos + 1],
                                 orc.Phi_dn[walker_pos:walker_pos + 1])
    err = max(rel_err(Gu_g, Gu[0]), rel_err(Gd_g, Gd[0]) if orc.Phi_dn.shape[2] else 0.0)
    assert err <= rtol, f"{label} Green's function rel err {err:.3e}"
    return err


def side_by_side(gpu, orc, n_steps, rtol, walkers=None, energy_at=(), label=""):
    """Advance both one step at a time and compare after every step."""
    worst = {}
    for s in range(1, n_steps + 1):
        gpu.afqmc_propagate(1)
        orc.step()
        r = compare_state(gpu, orc, rtol=rtol, walkers=walkers, label=f"{label} step {s}")
        if walkers is None:   # the whole population: the combs' log scale too
            d = abs(gpu.afqmc_log_weight_scale() - orc.log_scale)
            assert d <= rtol * max(1.0, abs(orc.log_scale)), f"{label} step {s} log scale {d:.3e}"
            r["log_scale"] = d
        for k, v in r.items():
            worst[k] = max(worst.get(k, 0.0), v)
        if s in energy_at:
            worst["energy"] = max(worst.get("energy", 0.0),
                                  compare_energy(gpu, orc, rtol=rtol, walkers=walkers,
                                                 label=f"{label} step {s}"))
    return worst
