"""Thin ctypes binding of libafqmc.so (include/afqmc.h).

Argument marshalling only: numpy arrays in, numpy arrays out, every step of
the walker propagation runs in the library's CUDA kernels. There is no CPU
fallback; loading fails loudly if the shared library is missing.
"""
from __future__ import annotations

import ctypes as C
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libafqmc.so")

AFQMC_FP64, AFQMC_FP32, AFQMC_TF32, AFQMC_TF32X3, AFQMC_BF16X3 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": AFQMC_FP64, "fp32": AFQMC_FP32, "tf32": AFQMC_TF32,
              "tf32x3": AFQMC_TF32X3, "bf16x3": AFQMC_BF16X3}
STATUS = {0: "OK", 1: "E_INVALID", 2: "E_OOM", 3: "E_CUDA", 4: "E_POPULATION",
          5: "E_TIMEOUT", 6: "E_NUMERIC", 7: "E_STATE"}
KERNEL_IDS = ["force_bias", "fields", "one_body", "propagate", "overlap",
              "weights", "orthonormalize", "energy", "comb"]


class afqmc_params(C.Structure):
    _fields_ = [("M", C.c_int32), ("n_up", C.c_int32), ("n_dn", C.c_int32),
                ("n_chol", C.c_int32), ("n_det", C.c_int32),
                ("n_walkers", C.c_int32), ("dtau", C.c_double),
                ("seed", C.c_uint64), ("run_id", C.c_int32),
                ("precision", C.c_int32), ("ortho_every", C.c_int32),
                ("measure_every", C.c_int32), ("pc_every", C.c_int32),
                ("taylor_order", C.c_int32), ("fb_cap", C.c_double),
                ("e_shift", C.c_double), ("fp64_islands", C.c_int32),
                ("graphs", C.c_int32), ("autotune", C.c_int32),
                ("weight_cap", C.c_int32), ("cs_group", C.c_int32),
                ("cs_size", C.c_int32), ("weight_mode", C.c_int32),
                ("mf_subtract", C.c_int32), ("block_sparse", C.c_int32),
                ("reserved", C.c_int32 * 3)]


class afqmc_tuning(C.Structure):
    _fields_ = [("xsplit", C.c_int32), ("bn_force_bias", C.c_int32),
                ("bn_one_body", C.c_int32), ("bn_energy", C.c_int32),
                ("bn_half_step", C.c_int32), ("taylor_fused", C.c_int32),
                ("reserved", C.c_int32 * 2)]


class afqmc_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_size_t), ("max_active", C.c_int32),
                ("device", C.c_int32), ("reserved", C.c_int32 * 4)]


class afqmc_run_info(C.Structure):
    _fields_ = [("state", C.c_int32), ("status", C.c_int32), ("n_blocks", C.c_int32),
                ("blocks_done", C.c_int32), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double),
                ("footprint", C.c_size_t), ("message", C.c_char * 160)]


class afqmc_block_result(C.Structure):
    _fields_ = [("t_start", C.c_double), ("t_end", C.c_double),
                ("device_ms", C.c_double), ("e_mixed", C.c_double),
                ("weight_sum", C.c_double), ("step", C.c_int64)]


class afqmc_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64),
                ("completed", C.c_int64), ("failed", C.c_int64), ("blocks", C.c_int64),
                ("walker_steps", C.c_double), ("p50_ms", C.c_double),
                ("p99_ms", C.c_double), ("elapsed_s", C.c_double),
                ("active", C.c_int32), ("queued", C.c_int32),
                ("max_active_seen", C.c_int32), ("reserved0", C.c_int32),
                ("bytes_in_use", C.c_size_t), ("peak_bytes", C.c_size_t)]


RUN_STATES = {0: "queued", 1: "active", 2: "done", 3: "failed"}


class AfqmcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load_library(path: str = LIB_PATH):
    """Load libafqmc.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with "
                          "`python -m paper_1804_03310_gb300.build`")
    lib = C.CDLL(path)
    P = C.POINTER
    d = P(C.c_double)
    i32 = P(C.c_int32)
    vp = C.c_void_p
    sig = {
        "afqmc_params_default": (None, [P(afqmc_params)]),
        "afqmc_create": (C.c_int, [P(afqmc_params), d, d, d, d, i32, i32, d, vp, P(vp)]),
        "afqmc_propagate": (C.c_int, [vp, C.c_int32]),
        "afqmc_orthonormalize": (C.c_int, [vp]),
        "afqmc_population_control": (C.c_int, [vp]),
        "afqmc_local_energy": (C.c_int, [vp, d, d]),
        "afqmc_weights": (C.c_int, [vp, d, d]),
        "afqmc_green": (C.c_int, [vp, C.c_int32, d, d]),
        "afqmc_force_bias": (C.c_int, [vp, d]),
        "afqmc_energy_shift": (C.c_int, [vp, d]),
        "afqmc_log_weight_scale": (C.c_int, [vp, d]),
        "afqmc_selftest_wait_timeout": (C.c_int, [vp, C.c_int64]),
        "afqmc_energy_history": (C.c_int, [vp, d, C.c_int32, i32]),
        "afqmc_get_state": (C.c_int, [vp, vp, P(C.c_size_t)]),
        "afqmc_set_state": (C.c_int, [vp, vp, C.c_size_t]),
        "afqmc_synchronize": (C.c_int, [vp]),
        "afqmc_set_kernel_timing": (C.c_int, [vp, C.c_int32]),
        "afqmc_kernel_stats": (C.c_int, [vp, C.c_int32, P(C.c_int64), d, d, i32]),
        "afqmc_launch_count": (C.c_int64, [vp]),
        "afqmc_last_error": (C.c_char_p, [vp]),
        "afqmc_destroy": (None, [vp]),
        "afqmc_comb_static": (C.c_int, [vp, C.c_int32, C.c_uint64, C.c_int32,
                                        C.c_int64, vp, vp, vp]),
        "afqmc_get_tuning": (C.c_int, [vp, P(afqmc_tuning)]),
        "afqmc_set_tuning": (C.c_int, [vp, P(afqmc_tuning)]),
        "afqmc_footprint": (C.c_int, [P(afqmc_params), i32, i32, P(C.c_size_t),
                                      P(C.c_size_t)]),
        "afqmc_device_bytes": (C.c_size_t, [vp]),
        "afqmc_graph_count": (C.c_int32, [vp]),
        "afqmc_batch_create": (C.c_int, [P(vp), C.c_int32, C.c_int32, P(vp)]),
        "afqmc_batch_propagate": (C.c_int, [vp, C.c_int32]),
        "afqmc_batch_launches": (C.c_int64, [vp]),
        "afqmc_batch_synchronize": (C.c_int, [vp]),
        "afqmc_batch_destroy": (None, [vp]),
        "afqmc_server_create": (C.c_int, [P(afqmc_server_config), P(vp)]),
        "afqmc_server_submit": (C.c_int, [vp, P(afqmc_params), d, d, d, d, i32, i32, d,
                                          C.c_int32, C.c_int32, P(C.c_int64)]),
        "afqmc_server_poll": (C.c_int, [vp, C.c_int64, P(afqmc_run_info),
                                        P(afqmc_block_result), C.c_int32]),
        "afqmc_server_wait": (C.c_int, [vp, C.c_int64, C.c_double]),
        "afqmc_server_stats_get": (C.c_int, [vp, P(afqmc_server_stats)]),
        "afqmc_server_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _dptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _iptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def default_params() -> afqmc_params:
    p = afqmc_params()
    load_library().afqmc_params_default(C.byref(p))
    return p


class Inputs:
    """afqmc_create's arguments as contiguous arrays plus the parameter block."""

    def __init__(self, h1, L, C_up, C_dn, occ_up, occ_dn, ci, *, dtau,
                 n_walkers, seed=0, run_id=0, precision="fp64", ortho_every=2,
                 measure_every=20, pc_every=20, taylor_order=6, fb_cap=1.0,
                 e_shift=None, fp64_islands=False, graphs=True, autotune=True,
                 weight_cap=0, cs_group=0, cs_size=0, weight_mode=0, mf_subtract=0,
                 block_sparse=0):
        self.h1 = np.ascontiguousarray(h1, dtype=np.float64)
        self.L = np.ascontiguousarray(L, dtype=np.float64)
        self.C_up = np.ascontiguousarray(C_up, dtype=np.float64)
        self.C_dn = np.ascontiguousarray(C_dn, dtype=np.float64)
        self.occ_up = np.ascontiguousarray(occ_up, dtype=np.int32)
        self.occ_dn = np.ascontiguousarray(occ_dn, dtype=np.int32)
        self.ci = np.ascontiguousarray(np.asarray(ci, dtype=np.complex128).view(np.float64))
        p = default_params()
        p.M = self.h1.shape[0]
        p.n_up = self.occ_up.shape[1]
        p.n_dn = self.occ_dn.shape[1]
        p.n_chol = self.L.shape[0]
        p.n_det = self.occ_up.shape[0]
        p.n_walkers = n_walkers
        p.dtau = dtau
        p.seed = seed
        p.run_id = run_id
        p.precision = PRECISIONS[precision] if isinstance(precision, str) else precision
        p.ortho_every = ortho_every
        p.measure_every = measure_every
        p.pc_every = pc_every
        p.taylor_order = taylor_order
        p.fb_cap = fb_cap
        p.e_shift = math.nan if e_shift is None else e_shift
        # False/True as 0/1; "qr" (or 2): the QR alone in FP64
        p.fp64_islands = 2 if fp64_islands == "qr" else int(fp64_islands)
        p.graphs = int(bool(graphs))
        p.autotune = int(bool(autotune))
        p.weight_cap = int(weight_cap)
        p.cs_group = int(cs_group)
        p.cs_size = int(cs_size)
        p.weight_mode = int(weight_mode)
        p.mf_subtract = int(mf_subtract)
        p.block_sparse = int(block_sparse)
        self.params = p

    @classmethod
    def from_system(cls, system, **kw):
        args = dict(dtau=system.dtau, n_walkers=system.n_walkers,
                    seed=system.seed, run_id=system.run_id,
                    ortho_every=system.ortho_every,
                    measure_every=system.measure_every,
                    pc_every=system.pc_every, taylor_order=system.taylor_order,
                    fb_cap=system.fb_cap, weight_cap=system.weight_cap,
                    weight_mode=system.weight_mode, mf_subtract=system.mf_subtract)
        args.update(kw)
        return cls(system.h1, system.L, system.C_up, system.C_dn,
                   system.occ_up, system.occ_dn, system.ci, **args)

    def args(self):
        """Pointer arguments h1, L, C_up, C_dn, occ_up, occ_dn, ci."""
        return (_dptr(self.h1), _dptr(self.L), _dptr(self.C_up), _dptr(self.C_dn),
                _iptr(self.occ_up), _iptr(self.occ_dn), _dptr(self.ci))


def afqmc_footprint(inputs: "Inputs"):
    """(resident, setup_peak) device bytes of a context (host-only call)."""
    lib = load_library()
    r = C.c_size_t()
    sp = C.c_size_t()
    s = lib.afqmc_footprint(C.byref(inputs.params), _iptr(inputs.occ_up),
                            _iptr(inputs.occ_dn), C.byref(r), C.byref(sp))
    if s != 0:
        raise AfqmcError(s, lib.afqmc_last_error(None).decode())
    return r.value, sp.value


class Afqmc:
    """One ph-AFQMC context (a population of walkers of one system)."""

    def __init__(self, *args, stream=None, **kw):
        lib = load_library()
        self._lib = lib
        self._h = C.c_void_p()
        inp = args[0] if len(args) == 1 and isinstance(args[0], Inputs) else Inputs(*args, **kw)
        p = inp.params
        self.params = p
        self.M, self.n_up, self.n_dn = p.M, p.n_up, p.n_dn
        self.n_chol, self.n_walkers = p.n_chol, p.n_walkers
        st = C.c_void_p(stream) if stream else None
        s = lib.afqmc_create(C.byref(p), *inp.args(), st, C.byref(self._h))
        if s != 0:
            raise AfqmcError(s, lib.afqmc_last_error(None).decode())

    @classmethod
    def from_system(cls, system, stream=None, **kw):
        return cls(Inputs.from_system(system, **kw), stream=stream)

    # -- helpers ------------------------------------------------------------
    def _check(self, s):
        if s != 0:
            raise AfqmcError(s, self._lib.afqmc_last_error(self._h).decode())

    def close(self):
        if self._h:
            self._lib.afqmc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the C calls ---------------------------------------------------------
    def afqmc_propagate(self, n_steps: int):
        self._check(self._lib.afqmc_propagate(self._h, n_steps))

    def afqmc_orthonormalize(self):
        self._check(self._lib.afqmc_orthonormalize(self._h))

    def afqmc_population_control(self):
        self._check(self._lib.afqmc_population_control(self._h))

    def afqmc_local_energy(self):
        e = np.zeros(2 * self.n_walkers)
        em = np.zeros(1)
        self._check(self._lib.afqmc_local_energy(self._h, _dptr(e), _dptr(em)))
        return e.view(np.complex128), float(em[0])

    def afqmc_weights(self):
        w = np.zeros(self.n_walkers)
        lo = np.zeros(2 * self.n_walkers)
        self._check(self._lib.afqmc_weights(self._h, _dptr(w), _dptr(lo)))
        return w, lo.view(np.complex128)

    def afqmc_green(self, walker: int):
        gu = np.zeros(2 * self.M * self.M)
        gd = np.zeros(2 * self.M * self.M)
        self._check(self._lib.afqmc_green(self._h, walker, _dptr(gu), _dptr(gd)))
        return (gu.view(np.complex128).reshape(self.M, self.M),
                gd.view(np.complex128).reshape(self.M, self.M))

    def afqmc_selftest_wait_timeout(self, limit_cycles: int):
        self._check(self._lib.afqmc_selftest_wait_timeout(self._h, int(limit_cycles)))

    def afqmc_energy_shift(self) -> float:
        e = np.zeros(1)
        self._check(self._lib.afqmc_energy_shift(self._h, _dptr(e)))
        return float(e[0])

    def afqmc_log_weight_scale(self) -> float:
        e = np.zeros(1)
        self._check(self._lib.afqmc_log_weight_scale(self._h, _dptr(e)))
        return float(e[0])

    def afqmc_force_bias(self):
        x = np.zeros(2 * self.n_walkers * self.n_chol)
        self._check(self._lib.afqmc_force_bias(self._h, _dptr(x)))
        return x.view(np.complex128).reshape(self.n_walkers, self.n_chol)

    def afqmc_energy_history(self):
        n = C.c_int32()
        self._check(self._lib.afqmc_energy_history(self._h, None, 0, C.byref(n)))
        k = min(n.value, 4096)
        out = np.zeros(2 * max(k, 1))
        self._check(self._lib.afqmc_energy_history(self._h, _dptr(out), k, C.byref(n)))
        return out[: 2 * k].reshape(k, 2)

    def afqmc_get_state(self) -> bytes:
        nb = C.c_size_t()
        self._check(self._lib.afqmc_get_state(self._h, None, C.byref(nb)))
        buf = C.create_string_buffer(nb.value)
        self._check(self._lib.afqmc_get_state(self._h, buf, C.byref(nb)))
        return buf.raw[: nb.value]

    def afqmc_set_state(self, state: bytes):
        buf = C.create_string_buffer(state, len(state))
        self._check(self._lib.afqmc_set_state(self._h, buf, len(state)))

    def afqmc_synchronize(self):
        self._check(self._lib.afqmc_synchronize(self._h))

    def afqmc_set_kernel_timing(self, enable: bool):
        self._check(self._lib.afqmc_set_kernel_timing(self._h, int(enable)))

    def afqmc_kernel_stats(self, kernel):
        kid = KERNEL_IDS.index(kernel) if isinstance(kernel, str) else kernel
        n = C.c_int64()
        ms = C.c_double()
        wk = C.c_double()
        isb = C.c_int32()
        self._check(self._lib.afqmc_kernel_stats(self._h, kid, C.byref(n), C.byref(ms),
                                                 C.byref(wk), C.byref(isb)))
        return dict(launches=n.value, total_ms=ms.value, work=wk.value,
                    is_bytes=bool(isb.value))

    def afqmc_launch_count(self) -> int:
        return int(self._lib.afqmc_launch_count(self._h))

    def afqmc_get_tuning(self) -> dict:
        t = afqmc_tuning()
        self._check(self._lib.afqmc_get_tuning(self._h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in afqmc_tuning._fields_ if f != "reserved"}

    def afqmc_set_tuning(self, **kw):
        t = afqmc_tuning()
        self._check(self._lib.afqmc_get_tuning(self._h, C.byref(t)))
        for k, v in kw.items():
            setattr(t, k, v)
        self._check(self._lib.afqmc_set_tuning(self._h, C.byref(t)))

    def afqmc_device_bytes(self) -> int:
        return int(self._lib.afqmc_device_bytes(self._h))

    def afqmc_graph_count(self) -> int:
        return int(self._lib.afqmc_graph_count(self._h))

    # -- views of the state --------------------------------------------------
    def walkers(self):
        """Walker orbitals as complex128 arrays Phi_up [W, M, n_up], Phi_dn [W, M, n_dn],
        plus weights, log-overlaps and the step counter, from a checkpoint image."""
        return decode_state(self.afqmc_get_state(), self.n_chol)


HEADER = np.dtype([("magic", "S8"), ("M", "<i4"), ("n_up", "<i4"), ("n_dn", "<i4"),
                   ("n_walkers", "<i4"), ("step", "<i8"), ("seed", "<u8"),
                   ("run_id", "<i4"), ("n_chol", "<i4")])


def decode_state(buf: bytes, n_chol=None):
    h = np.frombuffer(buf, dtype=HEADER, count=1)[0]
    M, nu, nd, W = int(h["M"]), int(h["n_up"]), int(h["n_dn"]), int(h["n_walkers"])
    N = nu + nd
    off = HEADER.itemsize
    z = np.frombuffer(buf, dtype=np.complex128, count=W * N * M, offset=off)
    z = z.reshape(W, N, M)
    off += W * N * M * 16
    w = np.frombuffer(buf, dtype=np.float64, count=W, offset=off).copy()
    off += W * 8
    lo = np.frombuffer(buf, dtype=np.complex128, count=W, offset=off).copy()
    Phi = np.swapaxes(z, 1, 2)
    return dict(Phi_up=Phi[:, :, :nu].copy(), Phi_dn=Phi[:, :, nu:].copy(), weight=w,
                logO=lo, step=int(h["step"]))


def encode_state(template: bytes, Phi_up, Phi_dn, weight, logO, step=None) -> bytes:
    """Replace the walkers of a checkpoint image (same sizes)."""
    h = np.frombuffer(template, dtype=HEADER, count=1).copy()
    if step is not None:
        h["step"] = step
    W = Phi_up.shape[0]
    z = np.concatenate([Phi_up, Phi_dn], axis=2)           # [W, M, N]
    z = np.ascontiguousarray(np.swapaxes(z, 1, 2), dtype=np.complex128)
    return (h.tobytes() + z.tobytes() + np.asarray(weight, np.float64).tobytes()
            + np.asarray(logO, np.complex128).tobytes())


COMB_STATIC_MAX_WALKERS = 65536


def afqmc_comb_static(d_weight: int, n_walkers: int, seed: int, run_id: int,
                      step: int, d_parent: int, d_wnew: int, stream: int = 0):
    """Comb population control on caller-owned device buffers (raw device
    pointers), allocating no device memory; see include/afqmc.h."""
    lib = load_library()
    s = lib.afqmc_comb_static(C.c_void_p(d_weight), n_walkers, seed, run_id, step,
                              C.c_void_p(d_parent), C.c_void_p(d_wnew),
                              C.c_void_p(stream) if stream else None)
    if s != 0:
        raise AfqmcError(s, lib.afqmc_last_error(None).decode())


class Batch:
    """Several contexts advanced together, one CUDA graph launch per block
    (afqmc_batch_* in include/afqmc.h). Keeps its members alive."""

    def __init__(self, contexts, steps_per_block):
        lib = load_library()
        self._lib = lib
        self.members = list(contexts)
        self.steps_per_block = steps_per_block
        arr = (C.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        self._h = C.c_void_p()
        s = lib.afqmc_batch_create(arr, len(self.members), steps_per_block, C.byref(self._h))
        if s != 0:
            raise AfqmcError(s, lib.afqmc_last_error(None).decode())

    def _check(self, s):
        if s != 0:
            raise AfqmcError(s, self._lib.afqmc_last_error(None).decode())

    def afqmc_batch_propagate(self, n_blocks: int):
        self._check(self._lib.afqmc_batch_propagate(self._h, n_blocks))

    def afqmc_batch_synchronize(self):
        self._check(self._lib.afqmc_batch_synchronize(self._h))

    def afqmc_batch_launches(self) -> int:
        return int(self._lib.afqmc_batch_launches(self._h))

    def close(self):
        if self._h:
            self._lib.afqmc_batch_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Serving loop (afqmc_server_* in include/afqmc.h): submit runs, poll
    their per-block results, read latency statistics."""

    def __init__(self, hbm_budget=0, max_active=0, device=0):
        lib = load_library()
        self._lib = lib
        cfg = afqmc_server_config()
        cfg.hbm_budget = hbm_budget
        cfg.max_active = max_active
        cfg.device = device
        self._h = C.c_void_p()
        s = lib.afqmc_server_create(C.byref(cfg), C.byref(self._h))
        if s != 0:
            raise AfqmcError(s, lib.afqmc_last_error(None).decode())

    def _check(self, s):
        if s != 0:
            raise AfqmcError(s, self._lib.afqmc_last_error(None).decode())

    def afqmc_server_submit(self, inputs: Inputs, n_blocks: int, steps_per_block: int) -> int:
        rid = C.c_int64()
        self._check(self._lib.afqmc_server_submit(self._h, C.byref(inputs.params),
                                                  *inputs.args(), n_blocks,
                                                  steps_per_block, C.byref(rid)))
        return rid.value

    def afqmc_server_poll(self, run_id: int):
        info = afqmc_run_info()
        self._check(self._lib.afqmc_server_poll(self._h, run_id, C.byref(info), None, 0))
        n = info.blocks_done
        blocks = (afqmc_block_result * max(n, 1))()
        self._check(self._lib.afqmc_server_poll(self._h, run_id, C.byref(info), blocks, n))
        out = {f: getattr(info, f) for f, _ in afqmc_run_info._fields_}
        out["state"] = RUN_STATES[info.state]
        out["message"] = info.message.decode(errors="replace")
        out["blocks"] = [{f: getattr(b, f) for f, _ in afqmc_block_result._fields_}
                         for b in blocks[:n]]
        return out

    def afqmc_server_wait(self, run_id: int = -1, timeout_s: float = -1.0):
        self._check(self._lib.afqmc_server_wait(self._h, run_id, timeout_s))

    def afqmc_server_stats(self) -> dict:
        st = afqmc_server_stats()
        self._check(self._lib.afqmc_server_stats_get(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in afqmc_server_stats._fields_}

    def close(self):
        if self._h:
            self._lib.afqmc_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
